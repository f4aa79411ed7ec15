#!/usr/bin/env python
"""Benchmark of the GB300 FFT power-spectrum path; prints ONE JSON line.

Workload (one step = one full power-spectrum evaluation of one catalog):
1e7 objects Poisson-sampled from a log-normal field (P ~ k^-1.5, sigma^2 ~ 1
at the cell scale) with a linear RSD displacement f = 0.75 along z, L = 1000
Mpc/h, FP32 positions resident in HBM; TSC + interlacing on Nmesh = 512,
compensated; (k, mu) bins dk = 0.005 to k_N with 10 mu bins and multipoles
l = 0, 2, 4, shot noise subtracted.  A step runs pk_paint (tile sort + tile
paint of both meshes), pk_compute (the library's own r2c transform of both
meshes: y and x passes, then the z transform fused with the compensate /
interlace / bin pass; reduce, finalize) and pk_result (host-visible
result).  Each step is bracketed by CUDA events on the plan's stream; the L2
is flushed (a 512 MB device write) between steps, outside the events.  The
end-to-end leg ("e2e") takes the catalog from pinned host memory every step
through pipeline.PowerStream (two plans on two streams), with the one-plan
loop beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 runs under torch.distributed.run: every rank evaluates its own
independent catalog (weak scaling, no data-path collective); value = catalogs
of all ranks / max-over-ranks device time.  --impl reference times the FP64
CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "P(k)/s + particles painted/s at Nmesh 512/2048, batched vs plain; p50/p99 latency"
L_BOX, NMESH, NPART, DK, NMU = 1000.0, 512, 10_000_000, 0.005, 10
WORKLOAD = ("lognormal 1e7 objects (P~k^-1.5, sigma^2~1, RSD f=0.75), L=1000 Mpc/h, FP32 positions, "
            "TSC + interlacing, Nmesh=512, compensated, dk=0.005 to k_N (321 k bins) x 10 mu bins, "
            "multipoles l=0,2,4, shot noise subtracted")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-2048", action="store_true", help="skip the 2048^3 Zel'dovich measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-mock batched measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--no-study", action="store_true", help="skip the window / interlacing accuracy study")
    ap.add_argument("--no-survey", action="store_true", help="skip the survey-multipole measurement")
    ap.add_argument("--no-windows", action="store_true", help="skip the paint time per window")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 mesh form of the main workload")
    ap.add_argument("--zeldovich-profile", action="store_true",
                    help="two paint + compute steps of the Nmesh 2048 Zel'dovich workload only (for a launch list)")
    ap.add_argument("--survey-profile", type=int, default=0, metavar="NMESH",
                    help="only run 3 survey-multipole evaluations of a small catalog (1e5 galaxies, 1e6 randoms, "
                         "1000 Mpc/h) on an NMESH^3 mesh and print their stage times: the workload of the "
                         "survey kernels' ncu summary")
    ap.add_argument("--profile", action="store_true",
                    help="timed steps only (no e2e leg, no CPU baseline, no clock sampler): for ncu")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.uuid and parts[1] != self.uuid:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ distributed --
def dist_setup(n):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest x over all ranks (the slowest rank's time sets the job's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds_max):
    """Whole-job throughput of a weak-scaling run: every rank processes its own
    units, the job ends with the slowest rank."""
    return world * units_per_rank / seconds_max


# --------------------------------------------------------------- oracle leg --
def oracle_step(pos64):
    """One full oracle evaluation of the workload on the host cores (OpenMP):
    the paint of every object on both interlaced TSC meshes, both FP64 r2c
    transforms (the oracle's own FFT), the whole mode loop and the finalize.
    Returns (seconds, result)."""
    import oracle
    t0 = time.perf_counter()
    res = oracle.fft_power(pos64, None, L_BOX, NMESH, "tsc", True, True, dk=DK, nmu=NMU)
    return time.perf_counter() - t0, res


def oracle_tiny():
    """The oracle on the tiny plain workload (1e5 uniform objects, FP64
    positions, L = 1000, CIC on 64^3, dk = 0.01, shot noise subtracted) on all
    host threads and on one, a few evaluations each (median seconds)."""
    import oracle
    import synth
    pos = synth.uniform_catalog(100_000, 1000.0, synth.seed_for(1))
    out = {"workload": "1e5 uniform objects, CIC, Nmesh 64, dk 0.01 (20 k bins)"}
    allc = oracle.threads()
    for label, nt in (("all_cores", allc), ("one_core", 1)):
        oracle.set_threads(nt)
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            oracle.fft_power(pos, None, 1000.0, 64, "cic", False, True, dk=0.01)
            ts.append(time.perf_counter() - t0)
        out[label] = {"threads": nt, "s_per_pk": statistics.median(ts), "pk_per_s": 1.0 / statistics.median(ts)}
    oracle.set_threads(allc)
    return out


def oracle_sample_text(threads):
    return ("per step: one full FP64 oracle evaluation of the same 1e7-object catalog (paint of every "
            "object on both TSC meshes, both 512^3 r2c transforms, the 512^2 x 257 mode loop, finalize), "
            "OpenMP over %d host threads" % threads)


def per_bin_errors(got, ref):
    """Largest |got - ref| of P(k), P(k, mu), P_0, P_2, P_4 over the bins,
    relative to the reference's pre-subtraction monopole of each bin; None if
    the mode counts differ (they must agree exactly)."""
    import numpy as np
    if not (np.array_equal(got["modes"], ref["modes"]) and np.array_equal(got["modes2d"], ref["modes2d"])):
        return None
    raw = ref["power_raw"] if "power_raw" in ref else ref["power"] + ref["shot_noise"]
    ok = ref["modes"] > 0
    out = {"P": float(np.max(np.abs(got["power"] - ref["power"])[ok] / raw[ok]))}
    for e in range(3):
        out["P%d" % (2 * e)] = float(np.max(np.abs(got["poles"][e] - ref["poles"][e])[ok] / raw[ok]))
    ok2 = ref["modes2d"] > 0
    raw2 = np.broadcast_to(raw[:, None], ok2.shape)
    out["Pkmu"] = float(np.max(np.abs(got["power2d"] - ref["power2d"])[ok2] / raw2[ok2]))
    return out


def binned_stored_modes(N=None, box=None, dk=None):
    """Stored half-grid modes that fall in a k bin (0 < |k|, kmin <= k < kmax):
    the modes the bin pass must read.  Same FP64 bin rule as the library."""
    import numpy as np
    N = N or NMESH
    L_box, DK_ = box or L_BOX, dk or DK
    kF = (2.0 * math.pi) / L_box
    nk = int(math.floor(((math.pi * N) / L_box) / DK_))
    f = np.where(np.arange(N) < N // 2, np.arange(N), np.arange(N) - N)
    r2 = (f[:, None] ** 2 + f[None, :] ** 2).reshape(-1)
    l2 = np.arange(N // 2 + 1) ** 2
    total = 0
    for chunk in np.array_split(r2, max(64, N * N // 8192)):
        m = chunk[:, None] + l2[None, :]
        b = np.floor((kF * np.sqrt(m.astype(np.float64)) - 0.0) / DK_)
        total += int(np.count_nonzero((m > 0) & (b >= 0) & (b < nk)))
    return total


def zbin_rows(N=None, box=None, dk=None):
    """Rows (kx, ky) of the stored half grid that hold a binned mode: the rows
    whose packed z transforms the fused z + bin pass reads (Same FP64 rule)."""
    import numpy as np
    N = N or NMESH
    L_box, DK_ = box or L_BOX, dk or DK
    kF = (2.0 * math.pi) / L_box
    nk = int(math.floor(((math.pi * N) / L_box) / DK_))
    f = np.where(np.arange(N) < N // 2, np.arange(N), np.arange(N) - N)
    r2 = (f[:, None] ** 2 + f[None, :] ** 2).reshape(-1)
    lmin = np.where(r2 == 0, 1, 0)                      # the smallest l of a row (DC excluded)
    b = np.floor((kF * np.sqrt((r2 + lmin ** 2).astype(np.float64))) / DK_)
    return int(np.count_nonzero(b < nk))


def make_catalog(rank, device):
    import synth
    return synth.lognormal_catalog(NPART, L_BOX, NMESH, synth.seed_for(2, rank), device=device)


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    import torch
    pos = make_catalog(0, "cuda" if torch.cuda.is_available() else "cpu").double().cpu().numpy()
    for _ in range(args.warmup):
        oracle_step(pos)
    ts = [oracle_step(pos)[0] for _ in range(args.steps)]
    tot = sum(ts)
    value = args.steps / tot
    threads = oracle.threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "P(k)/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nmesh": NMESH, "particles": NPART},
        "cpu_baseline": {"value": value, "unit": "P(k)/s", "cores": threads, "kind": "oracle",
                         "sample": oracle_sample_text(threads)},
        "e2e": {"value": value, "unit": "P(k)/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- GPU leg --
KERNEL_SOURCE = {"k_fft_axis": "pk_fft.cu", "k_zbin": "pk_fft.cu"}   # others: pk_kernels.cu


def traffic_record(kernel):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current source of the kernel."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    src = os.path.join(ROOT, "paper_1712_05834_gb300", "csrc", KERNEL_SOURCE.get(kernel, "pk_kernels.cu"))
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        with open(path) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[3] == sha:
                    return float(parts[2])
    except OSError:
        pass
    return None


def measure_pipelined(torch, cfg, pos, steps, depth=2):
    """Device throughput of the same workload through pipeline.PowerStream:
    `depth` plans on their own streams, catalogs resident in HBM and
    alternating between two copies of the catalog in different object order
    (240 MB together, above the 129 MB L2; each step also streams 4.3 GB of
    meshes).  Timed with CUDA events: one start event that every stream waits
    on, one end event per stream, the latest end."""
    from paper_1712_05834_gb300.pipeline import PowerStream
    gen = torch.Generator(device=pos.device).manual_seed(7)
    cats = [pos, pos[torch.randperm(len(pos), generator=gen, device=pos.device)].contiguous()]
    with PowerStream(cfg, depth=depth, own_fft=True) as ps:
        for _ in ps.map(cats * 2):                     # warm-up
            pass
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record(ps.streams[0])
        for s_ in ps.streams[1:]:
            s_.wait_event(e0)
        for _ in ps.map(cats[k % 2] for k in range(steps)):
            pass
        ends = []
        for s_ in ps.streams:
            e = torch.cuda.Event(enable_timing=True)
            e.record(s_)
            ends.append(e)
        torch.cuda.synchronize()
        ms = max(e0.elapsed_time(e) for e in ends)
    del cats
    return {"pk_per_s": steps / (ms / 1e3), "ms_per_step": ms / steps, "steps": steps, "depth": depth,
            "scope": "this rank's GPU",
            "api": "pipeline.PowerStream(cfg, depth=%d).map(device catalogs)" % depth,
            "l2": "inputs alternate between two device copies of the catalog (240 MB > 129 MB L2); "
                  "no flush between steps",
            "note": "kernels of consecutive catalogs overlap on the GPU (tails of the large kernels, the "
                    "small reduce / scan / finalize launches); the single-stream value above has none"}


def timed_plan_steps(pk, torch, stream, plan, pos, steps, warmup):
    """Device ms of each of `steps` paint + compute + result steps (after
    `warmup`), the median stage times and the last result."""
    pk.pk_enable_timing(plan, True)
    stages = {s_: [] for s_ in pk.STAGES}
    times = []
    res = None
    for k in range(warmup + steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pk.pk_paint(plan, pos)
        pk.pk_compute(plan)
        res = pk.pk_result(plan, 0)
        b.record(stream)
        st = pk.pk_stage_times(plan)
        b.synchronize()
        if k >= warmup:
            times.append(a.elapsed_time(b))
            for s_ in pk.STAGES:
                stages[s_].append(st[s_])
    return times, {s_: statistics.median(v) for s_, v in stages.items()}, res


def measure_2048(pk, torch, stream, world, steps=5, warmup=2):
    """The precision workload at scale: 1024^3 objects on a Zel'dovich lattice,
    L = 2000, PCS + interlacing on N = 2048 (FP32 mesh, int64 fixed-point
    paint, FP32 per-CTA bin partials summed in FP64), (k, mu) bins dk = 0.005
    x 10, multipoles; then the same catalog in the FP64 mesh form (FP64 mesh,
    D2Z, FP64 sums), whose result is the reference of the per-bin error."""
    import synth
    L, N, dk = 2000.0, 2048, 0.005
    pos = synth.zeldovich_lattice(1024, L, synth.seed_for(3), device="cuda")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    n = pos.shape[0]
    out = {}
    try:
        cfg = pk.make_config(L, N, "pcs", interlaced=True, dk=dk, nmu=NMU, precision="f32")
        plan = pk.pk_plan(cfg, stream)
        try:
            times, med, r32 = timed_plan_steps(pk, torch, stream, plan, pos, steps, warmup)
            free, total = torch.cuda.mem_get_info()
        finally:
            pk.pk_destroy(plan)
        torch.cuda.empty_cache()
        total_s = max_over_ranks(sum(times) / 1e3, world)
        out.update({"workload": "zeldovich 1024^3 objects (P~k^-2, rms 0.25 spacing), L=2000, FP32 positions, "
                                "PCS + interlacing, Nmesh=2048, dk=0.005 x 10 mu bins, l=0,2,4",
                    "pk_per_s": world * steps / total_s, "ms_per_step": 1e3 * total_s / steps,
                    "particles_painted_per_s": n / ((med["sort"] + med["paint"]) / 1e3),
                    "stage_ms_median": med, "device_mem_used_gb": (total - free) / 1e9})
        cfg64 = pk.make_config(L, N, "pcs", interlaced=True, dk=dk, nmu=NMU, precision="f64")
        plan = pk.pk_plan(cfg64, stream)
        try:
            t64, med64, r64 = timed_plan_steps(pk, torch, stream, plan, pos, 2, 1)
            free, total = torch.cuda.mem_get_info()
        finally:
            pk.pk_destroy(plan)
        out["fp64_form"] = {"ms_per_step": statistics.median(t64), "stage_ms_median": med64,
                            "device_mem_used_gb": (total - free) / 1e9}
        out["max_err_vs_fp64"] = per_bin_errors(r32, r64)
        out["max_err_note"] = ("FP32 form against the FP64 mesh form on the same catalog: max over bins of "
                               "|dX| / P_raw,0(b) for X = P, P(k,mu), P_0, P_2, P_4 (tolerance 1e-4)")
    finally:
        del pos
        torch.cuda.empty_cache()
    return out


def measure_fp64_form(pk, torch, stream, pos, flush, steps=10, warmup=3):
    """The FP64 mesh form of the main workload (FP64 deposits from the int64
    fixed-point cells, FP64 mesh, D2Z, FP64 per-mode arithmetic and sums),
    timed like the main line (L2 flushed between steps)."""
    cfg = pk.make_config(L_BOX, NMESH, "tsc", interlaced=True, dk=DK, nmu=NMU, precision="f64")
    plan = pk.pk_plan(cfg, stream)
    try:
        pk.pk_enable_timing(plan, True)
        for _ in range(warmup):
            pk.pk_paint(plan, pos)
            pk.pk_compute(plan)
            res = pk.pk_result(plan, 0)
        times, stages = [], {s_: [] for s_ in pk.STAGES}
        for k in range(steps):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pk.pk_paint(plan, pos)
            pk.pk_compute(plan)
            res = pk.pk_result(plan, 0)
            b.record(stream)
            st = pk.pk_stage_times(plan)
            b.synchronize()
            times.append(a.elapsed_time(b))
            for s_ in pk.STAGES:
                stages[s_].append(st[s_])
    finally:
        pk.pk_destroy(plan)
    ms = statistics.median(times)
    return {"ms_per_step": ms, "pk_per_s": 1e3 / ms, "stage_ms_median": {k: statistics.median(v) for k, v in
                                                                           stages.items()},
            "form": "FP64 mesh, int64 fixed-point paint, D2Z, FP64 per-mode arithmetic and bin sums"}, res


def max_rel_diff(a, b):
    """Largest |a - b| over the l = 0, 2, 4 rows, relative to a's
    pre-subtraction monopole per bin (mode counts must agree exactly)."""
    import numpy as np
    if not np.array_equal(a["modes"], b["modes"]):
        return float("inf")
    ok = a["modes"] > 0
    raw = (a["power"] + a["shot_noise"])[ok]
    return float(max(np.max(np.abs(a["poles"][e] - b["poles"][e])[ok] / raw) for e in range(3)))


MOCK_L, MOCK_DK = 1000.0, 0.01


def mock_catalogs(torch, specs):
    import synth
    from paper_1712_05834_gb300.batch import Catalog
    return [Catalog(synth.lognormal_catalog(s["n"], MOCK_L, s["nmesh"], s["seed"], device="cuda"),
                    s["nmesh"], s["window"]) for s in specs]


def plain_pass(pk, torch, cats, plans, stream):
    """One catalog at a time through the public API on resident batch-1 plans."""
    from paper_1712_05834_gb300.batch import class_key
    out = []
    for c in cats:
        key = class_key(c)
        if key not in plans:
            cfg = pk.make_config(MOCK_L, c.nmesh, c.window, interlaced=c.interlaced, dk=MOCK_DK)
            plans[key] = pk.pk_plan(cfg, stream)
        pk.pk_paint(plans[key], c.pos)
        pk.pk_compute(plans[key])
        out.append(pk.pk_result(plans[key], 0))
    return out


def generated_set(pk, torch, bp, specs, stream, runs):
    """Mock -> P(k) wholly on the device: every mock of the set is drawn by the
    library's log-normal generator (field grid = the mock's Nmesh) straight
    into the batch buffers, then the captured graph is replayed."""
    gens = {}
    try:
        for s in specs:
            if s["nmesh"] not in gens:
                gens[s["nmesh"]] = pk.LogNormalCatalog(MOCK_L, s["nmesh"], stream=stream)

        def draw_all(round_):
            for c in bp.classes:
                for j, i in enumerate(c.index):
                    a, b = int(c.offsets[j]), int(c.offsets[j + 1])
                    gens[specs[i]["nmesh"]].draw(specs[i]["seed"] + 7919 * round_, b - a, out=c.pos[a:b])

        draw_all(0)
        bp.launch()
        bp.results()
        times, gen_dev = [], []
        for r in range(runs):
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            draw_all(r + 1)
            b.record(stream)
            bp.launch()
            bp.results()
            times.append(time.perf_counter() - w0)
            gen_dev.append(a.elapsed_time(b) / 1e3)
        launches = sum(pk.load().pk_lognormal_launch_count(g.gen) for g in gens.values())
    finally:
        for g in gens.values():
            g.close()
    t = statistics.median(times)
    return {"mock_to_pk_per_s": len(specs) / t, "ms_per_set": 1e3 * t,
            "generate_device_ms_per_set": 1e3 * statistics.median(gen_dev),
            "generator_launches_total": int(launches),
            "note": "each mock drawn on the device (Philox field, log-normal weights, exact-integer "
                    "inverse-CDF placement, RSD) into the batch buffers, then the graph replayed"}


def measure_batched(pk, torch, world, rank, runs=5):
    """256 log-normal mocks (object counts log-uniform in [2e5, 4e6], Nmesh in
    {128, 192, 256}, CIC / TSC), L = 1000, dk = 0.01 to k_N, l = 0, 2, 4:
    size-class batches replayed from one CUDA graph, against the same mocks
    one at a time on resident plans."""
    import numpy as np
    import synth
    from paper_1712_05834_gb300 import batch
    specs = synth.mock_set_specs(256, synth.seed_for(4, 1000 * rank))
    cats = mock_catalogs(torch, specs)
    torch.cuda.synchronize()
    nobj = sum(c.n for c in cats)
    stream = torch.cuda.Stream()
    tuner = batch.Autotuner(sample=16, repeats=3)
    t0 = time.perf_counter()
    bp = batch.BatchPower(cats, MOCK_L, dk=MOCK_DK, tuner=tuner, graph=True, stream=stream)
    setup_s = time.perf_counter() - t0
    try:
        for _ in range(3):
            res_b = bp.run()
        barrier(world)
        times, dev = [], []
        for _ in range(runs):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            a.record(stream)
            bp.launch()
            b.record(stream)
            res_b = bp.results()
            times.append(time.perf_counter() - w0)
            dev.append(a.elapsed_time(b) / 1e3)
        launches = bp.launches_per_run
        classes = [{"nmesh": c.key[0], "window": c.key[1], "mocks": len(c.index),
                    "objects": int(c.offsets[-1]), "paint": "%s/%d" % c.choice} for c in bp.classes]
        gen = generated_set(pk, torch, bp, specs, stream, runs)
    finally:
        bp.close()
    plans = {}
    try:
        res_p = plain_pass(pk, torch, cats, plans, stream)
        barrier(world)
        ptimes = []
        for _ in range(runs):
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            res_p = plain_pass(pk, torch, cats, plans, stream)
            ptimes.append(time.perf_counter() - w0)
    finally:
        for p in plans.values():
            pk.pk_destroy(p)
    tb = max_over_ranks(statistics.median(times), world)
    tp = max_over_ranks(statistics.median(ptimes), world)
    diff = max(max_rel_diff(p, b) for p, b in zip(res_p, res_b))
    del cats
    torch.cuda.empty_cache()
    return {"workload": "256 lognormal mocks (L=1000, P~k^-1.5, RSD f=0.75), objects log-uniform in "
                        "[2e5, 4e6], Nmesh in {128,192,256}, CIC/TSC, no interlacing, dk=0.01 to k_N, "
                        "l=0,2,4; positions resident in HBM (%.2e objects, larger than L2)" % nobj,
            "batched_pk_per_s": world * 256 / tb, "plain_pk_per_s": world * 256 / tp,
            "speedup": tp / tb, "batched_ms_per_set": 1e3 * tb, "plain_ms_per_set": 1e3 * tp,
            "batched_device_ms_per_set": 1e3 * statistics.median(dev),
            "particles_painted_per_s_batched": world * nobj / tb,
            "max_rel_diff_batched_vs_plain": diff,
            "graph_launches_per_set": int(launches), "classes": classes,
            "generated_on_device": gen,
            "autotune": {k: {c: round(t, 4) for c, t in v.items()} for k, v in tuner.timings.items()},
            "setup_s": setup_s}


def measure_serving(pk, torch, world, rank, nreq, rate=200.0, repeats=3):
    """Poisson stream (mean 200 requests/s) of P(k) requests: 95% drawn from a
    pool of 64 mocks as in the batched workload, 5% large (Nmesh 1024, 1.3e8
    objects, TSC + interlacing); catalogs pre-staged on the device.  Served by
    the continuous-batching server and by the plain one-at-a-time path."""
    import numpy as np
    import synth
    from paper_1712_05834_gb300 import serve
    from paper_1712_05834_gb300.batch import Catalog
    pool = mock_catalogs(torch, synth.mock_set_specs(64, synth.seed_for(5, 1000 * rank)))
    big = Catalog(synth.lognormal_catalog(130_000_000, MOCK_L, 512, synth.seed_for(5, 999 + 1000 * rank),
                                          device="cuda"), 1024, "tsc", True)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    rng = np.random.default_rng(synth.seed_for(5, 2 + 1000 * rank))
    large = rng.random(nreq) < 0.05
    pick = rng.integers(0, len(pool), nreq)
    cats = [big if large[i] else pool[int(pick[i])] for i in range(nreq)]
    arr = serve.poisson_arrivals(nreq, rate, synth.seed_for(5, 3 + 1000 * rank))

    def reqs(times):
        return [serve.Request(i, c, float(t), tag="large" if large[i] else "pool")
                for i, (c, t) in enumerate(zip(cats, times))]

    out = {}
    warm = reqs(np.zeros(nreq))[: min(nreq, 64)] + [serve.Request(-1, big, 0.0)]
    with serve.PowerServer(MOCK_L, dk=MOCK_DK, large_nmesh=1024) as srv:
        srv.run(warm, realtime=False)
        barrier(world)
        served = srv.run(reqs(arr), realtime=True)
        out["served"] = serve.latency_summary(served)
        sat = [serve.latency_summary(srv.run(reqs(np.zeros(nreq)), realtime=False)) for _ in range(repeats)]
        out["served"]["slots"] = srv.slots_made
        out["served"]["evictions"] = srv.evictions
    serve.plain_serve(warm, MOCK_L, realtime=False, dk=MOCK_DK)
    barrier(world)
    plain = serve.plain_serve(reqs(arr), MOCK_L, realtime=True, dk=MOCK_DK)
    out["plain"] = serve.latency_summary(plain)
    plain_sat = [serve.latency_summary(serve.plain_serve(reqs(np.zeros(nreq)), MOCK_L, realtime=False, dk=MOCK_DK))
                 for _ in range(repeats)]
    pick = lambda runs: sorted(runs, key=lambda r: r["pk_per_s"])[len(runs) // 2]      # the median run
    out["served_saturated"] = pick(sat)
    out["plain_saturated"] = pick(plain_sat)
    sv = [r["pk_per_s"] for r in sat]
    pl = [r["pk_per_s"] for r in plain_sat]
    by_id = {r.rid: r for r in plain}
    out["max_rel_diff_served_vs_plain"] = max(max_rel_diff(by_id[r.rid].result, r.result) for r in served)
    # the headline: latency of the pool requests (95 % of the stream) at the
    # arrival rate, and the saturated throughput of both paths over repeats
    out = {"pool_p99_ms": {"served": out["served"]["by_tag"]["pool"]["p99_ms"],
                           "plain": out["plain"]["by_tag"]["pool"]["p99_ms"]},
           "pool_p50_ms": {"served": out["served"]["by_tag"]["pool"]["p50_ms"],
                           "plain": out["plain"]["by_tag"]["pool"]["p50_ms"]},
           "saturated_pk_per_s": {"served_runs": sv, "plain_runs": pl,
                                  "served_median": statistics.median(sv), "plain_median": statistics.median(pl),
                                  "ratio_median": statistics.median(sv) / statistics.median(pl),
                                  "served_min_over_plain_max": min(sv) / max(pl)},
           **out}
    out["workload"] = ("Poisson arrivals, mean %.0f req/s, %d requests: 95%% from a pool of 64 mocks as in the "
                       "batched workload, 5%% large (Nmesh 1024, 1.3e8 objects, TSC + interlacing); "
                       "catalogs pre-staged in HBM; latency = arrival -> result on the host" % (rate, nreq))
    del pool, big, cats
    torch.cuda.empty_cache()
    return out


def measure_window_study(torch, rank):
    """The paper's window comparison setup: a log-normal catalog of 5e7
    objects, L = 2500, Nmesh 512, each window +- interlacing against PCS +
    interlacing on 1024^3; max |P / P_ref - 1| below fractions of k_N.  Two
    controls at the same number density: a uniform (Poisson) catalog, whose
    power is pure shot noise, and the log-normal recipe on a 1024^3 generator
    grid (objects uniform inside 2.4 instead of 4.9 Mpc/h cells)."""
    import numpy as np
    import synth
    from paper_1712_05834_gb300 import accuracy
    n, L = 50_000_000, 2500.0
    pos = synth.lognormal_catalog(n, L, 512, synth.seed_for(6, 1000 * rank), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = accuracy.window_study(pos, L, 512)
    wall = time.perf_counter() - t0
    del pos
    torch.cuda.empty_cache()
    controls = {}
    gen = torch.Generator(device="cuda").manual_seed(synth.seed_for(6, 1000 * rank + 1))
    upos = torch.rand((n, 3), generator=gen, device="cuda", dtype=torch.float32) * L
    controls["uniform"] = accuracy.window_study(upos, L, 512)["max_abs_dev"]["pcs+interlacing"]
    del upos
    torch.cuda.empty_cache()
    fpos = synth.lognormal_catalog(n, L, 1024, synth.seed_for(6, 1000 * rank), device="cuda")
    controls["lognormal_generator_grid_1024"] = accuracy.window_study(fpos, L, 512)["max_abs_dev"]["pcs+interlacing"]
    del fpos
    torch.cuda.empty_cache()
    kk = st["k_over_kN"]
    pick = np.unique(np.searchsorted(kk, [0.25, 0.5, 0.75, 0.9, 0.99]).clip(0, len(kk) - 1))
    return {"workload": "lognormal 5e7 objects, L=2500, Nmesh 512 vs PCS + interlacing on 1024^3, "
                        "compensated, raw power (before shot-noise subtraction), dk = 2 kF to k_N",
            "max_abs_dev": st["max_abs_dev"],
            "ratio_minus_1_at": {"%.3f kN" % kk[i]: {n_: float(r[i] - 1.0) for n_, r in st["ratio"].items()}
                                 for i in pick},
            "pcs_interlaced_controls": controls,
            "wall_s": wall}


def measure_window_speed(pk, torch, stream, pos, reps=10, warmup=3):
    """Paint time (sort + tile paint) of the main catalog for each window,
    with and without interlacing, beside the paper's relative paint speeds
    (TSC about 10 %, PCS about 40 % slower than CIC, Sec. 3.3.2)."""
    out = {}
    try:
        for window in ("cic", "tsc", "pcs"):
            for il in (False, True):
                plan = pk.pk_plan(pk.make_config(L_BOX, NMESH, window, interlaced=il, dk=DK), stream)
                try:
                    pk.pk_enable_timing(plan, True)
                    ts = []
                    for k in range(warmup + reps):
                        pk.pk_paint(plan, pos)
                        pk.pk_compute(plan)
                        pk.pk_result(plan, 0)
                        st = pk.pk_stage_times(plan)
                        if k >= warmup:
                            ts.append(st["sort"] + st["paint"])
                finally:
                    pk.pk_destroy(plan)
                out[window + ("+interlacing" if il else "")] = statistics.median(ts)
    except Exception as e:             # a side measurement never costs the main line
        return {"error": repr(e)}
    base = out["cic"]
    return {"workload": "the main catalog (1e7 log-normal objects) on 512^3, sort + tile paint, median of %d"
                        % reps,
            "ms": out, "ratio_to_cic": {k: v / base for k, v in out.items()}}


def measure_survey(pk, torch, stream, world, rank, steps=5, warmup=2):
    """Survey multipoles (ConvolvedFFTPower) on the paper's "small" benchmark
    sample: 1e6 galaxies in a 2500 Mpc/h survey volume, Nmesh 1024, l = 0, 2,
    4 (1 + 5 + 9 = 15 r2c FFTs), here with 1e7 randoms, CIC, compensated."""
    import numpy as np
    import synth
    ext, N, dk = 2500.0, 1024, 0.005
    t0 = time.perf_counter()
    c = synth.survey_catalogs(1_000_000, 10_000_000, ext, synth.seed_for(9, 100 + rank), ngrid=256,
                              device="cuda")
    gen_s = time.perf_counter() - t0
    L, origin = 1.04 * ext, (-0.02 * ext,) * 3
    nd, nr = len(c["data"]), len(c["randoms"])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    dp, dw, dn, rp, rn = (dev(c["data"]), dev(c["data_wcomp"]), dev(c["data_nbar"]), dev(c["randoms"]),
                          dev(c["rand_nbar"]))
    del c
    gd = pk.survey_catalog(dp, wcomp=dw, nbar=dn)
    gr = pk.survey_catalog(rp, nbar=rn)
    cfg = pk.make_survey_config(L, origin, N, "cic", False, dk=dk, capacity=nd + nr)
    plan = pk.pk_survey_plan(cfg, stream)
    pk.pk_survey_enable_timing(plan, True)
    times, stages = [], {s: [] for s in pk.SURVEY_STAGES}
    try:
        for k in range(warmup + steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pk.pk_survey_paint(plan, gd, gr)
            pk.pk_survey_compute(plan)
            res = pk.pk_survey_result(plan)
            b.record(stream)
            b.synchronize()
            st = pk.pk_survey_stage_times(plan)
            if k >= warmup:
                times.append(a.elapsed_time(b))
                for s_ in pk.SURVEY_STAGES:
                    stages[s_].append(st[s_])
        launches = pk.pk_survey_launch_count(plan)
        free, total = torch.cuda.mem_get_info()
    finally:
        pk.pk_survey_destroy(plan)
    # The paper's companion benchmark: FFTPower, P(k, mu) in 10 mu bins on the
    # same mesh, here of the same galaxies in the survey's box frame.
    box_pos = (dp - torch.tensor(origin, dtype=torch.float32, device="cuda")).contiguous()
    fcfg = pk.make_config(L, N, "cic", dk=dk, nmu=10)
    fplan = pk.pk_plan(fcfg, stream)
    ftimes = []
    try:
        for k in range(warmup + steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pk.pk_paint(fplan, box_pos)
            pk.pk_compute(fplan)
            pk.pk_result(fplan, 0)
            b.record(stream)
            b.synchronize()
            if k >= warmup:
                ftimes.append(a.elapsed_time(b))
    finally:
        pk.pk_destroy(fplan)
        del box_pos
        del dp, dw, dn, rp, rn
        torch.cuda.empty_cache()
    total_s = max_over_ranks(sum(times) / 1e3, world)
    med = {s_: statistics.median(v) for s_, v in stages.items()}
    hbm, peak_kind = peaks()
    nbinned = binned_stored_modes(N, L, dk)
    cells = N ** 3
    bin_bytes = 15 * nbinned * 8                   # A_0 + 14 Y_lm transforms, complex64 per binned mode
    field_bytes = cells * (2 * 4 + 15 * 4)         # read D, R; write F (A_0) + 14 weighted copies
    roof = {
        "k_survey_bin": {"ms": med["bin"], "bytes": bin_bytes,
                         "per_unit": "8 B per binned stored mode per transform (15 transforms)"},
        "k_survey_ylm": {"ms": med["field"], "bytes": field_bytes,
                         "per_unit": "8 B read + 60 B written per cell (D, R in; F and 14 F Y_lm out)"},
    }
    for r in roof.values():
        r["achieved"] = r["bytes"] / r["ms"] / 1e6
        r["bound"], r["peak"], r["frac"], r["unit"] = "hbm", hbm, r["bytes"] / r["ms"] / 1e6 / hbm, "GB/s"
        r["peak_kind"] = peak_kind
    ok = res["modes"] > 0
    kk = res["k"][ok]
    pick = np.unique(np.searchsorted(kk, [0.02, 0.05, 0.1, 0.2, 0.5]).clip(0, len(kk) - 1))
    return {"workload": "survey octant (observer at the corner, radii 0.2-0.95 x 2500 Mpc/h, radial "
                        "selection), 1e6 clustered galaxies (log-normal) + 1e7 randoms, box 2600 Mpc/h, "
                        "Nmesh 1024, CIC, compensated, dk 0.005 to k_N, l = 0, 2, 4 (15 r2c FFTs), FKP sums FP64",
            "multipoles_per_s": world * steps / total_s, "ms_per_step": 1e3 * total_s / steps,
            "stage_ms_median": med, "fft_count_per_step": 15,
            "fftpower_same_mesh_ms": statistics.median(ftimes),
            "ratio_to_fftpower": (1e3 * total_s / steps) / statistics.median(ftimes),
            "objects_per_step": nd + nr, "rooflines": roof, "gpu_launches_per_step": launches // (warmup + steps),
            "alpha": res["alpha"], "shot_noise": res["shot_noise"],
            "poles_at": {"%.3f" % kk[i]: [float(res["poles"][r_][ok][i]) for r_ in range(3)] for i in pick},
            "device_mem_used_gb": (total - free) / 1e9, "generation_s": gen_s}


def survey_profile(nmesh):
    """Three paint + compute evaluations of the survey multipoles on a small
    catalog (the small case the survey kernels are profiled on)."""
    import numpy as np
    import torch
    import synth
    import paper_1712_05834_gb300 as pk
    pk.build()
    torch.cuda.set_device(0)
    ext = 1000.0
    c = synth.survey_catalogs(100_000, 1_000_000, ext, synth.seed_for(9, 7), ngrid=128, device="cuda")
    L, origin = 1.04 * ext, (-0.02 * ext,) * 3
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    gd = pk.survey_catalog(dev(c["data"]), wcomp=dev(c["data_wcomp"]), nbar=dev(c["data_nbar"]))
    gr = pk.survey_catalog(dev(c["randoms"]), nbar=dev(c["rand_nbar"]))
    stream = torch.cuda.Stream()
    plan = pk.pk_survey_plan(pk.make_survey_config(L, origin, nmesh, "cic", False, dk=0.005,
                                                   capacity=len(c["data"]) + len(c["randoms"])), stream)
    pk.pk_survey_enable_timing(plan, True)
    try:
        for _ in range(3):
            pk.pk_survey_paint(plan, gd, gr)
            pk.pk_survey_compute(plan)
            pk.pk_survey_result(plan)
            print(json.dumps(pk.pk_survey_stage_times(plan)), flush=True)
    finally:
        pk.pk_survey_destroy(plan)
    return 0


def zeldovich_profile():
    """Two paint + compute steps of the 1024^3-object Zel'dovich lattice on
    2048^3 meshes (PCS + interlacing), the workload of `nmesh_2048`, with
    per-stage times: the run a launch list of that configuration is taken on."""
    import torch
    import synth
    import paper_1712_05834_gb300 as pk
    pk.build()
    torch.cuda.set_device(0)
    L, N = 2000.0, 2048
    pos = synth.zeldovich_lattice(1024, L, synth.seed_for(3), device="cuda")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    stream = torch.cuda.Stream()
    plan = pk.pk_plan(pk.make_config(L, N, "pcs", interlaced=True, dk=DK, nmu=NMU, precision="f32"), stream)
    pk.pk_enable_timing(plan, True)
    try:
        for _ in range(2):
            pk.pk_paint(plan, pos)
            pk.pk_compute(plan)
            pk.pk_result(plan, 0)
            print(json.dumps(pk.pk_stage_times(plan)), flush=True)
    finally:
        pk.pk_destroy(plan)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.survey_profile:
        return survey_profile(args.survey_profile)
    if args.zeldovich_profile:
        return zeldovich_profile()
    import numpy as np
    import torch

    import paper_1712_05834_gb300 as pk
    world, rank, local = dist_setup(args.gpus)
    pk.build()
    pk.load()
    stream = torch.cuda.Stream()
    pos = make_catalog(rank, "cuda")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()                     # drop the generator's temporaries
    cfg = pk.make_config(L_BOX, NMESH, "tsc", interlaced=True, dk=DK, nmu=NMU, precision="f32")
    with torch.cuda.stream(stream):
        plan = pk.pk_plan(cfg, stream)
        pk.pk_use_own_fft(plan, True)            # the library's own FFT passes (its default at this size)
        pk.pk_enable_timing(plan, True)
        flush = torch.empty((1 if args.profile else 512) * 1024 * 1024, dtype=torch.uint8, device="cuda")

        def step():
            pk.pk_paint(plan, pos)
            pk.pk_compute(plan)
            return pk.pk_result(plan, 0)

        for _ in range(max(args.warmup, 3)):
            res = step()
        torch.cuda.synchronize()
        uuid = None
        try:
            uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
        except Exception:
            pass
        clocks = ClockSampler(None if args.profile else uuid)
        if not args.profile:
            clocks.start()
            time.sleep(0.3)
        barrier(world)
        torch.cuda.synchronize()
        launches0 = pk.pk_launch_count(plan)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        stages = {s: [] for s in pk.STAGES}
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)                      # L2 flush, outside the events
            ev[k][0].record(stream)
            res = step()
            ev[k][1].record(stream)
            st = pk.pk_stage_times(plan)
            for s in pk.STAGES:
                stages[s].append(st[s])
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - wall0
        launches = pk.pk_launch_count(plan) - launches0
        clk = clocks.stop()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        total_s = max_over_ranks(sum(step_ms) / 1e3, world)

        # e2e through the public API with host (pinned) buffers: every step
        # copies its catalog (12 B per object) to the device and reads its
        # result back
        e2e_steps, e2e_s, e2e_one_s = 0, float("nan"), float("nan")
        if not args.profile:
            from paper_1712_05834_gb300.pipeline import PowerStream
            host = pos.cpu().pin_memory()
            e2e_steps = max(3, min(args.steps, 50))
            # one plan, one catalog at a time: each copy waits for the
            # previous catalog's kernels and delays its own
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                pk.pk_paint(plan, host)
                pk.pk_compute(plan)
                pk.pk_result(plan, 0)
            torch.cuda.synchronize()
            e2e_one_s = max_over_ranks(time.perf_counter() - t0, world)
            # two plans deep (PowerStream): a catalog's copy and kernels run
            # while the previous catalog's kernels still occupy the GPU
            with PowerStream(cfg, depth=2, own_fft=True) as ps:
                for _ in ps.map([host] * 4):            # warm-up: staging buffers
                    pass
                torch.cuda.synchronize()
                barrier(world)
                t0 = time.perf_counter()
                for _ in ps.map([host] * e2e_steps):
                    pass
                torch.cuda.synchronize()
                e2e_s = max_over_ranks(time.perf_counter() - t0, world)
        pk.pk_destroy(plan)
        pipelined = None if args.profile else measure_pipelined(torch, cfg, pos, max(10, min(args.steps, 200)))
        fp64, res64 = (None, None) if (args.no_fp64 or args.profile) else measure_fp64_form(pk, torch, stream, pos,
                                                                                           flush)
        del flush
        torch.cuda.empty_cache()
        windows = None if (args.no_windows or args.profile) else measure_window_speed(pk, torch, stream, pos)
        big = None if (args.no_2048 or args.profile) else measure_2048(pk, torch, stream, world)
        batched = None if (args.no_batched or args.profile) else measure_batched(pk, torch, world, rank)
        served = None if (args.no_serve or args.profile) else measure_serving(pk, torch, world, rank,
                                                                              args.serve_requests)
        study = None if (args.no_study or args.profile) else measure_window_study(torch, rank)
        survey = None if (args.no_survey or args.profile) else measure_survey(pk, torch, stream, world, rank)

    if rank != 0:
        return 0
    K = args.steps
    value = job_rate(world, K, total_s)
    med = {s: statistics.median(v) for s, v in stages.items()}
    nmodes = NMESH * NMESH * (NMESH // 2 + 1)
    nbinned = binned_stored_modes()
    hbm, peak_kind = peaks()
    # algorithmic bytes per launch (what the step must move; extra traffic counts against it)
    tile_bytes = NPART * 16 + 2 * NMESH ** 3 * 4            # sorted float4 in + 2 FP32 meshes out
    stage_bytes = NPART * 12 + 2 * NMESH ** 3 * 4           # xyz FP32 in + 2 FP32 meshes out
    axis_bytes = 2 * 2 * NMESH ** 3 // 2 * 8                # read + write of 2 packed complex64 meshes
    zbin_bytes = 2 * zbin_rows() * (NMESH // 2) * 8          # the packed rows holding binned modes, 2 meshes
    roof = {
        "k_paint_tiles": {"achieved": tile_bytes / med["paint"] / 1e6, "ms": med["paint"], "bytes": tile_bytes,
                          "launches_per_step": 1,
                          "per_unit": "16 B per object (its sorted float4) + 4 B per cell per mesh"},
        "k_fft_axis": {"achieved": axis_bytes / (med["fft"] / 2) / 1e6, "ms": med["fft"] / 2, "bytes": axis_bytes,
                       "launches_per_step": 2,
                       "per_unit": "16 B per packed complex element (z pairs) per mesh: read and write once, "
                                   "one launch per axis (y, x)"},
        "k_zbin": {"achieved": zbin_bytes / med["bin"] / 1e6, "ms": med["bin"], "bytes": zbin_bytes,
                   "launches_per_step": 1,
                   "per_unit": "8 B per packed element of the rows (kx, ky) that hold a binned mode, per mesh"},
        "paint_stage": {"achieved": stage_bytes / (med["sort"] + med["paint"]) / 1e6,
                        "ms": med["sort"] + med["paint"], "bytes": stage_bytes,
                        "kernels": "k_sort_count + k_scan_* + k_sort_scatter + k_paint_tiles",
                        "per_unit": "12 B per object (FP32 xyz) + 4 B per cell per mesh"},
    }
    for r in roof.values():
        r["bound"] = "hbm"
        r["peak"] = hbm
        r["frac"] = r["achieved"] / hbm
    # the dominant kernel: the most device time per step
    dom = max((k for k in roof if k.startswith("k_")), key=lambda k: roof[k]["ms"] * roof[k]["launches_per_step"])
    rl = {"bound": "hbm", "achieved": roof[dom]["achieved"], "peak": hbm, "unit": "GB/s",
          "frac": roof[dom]["frac"], "traffic": traffic_record(dom), "kernel": dom,
          "peak_kind": peak_kind, "algorithmic_bytes_per_launch": roof[dom]["bytes"],
          "launch_ms": roof[dom]["ms"]}
    res_bytes = 8 * (len(res["power"]) * 4 + res["power2d"].size + 4)
    line = {
        "metric": METRIC, "value": value, "unit": "P(k)/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nmesh": NMESH, "particles": NPART,
                   "form": "FP32 mesh, int64 fixed-point paint, FP32 per-mode arithmetic and per-CTA bin "
                           "partials, FP64 cross-CTA sums and finalize",
                   "l2": "flushed between steps (512 MB device write outside the timed events)",
                   "parallelism": "replicas" if world == 1 else "dp%d (independent catalogs)" % world},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "particles_painted_per_s": NPART / ((med["sort"] + med["paint"]) / 1e3),
        "modes_binned_per_s": nbinned / (med["bin"] / 1e3),
        "stored_modes": nmodes, "binned_stored_modes": nbinned,
        "stage_ms_median": med,
        "fft_ms": med["fft"],
        "roofline": rl,
        "rooflines": roof,
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": {"value": world * e2e_steps / e2e_s, "unit": "P(k)/s",
                "h2d_bytes_per_step": int(NPART * 12), "d2h_bytes_per_step": int(res_bytes),
                "steps": e2e_steps,
                "api": "pipeline.PowerStream(cfg, depth=2).map(pinned host catalogs): pk_paint from host "
                       "memory, pk_compute, pk_result per catalog, two plans on two streams",
                "one_plan": {"value": world * e2e_steps / e2e_one_s, "unit": "P(k)/s",
                             "api": "pk_paint(plan, host), pk_compute, pk_result on one plan"}},
        "wall_s_timed": wall,
    }
    if pipelined is not None:
        line["pipelined"] = pipelined
    if big is not None:
        line["nmesh_2048"] = big
    if batched is not None:
        line["batched_mocks"] = batched
    if served is not None:
        line["serving"] = served
    if study is not None:
        line["window_study"] = study
    if survey is not None:
        line["survey_multipoles"] = survey
    if windows is not None:
        line["paint_by_window"] = windows
    if fp64 is not None:
        line["fp64_form"] = fp64
    if world == 1 and not args.no_cpu_baseline and not args.profile:
        import oracle
        oracle.build()
        pos64 = pos.double().cpu().numpy()
        t, ores = oracle_step(pos64)
        line["cpu_baseline"] = {"value": 1.0 / t, "unit": "P(k)/s", "cores": oracle.threads(), "kind": "oracle",
                                "sample": oracle_sample_text(oracle.threads())}
        # the same catalog's oracle result: per-bin error of each GPU form
        line["max_err_vs_oracle"] = {"f32_form": per_bin_errors(res, ores),
                                     "note": "max over bins of |dX| / P_raw,0(b), X = P, P(k,mu), P_0, P_2, "
                                             "P_4; tolerance 1e-4 (FP32 form), 1e-6 (FP64 form)"}
        if res64 is not None:
            line["max_err_vs_oracle"]["f64_form"] = per_bin_errors(res64, ores)
        line["cpu_baseline"]["tiny_workload"] = oracle_tiny()
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
