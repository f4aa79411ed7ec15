"""The catalog weight sums (sum w, sum w^2 of the painted amplitudes) that
normalize P(k) and set its shot noise (Sec. 3.4.1): each paint block keeps
its partial sums in a row of its own and one kernel adds the rows in a fixed
order, so repeated paints of the same catalog give the same bits, with both
paint variants, for weights given apart or as the fourth position component,
and painted values.  Against an FP64 sum on the host of the same FP32
amplitudes (W V is formed in FP32, one rounded product, then summed and
squared in FP64): 1e-12 relative."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk
    pk.build()
    pk.load()
    return pk


def _sums(pk, cfg, paint, runs=4):
    plan = pk.pk_plan(cfg)
    try:
        out = []
        for _ in range(runs):
            paint(plan)
            pk.pk_compute(plan)
            r = pk.pk_result(plan, 0)
            out.append((r["wsum"], r["w2sum"], r["shot_noise"]))
        return out
    finally:
        pk.pk_destroy(plan)


@pytest.mark.parametrize("variant", ["sort", "atomic"])
def test_weight_sums_are_run_to_run_identical(pk, variant):
    import torch
    n, L = 3_000_000, 500.0
    rng = np.random.default_rng(31)
    pos = (rng.random((n, 3)) * L).astype(np.float32)
    w = rng.uniform(0.5, 1.5, n).astype(np.float32)
    v = rng.normal(0.0, 1.0, n).astype(np.float32)
    dpos, dw, dv = torch.from_numpy(pos).cuda(), torch.from_numpy(w).cuda(), torch.from_numpy(v).cuda()
    xyzw = torch.cat([dpos, dw[:, None]], 1).contiguous()
    cfg = pk.make_config(L, 128, "tsc", interlaced=True, dk=0.05, paint_variant=variant)
    w64 = w.astype(np.float64)
    for paint, amp in ((lambda p: pk.pk_paint(p, dpos, dw), w64),
                       (lambda p: pk.pk_paint(p, xyzw), w64),
                       (lambda p: pk.pk_paint_values(p, dpos, dv, weights=dw), (w * v).astype(np.float64))):
        runs = _sums(pk, cfg, paint)
        assert all(r == runs[0] for r in runs[1:]), runs
        wsum, w2sum, _ = runs[0]
        assert abs(wsum - w64.sum()) <= 1e-12 * w64.sum()
        assert abs(w2sum - (amp * amp).sum()) <= 1e-12 * (amp * amp).sum()


def test_weight_sums_of_a_batch(pk):
    import torch
    L = 500.0
    rng = np.random.default_rng(32)
    sizes = [700_000, 1_300_000, 1]
    pos = torch.from_numpy((rng.random((sum(sizes), 3)) * L).astype(np.float32)).cuda()
    w = torch.from_numpy(rng.uniform(0.5, 1.5, sum(sizes)).astype(np.float32)).cuda()
    off = np.concatenate([[0], np.cumsum(sizes)])
    cfg = pk.make_config(L, 64, "cic", dk=0.1, batch=3)
    plan = pk.pk_plan(cfg)
    try:
        got = []
        for _ in range(3):
            pk.pk_paint_many(plan, pos, off, w)
            pk.pk_compute(plan)
            got.append([pk.pk_result(plan, k)["wsum"] for k in range(3)])
        assert got[1] == got[0] and got[2] == got[0]
        w64 = w.double().cpu().numpy()
        for k in range(3):
            ref = w64[off[k]:off[k + 1]].sum()
            assert abs(got[0][k] - ref) <= 1e-12 * ref
    finally:
        pk.pk_destroy(plan)
