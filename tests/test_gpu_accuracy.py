"""The window / interlacing accuracy study (Sec. 3.3.2) on a small version
of the paper's setup: a log-normal catalog at the paper's number density and
cell size (1e6 objects, L = 625, Nmesh 128; the paper uses 5e7 objects,
L = 2500, Nmesh 512), each window with and without interlacing against a
PCS + interlacing reference on a mesh twice as fine.

What the paper states and what is checked: with interlacing all three windows
are sub-percent up to the Nyquist wavenumber, interlacing always helps, and
the higher-order PCS window is the most accurate (at k < k_N / 2 it reaches
the ~1e-5 level)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def study():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1712_05834_gb300 as pk
    import synth
    from paper_1712_05834_gb300 import accuracy
    pk.build()
    pk.load()
    pos = synth.lognormal_catalog(1_000_000, 625.0, 128, synth.seed_for(6, 0), device="cuda")
    return accuracy.window_study(pos, 625.0, 128)


def test_interlaced_windows_are_sub_percent_to_nyquist(study):
    for w in ("cic", "tsc", "pcs"):
        assert study["max_abs_dev"][w + "+interlacing"]["k<1.00kN"] < 1e-2, w


def test_interlacing_always_reduces_the_error(study):
    for w in ("cic", "tsc", "pcs"):
        for f in ("k<0.50kN", "k<0.75kN", "k<1.00kN"):
            assert study["max_abs_dev"][w + "+interlacing"][f] < study["max_abs_dev"][w][f], (w, f)


def test_pcs_interlaced_is_the_most_accurate(study):
    dev = study["max_abs_dev"]
    for f in ("k<0.50kN", "k<0.75kN", "k<1.00kN"):
        assert dev["pcs+interlacing"][f] == min(d[f] for d in dev.values()), f
    assert dev["pcs+interlacing"]["k<0.50kN"] < 5e-5
    assert dev["pcs+interlacing"]["k<1.00kN"] < 1e-3


def test_modes_and_ratios_cover_the_bins(study):
    assert len(study["k"]) == len(study["modes"]) > 10
    assert study["k_over_kN"].max() < 1.0
    for r in study["ratio"].values():
        assert r.shape == study["k"].shape


@pytest.mark.parametrize("precision,tol", [("f32", 1e-4), ("f64", 1e-6)])
def test_study_ratios_equal_the_oracles(oracle, precision, tol):
    """The same study computed by the FP64 oracle (2e5 log-normal objects,
    L = 312.5, 64^3 against PCS + interlacing on 128^3): every scheme's per-bin
    ratio P / P_ref from the CUDA path equals the oracle's within the form's
    tolerance."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import synth
    from paper_1712_05834_gb300 import accuracy
    L, N = 312.5, 64
    pos = synth.lognormal_catalog(200_000, L, N, synth.seed_for(6, 1), device="cuda")
    got = accuracy.window_study(pos, L, N, precision=precision)
    host = pos.double().cpu().numpy()
    kF = 2.0 * math.pi / L
    dk = 2.0 * kF
    kmax = math.floor((math.pi * N / L) / dk) * dk
    ref = oracle.fft_power(host, None, L, 2 * N, "pcs", True, True, dk=dk, kmax=kmax, subtract_shot=False)
    ok = ref["modes"] > 0
    assert np.array_equal(got["modes"], ref["modes"][ok])
    for window, il in accuracy.SCHEMES:
        r = oracle.fft_power(host, None, L, N, window, il, True, dk=dk, kmax=kmax, subtract_shot=False)
        ratio = r["power"][ok] / ref["power"][ok]
        name = accuracy.scheme_name(window, il)
        err = np.max(np.abs(got["ratio"][name] - ratio))
        assert err <= tol, (name, err)
