"""Pins of the survey-multipole oracle (oracle/survey.py) to mathematics and
to the already pinned periodic-box oracle, independent of the oracle's own
code paths:

* distances: chi(z) against the closed forms of an Einstein-de Sitter
  universe (Om = 1) and of a pure cosmological constant (Om = 0), and
  against scipy's adaptive quadrature for Om = 0.31;
* sky -> Cartesian: the axes and the radius;
* the Cartesian-moment route to A_l equals the definition summed over every
  node for every mode (Legendre polynomials from numpy), for observers
  outside the box, inside it and exactly on a node;
* a far observer: the local line of sight becomes +z, and the survey bin sums
  equal the periodic-box multipole sums of the pinned FFTPower oracle on the
  same field (plain and interlaced, every window);
* the FKP field has zero mean with unit FKP weights, and a uniform
  full-box survey has I = (sum w)^2 / V;
* Poisson data and randoms: P_0 before shot-noise subtraction over the shot
  noise S follows the analytic aliased shot-noise factor of the box tests
  (chi^2 over seeds), which fixes the alpha^2 term of S; a planted S without
  it is rejected.
"""
import math

import numpy as np
import pytest

from test_oracle_pins import expected_shot


@pytest.fixture(scope="module")
def sv(oracle):
    import oracle.survey as survey
    return survey


def test_comoving_distance_closed_forms(sv):
    z = np.array([0.0, 0.01, 0.3, 0.57, 1.0, 2.5])
    eds = 2.0 * sv.C_OVER_H0 * (1.0 - 1.0 / np.sqrt(1.0 + z))
    np.testing.assert_allclose(sv.comoving_distance(z, 1.0), eds, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(sv.comoving_distance(z, 0.0), sv.C_OVER_H0 * z, rtol=1e-13, atol=1e-12)
    quad = pytest.importorskip("scipy.integrate").quad
    om = 0.31
    ref = [sv.C_OVER_H0 * quad(lambda x: 1.0 / math.sqrt(om * (1 + x) ** 3 + 1 - om), 0.0, zz,
                               epsabs=0, epsrel=1e-13)[0] for zz in z]
    np.testing.assert_allclose(sv.comoving_distance(z, om), ref, rtol=1e-12, atol=1e-12)


def test_sky_to_cartesian_axes(sv):
    z = np.array([0.5, 0.5, 0.5, 0.5])
    chi = sv.comoving_distance(0.5, 0.3)
    x = sv.sky_to_cartesian([0.0, 90.0, 123.0, 180.0], [0.0, 0.0, 90.0, -45.0], z, 0.3)
    want = np.array([[chi, 0, 0], [0, chi, 0], [0, 0, chi],
                     [-chi / math.sqrt(2), 0, -chi / math.sqrt(2)]])
    np.testing.assert_allclose(x, want, atol=1e-9 * chi)
    rng = np.random.default_rng(0)
    ra, dec, zz = rng.uniform(0, 360, 50), rng.uniform(-90, 90, 50), rng.uniform(0, 2, 50)
    r = np.linalg.norm(sv.sky_to_cartesian(ra, dec, zz, 0.3), axis=1)
    np.testing.assert_allclose(r, sv.comoving_distance(zz, 0.3), rtol=1e-14)


@pytest.mark.parametrize("N,L,origin", [
    (8, 80.0, (-3.0, 5.0, 20.0)),        # observer inside the box, off the nodes
    (8, 80.0, (-40.0, -40.0, -40.0)),    # observer exactly on node (4, 4, 4)
    (8, 80.0, (150.0, -300.0, 90.0)),    # observer outside the box
    (12, 60.0, (-31.0, -2.5, -17.0)),
])
def test_cartesian_moments_equal_definition(sv, N, L, origin):
    rng = np.random.default_rng(N + abs(int(origin[0])))
    F = rng.normal(size=(N, N, N))
    A = sv.multipole_fields(F, L, origin)
    B = sv.multipoles_direct(F, L, origin)
    scale = np.max(np.abs(B[0]))
    for ell in (0, 2, 4):
        assert np.max(np.abs(A[ell] - B[ell])) <= 1e-12 * scale, ell


@pytest.mark.parametrize("window,interlaced", [("cic", False), ("tsc", True), ("pcs", True), ("pcs", False)])
def test_far_observer_reduces_to_box_multipoles(oracle, sv, window, interlaced):
    N, L = 32, 200.0
    rng = np.random.default_rng(7)
    pos = rng.uniform(0, L, size=(6000, 3))
    pos[:3000, 2] = np.mod(pos[:3000, 2] + 8.0 * np.sin(2 * math.pi * pos[:3000, 0] / L), L)   # anisotropy
    w = rng.uniform(0.5, 1.5, len(pos))
    F1 = oracle.paint(pos, w, L, N, window, 0.0)
    F2 = oracle.paint(pos, w, L, N, window, 0.5) if interlaced else None
    dk = 2 * (2 * math.pi / L)
    box = oracle.bin_modes(oracle.r2c(F1), None if F2 is None else oracle.r2c(F2), L, window, True,
                           w.sum(), dk)
    origin = (-0.5 * L, -0.5 * L, 1e10)
    A = sv.multipole_fields(sv.interlaced_field(F1, F2), L, origin)
    got = sv.bin_multipoles(A, L, window, True, dk)
    assert np.array_equal(got["modes"], box["modes1d"])
    np.testing.assert_allclose(got["ksum"], box["ksum1d"], rtol=1e-12)
    conv = L ** 3 / w.sum() ** 2
    scale = box["psum1d"]
    for ell, key in ((0, "psum1d"), (2, "p2sum1d"), (4, "p4sum1d")):
        assert np.all(np.abs(got["sums"][ell] * conv - box[key]) <= 1e-6 * scale), ell


def test_fkp_field_zero_mean_and_uniform_normalization(sv):
    L, N = 300.0, 16
    rng = np.random.default_rng(11)
    nd, nr = 4000, 40000
    dpos, rpos = rng.uniform(0, L, (nd, 3)), rng.uniform(0, L, (nr, 3))
    wd, wr = rng.uniform(0.5, 1.5, nd), rng.uniform(0.5, 1.5, nr)
    ds, rs = sv.catalog_sums(wd, None, None, nd), sv.catalog_sums(wr, None, None, nr)
    alpha = ds["wsum"] / rs["wsum"]
    (F,) = sv.fkp_meshes(dpos, wd, rpos, wr, alpha, L, (0.0, 0.0, 0.0), N, "tsc", False)
    assert abs(F.sum()) <= 1e-11 * wd.sum()
    nbar = nd / L ** 3
    c = sv.fkp_constants(sv.catalog_sums(None, None, np.full(nd, nbar), nd),
                         sv.catalog_sums(None, None, np.full(nr, nbar), nr))
    assert abs(c["alpha"] - nd / nr) <= 1e-15
    assert abs(c["norm"] - nd ** 2 / L ** 3) <= 1e-12 * nd ** 2 / L ** 3
    assert abs(c["shot_noise"] - (nd + (nd / nr) ** 2 * nr) / (nd ** 2 / L ** 3)) <= 1e-12 * c["shot_noise"]


def _poisson_survey_chi2(sv, window, interlaced, seeds, drop_alpha2=False):
    from scipy import stats
    N, L, nd, nr = 32, 500.0, 30000, 150000
    p = {"cic": 2, "tsc": 3, "pcs": 4}[window]
    dk = 2 * (2 * math.pi / L)
    nk = int(math.floor((math.pi * N / L) / dk))
    Eb, var = expected_shot(N, L, p, interlaced, dk, nk)
    chi2, dof, zmax = 0.0, 0, 0.0
    for seed in seeds:
        rng = np.random.default_rng(seed)
        nbar = nd / L ** 3
        data = {"pos": rng.uniform(0, L, (nd, 3)), "wcomp": rng.uniform(0.5, 1.5, nd), "nbar": np.full(nd, nbar)}
        rand = {"pos": rng.uniform(0, L, (nr, 3)), "nbar": np.full(nr, nbar)}
        res = sv.convolved_power(data, rand, L, (-0.5 * L, -0.5 * L, 1e9), N, window, interlaced, True, dk,
                                 poles=(0,), subtract_shot=False)
        shot = res["shot_noise"]
        if drop_alpha2:
            shot = res["data_sums"]["w2sum"] / res["norm"]
        z = (res["power_raw"] / shot - Eb) / np.sqrt(var)
        chi2 += float(np.sum(z ** 2))
        dof += nk
        zmax = max(zmax, float(np.max(np.abs(z))))
    return chi2, dof, zmax, stats.chi2.sf(chi2, dof)


@pytest.mark.parametrize("window,interlaced", [("cic", False), ("pcs", True)])
def test_poisson_survey_gives_fkp_shot_noise(sv, window, interlaced):
    chi2, dof, zmax, pval = _poisson_survey_chi2(sv, window, interlaced, seeds=[301, 302, 303])
    assert zmax < 5.0 and pval > 1e-4, (chi2, dof, zmax, pval)


def test_planted_shot_noise_without_randoms_term_is_rejected(sv):
    chi2, dof, zmax, pval = _poisson_survey_chi2(sv, "cic", False, seeds=[301, 302, 303], drop_alpha2=True)
    assert pval < 1e-6, (chi2, dof, pval)


def test_planted_global_line_of_sight_is_rejected(sv):
    """Negative control for the per-node pin: multipoles about a fixed z axis
    (an observer far away) differ from the local-line-of-sight definition for
    an observer near the box, far beyond rounding."""
    N, L, near = 8, 80.0, (-40.0, -35.0, -30.0)
    rng = np.random.default_rng(5)
    F = rng.normal(size=(N, N, N))
    truth = sv.multipoles_direct(F, L, near)
    planted = sv.multipole_fields(F, L, (-0.5 * L, -0.5 * L, 1e12))
    scale = np.max(np.abs(truth[0]))
    assert np.max(np.abs(planted[2] - truth[2])) > 1e-2 * scale
    assert np.max(np.abs(planted[4] - truth[4])) > 1e-2 * scale
