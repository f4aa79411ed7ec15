"""The real spherical harmonics of the survey path (pk_survey_ylm, the same
functions the kernels evaluate), checked on the CPU against mathematics:
orthonormality on the sphere (a product rule exact for polynomials of degree
<= 15: Gauss-Legendre in cos(theta), equal steps in phi) and the addition
theorem sum_m Y_lm(a) Y_lm(b) = (2l + 1) / (4 pi) L_l(a.b) with Legendre
polynomials from numpy."""
import math

import numpy as np
import pytest

ELLS = [(2, m) for m in range(-2, 3)] + [(4, m) for m in range(-4, 5)]


@pytest.fixture(scope="module")
def pk():
    import paper_1712_05834_gb300 as pk
    pk.build()
    pk.load()
    return pk


def test_ylm_orthonormal_on_the_sphere(pk):
    ct, wt = np.polynomial.legendre.leggauss(12)
    phi = 2 * math.pi * np.arange(24) / 24
    pts, wts = [], []
    for c, w in zip(ct, wt):
        s = math.sqrt(1 - c * c)
        for p in phi:
            pts.append((s * math.cos(p), s * math.sin(p), c))
            wts.append(w * 2 * math.pi / 24)
    Y = np.array([[pk.pk_survey_ylm(l, m, *x) for x in pts] for l, m in ELLS])
    G = (Y * np.asarray(wts)[None, :]) @ Y.T
    np.testing.assert_allclose(G, np.eye(len(ELLS)), atol=1e-13)


@pytest.mark.parametrize("l", [2, 4])
def test_ylm_addition_theorem(pk, l):
    rng = np.random.default_rng(l)
    a = rng.normal(size=(40, 3))
    b = rng.normal(size=(40, 3))
    a /= np.linalg.norm(a, axis=1)[:, None]
    b /= np.linalg.norm(b, axis=1)[:, None]
    s = np.zeros(40)
    for m in range(-l, l + 1):
        s += np.array([pk.pk_survey_ylm(l, m, *x) * pk.pk_survey_ylm(l, m, *y) for x, y in zip(a, b)])
    coef = np.zeros(l + 1)
    coef[l] = 1.0
    want = (2 * l + 1) / (4 * math.pi) * np.polynomial.legendre.legval(np.sum(a * b, axis=1), coef)
    np.testing.assert_allclose(s, want, atol=1e-14)


def test_ylm_rejects_other_orders(pk):
    assert math.isnan(pk.pk_survey_ylm(3, 0, 0.0, 0.0, 1.0))
    assert math.isnan(pk.pk_survey_ylm(2, 3, 0.0, 0.0, 1.0))
