"""Pins of the oracle's lattice tables and entropic equilibrium.

The equilibrium is the minimiser of Eq. (3) under the mass and momentum
constraints stated after it.  Pins, none of which retypes the oracle's
product formula:
  * lattice tables: normalisation, isotropy up to fourth order (c_s^2 = 1/3),
    opposite-pair ordering;
  * the constraints hold to rounding;
  * ln(f^eq / W) lies in the span of the collision invariants {1, c}
    (stationarity of the constrained minimum);
  * H(f^eq + e d) > H(f^eq) for random d in the constraint null space;
  * agreement with an independent 60-digit Newton solve for the Lagrange
    multipliers;
  * per-axis second moment sum c_a^2 f^eq = rho (2 sqrt(1 + 3 u_a^2) - 1) / 3,
    a consequence of the minimiser derived separately.
"""
import itertools

import numpy as np
import pytest

import mp_reference as mpr

LATS = ["D1Q3", "D2Q9", "D3Q27"]


@pytest.mark.parametrize("lat", LATS)
def test_lattice_tables(orc, lat):
    c, w = orc.lattice(lat)
    d = orc.dim(lat)
    q = len(w)
    assert q == 3 ** d
    # every velocity of {-1,0,1}^d exactly once, rest first, +/- pairs
    vel = {tuple(ci[:d]) for ci in c}
    assert vel == set(itertools.product((-1, 0, 1), repeat=d))
    assert np.all(c[0] == 0)
    for k in range(1, q, 2):
        assert np.all(c[k] == -c[k + 1])
    assert np.all(c[:, d:] == 0)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    second = np.einsum("i,ia,ib->ab", w, c[:, :d], c[:, :d])
    assert np.allclose(second, np.eye(d) / 3.0, atol=1e-15)
    for a in range(d):
        assert abs(w @ c[:, a] ** 4 - 1.0 / 3.0) < 1e-15
        for b in range(d):
            if a != b:
                assert abs(w @ (c[:, a] ** 2 * c[:, b] ** 2) - 1.0 / 9.0) < 1e-15
    # weights are products of the D1Q3 weights (tensor-product lattice)
    w1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0, -1: 1.0 / 6.0}
    for ci, wi in zip(c, w):
        assert abs(wi - np.prod([w1[int(v)] for v in ci[:d]])) < 1e-16


def _random_states(rng, d, n=30):
    for _ in range(n):
        rho = rng.uniform(0.5, 2.0)
        u = rng.uniform(-0.4, 0.4, size=d)
        yield rho, u
    yield 1.0, np.zeros(d)
    yield 1.3, np.full(d, 0.9)     # close to the |u| < 1 limit


@pytest.mark.parametrize("lat", LATS)
def test_constraints_and_stationarity(orc, lat):
    c, w = orc.lattice(lat)
    d = orc.dim(lat)
    rng = np.random.default_rng(1)
    basis = np.column_stack([np.ones(len(w)), c[:, :d]])
    for rho, u in _random_states(rng, d):
        feq = orc.equilibrium(lat, rho, u)
        assert np.all(feq > 0)
        assert abs(feq.sum() - rho) <= 4e-15 * rho
        assert np.allclose(c[:, :d].T @ feq, rho * u, rtol=0, atol=8e-15 * rho)
        # ln(f^eq/W) = a + b.c exactly (entropic equilibrium structure)
        lg = np.log(feq / w)
        coef, *_ = np.linalg.lstsq(basis, lg, rcond=None)
        assert np.abs(basis @ coef - lg).max() < 2e-14 * (1 + np.abs(lg).max())


@pytest.mark.parametrize("lat", LATS)
def test_second_moment_closed_form(orc, lat):
    c, w = orc.lattice(lat)
    d = orc.dim(lat)
    rng = np.random.default_rng(2)
    for rho, u in _random_states(rng, d):
        feq = orc.equilibrium(lat, rho, u)
        for a in range(d):
            expect = rho * (2 * np.sqrt(1 + 3 * u[a] ** 2) - 1) / 3
            assert abs(c[:, a] ** 2 @ feq - expect) < 1e-14 * rho


@pytest.mark.parametrize("lat", LATS)
def test_minimality_under_null_space_perturbation(orc, lat):
    c, w = orc.lattice(lat)
    d = orc.dim(lat)
    rng = np.random.default_rng(3)
    A = np.vstack([np.ones(len(w)), c[:, :d].T])
    _, _, vt = np.linalg.svd(A)
    null = vt[d + 1:]                      # rows spanning {dl : A dl = 0}
    for rho, u in list(_random_states(rng, d))[:10]:
        feq = orc.equilibrium(lat, rho, u)
        h0 = np.sum(feq * np.log(feq / w))
        for _ in range(20):
            dl = rng.standard_normal(null.shape[0]) @ null
            eps = 1e-3 * feq.min() / np.abs(dl).max()
            f1 = feq + eps * dl
            assert np.abs(A @ (f1 - feq)).max() < 1e-15
            h1 = np.sum(f1 * np.log(f1 / w))
            assert h1 > h0


@pytest.mark.parametrize("lat", LATS)
def test_matches_independent_lagrange_newton(orc, lat):
    c, w = orc.lattice(lat)
    d = orc.dim(lat)
    rng = np.random.default_rng(4)
    cc = [[int(v) for v in ci[:d]] for ci in c]
    ww = mpr.mpf_vec(w)
    for rho, u in list(_random_states(rng, d))[:6]:
        feq = orc.equilibrium(lat, rho, u)
        ref = mpr.equilibrium(cc, ww, mpr.mp.mpf(rho),
                              [mpr.mp.mpf(rho) * mpr.mp.mpf(v) for v in u])
        ref = np.array([float(v) for v in ref])
        assert np.abs(feq - ref).max() <= 1e-13 * ref.max()


def test_invalid_velocity_rejected(orc):
    with pytest.raises(ValueError):
        orc.equilibrium("D2Q9", 1.0, [1.0, 0.0])
    with pytest.raises(ValueError):
        orc.equilibrium("D2Q9", -1.0, [0.0, 0.0])
