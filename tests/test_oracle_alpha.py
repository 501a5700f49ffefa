"""Pins of the oracle's entropy change Delta H(alpha) and its three choices
of alpha (Eq. (8)+(9) FORMULA, bisection ROOT, modified secant).

Every expected value comes from ``mp_reference`` (60-digit literal
H(f*) - H(f), equilibrium by an independent Newton solve, root of Eq. (4) by
200-step bisection) or from a property the paper states:
  * alpha_max > 1 and f*(alpha) >= 0 exactly on [0, alpha_max];
  * Delta H is convex and increasing on [1, alpha_max] (Fig. 1);
  * H(f*(alpha^(1))) <= H(f) for Eq. (9), and alpha^(1) <= alpha_bar
    (chord of a convex function);
  * the bisection stop rule -1e-13 <= Delta H <= 0;
  * the modified secant iterates keep Delta H <= 0 and converge to
    alpha_bar; its first iterate is Eq. (9).
A series identity derived for this build (Delta H(alpha) = sum_{k>=2}
(-1)^k (alpha^k - k alpha) / (k (k-1)) sum_i f_i x_i^k) is a further
independent check near equilibrium.
"""
import numpy as np
import pytest

import mp_reference as mpr

LATS = ["D1Q3", "D2Q9", "D3Q27"]
AMPS = [1e-6, 1e-4, 1e-2, 0.1, 0.45]


def _node(orc, lat, rng, amp):
    d = orc.dim(lat)
    rho = rng.uniform(0.8, 1.2)
    u = rng.uniform(-0.1, 0.1, size=d)
    feq = orc.equilibrium(lat, rho, u)
    return feq * (1.0 + amp * rng.uniform(-1, 1, size=len(feq)))


def _x(orc, lat, f):
    c, _ = orc.lattice(lat)
    d = orc.dim(lat)
    rho = f.sum()
    u = (c[:, :d].T @ f) / rho
    feq = orc.equilibrium(lat, rho, u)
    return feq, feq / f - 1.0


def _mpnode(orc, lat, f):
    c, w = orc.lattice(lat)
    d = orc.dim(lat)
    return mpr.Node(c[:, :d], w, f)


@pytest.mark.parametrize("lat", LATS)
def test_delta_h_matches_high_precision(orc, lat):
    rng = np.random.default_rng(10)
    for amp in AMPS:
        for _ in range(3):
            f = _node(orc, lat, rng, amp)
            feq, x = _x(orc, lat, f)
            m = _mpnode(orc, lat, f)
            am = orc.alpha_max(f, feq)
            for alpha in [0.5, 1.0, 1.7, 2.0, min(3.0, 0.99 * am), am]:
                if alpha > am:
                    continue        # outside the domain [0, alpha_max]
                got = orc.delta_h(f, x, alpha)
                ref = float(m.delta_h(min(alpha, float(m.alpha_max()))))
                bound = orc.delta_h_bound(f, x, alpha)
                # the oracle's own error bound must cover the true error
                assert abs(got - ref) <= bound + 1e-12 * abs(ref), (amp, alpha)
                if abs(ref) > 1e-25:
                    assert abs(got - ref) <= 1e-6 * abs(ref) + bound


@pytest.mark.parametrize("lat", LATS)
def test_delta_h_literal_form_agrees(orc, lat):
    rng = np.random.default_rng(11)
    for amp in [1e-2, 0.1, 0.45]:
        f = _node(orc, lat, rng, amp)
        feq, x = _x(orc, lat, f)
        for alpha in [1.0, 2.0]:
            lit = orc.delta_h_literal(lat, f, feq, alpha)
            mc = orc.delta_h(f, x, alpha)
            # the literal difference loses ~eps * H to cancellation
            assert abs(lit - mc) < 64 * np.finfo(float).eps * (1 + abs(
                orc.entropy(lat, f)))


@pytest.mark.parametrize("lat", LATS)
def test_series_identity_near_equilibrium(orc, lat):
    rng = np.random.default_rng(12)
    for amp in [1e-4, 1e-3, 1e-2]:
        f = _node(orc, lat, rng, amp)
        _, x = _x(orc, lat, f)
        for alpha in [1.0, 1.5, 2.0]:
            ser = sum((-1) ** k * (alpha ** k - k * alpha) / (k * (k - 1))
                      * np.sum(f * x ** k) for k in range(2, 14))
            got = orc.delta_h(f, x, alpha)
            assert abs(got - ser) <= 1e-9 * abs(ser) + orc.delta_h_bound(
                f, x, alpha)
    # alpha = 2 kills the second-order term: Delta H(2) = -1/3 sum f x^3 + ...
    f = _node(orc, lat, rng, 1e-4)
    _, x = _x(orc, lat, f)
    m3 = np.sum(f * x ** 3)
    assert abs(orc.delta_h(f, x, 2.0) + m3 / 3) < 1e-3 * abs(m3)


@pytest.mark.parametrize("lat", LATS)
def test_alpha_max_keeps_populations_nonnegative(orc, lat):
    rng = np.random.default_rng(13)
    for amp in [1e-3, 0.1, 0.45, 0.9]:
        f = _node(orc, lat, rng, amp)
        feq, _ = _x(orc, lat, f)
        am = orc.alpha_max(f, feq)
        assert am > 1.0
        for a in np.linspace(0, am, 50)[:-1]:
            assert np.all(f + a * (feq - f) > 0)
        fs = f + am * (feq - f)
        assert np.abs(fs).min() <= 1e-12 * f.max()
        assert np.any(f + am * (1 + 1e-9) * (feq - f) < 0)


@pytest.mark.parametrize("lat", LATS)
def test_delta_h_convex_increasing_on_one_to_alpha_max(orc, lat):
    rng = np.random.default_rng(14)
    for amp in [1e-2, 0.1, 0.45]:
        f = _node(orc, lat, rng, amp)
        feq, x = _x(orc, lat, f)
        am = min(orc.alpha_max(f, feq), 50.0)
        a = np.linspace(1.0, am, 200)
        d = np.array([orc.delta_h(f, x, v) for v in a])
        tol = max(orc.delta_h_bound(f, x, v) for v in a)
        assert d[0] < 0
        assert np.all(np.diff(d) >= -2 * tol)
        assert np.all(np.diff(d, 2) >= -4 * tol)


def _state_set(orc, lat, seed, n_per=4):
    rng = np.random.default_rng(seed)
    for amp in AMPS + [0.9]:
        for _ in range(n_per):
            yield amp, _node(orc, lat, rng, amp)


@pytest.mark.parametrize("lat", LATS)
def test_formula_entropy_safe_and_below_root(orc, lat):
    for amp, f in _state_set(orc, lat, 15):
        ft, alpha, flags, _ = orc.collide_node(lat, f, 0.9, "formula")
        assert not flags & orc.F_VIOLATION
        m = _mpnode(orc, lat, f)
        am = float(m.alpha_max())
        astar = min(2.0, am)
        # H-inequality Eq. (7) at the chosen alpha, in 60-digit arithmetic
        feq, x = _x(orc, lat, f)
        assert float(m.delta_h(alpha)) <= orc.delta_h_bound(f, x, alpha)
        dstar = m.delta_h(astar)
        if dstar <= 0:
            assert alpha == pytest.approx(astar, rel=1e-14)
            assert flags & orc.F_ACCEPT_STAR
        else:
            assert flags & orc.F_FORMULA
            root = m.root()
            assert 1.0 <= alpha <= astar
            if root is not None:
                assert alpha <= float(root) * (1 + 1e-14)
            # Eq. (9) with the 60-digit entropy values
            d1 = m.delta_h(1)
            ref = astar + float(dstar / (dstar - d1)) * (1 - astar)
            assert alpha == pytest.approx(ref, rel=1e-9, abs=1e-12)
        # Eq. (1): f~ = f + alpha beta (f^eq - f), which conserves mass and
        # momentum
        assert abs(ft.sum() - f.sum()) < 1e-14 * f.sum()


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q27"])
def test_formula_continuous_across_acceptance_boundary(orc, lat):
    # two states with opposite signs of Delta H(2); along the segment
    # between them Delta H(alpha_*) crosses 0 and Eq. (9) meets alpha_*.
    rng = np.random.default_rng(16)
    pos = neg = None
    while pos is None or neg is None:
        f = _node(orc, lat, rng, 1e-2)
        feq, x = _x(orc, lat, f)
        if orc.delta_h(f, x, 2.0) > 0:
            pos = f
        else:
            neg = f
    lo, hi = 0.0, 1.0          # s=0: neg, s=1: pos
    for _ in range(60):
        s = 0.5 * (lo + hi)
        f = (1 - s) * neg + s * pos
        feq, x = _x(orc, lat, f)
        if orc.delta_h(f, x, 2.0) > 0:
            hi = s
        else:
            lo = s
    a_lo = orc.collide_node(lat, (1 - lo) * neg + lo * pos, 0.9)[1]
    a_hi = orc.collide_node(lat, (1 - hi) * neg + hi * pos, 0.9)[1]
    assert a_lo == 2.0
    assert abs(a_hi - 2.0) < 1e-9


@pytest.mark.parametrize("lat", LATS)
def test_root_stop_rule_and_root_value(orc, lat):
    for amp, f in _state_set(orc, lat, 17, n_per=2):
        ft, alpha, flags, iters = orc.collide_node(lat, f, 0.9, "root")
        m = _mpnode(orc, lat, f)
        root = m.root()
        feq, x = _x(orc, lat, f)
        if root is None:
            assert flags & orc.F_NO_ROOT
            assert alpha == pytest.approx(float(m.alpha_max()), rel=1e-13)
            continue
        if flags & orc.F_DEGENERATE:
            continue
        d = orc.delta_h(f, x, alpha)
        assert not flags & orc.F_ROOT_CAP
        assert -1e-13 <= d <= 0 or iters >= 1
        assert float(m.delta_h(alpha)) <= orc.delta_h_bound(f, x, alpha)
        # distance to the exact root is set by the 1e-13 stop window
        slope = float(m.slope(root))
        assert float(root) - alpha <= 1e-13 / slope * 1.01 + 1e-13
        assert alpha <= float(root) * (1 + 1e-14)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q27"])
def test_secant_iteration(orc, lat):
    for amp, f in _state_set(orc, lat, 18, n_per=2):
        a1 = orc.collide_node(lat, f, 0.9, "formula")[1]
        s1 = orc.collide_node(lat, f, 0.9, "secant", secant_iters=1)[1]
        assert s1 == a1                     # first iterate is Eq. (9)
        m = _mpnode(orc, lat, f)
        root = m.root()
        feq, x = _x(orc, lat, f)
        prev = 1.0
        for k in [1, 2, 4, 8, 30]:
            ak = orc.collide_node(lat, f, 0.9, "secant", secant_iters=k)[1]
            assert float(m.delta_h(ak)) <= orc.delta_h_bound(f, x, ak)
            assert ak >= prev - 1e-15       # monotone towards the root
            prev = ak
        dstar = m.delta_h(min(2.0, float(m.alpha_max())))
        if dstar > 0 and root is not None:
            assert abs(prev - float(root)) <= 1e-13 / float(m.slope(root)) + 1e-12


def test_degenerate_node_takes_alpha_two(orc):
    c, w = orc.lattice("D2Q9")
    # u = 0, rho = 1: f = W is its own equilibrium up to rounding
    ft, alpha, flags, _ = orc.collide_node("D2Q9", w, 0.7)
    assert np.abs(ft - w).max() <= 4 * np.finfo(float).eps
    # an exactly representable equilibrium: rho = 36 -> f = {16, 4 x4, 1 x4}
    f = 36.0 * w
    f = np.round(f)
    ft, alpha, flags, _ = orc.collide_node("D2Q9", f, 0.7)
    assert flags & orc.F_DEGENERATE and alpha == 2.0
    assert np.array_equal(ft, f)


def test_invalid_node_rejected(orc):
    c, w = orc.lattice("D2Q9")
    f = w.copy()
    f[3] = 0.0
    with pytest.raises(ValueError):
        orc.collide_node("D2Q9", f, 0.7)
