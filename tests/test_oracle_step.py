"""Whole-lattice pins of the oracle's Eq. (1) step on periodic lattices.

  * mass and momentum are conserved (sum over the lattice) to 1e-13 relative;
  * the rest state and a uniform flow are fixed points (to rounding);
  * the mirror symmetries of the Taylor-Green vortex survive many steps
    (catches a wrong velocity table or streaming direction);
  * low-Re Taylor-Green kinetic energy decays as exp(-2 nu |k|^2 t) within
    0.5 % (the 64 x 64, nu = 0.01, u0 = 0.05, 1000-step case);
  * the discrete H-theorem Eq. (6): sum_x H is non-increasing, with zero
    per-node violations of Eq. (7);
  * push streaming Eq. (5b) moves each population by c_i exactly.
"""
import json
import math
import os

import numpy as np
import pytest

import elbm_workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_values.json")))


def test_streaming_moves_by_c(orc):
    # with beta -> 0 the collision is the identity: Eq. (1) is pure Eq. (5b)
    c, w = orc.lattice("D3Q27")
    L = orc.Lattice("D3Q27", 5, 4, 3, beta=0.0)
    rng = np.random.default_rng(0)
    f0 = 1.0 + 0.1 * rng.uniform(size=L.f.shape)
    L.set_populations(f0)
    L.step(1)
    for i in range(27):
        expect = np.roll(f0[i], shift=(c[i, 2], c[i, 1], c[i, 0]),
                         axis=(0, 1, 2))
        assert np.array_equal(L.f[i], expect)


@pytest.mark.parametrize("lat,shape", [("D2Q9", (1, 24, 20)),
                                       ("D3Q27", (6, 7, 8)),
                                       ("D1Q3", (1, 1, 30))])
def test_conservation(orc, lat, shape):
    nz, ny, nx = shape
    d = orc.dim(lat)
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, size=shape)
    u = 0.08 * rng.uniform(-1, 1, size=(d,) + shape)
    for mode in ["formula", "root"]:
        L = orc.Lattice(lat, nx, ny, nz, nu=1e-3)
        L.init_fields(rho, u)
        _, st = L.step(20, mode=mode, stats=True)
        m0, p0 = st[0]["mass"], np.array(st[0]["momentum"])
        r, uu = L.moments()
        m1 = r.sum()
        p1 = np.array([(r * uu[a]).sum() for a in range(d)])
        assert abs(m1 - m0) <= 1e-13 * m0
        assert np.abs(p1 - p0[:d]).max() <= 1e-13 * m0
        assert sum(s["n_violations"] for s in st) == 0


@pytest.mark.parametrize("lat,shape", [("D2Q9", (1, 8, 8)),
                                       ("D3Q27", (4, 4, 4))])
def test_rest_and_uniform_flow_fixed_points(orc, lat, shape):
    d = orc.dim(lat)
    for u0 in [np.zeros(d), np.array([0.05, -0.03, 0.02][:d])]:
        rho, u = W.uniform_flow(shape, u0)
        L = orc.Lattice(lat, shape[2], shape[1], shape[0], nu=0.01)
        L.init_fields(rho, u)
        f0 = L.f.copy()
        L.step(10)
        assert np.abs(L.f - f0).max() <= 32 * np.finfo(float).eps


def test_taylor_green_mirror_symmetry(orc):
    n = 32
    rho, u = W.taylor_green_2d(n, 0.05)
    L = orc.Lattice("D2Q9", n, n, 1, nu=0.005)
    L.init_fields(rho, u)
    L.step(200)
    r, uu = L.moments()
    r, ux, uy = r[0], uu[0, 0], uu[1, 0]
    mirror = (n // 2 - np.arange(n)) % n       # x -> N/2 - x
    assert np.abs(r - r[:, mirror]).max() < 1e-14
    assert np.abs(ux + ux[:, mirror]).max() < 1e-14
    assert np.abs(uy - uy[:, mirror]).max() < 1e-14
    assert np.abs(r - r[mirror, :]).max() < 1e-14     # y -> N/2 - y
    assert np.abs(ux - ux[mirror, :]).max() < 1e-14
    assert np.abs(uy + uy[mirror, :]).max() < 1e-14


def test_taylor_green_3d_mirror_symmetry(orc):
    n = 8
    rho, u = W.taylor_green_3d(n, 0.05)
    L = orc.Lattice("D3Q27", n, n, n, nu=0.01)
    L.init_fields(rho, u)
    L.step(20)
    r, uu = L.moments()
    m = (-np.arange(n)) % n
    # x -> -x mirror (u = u0 sin x cos y cos z): u -> -u, v, w unchanged
    assert np.abs(r - r[:, :, m]).max() < 1e-14
    assert np.abs(uu[0] + uu[0][:, :, m]).max() < 1e-14
    assert np.abs(uu[1] - uu[1][:, :, m]).max() < 1e-14
    # z -> -z mirror: w -> -w
    mz = (-np.arange(n)) % n
    assert np.abs(uu[2] + uu[2][mz]).max() < 1e-14
    assert np.abs(uu[0] - uu[0][mz]).max() < 1e-14


def test_taylor_green_energy_decay(orc):
    """The 64 x 64, nu = 0.01, u0 = 0.05 vortex for 1000 steps, FORMULA."""
    n, nu, steps = 64, 0.01, 1000
    rho, u = W.taylor_green_2d(n, 0.05)
    L = orc.Lattice("D2Q9", n, n, 1, nu=nu)
    L.init_fields(rho, u)
    _, st = L.step(steps, stats=True)
    r, uu = L.moments()
    e_end = 0.5 * np.sum(r * (uu ** 2).sum(0))
    k2 = 2 * (2 * math.pi / n) ** 2
    expect = math.exp(-2 * nu * k2 * steps)
    ratio = e_end / st[0]["kinetic_energy"]
    assert abs(ratio / expect - 1) < 5e-3
    assert sum(s["n_violations"] for s in st) == 0
    h = np.array([s["h_total"] for s in st])
    assert np.all(np.diff(h) <= 1e-12 * np.abs(h).max())


@pytest.mark.slow
def test_shear_layer_accept_two_proportion(orc):
    """Fig. 5: on the 128^2 double shear layer with nu = 1e-5, alpha = 2 is
    accepted at roughly half of the nodes through most of the run.  The figure's
    data is not printed, so the pin is a band: a median in [0.3, 0.7] over
    the first quarter of the run (t <= 0.25)."""
    g = GOLD["double_shear_layer"]
    n = g["M"]
    rho, u = W.shear_layer(n, g["U"], g["lambda"], g["perturbation"])
    L = orc.Lattice("D2Q9", n, n, 1, nu=g["nu"])
    L.init_fields(rho, u)
    _, st = L.step(g["T"], stats=True)
    prop = np.array([s["n_accept_two"] / s["n_nodes"] for s in st[100:]])
    target = GOLD["accept_two_proportion"]["value"]
    assert abs(np.median(prop) - target) < 0.1
    assert np.mean((prop > 0.3) & (prop < 0.7)) >= 0.8
    assert sum(s["n_violations"] for s in st) == 0
    h = np.array([s["h_total"] for s in st])
    assert np.all(np.diff(h) <= 1e-12 * np.abs(h).max())


@pytest.mark.parametrize("ends", ["zero_gradient", "periodic"])
def test_shock_tube_alpha_deviation(orc, ends):
    """1D shock tube of the paper's first experiment (Fig. 2): rho = 1.5 on
    [0, 400], 0.75 on (400, 800], u = 0, nu = 1e-5, t = 500; the largest
    deviation of the FORMULA alpha from 2 at the compressive shock front is
    printed as 3.96 %.  Readings (the paper gives neither): D1Q3, and either
    zero-gradient ends, realised by even reflection of the 801 nodes into a
    periodic lattice of 1602, or the 801 nodes wrapped periodically (a
    second step at the wrap); the deviation is taken over the collisions
    of the state at t = 500, at the nodes off equilibrium (the rest regions
    sit at f = f^eq to rounding).  The oscillating shock makes the value vary by
    ~0.5 % from step to step, so the pin is a band around the paper's
    number; both readings fall inside it."""
    g = GOLD["shock_tube"]
    rho, u = W.shock_tube(g["nodes"], g["rho_left"], g["rho_right"],
                          g["split"], ends=ends)
    n = rho.size
    L = orc.Lattice("D1Q3", n, 1, 1, nu=g["nu"])
    L.init_fields(rho, u)
    _, st = L.step(g["t"], stats=True)
    # nodes off equilibrium at t; where f = f^eq to rounding, f* = f for
    # every alpha and alpha only follows the sign of rounding noise
    c, _ = orc.lattice("D1Q3")
    fp = L.f.reshape(3, -1)[:, : g["nodes"] + 1]
    live = np.array([np.abs(orc.equilibrium(
        "D1Q3", fk.sum(), np.array([c[:, 0] @ fk / fk.sum()])) / fk - 1).max()
        > 1e-12 for fk in fp.T])
    maps, st1 = L.step(1, alpha_map=True, stats=True)
    st += st1
    a = np.where(live, maps[0].ravel()[: g["nodes"] + 1], 2.0)
    dev = (2.0 - a.min()) / 2.0
    assert a.max() <= 2.0 and maps[0].min() >= 1.0
    assert abs(dev - g["max_alpha_deviation_formula"]) < 0.005, dev
    # the minimum sits at the compressive front of the right-moving shock
    # (with periodic ends, where it meets the wave from the wrap)
    k = int(a.argmin())
    print("shock tube, %s ends: max alpha deviation %.5f at node %d"
          % (ends, dev, k))
    if ends == "periodic":
        # the periodic row is symmetric about x = 600.5: the front from the
        # step and the one from the wrap tie at nodes k and 1201 - k
        k = max(k, 1201 - k)
    assert 700 < k < 780
    assert sum(s["n_violations"] for s in st) == 0
