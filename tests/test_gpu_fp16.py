"""GPU parity of the FP16-shifted storage path against the FP64 oracle.

Storage: the deviation delta_i = f_i - W_i rho0 scaled by 2^k_i,
k_i = round(log2(1 / W_i)), in IEEE binary16; arithmetic in FP32 as for the
FP32-shifted path (the certified entropy decision sees the values as
loaded).  Tolerances:

  * initial state: binary16 rounding of the FP64 equilibrium deviation,
    within one binary16 ulp of numpy's correctly rounded conversion of the
    oracle's f^eq - W_i rho0 (both round to nearest even from FP64; a
    one-ulp difference can only come from the two FP64 evaluations
    straddling a rounding boundary);
  * one step from the same stored state: every population within the
    FP32 path's bound (2e-6 |f|) plus one binary16 rounding of the
    post-collision deviation (unit roundoff 2^-11, subnormal spacing
    2^-24 scaled by 2^-k_i);
  * multi-step: kinetic-energy and enstrophy histories within 1 % of the
    FP64 oracle (the tolerance the FP32 path is held to on turbulent
    flows); the velocity L2 error is printed;
  * mass and momentum drift at most the sum of the per-step rounding
    bounds 2^-11 sum |delta_i| (conservation holds to storage rounding);
  * zero Eq. (7) violations in the FP64 check.
"""
import os

import numpy as np
import pytest

import elbm_workloads as W

pytestmark = pytest.mark.gpu

U16 = 2.0 ** -11          # binary16 unit roundoff
SUB16 = 2.0 ** -24        # binary16 subnormal spacing


@pytest.fixture(scope="module")
def elbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_00866_gb300 as e
    if not os.path.exists(e.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    e.lib()
    return e


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.lib()
    return oracle


def _scales(orc, lat):
    """(W_i, 2^k_i) as arrays shaped for broadcasting over (q, nz, ny, nx)."""
    _, w = orc.lattice(lat)
    s = 2.0 ** np.round(np.log2(1.0 / w))
    return w[:, None, None, None], s[:, None, None, None]


def _fields(lat, shape, seed):
    nz, ny, nx = shape
    if lat == "D2Q9":
        return W.random_phase_2d(nx, seed=seed, umax=0.06, ny=ny)
    return W.random_phase_3d(nx, seed=seed, umax=0.06, ny=ny, nz=nz)


SHAPES = [("D2Q9", (1, 64, 64), 1e-5), ("D2Q9", (1, 23, 37), 1e-3),
          ("D3Q27", (12, 16, 20), 1e-4), ("D3Q27", (5, 7, 9), 2e-3)]


@pytest.mark.parametrize("lat,shape,nu", SHAPES)
def test_fp16_initial_state_is_rounded_equilibrium(elbm, orc, lat, shape, nu):
    nz, ny, nx = shape
    rho, u = _fields(lat, shape, 5)
    g = elbm.Lattice(lat, nx, ny, nz, nu=nu, dtype="fp16_shifted")
    g.init_fields(rho, u)
    o = orc.Lattice(lat, nx, ny, nz, nu=nu)
    o.init_fields(rho, u)
    w, s = _scales(orc, lat)
    r0 = g.rho0
    stored = (g.populations() - w * r0) * s
    expect = ((o.f - w * r0) * s).astype(np.float16).astype(np.float64)
    ulp = np.spacing(np.abs(expect).astype(np.float16)).astype(np.float64)
    diff = np.abs(stored - expect)
    assert np.all(diff <= ulp), diff.max()
    assert np.mean(diff == 0) > 0.999
    assert np.all(stored.astype(np.float16).astype(np.float64) == stored)


@pytest.mark.parametrize("lat,shape,nu", SHAPES)
def test_fp16_single_step_within_rounding_of_oracle(elbm, orc, lat, shape, nu):
    """One FP16 FORMULA step from an evolved, stored state vs the FP64
    oracle from the same (decoded) state; per-node alpha as for FP32."""
    nz, ny, nx = shape
    if lat == "D2Q9" and shape == (1, 64, 64):
        rho, u = W.shear_layer(nx, ny=ny)
    else:
        rho, u = _fields(lat, shape, 11)
    o = orc.Lattice(lat, nx, ny, nz, nu=nu)
    o.init_fields(rho, u)
    o.step(60)
    g = elbm.Lattice(lat, nx, ny, nz, nu=nu, dtype="fp16_shifted")
    g.set_populations(o.f)
    g.set_diagnostics(diag_every=1, check_every=1, alpha_map_every=1)
    loaded = g.populations()
    o.set_populations(loaded)
    amaps, _ = o.step(1, alpha_map=True, stats=True)
    g.step(1, "formula")
    f = g.populations()
    w, s = _scales(orc, lat)
    dev = np.abs(o.f - w * g.rho0)
    tol = 2e-6 * np.abs(o.f) + U16 * (dev + 2e-6 * np.abs(o.f)) + SUB16 / s
    bad = np.abs(f - o.f) > tol
    assert not bad.any(), (np.abs(f - o.f) / tol).max()
    ag = g.alpha_map().astype(np.float64)
    assert np.all(ag <= amaps[0] + 1e-12)
    st = g.entropy_stats()
    assert st["n_violations"] == 0 and st["checked"] == 1


def _energy(rho, u):
    return 0.5 * float(np.sum(rho * np.sum(u * u, axis=0)))


def test_fp16_taylor_green_2d_energy_history(elbm, orc):
    n, nu = 64, 0.01
    rho, u = W.taylor_green_2d(n, 0.05)
    g = elbm.Lattice("D2Q9", n, n, 1, nu=nu, dtype="fp16_shifted")
    g.set_diagnostics(diag_every=0, check_every=0)
    g.init_fields(rho, u)
    o = orc.Lattice("D2Q9", n, n, 1, nu=nu)
    o.init_fields(rho, u)
    worst = 0.0
    for _ in range(10):
        g.step(100, "formula")
        o.step(100)
        eg = _energy(*g.moments())
        eo = _energy(*o.moments())
        worst = max(worst, abs(eg / eo - 1))
    _, ug = g.moments()
    _, uo = o.moments()
    err = np.linalg.norm(ug - uo) / np.linalg.norm(uo)
    print("FP16 TGV-64: energy history max rel dev %.3e, velocity L2 rel "
          "error after 1000 steps %.3e" % (worst, err))
    assert worst < 1e-2


def test_fp16_taylor_green_3d_energy_and_enstrophy(elbm, orc):
    n, nu = 24, 0.005
    rho, u = W.taylor_green_3d(n, 0.05)
    g = elbm.Lattice("D3Q27", n, n, n, nu=nu, dtype="fp16_shifted")
    g.set_diagnostics(diag_every=0)
    g.init_fields(rho, u)
    o = orc.Lattice("D3Q27", n, n, n, nu=nu)
    o.init_fields(rho, u)
    for _ in range(4):
        g.step(50, "formula")
        o.step(50)
        eg, eo = _energy(*g.moments()), _energy(*o.moments())
        assert abs(eg / eo - 1) < 1e-2
        assert abs(g.enstrophy() / o.enstrophy() - 1) < 1e-2
    _, ug = g.moments()
    _, uo = o.moments()
    print("FP16 TGV-24^3 velocity L2 rel error after 200 steps: %.3e"
          % (np.linalg.norm(ug - uo) / np.linalg.norm(uo)))


def test_fp16_random_phase_zero_violations(elbm):
    n = 32
    rho, u = W.random_phase_3d(n, seed=2, umax=0.05)
    g = elbm.Lattice("D3Q27", n, n, n, nu=1e-5, dtype="fp16_shifted")
    g.set_diagnostics(diag_every=1, check_every=1)
    g.init_fields(rho, u)
    for _ in range(40):
        g.step(1, "formula")
        s = g.entropy_stats()
        assert s["n_violations"] == 0, s
    assert s["n_accept_two"] > 0 and s["n_formula"] > 0


def test_fp16_conservation_within_rounding(elbm, orc):
    n, steps = 48, 200
    rho, u = W.random_phase_2d(n, seed=4, umax=0.05)
    g = elbm.Lattice("D2Q9", n, n, 1, nu=1e-3, dtype="fp16_shifted")
    g.init_fields(rho, u)
    w, _ = _scales(orc, "D2Q9")
    f0 = g.populations()
    # per-step bound on the mass (and each momentum component) change:
    # one rounding of every stored deviation; the deviations' size is
    # bounded by twice its initial value for this slowly decaying flow
    per_step = U16 * 2.0 * np.abs(f0 - w * g.rho0).sum()
    r0, u0 = g.moments()
    m0 = r0.sum()
    p0 = (r0 * u0).reshape(2, -1).sum(1)
    g.step(steps, "formula")
    r1, u1 = g.moments()
    p1 = (r1 * u1).reshape(2, -1).sum(1)
    print("FP16 mass drift %.3e, momentum drift %.3e, bound %.3e"
          % (abs(r1.sum() - m0), np.abs(p1 - p0).max(), steps * per_step))
    assert abs(r1.sum() - m0) <= steps * per_step
    assert np.abs(p1 - p0).max() <= steps * per_step


@pytest.mark.parametrize("mode", ["root", "secant"])
def test_fp16_iterative_modes(elbm, orc, mode):
    lat, shape, nu = "D3Q27", (6, 8, 10), 1e-4
    nz, ny, nx = shape
    rho, u = _fields(lat, shape, 8)
    o = orc.Lattice(lat, nx, ny, nz, nu=nu)
    o.init_fields(rho, u)
    o.step(30)
    g = elbm.Lattice(lat, nx, ny, nz, nu=nu, dtype="fp16_shifted")
    g.set_populations(o.f)
    g.set_diagnostics(diag_every=1, check_every=1)
    o.set_populations(g.populations())
    o.step(1, mode=mode, secant_iters=4)
    g.step(1, mode)
    f = g.populations()
    w, s = _scales(orc, lat)
    dev = np.abs(o.f - w * g.rho0)
    # FP64 arithmetic with alpha rounded down to FP32 (as for FP32
    # storage): 2^-23 alpha |f^eq - f| < 2e-6 |f|
    tol = 2e-6 * np.abs(o.f) + U16 * (dev + 2e-6 * np.abs(o.f)) + SUB16 / s
    assert np.all(np.abs(f - o.f) <= tol), (np.abs(f - o.f) / tol).max()
    st = g.entropy_stats()
    assert st["n_violations"] == 0 and st["n_root_cap"] == 0
