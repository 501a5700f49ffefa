"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances:
  * FP64 storage, FORMULA: every population within 1e-12 relative (the two
    evaluate the same Eqs. (1)-(9) in FP64; differences are rounding order,
    FMA contraction and 1-ulp log differences);
  * FP64 ROOT / SECANT: iterative branch sequences can differ where Delta H
    is within rounding of a stop-rule edge, so fields agree to 1e-9 and the
    single-step check is that every GPU alpha (recovered from the FP64
    populations) satisfies the oracle's stop rule / H-inequality;
  * FP32 storage: velocity L2-relative 1e-5 against the FP64 oracle on
    laminar flows; per-node alpha never above the FP64 FORMULA alpha of the
    same stored state and within 1e-4 of it where the state is resolved
    (the certified decision rounds towards entropy safety);
  * zero Eq. (7) violations in the FP64 check of every path.
"""
import math
import os

import numpy as np
import pytest

import elbm_workloads as W

pytestmark = pytest.mark.gpu


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


def _pair(elbm, orc, lat, shape, nu, dtype, rho, u):
    nz, ny, nx = shape
    g = elbm.Lattice(lat, nx, ny, nz, nu=nu, dtype=dtype)
    g.init_fields(rho, u)
    o = orc.Lattice(lat, nx, ny, nz, nu=nu)
    o.init_fields(rho, u)
    return g, o


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_fp64_taylor_green_64_1000_steps(elbm, orc):
    """D2Q9 64 x 64 Taylor-Green, nu = 0.01, u0 = 0.05, FP64, FORMULA."""
    rho, u = W.taylor_green_2d(64, 0.05)
    g, o = _pair(elbm, orc, "D2Q9", (1, 64, 64), 0.01, "fp64", rho, u)
    g.set_diagnostics(diag_every=1, check_every=250)
    g.step(1000, "formula")
    _, st = o.step(1000, stats=True)
    f = g.populations()
    assert np.all(np.abs(f - o.f) <= 1e-12 * np.abs(o.f))
    s = g.entropy_stats()
    assert s["step"] == 999 and s["checked"] == 0
    ref = st[-1]
    assert abs(s["kinetic_energy"] / ref["kinetic_energy"] - 1) < 1e-11
    assert abs(s["mass"] - ref["mass"]) < 1e-12 * ref["mass"]
    assert abs(s["n_accept_two"] - ref["n_accept_two"]) <= 2
    k2 = 2 * (2 * math.pi / 64) ** 2
    r, uu = g.moments()
    e_end = 0.5 * np.sum(r * (uu ** 2).sum(0))
    assert abs(e_end / st[0]["kinetic_energy"] / math.exp(-2 * 0.01 * k2 * 1000)
               - 1) < 5e-3


@pytest.mark.parametrize("lat,shape", [("D2Q9", (1, 23, 37)),
                                       ("D3Q27", (11, 13, 19))])
def test_fp64_ragged_formula_parity(elbm, orc, lat, shape):
    nz, ny, nx = shape
    if lat == "D2Q9":
        rho, u = W.random_phase_2d(nx, seed=3, umax=0.1, ny=ny)
    else:
        rho, u = W.random_phase_3d(nx, seed=3, umax=0.1, ny=ny, nz=nz)
    g, o = _pair(elbm, orc, lat, shape, 2e-4, "fp64", rho, u)
    g.set_diagnostics(diag_every=1, check_every=1, alpha_map_every=1)
    for _ in range(3):
        g.step(10, "formula")
        amaps, _ = o.step(10, "formula", alpha_map=True)
        f = g.populations()
        assert np.all(np.abs(f - o.f) <= 1e-12 * np.abs(o.f)), _rel(f, o.f)
        assert np.abs(g.alpha_map() - amaps[-1]).max() < 2e-6   # FP32 map
    s = g.entropy_stats()
    assert s["checked"] == 1 and s["n_violations"] == 0


def _alpha_from_step(orc, lat, f_pre, f_post, beta):
    """alpha of every node recovered from an FP64 step: the post-collision
    f~_i(x) = f_post_i(x + c_i) = f_i + alpha beta (f^eq_i - f_i)."""
    c, w = orc.lattice(lat)
    d = orc.dim(lat)
    q = len(w)
    ft = np.stack([np.roll(f_post[i], shift=(-c[i, 2], -c[i, 1], -c[i, 0]),
                           axis=(0, 1, 2)) for i in range(q)])
    fp = f_pre.reshape(q, -1)
    ft = ft.reshape(q, -1)
    rho = fp.sum(0)
    alphas, xs = [], []
    for k in range(fp.shape[1]):
        feq = orc.equilibrium(lat, rho[k], (c[:, :d].T @ fp[:, k]) / rho[k])
        nk = feq - fp[:, k]
        alphas.append(float(np.dot(ft[:, k] - fp[:, k], nk) / (beta * np.dot(nk, nk))))
        xs.append(feq / fp[:, k] - 1)
    return np.array(alphas), xs


@pytest.mark.parametrize("lat,shape", [("D2Q9", (1, 20, 24)),
                                       ("D3Q27", (6, 7, 9))])
@pytest.mark.parametrize("mode", ["root", "secant"])
def test_fp64_iterative_modes_parity(elbm, orc, lat, shape, mode):
    """ROOT / SECANT: iterative branches can differ where Delta H is within
    rounding of a stop-rule edge, so fields agree to 1e-9 and every GPU alpha
    satisfies the stop rule (ROOT) or the H-inequality (SECANT) when
    re-evaluated by the oracle."""
    nz, ny, nx = shape
    if lat == "D2Q9":
        rho, u = W.random_phase_2d(nx, seed=5, umax=0.1, ny=ny)
    else:
        rho, u = W.random_phase_3d(nx, seed=5, umax=0.1, ny=ny, nz=nz)
    g, o = _pair(elbm, orc, lat, shape, 1e-4, "fp64", rho, u)
    g.set_diagnostics(diag_every=1, check_every=1)
    g.step(20, mode)
    o.step(20, mode, secant_iters=4)
    assert _rel(g.populations(), o.f) < 1e-9
    f_pre = g.populations()
    g.step(1, mode)
    alphas, xs = _alpha_from_step(orc, lat, f_pre, g.populations(), g.beta)
    fp = f_pre.reshape(len(f_pre), -1)
    for k in range(len(alphas)):
        if np.abs(xs[k]).max() < 1e-6:
            continue                    # alpha not recoverable at equilibrium
        fn, x, a = fp[:, k], xs[k], alphas[k]
        dh = orc.delta_h(fn, x, a)
        slope = abs(np.sum(fn * x * (np.log1p(a * x) - np.log1p(x))))
        tol = orc.delta_h_bound(fn, x, a) + slope * 1e-12 * a
        assert dh <= tol, (k, dh, tol)
        if mode == "root":
            feq = fn * (1 + x)
            assert dh >= -1e-13 - tol or orc.alpha_max(fn, feq) < 2.1
    s = g.entropy_stats()
    assert s["n_violations"] == 0 and s["n_root_cap"] == 0


@pytest.mark.parametrize("dtype,tol", [("fp32_shifted", 1e-5),
                                       ("fp32", 2e-4)])
def test_fp32_taylor_green_2d_vs_fp64_oracle(elbm, orc, dtype, tol):
    rho, u = W.taylor_green_2d(64, 0.05)
    g, o = _pair(elbm, orc, "D2Q9", (1, 64, 64), 0.01, dtype, rho, u)
    g.set_diagnostics(diag_every=1, check_every=100)
    g.step(1000, "formula")
    o.step(1000)
    _, ug = g.moments()
    _, uo = o.moments()
    err = np.linalg.norm(ug - uo) / np.linalg.norm(uo)
    print("FP32 %s TGV-64 velocity L2 rel error after 1000 steps: %.3e"
          % (dtype, err))
    assert err < tol
    g.set_diagnostics(diag_every=1, check_every=1)
    g.step(1, "formula")
    s = g.entropy_stats()
    assert s["n_violations"] == 0 and s["checked"] == 1


def test_fp32_taylor_green_3d_vs_fp64_oracle(elbm, orc):
    n = 24
    rho, u = W.taylor_green_3d(n, 0.05)
    g, o = _pair(elbm, orc, "D3Q27", (n, n, n), 0.005, "fp32_shifted", rho, u)
    g.set_diagnostics(diag_every=1, check_every=50)
    g.step(200, "formula")
    o.step(200)
    _, ug = g.moments()
    _, uo = o.moments()
    assert np.linalg.norm(ug - uo) / np.linalg.norm(uo) < 1e-5
    g.set_diagnostics(diag_every=1, check_every=1)
    g.step(1, "formula")
    s = g.entropy_stats()
    assert s["n_violations"] == 0 and s["checked"] == 1


@pytest.mark.parametrize("decision", ["exact", "certified"])
@pytest.mark.parametrize("lat,shape,nu", [("D2Q9", (1, 64, 64), 1e-5),
                                          ("D3Q27", (12, 16, 20), 1e-4)])
def test_fp32_single_step_alpha_against_fp64(elbm, orc, lat, shape, nu,
                                             decision):
    """One FP32 FORMULA step from an evolved state: per-node alpha vs the
    FP64 FORMULA alpha of the same stored state, and populations.  The
    exact decision takes the FP64 branch (acceptance of alpha = 2 or the
    Eq. (9) chord) at every node; the certified one never exceeds the FP64
    alpha."""
    nz, ny, nx = shape
    if lat == "D2Q9":
        rho, u = W.shear_layer(nx, ny=ny)
    else:
        rho, u = W.random_phase_3d(nx, seed=11, umax=0.08, ny=ny, nz=nz)
    o = orc.Lattice(lat, nx, ny, nz, nu=nu)
    o.init_fields(rho, u)
    o.step(60)
    g = elbm.Lattice(lat, nx, ny, nz, nu=nu, dtype="fp32_shifted")
    g.set_decision(decision)
    g.set_populations(o.f)
    g.set_diagnostics(diag_every=1, check_every=1, alpha_map_every=1)
    loaded = g.populations()          # the state as the GPU stores it
    o.set_populations(loaded)
    amaps, st = o.step(1, alpha_map=True, stats=True)
    g.step(1, "formula")
    ag = g.alpha_map().astype(np.float64)
    ao = amaps[0]
    s = g.entropy_stats()
    assert s["n_violations"] == 0 and s["checked"] == 1
    if decision == "exact":
        # the same branch as the FP64 decision at every node, alpha within
        # the FP32 evaluation of the chord (the accepted 2 exactly)
        assert s["n_decision_mismatch"] == 0
        assert np.all((ao == 2.0) == (ag == 2.0))
        assert np.abs(ag - ao).max() < 2e-5
        f = g.populations()
        assert np.all(np.abs(f - o.f) <= 2e-6 * np.abs(o.f))
        return
    assert np.all(ag <= ao + 1e-12)
    # nodes whose non-equilibrium part is resolved in FP32 (rms x > 1e-5)
    # follow the FP64 alpha to 1e-4; nodes within FP32 noise of equilibrium
    # may take the certified alpha = 1
    lf = loaded.reshape(len(loaded), -1)
    c, w = orc.lattice(lat)
    d = orc.dim(lat)
    rho_ = lf.sum(0)
    rms = np.empty(lf.shape[1])
    for k in range(lf.shape[1]):
        feq = orc.equilibrium(lat, rho_[k], (c[:, :d].T @ lf[:, k]) / rho_[k])
        rms[k] = np.sqrt(np.mean((feq / lf[:, k] - 1) ** 2))
    resolved = rms.reshape(ag.shape) > 1e-5
    close = (ao - ag) <= 1e-4
    assert close[resolved].mean() >= 0.999, close[resolved].mean()
    assert np.all((ag[~resolved] == 1.0) | close[~resolved])
    assert s["n_decision_mismatch"] <= s["n_band"]
    f = g.populations()
    assert np.all(np.abs(f - o.f) <= 2e-6 * np.abs(o.f))


@pytest.mark.parametrize("dtype", ["fp32_shifted", "fp16_shifted"])
@pytest.mark.parametrize("init", ["noise", "rough"])
@pytest.mark.parametrize("lat,shape", [("D2Q9", (1, 40, 36)),
                                       ("D3Q27", (8, 10, 12))])
def test_fp64_fixup_of_far_nodes_vs_oracle(elbm, orc, lat, shape, init,
                                           dtype):
    """Nodes far from equilibrium leave the FP32 kernels for the FP64
    fixup, which collides each node with a whole warp (one population per
    lane): populations multiplied by 1 + 0.3 U(-1, 1) ("noise"), or a flow
    rough at the grid scale with velocities up to 0.3 after a step
    ("rough": the components above 1/4 are the FP32 paths' velocity limit).
    One step without the FP64 check (the check's steps take the per-thread
    path) against the oracle's step of the same stored state: the FP64
    FORMULA's branch at every node, alpha within 2e-5 (the FP64 nodes' alpha
    rounded down to FP32; the FP32 nodes' Eq. (9) chord within its 2^-16
    certified width), populations within the FP32 arithmetic in units of
    W_i rho0 (2e-6 max(|f_i|, W_i rho0): at velocities near 1/4 some f_i
    lie far below W_i rho0, and FP32 forms f^eq_i - f_i to a fixed fraction
    of W_i rho) plus, for binary16 storage, 2^-10 of the stored deviation
    f - W rho0."""
    nz, ny, nx = shape
    um, km = (0.05, 4) if init == "noise" else (0.3, 8 if lat == "D2Q9" else 4)
    if lat == "D2Q9":
        rho, u = W.random_phase_2d(nx, 5, umax=um, ny=ny, kmax=km)
    else:
        rho, u = W.random_phase_3d(nx, 5, umax=um, ny=ny, nz=nz, kmax=km)
    nu = 2e-4
    g = elbm.Lattice(lat, nx, ny, nz, nu=nu, dtype=dtype)
    g.init_fields(rho, u)
    if init == "noise":
        f = g.populations()
        rng = np.random.default_rng(8)
        g.set_populations(f * (1.0 + 0.3 * rng.uniform(-1.0, 1.0, f.shape)))
    else:
        g.step(1, "formula")
    loaded = g.populations()
    g.set_diagnostics(diag_every=1, alpha_map_every=1)
    o = orc.Lattice(lat, nx, ny, nz, nu=nu)
    o.set_populations(loaded)
    amaps, _ = o.step(1, alpha_map=True, stats=True)
    g.step(1, "formula")
    s = g.entropy_stats()
    assert s["n_far"] > (0.2 * s["n_nodes"] if init == "noise" else 0), \
        s["n_far"]
    ag = g.alpha_map().astype(np.float64)
    ao = amaps[0]
    assert np.all((ao == 2.0) == (ag == 2.0))
    assert np.abs(ag - ao).max() < 2e-5
    fg = g.populations()
    _, w = orc.lattice(lat)
    wr = w.reshape((-1,) + (1,) * 3) * g.rho0
    tol = 2e-6 * np.maximum(np.abs(o.f), wr)
    if dtype == "fp16_shifted":
        tol += 2.0 ** -10 * np.abs(o.f - wr)
    assert np.all(np.abs(fg - o.f) <= tol), np.max(np.abs(fg - o.f) / tol)


@pytest.mark.parametrize("dtype", ["fp32_shifted", "fp16_shifted"])
def test_fixup_bulk_path_matches_per_lane_path(elbm, dtype):
    """The first step after initialisation leaves most nodes undecided in
    FP32 (n is rounding noise), so the fixup's queue is longer than its
    grid: each warp collects its FP64 nodes and runs them 32 at a time, one
    per lane (the last few of a warp, one per warp).  The same step with
    the FP64 check runs every FP64 node on its own lane directly.  The
    per-node arithmetic is the same except for the order of the sums in
    the one-per-warp remainder, so populations agree to the FP32 rounding
    of the relaxation and alpha maps to one FP32 rounding (2^-22
    relative).  The checked step also takes the FP64 branch at every
    non-degenerate node."""
    n = 96
    rho, u = W.taylor_green_3d(n, 0.05)
    res = []
    for check in (1, 0):
        g = elbm.Lattice("D3Q27", n, n, n, nu=1e-3, dtype=dtype)
        g.init_fields(rho, u)
        g.set_diagnostics(diag_every=check, check_every=check,
                          alpha_map_every=1)
        g.step(1, "formula")
        if check:
            s = g.entropy_stats()
            assert s["n_violations"] == 0
            assert s["n_decision_mismatch"] == 0
            # a fixup queue longer than its grid (304 x 256 threads)
            assert s["n_band"] + s["n_far"] > 77824
        res.append((g.populations(), g.alpha_map().astype(np.float64)))
        g.close()
    (f0, a0), (f1, a1) = res
    assert np.all(np.abs(f0 - f1) <= 2e-7 * np.abs(f0))
    assert np.all(np.abs(a0 - a1) <= 2.0 ** -22 * a0)


def test_pinned_host_buffers_match_pageable(elbm):
    """elbm_init_fields and elbm_moments read and write page-locked host
    buffers directly from their kernels (no device staging); pageable
    buffers go through a staging copy.  Both routes give the same
    populations and the same moments, bit for bit."""
    torch = pytest.importorskip("torch")
    import ctypes
    n = 24
    rho, u = W.taylor_green_3d(n, 0.05)
    rho_p = torch.empty(rho.shape, dtype=torch.float64, pin_memory=True)
    u_p = torch.empty(u.shape, dtype=torch.float64, pin_memory=True)
    rho_p.numpy()[...] = rho
    u_p.numpy()[...] = u
    out = []
    for pinned in (False, True):
        g = elbm.Lattice("D3Q27", n, n, n, nu=1e-3, dtype="fp32_shifted")
        if pinned:
            g.init_fields(rho_p.numpy(), u_p.numpy())
        else:
            g.init_fields(rho.copy(), u.copy())
        g.step(3, "formula")
        f = g.populations()
        if pinned:
            r_o = torch.empty(rho.shape, dtype=torch.float64, pin_memory=True)
            u_o = torch.empty(u.shape, dtype=torch.float64, pin_memory=True)
            assert elbm.lib().elbm_moments(
                g._h, ctypes.cast(r_o.data_ptr(), elbm._DP),
                ctypes.cast(u_o.data_ptr(), elbm._DP)) == 0
            m = (r_o.numpy().copy(), u_o.numpy().copy())
        else:
            m = g.moments()
        out.append((f, m))
        g.close()
    (f0, m0), (f1, m1) = out
    assert np.array_equal(f0, f1)
    assert np.array_equal(m0[0], m1[0]) and np.array_equal(m0[1], m1[1])


def test_fp32_random_phase_zero_violations(elbm):
    n = 32
    rho, u = W.random_phase_3d(n, seed=2, umax=0.05)
    g = elbm.Lattice("D3Q27", n, n, n, nu=1e-5, dtype="fp32_shifted")
    g.set_diagnostics(diag_every=1, check_every=1)
    g.init_fields(rho, u)
    for _ in range(40):
        g.step(1, "formula")
        s = g.entropy_stats()
        assert s["n_violations"] == 0, s
    assert s["n_accept_two"] > 0 and s["n_formula"] > 0


def test_conservation_on_gpu(elbm):
    rho, u = W.random_phase_2d(48, seed=4, umax=0.05)
    for dtype, tol in [("fp64", 1e-13), ("fp32_shifted", 1e-6)]:
        g = elbm.Lattice("D2Q9", 48, 48, 1, nu=1e-3, dtype=dtype)
        g.init_fields(rho, u)
        r0, u0 = g.moments()
        m0 = r0.sum()
        p0 = (r0 * u0).reshape(2, -1).sum(1)
        g.step(200, "formula")
        r1, u1 = g.moments()
        assert abs(r1.sum() - m0) <= tol * m0
        p1 = (r1 * u1).reshape(2, -1).sum(1)
        assert np.abs(p1 - p0).max() <= tol * m0


@pytest.mark.parametrize("lat,shape", [("D2Q9", (1, 1, 1)), ("D2Q9", (1, 1, 5)),
                                       ("D2Q9", (1, 7, 1)), ("D2Q9", (1, 3, 65)),
                                       ("D3Q27", (1, 1, 1)), ("D3Q27", (1, 4, 33)),
                                       ("D3Q27", (5, 1, 3)), ("D3Q27", (2, 3, 1))])
def test_edge_sizes(elbm, orc, lat, shape):
    nz, ny, nx = shape
    d = orc.dim(lat)
    rng = np.random.default_rng(sum(shape))
    rho = 1.0 + 0.02 * rng.uniform(-1, 1, size=shape)
    u = 0.05 * rng.uniform(-1, 1, size=(d,) + shape)
    for mode in ["formula", "root"]:
        g, o = _pair(elbm, orc, lat, shape, 1e-3, "fp64", rho, u)
        g.step(7, mode)
        o.step(7, mode)
        assert _rel(g.populations(), o.f) < (1e-12 if mode == "formula" else 1e-9)


def test_invalid_inputs_are_rejected(elbm):
    g = elbm.Lattice("D2Q9", 8, 8, 1, nu=0.01, dtype="fp32_shifted")
    rho = np.ones((1, 8, 8))
    u = np.zeros((2, 1, 8, 8))
    u[0, 0, 0, 0] = 1.0
    with pytest.raises(elbm.ElbmError) as e:
        g.init_fields(rho, u)
    assert e.value.status == 1
    with pytest.raises(elbm.ElbmError):
        g.alpha_map()            # nothing written yet
    f = np.full((9, 1, 8, 8), 0.1)
    f[3, 0, 2, 2] = 0.0
    with pytest.raises(elbm.ElbmError):
        g.set_populations(f)
    with pytest.raises(elbm.ElbmError):
        g.step(1, 9)


def test_device_resident_init_matches_host_init(elbm):
    import torch
    rho, u = W.taylor_green_3d(16, 0.05)
    a = elbm.Lattice("D3Q27", 16, 16, 16, nu=0.01, dtype="fp32_shifted")
    a.init_fields(rho, u)
    b = elbm.Lattice("D3Q27", 16, 16, 16, nu=0.01, dtype="fp32_shifted")
    b.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    a.step(5)
    b.step(5)
    assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("lat,shape,dtype,tol", [
    ("D2Q9", (1, 40, 48), "fp64", 1e-12),
    ("D3Q27", (12, 16, 20), "fp64", 1e-12),
    ("D3Q27", (16, 16, 16), "fp32_shifted", 1e-5)])
def test_enstrophy_matches_oracle(elbm, orc, lat, shape, dtype, tol):
    nz, ny, nx = shape
    if lat == "D2Q9":
        rho, u = W.taylor_green_2d(nx, 0.05, ny=ny)
    else:
        rho, u = W.taylor_green_3d(nx, 0.05, ny=ny, nz=nz)
    g, o = _pair(elbm, orc, lat, shape, 2e-3, dtype, rho, u)
    g.step(15)
    o.step(15)
    eg, eo = g.enstrophy(), o.enstrophy()
    assert eo > 0
    assert abs(eg / eo - 1) < tol
