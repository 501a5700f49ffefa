"""GPU tests of the batched multi-lattice stepper (elbm_batch_*).

Every member of a batch runs the same per-node arithmetic as the
single-lattice FP32-shifted FORMULA path, so after the same number of steps
its populations must equal those of a lone lattice (1e-6 relative covers
any difference in FP32 rounding order; none is expected).
"""
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


MIX = [("D2Q9", (1, 23, 37), 1e-3, 1), ("D3Q27", (9, 10, 12), 2e-3, 2),
       ("D2Q9", (1, 64, 64), 1e-5, 3), ("D3Q27", (20, 20, 20), 1e-4, 4),
       ("D2Q9", (1, 50, 100), 5e-3, 5)]


def _fields(lat, shape, seed):
    nz, ny, nx = shape
    if lat == "D2Q9":
        return W.random_phase_2d(nx, seed=seed, umax=0.05, ny=ny)
    return W.random_phase_3d(nx, seed=seed, umax=0.05, ny=ny, nz=nz)


def _alone(elbm, lat, shape, nu, seed, steps):
    nz, ny, nx = shape
    g = elbm.Lattice(lat, nx, ny, nz, nu=nu, dtype="fp32_shifted")
    g.set_diagnostics(diag_every=1)
    rho, u = _fields(lat, shape, seed)
    g.init_fields(rho, u)
    g.step(steps, "formula")
    return g


def _assert_same(a, b):
    assert np.all(np.abs(a - b) <= 1e-6 * np.abs(b)), np.abs(a - b).max()


@pytest.mark.parametrize("graphs", [True, False])
def test_batch_members_match_single_lattices(elbm, graphs):
    b = elbm.Batch(burst=8, use_graphs=graphs, autotune=True)
    ids = []
    for lat, shape, nu, seed in MIX:
        rho, u = _fields(lat, shape, seed)
        ids.append(b.add(lat, shape[2], shape[1], shape[0], nu, rho, u))
    b.step(21)     # two full bursts + a partial one
    t = b.tuning()
    assert t["threads"] in (128, 256) and t["blocks_per_sm"] >= 1
    for mid, (lat, shape, nu, seed) in zip(ids, MIX):
        g = _alone(elbm, lat, shape, nu, seed, 21)
        _assert_same(b.populations(mid), g.populations())
        assert b.info(mid)[0] == 21
    b.close()


def test_remaining_steps_freeze_members(elbm):
    b = elbm.Batch(burst=8)
    ids = []
    for (lat, shape, nu, seed), k in zip(MIX, [3, 8, 13, 0, 21]):
        rho, u = _fields(lat, shape, seed)
        mid = b.add(lat, shape[2], shape[1], shape[0], nu, rho, u)
        b.set_steps(mid, k)
        ids.append((mid, k))
    b.step(40)
    for (mid, k), (lat, shape, nu, seed) in zip(ids, MIX):
        done, rem = b.info(mid)
        assert done == k and rem == 0
        g = _alone(elbm, lat, shape, nu, seed, k)
        _assert_same(b.populations(mid), g.populations())


def test_members_join_and_leave_between_bursts(elbm):
    b = elbm.Batch(burst=4)
    (la, sa, na, ea), (lb, sb, nb, eb), (lc, sc, nc, ec) = MIX[:3]
    a = b.add(la, sa[2], sa[1], sa[0], na, *_fields(la, sa, ea))
    bb = b.add(lb, sb[2], sb[1], sb[0], nb, *_fields(lb, sb, eb))
    b.step(8)
    b.remove(a)
    c = b.add(lc, sc[2], sc[1], sc[0], nc, *_fields(lc, sc, ec))
    b.step(12)
    _assert_same(b.populations(bb), _alone(elbm, lb, sb, nb, eb, 20).populations())
    _assert_same(b.populations(c), _alone(elbm, lc, sc, nc, ec, 12).populations())


def test_batch_statistics_match_single_lattice(elbm):
    b = elbm.Batch(burst=5, diag_every=1)
    ids = []
    for lat, shape, nu, seed in MIX[:4]:
        rho, u = _fields(lat, shape, seed)
        ids.append(b.add(lat, shape[2], shape[1], shape[0], nu, rho, u))
    b.step(10)
    for mid, (lat, shape, nu, seed) in zip(ids, MIX[:4]):
        g = _alone(elbm, lat, shape, nu, seed, 10)
        s, r = b.entropy_stats(mid), g.entropy_stats()
        assert s["step"] == r["step"] == 9
        assert s["n_nodes"] == r["n_nodes"]
        for k in ["n_accept_two", "n_formula", "n_band", "n_far"]:
            assert s[k] == r[k], k
        for k in ["mass", "kinetic_energy"]:
            assert abs(s[k] - r[k]) <= 1e-9 * abs(r[k]), k
        assert abs(s["alpha_min"] - r["alpha_min"]) < 1e-7
        assert abs(s["alpha_max"] - r["alpha_max"]) < 1e-7


def test_batch_alpha_map_and_moments(elbm):
    b = elbm.Batch(burst=4)
    lat, shape, nu, seed = MIX[3]
    mid = b.add(lat, shape[2], shape[1], shape[0], nu, *_fields(lat, shape, seed))
    b.record_alpha(mid)
    b.step(6)
    g = elbm.Lattice(lat, shape[2], shape[1], shape[0], nu=nu,
                     dtype="fp32_shifted")
    g.set_diagnostics(diag_every=1, alpha_map_every=1)
    g.init_fields(*_fields(lat, shape, seed))
    g.step(6)
    assert np.array_equal(b.alpha_map(mid), g.alpha_map())
    rb, ub = b.moments(mid)
    rg, ug = g.moments()
    assert np.allclose(rb, rg, rtol=1e-12, atol=0) and np.allclose(ub, ug,
                                                                   atol=1e-12)


def test_batch_rejects_bad_input(elbm):
    b = elbm.Batch(max_members=1)
    lat, shape, nu, seed = MIX[0]
    b.add(lat, shape[2], shape[1], shape[0], nu, *_fields(lat, shape, seed))
    with pytest.raises(elbm.ElbmError):
        b.add(lat, shape[2], shape[1], shape[0], nu, *_fields(lat, shape, seed))
    with pytest.raises(elbm.ElbmError):
        b.remove(7)
