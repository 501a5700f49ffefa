"""The batched stepper and the serving loop against the CPU FP64 oracle.

The batched kernel has its own tile -> member lookup, descriptor staging and
deferred-node fixup, so its members are held to the oracle directly (not
only to the single-lattice CUDA path), at the FP32 tolerances:
  * one Eq. (1) step from the same stored state: every population within
    2e-6 |f| of the oracle's step (FP32 relaxation of the FP32-decided
    alpha, the bound the single-lattice FP32 tests use);
  * zero Eq. (7) violations: at every node the alpha the batch used keeps
    H(f*(alpha)) - H(f), evaluated by the oracle on the pre-collision state,
    within the oracle's rounding bound;
  * multi-step laminar runs (random-phase flows of the modes |k| <= 2,
    resolved by at least 12 nodes per axis, max |u| = 0.05): velocity
    within L2-relative 1e-5 of the oracle, for members that step from the
    start and for a member that joins while the others are between bursts
    (modes at the grid scale are not the laminar case this tolerance is
    stated for: a 9 x 10 x 12 lattice carrying |k| = 4 reaches 1.4e-5 after
    40 steps on the single-lattice FP32 path as well);
with CUDA graphs on and off.  Served requests (continuous batching, members
joining a running batch) are held to the oracle run of the same request.
"""
import os

import numpy as np
import pytest

import elbm_workloads as W

pytestmark = pytest.mark.gpu

VEL_TOL = 1e-5
POP_TOL = 2e-6

# one-step members: small and ragged, grid-scale modes (|k| <= 4)
MEMBERS = [("D2Q9", (1, 23, 37), 1e-3, 31), ("D3Q27", (9, 10, 12), 2e-3, 32)]
# multi-step laminar members (|k| <= 2 on >= 12 nodes per axis)
LAMINAR = [("D2Q9", (1, 24, 36), 1e-3, 31), ("D3Q27", (12, 14, 16), 2e-3, 32)]
LATE = ("D3Q27", (13, 12, 15), 5e-3, 33)


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


def _fields(lat, shape, seed, kmax=4):
    nz, ny, nx = shape
    if lat == "D2Q9":
        return W.random_phase_2d(nx, seed=seed, umax=0.05, ny=ny, kmax=kmax)
    return W.random_phase_3d(nx, seed=seed, umax=0.05, ny=ny, nz=nz,
                             kmax=kmax)


def _add(b, lat, shape, nu, seed, kmax=4):
    nz, ny, nx = shape
    return b.add(lat, nx, ny, nz, nu, *_fields(lat, shape, seed, kmax))


def _vel_err(ug, uo):
    return np.linalg.norm(ug - uo) / np.linalg.norm(uo)


def _eq7_violations(orc, lat, f_pre, alpha):
    """Nodes where Delta H(alpha) of the pre-collision state exceeds the
    oracle's rounding bound."""
    c, w = orc.lattice(lat)
    d = orc.dim(lat)
    fp = f_pre.reshape(len(w), -1)
    a = alpha.reshape(-1).astype(np.float64)
    bad = []
    for k in range(fp.shape[1]):
        f = fp[:, k]
        rho = f.sum()
        feq = orc.equilibrium(lat, rho, (c[:, :d].T @ f) / rho)
        x = feq / f - 1
        if orc.delta_h(f, x, a[k]) > orc.delta_h_bound(f, x, a[k]):
            bad.append(k)
    return bad


@pytest.mark.parametrize("graphs", [True, False])
def test_batch_one_step_vs_oracle(elbm, orc, graphs):
    b = elbm.Batch(burst=4, use_graphs=graphs, autotune=False)
    ids = [_add(b, *m) for m in MEMBERS]
    for mid in ids:
        b.record_alpha(mid)
    b.step(3)                       # leave equilibrium first
    f_pre = {mid: b.populations(mid) for mid in ids}
    b.step(1)
    for mid, (lat, shape, nu, _) in zip(ids, MEMBERS):
        nz, ny, nx = shape
        o = orc.Lattice(lat, nx, ny, nz, nu=nu)
        o.set_populations(f_pre[mid])
        o.step(1)
        f = b.populations(mid)
        err = np.abs(f - o.f) / np.abs(o.f)
        assert err.max() <= POP_TOL, (lat, err.max())
        assert _eq7_violations(orc, lat, f_pre[mid], b.alpha_map(mid)) == []
    b.close()


def test_batch_far_nodes_vs_oracle(elbm, orc):
    """Members whose flow is rough at the grid scale (modes |k| <= 8 at
    max |u| = 0.3) leave nodes far from equilibrium after a step; the
    batch fixup collides them in FP64, one node per warp.  One step from
    the same stored state against the oracle: populations within
    2e-6 max(|f_i|, W_i rho0) (at velocities near 1/4 some f_i lie far below
    W_i rho0, and FP32 forms f^eq_i - f_i to a fixed fraction of W_i rho),
    the FP64 FORMULA's branch at every node, alpha within 2e-5."""
    b = elbm.Batch(burst=1, use_graphs=False, autotune=False, diag_every=1)
    specs = [("D2Q9", (1, 30, 26), 2e-3, 51), ("D3Q27", (10, 9, 12), 2e-3, 52)]
    ids = []
    for lat, (nz, ny, nx), nu, seed in specs:
        if lat == "D2Q9":
            rho, u = W.random_phase_2d(nx, seed, umax=0.3, ny=ny, kmax=8)
        else:
            rho, u = W.random_phase_3d(nx, seed, umax=0.3, ny=ny, nz=nz,
                                       kmax=4)
        ids.append(b.add(lat, nx, ny, nz, nu, rho, u))
    for mid in ids:
        b.record_alpha(mid)
    b.step(1)
    f_pre = {mid: b.populations(mid) for mid in ids}
    b.step(1)
    for mid, (lat, (nz, ny, nx), nu, _) in zip(ids, specs):
        s = b.entropy_stats(mid)
        assert s["n_far"] > 0, (lat, s["n_far"])
        o = orc.Lattice(lat, nx, ny, nz, nu=nu)
        o.set_populations(f_pre[mid])
        amaps, _ = o.step(1, alpha_map=True, stats=True)
        f = b.populations(mid)
        _, w = orc.lattice(lat)
        wr = w.reshape((-1,) + (1,) * 3)
        err = np.abs(f - o.f) / np.maximum(np.abs(o.f), wr)
        assert err.max() <= POP_TOL, (lat, err.max())
        ag = b.alpha_map(mid).astype(np.float64)
        assert np.all((amaps[0] == 2.0) == (ag == 2.0))
        assert np.abs(ag - amaps[0]).max() < 2e-5
    b.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_batch_members_and_late_joiner_track_oracle(elbm, orc, graphs):
    b = elbm.Batch(burst=8, use_graphs=graphs, autotune=True)
    ids = [_add(b, *m, kmax=2) for m in LAMINAR]
    b.step(13)                      # one full burst and a partial one
    late = _add(b, *LATE, kmax=2)   # joins while the others are at step 13
    b.step(27)                      # three full bursts and a partial one
    runs = list(zip(ids, LAMINAR, [40, 40])) + [(late, LATE, 27)]
    for mid, (lat, shape, nu, seed), steps in runs:
        assert b.info(mid)[0] == steps
        nz, ny, nx = shape
        o = orc.Lattice(lat, nx, ny, nz, nu=nu)
        o.init_fields(*_fields(lat, shape, seed, kmax=2))
        o.step(steps)
        rg, ug = b.moments(mid)
        ro, uo = o.moments()
        e = _vel_err(ug, uo)
        print("batch %s %s after %d steps: velocity L2 rel %.2e"
              % (lat, shape, steps, e))
        assert e < VEL_TOL, (lat, e)
        assert np.abs(rg - ro).max() < 1e-6 * ro.max()
    b.close()


def test_served_requests_match_oracle(elbm, orc):
    from paper_1904_00866_gb300 import serve
    reqs = [
        {"id": 0, "arrival": 0.0, "lattice": "D2Q9", "n": 40, "nu": 1e-3,
         "steps": 30, "seed": 41},
        {"id": 1, "arrival": 0.0, "lattice": "D3Q27", "n": 24, "nu": 2e-3,
         "steps": 21, "seed": 42},
        {"id": 2, "arrival": 0.02, "lattice": "D2Q9", "n": 33, "nu": 5e-3,
         "steps": 45, "seed": 43},
        {"id": 3, "arrival": 0.03, "lattice": "D3Q27", "n": 20, "nu": 1e-2,
         "steps": 12, "seed": 44},
    ]
    srv = serve.Server(elbm.Batch(burst=8), W.fields_for, budget_bytes=4e9,
                       max_members=2, burst=8)
    for r in reqs:
        srv.submit(r)
    rep = srv.run()
    assert rep["completed"] == len(reqs)
    # requests 2 and 3 waited for a slot and joined a running batch
    assert any(srv.done[i]["admitted"] > 0 for i in (2, 3))
    for r in reqs:
        n = r["n"]
        nz = n if r["lattice"] == "D3Q27" else 1
        o = orc.Lattice(r["lattice"], n, n, nz, nu=r["nu"])
        o.init_fields(*W.fields_for(r["lattice"], n, r["seed"]))
        o.step(r["steps"])
        ro, uo = o.moments()
        rg, ug = srv.done[r["id"]]["result"]
        e = _vel_err(ug, uo)
        print("served request %d (%s n=%d, %d steps): velocity L2 rel %.2e"
              % (r["id"], r["lattice"], n, r["steps"], e))
        assert e < VEL_TOL, (r["id"], e)
        assert np.abs(rg - ro).max() < 1e-6 * ro.max()
