"""elbm_step_static: the step for callers that cannot allocate device memory.

Such callers (an application that reserves all of its device memory in its
own pool at start-up, or a latency-critical loop that must not wait on the
allocator's implicit synchronisation) own the population buffers and call
elbm_step_static, whose scratch lives in a fixed array inside the library.
This file checks, through the C ABI, that two consecutive static calls give
the same populations and statistics as two steps of the handle-based
elbm_step on the same state, and that oversized lattices are refused.  It is
collected last, and works alone or after the other tests.
"""
import ctypes
import os

import numpy as np
import pytest

import elbm_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_00866_gb300 as e
    if not os.path.exists(e.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    e.lib()
    import oracle
    return e, torch, oracle


def _to_pull_layout(orc, lat, f_pre, rho0):
    """Pre-collision f^n (FP64) -> FP32-shifted pull layout:
    buffer_i[x - c_i] = f_i(x) - W_i rho0."""
    c, w = orc.lattice(lat)
    out = np.empty(f_pre.shape, dtype=np.float32)
    for i in range(len(w)):
        dev = (f_pre[i] - w[i] * rho0).astype(np.float32)
        out[i] = np.roll(dev, shift=(-c[i, 2], -c[i, 1], -c[i, 0]),
                         axis=(0, 1, 2))
    return out


def _from_pull_layout(orc, lat, buf, rho0):
    c, w = orc.lattice(lat)
    out = np.empty(buf.shape)
    for i in range(len(w)):
        out[i] = w[i] * rho0 + np.roll(buf[i].astype(np.float64),
                                       shift=(c[i, 2], c[i, 1], c[i, 0]),
                                       axis=(0, 1, 2))
    return out


@pytest.mark.parametrize("lat,shape,nu", [("D3Q27", (14, 17, 40), 2e-3),
                                          ("D2Q9", (1, 61, 96), 1e-4)])
def test_static_step_matches_handle_step_twice(env, lat, shape, nu):
    elbm, torch, orc = env
    nz, ny, nx = shape
    if lat == "D2Q9":
        rho, u = W.random_phase_2d(nx, seed=21, umax=0.05, ny=ny)
    else:
        rho, u = W.random_phase_3d(nx, seed=21, umax=0.05, ny=ny, nz=nz)
    g = elbm.Lattice(lat, nx, ny, nz, nu=nu, dtype="fp32_shifted")
    g.init_fields(rho, u)
    g.step(5, "formula")                  # a state away from equilibrium
    f_pre = g.populations()
    g.set_populations(f_pre)              # handle state == static input
    rho0 = g.rho0
    bufs = [torch.from_numpy(_to_pull_layout(orc, lat, f_pre, rho0)).cuda(),
            torch.empty((len(f_pre),) + shape, dtype=torch.float32,
                        device="cuda")]
    stream = torch.cuda.current_stream().cuda_stream
    L = elbm.lib()
    lat_id = elbm.LATTICES[lat]
    g.set_diagnostics(diag_every=1)
    for call in range(2):
        src, dst = bufs[call % 2], bufs[(call + 1) % 2]
        st = elbm.EntropyStats()
        rc = L.elbm_step_static(lat_id, nx, ny, nz, nu, rho0,
                                ctypes.c_void_p(src.data_ptr()),
                                ctypes.c_void_p(dst.data_ptr()), None,
                                ctypes.c_void_p(stream), ctypes.byref(st))
        assert rc == 0, L.elbm_last_error(None)
        g.step(1, "formula")
        ref = g.populations()
        got = _from_pull_layout(orc, lat, dst.cpu().numpy(), rho0)
        assert np.all(np.abs(got - ref) <= 2e-6 * np.abs(ref)), call
        s_ref = g.entropy_stats()
        s = st.as_dict()
        assert s["n_nodes"] == s_ref["n_nodes"] == nx * ny * nz
        for k in ["n_accept_two", "n_formula", "n_band", "n_far"]:
            assert s[k] == s_ref[k], k
        for k in ["mass", "kinetic_energy", "alpha_min", "alpha_max"]:
            assert abs(s[k] - s_ref[k]) <= 1e-9 * max(1.0, abs(s_ref[k])), k


def test_static_step_rejects_oversized_lattice(env):
    elbm, torch, orc = env
    L = elbm.lib()
    x = torch.empty(16, dtype=torch.float32, device="cuda")
    y = torch.empty(16, dtype=torch.float32, device="cuda")
    rc = L.elbm_step_static(1, 129, 128, 128, 1e-3, 1.0,
                            ctypes.c_void_p(x.data_ptr()),
                            ctypes.c_void_p(y.data_ptr()), None, None, None)
    assert rc == 1
    assert b"at most 2097152" in L.elbm_last_error(None)
