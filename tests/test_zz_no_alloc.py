"""elbm_step_static: the step for callers that cannot allocate device memory.

Such callers (an application that reserves all of its device memory in its
own pool at start-up, or a latency-critical loop that must not wait on the
allocator's implicit synchronisation) own the population buffers and call
elbm_step_static, whose scratch lives in a fixed array inside the library.
This file checks, through the C ABI, that two consecutive static calls give
the same populations, alpha map and statistics as two steps of the
handle-based elbm_step on the same state, that the device's free memory does
not change across them, that the opt-in bulk-copy kernel variant gives the
same result through this entry point, and that oversized lattices are
refused.  It is collected last, and works alone or after the other tests.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import elbm_workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def _static(elbm, L, lat, shape, nu, rho0, src, dst, amap, stream, st):
    nz, ny, nx = shape
    return L.elbm_step_static(
        elbm.LATTICES[lat], nx, ny, nz, nu, rho0,
        ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
        ctypes.c_void_p(amap.data_ptr()) if amap is not None else None,
        ctypes.c_void_p(stream), ctypes.byref(st) if st is not None else None)


def _compare_two_calls(elbm, torch, orc, lat, shape, nu, seed):
    """Two static calls in a row against two elbm_step steps of a handle
    holding the same state.  Returns the largest relative population
    difference."""
    nz, ny, nx = shape
    if lat == "D2Q9":
        rho, u = W.random_phase_2d(nx, seed=seed, umax=0.05, ny=ny)
    else:
        rho, u = W.random_phase_3d(nx, seed=seed, umax=0.05, ny=ny, nz=nz)
    g = elbm.Lattice(lat, nx, ny, nz, nu=nu, dtype="fp32_shifted")
    g.init_fields(rho, u)
    g.step(5, "formula")                  # a state away from equilibrium
    f_pre = g.populations()
    g.set_populations(f_pre)              # handle state == static input
    rho0 = g.rho0
    q = len(f_pre)
    start = torch.from_numpy(_to_pull_layout(orc, lat, f_pre, rho0)).cuda()
    bufs = [start.clone(), torch.empty_like(start), torch.empty_like(start)]
    amaps = [torch.empty(shape, dtype=torch.float32, device="cuda")
             for _ in range(2)]
    stream = torch.cuda.current_stream().cuda_stream
    L = elbm.lib()
    # warm-up call: the first call on a device looks up the scratch array's
    # address, and lazy module loading may place the library's device code
    # and data then; its result is discarded
    warm = torch.empty_like(start)
    assert _static(elbm, L, lat, shape, nu, rho0, start, warm, None, stream,
                   elbm.EntropyStats()) == 0, L.elbm_last_error(None)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    stats = []
    for call in range(2):
        st = elbm.EntropyStats()
        rc = _static(elbm, L, lat, shape, nu, rho0, bufs[call],
                     bufs[call + 1], amaps[call], stream, st)
        assert rc == 0, L.elbm_last_error(None)
        stats.append(st.as_dict())
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before   # nothing allocated
    g.set_diagnostics(diag_every=1, alpha_map_every=1)
    worst = 0.0
    for call in range(2):
        g.step(1, "formula")
        ref = g.populations()
        got = _from_pull_layout(orc, lat, bufs[call + 1].cpu().numpy(), rho0)
        rel = np.abs(got - ref) / np.abs(ref)
        worst = max(worst, float(rel.max()))
        assert np.all(rel <= 2e-6), (call, rel.max())
        assert np.array_equal(amaps[call].cpu().numpy(), g.alpha_map()), call
        s_ref = g.entropy_stats()
        s = stats[call]
        assert s["n_nodes"] == s_ref["n_nodes"] == nx * ny * nz
        for k in ["n_accept_two", "n_formula", "n_band", "n_far"]:
            assert s[k] == s_ref[k], k
        for k in ["mass", "kinetic_energy", "alpha_min", "alpha_max"]:
            assert abs(s[k] - s_ref[k]) <= 1e-9 * max(1.0, abs(s_ref[k])), k
    assert q * nx * ny * nz == bufs[0].numel()
    return worst


@pytest.mark.parametrize("lat,shape,nu", [("D3Q27", (14, 17, 40), 2e-3),
                                          ("D2Q9", (1, 61, 96), 1e-4)])
def test_static_step_matches_handle_step_twice(env, lat, shape, nu):
    elbm, torch, orc = env
    _compare_two_calls(elbm, torch, orc, lat, shape, nu, seed=21)


_TMA_CHILD = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch
import paper_1904_00866_gb300 as elbm
import oracle
sys.path.insert(0, os.path.join({root!r}, "tests"))
import test_zz_no_alloc as t
worst = t._compare_two_calls(elbm, torch, oracle, "D3Q27", (6, 5, 256),
                             1e-3, seed=22)
print("tma static ok %.3e" % worst)
"""


def test_static_step_with_bulk_copy_variant(env):
    """The same check with the opt-in bulk-copy (TMA) kernel, which the
    static entry point reaches when ELBM_SC32_VARIANT=tma and nx % 256 == 0
    (the variant is chosen once per process, hence the child process)."""
    env_vars = dict(os.environ, ELBM_SC32_VARIANT="tma")
    r = subprocess.run([sys.executable, "-c", _TMA_CHILD.format(root=ROOT)],
                       env=env_vars, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "tma static ok" in r.stdout


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
