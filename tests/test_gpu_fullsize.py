"""Parity at the benchmark's full size: D3Q27 512^3 Taylor-Green (Re = 1600,
u0 = 0.05), FP32-shifted storage, FORMULA, in the launch configuration the
benchmark times.  The oracle collides sampled nodes one by one from the
GPU's pre-step populations; the GPU's post-step populations at x + c_i must
match, and the FP64 check must report zero violations over the lattice."""
import math
import os

import numpy as np
import pytest

import elbm_workloads as W

pytestmark = pytest.mark.gpu

N = 512
NU = 0.05 * (N / (2 * math.pi)) / 1600.0


@pytest.fixture(scope="module")
def elbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 40e9:
        pytest.skip("needs ~40 GB of free device memory")
    import paper_1904_00866_gb300 as e
    if not os.path.exists(e.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    e.lib()
    return e


def test_512_cubed_sampled_nodes(elbm):
    import oracle
    rho, u = W.taylor_green_3d(N, 0.05)
    g = elbm.Lattice("D3Q27", N, N, N, nu=NU, dtype="fp32_shifted")
    g.set_diagnostics(diag_every=1, check_every=0, alpha_map_every=1)
    g.init_fields(rho, u)
    del rho, u
    g.step(3, "formula")
    rng = np.random.default_rng(0)
    nodes = rng.integers(0, N ** 3, size=512)
    nodes[:4] = [0, N - 1, N * N * N - 1, N * N]     # wrap corners
    f_pre = g.populations_at(nodes)
    c, w = oracle.lattice("D3Q27")
    g.set_diagnostics(diag_every=1, check_every=1, alpha_map_every=1)
    g.step(1, "formula")
    amap = g.alpha_map().reshape(-1)
    x = nodes % N
    y = (nodes // N) % N
    z = nodes // (N * N)
    beta = oracle.beta_from_nu(NU)
    for i in range(27):
        dst = (((z + c[i, 2]) % N) * N + (y + c[i, 1]) % N) * N + (x + c[i, 0]) % N
        post = g.populations_at(dst)[:, i]
        for k in range(len(nodes)):
            ft, a, fl, _ = oracle.collide_node("D3Q27", f_pre[k], beta)
            assert amap[nodes[k]] <= a + 1e-12
            assert a - amap[nodes[k]] <= 1e-4
            assert abs(post[k] - ft[i]) <= 2e-6 * ft[i]
    s = g.entropy_stats()
    assert s["checked"] == 1 and s["n_violations"] == 0, s
    assert s["n_nodes"] == N ** 3
