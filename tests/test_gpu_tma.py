"""The bulk-copy (TMA) staging variant of the FP32-shifted FORMULA kernel
(selected by ELBM_SC32_VARIANT=tma when nx is a multiple of 256) must give the
same populations as the default per-thread gather kernel and stay within FP32
tolerance of the FP64 oracle.  The variant is chosen once per process, so
each case runs in a child process."""
import os
import subprocess
import sys

import numpy as np
import pytest

import elbm_workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, %(root)r)
import elbm_workloads as W, paper_1904_00866_gb300 as elbm
lat, nx, ny, nz, nu, seed, steps, out = %(args)r
if lat == "D2Q9":
    rho, u = W.shear_waves_2d(nx, seed) if nx == ny else W.random_phase_2d(nx, seed, ny=ny)
else:
    rho, u = W.random_phase_3d(nx, seed, ny=ny, nz=nz)
g = elbm.Lattice(lat, nx, ny, nz, nu=nu, dtype="fp32_shifted")
g.set_diagnostics(diag_every=1, check_every=1)
g.init_fields(rho, u)
g.step(steps, "formula")
np.save(out, g.populations())
np.save(out + ".u.npy", g.moments()[1])
s = g.entropy_stats()
assert s["n_violations"] == 0, s
"""


def _run(args, env_extra):
    env = dict(os.environ, **env_extra)
    code = SCRIPT % {"root": ROOT, "args": args}
    r = subprocess.run([sys.executable, "-c", code], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(args[-1])


@pytest.fixture(scope="module")
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_00866_gb300 as e
    if not os.path.exists(e.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    return e


@pytest.mark.parametrize("lat,nx,ny,nz", [("D3Q27", 256, 12, 10),
                                          ("D2Q9", 512, 40, 1)])
def test_tma_path_matches_gather_path(built, tmp_path, lat, nx, ny, nz):
    a = _run((lat, nx, ny, nz, 1e-4, 3, 12, str(tmp_path / "tma.npy")),
             {"ELBM_SC32_VARIANT": "tma"})
    b = _run((lat, nx, ny, nz, 1e-4, 3, 12, str(tmp_path / "gather.npy")), {})
    assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()


def test_tma_path_matches_oracle(built, tmp_path):
    import oracle
    nx, ny, nz, steps = 256, 6, 5, 40
    out = str(tmp_path / "tma_o.npy")
    _run(("D3Q27", nx, ny, nz, 5e-3, 9, steps, out),
         {"ELBM_SC32_VARIANT": "tma"})
    ug = np.load(out + ".u.npy")
    rho, u = W.random_phase_3d(nx, 9, ny=ny, nz=nz)
    o = oracle.Lattice("D3Q27", nx, ny, nz, nu=5e-3)
    o.init_fields(rho, u)
    o.step(steps)
    _, uo = o.moments()
    assert np.linalg.norm(ug - uo) / np.linalg.norm(uo) < 1e-5
