"""The FP32-shifted FORMULA step has three kernel variants that differ only
in how the pull gathers reach shared memory (ELBM_SC32_VARIANT: "cpasync"
per-element gathers, the default; "wide" 16-byte row-segment gathers when
nx is a multiple of 64; "tma" bulk-copy row staging).  All run the
same per-node arithmetic on the same values, so the populations after any
number of steps must be bit-identical, including nodes deferred to the FP64
fixup; statistics agree up to summation order (per-thread compensated
FP32 sums over different node sets: 1e-8 relative).  The variant is chosen once
per process, so each case runs in a child process."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, json, numpy as np
sys.path.insert(0, %(root)r)
import elbm_workloads as W, paper_1904_00866_gb300 as elbm
lat, nx, ny, nz, noise, steps, out = %(args)r
if lat == "D2Q9":
    rho, u = W.random_phase_2d(nx, 7, umax=0.05, ny=ny)
else:
    rho, u = W.random_phase_3d(nx, 7, umax=0.05, ny=ny, nz=nz)
g = elbm.Lattice(lat, nx, ny, nz, nu=2e-4, dtype="fp32_shifted")
g.set_diagnostics(diag_every=1, check_every=1)
g.init_fields(rho, u)
if noise > 0:
    # populations multiplied by 1 + noise * U(-1, 1): nodes far from
    # equilibrium, which the FP32 kernels defer to the FP64 fixup
    f = g.populations()
    rng = np.random.default_rng(3)
    g.set_populations(f * (1.0 + noise * rng.uniform(-1.0, 1.0, f.shape)))
g.step(steps, "formula")
np.save(out, g.populations())
s = g.entropy_stats()
json.dump(s, open(out + ".json", "w"))
"""


def _run(args, variant):
    env = dict(os.environ, ELBM_SC32_VARIANT=variant)
    code = SCRIPT % {"root": ROOT, "args": args}
    r = subprocess.run([sys.executable, "-c", code], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    import json
    return np.load(args[-1]), json.load(open(args[-1] + ".json"))


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


# nx = 64: one segment per row, both halo chunks wrap; noise 0.3 puts
# nodes beyond the FP32 range into the FP64 fixup queue
CASES = [("D3Q27", 64, 6, 5, 0.0, 9), ("D3Q27", 128, 3, 4, 0.0, 7),
         ("D3Q27", 64, 8, 8, 0.3, 3), ("D2Q9", 192, 7, 1, 0.0, 11),
         ("D2Q9", 64, 64, 1, 0.3, 3)]


@pytest.mark.parametrize("lat,nx,ny,nz,noise,steps", CASES)
def test_wide_gathers_match_per_element_gathers(built, tmp_path, lat, nx, ny,
                                                nz, noise, steps):
    a, sa = _run((lat, nx, ny, nz, noise, steps, str(tmp_path / "w.npy")),
                 "wide")
    b, sb = _run((lat, nx, ny, nz, noise, steps, str(tmp_path / "c.npy")),
                 "cpasync")
    assert np.array_equal(a, b), np.abs(a - b).max()
    for k in ["n_nodes", "n_accept_two", "n_formula", "n_band", "n_far",
              "n_violations", "n_degenerate"]:
        assert sa[k] == sb[k], k
    assert sa["n_violations"] == 0
    if noise > 0:
        assert sa["n_far"] > 0      # the fixup path was exercised
    for k in ["mass", "kinetic_energy", "alpha_min", "alpha_max"]:
        assert abs(sa[k] - sb[k]) <= 1e-8 * max(abs(sb[k]), 1e-30), k
