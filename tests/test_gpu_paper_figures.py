"""GPU runs of the paper's double shear layer (Figs. 3-5) against the oracle.

Fig. 5 plots, per step, the share of nodes where alpha = 2 is accepted
without Eq. (9) (H(f*(2)) <= H(f)).  The GPU counts it in the fused
statistics of every diagnostic step.  On the 128^2 layer with nu = 1e-5
(the figures' setting) the counts are compared with the oracle's at every
100th step of T = 3200:

  * FP64 storage: the same decisions up to nodes whose Delta H(2) lies
    within FP64 rounding of zero (at most 1e-3 of the nodes per step).
    Step 0 is left out: there f = f^eq up to the rounding of two
    independent initialisations, so every decision is rounding noise;
  * FP32-shifted storage: the certified decision accepts alpha = 2 only
    where Delta H(2) + e2 <= 0, so its count is at most the FP64 count of
    its own state and falls short by at most the band nodes; the FP32 and
    FP64 trajectories also drift apart slowly, so the comparison with the
    oracle's count allows the band share plus 0.5 %.
"""
import json
import os

import numpy as np
import pytest

import elbm_workloads as W

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_values.json")))


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
def oracle_counts():
    import oracle
    g = GOLD["double_shear_layer"]
    n = g["M"]
    rho, u = W.shear_layer(n, g["U"], g["lambda"], g["perturbation"])
    L = oracle.Lattice("D2Q9", n, n, 1, nu=g["nu"])
    L.init_fields(rho, u)
    _, st = L.step(g["T"], stats=True)
    return np.array([s["n_accept_two"] for s in st]), n * n


def _gpu_counts(elbm, dtype):
    g = GOLD["double_shear_layer"]
    n = g["M"]
    rho, u = W.shear_layer(n, g["U"], g["lambda"], g["perturbation"])
    lat = elbm.Lattice("D2Q9", n, n, 1, nu=g["nu"], dtype=dtype)
    lat.set_diagnostics(diag_every=100)
    lat.init_fields(rho, u)
    counts, bands = [], []
    for _ in range(g["T"] // 100):
        lat.step(100, "formula")        # statistics of its first step
        s = lat.entropy_stats()
        counts.append(s["n_accept_two"])
        bands.append(s["n_band"])
        assert s["n_violations"] == 0
    return np.array(counts), np.array(bands)


def test_fig5_counter_fp64_matches_oracle(elbm, oracle_counts):
    ref, nodes = oracle_counts
    got, _ = _gpu_counts(elbm, "fp64")
    want = ref[::100]
    d = np.abs(got - want)[1:]
    assert np.all(d <= 1e-3 * nodes), d.max()
    prop = got / nodes
    assert abs(np.median(prop[1:]) - GOLD["accept_two_proportion"]["value"]) < 0.1


def test_fig5_counter_fp32_within_band(elbm, oracle_counts):
    ref, nodes = oracle_counts
    got, band = _gpu_counts(elbm, "fp32_shifted")
    want = ref[::100]
    short = ((want - got) / nodes)[1:]
    band = band[1:]
    assert np.all(short >= -0.005), short.min()
    assert np.all(short <= band / nodes + 0.005), (short - band / nodes).max()
    print("Fig. 5 share, FP32 vs oracle: max shortfall %.4f, median share %.3f"
          % (short.max(), np.median(got[1:] / nodes)))


def _vorticity(u):
    """omega_z = dv/dx - du/dy (central differences, periodic), u: (2, 1, n, n)."""
    ux, uy = u[0, 0], u[1, 0]
    dvdx = 0.5 * (np.roll(uy, -1, axis=1) - np.roll(uy, 1, axis=1))
    dudy = 0.5 * (np.roll(ux, -1, axis=0) - np.roll(ux, 1, axis=0))
    return dvdx - dudy


def _run_to_t1(elbm, mode):
    """Vorticity at t = 1 (step T) and the alpha map of its collision."""
    g = GOLD["double_shear_layer"]
    n = g["M"]
    rho, u = W.shear_layer(n, g["U"], g["lambda"], g["perturbation"])
    lat = elbm.Lattice("D2Q9", n, n, 1, nu=g["nu"], dtype="fp64")
    lat.set_diagnostics(diag_every=100, alpha_map_every=g["T"])
    lat.init_fields(rho, u)
    lat.step(g["T"], mode)            # alpha of the collisions at step T
    omega = _vorticity(lat.moments()[1])
    lat.step(1, mode)
    return omega, lat.alpha_map()[0].astype(np.float64)


def _blocks(a, b):
    """Mean over b x b blocks of a square field."""
    n = a.shape[0] // b
    return a[:n * b, :n * b].reshape(n, b, n, b).mean(axis=(1, 3))


def test_fig3_fig4_formula_vs_root_at_t1(elbm):
    """Figs. 3-4 (t = 1, nu = 1e-5, 128^2): the vortex patterns of the
    formula and of the bisection match closely, and the formula's alpha
    drops below 2 at the vortices while staying near 2 away from them.  The figures' data is
    not printed, so these are bands around the stated behaviour."""
    wf, af = _run_to_t1(elbm, "formula")
    wr, ar = _run_to_t1(elbm, "root")
    out = {}
    out["rel_l2"] = np.linalg.norm(wf - wr) / np.linalg.norm(wr)
    out["corr"] = np.corrcoef(wf.ravel(), wr.ravel())[0, 1]
    for b in (4, 8, 16):
        out["corr_b%d" % b] = np.corrcoef(_blocks(wf, b).ravel(),
                                          _blocks(wr, b).ravel())[0, 1]
    out["enstrophy_ratio"] = np.mean(wf ** 2) / np.mean(wr ** 2)
    dev = 2.0 - af
    sm = np.abs(_blocks(wf, 4))
    dev4 = _blocks(dev, 4)
    hi = sm > np.quantile(sm, 0.9)
    lo = sm < np.quantile(sm, 0.5)
    out["dev_hi_over_lo_b4"] = dev4[hi].mean() / max(dev4[lo].mean(), 1e-300)
    out["corr_dev_absw_b4"] = np.corrcoef(dev4.ravel(), sm.ravel())[0, 1]
    out["share_alpha_lt2"] = np.mean(af < 2.0)
    out["root_share_lt2"] = np.mean(ar < 2.0)
    print("t=1:", {k: round(float(v), 4) for k, v in out.items()})
    # pointwise the two runs drift apart (Re = 512000 on 128^2 amplifies
    # the small alpha differences: correlation ~0.91), but at the scale of
    # the vortices the shapes agree
    assert out["corr_b8"] > 0.95 and out["corr_b16"] > 0.98
    # the formula's alpha is at most the root (Eq. (9) lower bound), so it
    # dissipates more: less enstrophy, by a bounded amount
    assert 0.7 < out["enstrophy_ratio"] <= 1.0
    # alpha deviates from 2 more where the flow is most vortical (measured
    # 1.23x in the top tenth of 4 x 4 blocks over the calmer half)
    assert out["dev_hi_over_lo_b4"] > 1.05
    # and about half of the nodes need Eq. (9) (Fig. 5)
    assert 0.3 < out["share_alpha_lt2"] < 0.7
