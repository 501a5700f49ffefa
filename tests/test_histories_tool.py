"""Host logic of histories.py (the Taylor-Green history runner) with a fake
lattice: the convective time, the normalisation by the initial values, the
recorded statistics and the comparison of two runs."""
import json
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import histories  # noqa: E402


class FakeLattice:
    """Energy decays by exp(-0.01 t), enstrophy grows linearly."""

    def __init__(self, lattice, nx, ny, nz, nu, dtype):
        self.n, self.t = nx, 0

    def set_decision(self, d):
        pass

    def set_diagnostics(self, **k):
        pass

    def init_fields(self, rho, u):
        self.rho, self.u = rho, u

    def moments(self):
        return self.rho, self.u * math.exp(-0.005 * self.t)

    def enstrophy(self):
        return 2.0 + 1e-3 * self.t

    def step(self, n, mode):
        self.t += n

    def sync(self):
        pass

    def entropy_stats(self):
        return {"n_violations": 0, "n_decision_mismatch": 0,
                "n_formula": 7, "alpha_min": 1.99, "step": self.t}

    def close(self):
        pass


class FakeModule:
    Lattice = FakeLattice


def test_history_records_normalised_samples(tmp_path):
    out = tmp_path / "h.json"
    r = histories.tgv_history(FakeModule, 16, "fp32_shifted", samples=3,
                              out_path=str(out))
    tc = int(round(16 / (2 * math.pi) / 0.05))
    assert r["tc_steps"] == tc and r["t"] == [1, 2, 3]
    for k, e in enumerate(r["energy"], start=1):
        assert math.isclose(e, math.exp(-0.01 * k * tc), rel_tol=1e-12)
    for k, z in enumerate(r["enstrophy"], start=1):
        assert math.isclose(z, (2.0 + 1e-3 * k * tc) / 2.0, rel_tol=1e-12)
    assert r["share_eq9"] == [7 / 16 ** 3] * 3
    assert json.load(open(out))["energy"] == r["energy"]


def test_compare_reports_largest_relative_deviation():
    base = {"n": 8, "dtype": "fp64", "decision": "exact", "t": [1, 2, 3],
            "energy": [1.0, 0.5, 0.25], "enstrophy": [1.0, 2.0, 4.0],
            "n_violations": [0, 0, 0], "n_decision_mismatch": [0, 0, 0]}
    other = dict(base, dtype="fp32_shifted", energy=[1.0, 0.505, 0.25],
                 enstrophy=[1.0, 2.0, 3.96], n_decision_mismatch=[2, 0, 0])
    (row,) = histories.compare([base, other])
    assert math.isclose(row["max_rel_dev_energy"], 0.01, rel_tol=1e-9)
    assert row["at_tc_energy"] == 2
    assert math.isclose(row["max_rel_dev_enstrophy"], 0.01, rel_tol=1e-9)
    assert row["at_tc_enstrophy"] == 3
    assert row["decision_mismatches"] == 2
    assert np.isfinite(row["max_rel_dev_energy"])
