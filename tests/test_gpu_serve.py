"""Serving on the GPU: requests admitted into a shared batch while others
are running must give the same result as the same request served alone
(the batched kernel advances each lattice independently), and the same as
the single-lattice path."""
import os

import numpy as np
import pytest

import elbm_workloads as W

pytestmark = pytest.mark.gpu

REQS = [
    {"id": 0, "arrival": 0.0, "lattice": "D2Q9", "n": 48, "nu": 1e-3, "steps": 40, "seed": 11},
    {"id": 1, "arrival": 0.0, "lattice": "D3Q27", "n": 16, "nu": 2e-3, "steps": 25, "seed": 12},
    {"id": 2, "arrival": 0.01, "lattice": "D2Q9", "n": 80, "nu": 1e-5, "steps": 9, "seed": 13},
    {"id": 3, "arrival": 0.02, "lattice": "D3Q27", "n": 24, "nu": 1e-4, "steps": 33, "seed": 14},
    {"id": 4, "arrival": 0.03, "lattice": "D2Q9", "n": 64, "nu": 5e-3, "steps": 17, "seed": 15},
    {"id": 5, "arrival": 0.04, "lattice": "D3Q27", "n": 20, "nu": 1e-3, "steps": 50, "seed": 16},
]


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


def _same(a, b):
    ra, ua = a
    rb, ub = b
    assert np.array_equal(ra, rb) and np.array_equal(ua, ub)


def test_results_same_alone_and_in_the_mix(elbm):
    from paper_1904_00866_gb300 import serve
    mix = serve.Server(elbm.Batch(burst=8), W.fields_for, budget_bytes=4e9,
                       max_members=3, burst=8)
    for r in REQS:
        mix.submit(r)
    rep = mix.run()
    assert rep["completed"] == len(REQS)
    assert rep["peak_resident"] <= 3
    # some request joined while another one was resident
    d = mix.done
    assert any(d[i]["admitted"] < d[j]["finished"] and d[i]["admitted"] >
               d[j]["admitted"] for i in d for j in d if i != j)
    for r in REQS:
        alone = serve.Server(elbm.Batch(burst=8), W.fields_for,
                             budget_bytes=4e9, max_members=1, burst=8)
        alone.submit(dict(r, arrival=0.0))
        alone.run()
        _same(d[r["id"]]["result"], alone.done[r["id"]]["result"])

    def make(req):
        n = req["n"]
        nz = n if req["lattice"] == "D3Q27" else 1
        return elbm.Lattice(req["lattice"], n, n, nz, nu=req["nu"],
                            dtype="fp32_shifted")
    seq, srep = serve.run_sequential([dict(r, arrival=0.0) for r in REQS],
                                     make, W.fields_for)
    for r in REQS:
        _same(d[r["id"]]["result"], seq[r["id"]]["result"])
