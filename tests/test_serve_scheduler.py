"""CPU tests of the continuous-batching scheduler (paper_1904_00866_gb300.serve)
with a simulated batch and clock: admission is first come first served,
bounded by the member slots and the device-memory budget; runs that arrive
while others are resident join at the next burst; every run gets exactly
its step count; latencies and throughput are accounted on the clock."""
import numpy as np
import pytest

from paper_1904_00866_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 0.0)


class FakeBatch:
    """Steps advance the clock by the work done at `rate` updates/s."""

    def __init__(self, clock, rate=1e9):
        self.clock, self.rate = clock, rate
        self.m = {}
        self.next = 0
        self.log = []

    def add(self, lattice, nx, ny, nz, nu, rho, u):
        mid = self.next
        self.next += 1
        self.m[mid] = {"nodes": nx * ny * nz, "done": 0, "left": 10 ** 18}
        self.log.append(("add", mid, self.clock()))
        return mid

    def set_steps(self, mid, k):
        self.m[mid]["left"] = k

    def step(self, k):
        work = 0
        for r in self.m.values():
            take = min(k, r["left"])
            r["left"] -= take
            r["done"] += take
            work += take * r["nodes"]
        self.clock.t += work / self.rate + 1e-4

    def sync(self):
        pass

    def info(self, mid):
        return self.m[mid]["done"], self.m[mid]["left"]

    def moments(self, mid):
        return np.zeros(1), np.zeros(1)

    def remove(self, mid):
        self.log.append(("remove", mid, self.clock()))
        del self.m[mid]


def fields(lattice, n, seed):
    return None, None


def make_requests(k, seed=1, rate=50.0):
    return serve_requests(k, seed, rate)


def serve_requests(k, seed, rate):
    import elbm_workloads as W
    return W.request_stream(seed=seed, count=k, rate=rate)


def test_all_requests_complete_with_exact_steps():
    clock = FakeClock()
    b = FakeBatch(clock)
    srv = serve.Server(b, fields, budget_bytes=150e9, max_members=8,
                       burst=16, clock=clock, sleep=clock.sleep)
    reqs = make_requests(40)
    for r in reqs:
        srv.submit(r)
    rep = srv.run(t0=0.0)
    assert rep["completed"] == 40
    for r in reqs:
        d = srv.done[r["id"]]
        assert d["steps"] == r["steps"]
        assert d["finished"] >= r["arrival"]
        assert d["latency"] > 0
    assert rep["peak_resident"] <= 8
    assert rep["p50_s"] <= rep["p99_s"]
    assert rep["mlups"] > 0


def test_fcfs_admission_and_budget():
    clock = FakeClock()
    b = FakeBatch(clock)
    reqs = make_requests(30)
    budget = max(serve.request_bytes(r) for r in reqs) * 1.5
    srv = serve.Server(b, fields, budget_bytes=budget, max_members=64,
                       burst=8, clock=clock, sleep=clock.sleep)
    for r in reqs:
        srv.submit(r)
    srv.run(t0=0.0)
    assert srv.peak_used <= budget
    admitted = [srv.done[r["id"]]["admitted"] for r in
                sorted(reqs, key=lambda r: (r["arrival"], r["id"]))]
    assert all(a <= b_ for a, b_ in zip(admitted, admitted[1:]))


def test_arrivals_join_running_batch():
    # a long run is resident; a short one arriving later joins before the
    # long one finishes (continuous batching, not a queue)
    clock = FakeClock()
    b = FakeBatch(clock, rate=1e7)
    long_req = {"id": 0, "arrival": 0.0, "lattice": "D3Q27", "n": 64,
                "nu": 1e-3, "steps": 5000, "seed": 1}
    short_req = {"id": 1, "arrival": 0.5, "lattice": "D2Q9", "n": 64,
                 "nu": 1e-3, "steps": 100, "seed": 2}
    srv = serve.Server(b, fields, budget_bytes=1e12, max_members=4,
                       burst=16, clock=clock, sleep=clock.sleep)
    srv.submit(long_req)
    srv.submit(short_req)
    srv.run(t0=0.0)
    d0, d1 = srv.done[0], srv.done[1]
    assert d1["admitted"] < d0["finished"]
    assert d1["finished"] < d0["finished"]
    assert d1["admitted"] - short_req["arrival"] < 1.0


def test_oversized_request_is_refused():
    clock = FakeClock()
    srv = serve.Server(FakeBatch(clock), fields, budget_bytes=1e6,
                       clock=clock, sleep=clock.sleep)
    with pytest.raises(ValueError):
        srv.submit({"id": 0, "arrival": 0.0, "lattice": "D3Q27", "n": 64,
                    "nu": 1e-3, "steps": 10, "seed": 1})


def test_sequential_baseline_accounting():
    clock = FakeClock()

    class FakeLattice:
        def __init__(self, req):
            self.nodes = serve.request_nodes(req)

        def init_fields(self, rho, u):
            pass

        def step(self, k):
            clock.t += k * self.nodes / 1e9

        def moments(self):
            return None

        def close(self):
            pass

    reqs = make_requests(10)
    done, rep = serve.run_sequential(reqs, FakeLattice, fields, clock=clock,
                                     sleep=clock.sleep)
    assert rep["completed"] == 10
    fin = [done[r["id"]]["finished"] for r in sorted(reqs,
                                                     key=lambda r: r["arrival"])]
    assert all(a <= b for a, b in zip(fin, fin[1:]))
