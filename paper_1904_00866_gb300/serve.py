"""Continuous-batching server of ELBM runs on one GPU.

Requests (a lattice type, size, viscosity and step count) arrive over time.
The server keeps every admitted run's populations resident in device memory
as a member of one ``Batch`` and advances all of them together in bursts
(one persistent launch per step, replayed from a CUDA graph).  Between
bursts it retires finished runs (reading back their final density and
velocity) and admits waiting requests, first come first served, as long as
a member slot is free and the device-memory budget holds them.  A run that
arrives while others are on the GPU therefore starts at the next burst
boundary instead of waiting for the GPU to drain, and all runs' work
overlaps in the same launches.

``run_sequential`` serves the same requests one after another with the
single-lattice path, the baseline the serving numbers are compared with.

The scheduling logic is independent of the GPU: ``Server`` takes any object
with the ``Batch`` interface (``add``, ``set_steps``, ``step``, ``info``,
``moments``, ``remove``, ``sync``) and any clock, which the CPU tests use.
"""
import heapq
import time

import numpy as np

Q = {"D2Q9": 9, "D3Q27": 27}
D = {"D2Q9": 2, "D3Q27": 3}


def request_nodes(req):
    n = int(req["n"])
    return n * n if req["lattice"] == "D2Q9" else n * n * n


def request_bytes(req):
    """Device bytes a resident run needs: two FP32 population buffers, its
    share of the deferred-node queue (8 B/node, +25 % headroom) and of the
    undecided-node buffer (one 128-byte record per sixteen nodes, 8 B/node),
    and the transient FP64 field staging of initialisation."""
    nodes = request_nodes(req)
    q, d = Q[req["lattice"]], D[req["lattice"]]
    return nodes * (2 * q * 4 + 18 + (1 + d) * 8)


def percentile(values, p):
    if not values:
        return None
    return float(np.percentile(np.asarray(values, dtype=np.float64), p))


class Server:
    """Admit / step / retire loop over one batch.

    batch: object with the Batch interface; fields: callable
    (lattice, n, seed) -> (rho, u); budget_bytes: device memory the resident
    runs may use; max_members: resident runs at most (the batch's member
    limit, 256, by default); burst: steps per
    burst; clock: seconds (monotonic); keep_results: store final fields.
    """

    def __init__(self, batch, fields, budget_bytes=150e9, max_members=256,
                 burst=16, clock=time.monotonic, sleep=time.sleep,
                 keep_results=True):
        self.batch = batch
        self.fields = fields
        self.budget = float(budget_bytes)
        self.max_members = int(max_members)
        self.burst = int(burst)
        self.clock = clock
        self.sleep = sleep
        self._t0 = 0.0
        self.keep_results = keep_results
        self.waiting = []          # heap of (arrival, id, request)
        self.active = {}           # member id -> request
        self.used = 0.0
        self.done = {}             # request id -> record
        self.lattice_updates = 0
        self.bursts = 0
        self.peak_used = 0.0
        self.peak_active = 0
        # host seconds spent admitting, waiting for bursts and retiring
        self.t_admit = self.t_burst = self.t_retire = 0.0

    # -- submission ----------------------------------------------------------
    def submit(self, req):
        if request_bytes(req) > self.budget:
            raise ValueError("request %r needs more than the whole budget"
                             % req["id"])
        heapq.heappush(self.waiting, (req["arrival"], req["id"], req))

    def _admit(self, now):
        admitted = 0
        while self.waiting and len(self.active) < self.max_members:
            arrival, rid, req = self.waiting[0]
            if arrival > now:
                break
            need = request_bytes(req)
            if self.used + need > self.budget:
                break                      # FCFS: the head waits for memory
            heapq.heappop(self.waiting)
            rho, u = self.fields(req["lattice"], req["n"], req["seed"])
            n = int(req["n"])
            nz = n if req["lattice"] == "D3Q27" else 1
            mid = self.batch.add(req["lattice"], n, n, nz, req["nu"], rho, u)
            self.batch.set_steps(mid, int(req["steps"]))
            self.active[mid] = dict(req, admitted=self.clock() - self._t0,
                                    bytes=need)
            self.used += need
            admitted += 1
        self.peak_used = max(self.peak_used, self.used)
        self.peak_active = max(self.peak_active, len(self.active))
        return admitted

    def _retire(self):
        finished = []
        for mid, req in list(self.active.items()):
            done, remaining = self.batch.info(mid)
            if remaining == 0:
                finished.append((mid, req))
        for mid, req in finished:
            result = self.batch.moments(mid) if self.keep_results else None
            self.batch.remove(mid)
            t = self.clock() - self._t0
            self.used -= req["bytes"]
            self.lattice_updates += request_nodes(req) * int(req["steps"])
            self.done[req["id"]] = {
                "arrival": req["arrival"], "admitted": req["admitted"],
                "finished": t, "latency": t - req["arrival"],
                "steps": int(req["steps"]), "nodes": request_nodes(req),
                "result": result}
            del self.active[mid]
        return len(finished)

    # -- main loop -------------------------------------------------------------
    def run(self, t0=None, idle_sleep=1e-3):
        """Serve until every submitted request is done.  Arrival times are
        seconds after t0 (default: now)."""
        t0 = self.clock() if t0 is None else t0
        self._t0 = t0
        while self.waiting or self.active:
            ta = self.clock()
            self._admit(ta - t0)
            tb = self.clock()
            self.t_admit += tb - ta
            if not self.active:
                if self.waiting:
                    wait = self.waiting[0][0] - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(min(wait, idle_sleep * 50))
                continue
            self.batch.step(self.burst)
            self.batch.sync()
            tc = self.clock()
            self.t_burst += tc - tb
            self.bursts += 1
            self._retire()
            self.t_retire += self.clock() - tc
        return self.report()

    def report(self):
        lat = [r["latency"] for r in self.done.values()]
        if not self.done:
            return {"completed": 0}
        first = min(r["arrival"] for r in self.done.values())
        last = max(r["finished"] for r in self.done.values())
        makespan = max(last - first, 1e-9)
        return {
            "completed": len(self.done),
            "p50_s": percentile(lat, 50),
            "p99_s": percentile(lat, 99),
            "mean_s": float(np.mean(lat)),
            "makespan_s": makespan,
            "mlups": self.lattice_updates / makespan / 1e6,
            "bursts": self.bursts,
            "peak_resident": self.peak_active,
            "peak_budget_bytes": self.peak_used,
            "host_s": {"admit": round(self.t_admit, 3),
                       "bursts": round(self.t_burst, 3),
                       "retire": round(self.t_retire, 3)},
        }


def run_sequential(requests, make_lattice, fields, clock=time.monotonic,
                   sleep=time.sleep):
    """Serve the requests one after another (arrival order) with the
    single-lattice path.  make_lattice(req) -> object with init_fields,
    step(n), moments(), close()."""
    t0 = clock()
    done = {}
    updates = 0
    for req in sorted(requests, key=lambda r: r["arrival"]):
        now = clock() - t0
        if req["arrival"] > now:
            sleep(req["arrival"] - now)
        g = make_lattice(req)
        g.init_fields(*fields(req["lattice"], req["n"], req["seed"]))
        g.step(int(req["steps"]))
        result = g.moments()
        g.close()
        t = clock() - t0
        updates += request_nodes(req) * int(req["steps"])
        done[req["id"]] = {"arrival": req["arrival"], "finished": t,
                           "latency": t - req["arrival"], "result": result}
    lat = [r["latency"] for r in done.values()]
    first = min(r["arrival"] for r in done.values())
    last = max(r["finished"] for r in done.values())
    makespan = max(last - first, 1e-9)
    return done, {"completed": len(done), "p50_s": percentile(lat, 50),
                  "p99_s": percentile(lat, 99), "mean_s": float(np.mean(lat)),
                  "makespan_s": makespan, "mlups": updates / makespan / 1e6}
