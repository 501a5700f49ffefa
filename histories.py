"""Kinetic-energy and enstrophy histories of the D3Q27 Taylor-Green vortex
at Re = 1600 on the GPU path, for comparing storage types, decision modes
and resolutions over many convective times.

The flow: u0 = 0.05 (Ma ~ 0.09), L = N / 2 pi, nu = u0 L / Re, initial
fields of the standard Taylor-Green vortex with its pressure, f = f^eq
(elbm_workloads.taylor_green_3d).  The time unit is the convective time
t_c = L / u0 (rounded to whole steps); after every t_c the run records
the kinetic energy 1/2 sum rho |u|^2 (from the moments) and the enstrophy
1/2 <|curl u|^2> (central differences, computed on the device), both
divided by their initial values so that runs at different resolutions are
comparable, and the entropy statistics of the diagnostic step of the
interval (its first step: 0, t_c, 2 t_c, ...): the FP64 check's
H-increase and decision-mismatch counts, the share of nodes on Eq. (9),
the smallest alpha.

    python histories.py run --n 256 --dtype fp64 --tc 20 --out a.json
    python histories.py run --n 256 --dtype fp32_shifted --out b.json
    python histories.py compare a.json b.json

`compare` prints, for each run against the first, the largest relative
deviation of the normalised energy and enstrophy over the common samples.
"""
import argparse
import json
import math
import sys
import time

import numpy as np

import elbm_workloads as W


def tgv_history(elbm, n, dtype, samples=20, re=1600.0, u0=0.05,
                decision="exact", log=None, out_path=None):
    """Run the vortex for `samples` convective times; returns the record
    (also rewritten to out_path after every sample, when given)."""
    L = n / (2 * math.pi)
    nu = u0 * L / re
    tc = int(round(L / u0))
    g = elbm.Lattice("D3Q27", n, n, n, nu=nu, dtype=dtype)
    if dtype != "fp64":
        g.set_decision(decision)
    g.set_diagnostics(diag_every=tc, check_every=tc)
    rho, u = W.taylor_green_3d(n, u0)
    g.init_fields(rho, u)
    del rho, u

    def energy():
        r, v = g.moments()
        return 0.5 * sum(float(np.vdot(r, v[a] * v[a]))
                         for a in range(v.shape[0]))

    e0, z0 = energy(), g.enstrophy()
    out = {"n": n, "dtype": dtype, "decision": decision, "re": re, "u0": u0,
           "nu": nu, "tc_steps": tc, "e0": e0, "z0": z0,
           "t": [], "energy": [], "enstrophy": [], "n_violations": [],
           "n_decision_mismatch": [], "share_eq9": [], "alpha_min": [],
           "stats_step": [], "seconds": []}
    for k in range(1, samples + 1):
        t0 = time.time()
        g.step(tc, "formula")
        g.sync()
        dt = time.time() - t0
        s = g.entropy_stats()
        out["t"].append(k)
        out["energy"].append(energy() / e0)
        out["enstrophy"].append(g.enstrophy() / z0)
        out["n_violations"].append(int(s["n_violations"]))
        out["n_decision_mismatch"].append(int(s["n_decision_mismatch"]))
        out["share_eq9"].append(float(s["n_formula"]) / float(n) ** 3)
        out["alpha_min"].append(float(s["alpha_min"]))
        out["stats_step"].append(int(s["step"]))
        out["seconds"].append(round(dt, 3))
        if out_path:
            with open(out_path, "w") as f:
                json.dump(out, f)
        if log:
            print("%s n=%d %s t=%d t_c: E/E0 %.6f  Z/Z0 %.6f  (%.1f s)"
                  % (dtype, n, decision, k, out["energy"][-1],
                     out["enstrophy"][-1], dt), file=log, flush=True)
    g.close()
    return out


def compare(runs):
    base = runs[0]
    rows = []
    for r in runs[1:]:
        m = min(len(base["t"]), len(r["t"]))
        e = np.abs(np.array(r["energy"][:m]) / np.array(base["energy"][:m])
                   - 1)
        z = np.abs(np.array(r["enstrophy"][:m])
                   / np.array(base["enstrophy"][:m]) - 1)
        rows.append({"run": "%s n=%d %s" % (r["dtype"], r["n"], r["decision"]),
                     "vs": "%s n=%d" % (base["dtype"], base["n"]),
                     "samples": m, "max_rel_dev_energy": float(e.max()),
                     "max_rel_dev_enstrophy": float(z.max()),
                     "at_tc_energy": int(np.argmax(e)) + 1,
                     "at_tc_enstrophy": int(np.argmax(z)) + 1,
                     "violations": int(sum(r["n_violations"])),
                     "decision_mismatches": int(sum(r["n_decision_mismatch"]))})
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("run")
    a.add_argument("--n", type=int, default=256)
    a.add_argument("--dtype", default="fp32_shifted",
                   choices=["fp64", "fp32", "fp32_shifted", "fp16_shifted"])
    a.add_argument("--decision", default="exact",
                   choices=["exact", "certified"])
    a.add_argument("--tc", type=int, default=20,
                   help="convective times to run (one sample each)")
    a.add_argument("--re", type=float, default=1600.0)
    a.add_argument("--out", required=True)
    c = sub.add_parser("compare")
    c.add_argument("files", nargs="+")
    args = ap.parse_args(argv)
    if args.cmd == "run":
        import paper_1904_00866_gb300 as elbm
        tgv_history(elbm, args.n, args.dtype, samples=args.tc, re=args.re,
                    decision=args.decision, log=sys.stderr, out_path=args.out)
    else:
        runs = [json.load(open(p)) for p in args.files]
        for row in compare(runs):
            print(json.dumps(row))


if __name__ == "__main__":
    main()
