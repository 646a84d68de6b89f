"""Writes the oracle's optima of one large instance of the batched
distribution (configs c4: M ~ U{256..8192}, N ~ U{8..128}) at the four
regularisation weights, computed by the FP64 oracle only (no GPU code is
imported):

    python tests/golden/make_fstar_c4.py [instance] [--max-newton K] [--gammas g1,g2,..]

Instance 178 of workloads.config_c4() is the largest of the distribution's
first 256 (M = 8063, N = 127, D = 16126).  For each gamma the oracle's solver
(Algorithm 3 from Theta = 1/N) runs to eps_KKT = 1e-11 or K Newton
iterations; the Frank-Wolfe gap of the result (orc_fw_gap, an upper bound of
f - f* by convexity) is recorded beside f, and a gamma counts as converged
when the oracle stopped on its KKT test.  Output:
tests/golden/fstar_c4_<instance>.json."""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle      # noqa: E402
import workloads   # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("instance", type=int, nargs="?", default=178)
    ap.add_argument("--max-newton", type=int, default=3000)
    ap.add_argument("--max-cg", type=int, default=10000)
    ap.add_argument("--gammas", default=",".join(str(g) for g in workloads.C4_GAMMAS))
    args = ap.parse_args()
    j = args.instance
    w = workloads.config_c4_instance(j)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"fstar_c4_{j}.json")
    out = {"config": w.name, "instance": j, "generator": f"workloads.config_c4_instance({j})",
           "M": w.M, "N": w.N, "D": w.D, "threads": oracle.num_threads(), "results": {}}
    if os.path.exists(path):
        with open(path) as fh:
            out["results"] = json.load(fh).get("results", {})
    for g in [float(x) for x in args.gammas.split(",")]:
        pr = oracle.Problem(w.M, w.N, w.lam, w.band_k, g)
        t0 = time.time()
        th, rep, hist = pr.fit(w.P, eps_kkt=1e-11, max_newton=args.max_newton, max_cg=args.max_cg)
        f, G = pr.gradient(w.P, th)
        gap = pr.fw_gap(th, G)
        res = {"gamma": g, "f": float(f), "fw_gap": float(gap), "kkt": float(rep["kkt"]),
               "status": int(rep["status"]), "converged": int(rep["status"]) == 0,
               "iters_s1": int(rep["iters_s1"]), "iters_s2": int(rep["iters_s2"]),
               "cg_total": int(rep["cg_total"]), "seconds": time.time() - t0,
               "max_cg": args.max_cg}
        print(json.dumps(res), flush=True)
        out["results"][repr(g)] = res
        with open(path, "w") as fh:
            json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
