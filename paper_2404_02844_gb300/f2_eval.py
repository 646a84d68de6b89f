"""The paper's reconstruction experiment on synthetic data: the loop
detector (R = 0.91644, eta_loop = 0.90524, eta_det = 0.528, 150 bins), probes
lambda_d = d^2, 5e5 trials per probe, reconstructed three ways (Fig.
results): (a) no regularisation, (b) gamma = 1e-5, (c) gamma = 1e-5 and the
long-range smoothing with a stage-2 refit; prints one JSON line with each
variant's solve time, Newton iterations, objective and infidelities (Eq.
fidelities) against the analytic POVM, with their mean and minimum over the
outcomes the probes cover (frequency >= 5 % for some probe).

    python -m paper_2404_02844_gb300.f2_eval [--m 100000] [--d 316] [--precision fp32]

The defaults are a scaled copy of the paper's geometry (D ~ sqrt(M));
--m 1210581 --d 1076 is the paper's size.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=100000)
    ap.add_argument("--d", type=int, default=316)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tc", "mixed", "fp64"])
    ap.add_argument("--eps-kkt", type=float, default=1e-9)
    ap.add_argument("--max-newton", type=int, default=600)
    ap.add_argument("--outcomes", type=int, default=50, help="report the first this many outcomes")
    ap.add_argument("--max-seconds", type=float, default=0.0,
                    help="> 0: wall-clock bound of every fit (the variant reports where it stopped)")
    ap.add_argument("--variants", default="a,b,c")
    args = ap.parse_args()

    import torch

    import paper_2404_02844_gb300 as tomo
    import workloads as W
    from paper_2404_02844_gb300 import build

    build.build()
    t0 = time.perf_counter()
    w = W.config_f2(M=args.m, D=args.d, gamma=0.0)
    t_data = time.perf_counter() - t0
    P = torch.from_numpy(w.P).cuda()
    T = torch.from_numpy(w.theta_true).cuda()
    out = {"workload": f"loop detector, M={w.M} N={w.N} D={w.D}, lambda_d = d^2, 5e5 trials",
           "precision": args.precision, "data_s": t_data, "variants": {}}
    K = args.outcomes
    # outcomes the probes cover: some probe sees them with frequency >= 5 %
    covered = np.nonzero(w.P.max(0) >= 0.05)[0]
    lim = dict(max_seconds=args.max_seconds) if args.max_seconds > 0 else {}
    want = set(args.variants.split(","))
    for name, gamma, smooth in (("a_no_regularisation", 0.0, False), ("b_gamma_1e-5", 1e-5, False),
                                ("c_gamma_1e-5_long_range", 1e-5, True)):
        if name[0] not in want:
            continue
        with tomo.Plan(w.M, w.N, w.lam, w.band_k, gamma, precision=args.precision) as pl:
            torch.cuda.synchronize()
            t = time.perf_counter()
            if smooth:
                Th, r1, r2 = pl.fit_smoothed(P, exclude=100, div=50.0, eps_kkt=args.eps_kkt,
                                             max_newton=args.max_newton, **lim)
                iters = [r1["iters_s1"] + r1["iters_s2"], r2["iters_s2"]]
                stop = [r1["stop_name"], r2["stop_name"]]
                kkt = r2["kkt"]
            else:
                Th, r = pl.fit(P, eps_kkt=args.eps_kkt, max_newton=args.max_newton, **lim)
                iters, stop, kkt = [r["iters_s1"] + r["iters_s2"]], [r["stop_name"]], r["kkt"]
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            inf = pl.infidelity(Th, T)[:K]
            f = pl.objective(P, Th)
        fid = 1.0 - inf
        cov = covered[covered < K]
        out["variants"][name] = {
            "seconds": dt, "newton_iters": iters, "stop": stop, "kkt": kkt, "f": f,
            "cg_products": (r1["cg_total"] + r2["cg_total"]) if smooth else r["cg_total"],
            "covered_outcomes": int(len(cov)),
            "mean_fidelity_covered": float(np.nanmean(fid[cov])),
            "min_fidelity_covered": float(np.nanmin(fid[cov])),
            "infidelity": [float(x) for x in inf]}
        print(json.dumps({name: {k: v for k, v in out["variants"][name].items() if k != "infidelity"}}),
              flush=True)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
