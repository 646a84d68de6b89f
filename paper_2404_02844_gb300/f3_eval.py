"""Solve times on the Liu-shaped near-dense geometry (Sec. Application to
other detector geometries; M ~ 6.6 N^1.06, D ~ 4.0 N^1.14; a synthetic
multiplexed-detector stand-in for the unavailable input generator):

    python -m paper_2404_02844_gb300.f3_eval [--n 30 100 300 1000] [--precision tc]

For each N: one full solve from Theta^(0) = 1/N to eps_KKT (default 1e-8) and
the device memory the plan holds; one JSON line.  The paper's CPU solver
needed 1450 s and 1.6 GiB at N = 1000 on its own (different) data.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[30, 100, 300, 1000])
    ap.add_argument("--precision", default="tc", choices=["tc", "fp32", "mixed", "fp64"])
    ap.add_argument("--eps-kkt", type=float, default=1e-8)
    ap.add_argument("--max-newton", type=int, default=500)
    args = ap.parse_args()

    import torch

    import paper_2404_02844_gb300 as tomo
    import workloads as W
    from paper_2404_02844_gb300 import build

    build.build()
    rows = []
    for N in args.n:
        t0 = time.perf_counter()
        w = W.config_f3(N)
        t_data = time.perf_counter() - t0
        P = torch.from_numpy(w.P).cuda()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        with tomo.Plan.from_workload(w, precision=args.precision) as pl:
            torch.cuda.synchronize()
            plan_bytes = free0 - torch.cuda.mem_get_info()[0]
            pl.fit(P, max_newton=2)        # configure kernels and capture the CG graphs
            torch.cuda.synchronize()
            t = time.perf_counter()
            Th, rep = pl.fit(P, eps_kkt=args.eps_kkt, max_newton=args.max_newton)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
        rows.append({"N": N, "M": w.M, "D": w.D, "free_variables": w.M * w.N, "seconds": dt,
                     "newton_iters": rep["iters_s1"] + rep["iters_s2"], "cg_total": rep["cg_total"],
                     "kkt": rep["kkt"], "stop": rep["stop_name"], "f": rep["f"],
                     "plan_device_bytes": int(plan_bytes), "data_s": t_data})
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"workload": "Liu-shaped (synthetic multiplexed detector, eta 0.9, 1e6 shots, gamma 1e-4)",
                      "precision": args.precision, "eps_kkt": args.eps_kkt, "rows": rows}), flush=True)


if __name__ == "__main__":
    main()
