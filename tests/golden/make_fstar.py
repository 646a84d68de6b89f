"""Writes the certified optimum of a synthetic configuration, computed by the
FP64 oracle only (no GPU code is imported):

    python tests/golden/make_fstar.py c1|c2

Output: tests/golden/fstar_<cfg>.json with f*, the KKT residual, iteration
counts, a Theta tolerance calibrated from two oracle runs (eps_KKT 1e-10 and
1e-12, difference x 10), and sampled rows of Theta* for parity checks."""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle      # noqa: E402
import workloads   # noqa: E402

CONFIGS = {"c1": workloads.config_c1, "c2": workloads.config_c2}


def main(name: str) -> None:
    w = CONFIGS[name]()
    pr = oracle.Problem.from_workload(w)
    t0 = time.time()
    th_lo, rep_lo, h_lo = pr.fit(w.P, eps_kkt=1e-10, max_newton=5000)
    t_lo = time.time() - t0
    print(name, "eps 1e-10:", rep_lo, f"{t_lo:.1f}s", flush=True)
    t0 = time.time()
    th, rep, hist = pr.fit(w.P, eps_kkt=1e-12, max_newton=5000)
    t_hi = time.time() - t0
    print(name, "eps 1e-12:", rep, f"{t_hi:.1f}s", flush=True)
    diff = np.abs(th - th_lo)
    rng = np.random.default_rng(workloads.BASE_SEED)
    rows = np.unique(np.concatenate([[0, 1, w.M // 2, w.M - 1],
                                     rng.choice(w.M, size=min(w.M, 60), replace=False)]))
    out = {
        "config": w.name,
        "generator": f"workloads.config_{name}()",
        "oracle": "oracle.Problem.fit, FP64, Algorithm 3",
        "f_star": rep["f"],
        "kkt": rep["kkt"],
        "status": rep["status"],
        "iters_s1": rep["iters_s1"],
        "iters_s2": rep["iters_s2"],
        "cg_total": rep["cg_total"],
        "ls_total": rep["ls_total"],
        "seconds": t_hi,
        "threads": oracle.num_threads(),
        "f_eps1e-10": rep_lo["f"],
        "theta_maxdiff_eps1e-10_vs_1e-12": float(diff.max()),
        "theta_tol": float(max(10 * diff.max(), 1e-9)),
        "rowsum_maxerr": float(np.abs(th.sum(1) - 1).max()),
        "f_history_head": [float(x) for x in hist[:40]],
        "sample_rows": [int(r) for r in rows],
        "theta_rows": [[float(v) for v in th[r]] for r in rows],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"fstar_{name}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main(sys.argv[1])
