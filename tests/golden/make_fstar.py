"""Writes the certified optimum of a synthetic configuration, computed by the
FP64 oracle only (no GPU code is imported):

    python tests/golden/make_fstar.py c1|c2            (iterative certification)
    python tests/golden/make_fstar.py c2 --exact       (exact KKT solve, below)
    python tests/golden/make_fstar.py c2 --theta-tol   (Theta tolerance, below)

The oracle's solver (Algorithm 3) runs in chunks of Newton iterations, each
chunk warm-started from the previous iterate (the first chunk is the plain
two-stage start from Theta = 1/N, the following ones run stage 2 with up to
250 CG products per Newton step; the optimum of the strictly convex problem
does not depend on the path).  After
each chunk the Frank-Wolfe duality gap of the iterate bounds f - f* from
above (convexity, see orc_fw_gap); the run stops once that bound is below
1e-11 * f, so f* is known to 1e-11 relative without trusting the solver,
or once f changes by less than 1e-14 (relative) over a chunk with the KKT
residual below 1e-11 (double-precision stagnation; the FW bound is then
limited by rounding in G and is reported as it stands).

Output tests/golden/fstar_<cfg>.json: f_star (the final objective, an upper
bound), f_lower (f - FW gap, a lower bound), the KKT residual, iteration
counts, sampled rows of Theta* and the change of those rows over the last
chunk (theta_drift), and theta_tol: 10 x the largest difference, on the
sampled rows, between Theta* and the oracle's iterate at KKT <= 1e-10 (a
separate run from Theta = 1/N, the calibration of the Theta tolerance:
Theta is poorly determined along the flat directions of the objective)."""
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
REL = 1e-11


def write(name, w, out):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"fstar_{name}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    return path


def main(name: str, chunk: int = 100, max_chunks: int = 400, cont_cg: int = 250) -> None:
    w = CONFIGS[name]()
    pr = oracle.Problem.from_workload(w)
    t0 = time.time()
    th, rep, hist = pr.fit(w.P, eps_kkt=0.0, max_newton=chunk)
    totals = {k: rep[k] for k in ("iters_s1", "iters_s2", "cg_total", "ls_total")}
    head = [float(x) for x in hist[:40]]
    prev = th.copy()
    rng = np.random.default_rng(workloads.BASE_SEED)
    rows = np.unique(np.concatenate([[0, 1, w.M // 2, w.M - 1],
                                     rng.choice(w.M, size=min(w.M, 60), replace=False)]))
    f_prev = np.inf
    for c in range(max_chunks):
        f, G = pr.gradient(w.P, th)
        gap = pr.fw_gap(th, G)
        kkt = pr.kkt(th, G)
        drift = float(np.abs(th[rows] - prev[rows]).max())
        print(f"{name} chunk {c}: f={f:.16e} fw_gap={gap:.3e} rel={gap / f:.3e} kkt={kkt:.3e} "
              f"iters={totals['iters_s1']}+{totals['iters_s2']} cg={totals['cg_total']} "
              f"drift={drift:.2e} t={time.time() - t0:.0f}s", flush=True)
        if gap <= REL * f:
            break
        if f_prev - f <= 1e-14 * f and kkt <= 1e-11:
            break
        f_prev = f
        prev = th.copy()
        # provisional record after every chunk (status "provisional" until a
        # stopping rule holds)
        write(name, w, {"config": w.name, "status": "provisional", "f_star": float(f),
                        "f_lower": float(f - gap), "fw_gap": float(gap), "kkt": float(kkt),
                        "iters_s1": totals["iters_s1"], "iters_s2": totals["iters_s2"],
                        "seconds": time.time() - t0,
                        "sample_rows": [int(r) for r in rows],
                        "theta_rows": [[float(v) for v in th[r]] for r in rows]})
        # continuation chunks: stage 2 (Algorithm 1) with longer CG solves
        th, rep, _ = pr.fit(w.P, Theta0=th, eps_kkt=0.0, max_newton=chunk, start_stage=2,
                            max_cg=cont_cg)
        for k in totals:
            totals[k] += rep[k]
        if rep["status"] == 3 and rep["iters_s2"] < 2:
            # the solver cannot decrease f any further in double precision
            f, G = pr.gradient(w.P, th)
            gap = pr.fw_gap(th, G)
            kkt = pr.kkt(th, G)
            print(f"{name}: stagnated at f={f:.16e} fw_gap={gap:.3e}", flush=True)
            break
    th10, rep10, _ = pr.fit(w.P, eps_kkt=1e-10, max_newton=100000)
    theta_tol = float(max(10.0 * np.abs(th10[rows] - th[rows]).max(), 1e-9))
    print(f"{name}: eps 1e-10 run: f={rep10['f']:.16e} kkt={rep10['kkt']:.3e} "
          f"theta_tol={theta_tol:.3e}", flush=True)
    out = {
        "config": w.name,
        "status": "certified",
        "generator": f"workloads.config_{name}()",
        "oracle": "oracle.Problem.fit (FP64, Algorithm 3, then warm-started stage-2 chunks)",
        "f_star": float(f),
        "f_lower": float(f - gap),
        "fw_gap": float(gap),
        "kkt": float(kkt),
        "iters_s1": totals["iters_s1"],
        "iters_s2": totals["iters_s2"],
        "cg_total": totals["cg_total"],
        "ls_total": totals["ls_total"],
        "seconds": time.time() - t0,
        "threads": oracle.num_threads(),
        "rowsum_maxerr": float(np.abs(th.sum(1) - 1).max()),
        "f_history_head": head,
        "sample_rows": [int(r) for r in rows],
        "theta_rows": [[float(v) for v in th[r]] for r in rows],
        "theta_drift": drift,
        "theta_tol": theta_tol,
        "f_eps1e-10": float(rep10["f"]),
    }
    print("wrote", write(name, w, out))


def main_exact(name: str, seed_iters: int = 100) -> None:
    """Certification by the exact KKT solve (oracle.exact_qp): the oracle's
    solver runs `seed_iters` Newton iterations (Algorithm 3) to provide a
    support, then the active-set KKT solve finishes exactly; f* is certified
    by the primal and dual violations of the final support."""
    from oracle import exact_qp
    w = CONFIGS[name]()
    pr = oracle.Problem.from_workload(w)
    t0 = time.time()
    th_it, rep, hist = pr.fit(w.P, eps_kkt=0.0, max_newton=seed_iters)
    print(f"{name}: seed solve f={rep['f']:.16e} kkt={rep['kkt']:.3e} t={time.time() - t0:.0f}s", flush=True)
    th, nu, info = exact_qp.exact_optimum(pr.dense_F(), w.P, w.gamma, th_it,
                                          log=lambda m: print(name, m, f"t={time.time() - t0:.0f}s", flush=True))
    f, G = pr.gradient(w.P, th)
    kkt = pr.kkt(th, G)
    gap = pr.fw_gap(th, G)
    print(f"{name}: exact f*={f:.16e} kkt={kkt:.3e} fw_gap={gap:.3e} {info}", flush=True)
    rng = np.random.default_rng(workloads.BASE_SEED)
    rows = np.unique(np.concatenate([[0, 1, w.M // 2, w.M - 1],
                                     rng.choice(w.M, size=min(w.M, 60), replace=False)]))
    out = {
        "config": w.name,
        "status": "certified" if info["converged"] else "provisional",
        "generator": f"workloads.config_{name}()",
        "oracle": "oracle.exact_qp.exact_optimum (active-set KKT solve) seeded by oracle.Problem.fit",
        "f_star": float(f),
        "f_lower": float(f - gap),
        "fw_gap": float(gap),
        "kkt": float(kkt),
        "kkt_primal_violation": info["primal_violation"],
        "kkt_dual_violation_rel": info["dual_violation"],
        "active_set_iterations": info["iterations"],
        "support": info["support"],
        "seed_iters": seed_iters,
        "seed_f": float(rep["f"]),
        "seconds": time.time() - t0,
        "threads": oracle.num_threads(),
        "rowsum_maxerr": float(np.abs(th.sum(1) - 1).max()),
        "f_history_head": [float(x) for x in hist[:40]],
        "sample_rows": [int(r) for r in rows],
        "theta_rows": [[float(v) for v in th[r]] for r in rows],
    }
    print("wrote", write(name, w, out))


def main_theta_tol(name: str) -> None:
    """Calibration of the Theta tolerance on the oracle: the oracle's solver
    (Algorithm 3 from Theta = 1/N, default options) runs until its objective
    is within the benchmark tolerance of the stored f* (f <= f* (1 + 0.5e-8),
    checked by the solver with f_target); theta_tol = 10 x the largest
    difference, on the stored sample rows, between that iterate and Theta*.
    Theta is poorly determined along the flat directions of the objective,
    so any solver that stops at this gap may differ from Theta* by that much.
    Adds theta_tol (and the run's counts) to tests/golden/fstar_<cfg>.json."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"fstar_{name}.json")
    with open(path) as fh:
        gold = json.load(fh)
    w = CONFIGS[name]()
    pr = oracle.Problem.from_workload(w)
    t0 = time.time()
    th, rep, _ = pr.fit(w.P, eps_kkt=0.0, max_newton=100000, f_target=gold["f_star"] * (1 + 0.5e-8))
    rows = np.array(gold["sample_rows"])
    diff = np.abs(th[rows] - np.array(gold["theta_rows"]))
    f = pr.objective(w.P, th)
    gold.update({
        "theta_tol": float(max(10.0 * diff.max(), 1e-9)),
        "theta_tol_run": {"f": float(f), "rel_gap": float((f - gold["f_star"]) / gold["f_star"]),
                          "iters_s1": int(rep["iters_s1"]), "iters_s2": int(rep["iters_s2"]),
                          "cg_total": int(rep["cg_total"]), "ls_total": int(rep["ls_total"]),
                          "seconds": time.time() - t0, "threads": oracle.num_threads(),
                          "max_diff": float(diff.max()),
                          "max_diff_row": int(rows[int(np.argmax(diff.max(1)))])},
    })
    print(json.dumps(gold["theta_tol_run"]), "theta_tol", gold["theta_tol"], flush=True)
    with open(path, "w") as fh:
        json.dump(gold, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    if len(sys.argv) > 2 and sys.argv[2] == "--exact":
        main_exact(sys.argv[1])
    elif len(sys.argv) > 2 and sys.argv[2] == "--theta-tol":
        main_theta_tol(sys.argv[1])
    else:
        main(sys.argv[1])
