"""Training and evaluation of the learned warm start on the detector
population of `workloads.config_c5_instance` (M = 1024 photon numbers,
D = 2048 probes with lambda linear in [0, 768], up to 64 outcomes, gamma 1e-3):

    python -m paper_2404_02844_gb300.warmstart_eval [--train 2000] [--steps 3000]
        [--test 16] [--precision fp32] [--save weights.bin]

Trains on `--train` instances whose targets are either the solver's own
optima (`--labels solver`, the default: every training instance is solved by
the batched solver to KKT 1e-8 first) or the simulator's true POVMs
(`--labels true`), then solves `--test` held-out instances three times: a
reference solve (KKT 1e-11) that fixes f_ref, and one solve from Theta^(0) =
1/N and one from the network's Theta0 (tomo_fit_warm, with its fallback),
both timed until f <= f_ref (1 + 1e-8).  Prints one JSON line: label
statistics, training and held-out loss, Newton iterations and solve time per
start, and how often the warm start won.
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
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--test", type=int, default=16)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tc", "fp64", "mixed"])
    ap.add_argument("--eps-kkt", type=float, default=1e-9)
    ap.add_argument("--labels", default="solver", choices=["solver", "true"])
    ap.add_argument("--label-precision", default="tc", choices=["fp32", "tc", "fp64", "mixed"])
    ap.add_argument("--concurrency", type=int, default=8)
    ap.add_argument("--fit-seconds", type=float, default=60.0, help="wall-clock bound of every evaluation fit")
    ap.add_argument("--label-newton", type=int, default=1000, help="Newton cap of the label solves")
    ap.add_argument("--save", default=None)
    ap.add_argument("--load", default=None, help="parameter file: skip the labels and the training")
    ap.add_argument("--zero-below", default="0",
                    help="comma-separated sparsification thresholds of Theta0 to compare")
    args = ap.parse_args()

    import torch

    import paper_2404_02844_gb300 as tomo
    import workloads as W
    from paper_2404_02844_gb300 import build

    build.build()
    lam = W.probe_intensities(W.C5_D, W.C5_X)
    F = W.dense_poisson(W.C5_M, lam)
    t0 = time.perf_counter()
    Ptr, Ttr, nctr, wtr = W.c5_batch(range(args.train), F=F)
    Pte, Tte, ncte, wte = W.c5_batch(range(100000, 100000 + args.test), F=F)
    t_data = time.perf_counter() - t0
    Ptr_d = torch.from_numpy(Ptr).cuda()
    Ttr_d = torch.from_numpy(Ttr).cuda()
    label_info = {"labels": args.labels if not args.load else f"loaded {args.load}"}
    if args.labels == "solver" and not args.load:
        # targets = the solver's optima of the training instances (batched)
        t0 = time.perf_counter()
        problems, outs = [], []
        for b, w in enumerate(wtr):
            P = Ptr_d[b, :, :w.N].contiguous()
            Th = torch.empty(w.M, w.N, dtype=torch.float64, device="cuda")
            problems.append((w.M, w.N, w.lam, w.band_k, w.gamma, P, Th))
            outs.append(Th)
        sts, reps = tomo.fit_batched(problems, precision=args.label_precision,
                                     concurrency=args.concurrency, eps_kkt=1e-8,
                                     max_newton=args.label_newton, max_seconds=args.fit_seconds)
        torch.cuda.synchronize()
        for b, w in enumerate(wtr):
            Ttr_d[b].zero_()
            Ttr_d[b, :, :w.N] = outs[b]
        t_lab = time.perf_counter() - t0
        kk = np.array([r["kkt"] for r in reps])
        print(json.dumps({"labels_done_s": t_lab}), flush=True)
        label_info.update({"label_s": t_lab, "label_precision": args.label_precision,
                           "label_solves_per_s": len(wtr) / t_lab,
                           "label_status_ok": int(sum(st in (0, 4) for st in sts)),
                           "label_kkt_median": float(np.median(kk)), "label_kkt_max": float(kk.max()),
                           "label_newton_mean": float(np.mean([r["iters_s1"] + r["iters_s2"] for r in reps])),
                           "label_vs_true_maxdiff_median": float(np.median(
                               [np.abs(outs[b].cpu().numpy() - w.theta_true).max() for b, w in enumerate(wtr[:64])]))})
        # held-out targets stay the true POVMs (loss only)
    ws = tomo.WarmStart(W.C5_D, W.C5_C0, W.C5_M, max_batch=args.batch, seed=1)
    rng = np.random.default_rng(0)
    Pte_d = torch.from_numpy(Pte[:args.batch]).cuda()
    Tte_d = torch.from_numpy(Tte[:args.batch]).cuda()
    l_test0, _ = ws.loss_grad(Pte_d, Tte_d, ncte[:args.batch])
    losses, t_train = [float("nan")], 0.0
    if args.load:
        ws.load(args.load)
    else:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        losses = []
        for s in range(args.steps):
            idx = torch.from_numpy(rng.choice(args.train, args.batch, replace=False)).cuda()
            losses.append(ws.train_step(Ptr_d[idx].contiguous(), Ttr_d[idx].contiguous(),
                                        nctr[idx.cpu().numpy()], lr=args.lr))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
    l_test1, _ = ws.loss_grad(Pte_d, Tte_d, ncte[:args.batch])
    if args.save:
        ws.save(args.save)

    zbs = [float(z) for z in args.zero_below.split(",")]
    rows = []
    for w in wte:
        with tomo.Plan.from_workload(w, precision=args.precision) as pl:
            P = torch.from_numpy(w.P).cuda()
            _, rref = pl.fit(P, eps_kkt=1e-10, max_newton=3000,
                             max_seconds=args.fit_seconds)   # f_ref (also warms the graphs)
            target = rref["f"] * (1.0 + 1e-8)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Thc, rc = pl.fit(P, f_target=target, eps_kkt=0.0, max_newton=3000, max_seconds=args.fit_seconds)
            torch.cuda.synchronize()
            tc = time.perf_counter() - t0
            fc = pl.objective(P, Thc)
            uni = torch.full((w.M, w.N), 1.0 / w.N, dtype=torch.float64, device="cuda")
            f0w, f0u = pl.objective(P, ws.infer(P)), pl.objective(P, uni)
            row = dict(N=w.N, cold_iters=rc["iters_s1"] + rc["iters_s2"], cold_s=tc,
                       cold_stop=rc["stop_name"], rel_gap_cold=(fc - rref["f"]) / rref["f"],
                       f0_warm_over_uniform=f0w / f0u, warm={})
            for zb in zbs:
                t0 = time.perf_counter()
                Thw, rw, used = tomo.fit_warm(pl, ws, P, zero_below=zb, f_target=target, eps_kkt=0.0,
                                              max_newton=3000, max_seconds=args.fit_seconds)
                torch.cuda.synchronize()
                tw = time.perf_counter() - t0
                fw = pl.objective(P, Thw)
                row["warm"][repr(zb)] = dict(iters=rw["iters_s1"] + rw["iters_s2"], s=tw, stop=rw["stop_name"],
                                             used_warm=bool(used), rel_gap=(fw - rref["f"]) / rref["f"])
        rows.append(row)
        print(json.dumps({"test": len(rows), **row}), flush=True)
    ci = np.array([r["cold_iters"] for r in rows])
    cs = np.array([r["cold_s"] for r in rows])
    warm = {}
    for zb in zbs:
        k = repr(zb)
        wi = np.array([r["warm"][k]["iters"] for r in rows])
        wsec = np.array([r["warm"][k]["s"] for r in rows])
        warm[k] = {"iters_mean": float(wi.mean()), "s_mean": float(wsec.mean()),
                   "s_median": float(np.median(wsec)), "s_total": float(wsec.sum()),
                   "faster_fraction": float(np.mean(wsec < cs)),
                   "used_warm": int(sum(r["warm"][k]["used_warm"] for r in rows)),
                   "max_rel_gap": float(max(r["warm"][k]["rel_gap"] for r in rows))}
    out = {
        "workload": "warm-start population: M=1024 D=2048 lambda lin [0,768], bins U{16..63}, "
                    "eta U[0.3,0.95], crosstalk U[0,1e-2], dark U[0,1e-3], 1e6 shots, gamma 1e-3",
        "params": ws.param_count, "train_instances": args.train, "steps": args.steps,
        "batch": args.batch, "lr": args.lr, "data_s": t_data, "train_s": t_train,
        "loss_first": losses[0], "loss_last_100": float(np.mean(losses[-100:])),
        "heldout_loss_before": l_test0, "heldout_loss_after": l_test1,
        "precision": args.precision, "test_instances": args.test,
        "cold_iters_mean": float(ci.mean()), "cold_s_mean": float(cs.mean()),
        "cold_s_median": float(np.median(cs)), "cold_s_total": float(cs.sum()),
        "max_rel_gap_cold": float(max(r["rel_gap_cold"] for r in rows)),
        "warm_by_zero_below": warm,
        **label_info,
        "f0_warm_over_uniform_median": float(np.median([r["f0_warm_over_uniform"] for r in rows])),
        "rows": rows,
    }
    print(json.dumps(out), flush=True)
    ws.close()


if __name__ == "__main__":
    main()
