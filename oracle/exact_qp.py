"""Exact optimum of the tomography QP from its KKT conditions (test
infrastructure, like the rest of the oracle).

With A = 2 (F^T F + gamma L) and C = -2 F^T P, the objective of Eq. min +
Eq. regul is f(Theta) = 1/2 sum_n theta_n^T A theta_n + sum_n c_n^T theta_n +
||P||^2 (theta_n = column n of Theta).  It is strictly convex on the row
simplices, and Theta is optimal iff, with multipliers nu_i of the row sums,
    A theta_n + c_n + nu = 0        on the support S_n of column n,
    A theta_n + c_n + nu >= 0       off the support,   theta >= 0,
    sum_n theta_{i,n} = 1.
For a given support the first and last conditions are a linear system:
theta_n[S_n] = -A_n^{-1} (c_n + nu)[S_n] with A_n = A[S_n, S_n], and
    K nu = -1 - sum_n P_n^T A_n^{-1} c_n[S_n],   K = sum_n P_n^T A_n^{-1} P_n
(P_n selects S_n), solved by dense Cholesky factorisations (scipy).  The
support is then corrected (entries with theta < 0 leave it, entries whose
reduced gradient is negative join it) until both inequalities hold.
Seeded with the support of an iterate of the oracle's solver, this reaches
the optimum in a few corrections; the result is certified by its KKT
violations, not by trusting any iteration."""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def laplacian(M: int) -> np.ndarray:
    L = np.zeros((M, M))
    idx = np.arange(M - 1)
    L[idx, idx] += 1.0
    L[idx + 1, idx + 1] += 1.0
    L[idx, idx + 1] -= 1.0
    L[idx + 1, idx] -= 1.0
    return L


def solve_support(A, C, S):
    """Theta and nu for a fixed support S (bool M x N, every row non-empty)."""
    M, N = C.shape
    K = np.zeros((M, M))
    r = -np.ones(M)
    facs = []
    for n in range(N):
        idx = np.flatnonzero(S[:, n])
        if idx.size == 0:
            facs.append(None)
            continue
        cf = sla.cho_factor(A[np.ix_(idx, idx)], lower=True, check_finite=False)
        inv = sla.cho_solve(cf, np.eye(idx.size), check_finite=False)
        K[np.ix_(idx, idx)] += inv
        r[idx] -= sla.cho_solve(cf, C[idx, n], check_finite=False)
        facs.append((idx, cf))
    nu = sla.solve(K, r, assume_a="pos", check_finite=False)
    Th = np.zeros((M, N))
    for n, fc in enumerate(facs):
        if fc is None:
            continue
        idx, cf = fc
        Th[idx, n] = -sla.cho_solve(cf, C[idx, n] + nu[idx], check_finite=False)
    return Th, nu


def exact_optimum(F, P, gamma, Theta_seed, seed_threshold=1e-10, max_iter=60, tol=1e-12,
                  dual_tol=1e-9, log=None):
    """Active-set KKT solve.  Stops when the primal violation (most negative
    theta on the support) is <= tol and the dual violation (most negative
    reduced gradient off the support, relative to max |C|) is <= dual_tol --
    the support then only changes by entries at the rounding level of the
    dense solves -- or after max_iter corrections.  Returns (Theta, nu, info)
    with the violations of the best support seen and whether the stopping
    rule held."""
    M = F.shape[1]
    A = 2.0 * (F.T @ F) + 2.0 * gamma * laplacian(M)
    C = -2.0 * (F.T @ P)
    S = Theta_seed > seed_threshold
    empty = ~S.any(axis=1)
    S[empty, np.argmax(Theta_seed[empty], axis=1)] = True
    scale = np.abs(C).max()
    best = None
    for it in range(max_iter):
        Th, nu = solve_support(A, C, S)
        G = A @ Th + C + nu[:, None]          # reduced gradient
        primal = max(-Th[S].min(), 0.0) if S.any() else 0.0
        dual = max(-(G[~S]).min(), 0.0) / scale if (~S).any() else 0.0
        if log:
            log(f"active set {it}: |S|={int(S.sum())} primal viol={primal:.3e} "
                f"dual viol={dual:.3e}")
        info = {"iterations": it + 1, "primal_violation": float(primal),
                "dual_violation": float(dual), "support": int(S.sum())}
        if best is None or max(primal, dual) < max(best[2]["primal_violation"], best[2]["dual_violation"]):
            best = (np.maximum(Th, 0.0), nu, dict(info))
        if primal <= tol and dual <= dual_tol:
            info["converged"] = True
            return np.maximum(Th, 0.0), nu, info
        drop = S & (Th < -tol)
        add = (~S) & (G < -dual_tol * scale)
        S = (S & ~drop) | add
        empty = ~S.any(axis=1)
        if empty.any():
            S[empty, np.argmax(Th[empty], axis=1)] = True
    Th, nu, info = best
    info["converged"] = False
    return Th, nu, info
