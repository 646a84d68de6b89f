"""The pins must catch plausible mistakes in the oracle.  Each case copies
oracle/tomo_oracle.c to a temporary directory, plants one mistake there by a
textual substitution (a dropped term, a wrong sign or index, a transposed
operand, a wrong constant), builds the copy and checks that at least one of
the independent checks below fails.  The committed oracle is never modified."""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest
from scipy.stats import poisson

import oracle
import workloads

SRC = os.path.join(os.path.dirname(oracle.__file__), "tomo_oracle.c")

MUTANTS = {
    "dropped_regulariser_gradient": ("        Y[i * N + n] += g2 * lx;", "        Y[i * N + n] += 0.0 * lx;"),
    "laplacian_wrong_neighbour": ("if (i > 0) lx += X[i * N + n] - X[(i - 1) * N + n];",
                                  "if (i > 0) lx += X[i * N + n] - X[(i + 1 < M ? i + 1 : i) * N + n];"),
    "gradient_missing_factor_2": ("for (int64_t k = 0; k < MN; ++k) G[k] *= 2.0;",
                                  "for (int64_t k = 0; k < MN; ++k) G[k] *= 1.0;"),
    "residual_sign": ("        O[k] -= P[k];", "        O[k] = P[k] + O[k];"),
    "poisson_off_by_one": ("lgammal((long double)i + 1.0L)", "lgammal((long double)i)"),
    "adjoint_transposed_index": ("            const double f = Fval(p, d, i);\n            const double *restrict y = Y + d * N;",
                                 "            const double f = Fval(p, d, i < p->M - 1 ? i + 1 : i);\n            const double *restrict y = Y + d * N;"),
    "projection_threshold": ("        double t = (cum - 1.0) / (double)(k + 1);", "        double t = (cum - 1.0) / (double)(k + 2);"),
    "stage2_reduced_gradient_sign": ("                    w->g[k] = w->G[k] - gm;", "                    w->g[k] = gm - w->G[k];"),
    "armijo_sign": ("        if (ft <= f + o->c * gts) {", "        if (ft <= f - o->c * gts) {"),
    "kkt_multiplier": ("        double lam = -mn > 0.0 ? -mn : 0.0;", "        double lam = mn > 0.0 ? mn : 0.0;"),
    "hess_diag_missing_square": ("            s += f * f;", "            s += f;"),
}


def build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"pattern of {name} not found"
    src = src.replace(old, new)  # every occurrence (full and sampled-row variants)
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-ffp-contract=off", "-o", str(so), str(c), "-lm"])
    return str(so)


class MutantOracle(oracle.Problem):
    """oracle.Problem bound to another build of the C file."""

    def __init__(self, L, *a, **kw):
        self._L = L
        saved = oracle._lib
        oracle._lib = L
        try:
            super().__init__(*a, **kw)
        finally:
            oracle._lib = saved


def load(so):
    saved = oracle._lib
    oracle._lib = None
    real_build = oracle.build
    oracle.build = lambda force=False: so
    try:
        L = oracle.lib()
    finally:
        oracle._lib = saved
        oracle.build = real_build
    return L


def laplacian(M):
    L = np.zeros((M, M))
    for i in range(M - 1):
        L[i, i] += 1
        L[i + 1, i + 1] += 1
        L[i, i + 1] -= 1
        L[i + 1, i] -= 1
    return L


def checks(L):
    """Independent checks; returns the list of those that fail."""
    saved = oracle._lib
    oracle._lib = L
    failed = []
    try:
        rng = np.random.default_rng(4)
        M, N, D, gamma = 12, 3, 20, 0.05
        lam = workloads.probe_intensities(D, 9.0)
        pr = oracle.Problem(M, N, lam, 0.0, gamma)
        F = np.stack([poisson.pmf(np.arange(M), l) for l in lam])
        A = 2 * (F.T @ F + gamma * laplacian(M))
        Th = workloads.random_feasible_theta(M, N, rng)
        P = rng.dirichlet(np.ones(N), D)
        V = rng.standard_normal((M, N))
        f, G = pr.gradient(P, Th)
        if not np.isclose(f, np.sum((P - F @ Th) ** 2) + gamma * np.sum(np.diff(Th, axis=0) ** 2), rtol=1e-10):
            failed.append("objective")
        if not np.allclose(G, A @ Th - 2 * F.T @ P, rtol=1e-9, atol=1e-12):
            failed.append("gradient")
        if not np.allclose(pr.hvp(V), A @ V, rtol=1e-9, atol=1e-12):
            failed.append("hvp")
        if not np.allclose(pr.hess_diag(), np.diag(A), rtol=1e-12):
            failed.append("hess_diag")
        x = rng.standard_normal(5)
        y = oracle.project_simplex(x)
        u = -np.sort(-x)
        cs = np.cumsum(u)
        rho = max(k for k in range(5) if u[k] - (cs[k] - 1) / (k + 1) > 0)
        if not np.allclose(y, np.maximum(x - (cs[rho] - 1) / (rho + 1), 0), atol=1e-14):
            failed.append("projection")
        Gh = np.array([[-1.0, -1.0, 2.0], [3.0, 4.0, 5.0]])
        ph = oracle.Problem(2, 3, np.array([1.0]), 0.0, 0.0)
        if not np.isclose(ph.kkt(np.array([[0.5, 0.5, 0.0], [1.0, 0.0, 0.0]]), Gh), np.sqrt(1.5)):
            failed.append("kkt")
        # full solve against brute force over row supports (tiny)
        Ms, Ns, Ds = 3, 3, 8
        lam2 = np.sort(rng.uniform(0, 5, Ds))
        F2 = np.stack([poisson.pmf(np.arange(Ms), l) for l in lam2])
        P2 = rng.dirichlet(np.ones(Ns), Ds)
        p2 = oracle.Problem(Ms, Ns, lam2, 0.0, gamma)
        Th2, rep, hist = p2.fit(P2, eps_kkt=1e-13)
        A2 = 2 * (F2.T @ F2 + gamma * laplacian(Ms))
        C2 = -2 * F2.T @ P2
        best = np.inf
        sups = [S for k in range(1, Ns + 1) for S in itertools.combinations(range(Ns), k)]
        for pat in itertools.product(sups, repeat=Ms):
            idx = [(i, n) for i in range(Ms) for n in pat[i]]
            nv = len(idx)
            K = np.zeros((nv + Ms, nv + Ms))
            rhs = np.zeros(nv + Ms)
            for a, (i, n) in enumerate(idx):
                for b, (j, m) in enumerate(idx):
                    if n == m:
                        K[a, b] = A2[i, j]
                K[a, nv + i] = K[nv + i, a] = 1.0
                rhs[a] = -C2[i, n]
            rhs[nv:] = 1.0
            sol = np.linalg.lstsq(K, rhs, rcond=None)[0]
            T = np.zeros((Ms, Ns))
            for a, (i, n) in enumerate(idx):
                T[i, n] = sol[a]
            if T.min() >= -1e-12:
                best = min(best, np.sum((P2 - F2 @ T) ** 2) + gamma * np.sum(np.diff(T, axis=0) ** 2))
        f_true = np.sum((P2 - F2 @ Th2) ** 2) + gamma * np.sum(np.diff(Th2, axis=0) ** 2)
        if not (abs(f_true - best) <= 1e-9 * best and abs(rep["f"] - f_true) <= 1e-9 * best
                and np.all(np.diff(hist) <= 1e-15 * hist[:-1])):
            failed.append("solve")
        if not (abs(oracle.poisson(7, 3.5) - poisson.pmf(7, 3.5)) <= 1e-13 * poisson.pmf(7, 3.5)):
            failed.append("poisson")
        # Armijo (App. B): every accepted step decreases f beyond rounding
        # (two small cases, 40 iterations with CG capped at 10 products so
        # that full steps overshoot and the rule has to reject trials; a
        # relative rise above 1e-12 is a rule violation, below it rounding)
        for w in (workloads.small_case(seed=101),
                  workloads.small_case(M=40, bins=5, D=60, X=30.0, seed=102)):
            pc = oracle.Problem.from_workload(w)
            _, _, hc = pc.fit(w.P, max_newton=40, eps_kkt=0.0, max_cg=10)
            if np.max(np.diff(hc) / hc[:-1]) > 1e-12:
                failed.append("monotone")
                break
    finally:
        oracle._lib = saved
    return failed


def test_unmutated_oracle_passes_the_checks():
    assert checks(oracle.lib()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    L = load(build_mutant(tmp_path, name))
    assert checks(L), f"mutation {name} was not detected"
