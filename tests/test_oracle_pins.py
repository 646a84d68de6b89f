"""Pins of the FP64 oracle against what the paper and the mathematics fix,
never against a retyping of the oracle itself: library routines (scipy's
Poisson pmf, mpmath at 50 digits, numpy dense algebra), closed forms,
invariants, brute force on tiny inputs and an independent solver."""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy.stats import poisson

import oracle
import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# helpers: an independent dense construction of F and H with scipy / numpy
# --------------------------------------------------------------------------
def dense_F(M, lam, band_k):
    """Dense D x M matrix of Poisson pmfs (scipy), zero outside the band."""
    D = len(lam)
    F = np.zeros((D, M))
    for d, l in enumerate(lam):
        lo, hi = oracle.band(M, band_k, l)
        if hi >= lo:
            i = np.arange(lo, hi + 1)
            F[d, lo:hi + 1] = poisson.pmf(i, l)
    return F


def laplacian(M):
    L = np.zeros((M, M))
    for i in range(M - 1):
        L[i, i] += 1
        L[i + 1, i + 1] += 1
        L[i, i + 1] -= 1
        L[i + 1, i] -= 1
    return L


def small_problem(M=30, N=5, D=45, X=25.0, band_k=10.0, gamma=1e-2, seed=3):
    rng = np.random.default_rng(seed)
    lam = workloads.probe_intensities(D, X)
    pr = oracle.Problem(M, N, lam, band_k, gamma)
    return pr, lam, rng


# --------------------------------------------------------------------------
# Eq. Fmatrix: Poisson weights
# --------------------------------------------------------------------------
def test_poisson_vs_scipy():
    rng = np.random.default_rng(0)
    for _ in range(400):
        lam = float(rng.choice([rng.uniform(0, 5), rng.uniform(5, 500), rng.uniform(500, 5e4)]))
        i = int(max(0, round(lam + rng.normal() * 4 * math.sqrt(lam + 1))))
        ref = poisson.pmf(i, lam)
        got = oracle.poisson(i, lam)
        # scipy's own pmf loses ~1e-10..1e-9 relative at lambda ~ 1e4-1e5
        # (mpmath below gives the tight pin)
        assert got == pytest.approx(ref, rel=(1e-12 if lam < 500 else 5e-9), abs=1e-300), (i, lam)


def test_poisson_vs_mpmath_large():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    cases = [(0, 3.0), (1, 1e-3), (7, 2.5), (1000, 990.0), (3000, 2951.3),
             (900000, 899000.0), (999999, 9.0e5 + 17.0), (10500, 1e4),
             (42964, 43227.35665631939)]
    rng = np.random.default_rng(9)
    for _ in range(40):
        lam = float(rng.uniform(1.0, 9e5))
        cases.append((int(max(0, round(lam + rng.normal() * 5 * math.sqrt(lam)))), lam))
    for i, lam in cases:
        ref = mp.exp(i * mp.log(lam) - lam - mp.loggamma(i + 1))
        got = oracle.poisson(i, lam)
        # long double evaluation: error ~ i*ln(lam)*2^-64 relative
        tol = 1e-14 + 4 * i * math.log(max(lam, 2.0)) * 2.0 ** -64
        assert abs(got - float(ref)) <= tol * float(ref), (i, lam, got, float(ref))


def test_poisson_vacuum_and_moments():
    assert oracle.poisson(0, 0.0) == 1.0
    assert oracle.poisson(3, 0.0) == 0.0
    for lam in (0.5, 7.0, 120.0):
        M = int(lam + 30 * math.sqrt(lam) + 40)
        w = np.array([oracle.poisson(i, lam) for i in range(M)])
        assert w.sum() == pytest.approx(1.0, abs=1e-13)
        assert (np.arange(M) * w).sum() == pytest.approx(lam, rel=1e-12)


def test_band_bounds_and_tail():
    # hand values: lambda = 100, k = 10: [100-100, 100+100] = [0, 200]
    assert oracle.band(1000, 10.0, 100.0) == (0, 200)
    # lambda = 3000: sqrt = 54.772..., lo = floor(2452.2) = 2452, hi = ceil(3547.7) = 3548
    assert oracle.band(4096, 10.0, 3000.0) == (2452, 3548)
    # small lambda keeps at least [0, 16]
    assert oracle.band(4096, 10.0, 1.0) == (0, 16)
    assert oracle.band(4096, 10.0, 0.0) == (0, 16)
    # cut-off at M - 1 and dense mode
    assert oracle.band(1000, 10.0, 990.0) == (675, 999)
    assert oracle.band(64, 0.0, 30.0) == (0, 63)
    # mass outside +-10 sqrt(lambda) is negligible (scipy cdf/sf)
    for lam in (1.0, 30.0, 3000.0, 9e5):
        lo, hi = oracle.band(10 ** 7, 10.0, lam)
        out = (poisson.cdf(lo - 1, lam) if lo > 0 else 0.0) + poisson.sf(hi, lam)
        assert out < 1e-9


# --------------------------------------------------------------------------
# Products with F, objective, gradient, Hessian
# --------------------------------------------------------------------------
@pytest.mark.parametrize("band_k", [10.0, 0.0, 3.0])
def test_apply_F_and_Ft_vs_dense(band_k):
    pr, lam, rng = small_problem(band_k=band_k)
    F = dense_F(pr.M, lam, band_k)
    X = rng.standard_normal((pr.M, pr.N))
    Y = rng.standard_normal((pr.D, pr.N))
    np.testing.assert_allclose(pr.apply_F(X), F @ X, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(pr.apply_Ft(Y), F.T @ Y, rtol=1e-11, atol=1e-13)
    # adjointness <F X, Y> = <X, F^T Y>
    a = np.sum(pr.apply_F(X) * Y)
    b = np.sum(X * pr.apply_Ft(Y))
    assert a == pytest.approx(b, rel=1e-12)


def test_row_sum_invariant_and_uniform_closed_form():
    pr, lam, rng = small_problem(M=60, N=7, D=50, X=30.0)
    Th = workloads.random_feasible_theta(pr.M, pr.N, rng)
    O = pr.apply_F(Th)
    s = pr.apply_F(np.ones((pr.M, 1)).repeat(pr.N, 1))[:, 0]  # sum_i F_{d,i}
    np.testing.assert_allclose(O.sum(1), s, rtol=1e-13)
    U = pr.apply_F(np.full((pr.M, pr.N), 1.0 / pr.N))
    np.testing.assert_allclose(U, np.repeat(s[:, None] / pr.N, pr.N, 1), rtol=1e-13)


def test_regulariser_closed_form():
    pr, lam, rng = small_problem(M=40, N=3, gamma=0.37)
    slopes = np.array([0.5, -2.0, 0.0])
    X = np.arange(40)[:, None] * slopes[None, :] + 1.0
    assert pr.regulariser(X) == pytest.approx(0.37 * 39 * np.sum(slopes ** 2), rel=1e-14)
    assert pr.regulariser(np.ones((40, 3))) == 0.0


def test_objective_vs_dense_definition():
    pr, lam, rng = small_problem()
    F = dense_F(pr.M, lam, pr.band_k)
    Th = workloads.random_feasible_theta(pr.M, pr.N, rng)
    P = rng.random((pr.D, pr.N))
    ref = np.sum((P - F @ Th) ** 2) + pr.gamma * np.sum(np.diff(Th, axis=0) ** 2)
    assert pr.objective(P, Th) == pytest.approx(ref, rel=1e-12)


def test_gradient_vs_central_differences():
    pr, lam, rng = small_problem(M=20, N=4, D=30, X=15.0)
    Th = workloads.random_feasible_theta(pr.M, pr.N, rng)
    P = rng.random((pr.D, pr.N))
    _, G = pr.gradient(P, Th)
    h = 1e-3
    for _ in range(25):
        i, n = rng.integers(pr.M), rng.integers(pr.N)
        E = np.zeros_like(Th)
        E[i, n] = h
        # f is quadratic: the central difference is exact up to rounding
        fd = (pr.objective(P, Th + E) - pr.objective(P, Th - E)) / (2 * h)
        assert G[i, n] == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_gradient_vs_dense_formula():
    pr, lam, rng = small_problem()
    F = dense_F(pr.M, lam, pr.band_k)
    Th = workloads.random_feasible_theta(pr.M, pr.N, rng)
    P = rng.random((pr.D, pr.N))
    _, G = pr.gradient(P, Th)
    ref = 2 * F.T @ (F @ Th - P) + 2 * pr.gamma * laplacian(pr.M) @ Th
    np.testing.assert_allclose(G, ref, rtol=1e-10, atol=1e-12)


def test_hvp_gradient_difference_symmetry_dense():
    pr, lam, rng = small_problem()
    Th = workloads.random_feasible_theta(pr.M, pr.N, rng)
    P = rng.random((pr.D, pr.N))
    V = rng.standard_normal((pr.M, pr.N))
    U = rng.standard_normal((pr.M, pr.N))
    _, G0 = pr.gradient(P, Th)
    _, G1 = pr.gradient(P, Th + V)
    HV = pr.hvp(V)
    np.testing.assert_allclose(G1 - G0, HV, rtol=1e-8, atol=1e-10)
    assert np.sum(U * HV) == pytest.approx(np.sum(V * pr.hvp(U)), rel=1e-11)
    F = dense_F(pr.M, lam, pr.band_k)
    A = 2 * (F.T @ F + pr.gamma * laplacian(pr.M))
    np.testing.assert_allclose(HV, A @ V, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(pr.hess_diag(), np.diag(A), rtol=1e-12)


# --------------------------------------------------------------------------
# Eq. Mp1_proj: simplex projection
# --------------------------------------------------------------------------
def brute_simplex(x):
    """Projection by enumerating supports: min ||x - y|| on each face."""
    n = len(x)
    best, bestd = None, np.inf
    for k in range(1, n + 1):
        for S in itertools.combinations(range(n), k):
            S = list(S)
            y = np.zeros(n)
            tau = (x[S].sum() - 1.0) / k
            y[S] = x[S] - tau
            if np.all(y[S] >= -1e-15):
                d = np.sum((x - y) ** 2)
                if d < bestd:
                    best, bestd = y, d
    return best


def test_simplex_projection_brute_force_and_condat():
    rng = np.random.default_rng(5)
    for _ in range(300):
        n = int(rng.integers(1, 9))
        x = rng.standard_normal(n) * rng.choice([0.1, 1.0, 10.0])
        y = oracle.project_simplex(x)
        np.testing.assert_allclose(y, brute_simplex(x), atol=1e-13)
        np.testing.assert_allclose(oracle.project_simplex(x, "condat"), y, atol=1e-13)


def test_simplex_projection_properties():
    rng = np.random.default_rng(6)
    for _ in range(200):
        n = int(rng.integers(2, 200))
        x = rng.standard_normal(n)
        y = oracle.project_simplex(x)
        assert y.min() >= 0.0
        assert y.sum() == pytest.approx(1.0, abs=1e-13 * n)
        np.testing.assert_allclose(oracle.project_simplex(y), y, atol=1e-15)  # idempotent
        np.testing.assert_allclose(oracle.project_simplex(x, "condat"), y, atol=1e-13)
        # variational inequality <x - P(x), z - P(x)> <= 0 for z in the simplex
        for _ in range(5):
            z = rng.dirichlet(np.ones(n))
            assert np.dot(x - y, z - y) <= 1e-12
    # special cases
    x = np.array([0.2, 0.3, 0.5])
    np.testing.assert_allclose(oracle.project_simplex(x), x, atol=1e-16)
    np.testing.assert_allclose(oracle.project_simplex(np.full(4, 7.0)), np.full(4, 0.25))
    np.testing.assert_allclose(oracle.project_simplex(np.array([5.0, -3.0])), [1.0, 0.0])


def test_kkt_definition_on_a_hand_case():
    pr = oracle.Problem(2, 3, np.array([1.0]), 0.0, 0.0)
    Th = np.array([[0.5, 0.5, 0.0], [1.0, 0.0, 0.0]])
    G = np.array([[-1.0, -1.0, 2.0], [3.0, 4.0, 5.0]])
    # row 0: lambda = 1, Theta (G + 1) = 0; row 1: lambda = 0, term = 1 * 3
    assert pr.kkt(Th, G) == pytest.approx(math.sqrt(9.0 / 6.0), rel=1e-15)


# --------------------------------------------------------------------------
# Full solve (Algorithm 3)
# --------------------------------------------------------------------------
def brute_force_qp(F, P, gamma):
    """Exact minimiser of ||P - F T||^2 + gamma tr(T^T L T) over row simplices
    by enumerating row supports and solving each equality-constrained KKT
    system (numpy), keeping the primal and dual feasible one."""
    D, M = F.shape
    N = P.shape[1]
    A = 2 * (F.T @ F + gamma * laplacian(M))  # per-column Hessian
    C = -2 * F.T @ P                           # linear term, M x N
    supports = [S for k in range(1, N + 1) for S in itertools.combinations(range(N), k)]
    best = None
    for pattern in itertools.product(supports, repeat=M):
        idx = [(i, n) for i in range(M) for n in pattern[i]]
        nv = len(idx)
        K = np.zeros((nv + M, nv + M))
        rhs = np.zeros(nv + M)
        for a, (i, n) in enumerate(idx):
            for b, (j, m) in enumerate(idx):
                if n == m:
                    K[a, b] = A[i, j]
            K[a, nv + i] = 1.0
            K[nv + i, a] = 1.0
            rhs[a] = -C[i, n]
        rhs[nv:] = 1.0
        try:
            sol = np.linalg.solve(K, rhs)
        except np.linalg.LinAlgError:
            continue
        T = np.zeros((M, N))
        for a, (i, n) in enumerate(idx):
            T[i, n] = sol[a]
        if T.min() < -1e-12:
            continue
        g = A @ T + C          # gradient of the quadratic
        nu = sol[nv:]          # multipliers of the row sums: g + nu >= 0 off-support
        if np.all(g + nu[:, None] >= -1e-9):
            best = np.maximum(T, 0.0)
            break
    return best


def test_fw_gap_bounds_the_objective_gap():
    """Convexity: f(Theta) - f* <= FW gap for every feasible Theta, and the
    gap vanishes at the brute-force optimum."""
    rng = np.random.default_rng(8)
    M, N, D = 4, 3, 9
    lam = np.sort(rng.uniform(0.0, 6.0, D))
    P = rng.dirichlet(np.ones(N), D)
    pr = oracle.Problem(M, N, lam, 0.0, 0.05)
    T_ref = brute_force_qp(dense_F(M, lam, 0.0), P, 0.05)
    f_star = pr.objective(P, T_ref)
    _, G = pr.gradient(P, T_ref)
    assert pr.fw_gap(T_ref, G) <= 1e-10
    for _ in range(50):
        Th = workloads.random_feasible_theta(M, N, rng)
        f, G = pr.gradient(P, Th)
        gap = pr.fw_gap(Th, G)
        assert f - f_star <= gap * (1 + 1e-12) + 1e-15
        # definition on a hand case: one row, G = (1, 3), Theta = (0.5, 0.5): 2 - 1 = 1
    h = oracle.Problem(1, 2, np.array([1.0]), 0.0, 0.0)
    assert h.fw_gap(np.array([[0.5, 0.5]]), np.array([[1.0, 3.0]])) == 1.0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fit_matches_brute_force_qp(seed):
    rng = np.random.default_rng(seed)
    M, N, D = 4, 3, 9
    lam = np.sort(rng.uniform(0.0, 6.0, D))
    P = rng.dirichlet(np.ones(N), D)
    gamma = 0.05
    pr = oracle.Problem(M, N, lam, 0.0, gamma)
    F = dense_F(M, lam, 0.0)
    T_ref = brute_force_qp(F, P, gamma)
    assert T_ref is not None
    Th, rep, hist = pr.fit(P, eps_kkt=1e-13)
    f_ref = pr.objective(P, T_ref)
    assert rep["f"] == pytest.approx(f_ref, rel=1e-10)
    np.testing.assert_allclose(Th, T_ref, atol=1e-7)


def fista_simplex(F, P, gamma, iters=60000):
    """Independent solver: accelerated projected gradient (FISTA) with
    numpy's sort-based simplex projection written out here."""
    M = F.shape[1]
    N = P.shape[1]
    A = 2 * (F.T @ F + gamma * laplacian(M))
    Lc = np.linalg.eigvalsh(A).max()
    C = -2 * F.T @ P

    def proj(X):
        U = -np.sort(-X, axis=1)
        cs = np.cumsum(U, axis=1) - 1.0
        k = np.arange(1, X.shape[1] + 1)
        cond = U - cs / k > 0
        rho = cond.shape[1] - 1 - np.argmax(cond[:, ::-1], axis=1)
        tau = cs[np.arange(X.shape[0]), rho] / (rho + 1)
        return np.maximum(X - tau[:, None], 0.0)

    X = np.full((M, N), 1.0 / N)
    Y, t = X.copy(), 1.0
    for _ in range(iters):
        Xn = proj(Y - (A @ Y + C) / Lc)
        tn = (1 + math.sqrt(1 + 4 * t * t)) / 2
        Y = Xn + (t - 1) / tn * (Xn - X)
        X, t = Xn, tn
    return X


def test_fit_matches_independent_fista():
    rng = np.random.default_rng(11)
    M, N, D = 10, 4, 24
    lam = workloads.probe_intensities(D, 9.0)
    theta = workloads.detector_povm(M, N - 1, 0.6)
    q = workloads.outcome_probabilities(lam, theta)
    P = workloads.sample_outcomes(q, 20000, rng)
    gamma = 1e-2
    pr = oracle.Problem(M, N, lam, 0.0, gamma)
    Th, rep, _ = pr.fit(P, eps_kkt=1e-13)
    Xf = fista_simplex(dense_F(M, lam, 0.0), P, gamma)
    assert rep["f"] == pytest.approx(pr.objective(P, Xf), rel=1e-9)
    assert rep["f"] <= pr.objective(P, Xf) * (1 + 1e-12)
    np.testing.assert_allclose(Th, Xf, atol=2e-5)


def test_noiseless_recovery():
    # gamma = 0, P = F Theta_true: the minimum is f* = 0 at Theta_true (F has
    # full column rank here, condition number ~2e3)
    M, N, D = 8, 4, 40
    lam = workloads.probe_intensities(D, 10.0)
    theta = workloads.detector_povm(M, N - 1, 0.8)
    P = dense_F(M, lam, 0.0) @ theta  # noise-free outcome statistics (scipy)
    pr = oracle.Problem(M, N, lam, 0.0, 0.0)
    Th, rep, _ = pr.fit(P, eps_kkt=1e-14, max_newton=3000)
    assert rep["status"] == 0
    assert rep["f"] < 1e-22
    np.testing.assert_allclose(Th, theta, atol=1e-8)


def test_fit_invariants_and_paper_constants_c1():
    with open(os.path.join(GOLD, "paper_constants.json")) as fh:
        gold = json.load(fh)
    o = oracle.Problem.default_opts()
    assert o["beta"] == gold["beta"]["value"]
    assert o["c"] == gold["c"]["value"]
    assert o["switch_tol"] == gold["switch_tol"]["value"]
    w = workloads.config_c1()
    pr = oracle.Problem.from_workload(w)
    Th, rep, hist = pr.fit(w.P, eps_kkt=1e-12)
    assert np.abs(Th.sum(1) - 1).max() <= 1e-13 * w.N
    assert Th.min() >= 0.0
    assert np.all(np.diff(hist) <= 1e-15 * hist[:-1])  # Armijo: f never increases
    assert rep["kkt"] < 1e-10
    # soft check against the iteration counts the paper reports (its CG count
    # per Newton step describes its own problem; the cap is a safety bound)
    assert rep["iters_s1"] <= 3 * gold["stage1_newton_iters"]["range"][1]
    assert rep["cg_total"] / max(1, rep["iters_s1"] + rep["iters_s2"]) <= o["max_cg"]


def test_two_stages_beat_stage_two_alone():
    """App. B, convergence of the two-stage approach: replacing the first
    iterations by the simplex-projected variant converges faster far from
    the minimum (gamma = 0 as in that comparison)."""
    w = workloads.config_c1()
    pr = oracle.Problem(w.M, w.N, w.lam, 0.0, 0.0)
    _, rep2, h2 = pr.fit(w.P, max_newton=25, start_stage=2, eps_kkt=0.0)
    _, rep12, h12 = pr.fit(w.P, max_newton=25, eps_kkt=0.0)
    assert h12[15] < h2[15]
    assert h12[-1] <= h2[-1]


def test_detector_model_occupancy_closed_form():
    """Pin of the workload generator: without dark counts and crosstalk,
    P(c clicked | k detected photons) = C(B,c) c! S(k,c) / B^k with Stirling
    numbers of the second kind, and k ~ Binomial(i, eta)."""
    from fractions import Fraction

    def stirling2(k, c):
        S = [[Fraction(0)] * (c + 1) for _ in range(k + 1)]
        S[0][0] = Fraction(1)
        for a in range(1, k + 1):
            for b in range(1, c + 1):
                S[a][b] = b * S[a - 1][b] + S[a - 1][b - 1]
        return S[k][c]

    B, eta = 5, Fraction(3, 4)
    theta = workloads.detector_povm(9, B, 0.75)
    for i in range(9):
        for c in range(B + 1):
            p = Fraction(0)
            for k in range(i + 1):
                pk = math.comb(i, k) * eta ** k * (1 - eta) ** (i - k)
                occ = Fraction(math.comb(B, c) * math.factorial(c)) * stirling2(k, c) / Fraction(B) ** k
                p += pk * occ
            assert theta[i, c] == pytest.approx(float(p), abs=1e-14)


def test_exact_kkt_solve_matches_brute_force_and_iterative_solver():
    """oracle.exact_qp: the active-set solution of the KKT conditions equals
    the brute-force optimum (tiny) from a poor seed, and the iterative
    oracle's optimum on c1."""
    from oracle import exact_qp
    rng = np.random.default_rng(21)
    for seed in range(3):
        M, N, D = 4, 3, 9
        lam = np.sort(rng.uniform(0.0, 6.0, D))
        P = rng.dirichlet(np.ones(N), D)
        F = dense_F(M, lam, 0.0)
        T_ref = brute_force_qp(F, P, 0.05)
        seed_th = np.full((M, N), 1.0 / N)      # full support: corrections needed
        Th, nu, info = exact_qp.exact_optimum(F, P, 0.05, seed_th)
        np.testing.assert_allclose(Th, T_ref, atol=1e-9)
    w = workloads.config_c1()
    pr = oracle.Problem.from_workload(w)
    Th_it, rep, _ = pr.fit(w.P, eps_kkt=1e-12)
    Th, nu, info = exact_qp.exact_optimum(pr.dense_F(), w.P, w.gamma, Th_it)
    f_exact = pr.objective(w.P, Th)
    assert info["converged"]
    assert info["primal_violation"] <= 1e-12 and info["dual_violation"] <= 1e-9
    assert f_exact <= rep["f"] * (1 + 1e-13)
    assert f_exact == pytest.approx(rep["f"], rel=1e-11)
    np.testing.assert_allclose(Th.sum(1), 1.0, atol=1e-12)


def test_smoothing_definition_and_closed_forms():
    """Eq. smoothing: direct window means (numpy), a linear profile is
    reproduced away from the clipped end, simplex rows stay simplex rows, rows
    below the exclusion are untouched."""
    rng = np.random.default_rng(12)
    M, N = 700, 5
    pr = oracle.Problem(M, N, np.array([1.0]), 0.0, 0.0)
    X = workloads.random_feasible_theta(M, N, rng)
    Y = pr.smooth(X, exclude=100, div=50.0)
    ref = X.copy()
    for i in range(100, M):
        w = i // 50
        a, b = max(0, i - w), min(M - 1, i + w)
        ref[i] = X[a:b + 1].mean(axis=0)
    np.testing.assert_allclose(Y, ref, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(Y.sum(1), 1.0, atol=1e-13)
    assert Y.min() >= 0.0
    np.testing.assert_array_equal(Y[:100], X[:100])
    # linear in i: the symmetric window mean is the centre value (unclipped rows)
    L = np.outer(np.arange(M, dtype=float), [1.0, -2.0, 0.5, 0.0, 3.0]) + 7.0
    YL = pr.smooth(L, exclude=0, div=50.0)
    rows = [i for i in range(M) if i + i // 50 <= M - 1]
    np.testing.assert_allclose(YL[rows], L[rows], rtol=1e-12)


def test_smoothed_refit_returns_to_the_unique_optimum():
    """Sec. Regularisation and smoothing: the stage-2-only refit starts from
    the smoothed POVM (feasible: a mean of simplex rows) and, the problem being
    strictly convex for gamma > 0, converges to the same optimum as the first
    fit.  A c1-sized case with a short exclusion and divisor (16, 8) so that
    the smoothing moves most rows; the paper's (100, 50) are parameters."""
    w = workloads.config_c1()
    pr = oracle.Problem.from_workload(w)
    Th1, rep1, _ = pr.fit(w.P, eps_kkt=1e-11, max_newton=800)
    Th, r1, r2, Ts = pr.fit_smoothed(w.P, exclude=16, div=8.0, eps_kkt=1e-11, max_newton=800)
    np.testing.assert_allclose(Ts.sum(1), 1.0, atol=1e-13)
    assert Ts.min() >= 0.0
    assert np.abs(Ts - Th1).max() > 1e-4      # the smoothing did move the POVM
    assert r2["iters_s1"] == 0 and r2["iters_s2"] > 0
    f1, f2, fs = (pr.objective(w.P, T) for T in (Th1, Th, Ts))
    assert fs > f1 * (1 + 1e-9)                # off the optimum after smoothing
    assert abs(f2 - f1) <= 1e-9 * f1, (f1, f2)
