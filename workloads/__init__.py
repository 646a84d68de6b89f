"""Seeded synthetic inputs for detector tomography (shared by the oracle tests,
the GPU tests and the benchmark).

This module simulates the *experiment*, not the reconstruction: it builds a
detector's true POVM matrix Theta_true (M photon numbers x N outcomes) from a
physical click-detector model, chooses coherent-probe intensities lambda_d, and
produces measured outcome frequencies P (D x N) by evaluating the probes'
photon-number statistics with ``scipy.stats.poisson`` and drawing multinomial
counts with numpy's PCG64.  It contains none of the solver's arithmetic
(objective, gradients, Hessian products, projections, Newton/CG/line-search
steps), so a mistake in either solver cannot be hidden by shared code here.

Detector model (a reading of the paper's multiplexed click detector, Sec.
"Detector under test"; the synthetic configurations use uniform bins):
B = N - 1 bins, outcome n = number of clicked bins.  Photons arrive one at a
time; each survives loss with probability eta and lands in a uniformly chosen
bin (a new click if that bin was still dark).  With probability ``crosstalk`` a
detected photon fires one extra uniformly chosen bin.  After all photons, each
still-dark bin fires a dark count with probability ``p_dark``.  Theta_true[i, :]
is the distribution of the clicked-bin count after i photons.  The chain is a
product of stochastic matrices (no alternating sums), so it is stable for any i.

Probe grid: lambda_d = X * d / (D - 1), d = 0..D-1, endpoints included.

Noise: P_d = multinomial(shots, q_d / sum(q_d)) / shots, where
q_d = sum_i Poisson(i; lambda_d) Theta_true[i, :] over i < M.  ``shots=None``
gives the noise-free q_d (not renormalised).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 2404028440


def probe_intensities(D: int, X: float) -> np.ndarray:
    """lambda_d = X*d/(D-1) for d = 0..D-1 (D == 1 gives [0])."""
    if D == 1:
        return np.zeros(1)
    return X * np.arange(D, dtype=np.float64) / (D - 1)


def quadratic_intensities(D: int, scale: float = 1.0) -> np.ndarray:
    """lambda_d = scale * d^2, the paper's experimental probe spacing."""
    return scale * np.arange(D, dtype=np.float64) ** 2


def _photon_transition(B: int, eta: float, crosstalk: float) -> np.ndarray:
    """(B+1)x(B+1) row-stochastic matrix of one arriving photon on the
    clicked-bin count c."""
    T = np.zeros((B + 1, B + 1))
    for c in range(B + 1):
        # photon lost
        T[c, c] += 1.0 - eta
        # photon detected: lands in a dark bin with probability (B-c)/B
        p_new = (B - c) / B
        for c1, w in ((c + 1, p_new), (c, 1.0 - p_new)):
            if w == 0.0:
                continue
            # no crosstalk
            T[c, c1] += eta * w * (1.0 - crosstalk)
            # crosstalk: one extra click in a uniformly chosen bin
            if crosstalk > 0.0:
                p_x = (B - c1) / B
                if p_x > 0.0:
                    T[c, c1 + 1] += eta * w * crosstalk * p_x
                T[c, c1] += eta * w * crosstalk * (1.0 - p_x)
    return T


def _dark_matrix(B: int, p_dark: float) -> np.ndarray:
    """(B+1)x(B+1) matrix: c -> c + Binomial(B - c, p_dark)."""
    K = np.zeros((B + 1, B + 1))
    for c in range(B + 1):
        k = np.arange(B - c + 1)
        logc = (math.lgamma(B - c + 1) - np.array([math.lgamma(j + 1) for j in k])
                - np.array([math.lgamma(B - c - j + 1) for j in k]))
        if p_dark == 0.0:
            w = (k == 0).astype(np.float64)
        else:
            w = np.exp(logc + k * math.log(p_dark) + (B - c - k) * math.log1p(-p_dark))
        K[c, c:] = w
    return K


def detector_povm(M: int, bins: int, eta: float, p_dark: float = 0.0,
                  crosstalk: float = 0.0) -> np.ndarray:
    """Theta_true, shape (M, bins+1), rows on the probability simplex."""
    B = int(bins)
    T = _photon_transition(B, eta, crosstalk)
    K = _dark_matrix(B, p_dark)
    theta = np.empty((M, B + 1))
    row = np.zeros(B + 1)
    row[0] = 1.0
    i = 0
    while i < M:
        theta[i] = row
        nxt = row @ T
        i += 1
        # once the chain has reached its absorbing state to the last bit,
        # every later row is identical
        if np.array_equal(nxt, row):
            theta[i:] = row
            break
        row = nxt
    theta = theta @ K
    # rows are stochastic up to rounding; renormalise exactly
    theta = np.maximum(theta, 0.0)
    theta /= theta.sum(axis=1, keepdims=True)
    return theta


def outcome_probabilities(lam: np.ndarray, theta: np.ndarray,
                          width_sigmas: float = 14.0) -> np.ndarray:
    """q_d = sum_{i<M} Poisson(i; lambda_d) Theta[i, :], using scipy's pmf on
    the photon numbers within +-width_sigmas*sqrt(lambda)+40 of lambda (the
    mass outside is below 1e-40)."""
    from scipy.stats import poisson

    M, N = theta.shape
    D = lam.shape[0]
    q = np.zeros((D, N))
    # rows identical from some index on: collapse the tail into one sf term
    last_change = M - 1
    while last_change > 0 and np.array_equal(theta[last_change], theta[last_change - 1]):
        last_change -= 1
    for d in range(D):
        l = float(lam[d])
        s = math.sqrt(l)
        a = max(0, int(math.floor(l - width_sigmas * s - 40)))
        b = min(M - 1, int(math.ceil(l + width_sigmas * s + 40)))
        if a > b:
            continue
        b_body = min(b, last_change - 1) if last_change < M - 1 else b
        if b_body >= a:
            i = np.arange(a, b_body + 1)
            w = poisson.pmf(i, l)
            q[d] += w @ theta[a:b_body + 1]
        if last_change < M - 1 and b >= last_change:
            start = max(a, last_change)
            # mass on [start, M-1] of the constant tail row
            mass = poisson.cdf(M - 1, l) - (poisson.cdf(start - 1, l) if start > 0 else 0.0)
            if mass < 0.0:
                mass = float(poisson.pmf(np.arange(start, min(M, start + 200000)), l).sum())
            q[d] += mass * theta[last_change]
    return q


def sample_outcomes(q: np.ndarray, shots, rng: np.random.Generator) -> np.ndarray:
    """Multinomial outcome frequencies per probe (shots=None: noise-free q)."""
    if shots is None:
        return q.copy()
    P = np.empty_like(q)
    for d in range(q.shape[0]):
        p = np.maximum(q[d], 0.0)
        p = p / p.sum()
        P[d] = rng.multinomial(int(shots), p) / float(shots)
    return P


@dataclasses.dataclass
class Workload:
    name: str
    M: int
    N: int
    D: int
    lam: np.ndarray
    P: np.ndarray
    theta_true: np.ndarray
    gamma: float
    band_k: float
    seed: int
    shots: object

    @property
    def MN(self) -> int:
        return self.M * self.N


def make_workload(name: str, M: int, bins: int, eta: float, D: int, X: float,
                  gamma: float, band_k: float, shots, seed: int,
                  p_dark: float = 0.0, crosstalk: float = 0.0,
                  lam: np.ndarray | None = None) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = detector_povm(M, bins, eta, p_dark=p_dark, crosstalk=crosstalk)
    if lam is None:
        lam = probe_intensities(D, X)
    q = outcome_probabilities(lam, theta)
    P = sample_outcomes(q, shots, rng)
    return Workload(name, M, bins + 1, D, lam, P, theta, gamma, band_k, seed, shots)


def config_c1(shots=1_000_000) -> Workload:
    """Plain FP64 fit: M=64, N=9 (8-bin detector, eta=0.7), D=100 probes with
    lambda linear in [0,30], 1e6 shots, gamma=1e-3, dense F."""
    return make_workload("c1_M64_N9_D100", 64, 8, 0.7, 100, 30.0, 1e-3, 0.0,
                         shots, BASE_SEED + 0)


def config_c2(shots=10_000_000) -> Workload:
    """FP64 vs FP32 fit: M=4096, N=128 (127 bins, eta=0.8, dark 1e-4/bin),
    D=8192 probes with lambda linear in [0,3000], 1e7 shots, gamma=1e-2,
    Poisson band +-10 sqrt(lambda)."""
    return make_workload("c2_M4096_N128_D8192", 4096, 127, 0.8, 8192, 3000.0,
                         1e-2, 10.0, shots, BASE_SEED + 1, p_dark=1e-4)


C4_GAMMAS = (1e-4, 1e-3, 1e-2, 1e-1)


def config_c4(n_instances=256, max_M=8192, shots=1_000_000):
    """Batched instances: M ~ U{256..max_M}, N ~ U{8..128} (bins = N - 1),
    efficiency U[0.3, 0.95], D = 2M probes with lambda linear in [0, 0.75 M],
    1e6 shots; each to be solved at gamma in C4_GAMMAS.  Instance j uses seed
    BASE_SEED + 3 + 1000 j."""
    return [config_c4_instance(j, max_M, shots) for j in range(n_instances)]


def config_c4_instance(j, max_M=8192, shots=1_000_000):
    """Instance j of config_c4 alone (same seed, same draws)."""
    seed = BASE_SEED + 3 + 1000 * j
    rng = np.random.Generator(np.random.PCG64(seed))
    M = int(rng.integers(256, max_M + 1))
    N = int(rng.integers(8, 129))
    eta = float(rng.uniform(0.3, 0.95))
    D = 2 * M
    return make_workload(f"c4_{j}_M{M}_N{N}", M, N - 1, eta, D, 0.75 * M, C4_GAMMAS[0],
                         10.0, shots, seed)


def small_case(M=48, bins=7, eta=0.75, D=80, X=40.0, gamma=1e-3, band_k=10.0,
               shots=100_000, seed=BASE_SEED + 77, p_dark=0.0, crosstalk=0.0):
    """A scaled-down instance of the same construction (tests)."""
    return make_workload(f"small_M{M}_N{bins+1}_D{D}", M, bins, eta, D, X, gamma,
                         band_k, shots, seed, p_dark=p_dark, crosstalk=crosstalk)


def random_feasible_theta(M: int, N: int, rng: np.random.Generator,
                          sparsity: float = 0.3) -> np.ndarray:
    """A random point of the row simplices with some exact zeros."""
    x = rng.random((M, N))
    x[rng.random((M, N)) < sparsity] = 0.0
    x[np.arange(M), rng.integers(0, N, M)] += 0.5
    return x / x.sum(axis=1, keepdims=True)


# ---- learned warm start: detector population -------------------------------
C5_M, C5_D, C5_X, C5_C0, C5_GAMMA, C5_SHOTS = 1024, 2048, 768.0, 64, 1e-3, 1_000_000


def dense_poisson(M: int, lam: np.ndarray) -> np.ndarray:
    """F_{d,i} = Poisson(i; lambda_d) for i < M from scipy's pmf (dense)."""
    from scipy.stats import poisson
    return poisson.pmf(np.arange(M)[None, :], np.asarray(lam)[:, None])


def config_c5_instance(j: int, F: np.ndarray | None = None, M: int = C5_M, D: int = C5_D,
                       X: float = C5_X, shots=C5_SHOTS, bins_range=(16, 63),
                       gamma: float = C5_GAMMA) -> Workload:
    """Instance j of the warm-start detector population: bins ~ U{16..63}
    (N = bins + 1 <= 64), efficiency U[0.3, 0.95], crosstalk U[0, 1e-2], dark
    counts U[0, 1e-3] per bin; D probes with lambda linear in [0, X]; dense
    outcome probabilities q = F Theta_true, multinomial shots.  Seed
    BASE_SEED + 4 + 1000 j.  F (D x M, from dense_poisson) may be passed in to
    share it across instances."""
    seed = BASE_SEED + 4 + 1000 * j
    rng = np.random.Generator(np.random.PCG64(seed))
    bins = int(rng.integers(bins_range[0], bins_range[1] + 1))
    eta = float(rng.uniform(0.3, 0.95))
    xt = float(rng.uniform(0.0, 1e-2))
    dark = float(rng.uniform(0.0, 1e-3))
    lam = probe_intensities(D, X)
    if F is None:
        F = dense_poisson(M, lam)
    theta = detector_povm(M, bins, eta, p_dark=dark, crosstalk=xt)
    q = F @ theta
    if shots is None:
        P = q
    else:
        p = np.maximum(q, 0.0)
        p /= p.sum(axis=1, keepdims=True)
        P = rng.multinomial(int(shots), p) / float(shots)
    return Workload(f"c5_{j}_N{bins + 1}", M, bins + 1, D, lam, P, theta, gamma, 10.0, seed, shots)


def c5_batch(js, F=None, C0: int = C5_C0, **kw):
    """Padded arrays of instances js: P (B, D, C0), Theta_true (B, M, C0),
    ncols (B,)."""
    ws = [config_c5_instance(j, F=F, **kw) for j in js]
    B, D, M = len(ws), ws[0].D, ws[0].M
    P = np.zeros((B, D, C0))
    T = np.zeros((B, M, C0))
    nc = np.zeros(B, dtype=np.int32)
    for b, w in enumerate(ws):
        P[b, :, :w.N] = w.P
        T[b, :, :w.N] = w.theta_true
        nc[b] = w.N
    return P, T, nc, ws


# ---- the paper's detector geometry (time-multiplexed loop detector) --------
# Sec. Experiment: out-coupling R, loop efficiency eta_loop, detector
# efficiency eta_det fitted by the paper; 150 time bins (N = 151 outcomes);
# D = 1076 coherent probes with |alpha_d|^2 ~ d^2; Hilbert space M = 1210581;
# 5e5 trials per probe.
LOOP_R, LOOP_ETA_LOOP, LOOP_ETA_DET = 0.91644, 0.90524, 0.528
F2_M, F2_D, F2_BINS, F2_SHOTS = 1210581, 1076, 150, 500_000


def loop_bin_click(bins: int = F2_BINS, R: float = LOOP_R, eta_loop: float = LOOP_ETA_LOOP,
                   eta_det: float = LOOP_ETA_DET) -> np.ndarray:
    """Per-photon click probability of time bin j = 1..bins (Eq. pj_fock at
    i = 1): q_1 = R eta_det, q_j = (1 - R)^2 R^-1 (R eta_loop)^(j-1) eta_det."""
    j = np.arange(1, bins + 1, dtype=np.float64)
    q = (1.0 - R) ** 2 / R * (R * eta_loop) ** (j - 1) * eta_det
    q[0] = R * eta_det
    return q


def loop_detector_povm(M: int, bins: int = F2_BINS, R: float = LOOP_R, eta_loop: float = LOOP_ETA_LOOP,
                       eta_det: float = LOOP_ETA_DET) -> np.ndarray:
    """Theta_true (M x (bins + 1)) of the loop detector: for i photons bin j
    clicks with p_j(i) = 1 - (1 - q_j)^i (Eq. pj_fock), bins independently, so
    the number of clicked bins is Poisson-binomial; computed by the exact
    recursion over bins (one bin at a time, column-major for speed)."""
    q = loop_bin_click(bins, R, eta_loop, eta_det)
    i = np.arange(M, dtype=np.float64)
    dist = np.zeros((bins + 1, M))
    dist[0] = 1.0
    tmp = np.empty(M)
    for j in range(bins):
        p = -np.expm1(i * np.log1p(-q[j]))
        omp = 1.0 - p
        for n in range(j + 1, 0, -1):
            np.multiply(dist[n], omp, out=dist[n])
            np.multiply(dist[n - 1], p, out=tmp)
            dist[n] += tmp
        dist[0] *= omp
    theta = np.ascontiguousarray(dist.T)
    theta = np.maximum(theta, 0.0)
    theta /= theta.sum(axis=1, keepdims=True)
    return theta


def config_f2(M: int = F2_M, D: int = F2_D, bins: int = F2_BINS, shots=F2_SHOTS, gamma: float = 1e-5,
              seed: int = BASE_SEED + 5) -> Workload:
    """The paper's geometry: loop-detector POVM, probes lambda_d = d^2
    (d = 0..D-1), multinomial trials per probe, band +-10 sqrt(lambda).
    Defaults are the paper's sizes; smaller M and D give the same geometry at
    a smaller scale (D should stay near sqrt(M))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = loop_detector_povm(M, bins)
    lam = quadratic_intensities(D)
    q = outcome_probabilities(lam, theta)
    P = sample_outcomes(q, shots, rng)
    return Workload(f"f2_M{M}_N{bins + 1}_D{D}", M, bins + 1, D, lam, P, theta, gamma, 10.0, seed, shots)


# ---- Liu-shaped near-dense geometry (Sec. Application to other detector
# geometries, Eq. liu_M, Eq. liu_D) --------------------------------------------
def liu_sizes(N: int) -> tuple[int, int]:
    """M ~ 6.6 N^1.06 and D ~ 4.0 N^1.14 (rounded)."""
    return int(round(6.6 * N ** 1.06)), int(round(4.0 * N ** 1.14))


def config_f3(N: int, eta: float = 0.9, shots=1_000_000, gamma: float = 1e-4,
              seed: int | None = None) -> Workload:
    """Synthetic stand-in for the spatially multiplexed detector of Liu et al.
    (whose input generator is not available): an equal-split network onto
    N - 1 click detectors of efficiency eta, outcome n = number of clicking
    detectors (the uniform-bin chain model of detector_povm), M and D from
    liu_sizes(N), lambda linear in [0, 0.75 M], multinomial shots.  Seed
    BASE_SEED + 6 + N unless given."""
    M, D = liu_sizes(N)
    return make_workload(f"f3_N{N}_M{M}_D{D}", M, N - 1, eta, D, 0.75 * M, gamma, 10.0, shots,
                         BASE_SEED + 6 + N if seed is None else seed)
