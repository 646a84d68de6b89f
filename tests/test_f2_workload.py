"""Pins of the paper-geometry workload (loop detector, Sec. Experiment) and
of the infidelity of Eq. fidelities (CPU)."""
import itertools

import numpy as np
import pytest

import oracle
import workloads


def test_poisson_binomial_matches_enumeration():
    bins = 8
    th = workloads.loop_detector_povm(41, bins)
    q = workloads.loop_bin_click(bins)
    for i in (0, 1, 5, 40):
        p = 1.0 - (1.0 - q) ** i          # Eq. pj_fock
        ref = np.zeros(bins + 1)
        for clicks in itertools.product((0, 1), repeat=bins):
            c = np.array(clicks)
            ref[c.sum()] += np.prod(np.where(c == 1, p, 1.0 - p))
        np.testing.assert_allclose(th[i], ref, rtol=1e-12, atol=1e-15)


def test_loop_povm_closed_forms():
    M, bins = 5000, 150
    th = workloads.loop_detector_povm(M, bins)
    q = workloads.loop_bin_click(bins)
    np.testing.assert_allclose(th.sum(1), 1.0, atol=1e-13)
    assert th[0, 0] == 1.0 and np.all(th[0, 1:] == 0.0)
    # the paper's parameters: bin 1 at i = 1 clicks with R eta_det
    assert q[0] == pytest.approx(0.91644 * 0.528, rel=1e-15)
    assert q[1] == pytest.approx((1 - 0.91644) ** 2 / 0.91644 * (0.91644 * 0.90524) * 0.528, rel=1e-14)
    # mean number of clicks = sum_j p_j(i) (linearity, whatever the correlations)
    for i in (1, 17, 333, 4999):
        mean = th[i] @ np.arange(bins + 1)
        assert mean == pytest.approx(np.sum(1.0 - (1.0 - q) ** i), rel=1e-11)


def test_coherent_bin_clicks_follow_from_fock_ones():
    """Eq. pj_coh from Eq. pj_fock and Eq. Fmatrix: for noise-free outcome
    frequencies of coherent probes, the mean number of clicked bins equals
    sum_j (1 - exp(-lambda q_j))."""
    w = workloads.config_f2(M=20000, D=120, shots=None)
    q = workloads.loop_bin_click(w.N - 1)
    mean = w.P @ np.arange(w.N)
    ref = np.array([np.sum(-np.expm1(-l * q)) for l in w.lam])
    np.testing.assert_allclose(mean, ref, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(w.lam, np.arange(120.0) ** 2)


def test_infidelity_definition():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(3)
    A = rng.random((12, 4))
    B = rng.random((12, 4))
    got = oracle.infidelity(A, B)
    for n in range(4):
        # the general definition with matrix square roots of the (diagonal) operators
        a, b = np.diag(A[:, n]), np.diag(B[:, n])
        sa = scipy_linalg.sqrtm(a)
        inner = scipy_linalg.sqrtm(sa @ b @ sa)
        F = np.real(np.trace(inner)) ** 2 / (np.trace(a) * np.trace(b))
        assert got[n] == pytest.approx(1.0 - F, abs=1e-12)
    assert np.allclose(oracle.infidelity(A, A), 0.0, atol=1e-14)
    # disjoint supports: fidelity 0
    C = np.array([[1.0, 0.0], [0.0, 1.0]])
    np.testing.assert_allclose(oracle.infidelity(C, C[::-1]), 1.0)
    # two-level hand value: (sqrt(.36*.64) + sqrt(.64*.36))^2 = 0.9216
    assert oracle.infidelity(np.array([[0.36], [0.64]]), np.array([[0.64], [0.36]]))[0] == pytest.approx(0.0784)


def test_liu_sizes_follow_the_papers_power_laws():
    """Eq. liu_M / liu_D; the paper quotes N M = 1.04e7 free variables at
    N = 1000 (the power laws are approximate: within 5 %)."""
    M, D = workloads.liu_sizes(1000)
    assert M == round(6.6 * 1000 ** 1.06) and D == round(4.0 * 1000 ** 1.14)
    assert abs(M * 1000 - 1.04e7) <= 0.05 * 1.04e7
    w = workloads.config_f3(30, shots=None)
    assert (w.M, w.D, w.N) == (*workloads.liu_sizes(30), 30)
    np.testing.assert_allclose(w.theta_true.sum(1), 1.0, atol=1e-13)
