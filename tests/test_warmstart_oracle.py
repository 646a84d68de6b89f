"""Pins of the learned-warm-start oracle (oracle/warmstart.py): its gradient
against central differences (and planted mistakes that this pin catches), its
convolution against numpy's correlate, the softmax's simplex rows, the first
Adam step's closed form, the bf16 rounding against torch's conversion, and
the warm-start population's outcome probabilities against the shared
generator's windowed sum."""
import numpy as np
import pytest

from oracle import warmstart as ws
import workloads

TINY = ws.Shape(D=16, C0=4, M=6, C1=3, C2=2, K=3, S1=2, S2=2, H=3)


def tiny_batch(rng, B=2):
    Ps = [rng.random((TINY.D, TINY.C0)) for _ in range(B)]
    ncols = [TINY.C0, TINY.C0 - 1][:B]
    Ts = []
    for b in range(B):
        T = rng.random((TINY.M, TINY.C0))
        T[:, ncols[b]:] = 0.0
        Ts.append(T / T.sum(1, keepdims=True))
    return Ps, Ts, ncols


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(TINY.count()) * 0.5
    Ps, Ts, ncols = tiny_batch(rng)
    L, g = ws.loss_and_grad(TINY, theta, Ps, Ts, ncols)
    h = 1e-6
    idx = rng.choice(TINY.count(), 60, replace=False)
    # every parameter block is represented
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in TINY.sizes()])
    idx = np.unique(np.concatenate([idx, offs[:-1]]))
    for j in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (ws.loss_and_grad(TINY, tp, Ps, Ts, ncols)[0] - ws.loss_and_grad(TINY, tm, Ps, Ts, ncols)[0]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, g[j])
    assert L > 0


def test_conv1d_matches_numpy_correlate():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((20, 3))
    W = rng.standard_normal((2, 3, 5))
    b = rng.standard_normal(2)
    for S in (1, 2, 4):
        Y = ws.conv1d(X, W, b, S)
        ref = np.zeros((20 // S, 2))
        for co in range(2):
            full = b[co] + sum(np.correlate(np.pad(X[:, ci], 2), W[co, ci], mode="valid") for ci in range(3))
            ref[:, co] = full[::S][:20 // S]
        np.testing.assert_allclose(Y, ref, rtol=1e-12, atol=1e-12)


def test_softmax_rows_are_simplex_rows_with_masked_columns():
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((7, 6)) * 30
    Th = ws.masked_softmax(Z, 4)
    np.testing.assert_allclose(Th.sum(1), 1.0, atol=1e-14)
    assert np.all(Th[:, 4:] == 0.0) and Th.min() >= 0.0
    # invariant to a per-row shift
    np.testing.assert_allclose(ws.masked_softmax(Z + 100.0, 4), Th, atol=1e-14)


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(6)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m, v = ws.adam_step(th, np.zeros(50), np.zeros(50), g, 1, 1e-3)
    # bias-corrected first moments equal g and g^2: the step is lr g / (|g| + eps)
    np.testing.assert_allclose(th - new, 1e-3 * g / (np.abs(g) + ws.ADAM_EPS), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.integers(-8, 8, 1000),
                        [0.0, 1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -1 - 2.0 ** -8]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ws.round_bf16(x), ref)
    # ties go to the even neighbour
    assert ws.round_bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0
    assert ws.round_bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6


# Plausible mistakes planted in copies of the oracle's functions: each must
# make the central-difference pin fail (the pin catches them).
def _fd_mismatch(loss_and_grad):
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(TINY.count()) * 0.5
    Ps, Ts, ncols = tiny_batch(rng)
    _, g = loss_and_grad(TINY, theta, Ps, Ts, ncols)
    h = 1e-6
    worst = 0.0
    for j in rng.choice(TINY.count(), 80, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (ws.loss_and_grad(TINY, tp, Ps, Ts, ncols)[0] - ws.loss_and_grad(TINY, tm, Ps, Ts, ncols)[0]) / (2 * h)
        worst = max(worst, abs(fd - g[j]) / max(1.0, abs(fd)))
    return worst


@pytest.mark.parametrize("mutant", ["leaky_forward_relu_backward", "softmax_columns_permuted",
                                    "conv_backward_stride_ignored"])
def test_gradient_pin_catches_planted_mistakes(monkeypatch, mutant):
    assert _fd_mismatch(ws.loss_and_grad) <= 1e-6
    if mutant == "leaky_forward_relu_backward":
        # the backward pass uses (Y > 0) masks; a leaky forward disagrees
        monkeypatch.setattr(ws, "relu", lambda x: np.where(x > 0, x, 0.1 * x))
    elif mutant == "softmax_columns_permuted":
        orig = ws.masked_softmax

        def bad(Z, ncols):
            out = orig(Z, ncols)
            return out[:, ::-1].copy() if ncols == Z.shape[1] else out
        monkeypatch.setattr(ws, "masked_softmax", bad)
    else:
        orig = ws.conv1d_backward
        monkeypatch.setattr(ws, "conv1d_backward", lambda X, W, dY, S: orig(X, W, dY, 1))
    assert _fd_mismatch(ws.loss_and_grad) > 1e-4


def test_c5_population_outcomes_match_the_windowed_generator():
    """The warm-start population's dense F q equals the windowed scipy sum
    of the shared generator (two independent evaluations)."""
    M, D, X = 300, 400, 200.0
    lam = workloads.probe_intensities(D, X)
    F = workloads.dense_poisson(M, lam)
    w = workloads.config_c5_instance(3, F=F, M=M, D=D, X=X, shots=None, bins_range=(4, 15))
    q = workloads.outcome_probabilities(lam, w.theta_true)
    np.testing.assert_allclose(w.P, q, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(w.theta_true.sum(1), 1.0, atol=1e-13)
