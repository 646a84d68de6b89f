"""Oracle of the learned warm start (test infrastructure: only tests/ and the
benchmark's CPU legs may import this module).

The learned warm start is not in the paper: it is this project's addition on
top of the solver (a feasible starting point for Algorithm 3 instead of
Theta^(0) = 1/N).  Its definition is the network below, written out in plain
numpy (float64 unless a function says otherwise), one operation per line,
for checking the CUDA kernels element by element.

Network (one sample; P is D x C0 with the outcome columns n >= ncols zero):
  Y1 = conv1d(P,  W1, b1, stride S1)          (T1 = D / S1) x C1
  Y2 = conv1d(relu(Y1), W2, b2, stride S2)    (T2 = T1 / S2) x C2
  Y3 = W3 flat(relu(Y2)) + b3                 H           (flat: t-major, then channel)
  Z  = W4 relu(Y3) + b4                       M x C0      (row-major logits)
  Theta0[i, :] = softmax over n < ncols of Z[i, :], 0 for n >= ncols
conv1d(X, W, b, S)[t, co] = b[co] + sum_{ci, k} W[co, ci, k] X[S t + k - K//2, ci]
(zero outside 0 <= S t + k - K//2 < rows of X).
Loss (row-wise cross-entropy against a target POVM T, rows summing to 1):
  L = -(1 / (B M)) sum_b sum_i sum_{n < ncols_b} T[b, i, n] log Theta0[b, i, n]
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
Parameters are laid out in one vector: W1, b1, W2, b2, W3, b3, W4, b4.
"""
from __future__ import annotations

import dataclasses

import numpy as np

ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


@dataclasses.dataclass(frozen=True)
class Shape:
    D: int
    C0: int
    M: int
    C1: int = 32
    C2: int = 32
    K: int = 5
    S1: int = 2
    S2: int = 4
    H: int = 32

    @property
    def T1(self):
        return self.D // self.S1

    @property
    def T2(self):
        return self.T1 // self.S2

    @property
    def F(self):
        return self.T2 * self.C2

    def sizes(self):
        return [("W1", (self.C1, self.C0, self.K)), ("b1", (self.C1,)),
                ("W2", (self.C2, self.C1, self.K)), ("b2", (self.C2,)),
                ("W3", (self.H, self.F)), ("b3", (self.H,)),
                ("W4", (self.M * self.C0, self.H)), ("b4", (self.M * self.C0,))]

    def count(self):
        return sum(int(np.prod(s)) for _, s in self.sizes())


def unpack(shape: Shape, theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, s in shape.sizes():
        n = int(np.prod(s))
        out[name] = theta[o:o + n].reshape(s)
        o += n
    return out


def pack(shape: Shape, params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in shape.sizes()])


def conv1d(X, W, b, S):
    """Direct definition: every output element is its own sum."""
    Tin, Cin = X.shape
    Cout, _, K = W.shape
    Tout = Tin // S
    Y = np.empty((Tout, Cout))
    for t in range(Tout):
        for co in range(Cout):
            acc = b[co]
            for k in range(K):
                s = S * t + k - K // 2
                if 0 <= s < Tin:
                    acc += np.dot(W[co, :, k], X[s, :])
            Y[t, co] = acc
    return Y


def relu(x):
    return np.maximum(x, 0.0)


def masked_softmax(Z, ncols):
    Zm = Z[:, :ncols]
    e = np.exp(Zm - Zm.max(axis=1, keepdims=True))
    out = np.zeros_like(Z)
    out[:, :ncols] = e / e.sum(axis=1, keepdims=True)
    return out


def forward(shape: Shape, theta: np.ndarray, P: np.ndarray, ncols: int) -> dict:
    """One sample; returns every intermediate (pre-activations and Theta0)."""
    p = unpack(shape, theta)
    X0 = np.array(P, dtype=np.float64)
    X0[:, ncols:] = 0.0
    Y1 = conv1d(X0, p["W1"], p["b1"], shape.S1)
    Y2 = conv1d(relu(Y1), p["W2"], p["b2"], shape.S2)
    A2 = relu(Y2).reshape(-1)
    Y3 = p["W3"] @ A2 + p["b3"]
    Z = (p["W4"] @ relu(Y3) + p["b4"]).reshape(shape.M, shape.C0)
    Th = masked_softmax(Z, ncols)
    return {"X0": X0, "Y1": Y1, "Y2": Y2, "Y3": Y3, "Z": Z, "Theta0": Th}


def loss_and_grad(shape: Shape, theta: np.ndarray, Ps, Ts, ncols) -> tuple[float, np.ndarray]:
    """Batch loss and its gradient by reverse-mode differentiation written out
    layer by layer."""
    B = len(Ps)
    p = unpack(shape, theta)
    g = {name: np.zeros(s) for name, s in shape.sizes()}
    L = 0.0
    scale = 1.0 / (B * shape.M)
    for b in range(B):
        nc = int(ncols[b])
        fw = forward(shape, theta, Ps[b], nc)
        Th = fw["Theta0"]
        T = np.array(Ts[b], dtype=np.float64)
        T[:, nc:] = 0.0
        with np.errstate(divide="ignore"):
            logs = np.where(T[:, :nc] > 0, np.log(np.maximum(Th[:, :nc], 1e-300)), 0.0)
        L += -scale * np.sum(T[:, :nc] * logs)
        # d L / d Z of softmax + cross-entropy (target rows sum to 1)
        dZ = np.zeros_like(Th)
        dZ[:, :nc] = scale * (Th[:, :nc] * T[:, :nc].sum(axis=1, keepdims=True) - T[:, :nc])
        dZ = dZ.reshape(-1)
        A3 = relu(fw["Y3"])
        g["W4"] += np.outer(dZ, A3)
        g["b4"] += dZ
        dY3 = (p["W4"].T @ dZ) * (fw["Y3"] > 0)
        A2 = relu(fw["Y2"]).reshape(-1)
        g["W3"] += np.outer(dY3, A2)
        g["b3"] += dY3
        dY2 = ((p["W3"].T @ dY3) * (fw["Y2"].reshape(-1) > 0)).reshape(shape.T2, shape.C2)
        A1 = relu(fw["Y1"])
        dW2, db2, dA1 = conv1d_backward(A1, p["W2"], dY2, shape.S2)
        g["W2"] += dW2
        g["b2"] += db2
        dY1 = dA1 * (fw["Y1"] > 0)
        dW1, db1, _ = conv1d_backward(fw["X0"], p["W1"], dY1, shape.S1)
        g["W1"] += dW1
        g["b1"] += db1
    return L, pack(shape, g)


def conv1d_backward(X, W, dY, S):
    """Gradients of conv1d(X, W, b, S) given dL/dY: (dW, db, dX)."""
    Tin, Cin = X.shape
    Cout, _, K = W.shape
    Tout = dY.shape[0]
    dW = np.zeros_like(W)
    dX = np.zeros_like(X)
    for t in range(Tout):
        for k in range(K):
            s = S * t + k - K // 2
            if 0 <= s < Tin:
                dW[:, :, k] += np.outer(dY[t, :], X[s, :])
                dX[s, :] += W[:, :, k].T @ dY[t, :]
    return dW, dY.sum(axis=0), dX


def adam_step(theta, m, v, grad, step, lr):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = ADAM_B1 * m + (1 - ADAM_B1) * grad
    v = ADAM_B2 * v + (1 - ADAM_B2) * grad * grad
    mh = m / (1 - ADAM_B1 ** step)
    vh = v / (1 - ADAM_B2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def round_bf16(x):
    """Round-to-nearest-even to bfloat16, returned as float64 (the rounding of
    the weights used at inference)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
