"""Plain FP64 CPU oracle of the warm-start perceptron and its features --
TEST INFRASTRUCTURE ONLY (tests/ and the package smoke check use it; the
solver library never does, and it shares no code with the CUDA path).

The network is the one include/spfom_mlp.h defines: x in R^16 ->
h1 = relu(W1 x + b1) -> h2 = relu(W2 h1 + b2) -> o = w3 . h2 + b3, trained on
the mean squared error (1/R) sum_r (o_r - t_r)^2. The warm start is a build
addition: the paper names data-driven modules only as future work (Section 7),
so what pins this oracle is mathematics, not the paper: central finite
differences of the loss for the gradients (exact arithmetic, rounding off),
numpy's matrix products for the forward pass, and torch's (or a hand-listed)
BF16 rounding for ``bf16``.

``rounding=True`` reproduces the precision the tensor-core kernels define:
inputs, weights, the hidden activations and the output gradients are rounded
to BF16 (round to nearest, ties to even) where they enter a product, while the
products themselves, biases, the loss and the gradients stay in binary64 here
(FP32 accumulation in the kernels). The rounded and the exact network differ by
O(2^-8) relative; the GPU and the rounded oracle differ only where an FP32 vs
binary64 accumulation lands on different sides of a BF16 rounding boundary.
"""
from __future__ import annotations

import numpy as np

F, H = 16, 256
PARAMS = H * F + H + H * H + H + H + 1


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64.
    Goes through binary32 first, as the kernels' FP32 values do."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def unpack(p):
    """Split the packed parameter vector: W1 [256,16], b1, W2 [256,256], b2, w3 [256], b3."""
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (PARAMS,)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def forward(p, X, rounding: bool = True):
    """Outputs o [R] and the cache of the backward pass."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    rnd = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    Xb, W1b, W2b, w3b = rnd(X), rnd(W1), rnd(W2), rnd(w3)
    h1 = rnd(np.maximum(Xb @ W1b.T + b1, 0.0))
    h2 = rnd(np.maximum(h1 @ W2b.T + b2, 0.0))
    o = h2 @ w3b + b3
    return o, (Xb, W1b, W2b, w3b, h1, h2)


def loss(p, X, t, rounding: bool = True) -> float:
    o, _ = forward(p, X, rounding)
    return float(np.mean((o - np.asarray(t, dtype=np.float64)) ** 2))


def loss_grad(p, X, t, rounding: bool = True):
    """(loss, gradient in the packed layout) by the chain rule, layer by layer."""
    o, (Xb, W1b, W2b, w3b, h1, h2) = forward(p, X, rounding)
    rnd = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    R = len(o)
    e = o - np.asarray(t, dtype=np.float64)
    L = float(np.mean(e ** 2))
    dO = rnd(2.0 * e / R)                      # dL/do_r
    dw3 = h2.T @ dO
    db3 = float(np.sum(dO))
    dH2 = rnd(np.outer(dO, w3b) * (h2 > 0))    # through o = w3 . h2 and the ReLU
    dW2 = dH2.T @ h1
    db2 = dH2.sum(axis=0)
    dH1 = rnd((dH2 @ W2b) * (h1 > 0))          # through h2 = relu(W2 h1 + b2) and the ReLU
    dW1 = dH1.T @ Xb
    db1 = dH1.sum(axis=0)
    return L, pack(dW1, db1, dW2, db2, dw3, db3)


def glorot(seed: int) -> np.ndarray:
    """A seeded parameter vector of the network's shape (test inputs only)."""
    rng = np.random.default_rng(seed)
    a1, a2, a3 = np.sqrt(6 / (F + H)), np.sqrt(6 / (2 * H)), np.sqrt(6 / (H + 1))
    return pack(rng.uniform(-a1, a1, (H, F)), rng.uniform(-0.1, 0.1, H), rng.uniform(-a2, a2, (H, H)),
                rng.uniform(-0.1, 0.1, H), rng.uniform(-a3, a3, H), 0.05)


# ---- features (the definition include/spfom_mlp.h states, written out) ----------------

def features(inst, s0) -> np.ndarray:
    """Per-resource features [m, 16] from the instance and the sales s0 [n] of
    the best assortments at y = 0, one resource at a time."""
    n, m = inst.n, inst.m
    a_val = inst.a_val if inst.a_val is not None else np.ones(len(inst.a_idx))
    users = [[] for _ in range(m)]          # (product, a_ij) per resource
    for j in range(n):
        for q in range(inst.a_ptr[j], inst.a_ptr[j + 1]):
            users[inst.a_idx[q]].append((j, float(a_val[q])))
    nres = np.diff(inst.a_ptr)
    d = np.array([sum(a * s0[j] for j, a in users[i]) for i in range(m)])
    mean_r, mean_c = float(np.mean(inst.r)), float(np.mean(inst.c))
    nnz_per_res = len(inst.a_idx) / m

    def ratio(di, ci):
        if di <= 0:
            return 0.0
        if ci <= 0:
            return 8.0
        return min(di / ci, 8.0)

    rho = np.array([max([ratio(d[k], inst.c[k]) for k in inst.a_idx[inst.a_ptr[j]:inst.a_ptr[j + 1]]] + [0.0])
                    for j in range(n)])
    out = np.zeros((m, 16))
    for i in range(m):
        c, di = float(inst.c[i]), float(d[i])
        w = sum(a * s0[j] for j, a in users[i])
        wr = sum(a * s0[j] * inst.r[j] for j, a in users[i])
        wr2 = sum(a * s0[j] * inst.r[j] ** 2 for j, a in users[i])
        mean = wr / w if w > 0 else 0.0
        var = wr2 / w - mean ** 2 if w > 0 else 0.0
        if di > 0 and c > 0:
            lr = float(np.clip(np.log(di / c), -6, 6))
        else:
            lr = 6.0 if di > 0 else -6.0
        out[i, 0] = c / mean_c
        out[i, 1] = di / mean_c
        out[i, 2] = min(c / di, 4.0) if di > 0 else 4.0
        out[i, 3] = lr
        out[i, 4] = mean / mean_r
        out[i, 5] = max([inst.r[j] for j, _ in users[i]] + [0.0]) / mean_r
        out[i, 6] = np.sqrt(max(var, 0.0)) / mean_r
        out[i, 7] = (sum(a * s0[j] * inst.r[j] / max(nres[j], 1) for j, a in users[i]) / w / mean_r) if w > 0 else 0.0
        out[i, 8] = len(users[i]) / nnz_per_res
        out[i, 9] = float(np.sum(inst.c) / np.sum(d)) if np.sum(d) > 0 else 4.0
        out[i, 10] = sum(a * s0[j] * rho[j] for j, a in users[i]) / w if w > 0 else 0.0
        out[i, 11] = 1.0
        out[i, 12] = 1.0 if di > c else 0.0
    return out
