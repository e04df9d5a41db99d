"""CPU oracle of the surrogate network -- TEST INFRASTRUCTURE.

A multilayer perceptron 36 -> 256 -> 256 -> 8 (ReLU, softmax cross-entropy)
over the bits of a 36-bit genome, written out in numpy float64.  The GPU path
stores its GEMM operands in bfloat16 and accumulates in float32; with
`bf16=True` this oracle rounds the same tensors to bfloat16 (round to nearest
even) at the same places and accumulates in float64, so the two agree up to
the float32 accumulation error and bfloat16 rounding-boundary flips.  With
`bf16=False` everything is float64 (used to pin the backward pass against
finite differences).

Layout (shared with the CUDA kernels by specification, not by code):
  x  [B, 48]   genome bits, feature j = bit (35 - j) of the genome, 36..47 zero
  W1 [48, 256], b1 [256];  W2 [256, 256], b2 [256];  W3 [256, 8], b3 [8]
  h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), logits = h2 W3 + b3
  loss = mean over the batch of -log softmax(logits)[label]
"""
from __future__ import annotations

import numpy as np

D_IN, D_PAD, D_H, D_OUT = 36, 48, 256, 8


def bf16_round(a):
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def genome_bits(genomes):
    """[B] packed 36-bit genomes -> [B, 48] features (MSB first, zero padding)."""
    g = np.asarray(genomes, dtype=np.uint64)
    x = np.zeros((g.shape[0], D_PAD), np.float64)
    for j in range(D_IN):
        x[:, j] = ((g >> np.uint64(D_IN - 1 - j)) & np.uint64(1)).astype(np.float64)
    return x


def class_of(results):
    """8 phenotype classes from classification results: 0 unbounded, 1 local
    non-determinism, 2 steric non-determinism, 3..7 deterministic bounded of
    size 1, 2-3, 4-7, 8-15, >= 16."""
    cls = np.asarray(results["cls"]).astype(np.int64)
    size = np.asarray(results["size"]).astype(np.int64)
    out = np.where(cls == 3, 0, np.where(cls == 1, 1, np.where(cls == 2, 2, 0)))
    det = cls == 0
    bucket = np.where(size >= 16, 7, np.where(size >= 8, 6, np.where(size >= 4, 5, np.where(size >= 2, 4, 3))))
    return np.where(det, bucket, out).astype(np.int64)


def forward_backward(params, x, labels, *, bf16=True):
    """Loss and gradients (dict with the names of params) of the mean loss."""
    r = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    W1, b1, W2, b2, W3, b3 = (np.asarray(params[k], np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    B = x.shape[0]
    xq = r(x)
    W1q, W2q, W3q = r(W1), r(W2), r(W3)
    z1 = xq @ W1q + b1
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2q + b2
    h2 = r(np.maximum(z2, 0.0))
    logits = h2 @ W3q + b3
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    p = e / e.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(p[np.arange(B), labels])))
    d = p.copy()
    d[np.arange(B), labels] -= 1.0
    d /= B
    dq = r(d)
    gW3 = h2.T @ dq
    gb3 = d.sum(axis=0)
    dh2 = r((dq @ W3q.T) * (h2 > 0))
    gW2 = h1.T @ dh2
    gb2 = dh2.sum(axis=0)
    dh1 = r((dh2 @ W2q.T) * (h1 > 0))
    gW1 = xq.T @ dh1
    gb1 = dh1.sum(axis=0)
    return loss, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3}, logits


def magnitude_sums(params, x, labels, *, bf16=True):
    """For every gradient element and every logit, the sum of the absolute
    values of the terms of the dot product (plus bias) that forms it --
    sum_i |a_i b_i| -- from the same rounded operands as forward_backward.
    A floating-point sum of K terms differs from the exact one by at most
    about K * u * sum_i |a_i b_i| (u the unit roundoff), which is what the
    element-wise tolerances of the parity tests are built from."""
    r = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    W1, b1, W2, b2, W3, b3 = (np.asarray(params[k], np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    B = x.shape[0]
    xq = r(x)
    W1q, W2q, W3q = r(W1), r(W2), r(W3)
    h1 = r(np.maximum(xq @ W1q + b1, 0.0))
    h2 = r(np.maximum(h1 @ W2q + b2, 0.0))
    logits = h2 @ W3q + b3
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    p = e / e.sum(axis=1, keepdims=True)
    d = p.copy()
    d[np.arange(B), labels] -= 1.0
    d /= B
    dq = r(d)
    dh2 = r((dq @ W3q.T) * (h2 > 0))
    dh1 = r((dh2 @ W2q.T) * (h1 > 0))
    a = np.abs
    return {"logits": a(h2) @ a(W3q) + a(b3),
            "W3": a(h2).T @ a(dq), "b3": a(d).sum(axis=0),
            "W2": a(h1).T @ a(dh2), "b2": a(dh2).sum(axis=0),
            "W1": a(xq).T @ a(dh1), "b1": a(dh1).sum(axis=0)}


def predict(params, x, *, bf16=True):
    r = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    h1 = r(np.maximum(r(x) @ r(params["W1"]) + params["b1"], 0.0))
    h2 = r(np.maximum(h1 @ r(params["W2"]) + params["b2"], 0.0))
    return h2 @ r(params["W3"]) + params["b3"]


def init_params(seed=0):
    """He-scaled normal initialisation (any fixed values serve the parity tests)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((D_PAD, D_H)) * np.sqrt(2.0 / D_IN),
        "b1": np.zeros(D_H),
        "W2": rng.standard_normal((D_H, D_H)) * np.sqrt(2.0 / D_H),
        "b2": np.zeros(D_H),
        "W3": rng.standard_normal((D_H, D_OUT)) * np.sqrt(1.0 / D_H),
        "b3": np.zeros(D_OUT),
    }


def adam_step(params, grads, state, *, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) in place; state holds m, v and t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params
