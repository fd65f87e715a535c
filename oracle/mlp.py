"""Reference for the learned quadrature order's network -- TEST INFRASTRUCTURE ONLY.

Plain numpy FP64 forward, softmax cross-entropy and backward of the 576 -> 64 -> 64 -> 6
ReLU network whose CUDA kernels the library provides.  Weights are rounded to FP16 for
the forward (as the kernels use them); the gradient with respect to the FP32 master
weights is the gradient with respect to the rounded weights (straight-through).
Parameter layout: W1 [576][64], b1 [64], W2 [64][64], b2 [64], W3 [64][6], b3 [6].
"""
from __future__ import annotations

import numpy as np

IN, H, C = 576, 64, 6
SIZES = [("W1", (IN, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, C)), ("b3", (C,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def fp16(a):
    return np.asarray(a, dtype=np.float32).astype(np.float16).astype(np.float64)


def forward(p, X, round_weights=True):
    """Hidden activations and logits for features X [B][576] (FP64 arithmetic)."""
    w = unpack(p)
    r = fp16 if round_weights else (lambda a: a)
    X = np.asarray(X, dtype=np.float64)
    H1 = np.maximum(X @ r(w["W1"]) + w["b1"], 0.0)
    H2 = np.maximum(H1 @ r(w["W2"]) + w["b2"], 0.0)
    Z = H2 @ r(w["W3"]) + w["b3"]
    return H1, H2, Z


def loss_and_grad(p, X, y, class_weight=None, round_weights=True):
    """Mean (class-weighted) softmax cross-entropy and its gradient (layout of p)."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y)
    B = X.shape[0]
    w = unpack(p)
    fp16 = globals()["fp16"] if round_weights else (lambda a: a)
    H1, H2, Z = forward(p, X, round_weights)
    m = Z.max(axis=1, keepdims=True)
    e = np.exp(Z - m)
    P = e / e.sum(axis=1, keepdims=True)
    cw = np.ones(C) if class_weight is None else np.asarray(class_weight, dtype=np.float64)
    sw = cw[y]
    loss = float(np.sum(sw * (np.log(e.sum(axis=1)) + m[:, 0] - Z[np.arange(B), y])) / B)
    dZ = P.copy()
    dZ[np.arange(B), y] -= 1.0
    dZ *= sw[:, None] / B
    g = {}
    g["W3"] = H2.T @ dZ
    g["b3"] = dZ.sum(axis=0)
    dH2 = (dZ @ fp16(w["W3"]).T) * (H2 > 0)
    g["W2"] = H1.T @ dH2
    g["b2"] = dH2.sum(axis=0)
    dH1 = (dH2 @ fp16(w["W2"]).T) * (H1 > 0)
    g["W1"] = X.T @ dH1
    g["b1"] = dH1.sum(axis=0)
    return loss, pack(g)


def softmax(Z):
    """Row-wise softmax of logits Z [B][C] (FP64)."""
    Z = np.asarray(Z, dtype=np.float64)
    e = np.exp(Z - Z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def ensemble_probs(params_list, X):
    """Class probabilities of an ensemble: the mean over its networks of their softmax outputs."""
    return np.mean([softmax(forward(p, X)[2]) for p in params_list], axis=0)


def risk_class(P, risk):
    """Class per row of probabilities P [B][C]: with risk > 0 the smallest class c whose higher
    classes c+1..C-1 hold at most `risk` of the probability (the last class if none does);
    with risk = 0 the most probable class."""
    P = np.asarray(P, dtype=np.float64)
    if risk <= 0:
        return P.argmax(axis=1)
    out = np.full(P.shape[0], P.shape[1] - 1)
    for i in range(P.shape[0]):
        above = 1.0
        for c in range(P.shape[1]):
            above -= P[i, c]
            if above <= risk:
                out[i] = c
                break
    return out
