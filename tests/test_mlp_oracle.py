"""Pins of the reference MLP (CPU): central finite differences of the loss, and the
softmax cross-entropy against its definition on a one-sample case."""
import numpy as np

from oracle import mlp


def small_problem(seed=0, B=5):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.1, mlp.NPARAMS)
    X = rng.normal(0, 1, (B, mlp.IN))
    y = rng.integers(0, mlp.C, B)
    return p, X, y


def test_gradient_matches_finite_differences():
    p, X, y = small_problem()
    cw = np.array([1.0, 2.0, 0.5, 1.5, 1.0, 3.0])
    loss, g = mlp.loss_and_grad(p, X, y, cw, round_weights=False)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(mlp.NPARAMS, 60, replace=False), np.arange(mlp.NPARAMS - 400, mlp.NPARAMS, 7)])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, y, cw, round_weights=False)[0] -
              mlp.loss_and_grad(pm, X, y, cw, round_weights=False)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_cross_entropy_definition_one_sample():
    p, X, y = small_problem(2, 1)
    _, _, Z = mlp.forward(p, X)
    z = Z[0]
    ref = -np.log(np.exp(z[y[0]]) / np.exp(z).sum())
    loss, _ = mlp.loss_and_grad(p, X, y)
    assert abs(loss - ref) < 1e-12


def test_forward_rounds_weights_to_fp16():
    p, X, y = small_problem(3, 2)
    p[:10] = 0.1  # 0.1 is not representable in FP16
    _, _, Z1 = mlp.forward(p, X, True)
    _, _, Z2 = mlp.forward(p, X, False)
    assert np.abs(Z1 - Z2).max() > 0
    w = mlp.unpack(p)
    assert mlp.fp16(w["W1"])[0, 0] == np.float64(np.float16(0.1))
