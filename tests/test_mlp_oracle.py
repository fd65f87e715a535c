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


def test_risk_rule_hand_cases():
    """The risk rule on probabilities worked by hand: tail sums after classes 0, 1, 2, ... are
    0.5, 0.2, 0.05, 0.01, 0.001, 0."""
    P = np.array([[0.5, 0.3, 0.15, 0.04, 0.009, 0.001]])
    assert mlp.risk_class(P, 0.0)[0] == 0          # argmax
    assert mlp.risk_class(P, 0.3)[0] == 1          # 0.2 <= 0.3
    assert mlp.risk_class(P, 0.05 + 1e-12)[0] == 2
    assert mlp.risk_class(P, 0.02)[0] == 3
    assert mlp.risk_class(P, 0.002)[0] == 4
    assert mlp.risk_class(P, 1e-6)[0] == 5         # only the last class leaves nothing above
    # a sharper distribution needs fewer classes at the same risk
    assert mlp.risk_class(np.array([[0.0, 0.999, 0.001, 0, 0, 0]]), 0.002)[0] == 1


def test_ensemble_probabilities():
    """One network alone is its softmax; identical members change nothing; the mean does not
    depend on the members' order and is a probability distribution."""
    rng = np.random.default_rng(3)
    X = rng.normal(0, 1, (7, mlp.IN))
    ps = [rng.normal(0, 0.1, mlp.NPARAMS) for _ in range(3)]
    one = mlp.softmax(mlp.forward(ps[0], X)[2])
    assert np.allclose(mlp.ensemble_probs([ps[0]], X), one, rtol=0, atol=1e-15)
    assert np.allclose(mlp.ensemble_probs([ps[0], ps[0]], X), one, rtol=0, atol=1e-15)
    a = mlp.ensemble_probs(ps, X)
    assert np.allclose(a, mlp.ensemble_probs(ps[::-1], X), rtol=0, atol=1e-15)
    assert np.allclose(a.sum(axis=1), 1.0) and (a > 0).all()
    manual = sum(mlp.softmax(mlp.forward(p, X)[2]) for p in ps) / 3
    assert np.allclose(a, manual, rtol=0, atol=1e-15)
