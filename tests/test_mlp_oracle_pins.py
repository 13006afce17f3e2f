"""Pins for the cost-model oracle (oracle/mlp.py), against things other than
its own code: central finite differences of the loss, closed forms, Adam's
first step, and planted mistakes in the backward pass."""
import numpy as np
import pytest

from oracle import mlp


def data(n=7, seed=1):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 20)), rng.normal(size=(n, 2))


def fd_grad(theta, X, T, h=1e-6):
    g = np.zeros_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        lp = mlp.loss(mlp.forward(theta + e, X)[0], T)
        lm = mlp.loss(mlp.forward(theta - e, X)[0], T)
        g[i] = (lp - lm) / (2 * h)
    return g


def test_parameter_count():
    assert mlp.n_params() == 20 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2 == 5634


def test_gradient_matches_central_differences():
    X, T = data()
    theta = mlp.init(3)
    Y, cache = mlp.forward(theta, X)
    g = mlp.backward(theta, cache, Y, T)
    np.testing.assert_allclose(g, fd_grad(theta, X, T), rtol=1e-5, atol=1e-8)


def test_zero_hidden_weights_give_bias_output():
    p = mlp.unflatten(mlp.init(0))
    for k in ("W1", "W2", "b1", "b2"):
        p[k] = np.zeros_like(p[k])
    p["b3"] = np.array([1.5, -2.0])
    theta = mlp.flatten(p)
    X, T = data()
    Y, cache = mlp.forward(theta, X)
    np.testing.assert_allclose(Y, np.tile([1.5, -2.0], (len(X), 1)))
    g = mlp.unflatten(mlp.backward(theta, cache, Y, T))
    np.testing.assert_allclose(g["b3"], (Y - T).mean(axis=0))   # d/db of the mean half squared error
    np.testing.assert_allclose(g["W3"], 0.0)


def test_hand_worked_single_sample():
    """x = e_0; W1 row j = delta_j0 so Z1 = e_0; W2 = identity on unit 0;
    W3 picks unit 0 into output 0 with weight 2. Then y = (2 + b3_0, b3_1)."""
    p = {k: np.zeros(s) for k, s in zip(mlp.NAMES, mlp.shapes())}
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["W3"][0, 0] = 2.0
    p["b3"][:] = [0.25, 0.5]
    x = np.zeros((1, 20))
    x[0, 0] = 1.0
    Y, _ = mlp.forward(mlp.flatten(p), x)
    np.testing.assert_allclose(Y, [[2.25, 0.5]])
    x[0, 0] = -1.0   # the ReLU cuts it
    Y, _ = mlp.forward(mlp.flatten(p), x)
    np.testing.assert_allclose(Y, [[0.25, 0.5]])


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    th, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), atol=1e-9)


def test_training_fits_a_linear_target():
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 1, size=(512, 20))
    T = np.stack([X[:, :5].sum(1), 2 * X[:, 5] - X[:, 6]], axis=1)
    theta = mlp.init(9)
    l0 = mlp.loss(mlp.forward(theta, X)[0], T)
    theta = mlp.train(theta, X, T, epochs=60, lr=3e-3, batch=64, seed=1)
    l1 = mlp.loss(mlp.forward(theta, X)[0], T)
    assert l1 < 0.02 * l0


PLANTS = {
    "relu mask dropped": lambda s: s.replace("* (Z2 > 0)", ""),
    "transposed weight": lambda s: s.replace('dZ1 = (dZ2 @ p["W2"])', 'dZ1 = (dZ2 @ p["W2"].T)'),
    "missing 1/N": lambda s: s.replace("dY = (Y - T) / N", "dY = (Y - T)"),
    "bias sums wrong axis": lambda s: s.replace('g["b2"] = dZ2.sum(axis=0)', 'g["b2"] = dZ2.sum(axis=0) * 0.5'),
}


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_backward_mistakes_fail_fd(name):
    import inspect
    import types
    src = inspect.getsource(mlp)
    bad = PLANTS[name](src)
    assert bad != src
    mod = types.ModuleType("mlp_bad")
    exec(compile(bad, "mlp_bad", "exec"), mod.__dict__)
    X, T = data()
    theta = mlp.init(3)
    Y, cache = mod.forward(theta, X)
    g = mod.backward(theta, cache, Y, T)
    assert not np.allclose(g, fd_grad(theta, X, T), rtol=1e-5, atol=1e-8)
