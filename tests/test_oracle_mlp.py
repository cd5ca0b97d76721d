"""Pins of the cost model's fp64 oracle (oracle/mlp.py) to facts outside it:
finite differences, a network computed by hand, a closed-form least-squares
optimum, and the first Adam step."""
import numpy as np

from oracle import mlp


def random_theta(rng, scale=0.3):
    return rng.normal(0.0, scale, size=mlp.N_PARAMS)


def test_layout_has_4801_parameters():
    assert mlp.N_PARAMS == 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1 == 4801
    theta = np.arange(mlp.N_PARAMS, dtype=np.float64)
    assert np.array_equal(mlp.pack(mlp.unpack(theta)), theta)
    p = mlp.unpack(theta)
    assert p["W1"][1, 0] == 8 and p["b1"][0] == 512 and p["W2"][0, 1] == 577
    assert p["b3"][0] == 4800


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    theta = random_theta(rng)
    X = rng.normal(size=(23, 8))
    y = rng.normal(size=23)
    L, g = mlp.gradient(theta, X, y)
    assert abs(L - mlp.loss(theta, X, y)) < 1e-12
    # every bias and output weight, and a sample of the hidden weights
    idx = np.concatenate([np.arange(512, 576), np.arange(4672, 4801),
                          rng.choice(512, 40, replace=False),
                          576 + rng.choice(4096, 80, replace=False)])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.loss(theta + e, X, y) - mlp.loss(theta - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_gradient_catches_a_planted_sign_error():
    # the same check must fail for a wrong gradient: flip the sign of dW2
    rng = np.random.default_rng(6)
    theta = random_theta(rng)
    X = rng.normal(size=(9, 8))
    y = rng.normal(size=9)
    _, g = mlp.gradient(theta, X, y)
    bad = g.copy()
    bad[576:576 + 4096] *= -1
    i = 576 + int(np.argmax(np.abs(g[576:576 + 4096])))
    e = np.zeros(mlp.N_PARAMS)
    e[i] = 1e-6
    fd = (mlp.loss(theta + e, X, y) - mlp.loss(theta - e, X, y)) / 2e-6
    assert abs(fd - g[i]) < 1e-6 and abs(fd - bad[i]) > 1e-4


def test_one_live_path_by_hand():
    # only W1[0,2], W2[0,0], w3[0] and the biases are non-zero
    parts = {name: np.zeros(shape) for name, shape in mlp.SIZES}
    parts["W1"][0, 2] = 1.5
    parts["b1"][0] = -0.5
    parts["W2"][0, 0] = 2.0
    parts["b2"][0] = 0.25
    parts["w3"][0] = -3.0
    parts["b3"][0] = 0.125
    theta = mlp.pack(parts)
    X = np.zeros((3, 8))
    X[:, 2] = [1.0, 0.2, 2.0]   # z1 = 1.0, -0.2 (dead), 2.5
    f, _ = mlp.forward(theta, X)
    # h1 = 1.0, 0, 2.5 ; h2 = 2.25, 0.25, 5.25 ; f = -3 h2 + 0.125
    assert np.allclose(f, [-6.625, -0.625, -15.625], rtol=0, atol=1e-15)
    # negative inputs to the ReLUs everywhere else: the other units add nothing
    assert np.count_nonzero(mlp.forward(theta, X)[1][1][:, 1:]) == 0


def test_linear_regime_reaches_the_least_squares_optimum():
    # With W1 = [I; -I] (unit j sees x_j or -x_j) and W2 = identity on those
    # units, every hidden unit passes its input through, relu(x) and relu(-x)
    # together carry x, and f is linear in x: the loss as a function of the
    # output weights is least squares, whose minimum is known in closed form.
    rng = np.random.default_rng(7)
    X = rng.normal(size=(200, 8))
    beta = rng.normal(size=8)
    y = X @ beta + 0.3 + 0.01 * rng.normal(size=200)
    parts = {name: np.zeros(shape) for name, shape in mlp.SIZES}
    for j in range(8):
        parts["W1"][j, j] = 1.0
        parts["W1"][8 + j, j] = -1.0
    for j in range(16):
        parts["W2"][j, j] = 1.0
    A = np.hstack([X, np.ones((200, 1))])
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    best = float(np.mean((A @ coef - y) ** 2))
    parts["w3"][:8] = coef[:8]
    parts["w3"][8:16] = -coef[:8]
    parts["b3"][0] = coef[8]
    theta = mlp.pack(parts)
    assert abs(mlp.loss(theta, X, y) - best) < 1e-12
    L, g = mlp.gradient(theta, X, y)
    # the normal equations: along w3[j] - w3[8 + j] (which moves f by x_j)
    # and along b3 the gradient vanishes at the optimum
    gw3 = g[4736:4800]
    assert np.max(np.abs(gw3[:8] - gw3[8:16])) < 1e-10
    assert abs(g[4800]) < 1e-10
    # the other output weights see dead units
    assert np.max(np.abs(gw3[16:])) == 0.0


def test_first_adam_step_moves_by_lr_sign():
    rng = np.random.default_rng(8)
    theta = rng.normal(size=mlp.N_PARAMS)
    g = rng.normal(size=mlp.N_PARAMS)
    lr, eps = 1e-3, 1e-8
    t1, m, v = mlp.adam_step(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr, eps=eps)
    # m^ = g and v^ = g^2 after one step
    assert np.allclose(theta - t1, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps the step at lr * sign(g) (m^ = g, v^ = g^2)
    t2, m, v = mlp.adam_step(t1, g, m, v, 2, lr, eps=0.0)
    assert np.allclose(t1 - t2, lr * np.sign(g), rtol=1e-12, atol=0)


def test_regret_definition():
    assert mlp.regret([3.0, 1.0, 2.0], [10.0, 12.0, 11.0]) == 12.0 / 10.0 - 1
    assert mlp.regret([0.0, 1.0], [5.0, 6.0]) == 0.0
