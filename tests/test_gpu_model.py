"""GPU parity of the learned cost model's kernels (mlp_forward_kernel,
mlp_grad_kernel, mlp_reduce_kernel) against the fp64 oracle (oracle/mlp.py),
and what the trained network gains over the method without it."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import mlp as O  # noqa: E402


@pytest.fixture(scope="module")
def cm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1405_5483_gb300 import build_lib
    build_lib.build()
    from paper_1405_5483_gb300 import cost_model
    return cost_model


def setup_model(cm, rng, scale=0.3):
    theta = (rng.normal(0.0, scale, size=4801)).astype(np.float32)
    mean = rng.normal(size=8).astype(np.float32)
    std = rng.uniform(0.5, 2.0, size=8).astype(np.float32)
    om, osd = np.float32(-0.7), np.float32(1.3)
    model = cm.Model(0)
    model.params = theta
    model.set_norm(mean, std, om, osd)
    return model, theta.astype(np.float64), mean, std, float(om), float(osd)


def test_forward_matches_oracle(cm):
    rng = np.random.default_rng(11)
    model, theta, mean, std, om, osd = setup_model(cm, rng)
    X = (rng.normal(size=(1000, 8)) * std + mean).astype(np.float32)   # 7 blocks + a tail
    got = model.predict(X)
    f, _ = O.forward(theta, O.standardise(X, mean, std))
    want = om + osd * f
    assert np.max(np.abs(got - want) / (1.0 + np.abs(want))) < 1e-5
    # device in, device out; and the empty call
    gd = model.predict(torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.array_equal(gd, got)
    assert model.predict(np.zeros((0, 8), np.float32)).size == 0


@pytest.mark.parametrize("N", [1, 64, 1000])
def test_gradient_matches_oracle(cm, N):
    rng = np.random.default_rng(N)
    model, theta, mean, std, om, osd = setup_model(cm, rng)
    X = (rng.normal(size=(N, 8)) * std + mean).astype(np.float32)
    y = (om + osd * rng.normal(size=N)).astype(np.float32)
    L, g = model.loss_grad(X, y)
    Lo, go = O.gradient(theta, O.standardise(X, mean, std), (y - om) / osd)
    assert abs(L - Lo) <= 1e-5 * max(1.0, Lo)
    scale = np.max(np.abs(go))
    assert np.max(np.abs(g - go)) <= 2e-5 * scale + 1e-7
    # every block of the layout is exercised (no silently zero gradient)
    for a, b in [(0, 512), (512, 576), (576, 4672), (4672, 4736), (4736, 4800), (4800, 4801)]:
        assert np.any(g[a:b] != 0)


def test_adam_steps_match_oracle(cm):
    rng = np.random.default_rng(21)
    model, theta, *_ = setup_model(cm, rng)
    m = np.zeros(4801)
    v = np.zeros(4801)
    for t in (1, 2):
        g = rng.normal(size=4801).astype(np.float32)
        model.adam_step(g, lr=1e-2, eps=1e-3)
        theta, m, v = O.adam_step(theta, g.astype(np.float64), m, v, t, 1e-2, eps=1e-3)
        assert np.max(np.abs(model.params - theta)) < 1e-6


def test_full_batch_training_equals_oracle_adam(cm):
    # one batch of all samples: each epoch is one Adam step on the full gradient
    rng = np.random.default_rng(31)
    model, theta, mean, std, om, osd = setup_model(cm, rng, scale=0.2)
    X = (rng.normal(size=(300, 8)) * std + mean).astype(np.float32)
    y = (om + osd * rng.normal(size=300)).astype(np.float32)
    losses = model.train(X, y, epochs=3, batch=300, lr=1e-3, eps=1e-3, seed=5)
    Xs, ys = O.standardise(X, mean, std), (y - om) / osd
    m = np.zeros(4801)
    v = np.zeros(4801)
    want_losses = []
    for t in (1, 2, 3):
        L, g = O.gradient(theta, Xs, ys)
        want_losses.append(L)
        theta, m, v = O.adam_step(theta, g, m, v, t, 1e-3, eps=1e-3)
    assert np.allclose(losses, want_losses, rtol=1e-5)
    assert np.max(np.abs(model.params - theta)) < 1e-5


def test_training_is_deterministic_and_learns(cm, tmp_path):
    rng = np.random.default_rng(41)
    X = rng.normal(size=(3000, 8)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] + 0.1 * X[:, 3]).astype(np.float32)
    runs = []
    for _ in range(2):
        model = cm.Model(3)
        model.fit_norm(X, y)
        losses = model.train(X, y, epochs=30, batch=128, lr=2e-3, seed=9)
        runs.append((model.params, losses, model))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    losses = runs[0][1]
    assert losses[-1] < 0.1 * losses[0]
    # the checkpoint carries the trained network
    model = runs[0][2]
    path = str(tmp_path / "m.bin")
    model.save(path)
    again = cm.Model.load(path)
    assert np.array_equal(again.predict(X[:100]), model.predict(X[:100]))


def test_choose_is_the_argmin_over_the_grid(cm):
    rng = np.random.default_rng(51)
    model, *_ = setup_model(cm, rng, scale=0.1)
    P = rng.integers(0x20, 0x7F, size=(200, 16)).astype(np.uint8)
    best, pred = model.choose(P, 95, 5.2, 1 << 22)
    g = cm.grid(P, 95)
    X = cm.features(95, 5.2, 16, 200, 1 << 22, [p for p, _ in g])
    y = model.predict(X)
    i = int(np.argmin(y))
    assert abs(pred - y[i]) < 1e-6
    assert {k: best[k] for k in ("q", "sigma_r", "k", "map_kind")} == \
        {k: g[i][0][k] for k in ("q", "sigma_r", "k", "map_kind")}


def test_trained_model_regret_and_gain(cm):
    """Train on the timing database's training sets with the library's own
    kernels; on the 200 held-out config-4-shaped sets the chosen parameters
    stay within 5% of the exhaustive tuner's best on average and beat the
    library's analytical default."""
    if not os.path.exists(cm.DB_PATH):
        pytest.skip("no timing database")
    db = cm.load_db()
    model, losses = cm.train_model(db)
    assert losses[-1] < losses[0]
    ev = cm.evaluate(model.predict, db)
    assert ev["sets"] >= 150
    assert ev["mean_regret"] <= 0.05, ev
    assert ev["geomean_speedup_over_default"] > 1.0, ev
