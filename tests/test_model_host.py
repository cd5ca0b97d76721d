"""Host-side parts of the learned cost model (no GPU): the parameter grid,
the feature vector, initialisation, and checkpoints."""
import math
import os

import numpy as np
import pytest

from paper_1405_5483_gb300 import build_lib


@pytest.fixture(scope="module")
def cm():
    build_lib.build()
    from paper_1405_5483_gb300 import cost_model
    return cost_model


def printable_set(rng, r, m):
    return rng.integers(0x20, 0x7F, size=(r, m)).astype(np.uint8)


@pytest.mark.parametrize("r,m", [(10, 8), (300, 16), (2000, 32), (50, 64)])
def test_grid_points_are_feasible_and_inside_the_grid(cm, r, m):
    import paper_1405_5483_gb300 as mpm
    P = printable_set(np.random.default_rng(r + m), r, m)
    g = cm.grid(P, 95)
    assert len(g) > 0
    seen = set()
    for p, info in g:
        key = (p["q"], p["sigma_r"], p["k"], p["map_kind"])
        assert key not in seen
        seen.add(key)
        assert 1 <= p["k"] <= 8 and info["positions"] <= 32
        assert info["table_bytes"] <= 16 << 20
        if p["map_kind"] == mpm.MAP_QHASH:
            assert 2 <= p["q"] <= 5 and p["sigma_r"] in (1 << 12, 1 << 14, 1 << 16)
        else:
            assert 2 <= p["q"] <= 6 and p["sigma_r"] in (2, 4, 8, 16)
        # the planner accepts the point as given and reports the same sizes
        p2, info2 = mpm.plan(P, 95, **p)
        assert (p2["q"], p2["sigma_r"], p2["k"], p2["map_kind"]) == key
        assert info2["positions"] == info["positions"]
    # m = 8 admits q <= 4 only (one non-overlapping q-gram per shift needs 2q - 1 <= m)
    if m == 8:
        assert max(p["q"] for p, _ in g) <= 4


def test_features_layout(cm):
    ps = [dict(q=3, sigma_r=16, k=2, map_kind=2), dict(q=4, sigma_r=1 << 16, k=1, map_kind=4)]
    X = cm.features(95, 5.25, 32, 1000, 1 << 22, ps)
    want = np.array([[95, 5.25, 5, 3, 22, 3, 4, 2], [95, 5.25, 5, 3, 22, 4, 16, 1]], np.float32)
    assert X.dtype == np.float32 and np.allclose(X, want, rtol=1e-6, atol=1e-6)


def test_model_initialisation_is_seeded_he_uniform(cm):
    a, b, c = cm.Model(7).params, cm.Model(7).params, cm.Model(8).params
    assert a.size == 4801 and np.array_equal(a, b) and not np.array_equal(a, c)
    w1, b1, w2, b2, w3, b3 = a[:512], a[512:576], a[576:4672], a[4672:4736], a[4736:4800], a[4800]
    assert np.all(np.abs(w1) <= math.sqrt(6 / 8)) and np.all(np.abs(w2) <= math.sqrt(6 / 64))
    assert np.all(np.abs(w3) <= math.sqrt(6 / 64))
    assert not np.any(b1) and not np.any(b2) and b3 == 0
    # uniform: the spread fills the bound (not all near zero)
    assert np.abs(w2).max() > 0.9 * math.sqrt(6 / 64)
    mean, std, om, osd = cm.Model(7).norm
    assert np.all(mean == 0) and np.all(std == 1) and om == 0 and osd == 1


def test_params_norm_and_checkpoint_round_trip(cm, tmp_path):
    rng = np.random.default_rng(3)
    m = cm.Model(1)
    theta = rng.normal(size=4801).astype(np.float32)
    m.params = theta
    assert np.array_equal(m.params, theta)
    m.set_norm(np.arange(8) * 0.5, np.arange(1, 9) * 0.25, -1.5, 2.0)
    path = str(tmp_path / "model.bin")
    m.save(path)
    assert os.path.getsize(path) == 8 + 4 + 20 * 4 + 8 + 3 * 4801 * 4
    m2 = cm.Model.load(path)
    assert np.array_equal(m2.params, theta)
    mean, std, om, osd = m2.norm
    assert np.allclose(mean, np.arange(8) * 0.5) and np.allclose(std, np.arange(1, 9) * 0.25)
    assert om == -1.5 and osd == 2.0


def test_bad_norm_and_bad_checkpoint_are_rejected(cm, tmp_path):
    import paper_1405_5483_gb300 as mpm
    m = cm.Model(1)
    with pytest.raises(mpm.MpmError):
        m.set_norm(np.zeros(8), np.zeros(8), 0.0, 1.0)
    with pytest.raises(mpm.MpmError):
        m.set_norm(np.zeros(8), np.ones(8), 0.0, -1.0)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a model at all")
    with pytest.raises(mpm.MpmError):
        cm.Model.load(str(bad))
    with pytest.raises(mpm.MpmError):
        cm.Model.load(str(tmp_path / "missing.bin"))


def test_committed_model_regret_on_heldout_sets(cm):
    """The committed network (trained on the GPU by the library's kernels on
    the timing database's 200 training sets), evaluated through the fp64
    oracle's forward pass: on the 200 held-out config-4-shaped sets its
    choice is within 5% of the best grid point on average and faster than
    the library's analytical default."""
    from oracle import mlp
    if not (os.path.exists(cm.DB_PATH) and os.path.exists(cm.MODEL_PATH)):
        pytest.skip("no committed timing database or model")
    db = cm.load_db()
    model = cm.Model.load()
    theta = model.params.astype(np.float64)
    mean, std, om, osd = model.norm

    def predict(X):
        f, _ = mlp.forward(theta, mlp.standardise(X, mean, std))
        return om + osd * f

    ev = cm.evaluate(predict, db)
    assert ev["sets"] == 200
    assert ev["mean_regret"] <= 0.05, ev
    assert ev["geomean_speedup_over_default"] > 1.0, ev
    # the training and held-out sets do not overlap
    assert not set(cm.TRAIN_SETS) & set(cm.HELDOUT_SETS)
