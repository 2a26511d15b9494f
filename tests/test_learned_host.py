"""Host logic of the learned propagator's driver: blob layout, constant and initial networks,
feature standardisation (no GPU)."""
import numpy as np

from oracle import learned as L
from paper_1505_07959_gb300 import fa, learned as LG


def test_blob_layout_is_the_oracles():
    lay = LG.blob_layout()
    p = L.init_params(2)
    blob = L.to_blob(p)
    for k, (off, shape) in lay.items():
        assert np.array_equal(blob[off:off + int(np.prod(shape))].reshape(shape),
                              np.asarray(p[k], dtype=np.float32)), k


def test_constant_blob_outputs_its_constant():
    blob = LG.constant_blob([0.5, 1.5, -2.0, 3.0])
    c, _ = L.forward(L.deployed(L.from_blob(blob)), np.random.default_rng(0).standard_normal((5, 8)))
    assert np.array_equal(c, np.tile([0.5, 1.5, -2.0, 3.0], (5, 1)))


def test_init_blob_starts_at_the_taylor_step():
    blob = LG.init_blob(np.arange(8.0), np.full(8, 2.0), seed=1)
    q = L.from_blob(blob)
    assert np.array_equal(q["mu"], np.arange(8.0)) and np.array_equal(q["sd"], np.full(8, 2.0))
    c, _ = L.forward(L.deployed(q), np.random.default_rng(0).standard_normal((3, 8)))
    assert np.array_equal(c, np.ones((3, 4)))
    assert np.std(q["W2"]) > 0.05


def test_standardisation_keeps_constant_features_finite():
    rec = np.zeros((10, fa.FA_RECORD_DOUBLES))
    rec[:, 0] = np.arange(10) / 10
    rec[:, 1] = 1 / 64                        # constant dT
    mu, sd = LG.standardisation(rec)
    assert abs(mu[0] - 0.45) < 1e-15 and sd[1] == 1.0 and np.all(np.isfinite(sd)) and np.all(sd > 0)


def test_log_uniform_sizes_are_seeded_and_in_range():
    a = LG.log_uniform_sizes(200, 256, 1024, 3)
    assert a == LG.log_uniform_sizes(200, 256, 1024, 3)
    assert min(a) >= 256 and max(a) <= 1024
    assert 0.3 < np.mean(np.array(a) < 512) < 0.7        # log-uniform: median near 512
