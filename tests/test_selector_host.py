"""Host-side logic of the selector module (no GPU): the Sec. 3
post-processing recovers thresholds planted in synthetic move records, and
the feature vector matches the oracle's definition."""
import math

import numpy as np

from oracle import mlp_oracle as M
from paper_2011_06636_gb300 import selector


def test_analysis_recovers_planted_thresholds():
    rng = np.random.default_rng(0)
    rec = []
    for _ in range(6000):
        r = rng.uniform(0, 1)
        lv = int(rng.integers(5, 15))
        best = 1 if r > 0.4 else (-1 if r > 0.2 else 0)
        for mv in (-1, 0, 1):
            rec.append((r, lv, mv, (0.01 if mv == best else 0.0) + rng.normal(0, 0.002)))
    out = selector.analyse(rec, n_set=60)
    assert 0.15 < out["keep_max_ratio"] < 0.2
    assert 0.2 < out["down_ratio_range"][0] and out["down_ratio_range"][1] < 0.4
    assert 0.4 < out["up_min_ratio"] < 0.45


def test_features_match_oracle_definition():
    hist = [math.log(0.5), math.log(0.3)]
    x = selector.features(hist, 4096 * 4096, 2, 17)
    ref = M.features([0.5, 0.3], 4096 * 4096, 2, 17)
    assert np.allclose(x, ref.astype(np.float32), rtol=0, atol=1e-7)


def test_bf16_conversion_matches_oracle():
    a = np.random.default_rng(1).standard_normal(5000).astype(np.float32)
    assert np.array_equal(selector.to_bf16_bits(a), M.bf16_bits(a))


def test_sec3_summary_fits_planted_thresholds():
    """sec3_summary on records whose best move switches at planted ratios
    0.26 and 0.58: Alg. 1's pair explains only part of the winners, the
    fitted pair lands on the planted one, and the rates are computed from the
    residual norms as Eq. average-convergence-rate states."""
    rng = np.random.default_rng(3)
    rows = []
    for _ in range(9000):
        r = rng.uniform(0, 1)
        lv = int(rng.integers(3, 12))
        best = 1 if r > 0.58 else (-1 if r > 0.26 else 0)
        for mv in (-1, 0, 1):
            rows.append((r, lv, mv, (0.01 if mv == best else 0.0) + rng.normal(0, 0.002)))
    out = selector.sec3_summary(np.asarray(rows), n_set=90)
    fit = out["best_fit_thresholds"]
    assert abs(fit["low"] - 0.26) <= 0.02 and abs(fit["high"] - 0.58) <= 0.02
    assert fit["agreement"] > 0.95
    assert out["alg1_agreement"] < fit["agreement"]
    # rates: -log(r_after / r_before) / M(level + action)
    dt = np.dtype([("prev_ratio", "<f8"), ("r_before", "<f8"), ("r_after", "<f8"),
                   ("level", "<i4"), ("action", "<i4")])
    rec = np.array([(0.5, 2.0, 1.0, 3, 1), (0.5, 1.0, 0.25, 0, 0)], dtype=dt)
    np.testing.assert_allclose(selector.sec3_rates(rec), [math.log(2) / 7, math.log(4) / 1])
