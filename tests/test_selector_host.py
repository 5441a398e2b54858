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
