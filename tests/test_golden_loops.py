"""The stored full-loop values (tests/golden/wgs_full_loops.json) and the
sub-ulp ensemble behind them (CPU): the file was written by the committed
script from the oracle alone, every ensemble start rounds to the given
float32 phase, and the 2D array's loop is determined by its inputs to 2e-4."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_wgs_golden as mk  # noqa: E402


def test_sub_ulp_offsets_round_back_to_the_float32_phase():
    rng = np.random.default_rng(0)
    ph = np.concatenate([rng.uniform(0.0, 2 * np.pi, 100000), [0.0, 1e-30, 1.0, 2.0, 6.2831855]]).astype(np.float32)
    for seed in (1000, 1001):
        off = mk.sub_ulp_offset(ph, seed)
        assert np.all((ph.astype(np.float64) + off).astype(np.float32) == ph)
        assert np.any(off != 0.0)


def test_stored_full_loops():
    with open(mk.OUT) as f:
        g = json.load(f)
    assert "oracle" in g["_source"] and "make_wgs_golden.py" in g["_source"]
    c2, c3 = g["c2"], g["c3_sampled"]
    assert (c2["nx"], c2["ny"], c2["N"], c2["D"], c2["iters"], c2["pixels_summed"]) == (1024, 1024, 400, 10, 50,
                                                                                         1024 * 1024)
    assert (c3["nx"], c3["ny"], c3["N"], c3["D"], c3["iters"]) == (1920, 1152, 2000, 11, 100)
    assert c3["sample_frac"] == mk.C3_FRAC and c3["sample_seed"] == mk.C3_SEED
    for c in (c2, c3):
        assert len(c["history"]) == c["iters"]
        assert len(c["ensemble"]) >= 4
        assert sorted(e["seed"] for e in c["ensemble"]) == list(range(mk.ENSEMBLE_SEED0,
                                                                      mk.ENSEMBLE_SEED0 + len(c["ensemble"])))
        assert 0.0 < c["uniformity"] <= 1.0 and 0.0 < c["efficiency"] <= 1.0
    u2 = [c2["uniformity"]] + [e["uniformity"] for e in c2["ensemble"]]
    assert max(u2) - min(u2) <= 2e-4
