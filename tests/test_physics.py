"""Physics metrics on simulation truth (paper Sec. 3), computed on the oracle's track candidates:
the 75 % hit-matching rule on hand-made rows, the efficiency turn-on at the 0.8 GeV threshold and
its plateau above 1 GeV, and small fake and duplicate rates on PU200-like events."""
import numpy as np
import pytest

import oracle
from paper_2207_08207_gb300 import gen, physics


def _rows(r):
    tc = r["tc"]
    return tc["type"], np.stack([tc[f"hit{k}"] for k in range(14)], axis=1)


def test_matching_rule():
    lut = np.array([0] * 20 + [1] * 20 + [-1] * 5)   # hits 0-19 particle 0, 20-39 particle 1, noise
    rows = np.full((6, 14), -1)
    rows[0, :10] = list(range(8)) + [20, 21]            # 8 of 10: matched to 0
    rows[1, :10] = list(range(7)) + [20, 21, 22]        # 7 of 10: fake
    rows[2, :14] = list(range(11)) + [20, 21, 40]       # 11 of 14 (0.79): matched
    rows[3, :14] = list(range(10)) + [20, 21, 40, 41]   # 10 of 14 (0.71): fake
    rows[4, :4] = [20, 21, 22, 23]                      # a 4-hit row of particle 1
    rows[5, :4] = [40, 41, 42, 43]                      # noise only: fake
    assert physics.match_tcs(rows, lut).tolist() == [0, -1, 0, -1, 1, -1]


def test_rates_count_duplicates_and_fakes():
    ev = gen.Event(x=np.zeros(40, np.float32), y=np.zeros(40, np.float32), z=np.zeros(40, np.float32),
                   sensor=np.zeros(40, np.int32), pls=np.zeros(0, dtype=gen.PLS_DTYPE),
                   hit_particle=np.array([0] * 20 + [1] * 20, np.int32), pls_particle=np.zeros(0, np.int32),
                   particles=dict(pt=np.array([2.0, 0.5, 3.0]), eta=np.array([0.1, -0.2, 1.0])))
    rows = np.full((3, 14), -1)
    rows[0, :10] = range(10)
    rows[1, :10] = range(5, 15)        # a second TC of particle 0: both are duplicates
    rows[2, :10] = list(range(20, 24)) + list(range(10, 16))   # mixed: fake
    c = physics.Counts()
    c.add(ev, np.array([2, 2, 2]), rows)
    s = c.summary()
    assert s["n_tc"] == 3 and abs(s["fake_rate"] - 1 / 3) < 1e-12 and abs(s["duplicate_rate"] - 2 / 3) < 1e-12
    i2 = int(np.digitize(2.0, physics.PT_BINS)) - 1
    assert s["eff_pt_den"][i2] == 1 and s["eff_pt"][i2] == 1.0
    i05 = int(np.digitize(0.5, physics.PT_BINS)) - 1
    assert s["eff_pt"][i05] == 0.0


@pytest.fixture(scope="module")
def low_pt_counts():
    c = physics.Counts()
    for seed in range(3):
        det, ev = gen.small_event(1200, seed=500 + seed, pt_min=0.4)
        c.add(ev, *_rows(oracle.run(det, ev)))
    return c.summary()


def test_turn_on_at_threshold(low_pt_counts):
    s = low_pt_counts
    b = np.array(s["pt_bins"][:-1])
    eff = np.array(s["eff_pt"])
    den = np.array(s["eff_pt_den"])
    below = (b < 0.7) & (den > 0)
    assert np.all(eff[below] < 0.05), eff[below]
    above = (b >= 0.8) & (den > 20)
    assert np.all(eff[above] > 0.95), eff[above]
    assert s["eff_above_1gev"] > 0.97
    assert s["fake_rate"] < 0.01 and s["duplicate_rate"] < 0.1


def test_pu200_rates():
    c = physics.Counts()
    det, ev = gen.config_event(2, 0)
    c.add(ev, *_rows(oracle.run(det, ev)))
    s = c.summary()
    assert s["eff_above_1gev"] > 0.95
    assert all(e > 0.9 for e in s["eff_eta"])
    assert s["fake_rate"] < 0.01
    assert s["duplicate_rate"] < 0.1
