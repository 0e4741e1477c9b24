"""The oracle's module-binned, map-driven search against an exhaustive all-pairs search.

The brute-force variant enumerates every ordered hit pair, every MD pair (testing module-map
membership by scanning the map row), every LS pair and T3 pair (testing the shared MD directly),
every (seed, T3/T5) pair (testing pixel-map membership) and every T5 pair in duplicate removal.
Both must give the same object sets and the same Track-Candidate list."""
import numpy as np
import pytest

import oracle
from paper_2207_08207_gb300 import gen


def key_sets(r):
    md = r["md"]

    def mdh(i):
        return (int(md["hit_lo"][i]), int(md["hit_up"][i]))
    out = {"md": {(mdh(i), bool(md["pass"][i])) for i in range(len(md["module"]))}}
    ls = r["ls"]
    out["ls"] = {(mdh(a) + mdh(b), bool(p)) for a, b, p in zip(ls["md_in"], ls["md_out"], ls["pass"])}
    t3 = r["t3"]
    t3k = [mdh(t3["md0"][i]) + mdh(t3["md1"][i]) + mdh(t3["md2"][i]) for i in range(len(t3["md0"]))]
    out["t3"] = {(k, bool(p)) for k, p in zip(t3k, t3["pass"])}
    t5 = r["t5"]
    t5k = [sum((mdh(t5[f"md{k}"][i]) for k in range(5)), ()) for i in range(len(t5["md0"]))]
    out["t5"] = {(k, bool(p)) for k, p in zip(t5k, t5["pass"])}
    out["pt3"] = {(int(p), t3k[o], bool(s)) for p, o, s in zip(r["pt3"]["pls"], r["pt3"]["obj"], r["pt3"]["pass"])}
    out["pt5"] = {(int(p), t5k[o], bool(s)) for p, o, s in zip(r["pt5"]["pls"], r["pt5"]["obj"], r["pt5"]["pass"])}
    tc = r["tc"]
    out["tc"] = [(int(tc["type"][i]),) + tuple(int(tc[f"hit{k}"][i]) for k in range(14)) for i in range(len(tc["type"]))]
    ext = r["tc_ext"]
    out["tc_ext"] = [(int(ext["n_add"][i]), t3k[ext["t3"][i]] if ext["t3"][i] >= 0 else None, bool(ext["definite"][i]))
                     + tuple(int(ext[f"hit{k}"][i]) for k in range(4)) for i in range(len(ext["t3"]))]
    return out


@pytest.mark.parametrize("seed", range(6))
def test_fifty_hit_events(seed):
    det, ev = gen.small_event(4, seed=100 + seed, noise_frac=0.05)
    assert 25 <= ev.n_hits <= 120
    a = key_sets(oracle.run(det, ev))
    b = key_sets(oracle.run(det, ev, brute_force=True))
    assert a == b


@pytest.mark.parametrize("seed", range(3))
def test_small_pu_events(seed):
    det, ev = gen.small_event(60, seed=200 + seed)
    a = key_sets(oracle.run(det, ev))
    b = key_sets(oracle.run(det, ev, brute_force=True))
    assert a == b
    assert len(a["t5"]) > 0 and len(a["pt3"]) > 0 and len(a["tc"]) > 0


def test_barrel_toy_event():
    det, ev = gen.config_event(1, 0)
    a = key_sets(oracle.run(det, ev))
    b = key_sets(oracle.run(det, ev, brute_force=True))
    assert a == b
