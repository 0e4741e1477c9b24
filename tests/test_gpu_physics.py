"""Physics metrics (paper Sec. 3) on the CUDA library's track candidates: the same counts as on the
oracle's candidates for the same events, the turn-on at the 0.8 GeV threshold and the plateau."""
import numpy as np
import pytest

import oracle
from paper_2207_08207_gb300 import gen, lst, physics

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_library_tcs_give_oracle_rates():
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    evs = [gen.small_event(1200, seed=500 + s, pt_min=0.4)[1] for s in range(3)] + [gen.config_event(2, 1)[1]]
    ctx = lst.Context(det)
    ctx.run(evs)
    cg, co = physics.Counts(), physics.Counts()
    for e, ev in enumerate(evs):
        tc = ctx.copy_tc(e)
        cg.add(ev, tc["type"], tc["hits"])
        r = oracle.run(det, ev)["tc"]
        co.add(ev, r["type"], np.stack([r[f"hit{k}"] for k in range(14)], axis=1))
    ctx.close()
    for f in ("eff_pt_num", "eff_pt_den", "eff_eta_num", "eff_eta_den", "eff_pt_by_type", "n_tc_type",
              "n_fake_type", "n_dup_type"):
        assert np.array_equal(getattr(cg, f), getattr(co, f)), f
    s = cg.summary()
    b = np.array(s["pt_bins"][:-1])
    eff, den = np.array(s["eff_pt"]), np.array(s["eff_pt_den"])
    assert np.all(eff[(b < 0.7) & (den > 0)] < 0.05)
    assert np.all(eff[(b >= 0.8) & (den > 20)] > 0.95)
    assert s["fake_rate"] < 0.01 and s["duplicate_rate"] < 0.1
