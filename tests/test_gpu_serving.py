"""Serving on the GPU: events of uneven pile-up arrive as a Poisson stream, several contexts run
batches concurrently on separate streams, and every event's track candidates are identical to the
same event processed alone."""
import numpy as np
import pytest

from paper_2207_08207_gb300 import gen, lst
from paper_2207_08207_gb300.serving import Server, poisson_arrivals

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_served_results_equal_alone():
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    evs = [gen.config_event(5, e, pu=float(p))[1] for e, p in enumerate([60, 250, 120, 300, 80, 180, 140, 220])]
    evs = evs * 3   # 24 requests
    alone = lst.Context(det)
    ref = []
    for ev in evs[:8]:
        alone.run([ev])
        ref.append(alone.copy_tc(0))
    alone.close()
    srv = Server(det, n_engines=2, max_batch=5, max_hits=max(e.n_hits for e in evs),
                 max_pls=max(e.n_pls for e in evs), budget=8e9)
    stats, reqs = srv.serve(evs, poisson_arrivals(400.0, len(evs), seed=3))
    srv.close()
    assert stats.n == len(evs) and stats.batches >= 2
    assert stats.max_inflight_bytes <= 8e9
    for i, r in enumerate(reqs):
        a, b = ref[i % 8], r.result
        for k in ("type", "obj", "hits", "pt", "eta", "phi"):
            assert np.array_equal(a[k], b[k]), (i, k)
