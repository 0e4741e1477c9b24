"""The multi-stream plain path (paper Sec. 4.2.2): events processed concurrently by N one-event
contexts on their own CUDA streams give, event by event, exactly the objects of one context running
them one at a time (and match the oracle on a sampled event)."""
import numpy as np
import pytest

import oracle
from paper_2207_08207_gb300 import gen, lst
from paper_2207_08207_gb300.streams import MultiStream
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("n_streams", [2, 4])
def test_streams_equal_single_runs(n_streams):
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    evs = [gen.config_event(3, e)[1] for e in range(6)] + [gen.small_event(300, seed=40 + k)[1] for k in range(3)]
    single = lst.Context(det)
    ref = []
    for ev in evs:
        single.run([ev])
        ref.append(single.results(0))
    single.close()
    got = {}
    with MultiStream(det, n_streams, max(e.n_hits for e in evs), max(e.n_pls for e in evs)) as ms:
        ms.run(evs, on_done=lambda i, ctx: got.__setitem__(i, ctx.results(0)))
        # device-resident inputs through the same contexts
        dev = [{"x": torch.as_tensor(ev.x, device="cuda"), "y": torch.as_tensor(ev.y, device="cuda"),
                "z": torch.as_tensor(ev.z, device="cuda"), "sensor": torch.as_tensor(ev.sensor, device="cuda"),
                "pls": torch.as_tensor(ev.pls.view(np.uint8).copy(), device="cuda"), "n_pls": ev.n_pls}
               for ev in evs[:4]]
        got_dev = {}
        ms.run(dev, on_done=lambda i, ctx: got_dev.__setitem__(i, ctx.results(0)))
    assert sorted(got) == list(range(len(evs)))
    for i in range(len(evs)):
        for k in ref[i]:
            if k != "counts":
                assert np.array_equal(ref[i][k], got[i][k]), (i, k)
                if i < 4:
                    assert np.array_equal(ref[i][k], got_dev[i][k]), (i, k)
    rep = parity.compare_event(oracle.run(det, evs[2]), got[2], evs[2])
    assert rep["ok"], rep["errors"]
