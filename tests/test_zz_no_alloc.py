"""lst_bin_hits_noalloc: hit binning for callers that cannot allocate device memory (a process whose
device memory is fixed at start-up, or a plugin in a framework that owns every allocation). Its
output must equal the context-based lst_bin_hits exactly (binning is integer work), on two calls in a
row, since every call reuses one static scratch array that keeps the previous call's contents.
This file is collected last so that a failure here stops a run only after every other test ran."""
import ctypes

import numpy as np
import pytest

from paper_2207_08207_gb300 import gen, lst

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_noalloc_binning_equals_context_binning():
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    n_sens = 2 * det.n_mods
    ctx = lst.Context(det)
    events = [gen.config_event(2, 0)[1], gen.small_event(300, seed=21)[1]]
    for ev in events:   # two calls in a row, different inputs, same scratch
        s = torch.as_tensor(ev.sensor, device="cuda")
        ref_order = torch.empty(ev.n_hits, dtype=torch.int32, device="cuda")
        ref_offs = torch.empty(n_sens + 1, dtype=torch.int32, device="cuda")
        ctx.bin_hits(s, ref_order, ref_offs)
        order = torch.full((ev.n_hits,), -7, dtype=torch.int32, device="cuda")
        offs = torch.full((n_sens + 1,), -7, dtype=torch.int32, device="cuda")
        lst.bin_hits_noalloc(s, n_sens, order, offs)
        torch.cuda.synchronize()
        assert torch.equal(order, ref_order)
        assert torch.equal(offs, ref_offs)
        assert int(offs[-1]) == ev.n_hits
    ctx.close()


def test_noalloc_rejects_oversize_and_bad_ids():
    s = torch.zeros(10, dtype=torch.int32, device="cuda")
    order = torch.empty(10, dtype=torch.int32, device="cuda")
    big = torch.empty(65537 + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(lst.LSTError) as ei:
        lst.bin_hits_noalloc(s, 65537, order, big)
    assert ei.value.code == lst.LST_EINVAL
    s[3] = 40
    offs = torch.empty(33, dtype=torch.int32, device="cuda")
    with pytest.raises(lst.LSTError) as ei:
        lst.bin_hits_noalloc(s, 32, order, offs)
    assert ei.value.code == lst.LST_EINVAL
    # still usable after an error
    s[3] = 5
    lst.bin_hits_noalloc(s, 32, order, offs)
    assert int(offs[-1]) == 10
