"""Half-precision storage of per-object floats (lst_config.half_floats, the "half precision floats"
of the paper's Sec. 5): the output-only columns are stored as IEEE binary16, everything else is
unchanged. The binary16 values must be exactly the float32 values of a default run rounded to
nearest binary16, every object and every other output identical, and the arenas smaller."""
import numpy as np
import pytest

from paper_2207_08207_gb300 import gen, lst

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_half_storage_matches_float32_run():
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    evs = [gen.config_event(2, 5)[1], gen.small_event(500, seed=31)[1]]
    full = lst.Context(det)
    half = lst.Context(det, half_floats=1)
    try:
        full.run(evs)
        half.run(evs)
        n_half_values = 0
        for e in range(len(evs)):
            a, b = full.results(e), half.results(e)
            assert a["counts"] == b["counts"]
            for f in a:
                if f == "counts":
                    continue
                if f in lst.HALF_FIELDS:
                    src = a[f[:-2]]          # the float32 column of the default run
                    assert a[f].size == 0 and b[f[:-2]].size == 0
                    assert b[f].dtype == np.float16 and b[f].shape == src.shape, f
                    with np.errstate(over="ignore"):   # beyond +-65504 binary16 holds +-inf, on both sides
                        want = src.astype(np.float16)
                    assert np.array_equal(b[f].view(np.uint16), want.view(np.uint16)), f
                    n_half_values += src.size
                elif f + "_h" not in lst.HALF_FIELDS:   # (float32 columns with a twin: checked above)
                    assert np.array_equal(a[f], b[f]), f
        assert n_half_values > 100_000
        nh, npls = sum(ev.n_hits for ev in evs), sum(ev.n_pls for ev in evs)
        assert half.predict_bytes(2, nh, npls) < full.predict_bytes(2, nh, npls)
    finally:
        full.close()
        half.close()
