"""The binding's column-wise input records (batches of host events, batches of tensor dicts) equal
the record-by-record ones: same pointers, sizes and memory spaces, in the C ABI's layout."""
import ctypes

import numpy as np
import pytest

from paper_2207_08207_gb300 import gen, lst


def _events(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nh = int(rng.integers(0, 50))
        k = int(rng.integers(0, 4)) if i % 3 else 0
        pls = np.zeros(k, dtype=gen.PLS_DTYPE)
        x = rng.normal(size=nh).astype(np.float64 if i % 2 else np.float32)   # converted to float32
        out.append(gen.Event(x=x, y=rng.normal(size=nh).astype(np.float32),
                             z=rng.normal(size=nh).astype(np.float32),
                             sensor=rng.integers(0, 10, nh).astype(np.int32), pls=pls,
                             hit_particle=np.zeros(nh, np.int32), pls_particle=np.zeros(k, np.int32),
                             particles={}))
    return out


def _records(arr, n):
    """The ctypes records at arr as tuples."""
    rec = ctypes.cast(arr, ctypes.POINTER(lst.EventIn))
    return [(r.x, r.y, r.z, r.sensor, r.n_hits, r.pls, r.n_pls, r.mem_space) for r in (rec[i] for i in range(n))]


def test_event_in_dtype_matches_the_structure():
    assert lst._EVENT_IN_DTYPE.itemsize == ctypes.sizeof(lst.EventIn)
    for f, _ in lst.EventIn._fields_:
        assert lst._EVENT_IN_DTYPE.fields[f][1] == getattr(lst.EventIn, f).offset


@pytest.mark.parametrize("host_async", [False, True])
def test_host_batch_records_match_record_by_record(host_async):
    evs = _events(7)
    buf, keep = lst._host_events_in(evs, host_async)
    ref, keep_ref = lst.Context._events_in(evs, host_async)
    got = _records(buf.ctypes.data, len(evs))
    want = _records(ctypes.addressof(ref), len(evs))
    # each path converts the float64 x arrays itself (different copies): x is compared by content,
    # every other field (the float32 arrays are used in place) by value
    for i, (g, w) in enumerate(zip(got, want)):
        assert g[1:] == w[1:]
        assert g[4] == len(evs[i].x) and g[6] == evs[i].n_pls
        assert g[7] == (lst.LST_MEM_HOST_ASYNC if host_async else lst.LST_MEM_HOST)
        x = np.ctypeslib.as_array(ctypes.cast(g[0], ctypes.POINTER(ctypes.c_float)), (g[4],)) if g[4] else np.zeros(0)
        np.testing.assert_array_equal(x, np.asarray(evs[i].x, dtype=np.float32))
        if evs[i].n_pls == 0:
            assert not g[5]


def test_tensor_batch_records_match_record_by_record():
    torch = pytest.importorskip("torch")
    evs = []
    for e in _events(5, seed=1):
        evs.append({"x": torch.as_tensor(np.asarray(e.x, np.float32)), "y": torch.as_tensor(e.y),
                    "z": torch.as_tensor(e.z), "sensor": torch.as_tensor(e.sensor),
                    "pls": torch.as_tensor(e.pls.view(np.uint8).copy()), "n_pls": e.n_pls})
    for host_async in (False, True):
        buf = lst._tensor_events_in(evs, host_async)
        ref, _ = lst.Context._events_in(evs, host_async)
        assert _records(buf.ctypes.data, len(evs)) == _records(ctypes.addressof(ref), len(evs))
