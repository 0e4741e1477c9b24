"""Parity of the CUDA chain (through the C ABI) with the CPU oracle, on seeded synthetic events:
the toy barrel tracker (200 helices), small and full PU200 events, a PU300 low-threshold event,
batches, device-resident inputs, degenerate events, invalid inputs and forced capacity overflow."""
import numpy as np
import pytest

import oracle
from paper_2207_08207_gb300 import gen, lst
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def det_full():
    return gen.make_detector(barrel_only=False, pt_thr=0.8)


@pytest.fixture(scope="module")
def ctx_full(det_full):
    c = lst.Context(det_full)
    yield c
    c.close()


def _check(ref, got, ev):
    rep = parity.compare_event(ref, got, ev)
    assert rep["ok"], (rep["errors"], got.get("counts"))
    return rep


def test_binning_bit_exact(det_full, ctx_full):
    _, ev = gen.config_event(2, 0)
    ref = oracle.run(det_full, ev)
    s = torch.as_tensor(ev.sensor, device="cuda")
    order = torch.empty(ev.n_hits, dtype=torch.int32, device="cuda")
    offs = torch.empty(2 * det_full.n_mods + 1, dtype=torch.int32, device="cuda")
    ctx_full.bin_hits(s, order, offs)
    assert np.array_equal(order.cpu().numpy(), ref["order"])
    assert np.array_equal(offs.cpu().numpy(), ref["offsets"])


def test_toy_barrel_config1():
    det, ev = gen.config_event(1, 0)
    ctx = lst.Context(det)
    ctx.run([ev])
    rep = _check(oracle.run(det, ev), ctx.results(0), ev)
    assert rep["n_t5"] > 100 and rep["n_tc"] > 100
    ctx.close()


@pytest.mark.parametrize("n,seed", [(5, 1), (50, 2), (400, 3), (1500, 4)])
def test_small_pu_events(ctx_full, n, seed):
    det, ev = gen.small_event(n, seed=seed)
    ctx_full.run([ev])
    _check(oracle.run(det, ev), ctx_full.results(0), ev)


def test_pu200_event(det_full, ctx_full):
    _, ev = gen.config_event(2, 0)
    ctx_full.run([ev])
    got = ctx_full.results(0)
    rep = _check(oracle.run(det_full, ev), got, ev)
    assert rep["n_tc"] > 5000
    assert got["counts"]["status"] == 0


def test_batch_equals_single_runs(det_full, ctx_full):
    evs = [gen.config_event(3, e)[1] for e in range(4)]
    ctx_full.run(evs)
    batched = [ctx_full.results(e) for e in range(4)]
    for e, ev in enumerate(evs):
        ctx_full.run([ev])
        single = ctx_full.results(0)
        for k in single:
            if k == "counts":
                continue
            assert np.array_equal(single[k], batched[e][k]), (e, k)
    _check(oracle.run(det_full, evs[1]), batched[1], evs[1])


def test_bench_batch_matches_single_runs_and_oracle(det_full, ctx_full):
    """The batched launch configuration the benchmark times (64 PU200 events per run, persistent LS
    work list, CUDA graph): every event of the batch equals its one-event run (a different launch
    shape: small-batch LS chunks, per-module tasks), and sampled events match the oracle."""
    evs = [gen.config_event(2, e, pu=200.0)[1] for e in range(64)]
    ctx = lst.Context(det_full, persistent=1, use_graph=1)
    try:
        ctx.run(evs)
        batched = [ctx.results(e) for e in range(64)]
    finally:
        ctx.close()
    for e, ev in enumerate(evs):
        ctx_full.run([ev])
        single = ctx_full.results(0)
        for k in single:
            if k != "counts":
                assert np.array_equal(single[k], batched[e][k]), (e, k)
    for e in (0, 37):
        _check(oracle.run(det_full, evs[e]), batched[e], evs[e])


def test_device_inputs_equal_host_inputs(det_full, ctx_full):
    _, ev = gen.small_event(800, seed=9)
    ctx_full.run([ev])
    host = ctx_full.results(0)
    pls = torch.as_tensor(ev.pls.view(np.uint8).copy(), device="cuda")
    dev_ev = {"x": torch.as_tensor(ev.x, device="cuda"), "y": torch.as_tensor(ev.y, device="cuda"),
              "z": torch.as_tensor(ev.z, device="cuda"), "sensor": torch.as_tensor(ev.sensor, device="cuda"),
              "pls": pls, "n_pls": ev.n_pls}
    ctx_full.run([dev_ev])
    dev = ctx_full.results(0)
    for k in host:
        if k != "counts":
            assert np.array_equal(host[k], dev[k]), k


def _pinned(a):
    t = torch.empty(a.nbytes, dtype=torch.uint8, pin_memory=True).numpy()
    t[:] = np.ascontiguousarray(a).view(np.uint8).reshape(-1)
    return t.view(a.dtype)


def test_async_host_inputs_equal_host_inputs(det_full, ctx_full):
    """LST_MEM_HOST_ASYNC: pinned arrays are gathered by the device in place, pageable ones where the
    host link is coherent (else packed); either way the results equal the LST_MEM_HOST run."""
    import dataclasses
    evs = [gen.small_event(700, seed=s)[1] for s in (21, 22)]
    ctx_full.run(evs)
    host = [ctx_full.results(e) for e in range(2)]
    pinned = [dataclasses.replace(ev, x=_pinned(ev.x), y=_pinned(ev.y), z=_pinned(ev.z),
                                  sensor=_pinned(ev.sensor), pls=_pinned(ev.pls)) for ev in evs]
    for batch in (pinned, evs):
        ctx_full.submit(batch, host_async=True)
        ctx_full.sync()
        for e in range(2):
            got = ctx_full.results(e)
            for k in host[e]:
                if k != "counts":
                    assert np.array_equal(host[e][k], got[k]), k


def test_degenerate_events(det_full, ctx_full):
    empty = gen.Event(x=np.zeros(0, np.float32), y=np.zeros(0, np.float32), z=np.zeros(0, np.float32),
                      sensor=np.zeros(0, np.int32), pls=np.zeros(0, dtype=gen.PLS_DTYPE),
                      hit_particle=np.zeros(0, np.int32), pls_particle=np.zeros(0, np.int32), particles={})
    _, noisy = gen.small_event(30, seed=5, noise_frac=0.5, with_pls=False)
    ctx_full.run([empty, noisy, empty])
    assert ctx_full.counts(0)["n_md"] == 0 and ctx_full.counts(0)["n_tc"] == 0
    assert ctx_full.counts(2)["n_tc"] == 0
    _check(oracle.run(det_full, noisy), ctx_full.results(1), noisy)


def test_invalid_inputs_rejected(det_full, ctx_full):
    _, ev = gen.small_event(20, seed=6)
    bad = gen.Event(x=ev.x.copy(), y=ev.y.copy(), z=ev.z.copy(), sensor=ev.sensor.copy(), pls=ev.pls,
                    hit_particle=ev.hit_particle, pls_particle=ev.pls_particle, particles={})
    bad.sensor[3] = 2 * det_full.n_mods + 5
    with pytest.raises(lst.LSTError) as ei:
        ctx_full.run([bad])
    assert ei.value.code == lst.LST_EINVAL
    nan = gen.Event(x=ev.x.copy(), y=ev.y.copy(), z=ev.z.copy(), sensor=ev.sensor.copy(), pls=ev.pls,
                    hit_particle=ev.hit_particle, pls_particle=ev.pls_particle, particles={})
    nan.x[0] = np.nan
    with pytest.raises(lst.LSTError) as ei:
        ctx_full.run([ev, nan])
    assert ei.value.code == lst.LST_EINVAL
    # the context stays usable
    ctx_full.run([ev])
    assert ctx_full.counts(0)["status"] == 0


def test_forced_overflow_is_counted_and_recovered(det_full):
    _, ev = gen.small_event(1500, seed=7)
    ctx = lst.Context(det_full, cap_scale=0.25)
    ctx.run([ev])
    c = ctx.counts(0)
    assert c["retries"] >= 1
    assert sum(c["overflow"].values()) > 0
    _check(oracle.run(det_full, ev), ctx.results(0), ev)
    ctx.close()


def test_cycle_budget_ends_run_with_timeout(det_full):
    """A warp past its cycle budget stops taking work: the run ends with LST_ETIMEOUT (no fault, no
    hang), the same context keeps answering, and a context without a budget gives full results."""
    _, ev = gen.small_event(400, seed=9)
    tight = lst.Context(det_full, cycle_budget=1)
    with pytest.raises(lst.LSTError) as ei:
        tight.run([ev])
    assert ei.value.code == lst.LST_ETIMEOUT
    assert tight.counts(0)["status"] == lst.LST_ETIMEOUT
    with pytest.raises(lst.LSTError):   # still usable, still over budget
        tight.run([ev])
    tight.close()
    free = lst.Context(det_full)
    free.run([ev])
    assert free.counts(0)["status"] == 0
    _check(oracle.run(det_full, ev), free.results(0), ev)
    free.close()


@pytest.mark.slow
def test_scan_wait_gives_up_at_its_bound():
    """The single-pass scan's wait on an earlier tile is bounded: with the first tile withheld the
    next tile's wait gives up (counted) instead of hanging, and the device stays usable."""
    assert lst.selftest_bounded_wait(0) >= 1
    torch.cuda.synchronize()
    assert torch.ones(4, device="cuda").sum().item() == 4.0


def test_pu300_low_threshold_config4():
    det, ev = gen.config_event(4, 0)
    ctx = lst.Context(det)
    ctx.run([ev])
    _check(oracle.run(det, ev), ctx.results(0), ev)
    ctx.close()


@pytest.mark.parametrize("persistent,graph", [(1, 0), (0, 1), (1, 1)])
def test_executor_modes_identical(det_full, ctx_full, persistent, graph):
    """The persistent work-queue LS kernel and the CUDA-graph replay give the same objects as the
    plain launches, for a full batch and then a smaller batch replayed through the same graph."""
    evs = [gen.config_event(3, e)[1] for e in range(3)]
    ctx_full.run(evs)
    ref = [ctx_full.results(e) for e in range(3)]
    ctx = lst.Context(det_full, persistent=persistent, use_graph=graph)
    ctx.reserve(3, max(e.n_hits for e in evs), max(e.n_pls for e in evs))
    for _ in range(2):
        ctx.run(evs)
        for e in range(3):
            got = ctx.results(e)
            for k in got:
                if k != "counts":
                    assert np.array_equal(got[k], ref[e][k]), (e, k)
    ctx.run(evs[1:2])   # fewer events than the graph's shape: padded with empty events
    got = ctx.results(0)
    for k in got:
        if k != "counts":
            assert np.array_equal(got[k], ref[1][k]), k
    if graph:
        n0 = ctx.launch_count()
        ctx.run(evs)
        assert ctx.launch_count() - n0 > 50   # graph replays count their kernel nodes
    ctx.close()


def test_double_float_outputs_agree_to_1e6(det_full, ctx_full):
    """The T3 / T5 / pT3 / pT5 and extension floats are computed in double-float (~1e-14 per
    operation) and stored as float32: they must agree with the float64 oracle to float32 storage
    precision, far inside the shipped 1e-4 tolerance. (A product contracted into a following
    addition by the compiler degrades the double-float operations to about float precision; this
    catches it.)"""
    _, ev = gen.config_event(2, 3)
    ctx_full.run([ev])
    rep = parity.compare_event(oracle.run(det_full, ev), ctx_full.results(0), ev, rel=1e-6, floor_scale=1e-3)
    assert rep["ok"], rep["errors"]
    assert rep["n_tc_ext"] > 1000
