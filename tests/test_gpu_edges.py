"""Edge cases of the CUDA chain beyond the parity events: more than 8192 track candidates of one
type in one event (the track-candidate sort's rank-count path, used above its shared-memory sort's
size), with duplicated seeds whose hit tuples are equal (the order must still be a permutation)."""
import numpy as np
import pytest

import oracle
from paper_2207_08207_gb300 import gen, lst

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _seeds_only_event(n, seed):
    """An event without outer-tracker hits and n pixel seeds: every seed becomes a pLS track
    candidate (no pT3 / pT5 can form, and pLS are not cleaned against each other). Seeds 2k and
    2k + 1 carry the same pixel hit ids, so their sorted hit tuples are equal."""
    rng = np.random.default_rng(seed)
    pls = np.zeros(n, dtype=gen.PLS_DTYPE)
    pls["pt"] = rng.uniform(1.0, 5.0, n)
    pls["eta"] = rng.uniform(-2.4, 2.4, n)
    pls["phi"] = rng.uniform(-np.pi, np.pi, n)
    pls["z0"] = rng.normal(0, 5, n)
    pls["charge"] = rng.choice([-1, 1], n)
    ids = rng.permutation(4 * n).reshape(n, 4).astype(np.int32)
    ids[1::2] = ids[0::2][: n // 2]
    pls["pix_hit"] = ids
    e = np.zeros(0, np.float32)
    return gen.Event(x=e, y=e, z=e, sensor=np.zeros(0, np.int32), pls=pls,
                     hit_particle=np.zeros(0, np.int32), pls_particle=np.arange(n, dtype=np.int32),
                     particles={})


@pytest.mark.parametrize("n", [9000, 8192])
def test_many_pls_candidates_sorted_as_permutation(n):
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    ev = _seeds_only_event(n, seed=n)
    ctx = lst.Context(det)
    try:
        ctx.run([ev])
        got = ctx.results(0)
    finally:
        ctx.close()
    assert got["counts"]["n_tc"] == n
    assert np.all(got["tc_type"] == lst.TC_TYPES.index("pLS"))
    obj = got["tc_obj"]
    assert np.array_equal(np.sort(obj), np.arange(n))          # every seed exactly once
    assert np.array_equal(got["tc_hits"][:, :4], ev.pls["pix_hit"][obj])   # each row holds its seed's hits
    assert np.all(got["tc_hits"][:, 4:] == -1)
    rows = np.sort(got["tc_hits"][:, :4], axis=1)
    keys = [tuple(r) for r in rows]
    assert keys == sorted(keys)                                 # rows ordered by sorted hit tuple
    ref = oracle.run(det, ev)
    rt = ref["tc"]
    ref_rows = sorted(tuple(sorted(int(rt[f"hit{k}"][i]) for k in range(4))) for i in range(len(rt["type"])))
    assert ref_rows == keys


@pytest.mark.parametrize("graph", [0, 1])
def test_stage_timing_with_and_without_graph(graph):
    """Per-stage and per-kernel timing works with plain launches and inside a captured graph, and
    switching it off and on again (a new capture each time) keeps the context usable, with device
    and in-place host inputs."""
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    evs = [gen.small_event(600, seed=80 + k)[1] for k in range(3)]
    ctx = lst.Context(det, use_graph=graph)
    try:
        ref = None
        for timing in (True, False, True):
            ctx.set_timing(timing)
            ctx.run(evs)
            got = [ctx.counts(e)["n_tc"] for e in range(3)]
            ref = ref or got
            assert got == ref
            if timing:
                st, km = ctx.stage_ms(), ctx.kernel_ms()
                assert st["total"] > 0 and km["ls"] > 0 and km["tc_ext"] > 0
            ctx.submit(evs, host_async=True)
            ctx.sync()
            assert [ctx.counts(e)["n_tc"] for e in range(3)] == ref
    finally:
        ctx.close()


def test_contexts_with_different_ls_blocks_coexist():
    """The LS kernel's shared-memory limit is process-wide: a context created later with smaller LS
    blocks must not break the launches of an earlier context with larger ones (graph capture and
    plain launches)."""
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    evs = [gen.small_event(400, seed=90 + k)[1] for k in range(2)]
    big = lst.Context(det, block_ls=256, use_graph=1)
    small = lst.Context(det, block_ls=64, use_graph=0)
    try:
        small.run(evs)
        ref = [small.counts(e)["n_tc"] for e in range(2)]
        big.set_timing(True)
        big.run(evs)
        big.set_timing(False)   # a new capture after the small context loaded its geometry
        big.run(evs)
        assert [big.counts(e)["n_tc"] for e in range(2)] == ref
    finally:
        big.close()
        small.close()


def test_ls_pair_count_lies_between_accepted_and_connected_pairs():
    """The LS search's work count (n_ls_pairs, the (inner MD, outer MD) pairs it evaluated inside its
    azimuth windows) is at least the number of LS it accepted and at most the pairs the module map
    connects (each module's MDs times those of its connected modules), in a batch of PU200 events,
    and is the same in every LS execution mode."""
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    evs = [gen.config_event(2, e)[1] for e in range(3)]
    seen = {}
    for persistent in (2, 1, 0):
        ctx = lst.Context(det, persistent=persistent)
        try:
            ctx.run(evs)
            n_ls, connected = 0, 0
            for e in range(len(evs)):
                r = ctx.results(e)
                n_ls += r["counts"]["n_ls"]
                na = np.bincount(r["md_module"], minlength=det.n_mods).astype(np.int64)
                cs = np.concatenate([[0], np.cumsum(na[det.conn_tgt])])
                nb = cs[det.conn_off[1:]] - cs[det.conn_off[:-1]]   # MDs of each module's connected modules
                connected += int((na * nb).sum())
            pairs = ctx.counts(0)["n_ls_pairs"]
            assert all(ctx.counts(e)["n_ls_pairs"] == pairs for e in range(len(evs)))
            assert n_ls <= pairs <= connected, (persistent, n_ls, pairs, connected)
            assert pairs < 0.7 * connected   # the windows remove a large share of the connected pairs
            seen[persistent] = pairs
        finally:
            ctx.close()
    # every execution mode evaluates the same windows (split into chunks or not)
    assert len(set(seen.values())) == 1, seen
