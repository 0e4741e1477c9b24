"""Host-side scheduling of the multi-stream plain path (streams.MultiStream) with fake contexts: event
i runs on context i mod N, a context never holds two events at once, every event completes exactly
once, and with N contexts at most N events are in flight."""
import pytest

from paper_2207_08207_gb300.streams import MultiStream


class FakeCtx:
    log = []

    def __init__(self, k):
        self.k = k
        self.current = None
        self.reserved = None

    def reserve(self, n, h, p):
        self.reserved = (n, h, p)

    def submit(self, events):
        assert self.current is None, "two events in flight on one context"
        assert len(events) == 1
        self.current = events[0]
        FakeCtx.log.append(("submit", self.k, events[0]))

    def sync(self):
        assert self.current is not None
        FakeCtx.log.append(("done", self.k, self.current))
        self.current = None
        return [0]

    def close(self):
        pass


@pytest.mark.parametrize("n_streams,n_events", [(1, 5), (3, 10), (4, 2), (8, 8)])
def test_round_robin(n_streams, n_events):
    FakeCtx.log = []
    made = []

    def factory():
        made.append(FakeCtx(len(made)))
        return made[-1]
    done = []
    ms = MultiStream(None, n_streams, 100, 10, context_factory=factory)
    assert all(c.reserved == (1, 100, 10) for c in made)
    ms.run(list(range(n_events)), on_done=lambda i, ctx: done.append((i, ctx.k)))
    assert sorted(i for i, _ in done) == list(range(n_events))
    assert all(k == i % n_streams for i, k in done)
    inflight = peak = 0
    for kind, k, ev in FakeCtx.log:
        inflight += 1 if kind == "submit" else -1
        peak = max(peak, inflight)
        if kind == "submit":
            assert k == ev % n_streams
    assert inflight == 0 and peak == min(n_streams, n_events)
    ms.close()


def test_rejects_zero_streams():
    with pytest.raises(ValueError):
        MultiStream(None, 0, 1, 1, context_factory=lambda: FakeCtx(0))
