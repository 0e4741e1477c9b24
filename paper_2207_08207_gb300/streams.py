"""Event-level parallelism over CUDA streams: the paper's multi-streaming (Sec. 4.2.2, Table 1).

The paper attaches whole events to streams so that the GPU's idle phases in one event's chain (short,
sparse kernels, host round trips) are filled with another event's work. Here each stream is a
library context shaped for one event (its own CUDA stream, arenas and captured graph, all on one
device): event i goes to context i mod N, and a context takes its next event as soon as its previous
one has finished, so up to N events are in flight. Every event's objects are those of a single
one-event run: contexts share nothing but the device.

This is the plain per-event path made concurrent, the comparison point between one event at a time
(N = 1) and the batched executor (many events per launch).
"""
from __future__ import annotations

import time

from . import lst


class MultiStream:
    """N one-event contexts on their own streams, fed round-robin.

    det: the detector (geometry, module map, pixel map) each context loads.
    max_hits, max_pls: the largest event the contexts are reserved for (they grow on demand).
    Further keyword arguments go to each context's configuration (e.g. persistent=1).
    context_factory: builds one context (default: lst.Context on `device`); the host-side
    scheduling can so be exercised without a GPU."""

    def __init__(self, det, n_streams: int, max_hits: int, max_pls: int, device: int = 0, use_graph: int = 1,
                 context_factory=None, **config):
        if n_streams < 1:
            raise ValueError("n_streams must be >= 1")
        make = context_factory or (lambda: lst.Context(det, device=device, use_graph=use_graph, **config))
        self.ctxs = []
        try:
            for _ in range(n_streams):
                c = make()
                c.reserve(1, max_hits, max_pls)
                self.ctxs.append(c)
        except Exception:
            self.close()
            raise

    @property
    def n_streams(self) -> int:
        return len(self.ctxs)

    def run(self, events, on_done=None) -> float:
        """Process `events` (gen.Event objects or dicts of device tensors, as Context.submit takes
        them) in order; event i runs on context i mod N. on_done(i, ctx) is called once event i has
        finished, with its results readable from ctx (e.g. ctx.results(0)) until that context takes
        its next event. Returns the wall time in seconds from the first submission to the last
        completion."""
        n = self.n_streams
        inflight = [None] * n
        t0 = time.perf_counter()
        for i, ev in enumerate(events):
            k = i % n
            if inflight[k] is not None:
                self.ctxs[k].sync()
                if on_done is not None:
                    on_done(inflight[k], self.ctxs[k])
            self.ctxs[k].submit([ev])
            inflight[k] = i
        # drain in submission order
        m = len(events)
        for j in range(max(0, m - n), m):
            k = j % n
            self.ctxs[k].sync()
            if on_done is not None:
                on_done(j, self.ctxs[k])
        return time.perf_counter() - t0

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
