"""Serving loop for the LST chain: events arrive over time, are admitted by their predicted
object-buffer memory against a fixed budget, and are processed by continuous batching.

Several resident engines (library contexts, each with its own CUDA stream and arenas, all sharing
the device-resident geometry's layout) run batches concurrently: whenever an engine is free, every
event that has arrived and fits the memory budget is taken into its next batch, so requests that
arrive while others are on the GPU are admitted as soon as an engine and memory free up, and their
work overlaps on the device with batches already running. Latency is measured from an event's
arrival to the host's observation of its batch's completion.

The scheduling (``Scheduler``) is independent of the engine so that it can be exercised on the host
with a fake engine; ``LSTEngine`` drives the CUDA library.
"""
from __future__ import annotations

import collections
import gc
import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    t_arrival: float          # seconds since the start of the run
    event: object
    n_hits: int
    n_pls: int
    pred_bytes: int = 0
    t_done: float = math.nan
    result: object = None


@dataclass
class ServeStats:
    n: int
    wall_s: float
    throughput: float
    p50_ms: float
    p99_ms: float
    p999_ms: float
    mean_batch: float
    max_inflight_bytes: int
    batches: int
    latencies_ms: list = field(default_factory=list)

    def as_dict(self):
        d = dict(self.__dict__)
        d.pop("latencies_ms")
        return d


class Engine:
    """Interface of one batch executor. `max_batch`: the most events it takes per batch."""

    max_batch = 64

    def submit(self, events):           # enqueue a batch; must not block on the GPU
        raise NotImplementedError

    def done(self) -> bool:             # has the last batch finished?
        raise NotImplementedError

    def collect(self, n):               # results of the last batch (after done()), list of n
        raise NotImplementedError


class Scheduler:
    """Continuous batching over several engines with memory-based admission.

    predict(n_hits, n_pls) -> bytes: the object-buffer memory one event is predicted to need.
    An event is admitted only while the predicted bytes of all events on the engines stay within
    `budget`; events are admitted in arrival order (no overtaking) up to `max_batch` per batch.
    """

    def __init__(self, engines, predict, budget=40e9, max_batch=64, clock=time.perf_counter, idle_sleep=0.0,
                 wakeup=None):
        self.engines = list(engines)
        self.predict = predict
        self.budget = float(budget)
        self.max_batch = int(max_batch)
        self.clock = clock
        self.idle_sleep = idle_sleep
        # wakeup: a threading.Event the engines set when a batch completes; with it the loop sleeps
        # until the next completion or arrival instead of polling
        self.wakeup = wakeup

    def run(self, requests):
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        for r in reqs:
            r.pred_bytes = int(self.predict(r.n_hits, r.n_pls))
            if r.pred_bytes > self.budget:
                raise ValueError(f"request {r.rid} alone exceeds the memory budget")
        pending = collections.deque(reqs)
        waiting = collections.deque()
        busy = {}                     # engine index -> list of requests
        t0 = self.clock()
        gc_was_enabled = gc.isenabled()
        gc.disable()   # no collector pauses inside the serving loop (collected after it)
        try:
            return self._loop(reqs, pending, waiting, busy, t0)
        finally:
            if gc_was_enabled:
                gc.enable()
            gc.collect()

    def _loop(self, reqs, pending, waiting, busy, t0):
        inflight = 0
        max_inflight = 0
        batches = 0
        batch_sizes = []
        self.iterations = 0
        while pending or waiting or busy:
            self.iterations += 1
            if self.wakeup is not None:
                self.wakeup.clear()   # a completion from here on wakes the wait below
            now = self.clock() - t0
            progressed = False
            while pending and pending[0].t_arrival <= now:
                waiting.append(pending.popleft())
                progressed = True
            # completions
            for k in list(busy):
                if self.engines[k].done():
                    progressed = True
                    batch = busy.pop(k)
                    res = self.engines[k].collect(len(batch))
                    t_done = self.clock() - t0
                    for r, out in zip(batch, res):
                        r.t_done = t_done
                        r.result = out
                    inflight -= sum(r.pred_bytes for r in batch)
            # admission onto free engines: the smallest free engine that takes everything waiting
            # (else the largest free one), so small bursts run on small launch shapes
            while waiting:
                free = [k for k in range(len(self.engines)) if k not in busy]
                if not free:
                    break
                cap = lambda k: min(self.max_batch, getattr(self.engines[k], "max_batch", self.max_batch))
                fits = [k for k in free if cap(k) >= len(waiting)]
                k = min(fits, key=cap) if fits else max(free, key=cap)
                batch = []
                while waiting and len(batch) < cap(k) and \
                        inflight + waiting[0].pred_bytes <= self.budget:
                    r = waiting.popleft()
                    inflight += r.pred_bytes
                    batch.append(r)
                if not batch:
                    break
                max_inflight = max(max_inflight, inflight)
                self.engines[k].submit([r.event for r in batch])
                progressed = True
                busy[k] = batch
                batches += 1
                batch_sizes.append(len(batch))
            if self.wakeup is not None:
                if not progressed:   # sleep until a batch completes or the next request arrives
                    wait = pending[0].t_arrival - (self.clock() - t0) if pending else 0.05
                    if wait > 0:
                        self.wakeup.wait(timeout=min(wait, 0.05))
            elif not busy and not waiting and pending:
                # idle until the next arrival
                wait = pending[0].t_arrival - (self.clock() - t0)
                if wait > 0 and self.idle_sleep > 0:
                    time.sleep(min(wait, self.idle_sleep))
        wall = self.clock() - t0
        lat = np.array([(r.t_done - r.t_arrival) * 1e3 for r in reqs])
        return ServeStats(
            n=len(reqs), wall_s=wall, throughput=len(reqs) / wall if wall > 0 else math.inf,
            p50_ms=float(np.percentile(lat, 50)) if lat.size else math.nan,
            p99_ms=float(np.percentile(lat, 99)) if lat.size else math.nan,
            p999_ms=float(np.percentile(lat, 99.9)) if lat.size else math.nan,
            mean_batch=float(np.mean(batch_sizes)) if batch_sizes else 0.0,
            max_inflight_bytes=int(max_inflight), batches=batches, latencies_ms=lat.tolist())


def poisson_arrivals(rate_hz, n, seed=0):
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, n))


class LSTEngine(Engine):
    """One library context with its own stream; batches of resident (device) or host events."""

    def __init__(self, det, max_batch, max_hits, max_pls, device=0, stream=None, keep="tc", notify=None, **cfg):
        import torch
        from . import lst
        self.max_batch = int(max_batch)
        self.ctx = lst.Context(det, device=device, **cfg)
        self.ctx.reserve(max_batch, max_hits, max_pls)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        self.keep = keep
        self._n = 0
        # a waiter thread blocks in lst_sync (the call releases the interpreter lock) for each
        # submitted batch and then marks it done and sets `notify`, so the scheduler needs no polling
        self.notify = notify
        self._done = threading.Event()
        self._err = None
        self._jobs = queue.SimpleQueue()
        self._waiter = threading.Thread(target=self._wait_loop, daemon=True)
        self._waiter.start()

    def _wait_loop(self):
        while self._jobs.get() is not None:
            try:
                self.ctx.sync()
            except Exception as ex:   # reported by collect()
                self._err = ex
            self._done.set()
            if self.notify is not None:
                self.notify.set()

    def predict(self, n_hits, n_pls):
        return self.ctx.predict_bytes(1, n_hits, n_pls)

    def submit(self, events):
        self._done.clear()
        self._err = None
        self.ctx.submit(events, stream=self.stream, host_async=True)   # events are held until sync
        self._n = len(events)
        self._jobs.put(True)

    def done(self):
        return self._done.is_set()

    def collect(self, n):
        self._done.wait()
        if self._err is not None:
            raise self._err
        if self.keep == "tc":   # the batch's track candidates, one transfer per array
            tc = self.ctx.copy_tc_all()
            o = tc["offsets"]
            return [{k: tc[k][o[e]:o[e + 1]] for k in ("type", "obj", "hits", "pt", "eta", "phi")}
                    for e in range(n)]
        if self.keep == "all":
            return [self.ctx.results(e) for e in range(n)]
        return [self.ctx.counts(e) for e in range(n)]

    def close(self):
        self._jobs.put(None)
        self._waiter.join(timeout=10)
        self.ctx.close()


class Server:
    """LST serving: resident contexts of different batch capacities (`batch_sizes`, default capacities
    growing by 4x up to `max_batch`), continuous batching, memory admission."""

    def __init__(self, det, n_engines=4, max_batch=64, max_hits=150_000, max_pls=12_000, budget=40e9, device=0,
                 keep="tc", batch_sizes=None, **cfg):
        if batch_sizes is None:
            # capacities growing by 4x up to max_batch (1, 4, 16, 64 for four engines): a burst goes
            # to the smallest free engine that takes it, whose capacity-shaped launches cost the least
            batch_sizes = [max(1, max_batch // 4 ** k) for k in range(n_engines)][::-1]
        self.wakeup = threading.Event()
        self.engines = [LSTEngine(det, b, max_hits, max_pls, device=device, keep=keep, notify=self.wakeup, **cfg)
                        for b in batch_sizes]
        self.scheduler = Scheduler(self.engines, self.engines[0].predict, budget=budget, max_batch=max(batch_sizes),
                                   wakeup=self.wakeup)

    def warmup(self, events):
        """Batches on every engine before a measurement: graph capture and arena first touch, then a
        full batch of the heaviest of `events`, so that the engines' arenas already hold any batch of
        these events (an arena that grows during serving makes its engine capture its graph again,
        a stall of a few hundred milliseconds for the requests waiting on it)."""
        heavy = max(events, key=lambda ev: (_n_hits(ev), _n_pls(ev)))
        for e in self.engines:
            for batch in (list(events[: e.max_batch]), [heavy] * e.max_batch):
                e.submit(batch)
                e.collect(len(batch))

    def serve(self, events, arrivals):
        reqs = [Request(i, float(t), ev, _n_hits(ev), _n_pls(ev)) for i, (t, ev) in enumerate(zip(arrivals, events))]
        stats = self.scheduler.run(reqs)
        return stats, reqs

    def close(self):
        for e in self.engines:
            e.close()


def _n_hits(ev):
    if isinstance(ev, dict):
        return int(ev["x"].shape[0])
    return ev.n_hits


def _n_pls(ev):
    if isinstance(ev, dict):
        return int(ev.get("n_pls", 0))
    return ev.n_pls
