"""Serving scheduler on the host, with a fake engine and a simulated clock: memory admission never
exceeds the budget, events are served in arrival order, requests arriving while batches run join the
next free engine (continuous batching), and every request completes."""
import pytest

from paper_2207_08207_gb300.serving import Engine, Request, Scheduler, poisson_arrivals


class FakeClock:
    def __init__(self, dt=1e-4):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeEngine(Engine):
    """Completes a batch `per_batch + per_event * n` seconds after submission."""

    def __init__(self, clock, per_batch=2e-3, per_event=1e-4, log=None):
        self.clock, self.per_batch, self.per_event = clock, per_batch, per_event
        self.t_end = None
        self.batch = None
        self.log = log if log is not None else []

    def submit(self, events):
        self.batch = list(events)
        self.t_end = self.clock.t + self.per_batch + self.per_event * len(events)
        self.log.append((self.clock.t, tuple(self.batch)))

    def done(self):
        return self.t_end is not None and self.clock.t >= self.t_end

    def collect(self, n):
        assert n == len(self.batch)
        self.t_end = None
        return [("result", e) for e in self.batch]


def _requests(n, rate, size=1000, seed=1):
    t = poisson_arrivals(rate, n, seed)
    return [Request(i, float(t[i]), i, size + (i % 7) * 100, 10) for i in range(n)]


def test_all_complete_in_order_with_results():
    clock = FakeClock()
    log = []
    engines = [FakeEngine(clock, log=log) for _ in range(3)]
    sched = Scheduler(engines, predict=lambda h, p: h, budget=1e9, max_batch=8, clock=clock)
    reqs = _requests(300, rate=2000)
    stats = sched.run(reqs)
    assert stats.n == 300
    assert all(r.result == ("result", r.rid) for r in reqs)
    assert all(r.t_done >= r.t_arrival for r in reqs)
    # arrival order is never overtaken across batches
    served = [e for _, batch in sorted(log) for e in batch]
    assert served == sorted(served)
    assert stats.p50_ms <= stats.p99_ms <= stats.p999_ms


def test_memory_budget_respected():
    clock = FakeClock()
    engines = [FakeEngine(clock, per_batch=5e-3) for _ in range(4)]
    budget = 5000
    sched = Scheduler(engines, predict=lambda h, p: h, budget=budget, max_batch=64, clock=clock)
    stats = sched.run(_requests(200, rate=20000))
    assert stats.max_inflight_bytes <= budget
    assert stats.n == 200


def test_continuous_batching_uses_free_engines():
    clock = FakeClock()
    log = []
    engines = [FakeEngine(clock, per_batch=10e-3, log=log) for _ in range(2)]
    sched = Scheduler(engines, predict=lambda h, p: 1, budget=1e9, max_batch=64, clock=clock)
    stats = sched.run(_requests(400, rate=10000))
    # a burst arriving while the first batch runs is taken by the second engine, not queued behind it
    assert log[1][0] < log[0][0] + 10e-3
    assert stats.batches < 400 and stats.mean_batch > 1


def test_request_larger_than_budget_rejected():
    clock = FakeClock()
    sched = Scheduler([FakeEngine(clock)], predict=lambda h, p: h, budget=10, clock=clock)
    with pytest.raises(ValueError):
        sched.run(_requests(3, rate=100))


class ThreadedEngine(Engine):
    """Completes each batch on a timer thread after `delay` seconds and sets the scheduler's wakeup
    event, as the library engine's waiter thread does."""

    def __init__(self, notify, delay=2e-3):
        import threading
        self.notify, self.delay, self.threading = notify, delay, threading
        self.batch = None
        self.flag = threading.Event()

    def submit(self, events):
        self.batch = list(events)
        self.flag.clear()

        def finish():
            self.flag.set()
            self.notify.set()
        self.threading.Timer(self.delay, finish).start()

    def done(self):
        return self.flag.is_set()

    def collect(self, n):
        self.flag.wait()
        return [("result", e) for e in self.batch]


def test_event_driven_loop_does_not_poll():
    import threading
    wake = threading.Event()
    engines = [ThreadedEngine(wake) for _ in range(2)]
    sched = Scheduler(engines, predict=lambda h, p: h, budget=1e9, max_batch=8, wakeup=wake)
    reqs = _requests(150, rate=1500)
    stats = sched.run(reqs)
    assert stats.n == 150 and all(r.result == ("result", r.rid) for r in reqs)
    # one pass per arrival, submission or completion (plus timeouts), not a busy poll
    assert sched.iterations < 10 * len(reqs), sched.iterations


def test_warmup_sizes_every_engine_for_a_full_batch_of_the_heaviest_event():
    """Server.warmup runs, on every engine, a batch of the given events and then a full batch of the
    heaviest of them, so that no batch of these events makes an engine grow its arenas (and capture
    its graph again) while it is being measured."""
    from types import SimpleNamespace

    from paper_2207_08207_gb300.serving import Server

    class Recorder(Engine):
        def __init__(self, max_batch):
            self.max_batch = max_batch
            self.batches = []

        def submit(self, events):
            self.batches.append(list(events))

        def done(self):
            return True

        def collect(self, n):
            assert n == len(self.batches[-1])
            return [None] * n

    events = [SimpleNamespace(n_hits=h, n_pls=p, name=i) for i, (h, p) in enumerate([(10, 5), (90, 1), (40, 9), (90, 3)])]
    srv = object.__new__(Server)
    srv.engines = [Recorder(1), Recorder(4), Recorder(16)]
    srv.warmup(events)
    for e in srv.engines:
        assert e.batches[0] == events[: e.max_batch]
        assert [ev.name for ev in e.batches[1]] == [3] * e.max_batch   # most hits, then most seeds
