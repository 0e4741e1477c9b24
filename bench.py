"""Benchmark of the GB300 Line Segment Tracking chain.

Workload: PU200 events of the full outer tracker (seeded synthetic events shaped like the paper's
ttbar + PU200 sample: ~6000 helices, pT ~ pT^-3 above 0.8 GeV, |eta| < 2.4, 3% noise, one pixel seed
per particle), processed in batches of --batch events (default 64). One step = one batch through the
whole chain (binning, MD, LS, T3, T5, pT3, pT5, TC) with the inputs already resident in HBM.

Printed (rank 0, one JSON line): events/s of the batched path (`value`), the plain one-event-at-a-time
path, p50/p99 per-event latency, the end-to-end number through the public API with host buffers,
the roofline of the dominant kernel, the CPU oracle baseline, and the SM clocks seen during timing.
`--impl reference` times the CPU oracle (the reference arm) on the same workload instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PU200 events/s on 1 GB300 (batched vs plain per-event) + p50/p99 event latency"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _pinned_copy(a):
    """A copy of the 1-D numpy array `a` in pinned (page-locked) host memory."""
    import torch
    t = torch.empty(a.nbytes, dtype=torch.uint8, pin_memory=True).numpy()
    t[:] = a.view(np.uint8).reshape(-1)
    return t.view(a.dtype)


def kernel_profile(kernel):
    """The ncu counters of a timed kernel (profiles/kernel_metrics.json), or None when there is no
    entry or the kernel's source file has changed since the capture (its SHA-1 differs)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "kernel_metrics.json")) as f:
            ent = json.load(f)["kernels"].get(kernel)
        if ent is None:
            return None
        with open(os.path.join(ROOT, ent["source"]), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != ent["source_sha1"]:
                return None
        return ent
    except (OSError, KeyError, ValueError):
        return None


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self):
        """Host time stamp (start / end of the timed region)."""
        return time.perf_counter()

    def stop(self, t0=None, t1=None):
        """Summary of the samples taken between t0 and t1 (all samples if none fall inside)."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for t, ln in self.lines if t0 is None or (t0 <= t <= t1)]
        for ln in inside or [ln for _, ln in self.lines]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "in_timed_region": bool(inside)}


def to_device(ev, torch):
    return {"x": torch.as_tensor(ev.x, device="cuda"), "y": torch.as_tensor(ev.y, device="cuda"),
            "z": torch.as_tensor(ev.z, device="cuda"), "sensor": torch.as_tensor(ev.sensor, device="cuda"),
            "pls": torch.as_tensor(ev.pls.view(np.uint8).copy(), device="cuda"), "n_pls": ev.n_pls}


def serving_run(det, events, rate, n_requests, batch_sizes, seed=0):
    """Poisson stream of `n_requests` events (drawn cyclically from `events`) at `rate` per second,
    served by resident engines of the given batch capacities."""
    from paper_2207_08207_gb300.serving import Server, poisson_arrivals
    srv = Server(det, batch_sizes=batch_sizes, max_hits=max(e.n_hits for e in events),
                 max_pls=max(e.n_pls for e in events), budget=40e9, keep="tc", use_graph=1, persistent=2)
    reqs = [events[i % len(events)] for i in range(n_requests)]
    srv.warmup(events)   # graph capture, arena first touch, arenas sized for the heaviest batch
    stats, _ = srv.serve(reqs, poisson_arrivals(rate, n_requests, seed))
    srv.close()
    d = stats.as_dict()
    d["rate_hz"] = rate
    return d


def rank_seed0(rank):
    """First event seed of a rank: ranks draw disjoint events (seeds 1000 rank + e, e < 1000)."""
    return 1000 * rank


def max_over_ranks(t_local, world, device):
    """The slowest rank's timed-region length (seconds): all-reduce MAX, then a barrier."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    return float(t.item())


def whole_job_rate(events_per_step, steps, world, t_max):
    """Whole-job throughput: the events all ranks processed over the slowest rank's time."""
    return events_per_step * steps * world / t_max


WORKLOADS = {
    1: "toy barrel events, 200 helices (barrel only, 5258 modules)",
    2: "PU200 events, full outer tracker (9138 modules)",
    3: "PU ~ U[140, 250] events, full outer tracker (9138 modules)",
    4: "PU300 events with 20 % loopers, pT threshold 0.6 GeV, full outer tracker (9138 modules)",
}


def make_events(n, seed0=0, config=2):
    """Events of a benchmark configuration (seed 1000 config + event); returns (detector, events)."""
    from paper_2207_08207_gb300 import gen
    if config == 2:
        det = gen.make_detector(barrel_only=False, pt_thr=0.8)
        return det, [gen.config_event(2, seed0 + e, pu=200.0)[1] for e in range(n)]
    pairs = [gen.config_event(config, seed0 + e) for e in range(n)]
    return pairs[0][0], [ev for _, ev in pairs]


def oracle_events_per_s(det, evs, threads):
    """CPU oracle on the given events (threads across events); returns (events/s, wall s)."""
    import concurrent.futures as cf
    import oracle
    oracle.build()
    t = time.perf_counter()
    if threads <= 1:
        for ev in evs:
            oracle.run(det, ev)
    else:
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda ev: oracle.run(det, ev), evs))
    dt = time.perf_counter() - t
    return len(evs) / dt, dt


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on the same PU200 workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = min(os.cpu_count() or 1, 16)
    det, evs = make_events(threads, seed0=0)
    for _ in range(args.warmup):
        oracle_events_per_s(det, evs[:1], 1)
    times = []
    for k in range(args.steps):
        r, dt = oracle_events_per_s(det, evs, threads)
        times.append(dt / len(evs))
    per_event = statistics.mean(times)
    value = 1.0 / per_event
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_event * len(evs) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"PU200 events (full outer tracker), {len(evs)} events per step on {threads} threads",
                   "events_per_step": len(evs)},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": threads, "kind": "oracle",
                         "sample": f"{len(evs)} PU200 events per step, one thread per event",
                         "cpu_model": cpu_model(), "host_cores": os.cpu_count()},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=None,
                    help="events per step (default: 16 for the PU300 stress workload, which is defined on 16, else 64)")
    ap.add_argument("--config", type=int, default=2, choices=sorted(WORKLOADS),
                    help="event configuration of the batched / plain measurement (2: PU200)")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-streams", action="store_true")
    ap.add_argument("--no-half", action="store_true")
    ap.add_argument("--serving-rates", default="500,1000,2000,3000",
                    help="comma-separated Poisson rates (events/s) of the serving measurement")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2207_08207_gb300 import lst

    B = args.batch if args.batch else (16 if args.config == 4 else 64)
    # every rank processes its own events (events are independent: no collective on the data path)
    det, evs = make_events(B, seed0=rank_seed0(rank), config=args.config)
    # inputs resident in HBM
    dev = [to_device(ev, torch) for ev in evs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.Stream()   # the library's work and the timing events share this stream
    torch.cuda.set_stream(stream)

    # batched executor: launch settings from the autotuner, chain replayed as a CUDA graph
    tuned = {"block_ls": 128, "warps_px": 4, "persistent": 2, "cap_scale": 1.0}
    if not args.no_tune:
        from paper_2207_08207_gb300 import autotune
        tuned = autotune.tune(det, dev, workload=f"config{args.config}")
    ctx = lst.Context(det, device=local, use_graph=1, **tuned)
    ctx.reserve(B, max(e.n_hits for e in evs), max(e.n_pls for e in evs))

    def step():
        ctx.submit(dev, stream=stream)
        ctx.sync()

    # per-kernel timing events are part of the captured graph: enable them before the warm-up so
    # that the graph used in the timed region is captured there
    ctx.set_timing(True)
    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(max(3, args.warmup)):
        step()
    launches0 = ctx.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_begin = sampler.mark()
    step_ms, stage_acc, kern_acc = [], {}, {}
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for k, v in ctx.stage_ms().items():
            stage_acc[k] = stage_acc.get(k, 0.0) + v
        for k, v in ctx.kernel_ms().items():
            kern_acc[k] = kern_acc.get(k, 0.0) + v
    torch.cuda.synchronize()
    t_end = sampler.mark()
    clocks = sampler.stop(t_begin, t_end)
    launches = ctx.launch_count() - launches0
    ctx.set_timing(False)
    t_local = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_local, world, "cuda")
    value = whole_job_rate(B, args.steps, world, t_max)
    counts = [ctx.counts(e) for e in range(B)]

    # roofline of the dominant kernel. The candidate kernels are bound by instruction issue (their
    # working set sits in L2), so the ceiling is the issue rate: SMs x 4 schedulers x max SM clock,
    # and the work per launch is the kernel's warp instructions per event (ncu, on this workload)
    # times the events of the launch. The HBM fraction (algorithmic bytes) is reported beside it.
    hbm_peak, peak_kind = _peaks()
    kavg = {k: v / args.steps for k, v in kern_acc.items()}
    dom = max(kavg, key=kavg.get) if kavg else None
    n_md = sum(c["n_md"] for c in counts)
    n_ls = sum(c["n_ls"] for c in counts)
    n_t3 = sum(c["n_t3"] for c in counts)
    n_t5 = sum(c["n_t5"] for c in counts)
    alg_bytes = ctx.kernel_algorithmic_bytes(dom, counts, sum(e.n_hits for e in evs), sum(e.n_pls for e in evs)) if dom else 0
    dur_s = kavg[dom] * 1e-3 if dom and kavg[dom] > 0 else float("nan")
    hbm_achieved = alg_bytes / dur_s / 1e9
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    issue_peak = n_sm * 4 * _sm_max_mhz() * 1e6 / 1e9          # G warp instructions / s
    prof = kernel_profile(dom) if args.config == 2 else None
    if prof is not None:
        per_ev = B / prof["events_per_launch"]
        inst = prof["warp_inst"] * per_ev
        achieved = inst / dur_s / 1e9
        roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": issue_peak,
                    "unit": "G warp-instructions/s", "frac": achieved / issue_peak,
                    "traffic": (prof["dram_read_bytes"] + prof["dram_write_bytes"]) * per_ev,
                    "peak_kind": "derived: SMs x 4 schedulers x max SM clock",
                    "warp_inst_per_launch": inst,
                    "profile": f"profiles/kernel_metrics.json ({prof['events_per_launch']}-event capture scaled to {B})"}
    else:
        roofline = {"bound": "hbm", "kernel": dom, "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_achieved / hbm_peak, "traffic": None, "peak_kind": peak_kind}
    # the LS search's work: windowed (inner MD, outer MD) pairs per event (counted by the kernel) and,
    # with the ncu instruction count, thread instructions per pair
    n_pairs = counts[0]["n_ls_pairs"] if counts else 0
    roofline["ls_pairs_per_event"] = n_pairs / B
    ls_prof = kernel_profile("ls") if args.config == 2 else None
    if ls_prof is not None and n_pairs:
        roofline["ls_thread_inst_per_pair"] = ls_prof["thread_inst"] * (B / ls_prof["events_per_launch"]) / n_pairs
    roofline.update({"kernel_ms": kavg.get(dom) if dom else None,
                     "hbm": {"algorithmic_bytes": alg_bytes, "achieved": hbm_achieved, "peak": hbm_peak,
                             "unit": "GB/s", "frac": hbm_achieved / hbm_peak, "peak_kind": peak_kind},
                     "kernels_ms": {k: round(v, 4) for k, v in sorted(kavg.items(), key=lambda kv: -kv[1])}})

    # plain path: one event per call (a context shaped for one event), inputs resident
    plain = None
    if not args.no_plain:
        pctx = lst.Context(det, device=local, use_graph=1)
        pctx.reserve(1, max(e.n_hits for e in evs), max(e.n_pls for e in evs))
        for i in range(3):
            pctx.submit([dev[i]], stream=stream)
            pctx.sync()
        lat = []
        for i in range(min(B, 32)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pctx.submit([dev[i]], stream=stream)
            pctx.sync()
            e1.record(stream)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1))
        pctx.close()
        lat_s = sorted(lat)
        plain = {"events_per_s": 1e3 / statistics.mean(lat), "p50_ms": float(np.percentile(lat_s, 50)),
                 "p99_ms": float(np.percentile(lat_s, 99)), "events": len(lat)}

    # half-precision storage of the output-only per-object floats (Sec. 5): the same batched launch
    # with binary16 columns; objects are identical (GPU test), the arenas smaller
    half = None
    if not args.no_half:
        hctx = lst.Context(det, device=local, use_graph=1, half_floats=1, **tuned)
        hctx.reserve(B, max(e.n_hits for e in evs), max(e.n_pls for e in evs))
        for _ in range(3):
            hctx.submit(dev, stream=stream)
            hctx.sync()
        hms = []
        for _ in range(max(5, args.steps // 2)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hctx.submit(dev, stream=stream)
            hctx.sync()
            e1.record(stream)
            e1.synchronize()
            hms.append(e0.elapsed_time(e1))
        nh, npl = sum(e.n_hits for e in evs), sum(e.n_pls for e in evs)
        b32, b16 = ctx.predict_bytes(B, nh, npl), hctx.predict_bytes(B, nh, npl)
        c = counts
        n_vals = sum(2 * x["n_md"] + 2 * x["n_ls"] + 4 * x["n_t3"] + 3 * x["n_t5"] + 2 * x["n_pt3"] + 2 * x["n_pt5"]
                     for x in c)
        half = {"events_per_s": B / (statistics.mean(hms) / 1e3), "ms_per_step": statistics.mean(hms),
                "arena_bytes_float32": b32, "arena_bytes_half": b16,
                "output_bytes_saved_per_event": 2 * n_vals / B}
        hctx.close()

    # the paper's multi-stream plain path (Sec. 4.2.2, Table 1): N one-event contexts on their own
    # streams, fed round-robin, inputs resident; events/s over the whole batch of events
    streams = None
    if not args.no_streams:
        from paper_2207_08207_gb300.streams import MultiStream
        streams = {"events": B, "events_per_s": {}}
        for n_st in (1, 2, 4, 8):
            with MultiStream(det, n_st, max(e.n_hits for e in evs), max(e.n_pls for e in evs),
                             device=local) as ms:
                ms.run(dev[: max(n_st, 4)])   # first runs: graph capture, arena first touch
                torch.cuda.synchronize()
                wall = ms.run(dev)
            streams["events_per_s"][str(n_st)] = B / wall

    # end to end through the public API: host buffers in, track candidates out
    e2e_ms = [float("nan")]
    h2d = sum(e.n_hits * 16 + e.n_pls * 48 for e in evs) + 2 * (B + 1) * 4
    d2h = 0
    # pinned host buffers for the results (one transfer per array for the whole batch)
    cap_tc = sum(e.n_pls for e in evs) + 20000 * B
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    tc_buf = {"offsets": pin((B + 1,), torch.int32), "type": pin((cap_tc,), torch.int32),
              "obj": pin((cap_tc,), torch.int32), "hits": pin((cap_tc, 14), torch.int32),
              "pt": pin((cap_tc,), torch.float32), "eta": pin((cap_tc,), torch.float32),
              "phi": pin((cap_tc,), torch.float32)}
    # the step's inputs in pinned host memory (the source of the host-to-device transfer)
    def pinned_event(ev):
        f32 = lambda a: _pinned_copy(np.ascontiguousarray(a, dtype=np.float32))
        return dataclasses.replace(ev, x=f32(ev.x), y=f32(ev.y), z=f32(ev.z),
                                   sensor=_pinned_copy(np.ascontiguousarray(ev.sensor, dtype=np.int32)),
                                   pls=_pinned_copy(np.ascontiguousarray(ev.pls)))
    evs_pin = [pinned_event(e) for e in evs] if not args.no_e2e else []
    for _ in range(0 if args.no_e2e else max(2, min(args.steps, 5)) + 1):
        if len(e2e_ms) == 1 and e2e_ms[0] != e2e_ms[0]:
            e2e_ms = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.submit(evs_pin, stream=stream, host_async=True)
        ctx.sync()
        tc = ctx.copy_tc_all(tc_buf)
        n_tc = tc["n"]
        d2h = n_tc * (4 * 5 + 14 * 4) + (B + 1) * 4
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    if len(e2e_ms) > 1:
        e2e_ms = e2e_ms[1:]   # first pass: host staging buffers
    e2e_value = B / (statistics.mean(e2e_ms) / 1e3)

    # physics performance of the copied-out track candidates on the generator's truth (Sec. 3):
    # efficiency at 75 % hit matching, fake and duplicate rates (host-side, after the timed region)
    phys = None
    if not args.no_e2e:
        from paper_2207_08207_gb300 import physics
        pc = physics.Counts()
        off = tc["offsets"]
        for e, ev in enumerate(evs):
            pc.add(ev, tc["type"][off[e]:off[e + 1]], tc["hits"][off[e]:off[e + 1]])
        ps = pc.summary()
        phys = {"events": B, "eff_above_1gev": ps["eff_above_1gev"], "fake_rate": ps["fake_rate"],
                "duplicate_rate": ps["duplicate_rate"],
                "eff_pt": {f"{lo:g}-{hi:g}": round(v, 4) for lo, hi, v in
                           zip(ps["pt_bins"][:-1], ps["pt_bins"][1:], ps["eff_pt"]) if v == v},
                "eff_eta_pt_gt_0.9": [round(v, 4) for v in ps["eff_eta"]],
                "by_type": ps["by_type"]}

    # serving: Poisson arrivals of PU ~ U[50, 300] events, continuous batching vs one at a time
    serving = None
    if not args.no_serving and rank == 0 and args.config == 2:
        from paper_2207_08207_gb300 import gen
        pool = [gen.config_event(5, e)[1] for e in range(24)]
        serving = {"workload": "Poisson stream of PU ~ U[50, 300] events (24 generated, cycled), 40 GB budget; "
                               "continuous batching over engines of 1, 4, 16 and 64 events vs one engine of 1",
                   "batched": [], "one_at_a_time": []}
        for rate in [float(r) for r in args.serving_rates.split(",")]:
            n_req = int(min(4000, max(200, rate * 2.0)))
            serving["batched"].append(serving_run(det, pool, rate, n_req, batch_sizes=[1, 4, 16, 64]))
            serving["one_at_a_time"].append(serving_run(det, pool, rate, min(n_req, 600), batch_sizes=[1]))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle in both of its modes: all host cores across events (the reported value) and
        # one thread, each on a bounded sample of the same events
        threads = min(os.cpu_count() or 1, 16)
        runs = [oracle_events_per_s(det, evs[:threads], threads) for _ in range(2)]
        r = len(runs) * threads / sum(dt for _, dt in runs)
        r1, dt1 = oracle_events_per_s(det, evs[:3], 1)
        cpu = {"value": r, "unit": "events/s", "cores": threads, "kind": "oracle",
               "sample": f"{threads} of the PU200 events, one thread per event, twice "
                         f"({sum(dt for _, dt in runs):.1f} s wall); single thread: 3 events ({dt1:.1f} s)",
               "single_thread": {"value": r1, "unit": "events/s", "cores": 1},
               "cpu_model": cpu_model(), "host_cores": os.cpu_count()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff", "data": "synthetic",
            "config": {"workload": f"{WORKLOADS[args.config]}, batch of {B} events per step",
                       "event_config": args.config,
                       "events_per_step": B, "l2": "256 MB buffer written between timed steps",
                       "parallelism": f"events sharded over {world} GPU(s)"},
            "latency_ms": {"batched_p50": float(np.percentile(step_ms, 50)),
                           "batched_p99": float(np.percentile(step_ms, 99))},
            "plain": plain,
            "streams": streams,
            "half_floats": half,
            "physics": phys,
            "serving": serving,
            "tuned": tuned,
            "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": launches,
            "stage_ms": {k: v / args.steps for k, v in stage_acc.items()},
            "objects_per_event": {"md": n_md / B, "ls": n_ls / B, "t3": n_t3 / B, "t5": n_t5 / B,
                                  "tc": sum(c["n_tc"] for c in counts) / B},
            "retries": max(c["retries"] for c in counts),
            "overflow_first_pass": counts[0]["overflow"],
            "exact_decisions_per_batch": counts[0]["recheck"],
        }
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
