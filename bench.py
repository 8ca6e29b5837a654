#!/usr/bin/env python
"""Benchmark of the MAGUS policy-step replay on one node of B300 GPUs.

One step = one replay of the batched workload: 4,096 synthetic traces x 100,000 intervals
(uint32 counter deltas, 1.64 GB) under one policy, every pair through Algorithm 1,
Algorithm 2, the jump-to-bound decision, the energy/EDP charge and the full change log,
in one persistent launch of the time-parallel kernel.  Inputs are resident in HBM when
the timed region starts (1.64 GB, larger than the 126 MB L2, so no flush is needed).
The same line carries the policy sweep (1,024 traces x 200,000 intervals x 256 policies)
and the uneven-length workload (16,384 traces, 1e3..1e6 intervals, 16 policies) under
the keys "sweep" and "uneven", each timed on its own with its roofline, one launch per
trace and the CPU oracle beside it.

With torchrun (N > 1) every rank replays its own 4,096 traces (weak scaling, no data-path
collective; a barrier and a max-reduction of the elapsed time only).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl magus|reference]

`--impl reference` times the CPU oracle (plain sequential C, OpenMP over pairs) on a
bounded sample of the same workload: the only reference this paper has.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import tracegen  # noqa: E402

METRIC = "policy-step samples/s & % HBM roofline vs plain launch; serve p50/p99 latency"
N_TRACES, N_INTERVALS = 4096, 100_000
LOG_CAP = 8192
WORKLOAD = "batched replay: 4096 traces x 100000 intervals (phase mean 40), 1 policy (W=5, inc=5, dec=-5, L=10, th=0.6)"
KERNEL_SOURCES = ["paper_2502_03796_b300/csrc/replay_tp.cu", "paper_2502_03796_b300/csrc/replay_seg.cu",
                  "paper_2502_03796_b300/csrc/replay_core.cuh", "paper_2502_03796_b300/csrc/magus_internal.h",
                  "paper_2502_03796_b300/csrc/tma.cuh"]


# the closed-loop kernels (their records: keys starting with "replay_closed")
CLOSED_SOURCES = ["paper_2502_03796_b300/csrc/replay_closed.cu", "paper_2502_03796_b300/csrc/replay_closed.h",
                  "paper_2502_03796_b300/csrc/replay_core.cuh", "paper_2502_03796_b300/csrc/magus_internal.h"]


# the static-baseline kernel (its records: keys starting with "replay_static")
STATIC_SOURCES = ["paper_2502_03796_b300/csrc/replay_static.cu", "paper_2502_03796_b300/csrc/replay_static.h",
                  "paper_2502_03796_b300/csrc/replay_core.cuh", "paper_2502_03796_b300/csrc/magus_internal.h"]


def kernel_sha(sources=None) -> str:
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured")
    return dict(hbm_gbs=6400.0, source="fallback")


def ncu_record(key: str) -> dict | None:
    """The committed ncu figures of a kernel (profiles/traffic.json), if they were taken on the
    current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(key)
    srcs = (CLOSED_SOURCES if key.startswith("replay_closed") else
            STATIC_SOURCES if key.startswith("replay_static") else KERNEL_SOURCES)
    if not e or e.get("kernel_sha") != kernel_sha(srcs):
        return None
    return e


def ncu_traffic(key: str) -> float | None:
    """Per-launch DRAM bytes of the batched replay from the committed ncu summary."""
    e = ncu_record(key)
    return float(e["dram_bytes_per_launch"]) if e else None


class _Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml ships with the driver)."""
    CLOCK_SM = 1
    REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
                   "hw_thermal_slowdown": 0x40, "hw_power_brake_slowdown": 0x80}

    def __init__(self):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")

    def handle(self, index: int):
        c = self.c
        h = c.c_void_p()
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        entry = vis.split(",")[index].strip() if vis else ""
        if entry.startswith("GPU-") or entry.startswith("MIG-"):
            rc = self.lib.nvmlDeviceGetHandleByUUID(entry.encode(), c.byref(h))
        else:
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(int(entry) if entry.isdigit() else index, c.byref(h))
        if rc != 0:
            raise RuntimeError(f"nvml handle lookup failed ({rc})")
        return h

    def clock(self, h, kind=CLOCK_SM, max_=False):
        v = self.c.c_uint()
        fn = self.lib.nvmlDeviceGetMaxClockInfo if max_ else self.lib.nvmlDeviceGetClockInfo
        if fn(h, kind, self.c.byref(v)) != 0:
            raise RuntimeError("nvml clock query failed")
        return float(v.value)

    def reasons(self, h):
        v = self.c.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        if fn(h, self.c.byref(v)) != 0:
            return set()
        return {n for n, bit in self.REASON_BITS.items() if v.value & bit}


class ClockSampler:
    """SM clock and clock-event (throttle) reasons polled through NVML every 2 ms while the
    timed region runs (read-only queries; no setting is changed)."""

    def __init__(self, index: int):
        self.samples, self.reasons = [], set()
        self.max_mhz = None
        try:
            self.nv = _Nvml()
            self.h = self.nv.handle(index)
            self.max_mhz = self.nv.clock(self.h, max_=True)
            self.ok = True
        except Exception as e:  # noqa: BLE001
            self.ok = False
            self.err = f"{type(e).__name__}: {e}"

    def _poll(self):
        while not self.stop_flag.is_set():
            try:
                self.samples.append(self.nv.clock(self.h))
                self.reasons |= self.nv.reasons(self.h)
            except Exception:  # noqa: BLE001
                pass
            time.sleep(0.002)

    def start(self):
        if not self.ok:
            return
        self.stop_flag = threading.Event()
        self.thread = threading.Thread(target=self._poll, daemon=True)
        self.thread.start()

    def stop(self) -> dict:
        if not self.ok:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=[], samples=0,
                        note="nvml unavailable: " + getattr(self, "err", "?"))
        self.stop_flag.set()
        self.thread.join(timeout=2)
        return dict(sm_mhz=float(np.median(self.samples)) if self.samples else None, sm_max_mhz=self.max_mhz,
                    reasons=sorted(self.reasons), samples=len(self.samples), source="nvml, 2 ms polling")


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float, device) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_traces(rank: int, n_traces: int = N_TRACES, n: int = N_INTERVALS) -> tracegen.TraceSet:
    # weak scaling: each rank owns a disjoint block of trace ids
    return tracegen.batched(n_traces=n_traces, n=n, seed=0, first_id=rank * n_traces)


def cpu_oracle_sample(ts: tracegen.TraceSet, policy, model, target_s: float = 6.0):
    """Time the CPU oracle on a bounded prefix of the workload's traces (~target_s wall on
    all host cores).  Returns (samples/s, threads, sample description)."""
    import oracle
    k = min(64, ts.n_traces)
    t0 = time.perf_counter()
    _, used = oracle.replay_batch(ts.data, ts.offsets[:k], ts.lengths[:k], [policy], model)
    dt = time.perf_counter() - t0
    rate = k / max(dt, 1e-9)
    k2 = int(min(ts.n_traces, max(k, rate * target_s)))
    t0 = time.perf_counter()
    _, used = oracle.replay_batch(ts.data, ts.offsets[:k2], ts.lengths[:k2], [policy], model)
    dt = time.perf_counter() - t0
    samples = int(ts.lengths[:k2].sum())
    return samples / dt, used, f"first {k2} of {ts.n_traces} traces x {N_INTERVALS} intervals, 1 policy ({dt:.1f} s wall)"


def bench_serve(seconds: float = 1.0, baseline_seconds: float = 0.25, device: int = 0) -> dict:
    """Serving workload: 100,000 node streams, Poisson arrivals at 200k requests/s, request
    sizes log-uniform in 1..4096 deltas, 8 GB admission budget; continuous batching (CUDA
    graph per launch) against one launch per request on the same arrival process."""
    from paper_2502_03796_b300 import magus
    model, policy = tracegen.default_model(), tracegen.default_policy()
    n_streams, rate = 100_000, 200_000.0
    pool = tracegen.batched(n_traces=64, n=1_000_000, seed=7).data        # delta pool
    out = {}
    for name, secs, max_req in (("batched", seconds, 0), ("per_request_launch", baseline_seconds, 1)):
        rq = tracegen.requests(int(rate * secs), rate_per_s=rate, n_streams=n_streams, seed=11)
        rng = np.random.default_rng(3)
        off = rng.integers(0, len(pool) - 4096, size=len(rq.size)).astype(np.uint64)
        sv = magus.Serve(model, policy, n_streams, mem_budget=8 << 30, device=device, max_batch_requests=max_req)
        # warm-up: a short burst through the same runtime
        sv.load(rq.arrival_s[:2000] * 0.0, rq.stream_id[:2000], rq.size[:2000], pool, off[:2000])
        st0 = sv.stats()
        lat, wall = sv.load(rq.arrival_s, rq.stream_id, rq.size, pool, off)
        st = sv.stats()
        sv.close()
        ok = lat[lat >= 0]
        samples = int(rq.size.sum())
        out[name] = dict(requests=int(len(lat)), offered_req_per_s=rate, duration_s=float(rq.arrival_s[-1]),
                         wall_s=wall, p50_ms=float(np.percentile(ok, 50) * 1e3), p99_ms=float(np.percentile(ok, 99) * 1e3),
                         p999_ms=float(np.percentile(ok, 99.9) * 1e3), max_ms=float(ok.max() * 1e3),
                         samples_per_s=samples / wall, launches=int(st["launches"] - st0["launches"]),
                         rejected=int(st["rejected"] - st0["rejected"]))
    out["streams"] = n_streams
    out["unit"] = "ms latency, samples/s"
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    model, policy = tracegen.default_model(), tracegen.default_policy()
    ts = rank_traces(0)
    import oracle
    # bounded per-step sample sized from a probe so K + W steps end within a few minutes
    k = 64
    t0 = time.perf_counter()
    oracle.replay_batch(ts.data, ts.offsets[:k], ts.lengths[:k], [policy], model)
    per_trace = (time.perf_counter() - t0) / k
    budget = 120.0 / max(args.steps + args.warmup, 1)
    k = int(min(ts.n_traces, max(16, budget / max(per_trace, 1e-9))))
    for _ in range(args.warmup):
        oracle.replay_batch(ts.data, ts.offsets[:k], ts.lengths[:k], [policy], model)
    t0 = time.perf_counter()
    used = 1
    for _ in range(args.steps):
        _, used = oracle.replay_batch(ts.data, ts.offsets[:k], ts.lengths[:k], [policy], model)
    dt = time.perf_counter() - t0
    samples = int(ts.lengths[:k].sum()) * args.steps
    value = samples / dt
    line = dict(metric=METRIC, value=value, unit="samples/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=dt / args.steps * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, sample_traces=k),
                cpu_baseline=dict(value=value, unit="samples/s", cores=used, kind="oracle",
                                  sample=f"first {k} of {ts.n_traces} traces per step"),
                e2e=dict(value=value, unit="samples/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


def static_savings(rp, d_tr, ts, policy, model, stream) -> dict:
    """The paper's metrics (Sec. 5.4) of the controlled policy against the static maximum
    (the default setting it is compared with, Sec. 5.3), per trace, averaged over traces;
    the static minimum (Sec. 6.3) for contrast.  One untimed replay of three policies."""
    import torch
    K = len(model["f_ghz"])
    pols = [policy, dict(policy, pin_level=K), dict(policy, pin_level=1)]
    out = rp.run(d_tr, ts.lengths, pols, stream=stream)
    torch.cuda.synchronize()
    E = out["energy_j"].view(-1, 3).cpu().numpy()
    T = out["time_s"].view(-1, 3).cpu().numpy()
    def metrics(k):
        e, t, e0, t0 = E[:, k], T[:, k], E[:, 1], T[:, 1]
        return dict(energy_saving_pct=float(np.mean(1 - e / e0) * 100),
                    edp_saving_pct=float(np.mean(1 - (e * t) / (e0 * t0)) * 100),
                    perf_loss_pct=float(np.mean(t / t0 - 1) * 100),
                    power_saving_pct=float(np.mean(1 - (e / t) / (e0 / t0)) * 100))
    return dict(policy=metrics(0), static_min=metrics(2),
                note="energy model of the synthetic workload, per-trace mean; not the paper's measured savings")


def time_steps(fn, steps: int, warmup: int, stream, after_warmup=None) -> float:
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if after_warmup is not None:
        after_warmup()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def sm_count(dev) -> int:
    """Streaming multiprocessors of the device (cudaDevAttrMultiProcessorCount)."""
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def alu_peak_lane_ops(sms: int, sm_mhz: float) -> float:
    """Integer-ALU pipe peak: per SM 4 partitions x 16 lanes per cycle, at the sampled clock."""
    return sms * 4 * 16 * sm_mhz * 1e6


def oracle_rate(ts, pols, model, target_s: float = 6.0):
    """The CPU oracle (all host cores, OpenMP over pairs) on a bounded prefix of the traces,
    sized from a one-trace probe to about target_s of wall time.  Returns (pair-samples/s,
    threads, sample description)."""
    import oracle
    t0 = time.perf_counter()
    oracle.replay_batch(ts.data, ts.offsets[:1], ts.lengths[:1], pols, model)
    per = max(time.perf_counter() - t0, 1e-6) / max(float(ts.lengths[0]), 1.0)
    k, tot = 0, 0.0
    while k < ts.n_traces and tot * per < target_s:
        tot += float(ts.lengths[k])
        k += 1
    t0 = time.perf_counter()
    _, used = oracle.replay_batch(ts.data, ts.offsets[:k], ts.lengths[:k], pols, model)
    dt = time.perf_counter() - t0
    n = float(ts.lengths[:k].sum()) * len(pols)
    return n / dt, used, f"first {k} of {ts.n_traces} traces x {len(pols)} policies ({dt:.1f} s wall)"


def per_trace_launches(rp, d_tr, ts, pols, stream, k: int = 256) -> dict:
    """The same replay entry point called once per trace (automatic kernel choice) on the
    first k traces: the one-launch-per-trace form the batched launch is compared with."""
    import torch
    k = min(k, ts.n_traces)
    total_ms, kernels, runs = 0.0, 0, 0
    rp.kernel_time()
    for i in range(k):
        sub_len = ts.lengths[i:i + 1]
        o = int(ts.offsets[i])
        sub = d_tr[o:o + int((sub_len[0] + 31) // 32 * 32) + 32]
        if i == 0:
            rp.run(sub, sub_len, pols, stream=stream)
            torch.cuda.synchronize()
            rp.kernel_time()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        rp.run(sub, sub_len, pols, stream=stream)
        t1.record(stream)
        torch.cuda.synchronize()
        total_ms += t0.elapsed_time(t1)
    _, _, runs, kernels = rp.kernel_time(detail=True)
    return dict(value=float(ts.lengths[:k].sum()) * len(pols) / (total_ms * 1e-3), unit="pair-interval samples/s",
                sample=f"first {k} traces, one call (automatic kernel choice) each", kernels_launched=kernels,
                ms_per_trace=total_ms / k)


def run_other(args, world, rank, local) -> int:
    """Lines for the other replay workloads: policy sweep, uneven lengths, single trace, few
    long traces."""
    line = measure_workload(args.workload, args, world, rank, local, args.steps, args.warmup,
                            plain=not args.no_plain, cpu=not args.no_cpu_baseline)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def measure_workload(kind, args, world, rank, local, steps, warmup, plain=True, cpu=True) -> dict:
    """One workload's line: the replay timed over `steps` calls after `warmup`, its roofline,
    and (rank 0) one launch per trace, the plain form and the CPU oracle beside it."""
    import torch
    from paper_2502_03796_b300 import magus
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    model = tracegen.default_model()
    if kind == "sweep":
        ts = tracegen.sweep(first_id=rank * 1024)
        pols = tracegen.sweep_policies()
        desc = "policy sweep: 1024 traces x 200000 intervals (bursty mean 10 / long mean 500 regimes), 256 policies"
    elif kind in ("ladder", "closed", "closed_ladder"):
        ts = tracegen.batched(n_traces=args.traces, seed=rank, first_id=rank * args.traces)
        mode = {"ladder": 1, "closed": 2, "closed_ladder": 3}[kind]
        pols = [dict(tracegen.default_policy(), step_mode=mode)]
        kern = "ladder kernel" if mode == 1 else ("literal kernel" if args.closed.startswith("-1") else
                                                  "segmented closed-loop kernels")
        what = {1: "one rung per decision", 2: "closed loop", 3: "closed loop, one rung per decision"}[mode]
        desc = (f"batched replay, {what} ({kern}): "
                f"{args.traces} traces x 100000 intervals (phase mean 40), 1 policy")
    elif kind == "static":
        ts = tracegen.batched(n_traces=args.traces, seed=rank, first_id=rank * args.traces)
        K = len(model["f_ghz"])
        pols = [dict(tracegen.default_policy(), pin_level=k) for k in range(1, K + 1)]
        desc = (f"static baselines at every rung ({K} pinned policies, one pass of the static kernel): "
                f"{args.traces} traces x 100000 intervals (phase mean 40)")
    elif kind == "long":
        ts = tracegen.batched(n_traces=16, n=4_000_000, seed=rank, first_id=rank * 16)
        pols = [tracegen.default_policy()]
        desc = "few long traces: 16 traces x 4000000 intervals (phase mean 40), 1 policy"
    elif kind == "uneven":
        nt = 16384 if args.traces == N_TRACES else args.traces
        ts = tracegen.uneven(n_traces=nt, seed=rank)
        pols = tracegen.sweep_policies()[:16]
        desc = f"uneven lengths: {nt} traces, log-uniform 1e3..1e6 intervals, 16 policies"
    else:
        ts = tracegen.single_trace()
        pols = [tracegen.default_policy()]
        desc = "single trace: 20000 intervals, 1 policy"
    d_tr = torch.from_numpy(ts.data.view(np.int32)).to(dev)
    rp = magus.Replay(model, device=local, mem_budget=4 << 30)
    stream = torch.cuda.current_stream(dev)
    n_pairs = ts.n_traces * len(pols)
    outs = rp.alloc(n_pairs, log_capacity=0)
    tuned = None
    if args.tile:
        rp.set_tile(*[int(x) for x in args.tile.split(",")])
    rp.set_segments(args.segments)
    if args.closed:
        rp.set_closed(*[int(x) for x in args.closed.split(",")])
    if kind in ("sweep", "uneven") and not args.tile and args.segments < 0:
        tuned, tms = rp.autotune(d_tr, ts.lengths, pols, stream=stream)
    clocks = ClockSampler(local)
    barrier(world)
    clocks.start()
    # the kernel events restart after the warm-up: they cover the timed steps only
    ms = time_steps(lambda: rp.run(d_tr, ts.lengths, pols, stream=stream, out=outs), steps, warmup, stream,
                    after_warmup=rp.kernel_time)
    clk = clocks.stop()
    barrier(world)
    ms = max_over_ranks(world, ms, dev)
    k_ms, k_main, k_n, k_kernels = rp.kernel_time(detail=True)
    pair_steps = ts.n_samples * len(pols)
    value = pair_steps * world / (ms * 1e-3)
    alg_bytes = 4 * ts.n_samples + 48 * n_pairs
    k_avg = k_ms / max(k_n, 1)
    peaks = measured_peaks()
    line = dict(metric=METRIC, value=value, unit="pair-interval samples/s", n_gpus=world, steps=steps,
                warmup=warmup, ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="u32/f64", data="synthetic",
                config=dict(workload=desc, traces=ts.n_traces, samples=ts.n_samples, policies=len(pols),
                            tile=list(tuned) if tuned else None, outputs="energy, EDP, time, counts, hash (no entries)"),
                roofline=dict(bound="hbm", achieved=alg_bytes / (k_avg * 1e-3) / 1e9,
                              peak=peaks["hbm_gbs"], unit="GB/s", frac=alg_bytes / (k_avg * 1e-3) / 1e9 / peaks["hbm_gbs"],
                              traffic=None, kernel_ms=k_avg, main_kernel_ms=k_main / max(k_n, 1),
                              alg_bytes_per_launch=alg_bytes),
                gpu_launches=k_kernels, clocks=clk)
    if kind in ("closed", "closed_ladder"):
        segs, second, final, logged = rp.closed_stats()
        line["config"]["closed_replay"] = dict(segments=segs, second_replays=second, final_pass_replays=final,
                                               log_pass_replays=logged)
    # many policies per byte read: the integer ALU pipe bounds these launches; report that
    # roofline (ncu lane-operations per (interval, policy), committed with the source hash,
    # against the device's SMs x 64 integer lanes per cycle at the sampled SM clock)
    # (the closed loop: one thread per segment replays its rounds in order, integer ALU work;
    # its record holds for the benchmark's 4,096 traces, whose automatic segments fix the
    # share of burn-in rounds)
    if kind in ("closed", "closed_ladder"):
        key = "replay_closed_batched" if kind == "closed" else "replay_closed_ladder_batched"
        rec = ncu_record(key) if ts.n_traces == N_TRACES else None
    elif kind == "static":
        # one pass over the traces: the HBM roofline stands; the record gives the DRAM bytes
        # of one launch on the benchmark's 4,096 traces
        rec = ncu_record("replay_static_batched") if ts.n_traces == N_TRACES else None
        if rec:
            line["roofline"]["traffic"] = rec["dram_bytes_per_launch"]
            line["roofline"]["kernel"] = "replay_static_kernel"
        rec = None
    else:
        rec = ncu_record(f"replay_tp_{kind}")
    sms = sm_count(dev)
    line["config"]["sms"] = sms
    if rec and rec.get("alu_lane_ops_per_pair_interval") and clk.get("sm_mhz"):
        alu_ach = rec["alu_lane_ops_per_pair_interval"] * pair_steps / (k_avg * 1e-3)
        alu_peak = alu_peak_lane_ops(sms, clk["sm_mhz"])
        hbm = dict(line["roofline"])
        line["roofline"] = dict(bound="alu", achieved=alu_ach, peak=alu_peak, unit="lane-ops/s",
                                frac=alu_ach / alu_peak, ops_per_pair_interval=rec["alu_lane_ops_per_pair_interval"],
                                peak_source=f"derived: {sms} SMs (device query) x 64 integer lanes per cycle x "
                                            "sampled SM clock",
                                traffic=None, kernel_ms=k_avg, hbm=hbm)
    if plain and rank == 0:
        line["one_launch_per_trace"] = per_trace_launches(rp, d_tr, ts, pols, stream)
        # plain form (one launch per trace, literal FP64) on a small sample
        if kind == "long":
            kp, p_len = 1, np.array([200_000], dtype=np.uint64)     # a prefix of the first trace
        else:
            kp = 4 if kind != "single" else 1
            p_len = ts.lengths[:kp]
        sub = d_tr[:int(ts.offsets[kp - 1]) + int((ts.lengths[kp - 1] + 31) // 32 * 32)] if kp > 1 else d_tr
        rp.plain(sub, p_len, pols, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rp.plain(sub, p_len, pols, stream=stream)
        torch.cuda.synchronize()
        line["plain_launch"] = dict(value=float(p_len.sum()) * len(pols) / (time.perf_counter() - t0),
                                    unit="pair-interval samples/s",
                                    sample=f"first {kp} traces" if kind != "long" else "first 200000 intervals of trace 0")
    if cpu and rank == 0:
        rate, used, sample = oracle_rate(ts, pols, model)
        line["cpu_baseline"] = dict(value=rate, unit="pair-interval samples/s", cores=used, kind="oracle",
                                    sample=sample)
    rp.close()
    del d_tr
    torch.cuda.empty_cache()
    return line


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="magus", choices=["magus", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--tile", default="", help="time_groups,policy_slots (default: automatic)")
    ap.add_argument("--closed", default="",
                    help="closed loop: seg_rounds[,burn_rounds] (default automatic; -1: literal kernel)")
    ap.add_argument("--segments", type=int, default=-1,
                    help="-1 automatic, 0 tile kernel, >0 segment kernel with this many rounds per segment")
    ap.add_argument("--traces", type=int, default=N_TRACES, help="traces per GPU (profiling runs use fewer)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-savings", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="leave the policy-sweep workload out of the default line")
    ap.add_argument("--no-uneven", action="store_true", help="leave the uneven-length workload out of the default line")
    ap.add_argument("--mw-steps", type=int, default=10, help="timed steps of the sweep / uneven workloads")
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "sweep", "uneven", "single", "long", "ladder", "closed", "closed_ladder",
                             "static"],
                    help="batched (default, the headline line); sweep / uneven / single print their own line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload != "batched":
        return run_other(args, world, rank, local)

    import torch
    from paper_2502_03796_b300 import magus

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    model, policy = tracegen.default_model(), tracegen.default_policy()
    ts = rank_traces(rank, n_traces=args.traces)
    samples_per_step = ts.n_samples
    d_tr = torch.from_numpy(ts.data.view(np.int32)).to(dev)
    rp = magus.Replay(model, device=local, mem_budget=2 << 30)
    if args.tile:
        rp.set_tile(*[int(x) for x in args.tile.split(",")])
    rp.set_segments(args.segments)
    outs = rp.alloc(ts.n_traces, log_capacity=LOG_CAP)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        rp.run(d_tr, ts.lengths, [policy], stream=stream, out=outs)
    torch.cuda.synchronize(dev)
    rp.kernel_time()
    rp.status()

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rp.run(d_tr, ts.lengths, [policy], stream=stream, out=outs)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(world, ms, dev)
    k_ms, k_main_ms, k_n, k_kernels = rp.kernel_time(detail=True)
    if rp.status() != 0:
        raise RuntimeError("device-side status error during the timed region")
    seg_path = k_kernels > k_n
    value = samples_per_step * world * args.steps / (ms * 1e-3)

    # algorithmic bytes of one launch: every delta read once, per-pair totals written once,
    # every change-log entry written once
    out_np = outs[0]
    n_changes = int(out_np["n_changes"].sum().item())
    alg_bytes = 4 * samples_per_step + 48 * ts.n_traces + 4 * min(n_changes, LOG_CAP * ts.n_traces)
    k_avg_ms = k_ms / max(k_n, 1)
    peaks = measured_peaks()
    # the replay (all of its kernels) against the HBM roofline: for the segment path the
    # combine kernel's time is included, so the fraction is the replay's, not flattering
    achieved = alg_bytes / (k_avg_ms * 1e-3) / 1e9
    traffic = ncu_traffic("replay_seg_batched" if seg_path else "replay_tp_batched")
    roofline = dict(bound="hbm", achieved=achieved, peak=peaks["hbm_gbs"], unit="GB/s",
                    frac=achieved / peaks["hbm_gbs"], traffic=traffic,
                    peak_source=f"{peaks['source']} (MEASURED_PEAKS.json hbm_gbs)" if peaks["source"] == "measured"
                    else "fallback 6.4 TB/s",
                    kernel=("replay_seg_kernel<1> + combine_kernel" if seg_path else
                            f"replay_tp_kernel<4,1,1,{policy['direv_length']}> (the automatic tile for one "
                            f"policy group, its instance for W = {policy['direv_length']})"),
                    kernel_ms=k_avg_ms, main_kernel_ms=k_main_ms / max(k_n, 1),
                    alg_bytes_per_launch=alg_bytes, frac_of_nominal_8tbs=achieved / 8000.0)
    # the pipe that actually bounds the kernel: integer ALU lane-operations per interval
    # (ncu, committed with the kernel-source hash) against 148 SMs x 4 partitions x 16 lanes
    # x the SM clock sampled during the timed region
    rec = ncu_record("replay_tp_batched") if not seg_path else None
    sms = sm_count(dev)
    if rec and rec.get("alu_lane_ops_per_interval") and clk.get("sm_mhz"):
        alu_ach = rec["alu_lane_ops_per_interval"] * samples_per_step / (k_main_ms / max(k_n, 1) * 1e-3)
        alu_peak = alu_peak_lane_ops(sms, clk["sm_mhz"])
        roofline["alu"] = dict(achieved=alu_ach, peak=alu_peak, unit="lane-ops/s", frac=alu_ach / alu_peak,
                               ops_per_interval=rec["alu_lane_ops_per_interval"],
                               peak_source=f"derived: {sms} SMs (device query) x 64 integer lanes per cycle x "
                                           "sampled SM clock")

    line = dict(metric=METRIC, value=value, unit="samples/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="u32/f64", data="synthetic",
                config=dict(workload=WORKLOAD if args.traces == N_TRACES else
                            WORKLOAD.replace(str(N_TRACES), str(args.traces)), traces_per_gpu=ts.n_traces, intervals=N_INTERVALS, policies=1,
                            outputs="energy, EDP, time, change count, change hash, hf count, full change log",
                            l2="inputs 1.64 GB per GPU > 126 MB L2 (no flush needed)",
                            parallelism=f"dp{world} (traces sharded, no collective)"),
                roofline=roofline, gpu_launches=k_kernels, clocks=clk)

    if rank == 0 and not args.no_plain:
        # the plain form: one launch per trace, one thread per policy, literal FP64
        k = 16
        sub = tracegen.TraceSet(ts.lengths[:k], ts.offsets[:k], ts.data[:int(ts.offsets[k])])
        d_sub = d_tr[:int(ts.offsets[k])]
        rp.plain(d_sub, sub.lengths, [policy], stream=stream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rp.plain(d_sub, sub.lengths, [policy], stream=stream)
        torch.cuda.synchronize(dev)
        pdt = time.perf_counter() - t0
        plain_rate = sub.n_samples / pdt
        line["plain_launch"] = dict(value=plain_rate, unit="samples/s", sample=f"{k} traces, {k} launches",
                                    speedup=value / world / plain_rate)
        # the same entry point called once per trace (the time-parallel kernels, chosen
        # automatically per call) on the first 256 traces
        olt = per_trace_launches(rp, d_tr, ts, [policy], stream)
        olt["speedup"] = value / world / olt["value"]
        line["one_launch_per_trace"] = olt

    if rank == 0 and not args.no_e2e:
        # end to end through the public API with host buffers: pinned host traces in,
        # host outputs back, copies inside the timed region
        pinned = torch.from_numpy(ts.data.view(np.int32)).pin_memory()
        host_tr = pinned.numpy().view(np.uint32)
        n_pairs = ts.n_traces
        hout = {k: torch.zeros(n_pairs, dtype=torch.float64).pin_memory().numpy()
                for k in ("energy_j", "edp_js", "time_s")}
        for k in ("n_changes", "change_hash", "n_hf"):
            hout[k] = torch.zeros(n_pairs, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
        # the full change log comes back too: the same work as the device-timed replay
        hout["log"] = torch.zeros(n_pairs * LOG_CAP, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        rp.run_host(host_tr, ts.lengths, [policy], out=hout)
        ksteps = max(10, min(args.steps, 20))
        t0 = time.perf_counter()
        for _ in range(ksteps):
            rp.run_host(host_tr, ts.lengths, [policy], out=hout)
        edt = time.perf_counter() - t0
        # the bound of this path: the host-to-device link, measured with one plain pinned
        # copy of the same bytes outside the timed loop
        dst = torch.empty(ts.data.nbytes // 4, dtype=torch.int32, device=dev)
        dst.copy_(pinned, non_blocking=True)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        dst.copy_(pinned, non_blocking=True)
        torch.cuda.synchronize(dev)
        link_gbs = ts.data.nbytes / (time.perf_counter() - t1) / 1e9
        del dst
        h2d_gbs = ts.data.nbytes * ksteps / edt / 1e9
        line["e2e"] = dict(value=samples_per_step * ksteps / edt, unit="samples/s",
                           h2d_bytes_per_step=int(ts.data.nbytes), d2h_bytes_per_step=48 * n_pairs + 4 * LOG_CAP * n_pairs,
                           steps=ksteps, api="magus_replay_run_host", log="full change log copied back",
                           h2d_gbs=h2d_gbs, link_gbs=link_gbs, link_frac=h2d_gbs / link_gbs)
        del hout
        rp.kernel_time()

    if rank == 0 and not args.no_savings:
        line["savings_vs_static_max"] = static_savings(rp, d_tr, ts, policy, model, stream)

    if rank == 0 and not args.no_serve:
        line["serve"] = bench_serve(device=local)

    if rank == 0 and not args.no_cpu_baseline:
        rate, used, sample = cpu_oracle_sample(ts, policy, model)
        line["cpu_baseline"] = dict(value=rate, unit="samples/s", cores=used, kind="oracle", sample=sample)

    rp.close()
    del d_tr, outs
    torch.cuda.empty_cache()
    # the many-policy workloads (policy sweep, uneven lengths) at full size: each with its own
    # timing, roofline, one launch per trace and CPU oracle
    for kind, skip in (("sweep", args.no_sweep), ("uneven", args.no_uneven)):
        if skip:
            continue
        sub = argparse.Namespace(**vars(args))
        sub.traces = N_TRACES
        w = measure_workload(kind, sub, world, rank, local, args.mw_steps, 3, plain=not args.no_plain,
                             cpu=not args.no_cpu_baseline)
        line[kind] = {k: w[k] for k in ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "config",
                                        "roofline", "gpu_launches", "clocks", "one_launch_per_trace",
                                        "plain_launch", "cpu_baseline") if k in w}

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
