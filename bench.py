"""Throughput benchmark of the TVOLAP hot path on GB300.

Workload (default): 64 independent channels, L = 256 (2L = 512, 4L = 1024),
480000 samples per channel (10 s at 48 kHz, pink-ish noise), eight stored
48000-tap impulse responses per channel (M = 94 partitions), a new filter at
every block mixed from two stored responses by a random walk. One step is the
whole path over that batch: transform the 512 stored responses into the
partition bank (Eqs. 2, 4, 6), then the offline TVOLAP of all channels
(forward transforms, Eq. 7 multiply-accumulate, inverse transforms and
overlap-add). Inputs are resident in device memory when the timed region
starts; the step's working set (about 1.5 GB) is far larger than the 129 MB
L2, so no flush is needed between steps.

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "channel-samples/s"
UNIT = "channel-samples/s"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP32 FMA peak from unit counts and clocks: 152 SMs x 128 FP32 lanes x 2 flops x clock.
SMS, FP32_LANES = 152, 128

# DRAM bytes (read + write) of one launch of the persistent multiply-accumulate kernel at
# the default 64-channel workload: an ncu capture of the same kernel at 32 channels, scaled
# by the channel count (the traffic grows in proportion to it).
MAC_TRAFFIC_BYTES = 2 * (309.411072e6 + 215.104000e6)

# DRAM bytes (read + write) of one launch of the fused adjoint kernel at the
# 16-channel differentiable workload: an ncu capture of the same kernel at 2
# channels, scaled by the channel count.
ADJ_TRAFFIC_BYTES = 8 * (369.795072e6 + 310.738688e6)


def fp32_peak_tflops(mhz: float) -> float:
    return SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12


def _is_num(v: str) -> bool:
    try:
        float(v)
        return True
    except ValueError:
        return False


def smi_index_of(uuid: str, listing: str, fallback: str) -> str:
    """nvidia-smi's index of the GPU whose UUID is ``uuid``, from the lines
    ``index, uuid`` of ``listing``; ``fallback`` when none matches."""
    want = uuid.strip().lower()
    want = want[4:] if want.startswith("gpu-") else want
    for line in listing.splitlines():
        p = [v.strip() for v in line.split(",")]
        if len(p) == 2:
            u = p[1].lower()
            if (u[4:] if u.startswith("gpu-") else u) == want and want:
                return p[0]
    return fallback


def smi_index(dev) -> str:
    """nvidia-smi's id of torch device ``dev``. CUDA's device order and
    CUDA_VISIBLE_DEVICES need not follow nvidia-smi's numbering, so the device
    is found by its UUID; the CUDA index is the fallback."""
    fallback = str(dev.index if dev.index is not None else 0)
    try:
        import torch
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        listing = subprocess.run(["nvidia-smi", "--query-gpu=index,uuid", "--format=csv,noheader"],
                                 capture_output=True, text=True, timeout=20).stdout
    except Exception:
        return fallback
    return smi_index_of(uuid, listing, fallback)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during a timed region.

    ``start(prime)`` launches nvidia-smi (a row every PERIOD_MS) and, given
    ``prime`` (one untimed step, synchronised), keeps the GPU busy with it until
    the sampler's first row has arrived (at most ``wait_s``), so that sampling
    is live and the clocks are those under load when the region opens. The
    region is the ``with`` block. Every row carries nvidia-smi's own timestamp
    (else the time it was read) and only rows stamped inside the region are
    summarised; a region shorter than the sampling period reports the row
    nearest to it, with its distance.
    """
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    PERIOD_MS = 25

    def __init__(self, index):
        self.index = index               # nvidia-smi's id of the GPU (see smi_index)
        self.proc = None
        self.reader = None
        self.lines = []
        self.first = threading.Event()
        self.primed = 0
        self.t_open = self.t_close = None

    def start(self, prime=None, wait_s: float = 3.0):
        if self.proc is not None:
            return self
        try:
            self.proc = subprocess.Popen(self.command(), stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        deadline = time.time() + wait_s
        try:
            while prime is not None and not self.first.is_set() and time.time() < deadline:
                prime()
                self.primed += 1
        except BaseException:
            self._stop()
            raise
        return self

    def command(self):
        return ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)]

    def _read(self):
        try:
            for line in self.proc.stdout:
                self.lines.append((time.time(), line))
                self.first.set()
        except (OSError, ValueError):
            pass

    def __enter__(self):
        self.start()
        self.t_open = time.time()
        return self

    def __exit__(self, *exc):
        self.t_close = time.time()
        self._stop()

    def _stop(self):
        if self.proc is None or self.proc.poll() is not None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.reader.join(timeout=5)

    def _rows(self):
        rows = []
        for arrived, line in list(self.lines):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = arrived                 # unparsed stamp: the time the row was read
            rows.append((ts, p))
        return rows

    def summary(self):
        rows = self._rows()
        if not rows or self.t_open is None or self.t_close is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        inside = [p for ts, p in rows if self.t_open <= ts <= self.t_close]
        res = {}
        if inside:
            res["samples"] = len(inside)
        else:
            mid = 0.5 * (self.t_open + self.t_close)
            ts, p = min(rows, key=lambda r: abs(r[0] - mid))
            inside = [p]
            res["samples"] = 0
            res["nearest_ms"] = round(1e3 * max(self.t_open - ts, ts - self.t_close, 0.0), 1)
        mhz = [float(p[2]) for p in inside if _is_num(p[2])]
        mx = [float(p[3]) for p in inside if _is_num(p[3])]
        reasons = sorted({self.REASONS[i] for p in inside for i in range(4)
                          if p[6 + i].lower().startswith("active")})
        res.update({"sm_mhz": statistics.median(mhz) if mhz else None,
                    "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                    "region_ms": round(1e3 * (self.t_close - self.t_open), 1),
                    "smi_id": str(self.index)})
        if self.primed:
            res["prime_steps"] = self.primed
        return res


def workload(args):
    from synth import workloads as W
    return W.plain_at_scale(n_ch=args.channels, N=args.samples, ir_len=args.ir_len)


def mac_terms(nb: int, M: int) -> int:
    """Number of (block, partition) products of Eq. 7 with t - 2m >= 0."""
    t = np.arange(nb)
    return int(np.minimum(M, t // 2 + 1).sum())


def job_rate(elapsed_ms: float, units_per_rank_step: float, ws: int, steps: int, device):
    """Whole-job rate of a replicated run: the slowest rank's elapsed time (an
    all-reduce MAX; every rank gets it) and the units all ranks processed per
    second. With one rank no collective is called."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed_ms = float(tt.item())
    return elapsed_ms, units_per_rank_step * ws * steps / (elapsed_ms * 1e-3)


# --------------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2310_00319_gb300 import Plan, costmodel
    from paper_2310_00319_gb300.tvolap import n_blocks_for

    ws, rank, local = _dist()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    wl = workload(args)
    L, M, P = wl.L, wl.M, 2 * wl.L
    n_ch, N = wl.n_in, wl.N
    nb = n_blocks_for(wl.out_len, L)
    stream = torch.cuda.current_stream(dev)

    plan = Plan(L, M, n_in=n_ch, n_out=wl.n_out, out_to_in=wl.out_to_in,
                n_slots=wl.irs.shape[0], device=dev)
    if args.staging is not None:
        plan.set_option(1, args.staging)
    x = torch.from_numpy(wl.x).to(dev)
    irs = torch.from_numpy(wl.irs).to(dev)
    sa = torch.from_numpy(wl.sched_a).to(dev)
    sb = torch.from_numpy(wl.sched_b).to(dev)
    sal = torch.from_numpy(wl.sched_alpha).to(dev)
    X = torch.empty((n_ch, nb, P), dtype=torch.complex64, device=dev)
    Y = torch.empty((wl.n_out, nb, P), dtype=torch.complex64, device=dev)
    y = torch.empty((wl.n_out, wl.out_len), dtype=torch.float32, device=dev)
    lib, h = plan.lib, plan.h
    from paper_2310_00319_gb300.tvolap import _ptr
    from paper_2310_00319_gb300 import _lib as L_

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        L_.check(lib.tvolap_load_bank(h, 0, irs.shape[0], _ptr(irs), irs.shape[1], irs.shape[1]),
                 "load_bank")
        if ev:
            ev[1].record(stream)
        L_.check(lib.tvolap_forward_spectra(h, _ptr(x), N, N, nb, _ptr(X)), "forward")
        if ev:
            ev[2].record(stream)
        L_.check(lib.tvolap_mac(h, _ptr(X), nb, _ptr(sa), _ptr(sb), _ptr(sal), sa.shape[1],
                                _ptr(Y)), "mac")
        if ev:
            ev[3].record(stream)
        L_.check(lib.tvolap_inverse_ola(h, _ptr(Y), nb, _ptr(y), wl.out_len, wl.out_len),
                 "inverse")
        if ev:
            ev[4].record(stream)

    launches_per_step = 5     # bank, forward, MAC group + overflow, inverse
    for _ in range(args.warmup):
        step()
    plan.check()
    torch.cuda.synchronize(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(smi_index(dev)).start(prime=lambda: (step(), torch.cuda.synchronize(dev)))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with clk:
        t0.record(stream)
        for i in range(args.steps):
            step(evs[i])
        t1.record(stream)
        torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    elapsed_ms = t0.elapsed_time(t1)
    stage_ms = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(4)] for e in evs])
    plan.check()
    elapsed_ms, value = job_rate(elapsed_ms, wl.n_out * wl.out_len, ws, args.steps, dev)
    ms_per_step = elapsed_ms / args.steps

    # dominant kernel: the Eq. 7 multiply-accumulate, FP32 ALU bound
    peaks, peak_kind = _peaks()
    clocks = clk.summary()
    mac_ms = float(stage_ms[:, 2].mean())
    flops = mac_terms(nb, M) * P * wl.n_out * costmodel.mac_flops_per_block_bin_partition(True)
    achieved = flops / (mac_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    staging = 0 if args.staging is None else args.staging
    traffic = args.traffic
    if (traffic is None and staging == 0 and args.channels == 64 and args.samples == 480000
            and args.ir_len == 48000):
        traffic = MAC_TRAFFIC_BYTES
    kernel = {0: "k_mac_signal_persist", 1: "k_mac_signal_lsu"}.get(staging, "k_mac_signal_group")
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "kernel": kernel,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock (derived)"}
    # the transform stages are memory bound: algorithmic bytes / time vs measured HBM copy
    bytes_fwd = 4.0 * n_ch * N + 8.0 * P * n_ch * nb
    bytes_inv = 8.0 * P * wl.n_out * nb + 4.0 * wl.n_out * wl.out_len
    bytes_bank = 4.0 * irs.numel() + 8.0 * P * M * irs.shape[0]
    hbm = peaks.get("hbm_gbs", 6800.0)
    st = stage_ms.mean(0)
    stages = {
        "bank_fft": {"ms": round(float(st[0]), 4),
                     "gbs": round(bytes_bank / (st[0] * 1e-3) / 1e9, 1)},
        "forward_fft": {"ms": round(float(st[1]), 4),
                        "gbs": round(bytes_fwd / (st[1] * 1e-3) / 1e9, 1)},
        "mac": {"ms": round(float(st[2]), 4), "tflops": round(achieved, 3)},
        "inverse_ola": {"ms": round(float(st[3]), 4),
                        "gbs": round(bytes_inv / (st[3] * 1e-3) / 1e9, 1)},
        "hbm_peak_gbs": hbm,
    }
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name + f"_N{N}_ir{wl.ir_len}", "channels": wl.n_out,
                   "L": L, "M": M, "fft_len": 4 * L, "ir_len": wl.ir_len,
                   "stored_irs_per_channel": 8, "filter": "new mix every block",
                   "samples_per_channel": wl.out_len, "blocks": nb,
                   "per_gpu_units": wl.n_out * wl.out_len,
                   "l2": "working set ~1.5 GB >> 129 MB L2; no flush",
                   "parallelism": f"replicas x{ws}"},
        "roofline": roofline, "stages": stages, "peaks": peak_kind,
        "clocks": clocks, "gpu_launches": launches_per_step * args.steps,
    }
    if rank == 0 and not args.skip_extras:
        out["e2e"] = run_e2e(args, plan, wl, dev, stream)
        out["vs_per_source"] = run_per_source(args, wl, dev, stream, ms_per_step)
        out["stream"] = run_stream(args, wl, dev, stream)
        out["static_scratch"] = run_static(args, wl, dev, stream)
        # the same streaming ticks at 4x the channels: the tick reads about
        # 296 MB of delay line and filter spectra, more than the L2 holds
        from synth import workloads as W
        wl4 = W.plain_at_scale(n_ch=4 * args.channels, N=650 * wl.L, ir_len=args.ir_len)
        out["stream_beyond_l2"] = run_stream(args, wl4, dev, stream)
        del wl4
    if rank == 0 and not args.skip_extras and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(args, wl, budget_s=args.cpu_seconds,
                                           y_channel0=y[0].cpu().numpy())
        out["accuracy_plain_mono"] = accuracy_plain_mono(dev)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


def run_e2e(args, plan, wl, dev, stream):
    """Same metric through the public API with host buffers: every step copies
    its inputs from pinned host memory, processes them and copies its output
    back, all inside the timed region. Two sets of device buffers let step k+1's
    copies run on their own streams while step k computes (copy-in, compute
    and copy-out of one step stay in order through events)."""
    import torch
    xh = torch.from_numpy(wl.x).pin_memory()
    irh = torch.from_numpy(wl.irs).pin_memory()
    sah = torch.from_numpy(wl.sched_a).pin_memory()
    sbh = torch.from_numpy(wl.sched_b).pin_memory()
    salh = torch.from_numpy(wl.sched_alpha).pin_memory()
    host_in = (xh, irh, sah, sbh, salh)
    yh = [torch.empty((wl.n_out, wl.out_len), dtype=torch.float32).pin_memory() for _ in range(2)]
    dev_in = [[torch.empty_like(t, device=dev) for t in host_in] for _ in range(2)]
    yd = [torch.empty((wl.n_out, wl.out_len), dtype=torch.float32, device=dev) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_free = [torch.cuda.Event() for _ in range(2)]
    for b in range(2):
        ev_free[b].record(s_out)

    def step(k):
        b = k & 1
        s_in.wait_event(ev_free[b])                 # step k-2 has left this buffer set
        with torch.cuda.stream(s_in):
            for d, h in zip(dev_in[b], host_in):
                d.copy_(h, non_blocking=True)
        ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        xd, ird, sad, sbd, sald = dev_in[b]
        plan.load_bank(0, ird)
        plan.process_signal(xd, sad, sbd, sald, out_len=wl.out_len, out=yd[b])
        ev_comp[b].record(stream)
        s_out.wait_event(ev_comp[b])
        with torch.cuda.stream(s_out):
            yh[b].copy_(yd[b], non_blocking=True)
        ev_free[b].record(s_out)

    steps = max(3, args.steps)
    for k in range(3):
        step(k)
    torch.cuda.synchronize(dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(s_in)
    for k in range(steps):
        step(k)
    t1.record(s_out)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1) / steps
    h2d = sum(t.numel() * t.element_size() for t in host_in)
    d2h = yh[0].numel() * yh[0].element_size()
    return {"value": round(wl.n_out * wl.out_len / (ms * 1e-3), 1), "unit": UNIT,
            "ms_per_step": round(ms, 4), "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps,
            "note": "copies of consecutive steps overlap compute on separate streams"}


def run_per_source(args, wl, dev, stream, batched_ms):
    """The plain per-source form: one single-channel process_signal call per
    channel in a Python loop, same kernels, no batching."""
    import torch
    from paper_2310_00319_gb300 import Plan
    plans = []
    x = torch.from_numpy(wl.x).to(dev)
    sa = torch.from_numpy(wl.sched_a).to(dev)
    sb = torch.from_numpy(wl.sched_b).to(dev)
    sal = torch.from_numpy(wl.sched_alpha).to(dev)
    irs = torch.from_numpy(wl.irs).to(dev)
    n_ir = irs.shape[0] // wl.n_out
    ys = torch.empty((wl.n_out, wl.out_len), dtype=torch.float32, device=dev)
    p = Plan(wl.L, wl.M, n_in=1, n_out=1, n_slots=n_ir, device=dev)
    sa_l = (sa - (torch.arange(wl.n_out, device=dev, dtype=torch.int32) * n_ir)[:, None]).contiguous()
    sb_l = (sb - (torch.arange(wl.n_out, device=dev, dtype=torch.int32) * n_ir)[:, None]).contiguous()

    def step():
        for c in range(wl.n_out):
            p.load_bank(0, irs[c * n_ir:(c + 1) * n_ir])
            p.process_signal(x[c:c + 1], sa_l[c:c + 1], sb_l[c:c + 1], sal[c:c + 1],
                             out_len=wl.out_len, out=ys[c:c + 1])

    step()
    torch.cuda.synchronize(dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 3
    t0.record(stream)
    for _ in range(n):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1) / n
    p.check()
    p.close()
    return {"per_source_ms_per_step": round(ms, 4), "batched_ms_per_step": round(batched_ms, 4),
            "ratio": round(ms / batched_ms, 3)}


def run_stream(args, wl, dev, stream, ticks=600, warm=50):
    """Streaming ticks (process_block) on the same channels and filters: per
    tick device time, p50 / p99, against the L / fs deadline."""
    import torch
    from paper_2310_00319_gb300 import Plan, costmodel
    p = Plan(wl.L, wl.M, n_in=wl.n_in, n_out=wl.n_out, out_to_in=wl.out_to_in,
             n_slots=wl.irs.shape[0], device=dev)
    p.load_bank(0, torch.from_numpy(wl.irs).to(dev))
    L = wl.L
    x = torch.from_numpy(wl.x[:, :(ticks + warm) * L]).to(dev)
    sa = torch.from_numpy(np.ascontiguousarray(wl.sched_a.T)).to(dev)
    sb = torch.from_numpy(np.ascontiguousarray(wl.sched_b.T)).to(dev)
    sal = torch.from_numpy(np.ascontiguousarray(wl.sched_alpha.T)).to(dev)
    blocks = [x[:, t * L:(t + 1) * L].contiguous() for t in range(ticks + warm)]
    out = torch.empty((wl.n_out, L), dtype=torch.float32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(ticks)]
    for t in range(warm):
        p.process_block(blocks[t], out, sa[t], sb[t], sal[t])
    torch.cuda.synchronize(dev)
    for i in range(ticks):
        t = warm + i
        evs[i][0].record(stream)
        p.process_block(blocks[t], out, sa[t], sb[t], sal[t])
        evs[i][1].record(stream)
    torch.cuda.synchronize(dev)
    # constant load (Section 4): the same ticks with one selection kept for all
    # blocks (no filter switch) cost the same as a new selection every block
    fixed = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(ticks)]
    for i in range(ticks):
        t = warm + i
        fixed[i][0].record(stream)
        p.process_block(blocks[t], out, sa[warm], sb[warm], sal[warm])
        fixed[i][1].record(stream)
    torch.cuda.synchronize(dev)
    # the three stages timed on their own (events around each; the next tick
    # waits for the previous one's events)
    from paper_2310_00319_gb300.tvolap import OPT_STAGE_TIMING
    p.set_option(OPT_STAGE_TIMING, 1)
    for i in range(ticks):
        t = warm + i
        p.process_block(blocks[t], out, sa[t], sb[t], sal[t])
    st_ms, n_timed = p.stage_times()
    p.set_option(OPT_STAGE_TIMING, 0)
    p.check()
    ms = np.array([a.elapsed_time(b) for a, b in evs])
    ms_fixed = np.array([a.elapsed_time(b) for a, b in fixed])
    p.close()
    deadline_ms = L / 48000 * 1e3
    bpt = costmodel.stream_mac_bytes_per_tick(wl.n_out, 2 * L, wl.M, 2)
    mac_ms = st_ms[1] / n_timed
    peaks, _ = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    mac_gbs = bpt / (mac_ms * 1e-3) / 1e9
    return {"ticks": ticks, "channels": wl.n_out,
            "tick_ms_p50": round(float(np.percentile(ms, 50)), 4),
            "tick_ms_p99": round(float(np.percentile(ms, 99)), 4),
            "deadline_ms": round(deadline_ms, 4),
            "channel_samples_per_s": round(wl.n_out * L / (ms.mean() * 1e-3), 1),
            "mac_bytes_per_tick": bpt,
            "logical_gbs_per_tick": round(bpt / (ms.mean() * 1e-3) / 1e9, 1),
            "stages_ms_per_tick": {"forward": round(st_ms[0] / n_timed, 5),
                                   "mac": round(mac_ms, 5),
                                   "inverse": round(st_ms[2] / n_timed, 5)},
            "mac_roofline": {"bound": "hbm", "achieved": round(mac_gbs, 1), "peak": hbm,
                             "unit": "GB/s", "frac": round(mac_gbs / hbm, 4),
                             "kernel": "k_mac_stream (delay line + 2 filter spectra read, "
                                       "Y written; algorithmic bytes)",
                             "working_set_mb": round(bpt / 1e6, 1),
                             "l2_mb": round(torch.cuda.get_device_properties(dev).L2_cache_size
                                            / 1e6, 1)},
            "constant_load": {"switching_every_block_ms_mean": round(float(ms.mean()), 5),
                              "fixed_selection_ms_mean": round(float(ms_fixed.mean()), 5)}}


def run_stream_only(args):
    """Streaming ticks alone (process_block, one hop per call) on
    ``--channels`` channels of the default workload's shape (L = 256, M = 94,
    eight stored responses per channel, a new mixed filter every block)."""
    import torch
    from synth import workloads as W
    dev = torch.device("cuda", 0)
    ticks = max(args.steps, 10)
    wl = W.plain_at_scale(n_ch=args.channels, N=(ticks + 50) * 256, ir_len=args.ir_len)
    r = run_stream(args, wl, dev, torch.cuda.current_stream(dev), ticks=ticks)
    return {"metric": "channel-samples/s (streaming ticks)",
            "value": r["channel_samples_per_s"], "unit": UNIT, "n_gpus": 1, "steps": ticks,
            "warmup": 50, "ms_per_step": r["tick_ms_p50"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"plain_at_scale_streaming_{args.channels}ch_L256_M94"},
            "roofline": dict(r["mac_roofline"], traffic=None), "stream": r}


def run_static(args, wl, dev, stream, reps=10):
    """tvolap_process_signal_static (its scratch in the library's fixed device
    array, no allocation) against tvolap_process_signal (workspace from
    cudaMalloc) on two channels of the default workload: the largest slice
    whose block spectra fit the 32 MiB array."""
    import torch
    from paper_2310_00319_gb300 import Plan
    from paper_2310_00319_gb300 import _lib as L_
    from paper_2310_00319_gb300.tvolap import _ptr
    ch = 2
    p = Plan(wl.L, wl.M, n_in=ch, n_out=ch, n_slots=wl.irs.shape[0], device=dev)
    p.load_bank(0, torch.from_numpy(wl.irs).to(dev))
    x = torch.from_numpy(wl.x[:ch]).to(dev)
    sa, sb, sal = (torch.from_numpy(a[:ch]).to(dev) for a in (wl.sched_a, wl.sched_b,
                                                             wl.sched_alpha))
    y = torch.empty((ch, wl.out_len), dtype=torch.float32, device=dev)
    N = wl.N

    def static():
        L_.check(p.lib.tvolap_process_signal_static(
            p.h, _ptr(x), N, N, _ptr(sa), _ptr(sb), _ptr(sal), sa.shape[1], _ptr(y),
            wl.out_len, wl.out_len), "tvolap_process_signal_static")

    def plain():
        p.process_signal(x, sa, sb, sal, out_len=wl.out_len, out=y)

    res = {}
    for name, fn in (("static_ms", static), ("process_signal_ms", plain)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        res[name] = round(a.elapsed_time(b) / reps, 4)
    p.check()
    p.close()
    return {"channels": ch, "samples_per_channel": wl.out_len, **res,
            "note": "the static entry point runs the cp.async multiply-accumulate (no scratch "
                    "beyond the fixed array)"}


# --------------------------------------------------------------------------- adjoint
def run_adjoint(args):
    """Differentiable model at 16 channels x 240000 samples, L = 256, M = 47:
    one training step = forward (block spectra, Eq. 7 with per-block parameter
    spectra, inverse + overlap-add) and backward (gradient spectra, adjoint of
    Eq. 7, input gradient). The backward recomputes each block's input spectrum
    inside the adjoint kernel (no spectra kept); the same step with the spectra
    recomputed per segment of 32 blocks by the transform kernel is reported
    beside it. The parameter kernels stream P (2.9 GB) and dP: HBM-bound."""
    import torch
    from paper_2310_00319_gb300 import Plan
    from synth import workloads as W
    dev = torch.device("cuda", 0)
    d = W.differentiable(seed=4, n_ch=args.adj_channels)
    C, N = d["x"].shape
    L, M, nb, P = d["L"], d["M"], d["n_blocks"], 2 * d["L"]
    plan = Plan(L, M, n_in=C, n_out=C, n_slots=1, device=dev)
    x = torch.from_numpy(d["x"]).to(dev)
    Pm = torch.from_numpy(d["P"]).to(dev)
    r = torch.from_numpy(d["r"]).to(dev)
    stream = torch.cuda.current_stream(dev)
    K = 32
    Y = torch.empty((C, nb, P), dtype=torch.complex64, device=dev)
    dP = torch.empty_like(Pm)
    dX = torch.empty((C, nb, P), dtype=torch.complex64, device=dev)
    dx = torch.empty_like(x)
    names = ["fwd_spectra", "mac_params", "inverse_ola", "adjoint_output", "bwd_spectra",
             "adjoint_mac", "adjoint_input"]

    def step(ev, fused=True):
        marks = []

        def mark(name):
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            marks.append((name, e))
        mark("start")
        X = plan.block_spectra(x, 0, nb)                 # forward: all blocks at once
        mark("fwd_spectra")
        plan.mac_params(X, 0, Pm, 0, nb, out=Y)
        mark("mac_params")
        plan.inverse_ola(Y, N)
        mark("inverse_ola")
        G = plan.adjoint_output(r, 0, nb)
        mark("adjoint_output")
        if fused:                                        # X(q) recomputed in the kernel
            mark("bwd_spectra")
            plan.adjoint_mac_x(G, 0, x, Pm, 0, nb, dP, dX=dX, dx_row=0)
            mark("adjoint_mac")
        else:
            for q0 in range(0, nb, K):                   # X recomputed per segment
                qc = min(K, nb - q0)
                Xs = plan.block_spectra(x, q0, qc)
                mark("bwd_spectra")
                plan.adjoint_mac(G, 0, Xs, q0, Pm, q0, qc, dP, dX=dX, dx_row=q0)
                mark("adjoint_mac")
        dx.zero_()
        mark("copy")
        plan.adjoint_input(dX, 0, dx)
        mark("adjoint_input")
        ev.append(marks)

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize(dev)
    evs = []
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(smi_index(dev)).start(prime=lambda: (step([]), torch.cuda.synchronize(dev))) \
            as clk:
        t0e.record(stream)
        for _ in range(args.steps):
            step(evs)
        t1e.record(stream)
        torch.cuda.synchronize(dev)
    plan.check()
    ms = t0e.elapsed_time(t1e) / args.steps
    grad_acc = None if args.no_cpu else adjoint_accuracy(d, dP, dx, dX, plan, x, r)
    # the same step with segments of K blocks recomputed by the transform kernel
    for _ in range(2):
        step([], fused=False)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(args.steps):
        step([], fused=False)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    seg_ms = s0.elapsed_time(s1) / args.steps
    tot = {k: 0.0 for k in names + ["copy"]}
    for marks in evs:
        for (n0, e0), (n1, e1) in zip(marks[:-1], marks[1:]):
            tot[n1] += e0.elapsed_time(e1)
    tot = {k: v / args.steps for k, v in tot.items()}
    pbytes = float(Pm.numel() * 8)
    peaks, kind = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    adj_gbs = 2 * pbytes / (tot["adjoint_mac"] * 1e-3) / 1e9      # read P, write dP
    fwd_gbs = pbytes / (tot["mac_params"] * 1e-3) / 1e9           # read P
    return {"metric": "channel-samples/s (forward + backward)",
            "value": round(C * N / (ms * 1e-3), 1), "unit": "channel-samples/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"differentiable_{C}ch_L256_M47_N240000",
                       "backward": "input spectra recomputed inside the adjoint kernel",
                       "param_bytes": pbytes,
                       "l2": f"parameters ({pbytes / 1e9:.2f} GB) read and written per step, "
                             "larger than the 129 MB L2; no flush"},
            "segmented_k32_ms_per_step": round(seg_ms, 4),
            "roofline": {"bound": "hbm", "achieved": round(adj_gbs, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(adj_gbs / hbm, 4),
                         "traffic": ADJ_TRAFFIC_BYTES if C == 16 else None,
                         "kernel": "k_adjoint_mac_x (read P, write dP; X recomputed)"},
            "mac_params_gbs": round(fwd_gbs, 1),
            "stages_ms": {k: round(v, 4) for k, v in tot.items()},
            "peaks": kind, "clocks": clk.summary(), "gradient_accuracy": grad_acc}


def adjoint_accuracy(d, dP, dx, dX, plan, x, r, seed=5):
    """Sampled gradient entries of the timed step against the oracle: 26
    parameter entries and 8 input samples in each of 3 channels, each computed
    on its own in FP64 from the definitions."""
    import oracle
    dx.zero_()
    plan.adjoint_input(dX, 0, dx)                      # the step's input gradient
    L, M, nb = d["L"], d["M"], d["n_blocks"]
    rng = np.random.default_rng(seed)
    C = d["x"].shape[0]
    errs_p, errs_x = [], []
    for c in sorted({0, C // 2, C - 1}):
        idx = [(int(rng.integers(0, nb)), int(rng.integers(0, M)), int(rng.integers(0, 2 * L)))
               for _ in range(24)] + [(nb - 1, M - 1, 5), (3, M - 1, 0)]
        sidx = [int(v) for v in rng.integers(0, d["x"].shape[1], 6)] + [0, d["x"].shape[1] - 1]
        sP, sx = oracle.params_grad_sampled(d["x"][c], d["P"][c], L, d["r"][c], idx, sidx)
        gP = np.array([dP[c, t, m, k].item() for (t, m, k) in idx])
        gx = dx[c, sidx].cpu().numpy()
        peak = float(dP[c].abs().max())
        errs_p.append(float(np.max(np.abs(gP - sP))) / peak)
        errs_x.append(float(np.linalg.norm(gx - sx) / np.linalg.norm(sx)))
    return {"dP_max_abs_over_peak": max(errs_p), "dx_rel_l2": max(errs_x),
            "entries": "26 dP entries and 8 dx samples in each of 3 channels",
            "tolerance": "1e-3 (gradients)"}


# --------------------------------------------------------------------------- batched
def run_batched(args):
    """512 independent sources with uneven hops (64..512), response lengths
    (4800..96000 taps) and signal lengths (1..20 s): the sources are grouped by
    hop, each group runs as one ragged call (forward transforms, Eq. 7,
    inverse + overlap-add), the MAC staging is autotuned per group, and the
    whole batch is replayed as one CUDA graph. Compared with the plain
    per-source form: one single-channel process_signal call per source in a
    loop, same kernels. Filter banks are resident in both forms."""
    import torch
    from paper_2310_00319_gb300 import Plan, costmodel
    from paper_2310_00319_gb300.batch import BatchedTvolap
    from paper_2310_00319_gb300.tvolap import n_blocks_for
    from synth import workloads as W
    dev = torch.device("cuda", 0)
    S = W.batched_uneven()
    total = sum(s.out_len for s in S)
    B = BatchedTvolap(S, device=dev)
    if args.staging is None:
        tuned = B.autotune(reps=2)
    else:                                  # fixed staging (profiling: the timing would differ)
        B.set_staging(args.staging)
        tuned = {B.group_info(g)[0]: args.staging for g in range(B.n_groups)}
    B.capture()
    for _ in range(args.warmup):
        B.replay()
    torch.cuda.synchronize(dev)
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(smi_index(dev)).start(prime=lambda: (B.replay(), torch.cuda.synchronize(dev))) \
            as clk:
        t0e.record(B.stream)
        for _ in range(args.steps):
            B.replay()
        t1e.record(B.stream)
        torch.cuda.synchronize(dev)
    B.check()
    ms = t0e.elapsed_time(t1e) / args.steps
    launches = 4 * B.n_groups       # per hop group: forward, MAC group + overflow, inverse

    # plain per-source form: one single-channel process_signal per source in a
    # loop, with the staging the autotuner chose for the source's hop (same
    # kernels), and again with the default staging (skipped by --skip-extras)
    stream = torch.cuda.current_stream(dev)
    per = []
    for s in (S if not args.skip_extras else []):
        p = Plan(s.L, s.M, n_slots=s.irs.shape[0], device=dev)
        p.load_bank(0, torch.from_numpy(s.irs).to(dev))
        per.append((p, torch.from_numpy(s.x[None, :]).to(dev),
                    torch.from_numpy(s.sched[None, :]).to(dev),
                    torch.empty((1, s.out_len), dtype=torch.float32, device=dev), s.out_len, s.L))

    def loop():
        for p, x, sc, y, ol, _ in per:
            p.process_signal(x, sc, out_len=ol, out=y)

    def time_loop():
        loop()
        torch.cuda.synchronize(dev)
        reps = max(1, min(3, args.steps))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            loop()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    if args.skip_extras:
        default_ms = per_ms = None
    else:
        default_ms = time_loop()
        tiling = {B.group_info(g)[0]: B.group_tiling(g) for g in range(B.n_groups)}
        for p, *_, L in per:                 # the batch's choices for the source's hop
            p.set_option(1, tiling[L][0])
            p.set_option(3, tiling[L][1])
        per_ms = time_loop()
    for p, *_ in per:
        p.check()
        p.close()

    cpu = None if args.no_cpu else batched_oracle(S, B, budget_s=args.cpu_seconds)
    flops = 0.0
    for s in S:
        nb = n_blocks_for(s.out_len, s.L)
        flops += mac_terms(nb, s.M) * 2 * s.L * costmodel.mac_flops_per_block_bin_partition(False)
    clocks = clk.summary()
    mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = fp32_peak_tflops(mhz)
    ach = flops / (ms * 1e-3) / 1e12
    hops = sorted({s.L for s in S})
    return {"metric": METRIC, "value": round(total / (ms * 1e-3), 1), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batched_uneven_512src", "sources": len(S),
                       "channel_samples": total, "hops": hops,
                       "l2": "inputs larger than L2 (about 1 GB of input, 10 GB of spectra)"},
            "vs_per_source": None if per_ms is None else {
                "per_source_ms_per_step": round(per_ms, 4), "batched_ms_per_step": round(ms, 4),
                "ratio": round(per_ms / ms, 3),
                "per_source_default_staging_ms": round(default_ms, 4),
                "note": "per-source loop with the staging and transform CTA size chosen for "
                        "its hop"},
            "roofline": {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 1),
                         "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": None,
                         "kernel": "whole step: Eq. 7 flops / replay time (lower bound on "
                                   "the multiply-accumulate kernels)"},
            "autotune": {str(B.group_info(g)[0]): {"mac_staging": B.group_tiling(g)[0],
                                                   "xform_threads": B.group_tiling(g)[1]}
                         for g in range(B.n_groups)},
            "gpu_launches": launches * args.steps, "clocks": clocks, "cpu_baseline": cpu}


def batched_oracle(S, B, budget_s=15.0, n_src=32, seed=11):
    """The FP64 oracle on a seeded subset of the batched sources: per source a
    window of consecutive outputs from the middle of its signal, sized so the
    subset takes about budget_s; also the GPU's accuracy on those samples."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = sorted(int(i) for i in rng.choice(len(S), min(n_src, len(S)), replace=False))
    probe = 64
    cost = 0.0
    for i in idx:
        s = S[i]
        t = time.perf_counter()
        oracle.tvolap_samples(s.x, s.irs, s.L, s.sched[None, :], None, None,
                              np.zeros(probe, np.int32),
                              np.arange(s.out_len // 2, s.out_len // 2 + probe, dtype=np.int64))
        cost += (time.perf_counter() - t) / probe
    n = int(max(probe, budget_s / max(cost, 1e-9)))
    got, ref, total, dt = [], [], 0, 0.0
    for i in idx:
        s = S[i]
        a = s.out_len // 2
        k = min(n, s.out_len - a)
        ni = np.arange(a, a + k, dtype=np.int64)
        t = time.perf_counter()
        r = oracle.tvolap_samples(s.x, s.irs, s.L, s.sched[None, :], None, None,
                                  np.zeros(k, np.int32), ni)
        dt += time.perf_counter() - t
        total += k
        ref.append(r)
        got.append(B.output(i)[a:a + k].cpu().numpy())
    return {"value": round(total / dt, 1), "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": round(dt, 2),
            "sample": f"{len(idx)} sources (seed {seed}), up to {n} consecutive outputs each "
                      "from the middle of the signal",
            "accuracy": accuracy(np.concatenate(got), np.concatenate(ref))}


# --------------------------------------------------------------------------- serving
def run_serve(args):
    """Streaming server: 1000 streams present at the start, Poisson arrivals
    at 50/s with lifetimes of 2..30 s, hop 64/128/256, binaural banks of 36
    pairs of 12000..144000 taps, a head-orientation walk choosing the pair of
    every block. Base tick 64 samples (1.333 ms at 48 kHz). Three measurements
    over consecutive ticks: latency (one tick at a time: host-to-host time from
    the tick call to its outputs in host memory, and device time), throughput
    (ticks pipelined two deep, device time), and the multiply-accumulate
    kernel alone (direct launches between CUDA events)."""
    import torch
    from paper_2310_00319_gb300.server import OPT_TIMING, Server
    from synth import workloads as W
    dev = torch.device("cuda", 0)
    lat_ticks = args.serve_ticks
    thr_ticks = max(10, args.serve_ticks * 3 // 4)
    timed_ticks = max(10, args.serve_ticks // 13)
    warm = max(args.warmup, 20)
    n_streams = args.streams
    fs, base, top, n_pairs = 48000, 64, 256, 36
    cap = n_streams if n_streams < 1000 else 1000
    rng = np.random.default_rng(5)
    # response banks: K distinct banks (lengths uniform 12000..144000), each
    # stream takes one at random and transforms it into its own arena piece
    K = 16
    lens = rng.integers(12000, 144001, K)
    banks_np = [W.serving_bank(rng, int(n), n_pairs) for n in lens]
    banks = [torch.from_numpy(b).to(dev) for b in banks_np]
    hops = np.array([64, 128, 256])
    total_ticks = warm + lat_ticks + thr_ticks + timed_ticks
    ev = W.serving_arrivals(seed=5, duration_s=total_ticks * base / fs, prefill=n_streams,
                            base_hop=base, fs=fs)
    n_ev = ev.shape[0]
    L_of = hops[rng.integers(0, 3, n_ev)]
    bank_of = rng.integers(0, K, n_ev)
    stream = torch.cuda.Stream(dev)
    free_b = torch.cuda.mem_get_info(dev)[0]
    # a stream takes at most (36 pairs x 2 + 2) x 144000 taps x 8 B (about 85 MB)
    arena = int(min(0.6 * free_b, 140e9, cap * 90e6))
    srv = Server(base, top, cap, max_out=2, arena_bytes=arena, device=dev, stream=stream)
    live = {}                 # stream id -> event index
    leave_at = {}
    track, done_tracks = {}, []
    ticket_ev = {}            # waiting request -> event index
    waits = []                # base ticks each admitted request waited
    nxt = 0

    def arrivals(tick):
        """Requests of this tick join the admission queue (none is dropped);
        those the queue admitted (now or at the last due) start their lifetime;
        streams whose lifetime is over retire and free their slot and memory."""
        nonlocal nxt
        while nxt < n_ev and ev[nxt, 0] <= tick:
            ticket_ev[srv.submit(int(L_of[nxt]), banks[bank_of[nxt]])] = nxt
            nxt += 1
        admitted(tick)
        for i in [i for i, t in leave_at.items() if t <= tick]:
            srv.retire(i)
            del live[i], leave_at[i]
            if i in track:                       # the id may be reused: close the record
                done_tracks.append(track.pop(i))

    def admitted(tick):
        for t, i, w in srv.admitted():
            e = ticket_ev.pop(t)
            live[i] = e
            leave_at[i] = tick + int(ev[e, 1] - ev[e, 0])     # lifetime from admission
            srv.sel[i] = int(rng.integers(0, n_pairs))
            waits.append(w)

    pool = (0.1 * rng.standard_normal((4096, top))).astype(np.float32)
    steps = np.array([-1, 0, 1], np.int32)

    def stage(ids, tick):
        srv.inp[ids] = pool[(ids * 7 + tick) % 4096]
        srv.sel[ids] = (srv.sel[ids] + steps[rng.integers(0, 3, ids.shape[0])]) % n_pairs

    # record the first blocks of 16 streams present from the start, for the oracle
    REC = 120
    tick = 0
    arrivals(0)
    track.update({i: {"ev": e, "x": [], "sel": [], "y": []} for i, e in list(live.items())[:16]})
    srv.wait()

    def record_in(ids):
        for i in ids:
            tr = track.get(int(i))
            if tr is not None and len(tr["x"]) < REC:
                L = int(L_of[tr["ev"]])
                tr["x"].append(srv.inp[i, :L].copy())
                tr["sel"].append(int(srv.sel[i]))

    def record_out(ids):
        for i in ids:
            tr = track.get(int(i))
            if tr is not None and len(tr["y"]) < len(tr["x"]):
                L = int(L_of[tr["ev"]])
                tr["y"].append(srv.out[i, :, :L].copy())

    for _ in range(warm):
        arrivals(tick)
        ids = srv.due()
        admitted(tick)
        stage(ids, tick)
        record_in(ids)
        srv.tick()
        srv.wait()
        record_out(ids)
        tick += 1
    srv.wait()
    # latency: one tick at a time
    h2h, gpu, live_n, queued_n = [], [], [], []
    e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
         for _ in range(lat_ticks)]
    s0 = srv.stats()
    waits_before = len(waits)
    with ClockSampler(smi_index(dev)) as clk:
        for k in range(lat_ticks):
            arrivals(tick)
            ids = srv.due()
            admitted(tick)
            live_n.append(len(live))
            queued_n.append(len(ticket_ev))
            stage(ids, tick)
            record_in(ids)
            t0 = time.perf_counter()
            e[k][0].record(stream)
            srv.tick()
            e[k][1].record(stream)
            srv.wait()
            h2h.append(time.perf_counter() - t0)
            record_out(ids)
            tick += 1
        torch.cuda.synchronize(dev)
        gpu = [a.elapsed_time(b) for a, b in e]
        s1 = srv.stats()
        # throughput: pipelined, device time over the whole run
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_host = time.perf_counter()
        a.record(stream)
        for k in range(thr_ticks):
            arrivals(tick)
            ids = srv.due()
            admitted(tick)
            stage(ids, tick)
            srv.tick()
            tick += 1
        b.record(stream)
        srv.wait()
        t_host = time.perf_counter() - t_host
        s2 = srv.stats()
    thr_ms = a.elapsed_time(b)
    # the multiply-accumulate kernel alone: direct launches with stage events
    srv.set_option(OPT_TIMING, 1)
    s3 = srv.stats()
    for k in range(timed_ticks):
        arrivals(tick)
        ids = srv.due()
        admitted(tick)
        stage(ids, tick)
        srv.tick()
        tick += 1
    srv.wait()
    s4 = srv.stats()
    srv.set_option(OPT_TIMING, 0)
    st = s4
    q = srv.queue()
    srv.close()
    cpu = None
    if not args.no_cpu:
        cpu = serve_oracle(list(track.values()) + done_tracks, banks_np, bank_of, L_of)
    stage_ms = [s4["stage_ms"][i] - s3["stage_ms"][i] for i in range(3)]
    mac_bytes = s4["mac_bytes"] - s3["mac_bytes"]
    mac_gbs = mac_bytes / (stage_ms[1] * 1e-3) / 1e9
    peaks, kind = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    samples = s2["channel_samples"] - s1["channel_samples"]
    deadline = base / fs * 1e3
    h2h_ms = np.array(h2h) * 1e3
    gpu = np.array(gpu)
    return {"metric": f"channel-samples/s (streaming, {n_streams} binaural streams)",
            "value": round(samples / (thr_ms * 1e-3), 1), "unit": "channel-samples/s",
            "n_gpus": 1, "steps": thr_ticks, "warmup": warm,
            "ms_per_step": round(thr_ms / thr_ticks, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving_{n_streams}_streams", "base_tick_samples": base,
                       "hops": [64, 128, 256], "pairs_per_stream": n_pairs,
                       "ir_len": "uniform 12000..144000 (16 banks)", "capacity": cap,
                       "arena_gb": round(arena / 1e9, 1),
                       "l2": "banks and delay lines (tens of GB) far larger than L2"},
            "latency": {"ticks": lat_ticks, "deadline_ms": round(deadline, 4),
                        "host_to_host_ms_p50": round(float(np.percentile(h2h_ms, 50)), 4),
                        "host_to_host_ms_p99": round(float(np.percentile(h2h_ms, 99)), 4),
                        "gpu_ms_p50": round(float(np.percentile(gpu, 50)), 4),
                        "gpu_ms_p99": round(float(np.percentile(gpu, 99)), 4),
                        "missed_deadline": int((h2h_ms > deadline).sum())},
            "streams": {"live_end": st["live"], "dropped": 0,
                        "submitted": nxt, "admitted": len(waits), "waiting_end": q["waiting"],
                        "live_during_latency": {"min": int(min(live_n)), "max": int(max(live_n)),
                                                "mean": round(float(np.mean(live_n)), 1)},
                        "waiting_during_latency_max": int(max(queued_n)),
                        "queue_wait_ticks": {
                            "p50": float(np.percentile(waits, 50)),
                            "p99": float(np.percentile(waits, 99)),
                            "max": int(max(waits)),
                            "admitted_after_waiting": int(sum(1 for w in waits if w > 0))},
                        "mean_due_per_tick": round((s2["stream_blocks"] - s1["stream_blocks"]) /
                                                   thr_ticks, 1)},
            "throughput_host_s": round(t_host, 3),
            "roofline": {"bound": "hbm", "achieved": round(mac_gbs, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(mac_gbs / hbm, 4), "traffic": None,
                         "kernel": "k_srv_mac (delay line + 2 bank spectra read, Y written)"},
            "stages_ms_per_tick": {"forward": round(stage_ms[0] / timed_ticks, 4),
                                   "mac": round(stage_ms[1] / timed_ticks, 4),
                                   "inverse": round(stage_ms[2] / timed_ticks, 4)},
            "gpu_launches": 3 * thr_ticks,           # forward, MAC, inverse per tick
            "peaks": kind, "clocks": clk.summary(), "cpu_baseline": cpu}


def serve_oracle(tracks, banks_np, bank_of, L_of):
    """The FP64 oracle on the recorded first blocks of up to 16 streams: each
    stream's output (delayed by L) recomputed from its inputs and pair indices;
    also the server's accuracy on them."""
    import oracle
    got, ref, dt, n = [], [], 0.0, 0
    for tr in tracks:
        nb = len(tr["y"])
        if nb < 8:
            continue
        L = int(L_of[tr["ev"]])
        bank = banks_np[bank_of[tr["ev"]]]                   # [pairs, 2, ir_len]
        F, _, ir_len = bank.shape
        x = np.concatenate(tr["x"][:nb])
        sel = np.array(tr["sel"][:nb], np.int32)
        sched = np.stack([sel * 2, sel * 2 + 1]).astype(np.int32)
        t = time.perf_counter()
        r = oracle.tvolap_direct(x[None, :], bank.reshape(F * 2, ir_len), L, sched,
                                 out_len=(nb - 1) * L, out_to_in=[0, 0])
        dt += time.perf_counter() - t
        y = np.concatenate(tr["y"][:nb], axis=1)[:, L:]      # delayed by L
        got.append(y.ravel())
        ref.append(r.ravel())
        n += r.size
    if not ref:
        return None
    return {"value": round(n / dt, 1), "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": round(dt, 2),
            "sample": f"first blocks of {len(ref)} streams present from the start "
                      "(both outputs, up to 120 blocks each)",
            "accuracy": accuracy(np.concatenate(got), np.concatenate(ref))}


# --------------------------------------------------------------------------- sub-records
SUBRECORD_RUNS = (
    # name, runner, bounded settings
    ("batched", "run_batched", {"steps": 5, "warmup": 3}),
    ("adjoint", "run_adjoint", {"steps": 5, "warmup": 3}),
    ("serve", "run_serve", {"serve_ticks": 2000, "warmup": 3}),
)


def compact_record(name: str, r: dict, wall_s: float) -> dict:
    """The figures of a workload's full line that the default line carries:
    value, per-step time, roofline (kernel, traffic), clocks, the accuracy
    against the oracle on its seeded subset, and the workload's own
    comparison (per-source loop, latency and queue, segmented backward)."""
    keep = ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "roofline", "clocks",
            "gpu_launches", "vs_per_source", "autotune", "latency", "streams",
            "segmented_k32_ms_per_step", "mac_params_gbs", "stages_ms_per_tick")
    out = {k: r[k] for k in keep if k in r}
    out["workload"] = r["config"]["workload"]
    cpu = r.get("cpu_baseline")
    if cpu:
        out["accuracy"] = cpu.get("accuracy")
        out["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "sample")}
    if r.get("gradient_accuracy"):
        out["accuracy"] = r["gradient_accuracy"]
    out["wall_s"] = round(wall_s, 1)
    return out


def workload_subrecords(args) -> dict:
    """The batched, differentiable and serving workloads, each run with
    bounded settings after the default workload's timed region, as compact
    records of the default line (one GPU)."""
    import copy

    import torch
    out = {}
    for name, fn, over in SUBRECORD_RUNS:
        a = copy.copy(args)
        a.__dict__.update(over)
        a.staging = None
        torch.cuda.empty_cache()
        t = time.perf_counter()
        out[name] = compact_record(name, globals()[fn](a), time.perf_counter() - t)
    return out


# --------------------------------------------------------------------------- oracle
_F64 = {}


def _oracle_sample(wl, n_samples, channel=0, start=None, values=False):
    """Time the oracle on n_samples consecutive outputs of one channel (inputs
    are converted to FP64 once, outside the timing); with values, also return
    the outputs."""
    import oracle
    if id(wl) not in _F64:
        _F64.clear()
        _F64[id(wl)] = (np.ascontiguousarray(wl.x, np.float64),
                        np.ascontiguousarray(wl.irs, np.float64),
                        np.ascontiguousarray(wl.sched_alpha, np.float64))
    x64, irs64, al64 = _F64[id(wl)]
    start = wl.out_len // 2 if start is None else start
    n_idx = np.arange(start, start + n_samples, dtype=np.int64)
    oc = np.full(n_samples, channel, dtype=np.int32)
    t = time.perf_counter()
    y = oracle.tvolap_samples(x64, irs64, wl.L, wl.sched_a, wl.sched_b, al64, oc, n_idx,
                              out_to_in=wl.out_to_in)
    dt = time.perf_counter() - t
    return (dt, y) if values else dt


def run_mixdown(args):
    """Binaural mixdown: S = channels / 2 sources, each rendered to two ears
    through its own time-variant responses (plan output 2s + e reads source s),
    the ears' spectra summed before one inverse transform per ear. A step is
    the bank transform, the forward transforms of the S sources, the MAC of
    the 2S paths, the mixdown and the two inverse transforms with the
    overlap-add; beside it the same step with 2S inverse transforms and no
    mixdown."""
    import torch
    import oracle
    from paper_2310_00319_gb300 import Plan, costmodel, _lib as L_
    from paper_2310_00319_gb300.tvolap import n_blocks_for, _ptr
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    base = workload(args)                                   # 2S paths of the default recipe
    S = base.n_out // 2
    L, M, P, N = base.L, base.M, 2 * base.L, base.N
    nb = n_blocks_for(base.out_len, L)
    o2i = [o // 2 for o in range(2 * S)]
    mix = [o % 2 for o in range(2 * S)]
    stream = torch.cuda.current_stream(dev)
    plan = Plan(L, M, n_in=S, n_out=2 * S, out_to_in=o2i, n_slots=base.irs.shape[0], device=dev)
    plan.set_mix(mix)
    ears = Plan(L, M, n_in=2, n_out=2, n_slots=1, device=dev)   # inverse of the two mixed rows
    x = torch.from_numpy(np.ascontiguousarray(base.x[:S])).to(dev)
    irs = torch.from_numpy(base.irs).to(dev)
    sa, sb, sal = (torch.from_numpy(a).to(dev) for a in (base.sched_a, base.sched_b,
                                                           base.sched_alpha))
    X = torch.empty((S, nb, P), dtype=torch.complex64, device=dev)
    Y = torch.empty((2 * S, nb, P), dtype=torch.complex64, device=dev)
    Ym = torch.empty((2, nb, P), dtype=torch.complex64, device=dev)
    y2 = torch.empty((2, base.out_len), dtype=torch.float32, device=dev)
    yall = torch.empty((2 * S, base.out_len), dtype=torch.float32, device=dev)
    lib, h = plan.lib, plan.h

    def step(mixdown, ev=None):
        rec = (lambda i: ev[i].record(stream)) if ev else (lambda i: None)
        rec(0)
        L_.check(lib.tvolap_load_bank(h, 0, irs.shape[0], _ptr(irs), irs.shape[1], irs.shape[1]),
                 "load_bank")
        L_.check(lib.tvolap_forward_spectra(h, _ptr(x), N, N, nb, _ptr(X)), "forward")
        rec(1)
        L_.check(lib.tvolap_mac(h, _ptr(X), nb, _ptr(sa), _ptr(sb), _ptr(sal), sa.shape[1],
                                _ptr(Y)), "mac")
        rec(2)
        if mixdown:
            L_.check(lib.tvolap_mix(h, _ptr(Y), nb, _ptr(Ym)), "mix")
            rec(3)
            L_.check(lib.tvolap_inverse_ola(ears.h, _ptr(Ym), nb, _ptr(y2), base.out_len,
                                            base.out_len), "inverse")
        else:
            rec(3)
            L_.check(lib.tvolap_inverse_ola(h, _ptr(Y), nb, _ptr(yall), base.out_len,
                                            base.out_len), "inverse")
        rec(4)

    def timed(mixdown):
        for _ in range(args.warmup):
            step(mixdown)
        plan.check()
        torch.cuda.synchronize(dev)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        prime = lambda: (step(mixdown), torch.cuda.synchronize(dev))  # noqa: E731
        with ClockSampler(smi_index(dev)).start(prime=prime) as clk:
            t0.record(stream)
            for i in range(args.steps):
                step(mixdown, evs[i])
            t1.record(stream)
            torch.cuda.synchronize(dev)
        plan.check()
        st = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(4)] for e in evs]).mean(0)
        return t0.elapsed_time(t1) / args.steps, st, clk.summary()

    ms_mix, st_mix, clocks = timed(True)
    ms_plain, st_plain, _ = timed(False)
    # the user call for the whole signal (forward, MAC, mixdown, two inverses)
    for _ in range(2):
        plan.process_signal_mix(x, sa, sb, sal, out_len=base.out_len)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        ym = plan.process_signal_mix(x, sa, sb, sal, out_len=base.out_len)
    b.record(stream)
    torch.cuda.synchronize(dev)
    plan.check()
    ms_call = a.elapsed_time(b) / args.steps
    units = 2 * S * base.out_len                            # path-samples per step
    flops = mac_terms(nb, M) * P * 2 * S * costmodel.mac_flops_per_block_bin_partition(True)
    peak = fp32_peak_tflops(_peaks()[0].get("sm_max_mhz", 2070.0))
    achieved = flops / (st_mix[1] * 1e-3) / 1e12
    hbm = _peaks()[0].get("hbm_gbs", 6800.0)
    mix_bytes = 8.0 * P * nb * (2 * S + 2)
    out = {
        "metric": METRIC, "value": round(units / (ms_mix * 1e-3), 1), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_mix, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"binaural_mixdown_{S}src_L{L}_N{N}_ir{base.ir_len}",
                   "sources": S, "ears": 2, "paths": 2 * S, "L": L, "M": M,
                   "samples_per_path": base.out_len, "per_gpu_units": units,
                   "unit_note": "path-samples (sources x ears x output samples)",
                   "l2": "working set ~1.3 GB >> 129 MB L2; no flush"},
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2),
                     "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "k_mac_signal_persist"},
        "stages": {"bank_and_forward": {"ms": round(float(st_mix[0]), 4)},
                   "mac": {"ms": round(float(st_mix[1]), 4), "tflops": round(achieved, 3)},
                   "mix": {"ms": round(float(st_mix[2]), 4),
                           "gbs": round(mix_bytes / (st_mix[2] * 1e-3) / 1e9, 1),
                           "of_hbm": round(mix_bytes / (st_mix[2] * 1e-3) / 1e9 / hbm, 3)},
                   "inverse_2_ears": {"ms": round(float(st_mix[3]), 4)}},
        "without_mixdown": {"ms_per_step": round(ms_plain, 4),
                            "inverse_all_paths_ms": round(float(st_plain[3]), 4),
                            "speedup": round(ms_plain / ms_mix, 3),
                            "note": f"{2 * S} inverse transforms and {2 * S} output rows; the "
                                    "ears would still need a sum"},
        "process_signal_mix_ms": round(ms_call, 4),
        "clocks": clocks, "gpu_launches": 6 * args.steps,
    }
    if not args.no_cpu:
        # ear e at 128 samples in the steady state: the sum of its paths' oracle outputs
        n_idx = np.arange(base.out_len // 2, base.out_len // 2 + 128, dtype=np.int64)
        x64 = np.ascontiguousarray(base.x[:S], np.float64)
        irs64 = np.ascontiguousarray(base.irs, np.float64)
        al64 = np.ascontiguousarray(base.sched_alpha, np.float64)
        oc = np.repeat(np.arange(2 * S, dtype=np.int32), n_idx.size)
        t = time.perf_counter()
        per_path = oracle.tvolap_samples(x64, irs64, L, base.sched_a, base.sched_b, al64, oc,
                                         np.tile(n_idx, 2 * S), out_to_in=o2i)
        dt = time.perf_counter() - t
        ref = oracle.mixdown(per_path.reshape(2 * S, n_idx.size), mix)
        got = ym[:, n_idx.min():n_idx.max() + 1].cpu().numpy()
        out["accuracy"] = accuracy(got, ref)
        out["cpu_baseline"] = {"value": round(oc.size / dt, 1), "unit": UNIT,
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": f"{n_idx.size} samples of both ears: {oc.size} path "
                                         "samples of the FP64 time-domain oracle, summed"}
    plan.close()
    ears.close()
    return out


def run_nonuniform(args):
    """Two-level non-uniform partitions for long responses at a short hop:
    16 channels, responses of 96000 taps (2 s at 48 kHz), head hop 64 (latency
    128 samples) with 15 partitions, tail hop 1024 with 46 partitions, against
    one uniform plan at hop 64 (750 partitions, the same latency). Offline:
    one process_signal of 480000 samples per channel; streaming: mean time of
    a hop-64 tick (every 16th also runs the tail's hop)."""
    import torch
    import oracle
    from synth import workloads as W
    from paper_2310_00319_gb300 import Plan
    from paper_2310_00319_gb300.nonuniform import NonUniform
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    La, Ma, ratio, Mb, n_ch, ir_len = 64, 15, 16, 46, 16, 96000
    # the default workload's filter walk (step 0.05 per 256 samples) at the same speed in
    # time: four times the steps, half the step size
    wl = W.plain_at_scale(n_ch=n_ch, N=args.samples, L=La, ir_len=ir_len, step_sigma=0.025)
    nb = wl.sched_a.shape[1]
    stream = torch.cuda.current_stream(dev)
    nu = NonUniform(La, Ma, ratio, Mb, n_in=n_ch, n_slots=wl.irs.shape[0], device=dev)
    uni = Plan(La, wl.M, n_in=n_ch, n_slots=wl.irs.shape[0], device=dev)
    irs = torch.from_numpy(wl.irs).to(dev)
    nu.load_bank(0, irs)
    uni.load_bank(0, irs)
    x = torch.from_numpy(wl.x).to(dev)
    sa, sb, sal = (torch.from_numpy(a).to(dev) for a in (wl.sched_a, wl.sched_b, wl.sched_alpha))

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / steps

    # the tail's filters move 16 head steps per block: keep its faster MAC staging
    tail_ms = {}
    for stg in (0, 2):
        nu.set_option(1, stg, level=1)
        tail_ms[stg] = timed(lambda: nu.process_signal(x, sa, sb, sal, out_len=wl.out_len), 3)
    tail_staging = min(tail_ms, key=tail_ms.get)
    nu.set_option(1, tail_staging, level=1)
    run_nu = lambda: nu.process_signal(x, sa, sb, sal, out_len=wl.out_len)  # noqa: E731
    with ClockSampler(smi_index(dev)).start(prime=lambda: (run_nu(), torch.cuda.synchronize(dev))) \
            as clk:
        ms_nu = timed(run_nu, args.steps)
    clocks = clk.summary()
    ms_uni = timed(lambda: uni.process_signal(x, sa, sb, sal, out_len=wl.out_len), max(3, args.steps // 4))
    nu.check()
    uni.check()
    # streaming ticks (hop 64): 1600 ticks = 100 tail hops
    n_ticks = 1600
    xs = x[:, :n_ticks * La].contiguous()
    blocks = [xs[:, t * La:(t + 1) * La].contiguous() for t in range(n_ticks)]
    out = torch.empty((n_ch, La), dtype=torch.float32, device=dev)
    sat = sa.t().contiguous()

    def ticks(obj):
        obj.reset()
        for t in range(n_ticks):
            obj.process_block(blocks[t], out, sat[t])

    tick_nu = timed(lambda: ticks(nu), 2) / n_ticks
    tick_uni = timed(lambda: ticks(uni), 2) / n_ticks
    units = n_ch * wl.out_len
    res = {
        "metric": METRIC, "value": round(units / (ms_nu * 1e-3), 1), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_nu, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"nonuniform_{n_ch}ch_La{La}x{ratio}_ir{ir_len}_N{wl.N}",
                   "channels": n_ch, "head": {"hop": La, "partitions": Ma, "taps": 2 * La * Ma},
                   "tail": {"hop": La * ratio, "partitions": Mb, "mac_staging": tail_staging},
                   "ir_len": ir_len, "filter": "walk step 0.025 per 64 samples, new mix every block",
                   "latency_samples": 2 * La, "per_gpu_units": units,
                   "l2": "working set > 129 MB L2; no flush"},
        "uniform_hop64": {"partitions": wl.M, "ms_per_step": round(ms_uni, 4),
                          "speedup": round(ms_uni / ms_nu, 2)},
        "stream_tick_ms": {"nonuniform": round(tick_nu, 4), "uniform_hop64": round(tick_uni, 4),
                           "deadline_ms": round(La / 48.0, 4)},
        "clocks": clocks,
        # per process_signal: two plans' forward, MAC (+ overflow), inverse, the
        # tail schedule and the shifted add
        "gpu_launches": 10 * args.steps,
    }
    if not args.no_cpu:
        # the oracle's two-level definition on the first 6000 samples of channel 0
        n = 6000
        nb_n = oracle.n_out_blocks(n, La)
        t = time.perf_counter()
        ref = oracle.tvolap_nonuniform(wl.x[0, :n], wl.irs, La, Ma, ratio, Mb,
                                       wl.sched_a[:1, :nb_n], wl.sched_b[:1, :nb_n],
                                       wl.sched_alpha[:1, :nb_n], out_len=n)
        dt = time.perf_counter() - t
        y = nu.process_signal(x[:, :n].contiguous(), sa[:, :nb_n].contiguous(),
                              sb[:, :nb_n].contiguous(), sal[:, :nb_n].contiguous(),
                              out_len=n)[:1].cpu().numpy()
        res["accuracy"] = accuracy(y, ref)
        res["cpu_baseline"] = {"value": round(n / dt, 1), "unit": UNIT, "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": f"{n} samples of channel 0 (both levels)"}
    nu.close()
    uni.close()
    return res


def accuracy_plain_mono(dev):
    """The mono configuration (L = 128, 96000 samples, 4 responses of 4096 taps
    switched every 16 blocks) through process_signal, against the FP64 oracle
    over the whole signal."""
    import torch
    import oracle
    from paper_2310_00319_gb300 import Plan
    from synth import workloads as W
    wl = W.plain_mono()
    p = Plan(wl.L, wl.M, n_slots=wl.irs.shape[0], device=dev)
    p.load_bank(0, torch.from_numpy(wl.irs).to(dev))
    y = p.process_signal(torch.from_numpy(wl.x).to(dev), torch.from_numpy(wl.sched_a).to(dev),
                         out_len=wl.out_len).cpu().numpy()
    p.check()
    p.close()
    ref = oracle.tvolap_direct(wl.x, wl.irs, wl.L, wl.sched_a, out_len=wl.out_len)
    out = accuracy(y, ref)
    out["workload"] = "plain_mono_L128_N96000_ir4096 (whole signal)"
    return out


def accuracy(y, ref):
    """FP32 result against the FP64 oracle on the same samples."""
    y = np.asarray(y, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    peak = float(np.max(np.abs(ref))) or 1.0
    return {"rel_l2": float(np.linalg.norm(y - ref) / (np.linalg.norm(ref) or 1.0)),
            "max_abs_over_peak": float(np.max(np.abs(y - ref)) / peak), "samples": int(y.size),
            "tolerance": "rel-L2 <= 1e-5 and max-abs <= 1e-4 x peak"}


def cpu_baseline(args, wl, budget_s=15.0, y_channel0=None):
    """The FP64 oracle on the host cores: a contiguous run of output samples of
    one channel in the steady state, sized to about budget_s seconds. With the
    GPU's output of that channel, also its accuracy on those samples."""
    import oracle
    probe = 256
    dt = _oracle_sample(wl, probe)
    n = int(max(probe, min(wl.out_len // 2, probe * budget_s / max(dt, 1e-6))))
    start = wl.out_len // 2
    dt, ref = _oracle_sample(wl, n, start=start, values=True)
    out = {"value": round(n / dt, 1), "unit": UNIT, "cores": oracle.num_threads(),
           "kind": "oracle", "seconds": round(dt, 2),
           "sample": f"{n} consecutive output samples of channel 0 from n={start} "
                     f"(FP64 time-domain oracle, {2 * wl.ir_len} flop-pairs per sample)"}
    if y_channel0 is not None:
        out["accuracy"] = accuracy(y_channel0[start:start + n], ref)
    return out


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return None
    import oracle
    wl = workload(args)
    probe = 128
    dt = _oracle_sample(wl, probe)
    # every step a bounded sample: the whole run stays within about 150 s
    step_s = min(args.ref_step_seconds, 150.0 / max(1, args.steps + args.warmup))
    per_step = int(max(probe, probe * step_s / max(dt, 1e-6)))
    for _ in range(args.warmup):
        _oracle_sample(wl, per_step)
    total = 0.0
    for _ in range(args.steps):
        total += _oracle_sample(wl, per_step)
    value = per_step * args.steps / total
    return {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl.name + f"_N{wl.N}_ir{wl.ir_len}", "channels": wl.n_out,
                       "L": wl.L, "M": wl.M, "per_step_units": per_step},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{per_step} consecutive output samples of channel 0 "
                                       "per step (FP64 time-domain oracle)"},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain_at_scale",
                    choices=["plain_at_scale", "adjoint", "batched", "serve", "mixdown",
                             "nonuniform", "stream"])
    ap.add_argument("--channels", type=int, default=64)
    ap.add_argument("--samples", type=int, default=480000)
    ap.add_argument("--ir-len", type=int, default=48000,
                    help="taps of the stored responses of the default workload")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the multiply-accumulate kernel")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=4.0)
    ap.add_argument("--streams", type=int, default=1000,
                    help="serve: streams present at the start (slots capped at 1000)")
    ap.add_argument("--serve-ticks", type=int, default=10000,
                    help="serve: ticks of the latency run (throughput run: 3/4 of it)")
    ap.add_argument("--adj-channels", type=int, default=16,
                    help="adjoint: channels of the differentiable workload")
    ap.add_argument("--staging", type=int, default=None, choices=[0, 1, 2, 3, 4, 5],
                    help="multiply-accumulate staging (default workload: instead of the default; "
                         "batched: instead of the autotuner)")
    ap.add_argument("--skip-extras", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="default workload: leave out the batched, adjoint and serve records")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl != "reference" and args.workload != "plain_at_scale" and _dist()[0] > 1:
        # the other workloads are single-GPU measurements on cuda:0
        sys.exit(f"bench.py: --workload {args.workload} runs on one GPU; launch it without torchrun")
    if args.impl == "reference":
        out = run_reference(args)
    elif args.workload == "adjoint":
        out = run_adjoint(args)
    elif args.workload == "batched":
        out = run_batched(args)
    elif args.workload == "serve":
        out = run_serve(args)
    elif args.workload == "mixdown":
        out = run_mixdown(args)
    elif args.workload == "nonuniform":
        out = run_nonuniform(args)
    elif args.workload == "stream":
        out = run_stream_only(args)
    else:
        out = run_ours(args)
        if (out is not None and _dist()[0] == 1 and not args.skip_extras
                and not args.no_workloads):
            out["workloads"] = workload_subrecords(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
