"""Benchmark of the dedispersion hot path on GB300.

One step = one pass of the hot path over one block of synthetic filterbank data:
per-channel noise statistics, profiled dedispersion of every trial (eq. p_dedisp),
the boxcar normaliser and the boxcar S/N scan over all widths (eq. snr).  The default
workload is the CRAFT-like configuration (336 x 1 MHz channels over 1130-1466 MHz,
dt = 1 ms, 65536 fp32 samples, 4096 trial DMs of eq. trial DMs over 0-4000 pc cm^-3,
weights proportional to nu^-1.4 on every tap, boxcar widths 1-32).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

prints one JSON line.  `value` is dedispersed DM-trial*samples per second for the
whole job (N ranks each process their own block: weak scaling, no collective on the
data path).  `--impl reference` times the CPU oracle (tests' reference) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "dedispersed DM-trial·samples/s on 1 GB300 and % roofline; fwd+bwd vs plain fwd"
UNIT = "DM-trial·samples/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
FP32_LANES_PER_SM = 128
SMEM_BYTES_PER_CLK_PER_SM = 128
LAUNCHES_PER_STEP = 4    # channel stats, dedispersion, normaliser, boxcar scan


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return dict(FALLBACK_PEAKS), "fallback"


# ----------------------------------------------------------------------------- workload


def dm_shards(cost, ws, align=16):
    """Contiguous trial ranges, one per rank, of about equal cost (cost[d]: taps of trial
    d), with boundaries on multiples of `align` trials (one CTA's trial block) where the
    list allows.  Returns [(lo, hi)] * ws covering 0 .. len(cost)."""
    cost = np.asarray(cost, np.float64)
    D = len(cost)
    cum = np.concatenate([[0.0], np.cumsum(cost)])
    bounds = [0]
    for r in range(1, ws):
        d = int(np.searchsorted(cum, cum[-1] * r / ws))
        d = int(round(d / align)) * align if D >= ws * align else d
        bounds.append(min(max(d, bounds[-1]), D))
    bounds.append(D)
    return [(bounds[r], bounds[r + 1]) for r in range(ws)]


def craft_workload(dd, dev, ndm=None, rank=0, ws=1):
    """The CRAFT-like block; with ws > 1 ranks, this rank's contiguous range of its trial
    list (cost-balanced), every rank computing the same output span as one GPU would
    (the full list's t_out) from a full replica of the input."""
    import torch
    import synth
    cfg = synth.make_craft()
    b = cfg["band"]
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, cfg["nsamp"], "f32")
    dms, eps = dd.trial_dms(band, 0.0, cfg["dm_max"], cfg["ndm"], tau_av_ms=1.0)
    if ndm:   # a smaller profiling case: a contiguous block from the middle of the list
        m = max(0, len(dms) // 2 - ndm // 2)
        dms = dms[m:m + ndm]
    full = dd.Plan(band, dms)
    delay_f, taps_f = full.tables()
    t_out = cfg["nsamp"] - full.d_max
    full.close()
    shards = dm_shards(taps_f.astype(np.int64).sum(axis=1), ws)
    lo, hi = shards[rank]
    plan = dd.Plan(band, dms[lo:hi])
    delay, taps = plan.tables()
    K = int(taps_f.max())
    w = np.where(np.arange(K)[None, None, :] < taps[:, :, None], cfg["wchan"][None, :, None], 0.0)
    w = np.ascontiguousarray(w, dtype=np.float32)
    plan.set_profiles(weights=w)
    x = torch.from_numpy(cfg["data"]).to(dev)
    info = plan.info()
    return dict(
        name="CRAFT-like",
        desc=("CRAFT-like: 336 ch x 1 MHz (1130-1466 MHz), dt 1 ms, 65536 fp32 samples, "
              f"{len(dms)} trial DMs 0-{dms[-1]:.0f} (eq. trial DMs, eps={eps:.4f}), "
              "weights ~ nu^-1.4 on every tap, boxcar widths 1-32"),
        plan=plan, x=x, host=cfg["data"], nsamp=t_out + info["d_max"], t_out=t_out,
        nsamp_in=cfg["nsamp"],
        ndm=hi - lo, ndm_total=len(dms), shards=shards, dms=dms, wchan=cfg["wchan"], band=band,
        widths=cfg["widths"], delay=delay, taps=taps, w=w, dtype="f32",
        flops=2.0 * float(taps.astype(np.int64).sum()) * t_out, ns_total=int(info["ns_total"]),
    )


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [v.strip() for v in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax = float(p[2])
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- timing


def _dist():
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1 and not dist.is_initialized():
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    rank = int(os.environ.get("RANK", "0"))
    return rank, ws


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args):
    import torch
    import paper_1301_3968_gb300 as dd
    from paper_1301_3968_gb300 import build as dd_build

    rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dd_build.build()
    W = craft_workload(dd, dev, args.ndm, rank, ws)
    plan, x = W["plan"], W["x"]
    widths = W["widths"]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)      # 256 MiB > 129 MB L2
    out = torch.empty((W["ndm"], W["t_out"]), dtype=torch.float32, device=dev)

    def step(ev=None):
        mean, sd = plan.channel_stats(x, nsamp=W["nsamp_in"])
        if ev is not None:
            ev[0].record(stream)
        plan.dedisperse(x, nsamp=W["nsamp"], out=out)
        if ev is not None:
            ev[1].record(stream)
        return plan.boxcar_snr(out, widths, mean, sd, t_len=W["t_out"])

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()

    clk = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clk:
        clk.start()
        time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    _barrier(ws)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                     # evict the input from L2 between steps
        evs[i][0].record(stream)
        step(kev[i])
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    k_ms = [a.elapsed_time(b) for a, b in kev]
    clocks = clk.stop() if clk else None
    ms = _max_over_ranks(sum(step_ms) / len(step_ms), ws)
    units = float(W["ndm_total"]) * W["t_out"]      # every rank's trials, one output span
    value = units / (ms / 1e3)

    e2e = None if args.no_e2e else e2e_run(args, W, ws, plan, x, out, widths, stream)
    shard = merge_check(dd, dev, W, rank, ws, plan, x, out, widths) if ws > 1 else None
    # the device's measured FP32 FMA (scalar and packed pairs) and INT32 add rates (after
    # the timed region), and its SM count
    live = {"fma_tflops": dd.alu_peak("fma") / 1e12, "fma2_tflops": dd.alu_peak("fma2") / 1e12,
            "iadd_tops": dd.alu_peak("iadd") / 1e12,
            "sms": torch.cuda.get_device_properties(dev).multi_processor_count}
    extras = None
    if rank == 0 and ws == 1 and not args.no_extras:
        extras = {"craft_fused": craft_fused_extra(W, plan, x, out, widths, flush, stream, ms),
                  "plain": plain_extra(dd, dev, flush, stream),
                  "fwd_bwd": diff_extra(dd, dev, flush, stream),
                  "batched": batched_extra(dd, dev, flush, stream, iadd_tops=live["iadd_tops"]),
                  "large_lowband": large_extra(dd, dev, flush, stream, iadd_tops=live["iadd_tops"],
                                               sms=live["sms"])}
    return _result(args, W, ws, rank, ms, value, k_ms, clocks, e2e, extras, live, shard)


def merge_check(dd, dev, W, rank, ws, plan, x, out, widths):
    """After the timed region: gathers every rank's peak S/N and peak times on rank 0 and
    compares the merged tables with one plan over the whole trial list on rank 0's GPU."""
    import torch
    import torch.distributed as dist
    mean, sd = plan.channel_stats(x, nsamp=W["nsamp_in"])
    plan.dedisperse(x, nsamp=W["nsamp"], out=out)
    pk, ag, _ = plan.boxcar_snr(out, widths, mean, sd, t_len=W["t_out"])
    mine = (pk.cpu().numpy(), ag.cpu().numpy())
    got = [None] * ws if rank == 0 else None
    dist.gather_object(mine, got, dst=0)
    if rank != 0:
        return None
    peak = np.concatenate([g[0] for g in got])
    arg = np.concatenate([g[1] for g in got])
    fp = dd.Plan(W["band"], W["dms"])
    _, taps = fp.tables()
    K = W["w"].shape[2]
    w = np.where(np.arange(K)[None, None, :] < taps[:, :, None], W["wchan"][None, :, None], 0.0)
    fp.set_profiles(weights=np.ascontiguousarray(w, dtype=np.float32))
    nsamp = W["t_out"] + fp.d_max
    fout = torch.empty((fp.ndm, W["t_out"]), dtype=torch.float32, device=dev)
    m1, s1 = fp.channel_stats(x, nsamp=W["nsamp_in"])
    fp.dedisperse(x, nsamp=nsamp, out=fout)
    p1, a1, _ = fp.boxcar_snr(fout, widths, m1, s1, t_len=W["t_out"])
    p1, a1 = p1.cpu().numpy(), a1.cpu().numpy()
    fp.close()
    return {"trials_per_rank": [hi - lo for lo, hi in W["shards"]],
            "trial_ranges": W["shards"],
            "merged_peak_snr_equal_one_gpu": bool(np.array_equal(peak, p1)),
            "merged_peak_t_equal_one_gpu": bool(np.array_equal(arg, a1)),
            "max_abs_snr_diff": float(np.max(np.abs(peak - p1)))}


def e2e_run(args, W, ws, plan, x, out, widths, stream):
    """End to end through the public API: every step copies its input block from pinned host
    memory to the device, runs the hot path and copies the peak S/N and times back.  The
    copy of step i + 1's input runs on a copy stream into a second buffer while step i
    computes (a streaming pipeline's double buffering); every copy is inside the timed
    region."""
    import torch

    host = torch.from_numpy(W["host"]).pin_memory()
    peak_h = torch.empty((W["ndm"], len(widths)), dtype=torch.float32).pin_memory()
    arg_h = torch.empty((W["ndm"], len(widths)), dtype=torch.int32).pin_memory()
    xin = [torch.empty_like(x), torch.empty_like(x)]
    cs = torch.cuda.Stream(device=x.device)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    freed = [torch.cuda.Event(), torch.cuda.Event()]

    def steps(n):
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            xin[0].copy_(host, non_blocking=True)
            copied[0].record(cs)
        for i in range(n):
            b = i & 1
            if i + 1 < n:  # the next input, once step i - 1 is done with that buffer
                with torch.cuda.stream(cs):
                    if i >= 1:
                        cs.wait_event(freed[b ^ 1])
                    xin[b ^ 1].copy_(host, non_blocking=True)
                    copied[b ^ 1].record(cs)
            stream.wait_event(copied[b])
            mean, sd = plan.channel_stats(xin[b], nsamp=W["nsamp_in"])
            plan.dedisperse(xin[b], nsamp=W["nsamp"], out=out)
            freed[b].record(stream)
            pk, ag, _ = plan.boxcar_snr(out, widths, mean, sd, t_len=W["t_out"])
            peak_h.copy_(pk, non_blocking=True)
            arg_h.copy_(ag, non_blocking=True)

    steps(max(2, args.warmup))
    torch.cuda.synchronize()
    _barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    steps(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms = _max_over_ranks(e0.elapsed_time(e1) / args.steps, ws)
    # bytes of the whole job: every rank copies the input in and its peaks out
    h2d = ws * host.numel() * host.element_size()
    d2h = W["ndm_total"] * len(widths) * 8
    units = float(W["ndm_total"]) * W["t_out"]
    return {"value": units / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": e_ms,
            "copies": "input H2D on a copy stream, double-buffered against the previous step"}


# ----------------------------------------------------------------------------- extras


def _ev_time(fn, reps, flush, stream):
    """Mean device time (ms) of fn over `reps` calls, L2 flushed before each, events on
    the launching stream."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for i in range(reps):
        flush.fill_(i & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sum(ts) / len(ts)


def craft_fused_extra(W, plan, x, out, widths, flush, stream, step_ms, reps=10):
    """The CRAFT-like step with the boxcar scan fused into the dedispersion CTAs
    (dd_dedisperse_boxcar: the 4096 x 60261 fp32 series is never stored): its time against
    the unfused step's, and its peak S/N and times against the unfused step's, bit for bit."""
    import torch

    def fstep():
        mean, sd = plan.channel_stats(x, nsamp=W["nsamp_in"])
        return plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=W["nsamp"])

    ms = _ev_time(fstep, reps, flush, stream)
    pf, af, _ = fstep()
    mean, sd = plan.channel_stats(x, nsamp=W["nsamp_in"])
    plan.dedisperse(x, nsamp=W["nsamp"], out=out)
    pu, au, _ = plan.boxcar_snr(out, widths, mean, sd, t_len=W["t_out"])
    units = float(W["ndm"]) * W["t_out"]
    return {"step_ms": ms, "value": units / (ms / 1e3), "unit": "DM-trial\u00b7samples/s",
            "unfused_step_ms": step_ms, "fused_over_unfused": ms / step_ms if step_ms else None,
            "peaks_equal_unfused_bitwise": bool(torch.equal(pf.view(torch.int32), pu.view(torch.int32))
                                                and torch.equal(af, au)),
            "status": plan.device_status(),
            "series_bytes_not_stored": int(W["ndm"]) * W["t_out"] * 4}


def diff_extra(dd, dev, flush, stream, reps=5):
    """Differentiable configuration: 336 ch, 16384 fp32 samples, 1024 trial DMs to 2000,
    32 learnable fp32 taps per channel.  Plain forward (fixed weights) against one
    forward + backward through DDFunction (weights copied in, the dedispersed series,
    then the adjoint for the weight and input gradients)."""
    import torch
    import synth
    cfg = synth.make_diff(npulse=0)          # timing does not depend on the pulses
    b, T, D, K = cfg["band"], cfg["nsamp"], 1024, 32
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "f32")
    dms, _ = dd.trial_dms(band, 0.0, 2000.0, D, tau_av_ms=1.0)
    plan = dd.Plan(band, dms)
    delay, taps0 = plan.tables()
    rng = np.random.default_rng(synth.sub_seed("diff-weights"))
    w0 = (rng.uniform(0.5, 1.5, size=(D, b.nchan, K))
          * (np.arange(K)[None, None, :] < taps0[:, :, None])).astype(np.float32)
    plan.set_profiles(delay=delay, taps=np.full_like(taps0, K), weights=w0)
    t_out = T - plan.d_max
    x = torch.from_numpy(cfg["data"]).to(dev)
    w = torch.from_numpy(w0).to(dev)
    out = torch.empty((D, t_out), dtype=torch.float32, device=dev)
    g = torch.from_numpy(rng.standard_normal((D, t_out)).astype(np.float32)).to(dev)
    plan.set_weights(w)
    fwd_ms = _ev_time(lambda: plan.dedisperse(x, nsamp=T, out=out), reps, flush, stream)
    xr = x.clone().requires_grad_(True)
    wr = w.clone().requires_grad_(True)

    def fwd_bwd():
        xr.grad = None
        wr.grad = None
        y = dd.DDFunction.apply(xr, wr, plan, 0, T)
        y.backward(g)

    fb_ms = _ev_time(fwd_bwd, reps, flush, stream)
    bw_ms = _ev_time(lambda: plan.backward(x, g, nsamp=T, want_gin=False), reps, flush, stream)
    bi_ms = _ev_time(lambda: plan.backward(x, g, nsamp=T, want_gw=False), reps, flush, stream)
    units = float(D) * t_out
    flops = 2.0 * D * b.nchan * K * t_out
    plan.close()
    return {
        "workload": (f"differentiable: {b.nchan} ch, {T} fp32 samples (noise), {D} trial DMs "
                     f"0-2000, {K} learnable taps per channel"),
        "fwd_ms": fwd_ms, "fwd_bwd_ms": fb_ms, "bwd_w_ms": bw_ms, "bwd_in_ms": bi_ms,
        "fwd_value": units / (fwd_ms / 1e3), "fwd_bwd_value": units / (fb_ms / 1e3), "unit": UNIT,
        "fwd_bwd_over_fwd": fb_ms / fwd_ms,
        "fwd_tflops": flops / (fwd_ms / 1e3) / 1e12,
        "bwd_w_tflops": flops / (bw_ms / 1e3) / 1e12,
        "bwd_in_tflops": flops / (bi_ms / 1e3) / 1e12,
    }


def plain_extra(dd, dev, flush, stream, reps=20):
    """Plain configuration: 64 channels over 1200-1500 MHz, dt 1 ms, 4096 uint8 samples,
    128 trial DMs 0-500, unit weights (exact integer sums), boxcar widths 1-16.  About
    2 MB of data: launch- and latency-bound, reported but not held to a roofline."""
    import torch
    import synth
    cfg = synth.make_plain()
    b = cfg["band"]
    plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, cfg["nsamp"], "u8"), cfg["dms"])
    x = torch.from_numpy(cfg["data"]).to(dev)
    out = torch.empty((plan.ndm, cfg["nsamp"] - plan.d_max), dtype=torch.int32, device=dev)
    widths = np.arange(1, 17, dtype=np.int32)

    def step():
        m, s = plan.channel_stats(x, nsamp=cfg["nsamp"])
        plan.dedisperse(x, nsamp=cfg["nsamp"], out=out)
        plan.boxcar_snr(out, widths, m, s)

    dd_ms = _ev_time(lambda: plan.dedisperse(x, nsamp=cfg["nsamp"], out=out), reps, flush, stream)
    st_ms = _ev_time(step, reps, flush, stream)
    units = float(plan.ndm) * out.shape[1]
    plan.close()
    return {"workload": "plain: 64 ch 1200-1500 MHz, dt 1 ms, 4096 uint8 samples, 128 trial DMs 0-500, "
                        "unit weights, int32 out, boxcar widths 1-16",
            "dedisp_ms": dd_ms, "step_ms": st_ms, "dedisp_value": units / (dd_ms / 1e3),
            "step_value": units / (st_ms / 1e3), "unit": UNIT}


def _batch_case(dd, dev, flush, stream, cfg, reps, tune, widths, graph=True):
    """Plans for a set of beams (default schedules timed one launch after another, then
    autotuned), their batched launch, and optionally the graph of the whole block."""
    import torch
    import synth
    b = cfg["band"]
    plans, xs, outs = [], [], []
    for beam in cfg["beams"]:
        band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, beam["nsamp"], "u8")
        dms, _ = dd.trial_dms(band, 0.0, beam["dm_max"], beam["ndm"], tau_av_ms=1.0)
        plans.append(dd.Plan(band, dms))
        xs.append(torch.from_numpy(synth.make_beam_data(beam)).to(dev))
        outs.append(torch.empty((len(dms), beam["nsamp"] - plans[-1].d_max), dtype=torch.int32, device=dev))

    def per_beam_fwd():
        for p, x, o in zip(plans, xs, outs):
            p.dedisperse(x, nsamp=p.band.nsamp, out=o)

    gs = torch.cuda.Stream(dev)
    gs.wait_stream(stream)
    res = {}
    with torch.cuda.stream(gs):
        res["default_fwd_ms"] = _ev_time(per_beam_fwd, reps, flush, gs)
        for p, x, o in zip(plans, xs, outs):
            p.autotune(x, o, cache_path=tune)
        batch = dd.Batch(plans)
        batch.bind(xs, outs)
        res["plain_fwd_ms"] = _ev_time(per_beam_fwd, reps, flush, gs)
        res["batched_fwd_ms"] = _ev_time(lambda: batch.dedisperse(gs), reps, flush, gs)
        if graph:
            means = [torch.empty(b.nchan, dtype=torch.float64, device=dev) for _ in plans]
            sds = [torch.empty_like(m) for m in means]
            peaks = [torch.empty((p.ndm, len(widths)), dtype=torch.float32, device=dev) for p in plans]
            args = [torch.empty((p.ndm, len(widths)), dtype=torch.int32, device=dev) for p in plans]
            batch.bind_boxcar(widths, means, sds, peaks, args)

            def per_beam_step():
                for p, x, o in zip(plans, xs, outs):
                    m, s = p.channel_stats(x, nsamp=p.band.nsamp)
                    p.dedisperse(x, nsamp=p.band.nsamp, out=o)
                    p.boxcar_snr(o, widths, m, s)

            res["plain_step_ms"] = _ev_time(per_beam_step, reps, flush, gs)
            batch.capture(gs)
            res["graph_step_ms"] = _ev_time(lambda: batch.replay(gs), reps, flush, gs)
    info = batch.info()
    # work: trial x output samples; additions the direct path executes (one per tap,
    # trial and output) and the graded exact count (min(n, 2) per trial, channel and
    # output plus one per input sample for a prefix pass)
    units = executed = graded = 0.0
    for p, o in zip(plans, outs):
        _, taps = p.tables()
        t_out = o.shape[1]
        units += float(p.ndm) * t_out
        executed += float(taps.astype(np.int64).sum()) * t_out
        graded += float(np.minimum(taps, 2).astype(np.int64).sum()) * t_out + float(b.nchan) * p.band.nsamp
    batch.close()
    for p in plans:
        p.close()
    res.update(units=units, executed_adds=executed, graded_adds=graded, items=info["items"],
               grid=info["grid"], nbeams=len(plans), samples=sum(x.shape[1] for x in xs),
               trials=sum(o.shape[0] for o in outs))
    return res


def batched_extra(dd, dev, flush, stream, reps=3, iadd_tops=None):
    """Batched configuration: 36 beams on the CRAFT band, uint8 in / int32 out, per-beam
    lengths 2^14-2^17 and 512-8192 trial DMs (seeded log-uniform), each plan autotuned.
    One batched launch (and the CUDA graph of the whole block, boxcars included)
    against the same beams run one plain launch after another; the autotuner's gain over
    the default schedules; and 36 beams from the lower end of both ranges (2^14-2^15
    samples, 512-1024 trials), where each beam's own launch is a few waves."""
    import tempfile
    import synth
    widths = np.arange(1, 33, dtype=np.int32)
    tune = os.path.join(tempfile.mkdtemp(prefix="dd_tune_"), "schedule.txt")
    r = _batch_case(dd, dev, flush, stream, synth.make_batched_beams(), reps, tune, widths)
    small = _batch_case(dd, dev, flush, stream,
                        synth.make_batched_beams(seed=synth.sub_seed("batched-small"), t_exp=(14, 15),
                                                 d_exp=(9, 10)), 5, tune, widths, graph=False)
    units = r["units"]
    res = {
        "workload": (f"batched: {r['nbeams']} beams, 336 ch, {r['samples']} uint8 samples in all, "
                     f"{r['trials']} trials in all, int32 out, boxcar widths 1-32, autotuned schedules"),
        "units": units, "items": r["items"], "grid": r["grid"],
        "default_schedule_fwd_ms": r["default_fwd_ms"], "plain_fwd_ms": r["plain_fwd_ms"],
        "autotune_gain": r["default_fwd_ms"] / r["plain_fwd_ms"],
        "batched_fwd_ms": r["batched_fwd_ms"],
        "plain_step_ms": r["plain_step_ms"], "graph_step_ms": r["graph_step_ms"],
        "plain_fwd_value": units / (r["plain_fwd_ms"] / 1e3),
        "batched_fwd_value": units / (r["batched_fwd_ms"] / 1e3),
        "graph_step_value": units / (r["graph_step_ms"] / 1e3), "unit": UNIT,
        "batched_over_plain_fwd": r["plain_fwd_ms"] / r["batched_fwd_ms"],
        "executed_adds_per_block": r["executed_adds"], "graded_adds_per_block": r["graded_adds"],
        "small_beams": {
            "workload": (f"{small['nbeams']} beams, 336 ch, 2^14-2^15 samples and 512-1024 trials each "
                         f"({small['samples']} samples, {small['trials']} trials in all), autotuned"),
            "plain_fwd_ms": small["plain_fwd_ms"], "batched_fwd_ms": small["batched_fwd_ms"],
            "batched_over_plain_fwd": small["plain_fwd_ms"] / small["batched_fwd_ms"],
            "autotune_gain": small["default_fwd_ms"] / small["plain_fwd_ms"],
            "batched_fwd_value": small["units"] / (small["batched_fwd_ms"] / 1e3)},
    }
    if iadd_tops:
        # the direct integer path: one add per tap (two per three-input add); graded: the
        # exact minimum of a prefix-difference method
        res["executed_frac_of_measured_iadd"] = r["executed_adds"] / (r["batched_fwd_ms"] / 1e3) / 1e12 / iadd_tops
        res["graded_frac_of_measured_iadd"] = r["graded_adds"] / (r["batched_fwd_ms"] / 1e3) / 1e12 / iadd_tops
    return res


def large_extra(dd, dev, flush, stream, chunk=1 << 18, nsamp=1 << 20, ndm=8192, iadd_tops=None,
                sm_mhz=None, sms=None, dm_range=None):
    """Large low-band configuration: 1024 ch over 700-1000 MHz, dt 64 us, 2^20 uint8
    samples, 8192 trial DMs 0-2000 (unit weights, run-length sums), streamed in
    overlapping chunks of `chunk` outputs (each chunk reads its outputs plus d_max
    samples), int32 out, then boxcar S/N over widths 1-256 per chunk."""
    import torch
    import synth
    if sm_mhz is None:
        sm_mhz = float(_peaks()[0].get("sm_max_mhz", 2070.0))
    if sms is None:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cfg = synth.make_large(nsamp=nsamp)
    b, T = cfg["band"], cfg["nsamp"]
    if dm_range is not None:   # a profiling case: part of the list at the same spacing
        dms = np.linspace(dm_range[0], dm_range[1], ndm)
    else:
        dms = cfg["dms"] if ndm == len(cfg["dms"]) else np.linspace(0.0, cfg["dms"][-1], ndm)
    plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "u8"), dms)
    x = torch.from_numpy(cfg["data"]).to(dev)
    dmax = plan.d_max
    t_out = T - dmax
    starts = list(range(0, t_out, chunk))
    out = torch.empty((plan.ndm, chunk), dtype=torch.int32, device=dev)
    widths = np.arange(1, 257, dtype=np.int32)
    mean, sd = plan.channel_stats(x, nsamp=T)

    def dedisp_all():
        for t0 in starts:
            n = min(chunk, t_out - t0)
            plan.dedisperse(x, t_offset=t0, nsamp=n + dmax, out=out)

    def step_all():
        for t0 in starts:
            n = min(chunk, t_out - t0)
            plan.dedisperse(x, t_offset=t0, nsamp=n + dmax, out=out)
            plan.boxcar_snr(out, widths, mean, sd, t_len=n)

    def fused_all():
        for t0 in starts:
            n = min(chunk, t_out - t0)
            plan.dedisperse_boxcar(x, widths, mean, sd, t_offset=t0, nsamp=n + dmax)

    dd_ms = _ev_time(dedisp_all, 2, flush, stream)
    st_ms = _ev_time(step_all, 2, flush, stream)
    fu_ms = _ev_time(fused_all, 2, flush, stream)
    fu_status = plan.device_status()
    units = float(plan.ndm) * t_out
    dct = units * b.nchan
    # graded work of exact unit-weight sums: min(n, 2) additions per (trial, channel,
    # output) plus one per input sample for the prefix pass
    _, taps = plan.tables()
    graded = float(np.minimum(taps, 2).astype(np.int64).sum()) * t_out + float(b.nchan) * T
    res = {
        "workload": (f"large low-band: {b.nchan} ch 700-1000 MHz, dt 64 us, {T} uint8 samples, "
                     f"{plan.ndm} trial DMs {dms[0]:.0f}-{dms[-1]:.0f}, {len(starts)} overlapping chunks of {chunk} "
                     "outputs, int32 out, boxcar widths 1-256"),
        "method": plan.method, "d_max": dmax, "t_out": t_out,
        "dedisp_ms": dd_ms, "step_ms": st_ms,
        "dedisp_value": units / (dd_ms / 1e3), "step_value": units / (st_ms / 1e3), "unit": UNIT,
        "trial_channel_samples_per_s": dct / (dd_ms / 1e3),
        "realtime_factor": (t_out * b.dt_ms / 1e3) / (st_ms / 1e3),
        "fused_step_ms": fu_ms, "fused_value": units / (fu_ms / 1e3), "fused_over_step": fu_ms / st_ms,
        "fused_status": fu_status,
        "fused_series_bytes_not_stored": plan.ndm * chunk * 4,
        # the run-length kernel's bound: shared-memory reads, one 4-byte word per (trial,
        # channel, output) from the CTA's difference rows (two without them), against
        # the SMs x 128 B/clk at the measured clock
        "smem_read_bytes_per_block": 4.0 * dct,
        "smem_read_tbps": 4.0 * dct / (dd_ms / 1e3) / 1e12,
        "smem_peak_tbps": sms * SMEM_BYTES_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12,
        "graded_adds_per_block": graded,
        "graded_tops": graded / (dd_ms / 1e3) / 1e12,
        "bound": "shared-memory reads (1 word per trial, channel and output with the CTA's difference rows; see profiles)",
    }
    res["smem_read_frac"] = res["smem_read_tbps"] / res["smem_peak_tbps"]
    res["smem_peak_kind"] = f"derived: {sms} SMs x {SMEM_BYTES_PER_CLK_PER_SM} B/clk x {sm_mhz:.0f} MHz"
    if iadd_tops:
        res["graded_frac_of_measured_iadd"] = res["graded_tops"] / iadd_tops
    plan.close()
    return res


TRAFFIC_SOURCES = ["dd_tile.cuh", "dd_dedisp.cu", "dd_internal.h", "dd_packed.cuh", "dd_fused_scan.cuh",
                   "dd_debug.cuh"]


def kernel_source_sha():
    """sha256 over the sources the dedispersion kernel is compiled from, in a fixed order."""
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1301_3968_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _profile_traffic():
    """DRAM bytes per dedispersion launch from the ncu capture recorded in
    profiles/traffic.json, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)["k_dedisp_f32_craft"]
        sha = kernel_source_sha()
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("source_sha256") != sha:
        return None
    try:
        return float(rec["dram_bytes_per_launch"])
    except (KeyError, TypeError, ValueError):
        return None


def _result(args, W, ws, rank, ms, value, k_ms, clocks, e2e, extras=None, live=None, shard=None):
    if rank != 0:
        return None
    peaks, kind = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = live["sms"] if live else 152
    derived = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    # the denominator is the largest of the derived FP32 rate and the measured scalar and
    # packed FMA rates
    cands = {"derived": derived}
    if live:
        cands["measured_fma"] = live["fma_tflops"]
        cands["measured_fma2"] = live["fma2_tflops"]
    peak_name = max(cands, key=cands.get)
    peak_tflops = cands[peak_name]
    k_avg = sum(k_ms) / len(k_ms)
    achieved = W["flops"] / (k_avg / 1e3) / 1e12
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": W["dtype"], "data": "synthetic",
        "config": {"workload": W["desc"], "trials": W["ndm_total"], "t_out": W["t_out"],
                   "channels": 336, "nsamp": int(W["host"].shape[1]), "taps_total": W["ns_total"],
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": (f"dm{ws}: contiguous cost-balanced trial ranges per GPU, a full "
                                   "input replica each, peaks merged on the host; no collective "
                                   "on the data path")},
        "e2e": e2e,
        "gpu_launches": LAUNCHES_PER_STEP * args.steps * ws,   # every rank launches its own
        "roofline": {"bound": "alu", "kernel": "k_dedisp<float,float,weighted>",
                     "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops,
                     "traffic": args.traffic if args.traffic is not None else _profile_traffic(),
                     "peak_kind": (f"{peak_name}: the largest of the derived rate ({sms} SMs x "
                                   f"{FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_max:.0f} MHz, {kind} "
                                   "sm_max_mhz = %.1f) and the measured scalar and packed FMA rates" % derived),
                     "peak_candidates": cands,
                     "kernel_ms": k_avg, "flops_per_launch": W["flops"]},
        "alu_peaks_measured": live,
        "clocks": clocks,
    }
    if live:
        res["roofline"]["frac_of_measured_fma"] = achieved / live["fma_tflops"]
        res["roofline"]["frac_of_measured_fma2"] = achieved / live["fma2_tflops"]
        res["config"]["sms"] = sms
    if shard is not None:
        res["shard"] = shard
    if extras is not None:
        res["extras"] = extras
    if ws == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(W, budget_s=args.cpu_seconds)
    return res


# ----------------------------------------------------------------------------- oracle


def cpu_baseline(W, budget_s=12.0):
    """The oracle as it stands (C brute force + numpy boxcar) on a bounded sample of
    trial rows of the same workload, on this host's cores."""
    import oracle
    from oracle import ref
    I, delay, taps, w = W["host"], W["delay"], W["taps"], W["w"]
    nsamp, t_out, widths = W["nsamp"], W["t_out"], W["widths"]
    mu_c, sd_c = ref.channel_stats(I, nsamp=nsamp)
    rng = np.random.default_rng(7)
    order = rng.permutation(W["ndm"])
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s and done < W["ndm"]:
        rows = np.sort(order[done:done + 16])
        x = oracle.c_dedisperse(I, delay, taps, w=w, nsamp=nsamp, rows=rows)
        mu, sd = ref.boxcar_norm(taps[rows], widths, mu_c, sd_c, w=w[rows])
        ref.boxcar_snr(x, widths, mu, sd)
        done += len(rows)
    el = time.perf_counter() - t0
    return {"value": done * t_out / el, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{done} of {W['ndm']} trial rows (random), full {t_out} outputs each, "
                      f"dedispersion + boxcar normaliser + boxcar S/N, {el:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    from oracle import ref
    import synth
    cfg = synth.make_craft()
    b = cfg["band"]
    dms, eps = ref.trial_dms(0.0, cfg["dm_max"], cfg["ndm"], b.nchan, b.f_lo_mhz, b.df_mhz,
                             b.dt_ms, 1.0)
    delay, _ = ref.delay_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms)
    taps, _ = ref.taps_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms)
    K = int(taps.max())
    w = np.where(np.arange(K)[None, None, :] < taps[:, :, None], cfg["wchan"][None, :, None], 0.0)
    w = np.ascontiguousarray(w, dtype=np.float32)
    nsamp = cfg["nsamp"]
    t_out = nsamp - ref.d_max(delay, taps)
    widths = cfg["widths"]
    rows_per_step = 8
    rng = np.random.default_rng(11)

    def step():
        rows = np.sort(rng.choice(len(dms), rows_per_step, replace=False))
        mu_c, sd_c = ref.channel_stats(cfg["data"], nsamp=nsamp)
        x = oracle.c_dedisperse(cfg["data"], delay, taps, w=w, nsamp=nsamp, rows=rows)
        mu, sd = ref.boxcar_norm(taps[rows], widths, mu_c, sd_c, w=w[rows])
        ref.boxcar_snr(x, widths, mu, sd)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    ms = el / args.steps * 1e3
    value = rows_per_step * t_out / (el / args.steps)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "CRAFT-like: 336 ch x 1 MHz, dt 1 ms, 65536 fp32 samples, 4096 trial "
                               "DMs 0-4000 (eq. trial DMs), weights ~ nu^-1.4, boxcar widths 1-32",
                   "sample": f"{rows_per_step} random trial rows per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{rows_per_step} random trial rows of 4096 per step, full "
                                   f"{t_out} outputs, stats + dedispersion + normaliser + boxcar"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_only(args):
    """One extra measurement alone (rank 0, no headline step): for profiling a kernel of
    that configuration."""
    import torch
    import paper_1301_3968_gb300 as dd
    from paper_1301_3968_gb300 import build as dd_build
    dd_build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    if args.only == "plain":
        r = plain_extra(dd, dev, flush, stream)
    elif args.only == "craft_fused":
        W = craft_workload(dd, dev, args.ndm)
        out = torch.empty((W["ndm"], W["t_out"]), dtype=torch.float32, device=dev)
        plan, x = W["plan"], W["x"]

        def ustep():
            mean, sd = plan.channel_stats(x, nsamp=W["nsamp_in"])
            plan.dedisperse(x, nsamp=W["nsamp"], out=out)
            return plan.boxcar_snr(out, W["widths"], mean, sd, t_len=W["t_out"])

        r = craft_fused_extra(W, plan, x, out, W["widths"], flush, stream, _ev_time(ustep, 10, flush, stream))
    elif args.only == "fwd_bwd":
        r = diff_extra(dd, dev, flush, stream)
    elif args.only == "batched":
        r = batched_extra(dd, dev, flush, stream, iadd_tops=dd.alu_peak("iadd") / 1e12)
    else:
        rng = None if args.large_dm_range is None else tuple(args.large_dm_range)
        r = large_extra(dd, dev, flush, stream, nsamp=args.large_nsamp, ndm=args.large_ndm,
                        iadd_tops=dd.alu_peak("iadd") / 1e12, dm_range=rng,
                        chunk=min(1 << 18, args.large_nsamp))
    return {"only": args.only, **r}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ndm", type=int, default=None,
                    help="profiling case: this many consecutive trials from the middle of the "
                         "4096-trial list")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--only", default=None, choices=["plain", "craft_fused", "fwd_bwd", "batched", "large_lowband"],
                    help="run one extra measurement alone (profiling)")
    ap.add_argument("--large-nsamp", type=int, default=1 << 20)
    ap.add_argument("--large-ndm", type=int, default=8192)
    ap.add_argument("--large-dm-range", type=float, nargs=2, default=None,
                    help="profiling case: --large-ndm trials evenly over this DM range")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the forward+backward, batched-beam and large low-band measurements")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per dedispersion launch from an ncu capture")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ and not args.only:
        # not started by a launcher: start one rank per GPU on this node
        import socket
        sk = socket.socket()
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
        sk.close()
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
               f"--nproc-per-node={args.gpus}", "--master-addr=127.0.0.1", f"--master-port={port}",
               os.path.abspath(__file__)] + sys.argv[1:]
        sys.exit(subprocess.run(cmd).returncode)
    if args.only:
        res = run_only(args)
    elif args.impl == "reference":
        res = run_reference(args)
    else:
        res = run_gpu(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
