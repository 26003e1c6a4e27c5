#!/usr/bin/env python
"""Throughput of the signal-simulation hot path on one GB300 (or N, weak scaling).

A step simulates one event on the three-plane detector (800/800/960 wires x
6000 ticks, 100,000 track depos, binomial fluctuation with survival 0.7):
for every plane, diffusion + raster + fluctuation + scatter-add into the
grid, then the FFT convolution with that plane's response.  The metric is
depos per second through the whole path (a depo counts once per plane it is
simulated on), with planes per second and the raster+scatter-only rate
reported beside it.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 oracle
on the host cores instead (the CPU baseline arm).

Timing: the event's batch (wave size picked by timing) is captured into a
CUDA graph; W untimed warm-up replays; then K replays, each bracketed by
CUDA events on the launching stream, with L2 flushed (a 512 MiB write)
between steps, outside the events; barrier + synchronize on both sides; the
max over ranks.  Per-kernel device times come from the library's own launch
trace (CUDA events around every launch, on the launching stream) over K
steps of the same event launched one stage at a time.

Under torchrun each rank simulates its own event (its own seed and event id):
the units are independent, so there is no collective on the data path, only
the barrier and the max/sum reductions of the timing (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_02479_gb300 import inputs  # noqa: E402

METRIC = "depos/sec and planes/sec (raster+scatter+FFT conv) at 1 GB300; % of HBM roofline"
UNIT = "depos/s"
FP32_LANES_PER_SM = 128
NUM_SMS_GB300 = 152


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(prefix="clocks_", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.close()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------ distributed
def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _init_pg(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend=backend)
    return dist


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, value: float, device) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(dist, value: float, device) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# -------------------------------------------------------------- workloads
def make_workload(name: str, rank: int):
    if name == "three_planes":
        return inputs.three_planes(seed=1001 + 7919 * rank)
    if name == "single_plane":
        return inputs.single_plane(seed=1000 + 7919 * rank)
    raise SystemExit(f"unknown workload {name}")


def algorithmic_bytes(kernel: str, nw: int, nt: int, nfreq: int, kw: int, ndepo: int) -> float:
    """Bytes a kernel's step must move at minimum (inputs read once, outputs
    written once), per launch on one plane."""
    spec = 8.0 * nfreq * nw
    if kernel == "raster_scatter":
        return 12.0 * ndepo + 4.0 * nw * nt
    if kernel == "fwd_rows":
        return 4.0 * nw * nt + spec
    if kernel == "wire_conv":
        return 2.0 * spec + 8.0 * nfreq * kw
    if kernel == "inv_rows":
        return spec + 4.0 * nw * nt
    if kernel == "memset_grid":
        return 4.0 * nw * nt
    return 0.0


# ------------------------------------------------------------------ oracle
_ORACLE_NEXT = [0]


def oracle_sample(w, budget_s: float, keep=None):
    """Run the FP64 oracle over the workload's planes (cycling through them
    across calls) for about budget_s seconds, at least one plane; returns
    (depo-planes processed, seconds, planes).  keep: a dict that receives
    the first waveform computed for each plane index (event 0)."""
    import oracle
    done = 0
    planes = 0
    t0 = time.perf_counter()
    while True:
        i = _ORACLE_NEXT[0]
        _ORACLE_NEXT[0] += 1
        sp = w.planes[i % len(w.planes)]
        d = w.events[0][i % len(w.planes)]
        S = oracle.raster_scatter(d.q, d.x_mm, d.t_us, sp.nwires, sp.nticks, fluctuate=w.fluctuate,
                                  p=w.p_survive, seed=w.seed, event_id=0, plane_id=sp.plane_id)
        M = oracle.convolve_fft(S, sp.response, 10)
        if keep is not None and i % len(w.planes) not in keep:
            keep[i % len(w.planes)] = M
        done += d.n
        planes += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return done, time.perf_counter() - t0, planes


def oracle_error_of(gpu_out, kept, w):
    """Error of the timed event's waveforms against the FP64 oracle for the
    planes the CPU baseline computed: relative L2 over the plane and the
    largest absolute difference over the largest |M|.  Fluctuated events
    use the same counters on both sides; bins where FP32 and FP64 round
    q w to different electron counts differ by one electron."""
    out = []
    for i in sorted(kept):
        M = kept[i]
        diff = gpu_out[i].astype(np.float64) - M
        out.append({"plane_id": w.planes[i].plane_id,
                    "rel_l2": float(np.linalg.norm(diff) / max(np.linalg.norm(M), 1e-300)),
                    "max_abs_over_max": float(np.abs(diff).max() / max(np.abs(M).max(), 1e-300))})
    return {"planes": out, "mode": "binomial" if w.fluctuate else "expected value",
            "note": "same seed and counters as the GPU; FP32 on the GPU against FP64"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    w = make_workload(args.workload, 0)
    # a step is one plane of the event through the oracle (~0.5 s on one
    # thread); warm-up and timed steps stop early once the time budget is
    # spent so that any --steps ends within a few minutes
    t_start = time.perf_counter()
    for _ in range(args.warmup):
        oracle_sample(w, 0.0)
        if time.perf_counter() - t_start > 0.2 * args.reference_seconds:
            break
    t0 = time.perf_counter()
    done = 0
    planes = 0
    steps = 0
    for _ in range(args.steps):
        d, _, p = oracle_sample(w, 0.0)   # one plane per step
        done += d
        planes += p
        steps += 1
        if time.perf_counter() - t0 > args.reference_seconds:
            break
    dt = time.perf_counter() - t0
    value = done / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "sample": "one plane of the event per step (cycling U, V, W)",
                   "depos_per_plane": w.events[0][0].n, "steps_requested": args.steps,
                   "time_budget_s": args.reference_seconds},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{steps} steps (of {args.steps} requested, {args.reference_seconds:.0f} s "
                                   f"budget) x one plane of {w.events[0][0].n} depos"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "planes_per_s": planes / dt,
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- main
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x max SM clock
INT_MUL_PEAK_T = 152 * 64 * 2.070e9 / 1e12          # 152 SMs x 64 INT32 multiply lanes x max SM clock
PHILOX_MULS = 40    # 32-bit multiplies per Philox4x32-10 block: 10 rounds x 2 products x (low, high)

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture of the three-plane step with one launch per stage over the
# three planes (the configuration of the per-kernel table), as of the current
# kernels.
# DRAM bytes per launch (read + write) from one ncu --set full capture of the
# step's kernels (one launch per stage over the three planes; wire
# convolution variant 9 on every plane); see profiles/.
# the raster's share of issue slots in the same capture (it is issue-bound)
NCU_ISSUE_ACTIVE = {"three_planes_800_800_960x6000": 0.688}
NCU_TRAFFIC = {"three_planes_800_800_960x6000": {
    "raster_scatter": 8.39e6, "fwd_rows": 74.5e6, "wire_conv": 94.0e6, "inv_rows": 72.1e6, "memset_grid": 3.12e6}}


def drawing_bins(wiresim, planes, depos) -> int:
    """Bins that draw one Philox block in binomial mode: in-grid bins holding
    N = floor(q w + 1/2) >= 1 electrons, counted on the expected-value
    patches of the same depos."""
    n = 0
    for pl, dd in zip(planes, depos):
        pt = pl.rasterize(dd, wiresim.Params(p_survive=1.0))
        n += int((pt["val"][:pt["capacity"]] >= 0.5).sum().item())
    return n


def algorithmic_flops(kernel: str, nw: int, nt: int, L: int, nfreq: int, kw: int) -> float:
    """FP32 flops a kernel's step needs by the usual count, per launch on one
    plane: 5 L log2 L per complex L-point FFT (two real rows per transform),
    8 per complex multiply-add of the wire-axis sum."""
    import math
    if kernel in ("fwd_rows", "inv_rows"):
        return (nw + 1) // 2 * 5.0 * L * math.log2(L)
    if kernel == "wire_conv":
        return 8.0 * kw * nfreq * nw
    return 0.0


def _time_steps(step, steps, stream, flush):
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def batched_workload_comparison(wiresim, dev, stream, flush, steps: int):
    """64 events x 3 planes with log-uniform depo counts: the batched path
    (one launch per stage per wave, replayed from a CUDA graph; wave size
    picked by timing) against one ws_simulate call per (event, plane)."""
    import torch
    w = inputs.batched_events()
    planes = [wiresim.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id, device=dev) for sp in w.planes]
    events = [[wiresim.DeviceDepos.from_plane_depos(d, device=dev) for d in ev] for ev in w.events]
    params = wiresim.Params(fluctuate=w.fluctuate, p_survive=w.p_survive, seed=w.seed)
    ndp = sum(d.n for ev in w.events for d in ev)
    best = None
    for upw in (3, 6, 12, 16, 24, 32):
        b = wiresim.Batch(planes, events, params, units_per_wave=upw, device=dev)
        b.run(stream)
        torch.cuda.synchronize()
        ms = sum(_time_steps(lambda: b.run(stream), 2, stream, flush)) / 2
        if best is None or ms < best[0]:
            best = (ms, upw, b)
        else:
            del b
    _, upw, b = best
    b.capture()
    b.replay()
    torch.cuda.synchronize()
    graph_ms = _time_steps(b.replay, steps, stream, flush)
    outs = [torch.empty((pl.nwires, pl.nticks), dtype=torch.float32, device=dev) for pl in planes]

    def per_plane():
        for e, ev in enumerate(events):
            pe = wiresim.Params(**{**params.__dict__, "event_id": e})
            for pl, d, o in zip(planes, ev, outs):
                pl.simulate(d, pe, out=o, stream=stream)

    per_plane()
    torch.cuda.synchronize()
    pp_ms = _time_steps(per_plane, steps, stream, flush)
    g = sum(graph_ms) / len(graph_ms)
    pp = sum(pp_ms) / len(pp_ms)
    return {"workload": w.name, "events": len(w.events), "depo_planes": ndp,
            "units_per_wave": upw, "batched_graph_depos_per_s": ndp / (g * 1e-3),
            "per_plane_depos_per_s": ndp / (pp * 1e-3), "speedup": pp / g,
            "batched_ms": g, "per_plane_ms": pp}


def _profiled_once(step, enabled: bool):
    """One more step bracketed by cudaProfilerStart/Stop (for an ncu launch
    list taken with --profile-from-start off)."""
    if not enabled:
        return
    import torch
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    step()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()


def noise_leg(wiresim, dev, stream, flush, steps: int, units_per_wave: int, plain_ms: float,
              profile: bool = False, wire_conv_variant: int = -1):
    """The benchmark event with the noise term of Eq. 1 switched on (an
    incoherent spectrum per wire plus a coherent one per group of 32 wires,
    synthetic shapes), replayed from a CUDA graph like the timed step."""
    import torch
    w = make_workload("three_planes", 0)
    planes = [wiresim.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id, device=dev) for sp in w.planes]
    L = planes[0].info.fft_len_tick
    for pl in planes:
        pl.set_noise(inputs.noise_amplitudes(L), inputs.noise_amplitudes(L, "coherent"), 32)
        if wire_conv_variant >= 0:
            pl.set_wire_conv_variant(wire_conv_variant)
    depos = [wiresim.DeviceDepos.from_plane_depos(d, device=dev) for d in w.events[0]]
    params = wiresim.Params(fluctuate=w.fluctuate, p_survive=w.p_survive, seed=w.seed)
    b = wiresim.Batch(planes, [depos], params, units_per_wave=units_per_wave, device=dev)
    b.capture()
    for _ in range(3):
        b.replay()
    torch.cuda.synchronize(dev)
    ms = sorted(_time_steps(b.replay, steps, stream, flush))[steps // 2]
    _profiled_once(b.replay, profile)
    ndp = sum(d.n for d in w.events[0])
    for pl in planes:
        pl.close()
    return {"workload": w.name + " + noise (incoherent, coherent groups of 32)", "ms_per_step": ms,
            "value": ndp / (ms * 1e-3), "unit": UNIT, "over_plain": ms / plain_ms,
            "where": "noise drawn per (wire, bin) and added to the half spectra between the wire convolution "
                     "and the inverse transform (one more launch per wave)"}


def multinomial_leg(wiresim, dev, stream, flush, steps: int, units_per_wave: int, plain_ms: float,
                    profile: bool = False, wire_conv_variant: int = -1):
    """The benchmark event with the charge-conserving fluctuation
    (fluctuate = 2: binomial survivors per depo, multinomial split over the
    patch), replayed from a CUDA graph like the timed step."""
    import torch
    w = make_workload("three_planes", 0)
    planes = [wiresim.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id, device=dev) for sp in w.planes]
    if wire_conv_variant >= 0:
        for pl in planes:
            pl.set_wire_conv_variant(wire_conv_variant)
    depos = [wiresim.DeviceDepos.from_plane_depos(d, device=dev) for d in w.events[0]]
    params = wiresim.Params(fluctuate=2, p_survive=w.p_survive, seed=w.seed)
    b = wiresim.Batch(planes, [depos], params, units_per_wave=units_per_wave, device=dev)
    b.capture()
    for _ in range(3):
        b.replay()
    torch.cuda.synchronize(dev)
    ms = sorted(_time_steps(b.replay, steps, stream, flush))[steps // 2]
    _profiled_once(b.replay, profile)
    # the raster stage alone, traced
    planes[0].trace(steps * 16 + 16)
    for _ in range(steps):
        flush.zero_()
        b.run(stream)
    torch.cuda.synchronize(dev)
    st = planes[0].trace_read()
    planes[0].trace(0)
    ndp = sum(d.n for d in w.events[0])
    for pl in planes:
        pl.close()
    rn, rms = st.get("raster_scatter", (1, 0.0))
    return {"workload": w.name + ", fluctuate = 2 (charge-conserving multinomial)", "ms_per_step": ms,
            "value": ndp / (ms * 1e-3), "unit": UNIT, "over_plain": ms / plain_ms,
            "raster_ms_per_launch": rms / max(rn, 1)}


def impacts_leg(wiresim, dev, stream, flush, steps: int, impacts: int = 10, profile: bool = False):
    """The benchmark event on planes whose response depends on the charge's
    position inside the pitch (10 sub-pitch positions, synthetic slices):
    the raster bins the pitch axis at pitch/10 and the forward transform
    runs over 10x the rows; one ws_simulate per plane."""
    import torch
    w = make_workload("three_planes", 0)
    kinds = ["bipolar", "bipolar", "unipolar"]
    planes = [wiresim.Plane(sp.nwires, sp.nticks, inputs.impact_response(kinds[i], impacts=impacts),
                            plane_id=sp.plane_id, device=dev) for i, sp in enumerate(w.planes)]
    depos = [wiresim.DeviceDepos.from_plane_depos(d, device=dev) for d in w.events[0]]
    params = wiresim.Params(fluctuate=w.fluctuate, p_survive=w.p_survive, seed=w.seed)
    outs = [torch.empty((sp.nwires, sp.nticks), dtype=torch.float32, device=dev) for sp in w.planes]

    def step():
        for pl, d, o in zip(planes, depos, outs):
            pl.simulate(d, params, out=o, stream=stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    ms = sorted(_time_steps(step, steps, stream, flush))[steps // 2]
    _profiled_once(step, profile)
    for pl in planes:
        pl.trace(16 * steps + 16)
    for _ in range(steps):
        flush.zero_()
        step()
    torch.cuda.synchronize(dev)
    kern = {}
    for pl in planes:
        for name, (n, t) in pl.trace_read().items():
            kern[name] = kern.get(name, 0.0) + t / steps
        pl.trace(0)
        pl.close()
    ndp = sum(d.n for d in w.events[0])
    return {"workload": w.name + f", {impacts} sub-pitch response positions per plane", "ms_per_step": ms,
            "value": ndp / (ms * 1e-3), "unit": UNIT, "kernels_ms_per_step": kern,
            "path": "ws_simulate per plane (fine grid of nwires*10 rows, per-impact wire convolution)"}


def adjoint_leg(wiresim, dev, stream, flush, steps: int):
    """Forward and adjoint (ws_simulate_backward: gradients for q, x, t of
    every depo, D_L, D_T and the response) of one 960 x 6000 plane with
    20,000 depos (t >= 1 us), expected-value mode."""
    import torch
    w = inputs.single_plane(n=20000, seed=1003, t_min_us=1.0)
    sp, d = w.planes[0], w.events[0][0]
    plane = wiresim.Plane(sp.nwires, sp.nticks, sp.response, device=dev)
    dd = wiresim.DeviceDepos.from_plane_depos(d, device=dev)
    params = wiresim.Params()
    out = torch.empty((sp.nwires, sp.nticks), dtype=torch.float32, device=dev)
    g = torch.randn((sp.nwires, sp.nticks), generator=torch.Generator().manual_seed(1003)).to(dev)
    fwd = lambda: plane.simulate(dd, params, out=out, stream=stream)
    bwd = lambda: plane.backward(dd, params, g, want_response=True, stream=stream)
    for _ in range(3):
        fwd()
        bwd()
    torch.cuda.synchronize(dev)
    f_ms = sorted(_time_steps(fwd, steps, stream, flush))[steps // 2]
    b_ms = sorted(_time_steps(bwd, steps, stream, flush))[steps // 2]
    plane.close()
    return {"workload": "single_plane_960x6000, 20000 depos (t >= 1 us), expected value",
            "forward_ms": f_ms, "backward_ms": b_ms, "backward_over_forward": b_ms / f_ms,
            "backward_outputs": "dL/dq, dL/dx, dL/dt per depo; dL/dD_L, dL/dD_T; dL/dR (21 x 200)"}


def run_gpu(args):
    import torch
    from paper_2203_02479_gb300 import wiresim

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = _init_pg(world, "nccl")
    wiresim.load_library()

    w = make_workload(args.workload, rank)
    ev = w.events[0]
    planes = [wiresim.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id, device=dev)
              for sp in w.planes]
    depos = [wiresim.DeviceDepos.from_plane_depos(d, device=dev) for d in ev]
    params = wiresim.Params(fluctuate=w.fluctuate, p_survive=w.p_survive, seed=w.seed, event_id=rank)
    if args.wire_conv_variant >= 0:
        for pl in planes:
            pl.set_wire_conv_variant(args.wire_conv_variant)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    # wave size of the event's batch, picked by timing graph replays: with
    # fewer units per wave than planes, the later waves run on the library's
    # extra streams beside the first (wave k on stream k % 3)
    best = None
    choices = [args.units_per_wave] if args.units_per_wave > 0 else list(range(len(planes), 0, -1))
    for upw in choices:
        cand = wiresim.Batch(planes, [depos], params, units_per_wave=upw, device=dev)
        cand.capture()
        for _ in range(3):
            cand.replay()
        torch.cuda.synchronize(dev)
        t = sorted(_time_steps(cand.replay, 20, torch.cuda.current_stream(dev), flush))[10]
        if best is None or t < best[0]:
            best = (t, upw, cand)
        else:
            del cand
    _, upw_event, batch = best
    outs = [torch.empty((sp.nwires, sp.nticks), dtype=torch.float32, device=dev) for sp in w.planes]
    ndepo_planes = sum(d.n for d in ev)
    stream = torch.cuda.current_stream(dev)

    # one launch per stage over all planes (no concurrent kernels): its
    # traced launches give the per-kernel device times and the roofline
    serial = wiresim.Batch(planes, [depos], params, units_per_wave=len(planes), device=dev)

    def step():
        serial.run(stream)

    def step_per_plane():
        for pl, dd, o in zip(planes, depos, outs):
            pl.simulate(dd, params, out=o, stream=stream)

    for _ in range(max(args.warmup, 0)):
        step()
        step_per_plane()
    torch.cuda.synchronize(dev)

    # the batched path launched kernel by kernel, with the library's launch
    # trace (per-kernel device times for the roofline)
    planes[0].trace(args.steps * 16 + 16)
    stream_ms = _time_steps(step, args.steps, stream, flush)
    stats = planes[0].trace_read()
    planes[0].trace(0)
    # kernels per step of the timed batch (its waves), from the same trace
    planes[0].trace(20 * 32 + 16)
    for _ in range(20):
        batch.run(stream)
    torch.cuda.synchronize(dev)
    per_step_launches = sum(n * (2 if name == "raster_scatter" else 1)
                            for name, (n, _) in planes[0].trace_read().items()) / 20.0
    planes[0].trace(0)

    # the same event one plane at a time
    pp_ms = _time_steps(step_per_plane, args.steps, stream, flush)

    # timed region: the batched step replayed from a CUDA graph (the
    # production path: one graph launch per event)
    batch.capture()
    for _ in range(max(args.warmup, 0)):
        batch.replay()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local) if local == 0 else None
    _barrier(dist)
    torch.cuda.synchronize(dev)
    if args.profile_timed:
        torch.cuda.profiler.start()
    graph_ms = _time_steps(batch.replay, args.steps, stream, flush)
    if args.profile_timed:
        torch.cuda.profiler.stop()
    _barrier(dist)
    clocks = sampler.stop() if sampler else None
    total_ms = _max_over_ranks(dist, float(sum(graph_ms)), dev)
    # the event's waveforms as the timed graph left them, for the error
    # against the oracle (rank 0 at N = 1, beside the CPU baseline)
    check_oracle = world == 1 and not args.no_cpu_baseline
    gpu_out = [o.cpu().numpy() for o in batch.outs] if check_oracle else None

    # per-kernel algorithmic work (sum over the event's planes per launch)
    kern = {name: [n, ms] for name, (n, ms) in stats.items()}
    # each traced raster_scatter entry is two kernels (lane per depo + large-patch)
    launches = int(round(per_step_launches * args.steps))
    per_launch_bytes, per_launch_flops = {}, {}
    for name in kern:
        per_launch_bytes[name] = sum(algorithmic_bytes(name, sp.nwires, sp.nticks, pl.info.nfreq,
                                                       sp.response.shape[0], d.n)
                                     for pl, sp, d in zip(planes, w.planes, ev))
        per_launch_flops[name] = sum(algorithmic_flops(name, sp.nwires, sp.nticks, pl.info.fft_len_tick,
                                                       pl.info.nfreq, sp.response.shape[0])
                                     for pl, sp in zip(planes, w.planes))
    # raster: the Philox multiplies of the binomial draws are its irreducible
    # arithmetic (INT32 multiply pipe)
    per_launch_muls = {name: 0.0 for name in kern}
    if w.fluctuate and 0.0 < w.p_survive < 1.0 and "raster_scatter" in kern:
        per_launch_muls["raster_scatter"] = PHILOX_MULS * float(drawing_bins(wiresim, planes, depos))
    dominant = max(kern, key=lambda k: kern[k][1])
    dn, dms = kern[dominant]
    avg_s = dms / dn * 1e-3
    peak_gbs, sm_max, peak_src = _peaks()
    bw = per_launch_bytes[dominant] / avg_s / 1e9
    fl = per_launch_flops[dominant] / avg_s / 1e12
    im = per_launch_muls[dominant] / avg_s / 1e12
    t_hbm = per_launch_bytes[dominant] / (peak_gbs * 1e9)
    t_alu = per_launch_flops[dominant] / (FP32_PEAK_TFLOPS * 1e12)
    t_int = per_launch_muls[dominant] / (INT_MUL_PEAK_T * 1e12)
    traffic = NCU_TRAFFIC.get(w.name, {}).get(dominant)
    if t_int > max(t_alu, t_hbm):
        roof = {"kernel": dominant, "bound": "alu", "achieved": im, "peak": INT_MUL_PEAK_T,
                "unit": "T int32-mul/s", "frac": im / INT_MUL_PEAK_T, "traffic": traffic,
                "peak_source": "derived: 152 SMs x 64 INT32 multiply lanes x 2.07 GHz "
                               "(a Philox-only loop reaches 19.0, 94%)",
                "work": f"{PHILOX_MULS} multiplies per Philox block x one block per drawing bin "
                        f"({per_launch_muls[dominant] / PHILOX_MULS:.0f} bins)",
                "hbm_frac_of_measured": bw / peak_gbs}
    elif t_alu > t_hbm:
        roof = {"kernel": dominant, "bound": "alu", "achieved": fl, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": fl / FP32_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz",
                "hbm_frac_of_measured": bw / peak_gbs}
    else:
        roof = {"kernel": dominant, "bound": "hbm", "achieved": bw, "peak": peak_gbs, "unit": "GB/s",
                "frac": bw / peak_gbs, "traffic": traffic, "peak_source": f"{peak_src} hbm_gbs",
                "alu_frac_of_derived": fl / FP32_PEAK_TFLOPS}
    kernels = {}
    for name, (n, ms) in sorted(kern.items()):
        a = ms / n * 1e-3
        kernels[name] = {"ms_per_step": ms / args.steps, "launches_per_step": n / args.steps,
                         "hbm_gbs": per_launch_bytes[name] / a / 1e9,
                         "hbm_frac": per_launch_bytes[name] / a / 1e9 / peak_gbs,
                         "fp32_tflops": per_launch_flops[name] / a / 1e12,
                         "fp32_frac": per_launch_flops[name] / a / 1e12 / FP32_PEAK_TFLOPS,
                         "int_mul_frac": per_launch_muls[name] / a / 1e12 / INT_MUL_PEAK_T,
                         "ncu_dram_bytes": NCU_TRAFFIC.get(w.name, {}).get(name)}
    if "raster_scatter" in kernels:
        kernels["raster_scatter"]["ncu_issue_active"] = NCU_ISSUE_ACTIVE.get(w.name)
    if roof["kernel"] == "raster_scatter":
        roof["ncu_issue_active"] = NCU_ISSUE_ACTIVE.get(w.name)
    # the FFT convolution (a5-a7) as a whole: its three kernels' time against
    # the bytes each pass reads and writes, and against the least any
    # convolution must move (the grid in, the waveform out, the response)
    conv_names = [k for k in ("fwd_rows", "wire_conv", "inv_rows") if k in kern]
    convolution = None
    if len(conv_names) == 3:
        c_s = sum(kern[k][1] / kern[k][0] for k in conv_names) * 1e-3
        pass_bytes = sum(per_launch_bytes[k] for k in conv_names)
        min_bytes = sum(8.0 * sp.nwires * sp.nticks + 4.0 * sp.response.size for sp in w.planes)
        convolution = {"kernels": conv_names, "ms_per_step": c_s * 1e3,
                       "pass_bytes": pass_bytes, "hbm_frac_pass_bytes": pass_bytes / c_s / 1e9 / peak_gbs,
                       "min_bytes": min_bytes, "hbm_frac_min_bytes": min_bytes / c_s / 1e9 / peak_gbs,
                       "note": "pass bytes: each of the three passes reads its input and writes its output once "
                               "(about 25 B per grid cell in all); min bytes: the grid in and the waveform out "
                               "(8 B per grid cell) plus the response"}

    # end to end through the public API with host buffers: every step copies
    # its depos in from pinned host memory, replays the event's graph and
    # copies the three waveforms out; two pipelines (own planes, buffers,
    # graph and stream) alternate so that one step's copies overlap the
    # other's kernels
    e2e = None
    two_event = None
    if not args.no_e2e:
        host_in = [[torch.from_numpy(a).pin_memory() for a in (d.q, d.x_mm, d.t_us)] for d in ev]
        h2d = sum(a.numel() * 4 for trip in host_in for a in trip)
        pipes = []
        for _ in range(2):
            pl2 = [wiresim.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id, device=dev)
                   for sp in w.planes]
            dev_in = [[torch.empty_like(a, device=dev) for a in trip] for trip in host_in]
            dd2 = [wiresim.DeviceDepos(*trip, device=dev) for trip in dev_in]
            b2 = wiresim.Batch(pl2, [dd2], params, units_per_wave=upw_event, device=dev)
            b2.capture()
            host_out = [torch.empty((sp.nwires, sp.nticks), dtype=torch.float32).pin_memory() for sp in w.planes]
            pipes.append((pl2, dev_in, b2, host_out, torch.cuda.Stream(dev)))
        d2h = sum(o.numel() * 4 for o in pipes[0][3])

        def e2e_step(j):
            _, dev_in, b2, host_out, st = pipes[j % 2]
            with torch.cuda.stream(st):
                for trip_h, trip_d in zip(host_in, dev_in):
                    for a_h, a_d in zip(trip_h, trip_d):
                        a_d.copy_(a_h, non_blocking=True)
                b2.replay()
                for o, oh in zip(b2.outs, host_out):
                    oh.copy_(o, non_blocking=True)

        # the same two pipelines without the copies: events overlap on the
        # device (one event's raster next to the other's transforms)
        def overlap_step(j):
            _, _, b2, _, st = pipes[j % 2]
            with torch.cuda.stream(st):
                b2.replay()

        for j in range(max(args.warmup, 2)):
            overlap_step(j)
        torch.cuda.synchronize(dev)
        o0 = torch.cuda.Event(enable_timing=True)
        o1 = torch.cuda.Event(enable_timing=True)
        o_steps = max(2, args.steps)
        o0.record(pipes[0][4])
        pipes[1][4].wait_event(o0)
        for j in range(o_steps):
            overlap_step(j)
        pipes[0][4].wait_stream(pipes[1][4])
        o1.record(pipes[0][4])
        torch.cuda.synchronize(dev)
        overlap_ms = o0.elapsed_time(o1) / o_steps

        for j in range(max(args.warmup, 2)):
            e2e_step(j)
        torch.cuda.synchronize(dev)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        e_steps = max(2, args.steps)
        _barrier(dist)
        torch.cuda.synchronize(dev)
        s0.record(pipes[0][4])
        pipes[1][4].wait_event(s0)
        for j in range(e_steps):
            e2e_step(j)
        pipes[0][4].wait_stream(pipes[1][4])
        s1.record(pipes[0][4])
        torch.cuda.synchronize(dev)
        _barrier(dist)
        e_ms = _max_over_ranks(dist, s0.elapsed_time(s1), dev)
        e_total = _sum_over_ranks(dist, float(ndepo_planes * e_steps), dev)
        # the host link's own rate: the step's device-to-host copies alone,
        # back to back (the direction that bounds the pipelined step, whose
        # kernels and host-to-device copies hide behind it)
        def d2h_only():
            _, _, b2, host_out, st = pipes[0]
            with torch.cuda.stream(st):
                for o, oh in zip(b2.outs, host_out):
                    oh.copy_(o, non_blocking=True)

        d2h_only()
        torch.cuda.synchronize(dev)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(pipes[0][4])
        for _ in range(10):
            d2h_only()
        c1.record(pipes[0][4])
        torch.cuda.synchronize(dev)
        copy_ms = c0.elapsed_time(c1) / 10
        e2e = {"value": e_total / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e_ms / e_steps,
               "d2h_alone_ms_per_step": copy_ms,
               "d2h_gbs_measured": d2h / (copy_ms * 1e-3) / 1e9,
               "frac_of_d2h_bound": copy_ms / (e_ms / e_steps),
               "path": "Batch.replay (CUDA graph) per step; pinned host copies in and out on the step's stream; "
                       "two alternating pipelines overlap one step's copies with the other's kernels"}
        two_event = {"ms_per_step": overlap_ms, "value": ndepo_planes / (overlap_ms * 1e-3),
                     "note": "events alternating between two graph pipelines on two streams (two events in "
                             "flight), no host copies, no L2 flush between events (an event's buffers, ~190 MB, "
                             "exceed L2)"}
        for p2 in pipes:
            for pl in p2[0]:
                pl.close()

    all_depos = _sum_over_ranks(dist, float(ndepo_planes * args.steps), dev)
    all_planes = _sum_over_ranks(dist, float(len(planes) * args.steps), dev)
    batched = None
    adjoint = None
    noise = None
    multinomial = None
    impacts = None
    if rank == 0 and world == 1 and not args.no_batched_workload:
        batched = batched_workload_comparison(wiresim, dev, stream, flush, max(3, min(args.steps, 10)))
        adjoint = adjoint_leg(wiresim, dev, stream, flush, max(5, min(args.steps, 50)))
        noise = noise_leg(wiresim, dev, stream, flush, max(5, min(args.steps, 200)), upw_event,
                          sorted(graph_ms)[len(graph_ms) // 2], args.profile_legs, args.wire_conv_variant)
        impacts = impacts_leg(wiresim, dev, stream, flush, max(5, min(args.steps, 50)), profile=args.profile_legs)
        multinomial = multinomial_leg(wiresim, dev, stream, flush, max(5, min(args.steps, 200)), upw_event,
                                      sorted(graph_ms)[len(graph_ms) // 2], args.profile_legs,
                                      args.wire_conv_variant)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    value = all_depos / (total_ms * 1e-3)
    raster_ms = kern.get("raster_scatter", [0, 0.0])[1] + kern.get("memset_grid", [0, 0.0])[1]
    cpu = None
    oracle_error = None
    if check_oracle:
        kept = {}
        done, secs, nplanes = oracle_sample(w, args.cpu_seconds, keep=kept)
        cpu = {"value": done / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nplanes} planes of this event ({done} depo-planes), FP64, single thread"}
        oracle_error = oracle_error_of(gpu_out, kept, w)
    pp = sum(pp_ms) / len(pp_ms)
    sl = sum(stream_ms) / len(stream_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "depos_per_event": ev[0].n, "planes": len(planes),
                   "wires": [sp.nwires for sp in w.planes], "nticks": w.planes[0].nticks,
                   "fluctuate": w.fluctuate, "p_survive": w.p_survive,
                   "seed": w.seed, "event_id": rank,
                   "fft_len_tick": planes[0].info.fft_len_tick,
                   "units_per_wave": upw_event,
                   "wire_conv_variant": [pl.info.wire_conv_variant for pl in planes],
                   "path": "ws_simulate_batch over the event's planes in waves of units_per_wave (wave k on "
                           "stream k % 3), replayed from a CUDA graph",
                   "l2": "flushed between timed steps (512 MiB write)"},
        "planes_per_s": all_planes / (total_ms * 1e-3),
        "raster_scatter_depos_per_s": all_depos / (raster_ms * 1e-3) if raster_ms > 0 else None,
        "per_plane_path": {"ms_per_step": pp, "value": ndepo_planes / (pp * 1e-3)},
        "stream_launch": {"ms_per_step": sl, "value": ndepo_planes / (sl * 1e-3),
                          "note": "one launch per stage over the three planes, launched kernel by kernel "
                                  "(traced: kernels, roofline)"},
        "two_event_overlap": two_event,
        "kernels": kernels,
        "convolution": convolution,
        "roofline": roof,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "oracle_error": oracle_error,
        "gpu": torch.cuda.get_device_name(dev),
        "host_cores": os.cpu_count(),
        "batched_workload": batched,
        "adjoint": adjoint,
        "noise": noise,
        "multinomial": multinomial,
        "impacts": impacts,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="wiresim", choices=["wiresim", "reference"])
    ap.add_argument("--workload", default="three_planes", choices=["three_planes", "single_plane"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched-workload", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--reference-seconds", type=float, default=150.0,
                    help="time budget of the --impl reference timed steps")
    ap.add_argument("--wire-conv-variant", type=int, default=-1,
                    help="force the planes' wire-convolution kernel (default: each plane's autotuned choice)")
    ap.add_argument("--units-per-wave", type=int, default=0,
                    help="force the event's wave size (default: picked by timing)")
    ap.add_argument("--profile-timed", action="store_true",
                    help="bracket the timed graph replays with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--profile-legs", action="store_true",
                    help="bracket one more step of the noise, impact and multinomial legs with "
                         "cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "wiresim":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
