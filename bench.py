#!/usr/bin/env python
"""Masked forward+backward throughput of the differentiable Gaussian-splat step.

Workload (default): one oblique aerial view at 5472x3648 of 40 box buildings
covered by 1.5M flat Gaussians (synthetic stand-in for a GauU-Scene building
group at the original resolution), building mask ~37% of the pixels.  One
step = preprocess -> bin -> masked render -> L1 + boundary-aware normal loss ->
per-tile / per-pixel Gaussian statistics -> render adjoint -> preprocess
adjoint, through the fused autograd Function.  Metric: building-mask pixels
per second (Mpix/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica of the workload (independent
sub-regions; weak scaling); the value is the total over ranks divided by the
slowest rank's time.
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


def _load_json(path):
    with open(path) as f:
        return json.load(f)


ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "masked fwd+bwd Mpix/s @5472x3648, 1.5M Gaussians; % HBM roofline; batched vs plain"
UNIT = "Mpix/s"
WORKLOAD = "aerial view 5472x3648, 1.5M Gaussians on 40 box buildings, building mask ~37%"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", default="16x16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="aerial",
                    choices=["aerial", "aerial-crop2048", "batched", "capacity", "vote", "tsdf", "train"],
                    help="aerial: the 5472x3648 view; aerial-crop2048: its 2048x2048 window with the most "
                         "mask pixels, all 1.5M Gaussians (a smaller case for profiler captures); batched: 8 "
                         "uneven sub-regions (200k-3M Gaussians) x 4 mixed-resolution views, one graph-captured "
                         "persistent step vs 32 sequential per-view steps; capacity: 12 sub-regions, 20M "
                         "Gaussians, 72 views at 6000x4000 with Adam; vote: the multi-view voting filter, 1M "
                         "sparse points against 32 coarse masks at 5472x3648; tsdf: mean fusion of 32 building / "
                         "background depth-map pairs at 2736x1824 and their TSDF integration into 640x640x200 voxels; train: "
                         "group training of the 8 sub-regions (10.5M Gaussians), one view per group per iteration, "
                         "graph-replayed iterations with fused Adam")
    ap.add_argument("--scale", type=float, default=1.0, help="batched workload: fraction of the Gaussians")
    ap.add_argument("--dssim", action="store_true",
                    help="aerial workloads: L_rgb with the masked D-SSIM term (0.8 L1 + 0.2 (1 - SSIM))")
    ap.add_argument("--objective", default="pg", choices=["pg", "eq11"],
                    help="aerial workloads: pg = L_rgb + lambda_4 L_ban (GC-load value only); eq11 = Eq. 11 with "
                         "the flattening loss and the soft-count GC-load, all differentiated")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched workload: use the launch shape the autotuner chose on B300 (16x16 tiles, "
                         "occupancy-deep persistent queue, index order) instead of tuning")
    ap.add_argument("--retune", action="store_true", help="batched workload: ignore the autotune cache")
    ap.add_argument("--ncu-region", default="none", choices=["none", "plain"],
                    help="batched workload: run one more eager plain step between cudaProfilerStart/Stop, for "
                         "ncu --profile-from-start off (a launch list of one plain step)")
    ap.add_argument("--no-batched", action="store_true",
                    help="aerial workload: leave out the batched-vs-plain sub-record (8 sub-regions, 32 views)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- workload

def workload(name="aerial"):
    import pgsag_synth as syn
    g, views, boxes = syn.config1()
    if name == "aerial-crop2048":
        x0, y0 = syn.densest_window(views[0].mask, 2048, 2048, step=256)
        views = [syn.crop_view(views[0], x0, y0, 2048, 2048)]
    return g, views


def cpu_crop_sample(views):
    import pgsag_synth as syn
    v = views[0]
    w = 128
    x0, y0 = syn.densest_window(v.mask, w, w)
    return syn.crop_view(v, x0, y0, w, w), f"{w}x{w} window (densest mask) of the 5472x3648 view, all 1.5M Gaussians projected"


def run_oracle_steps(g, cv, n):
    import torch
    from oracle import pgsag_oracle as O
    times = []
    for _ in range(n):
        t = time.perf_counter()
        O.step(g, cv)
        times.append(time.perf_counter() - t)
    return times, torch.get_num_threads()


# ---------------------------------------------------------------------------- algorithmic bytes

def algorithmic_bytes(plan, K, n_binned):
    """DRAM bytes each stage of this design moves per step (each item read or
    written once by the stage that needs it), from the measured sizes: N
    Gaussians, NP pairs, n_binned binned pairs (one view: also the Gaussians
    with a binned pair), K duplicates, P rendered and M mask pixels, A tiles."""
    N, NP, P, A = plan.n_gauss, plan.n_pairs, plan.n_render, plan.n_active
    M = plan.n_mask
    return {
        # means, scales, quats, opacity 44 B/G; per pair: key 4 + bininfo 16;
        # per binned pair: SH row 192 + rec 64 + tile mask 8 + zeroed grad2d row 64 (read back by the
        # adjoint's atomics)
        "preprocess": 44 * N + 20 * NP + 328 * n_binned,
        # bininfo 16 per pair, tile mask 8 per binned pair; per duplicate: emit (tile, pair) 8, scatter reads 8
        # + writes 4, sort reads 4 + depth key 4 + writes 4; per tile: count 4 + range 8
        "bin": 16 * NP + 8 * n_binned + 32 * K + 12 * A,
        # per pixel: list 4 + out8 32 + depth 4 + aux 16; per duplicate: id 4 + record 64
        "render_fwd": 56 * P + 68 * K,
        # pass A: flags 1 + pixel index 4 + out8 32 + depth 4 + dout8 32 + aux 16 + GC weight 4;
        # on mask pixels target 12 + scratch 24
        "loss": 93 * P + 36 * M,
        "tile_stats": 8 * A,
        # per pixel: list 4 + aux 16 + dout8 32 + depth 4 (Eq. 4 chain; the Eq. 11 objective also reads
        # the 16-byte normal half of out8) + neighbour gather (index 4, scratch 12);
        # per duplicate: id 4 + record 64; grad2d read + write-back 2x64 per binned pair (its zeroing is
        # the projection's, above); the step's gradient buffers cleared on the side, 236 B/G
        "render_bwd": (89 if plan.objective == "eq11" else 73) * P + 68 * K + 128 * n_binned + 236 * N,
        # gradient rows of the Gaussians with a binned pair written, 236 B (the others keep the clear's
        # zeros); bininfo 16/pair; binned: params 236 + grad2d 64
        "preprocess_bwd": 16 * NP + 536 * n_binned,
    }


# FP32 work per (pixel, Gaussian) pair: ~10 FLOP to test alpha >= 1/255 (offset,
# quadratic form); a contributing pair adds ~20 FLOP forward (exp, alpha,
# transmittance, 7 blended channels) and ~90 backward (transmittance recovery,
# the suffix term, d alpha, 13 gradient terms).  FMA counts as 2.
FLOP_TEST, FLOP_FWD_CONTRIB, FLOP_BWD_CONTRIB = 10, 20, 90


def pair_counts(plan):
    """E_eval = sum over active tiles of (rendered pixels x list length): the
    pairs the tile lists put in front of the pixels; E_contrib = sum of n_contrib."""
    import numpy as np
    A = plan.n_active
    rg = plan.ranges[:A].cpu().numpy().astype(np.int64)
    npix = plan.act_tiles[:A, 3].cpu().numpy().astype(np.int64)
    e_eval = int((npix * (rg[:, 1] - rg[:, 0])).sum())
    e_contrib = int(plan.aux[:, 2].sum().item())
    return e_eval, e_contrib


def fp32_peak_tflops(sm_mhz):
    """148 SMs x 128 FP32 lanes x 2 FLOP per FMA x clock (nominal, for context)."""
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12


def measured_alu_peaks():
    """FP32 FMA (scalar and packed f32x2, TFLOP/s) and ex2 (Gop/s) throughput
    measured on this GPU by libpgsag_probe.so; None if the probe is missing."""
    import ctypes
    path = os.path.join(ROOT, "paper_2501_01677_b300", "libpgsag_probe.so")
    if not os.path.exists(path):
        return None
    lib = ctypes.CDLL(path)
    f = lib.pgsag_probe_throughput
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    out = {}
    for kind, name, iters in ((0, "ffma_tflops", 1 << 15), (1, "ffma2_tflops", 1 << 14), (2, "ex2_gops", 1 << 13)):
        r = ctypes.c_double(0.0)
        if f(kind, iters, ctypes.byref(r), None) != 0:
            return None
        out[name] = r.value
    return out


# Compulsory DRAM bytes per unit of work (each item read or written once per
# step): per binned (view, Gaussian) pair 904 B (projection read 236 + write 68,
# binning 24, grad2d zero 52 + read 52, adjoint read 236 + write 236), per
# duplicate 156 B (emit 12, sort 24, range 8, forward gather 56, adjoint gather
# 56), per rendered pixel 165 B (forward 44, loss 77, adjoint 44).
BYTES_PER_PAIR, BYTES_PER_DUP, BYTES_PER_PIXEL = 904, 156, 165
BYTES_GRAD_ROW = 236  # one Gaussian's parameter-gradient row (59 floats)
HBM_NOMINAL_GBS = 7700.0  # B300 HBM3e nominal, for context beside the measured copy bandwidth


def frustum_visible(g, cam) -> int:
    """Gaussians whose centre lies in the view frustum: camera-space z above the
    near plane and the projected centre inside the image."""
    import numpy as np
    m = np.asarray(g.means, np.float64)
    mc = m @ np.asarray(cam.R, np.float64).T + np.asarray(cam.t, np.float64)
    z = mc[:, 2]
    ok = z > cam.znear
    zs = np.where(ok, z, 1.0)
    u = cam.fx * mc[:, 0] / zs + cam.cx
    w = cam.fy * mc[:, 1] / zs + cam.cy
    return int((ok & (u >= 0) & (u < cam.width) & (w >= 0) & (w < cam.height)).sum())


def read_traffic(kernel: str, summary: str = "traffic_aerial_5472x3648.txt"):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if any."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 2 and parts[0] == kernel:
            try:
                return float(parts[1])
            except ValueError:
                return None
    return None


def aggregate(ms_local: float, units_local: float, steps: int, world: int, dist_mod=None, device=None):
    """Whole-job throughput over ranks: the slowest rank's time (max over ranks)
    and the units all ranks processed.  Returns (max ms, value in units / s)."""
    if world > 1 and dist_mod is not None:
        import torch
        t = torch.tensor([ms_local, units_local], dtype=torch.float64, device=device)
        mx = t[:1].clone()
        dist_mod.all_reduce(mx, op=dist_mod.ReduceOp.MAX)
        tot = t[1:].clone()
        dist_mod.all_reduce(tot, op=dist_mod.ReduceOp.SUM)
        ms, units = float(mx.item()), float(tot.item())
    else:
        ms, units = ms_local, units_local
    return ms, units * steps / (ms / 1e3)


def peaks():
    try:
        return _load_json(os.path.join(ROOT, "MEASURED_PEAKS.json")), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0}, "fallback"


# ---------------------------------------------------------------------------- arms

def ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2501_01677_b300 import raster

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    tw, th = (int(x) for x in args.tile.split("x"))
    g, views = workload(args.workload)
    v = views[0]
    P = raster.GaussianParams.from_numpy(g, requires_grad=True)
    plan = raster.Plan([v.cam], [v.mask], [v.target], g.n, tile=(tw, th))
    plan.set_objective(args.objective)
    if args.dssim:
        plan.set_dssim(0.2)

    def step(check=False):
        for t in P.tensors():
            t.grad = None
        loss = raster.render_loss(plan, P, check=check)
        loss.backward()
        return loss

    step(check=True)
    for _ in range(max(args.warmup - 1, 0)):
        step()
    torch.cuda.synchronize()
    plan.check_status()
    K_dup = plan.k_value()
    stream = torch.cuda.current_stream()

    # eager autograd steps with per-stage events (the split; events cost a little).
    # A host slower than the GPU would leave launch gaps between a stage's two
    # events, so the stream is first held by a bounded spin kernel (torch's
    # cycle-count sleep) for longer than the host takes to enqueue the steps.
    n_stage = max(1, min(args.steps, 5))
    host_ms = host_enqueue_ms(step)
    plan.stage_events = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hold_stream(host_ms * n_stage)
    e0.record(stream)
    for _ in range(n_stage):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_eager = e0.elapsed_time(e1) / n_stage
    stage_ms = {}
    for name, a, b in plan.stage_events:
        stage_ms[name] = stage_ms.get(name, 0.0) + a.elapsed_time(b)
    plan.stage_events = None
    stage_ms = {k: v / n_stage for k, v in stage_ms.items()}
    plan.check_status()

    # the same autograd step (forward through the autograd.Function, backward,
    # gradients into .grad) captured once as a CUDA graph: no host work between
    # the kernels.  The timed region replays it.
    for t in P.tensors():
        t.grad = None
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()                                   # warm the side stream
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    for t in P.tensors():
        t.grad = None
    with torch.cuda.graph(graph):
        g_loss = raster.render_loss(plan, P, check=False)
        g_loss.backward()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    plan.check_status()

    # timed region (device time, CUDA events on the launching stream)
    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    plan.check_status()
    mpix = plan.n_mask / 1e6
    # per-step device times of as many further replays (an event pair around
    # each), for the median the measurement protocol quotes
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for ea, eb in ev:
        ea.record(stream)
        graph.replay()
        eb.record(stream)
    torch.cuda.synchronize()
    per_step = sorted(ea.elapsed_time(eb) for ea, eb in ev)
    median_ms = per_step[len(per_step) // 2]
    ms, value = aggregate(ms, mpix, args.steps, ws, dist if ws > 1 else None, device="cuda")

    # end to end through the public API with host buffers: every step uploads its
    # inputs (all Gaussian parameters, from pinned host memory) and reads back its
    # result (the gradients of all parameters and the loss, into pinned host
    # memory).  Two parameter buffers, each with its own captured step, let step
    # i+1's upload (copy-in stream) and step i-1's read-back (copy-out stream) run
    # while step i computes; a buffer's next upload waits for the step that read
    # it, its next step for the read-back of its previous gradients.
    e2e = None
    if not args.no_e2e:
        n_e2e = max(4, args.steps // 2)
        P2 = raster.GaussianParams(*[t.detach().clone().requires_grad_(True) for t in P.tensors()])
        for t in P2.tensors():
            t.grad = None
        side2 = torch.cuda.Stream()
        side2.wait_stream(stream)
        with torch.cuda.stream(side2):
            raster.render_loss(plan, P2, check=False).backward()
        stream.wait_stream(side2)
        torch.cuda.synchronize()
        graph2 = torch.cuda.CUDAGraph()
        for t in P2.tensors():
            t.grad = None
        with torch.cuda.graph(graph2):
            g_loss2 = raster.render_loss(plan, P2, check=False)
            g_loss2.backward()
        bufs = [(P, graph, g_loss), (P2, graph2, g_loss2)]
        host = [t.detach().cpu().pin_memory() for t in P.tensors()]
        host_grads = [[torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in P.tensors()] for _ in range(2)]
        loss_host = torch.empty(n_e2e, dtype=torch.float32, pin_memory=True)
        h2d = sum(t.numel() * t.element_size() for t in host)
        d2h = sum(t.numel() * t.element_size() for t in host_grads[0]) + 4
        copy_in, copy_out = torch.cuda.Stream(), torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        computed = [torch.cuda.Event(), torch.cuda.Event()]
        read_back = [torch.cuda.Event(), torch.cuda.Event()]
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        copy_in.wait_stream(stream)
        copy_out.wait_stream(stream)
        for i in range(n_e2e):
            cur = i & 1
            Pc, gr, lo = bufs[cur]
            with torch.cuda.stream(copy_in):
                if i >= 2:
                    copy_in.wait_event(computed[cur])   # the step that last read this buffer
                with torch.no_grad():
                    for d, h in zip(Pc.tensors(), host):
                        d.copy_(h, non_blocking=True)
                copied[cur].record(copy_in)
            stream.wait_event(copied[cur])
            if i >= 2:
                stream.wait_event(read_back[cur])       # this buffer's previous gradients were read out
            gr.replay()
            computed[cur].record(stream)
            with torch.cuda.stream(copy_out):
                copy_out.wait_event(computed[cur])
                for h, t in zip(host_grads[cur], Pc.tensors()):
                    h.copy_(t.grad, non_blocking=True)
                loss_host[i].copy_(lo.detach(), non_blocking=True)
                read_back[cur].record(copy_out)
        stream.wait_event(read_back[(n_e2e - 1) & 1])
        stream.wait_event(read_back[n_e2e & 1])
        b.record(stream)
        torch.cuda.synchronize()
        plan.check_status()
        assert bool(torch.isfinite(loss_host).all())
        assert all(bool(torch.isfinite(h).all()) for h in host_grads[0] + host_grads[1])
        ms_e2e, v_e2e = aggregate(a.elapsed_time(b), mpix, n_e2e, ws, dist if ws > 1 else None, device="cuda")
        e2e = {"value": v_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "result_read_back": "gradients of all parameters (354 MB) and the loss",
               "overlap": "step i+1's parameter upload and step i-1's gradient read-back run on two copy "
                          "streams during step i",
               "ms_per_step": ms_e2e / n_e2e}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    # roofline of the dominant single-kernel stage
    pk, pk_src = peaks()
    n_binned = int((plan.bininfo[:plan.n_pairs, 3] > 0).sum().item())
    ab = algorithmic_bytes(plan, K_dup, n_binned)
    single = ("preprocess", "render_fwd", "render_bwd", "preprocess_bwd")
    dom = max(single, key=lambda k: stage_ms.get(k, 0.0))
    kernel_name = {"preprocess": "k_preprocess", "render_fwd": "k_render_fwd", "render_bwd": "k_render_bwd",
                   "preprocess_bwd": "k_preprocess_bwd"}[dom]
    traffic = read_traffic(kernel_name)
    e_eval, e_contrib = pair_counts(plan)
    if dom in ("render_fwd", "render_bwd"):
        per = FLOP_FWD_CONTRIB if dom == "render_fwd" else FLOP_BWD_CONTRIB
        flops = FLOP_TEST * e_eval + per * e_contrib
        alu = measured_alu_peaks()
        if alu:
            peak = max(alu["ffma_tflops"], alu["ffma2_tflops"])
            peak_src = "measured in this run: FP32 FMA throughput probe (best of scalar and f32x2)"
        else:
            peak = fp32_peak_tflops(pk.get("sm_max_mhz", 2032.0))
            peak_src = "derived: 148 SMs x 128 FP32 lanes x 2 x max SM clock"
        achieved = flops / (stage_ms[dom] / 1e3) / 1e12
        # special-function unit: an exponential per contributing pair forward, an
        # exponential and a reciprocal backward
        xu_ops = (1 if dom == "render_fwd" else 2) * e_contrib
        xu_gops = xu_ops / (stage_ms[dom] / 1e3) / 1e9
        roofline = {"bound": "alu", "kernel": kernel_name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "peak_source": peak_src, "alu_probe": alu,
                    "xu": {"ops": xu_ops, "achieved_gops": xu_gops,
                           "peak_gops": alu["ex2_gops"] if alu else None,
                           "frac": xu_gops / alu["ex2_gops"] if alu else None},
                    "traffic": traffic, "algorithmic_flops": flops, "pairs_evaluated": e_eval,
                    "pairs_contributing": e_contrib,
                    "hbm_achieved_gbs": ab[dom] / (stage_ms[dom] / 1e3) / 1e9, "algorithmic_bytes": ab[dom]}
    else:
        achieved = ab[dom] / (stage_ms[dom] / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": pk["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "peak_source": pk_src, "traffic": traffic,
                    "algorithmic_bytes": ab[dom]}
    # whole step against HBM: compulsory bytes from the per-unit figures and the
    # measured units.  Two readings of "visible Gaussian" (the per-unit figure's unit): (a)
    # a Gaussian whose centre lies in the view frustum (in front of the near plane,
    # projecting inside the image), counted on the host; (b) a (view, Gaussian)
    # pair the projection bins to at least one active tile (the pairs every later
    # stage touches).  The 904 B of a visible Gaussian include its 236 B gradient
    # write; the API writes every Gaussian's gradient row, so the rows of the
    # others (236 B each, zeros) are a further term, reported separately.
    n_vis = frustum_visible(g, v.cam)
    sec = ms / args.steps / 1e3

    def frac(nbytes):
        return nbytes / sec / 1e9 / pk["hbm_gbs"]

    dup_pix = BYTES_PER_DUP * K_dup + BYTES_PER_PIXEL * plan.n_render
    bytes_vis = BYTES_PER_PAIR * n_vis + dup_pix
    bytes_binned = BYTES_PER_PAIR * n_binned + dup_pix
    grad_rest = BYTES_GRAD_ROW * (g.n - n_vis)
    whole = {"algorithmic_bytes": bytes_vis, "achieved_gbs": bytes_vis / sec / 1e9, "frac": frac(bytes_vis),
             "frac_of_nominal_7700_gbs": bytes_vis / sec / 1e9 / HBM_NOMINAL_GBS,
             "unit_reading": "904 B per Gaussian with its centre in the view frustum",
             "units": {"visible_gaussians": n_vis, "binned_pairs": n_binned, "duplicates": K_dup,
                       "rendered_pixels": plan.n_render, "gaussians": g.n},
             "bytes_per_unit": {"visible_gaussian": BYTES_PER_PAIR, "duplicate": BYTES_PER_DUP,
                                "rendered_pixel": BYTES_PER_PIXEL, "gradient_row": BYTES_GRAD_ROW},
             "binned_pairs_reading": {"algorithmic_bytes": bytes_binned, "frac": frac(bytes_binned)},
             "with_all_gradient_rows": {"algorithmic_bytes": bytes_vis + grad_rest,
                                        "frac": frac(bytes_vis + grad_rest),
                                        "extra_bytes": grad_rest},
             "stage_model_bytes": sum(ab.values()),
             "stage_model_frac": frac(sum(ab.values()))}

    cpu = None
    if not args.no_cpu_baseline and ws == 1 and args.workload == "aerial" and args.objective == "pg" and \
            not args.dssim:
        cv, sample = cpu_crop_sample(views)
        times, cores = run_oracle_steps(g, cv, 2)
        t = min(times)
        cpu = {"value": float(cv.mask.sum()) / 1e6 / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": sample, "s_per_step": t}
        # the same oracle step on one host thread (its single-core figure)
        nt = torch.get_num_threads()
        torch.set_num_threads(1)
        try:
            t1 = min(run_oracle_steps(g, cv, 1)[0])
        finally:
            torch.set_num_threads(nt)
        cpu["single_core"] = {"value": float(cv.mask.sum()) / 1e6 / t1, "s_per_step": t1}

    # batched vs plain (the metric's third clause): the 8-sub-region workload,
    # timed after the headline so that its setup does not touch the timed region
    batched_rec = None
    if not args.no_batched and ws == 1 and args.workload == "aerial" and args.objective == "pg" and not args.dssim:
        graph = graph2 = bufs = None  # release the headline's graph pools first
        torch.cuda.empty_cache()
        batched_rec = batched_summary(run_batched(args, False, args.steps, max(args.warmup, 3)), False)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "median_ms_per_step": median_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == "aerial" else args.workload, "width": v.cam.width, "height": v.cam.height, "n_gaussians": g.n,
                   "mask_pixels": plan.n_mask, "rendered_pixels": plan.n_render, "active_tiles": plan.n_active,
                   "duplicates_K": K_dup, "tile": args.tile, "parallelism": f"replicas x{ws}",
                   "objective": args.objective, "dssim": bool(args.dssim),
                   "l2": "inputs larger than L2 (params 354 MB, per-pixel buffers > 2 GB)"},
        "roofline": roofline, "step_roofline": whole,
        "stages_ms": stage_ms, "eager_ms_per_step": ms_eager, "graph": True,
        "cpu_baseline": cpu, "e2e": e2e, "batched": batched_rec,
        "gpu_launches": plan.kernel_launches_per_step() * args.steps,
        "clocks": ck,
    }
    print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()


# launch shape the autotuner chose for the 8-sub-region workload on B300 (16x16
# tiles, persistent render launches as deep as the occupancy allows, tiles in
# index order); the default bench line uses it without re-tuning
BATCHED_DEFAULT_SHAPE = (16, 16, 0, False)


def run_batched(args, tune: bool, steps: int, warmup: int):
    """Uneven sub-regions in one step (Sec. 4.1 grouping, parallel groups Sec. 5.1):
    plain = one plan per view, run one after the other on one stream (same
    kernels, no graph); batched = one plan over all views with a persistent
    render queue, the whole step replayed as one CUDA graph.  Both use the same
    tile shape and compute identical per-view outputs and summed gradients.
    tune=True runs the autotuner (cached) for the launch shape."""
    import torch
    import pgsag_synth as syn
    from paper_2501_01677_b300 import autotune, raster

    ws, rank, local = dist_env()
    g, ranges, views, owner = syn.config3(scale=args.scale)
    g_ranges = [ranges[o] for o in owner]
    P = raster.GaussianParams.from_numpy(g)
    stream = torch.cuda.current_stream()
    cams, masks, targets = [v.cam for v in views], [v.mask for v in views], [v.target for v in views]
    table, t_tune = None, None
    if tune:
        t0 = time.perf_counter()
        shape, table = autotune.autotune(cams, masks, targets, P, g_ranges, use_cache=not args.retune)
        t_tune = time.perf_counter() - t0
    else:
        shape = autotune.LaunchShape(*BATCHED_DEFAULT_SHAPE)
    tw, th = shape.tile

    def timed(fn, n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    # plain: one plan per view
    plans = []
    for v, view in enumerate(views):
        pl = raster.Plan([view.cam], [view.mask], [view.target], g.n, g_ranges=[g_ranges[v]], tile=(tw, th))
        pl.forward(P)
        plans.append(pl)
    grads_plain = raster.new_param_grads(P)

    def plain_step():
        # each plan covers its sub-region's Gaussian span only: the first view of
        # a sub-region writes the span's gradients, its other views add to them
        seen = set()
        for i, pl in enumerate(plans):
            pl.step(P, grads_plain, accumulate=owner[i] in seen)
            seen.add(owner[i])

    for _ in range(warmup):
        plain_step()
    ms_plain = timed(plain_step, steps)
    for pl in plans:
        pl.check_status()
    # the same per-view launches captured as one CUDA graph: the plain form's GPU
    # cost without the host's launch overhead
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        plain_step()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph_plain = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_plain):
        plain_step()
    for _ in range(warmup):
        graph_plain.replay()
    ms_plain_graph = timed(graph_plain.replay, steps)
    del graph_plain
    for pl in plans:
        pl.check_status()
    # per-stage split of one eager plain step (CUDA events around each stage call)
    host_ms = host_enqueue_ms(plain_step)
    for pl in plans:
        pl.stage_events = []
    hold_stream(host_ms)
    plain_step()
    torch.cuda.synchronize()
    stages_plain = {}
    for pl in plans:
        for name, a, b in pl.stage_events:
            stages_plain[name] = stages_plain.get(name, 0.0) + a.elapsed_time(b)
        pl.stage_events = None
    if getattr(args, "ncu_region", "none") == "plain":
        # one eager plain step between cudaProfilerStart/Stop (ncu --profile-from-start off)
        torch.cuda.profiler.start()
        plain_step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    n_mask = sum(pl.n_mask for pl in plans)
    launches_plain = sum(pl.kernel_launches_per_step() for pl in plans)
    del plans
    torch.cuda.empty_cache()

    # batched: one plan, the launch shape, one graph
    plan = autotune.plan_for(cams, masks, targets, P, shape, g_ranges)
    grads = raster.new_param_grads(P)
    graph = plan.capture(P, grads)
    for _ in range(warmup):
        graph.replay()
    clocks = ClockSampler(local)
    clocks.start()
    ms_batched = timed(graph.replay, steps)
    ck = clocks.stop()
    plan.check_status()
    # per-stage split of one eager batched step
    host_ms = host_enqueue_ms(lambda: plan.step(P, grads))
    plan.stage_events = []
    hold_stream(host_ms)
    plan.step(P, grads)
    torch.cuda.synchronize()
    stages_batched = {}
    for name, a, b in plan.stage_events:
        stages_batched[name] = stages_batched.get(name, 0.0) + a.elapsed_time(b)
    plan.stage_events = None
    plan.check_status()
    assert plan.n_mask == n_mask
    diff = max(float((a - b).abs().max() / (b.abs().max() + 1e-30)) for a, b in zip(grads, grads_plain))
    return {
        "n_gauss": g.n, "views": len(views), "mask_pixels": n_mask, "pairs": plan.n_pairs,
        "duplicates_K": plan.k_value(), "active_tiles": plan.n_active,
        "ms_plain": ms_plain, "ms_batched": ms_batched, "ratio": ms_plain / ms_batched,
        "ms_plain_graph": ms_plain_graph, "ratio_vs_plain_graph": ms_plain_graph / ms_batched,
        "launches_plain": launches_plain, "launches_batched": plan.kernel_launches_per_step(),
        "shape": shape, "table": table, "t_tune": t_tune, "clocks": ck, "grad_diff": diff,
        "stages_plain": stages_plain, "stages_batched": stages_batched,
    }


def host_enqueue_ms(fn) -> float:
    """Host time to enqueue fn()'s GPU work, taken while the stream is held by a
    bounded spin kernel (torch's cycle-count sleep, ~0.3 s) so the GPU cannot
    drain the queue meanwhile."""
    import torch
    torch.cuda.synchronize()
    torch.cuda._sleep(int(0.3 * 2.0e9))
    t = time.perf_counter()
    fn()
    ms = (time.perf_counter() - t) * 1e3
    torch.cuda.synchronize()
    return ms


def hold_stream(host_ms: float):
    """Hold the current stream (bounded cycle-count spin, ~2 GHz clock) for about
    four times the host time needed to enqueue what follows, so per-stage CUDA
    events record GPU time only, not host launch gaps of a slow host."""
    import torch
    torch.cuda._sleep(int((4.0 * host_ms + 5.0) * 2.0e6))


def batched_summary(r, tuned: bool) -> dict:
    sh = r["shape"]
    return {"workload": "8 sub-regions (200k..3M Gaussians, %d total) x 4 views at 1920x1080 / 4000x3000 / "
                        "5472x3648, rectangle masks 20-60%%" % r["n_gauss"],
            "ms": r["ms_batched"], "plain_ms": r["ms_plain"], "ratio": r["ratio"],
            "value": r["mask_pixels"] / 1e6 / (r["ms_batched"] / 1e3),
            "plain_value": r["mask_pixels"] / 1e6 / (r["ms_plain"] / 1e3), "unit": UNIT,
            "mask_pixels": r["mask_pixels"],
            "plain": "32 per-view plans run one after the other on one stream (same kernels, no graph)",
            "plain_graph_ms": r["ms_plain_graph"], "ratio_vs_plain_graph": r["ratio_vs_plain_graph"],
            "plain_graph": "the same 32 per-view plans' launches captured as one CUDA graph (no host overhead)",
            "batched": "one plan over the 32 views, persistent render launches, one CUDA-graph replay",
            "launch_shape": {"tile": f"{sh.tile_w}x{sh.tile_h}", "ctas_per_sm": sh.ctas_per_sm, "lpt": sh.lpt,
                             "source": "autotuned in this run" if tuned else "the autotuner's choice on B300"},
            "gpu_launches_per_step": {"plain": r["launches_plain"], "batched": r["launches_batched"]},
            "eager_stages_ms": {"plain": r["stages_plain"], "batched": r["stages_batched"]},
            "grad_max_rel_diff_batched_vs_plain": r["grad_diff"], "clocks": r["clocks"]}


def batched(args):
    tuned = not args.no_autotune
    r = run_batched(args, tuned, args.steps, args.warmup)
    sh = r["shape"]
    out = {
        "metric": METRIC, "value": r["mask_pixels"] / 1e6 / (r["ms_batched"] / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_batched"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "8 sub-regions (200k..3M Gaussians, %d total) x 4 views at 1920x1080 / "
                               "4000x3000 / 5472x3648, rectangle masks 20-60%%" % r["n_gauss"],
                   "views": r["views"], "mask_pixels": r["mask_pixels"], "pairs": r["pairs"],
                   "duplicates_K": r["duplicates_K"], "active_tiles": r["active_tiles"],
                   "tile": f"{sh.tile_w}x{sh.tile_h}", "scale": args.scale},
        "batched_vs_plain": r["ratio"],
        "batched": batched_summary(r, tuned),
        "autotune": None if r["table"] is None else {
            "chosen": {"tile": f"{sh.tile_w}x{sh.tile_h}", "ctas_per_sm": sh.ctas_per_sm, "lpt": sh.lpt},
            "table_ms": r["table"], "seconds": r["t_tune"]},
        "gpu_launches": r["launches_batched"] * args.steps,
        "clocks": r["clocks"],
    }
    print(json.dumps(out))


def capacity(args):
    """City block at HBM capacity: 12 sub-regions, 20M Gaussians, 6 views each at
    6000x4000, all 72 views in one plan (persistent longest-first render launches,
    whole step as one CUDA graph) followed by the fused Adam update of every
    parameter; reports the step time and the peak device memory."""
    import torch
    import pgsag_synth as syn
    from paper_2501_01677_b300 import raster

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    g, ranges, cams, owner, masks, targets = syn.config4(scale=args.scale)
    t_gen = time.perf_counter() - t0
    g_ranges = [ranges[o] for o in owner]
    tw, th = (int(x) for x in args.tile.split("x"))
    torch.cuda.reset_peak_memory_stats()
    P = raster.GaussianParams.from_numpy(g, requires_grad=False)
    n_gauss = g.n
    del g
    t0 = time.perf_counter()
    plan = raster.Plan(cams, masks, targets, n_gauss, g_ranges=g_ranges, tile=(tw, th))
    plan.release_prep_buffers()
    plan.forward(P)
    t_plan = time.perf_counter() - t0
    plan.use_persistent_schedule(ctas_per_sm=0, lpt=True)
    grads = raster.new_param_grads(P)
    m = [torch.zeros_like(t) for t in P.tensors()]
    v = [torch.zeros_like(t) for t in P.tensors()]
    lrs = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]
    graph = plan.capture(P, grads)
    stream = torch.cuda.current_stream()
    it = [0]

    def one_step():
        graph.replay()
        it[0] += 1
        raster.adam_step(list(P.tensors()), grads, m, v, lrs, it[0])

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    plan.check_status()
    clocks = ClockSampler(local)
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        one_step()
    b.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    plan.check_status()
    ms = a.elapsed_time(b) / args.steps
    free, total = torch.cuda.mem_get_info()
    peak = torch.cuda.max_memory_allocated()
    pb = plan.device_bytes()
    opt = sum(3 * t.numel() * t.element_size() for t in P.tensors())  # grads, m, v
    out = {
        "metric": METRIC, "value": plan.n_mask / 1e6 / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "city block: 12 sub-regions, %d Gaussians, %d views at %dx%d (fx = 1.2 W), "
                               "rectangle masks 20-60%%; fwd + bwd + Adam" % (n_gauss, len(cams), cams[0].width,
                                                                             cams[0].height),
                   "views": len(cams), "mask_pixels": plan.n_mask, "rendered_pixels": plan.n_render,
                   "image_pixels": plan.n_pix, "pairs": plan.n_pairs, "duplicates_K": plan.k_value(),
                   "active_tiles": plan.n_active, "tile": args.tile, "scale": args.scale},
        "memory_gb": {"peak_allocated": peak / 1e9, "budget": 180.0, "device_total": total / 1e9,
                      "device_used_at_end": (total - free) / 1e9,
                      "params": sum(t.numel() * t.element_size() for t in P.tensors()) / 1e9,
                      "grads_adam_state": opt / 1e9, **{k: b_ / 1e9 for k, b_ in pb.items()}},
        "setup_s": {"generate": t_gen, "plan_and_first_forward": t_plan},
        "gpu_launches": (plan.kernel_launches_per_step() + 5) * args.steps,
        "clocks": ck,
    }
    print(json.dumps(out))


VOTE_METRIC = "voting filter Gprojections/s (points x views / s), 1M points x 32 views @5472x3648"
VOTE_UNIT = "Gprojections/s"
# FP32 operations per (point, view) projection, each its own instruction:
# x_c = R x + t (9 mul + 9 add), 1 / z_c, u and v (4 mul + 2 add)
VOTE_FLOP_PER_PROJ = 25


def vote_bytes(M, packed, n_rel):
    """Compulsory DRAM bytes of one vote + compaction: points 12 B, packed masks
    once, counts 4 + 4 and flag 1 B written per point; compaction reads the flags
    twice and writes 4 B per kept point."""
    mask_b = sum(4 * h * w for h, w in zip(packed.heights, packed.words_per_row))
    return {"vote": 12 * M + mask_b + 9 * M, "compact": 2 * M + 4 * n_rel, "masks": mask_b}


def vote_bench(args):
    """The multi-view voting filter (Sec. 4.1, Eq. 5-7): 1M sparse points of the
    40-building scene against 32 coarse masks at 5472x3648 (one vote launch for
    all views + the three compaction launches per step).  Masks are packed once
    before timing (they are fixed, like the render masks).  The inputs (points
    12 MB, packed masks 80 MB) fit in L2, so L2 is flushed between timed steps
    by writing a 256 MB buffer, outside the timed region."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import pgsag_synth as syn
    from paper_2501_01677_b300 import vote

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    w = syn.vote_workload()
    M, V = int(w.points.shape[0]), len(w.cams)
    masks_d = [torch.from_numpy(m).cuda() for m in w.masks]
    packed = vote.pack_masks(masks_d)
    del masks_d
    pts = torch.from_numpy(w.points).cuda()
    out = vote.VoteResult(torch.empty(M, dtype=torch.int32, device="cuda"),
                          torch.empty(M, dtype=torch.int32, device="cuda"),
                          torch.empty(M, dtype=torch.uint8, device="cuda"),
                          torch.zeros(1, dtype=torch.int32, device="cuda"))
    table = vote.vote_views(w.cams, packed)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()
    idx_d = torch.empty(M, dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    cws = vote.compact_workspace(M)

    def step():
        vote.vote_filter(pts, w.cams, packed, w.tau, out=out, table=table)
        return vote.compact(out.reliable)

    for _ in range(args.warmup):
        idx = step()
    torch.cuda.synchronize()
    assert int(out.status.item()) == 0
    n_rel = int(idx.numel())
    # per-kernel time of the vote launch alone and of the whole step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for e in ev:
        flush.zero_()
        e[0].record(stream)
        vote.vote_filter(pts, w.cams, packed, w.tau, out=out, table=table)
        e[1].record(stream)
        vote.compact_async(out.reliable, idx_d, n_out, cws, out.status)
        e[2].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms_step = sum(e[0].elapsed_time(e[2]) for e in ev)
    ms_vote = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
    ms, value = aggregate(ms_step, M * V / 1e9, args.steps, ws, dist if ws > 1 else None, device="cuda")

    # end to end through the public calls: points from pinned host memory, the
    # reliable indices back to the host, every step
    host_pts = w.points.copy()
    hp = torch.from_numpy(host_pts).pin_memory()
    idx_host = torch.empty(M, dtype=torch.int32, pin_memory=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d2h = 0
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        pts.copy_(hp, non_blocking=True)
        vote.vote_filter(pts, w.cams, packed, w.tau, out=out, table=table)
        idx = vote.compact(out.reliable)   # reads the count back (a host sync)
        idx_host[:idx.numel()].copy_(idx, non_blocking=True)
        d2h = 4 * idx.numel() + 4
    b.record(stream)
    torch.cuda.synchronize()
    ms_e2e, v_e2e = aggregate(a.elapsed_time(b), M * V / 1e9, args.steps, ws, dist if ws > 1 else None,
                              device="cuda")
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    pk, pk_src = peaks()
    vb = vote_bytes(M, packed, n_rel)
    alu = measured_alu_peaks()
    ffma = max(alu["ffma_tflops"], alu["ffma2_tflops"]) if alu else fp32_peak_tflops(2032.0)
    flops = VOTE_FLOP_PER_PROJ * M * V
    alu_ach = flops / (ms_vote / 1e3) / 1e12
    alu_peak = ffma / 2  # unfused mul / add: one FLOP per FP32 lane per issue
    hbm_ach = vb["vote"] / (ms_vote / 1e3) / 1e9
    roofline = {"bound": "alu", "kernel": "k_vote", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": alu_ach / alu_peak,
                "peak_source": "half the FP32 FMA throughput measured in this run (separate mul / add, no FMA)",
                "algorithmic_flops": flops, "flop_per_projection": VOTE_FLOP_PER_PROJ,
                "hbm": {"achieved": hbm_ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": hbm_ach / pk["hbm_gbs"],
                        "peak_source": pk_src, "algorithmic_bytes": vb["vote"]},
                "traffic": read_traffic("k_vote", "traffic_vote_1M_32x5472x3648.txt"), "ms_per_launch": ms_vote}
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        from oracle import vote_oracle as VO
        t0 = time.perf_counter()
        VO.vote_filter(w.points, w.cams, w.masks, w.tau)
        t_cpu = time.perf_counter() - t0
        cpu = {"value": M * V / 1e9 / t_cpu, "unit": VOTE_UNIT, "cores": 1, "kind": "oracle",
               "sample": "the full workload (numpy float32, one thread)", "s_per_step": t_cpu}
    res = {
        "metric": VOTE_METRIC, "value": value, "unit": VOTE_UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "voting filter: %d sparse points of the 40-building scene x %d coarse masks at "
                               "%dx%d, tau %d" % (M, V, w.cams[0].width, w.cams[0].height, w.tau),
                   "points": M, "views": V, "tau": w.tau, "reliable": n_rel,
                   "l2": "inputs fit in L2: a 256 MB buffer is written between timed steps"},
        "roofline": roofline, "bytes": vb, "cpu_baseline": cpu,
        "e2e": {"value": v_e2e, "unit": VOTE_UNIT, "h2d_bytes_per_step": 12 * M, "d2h_bytes_per_step": d2h,
                "ms_per_step": ms_e2e / args.steps},
        "gpu_launches": 4 * args.steps, "clocks": ck,
    }
    print(json.dumps(res))
    if ws > 1:
        dist.destroy_process_group()


TSDF_METRIC = "TSDF integration Gvoxel-views/s (voxels x views / s), 640x640x200 voxels x 32 views @2736x1824"
TSDF_UNIT = "Gvoxel-views/s"


def tsdf_bench(args):
    """Depth-map fusion and TSDF integration (Sec. 4.4): per step, one fusion
    launch over the 32 building / background depth-map pairs (2736x1824) and one
    integration launch of the 32 fused maps into a 640x640x200 grid at 0.25 m
    (overwrite).  Inputs (two 640 MB map stacks) and the grids (655 MB) are larger
    than L2."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import pgsag_synth as syn
    from paper_2501_01677_b300 import tsdf as T

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    w = syn.tsdf_workload()
    V = len(w.cams)
    H, W = w.cams[0].height, w.cams[0].width
    npix = H * W
    host_maps = np.stack([np.stack(w.building), np.stack(w.background)]).reshape(2, V * npix)
    maps = torch.from_numpy(host_maps).cuda()
    fused = torch.empty(V * npix, dtype=torch.float32, device="cuda")
    nx, ny, nz = w.dims
    nvox = nx * ny * nz
    tsdf = torch.empty(nz, ny, nx, dtype=torch.float32, device="cuda")
    weight = torch.empty_like(tsdf)
    g = T.grid(w.origin, w.voxel, w.dims, w.trunc)
    offs = [v * npix for v in range(V)]
    table = T.depth_views(w.cams, offs)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        T.fuse(maps, out=fused)
        T.integrate(g, w.cams, fused, offs, tsdf, weight, status=status, table=table)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for e in ev:
        e[0].record(stream)
        T.fuse(maps, out=fused)
        e[1].record(stream)
        T.integrate(g, w.cams, fused, offs, tsdf, weight, status=status, table=table)
        e[2].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms_step = sum(e[0].elapsed_time(e[2]) for e in ev)
    ms_fuse = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
    ms_int = sum(e[1].elapsed_time(e[2]) for e in ev) / args.steps
    ms, value = aggregate(ms_step, nvox * V / 1e9, args.steps, ws, dist if ws > 1 else None, device="cuda")
    # end to end: both map stacks from pinned host memory, the TSDF grid back
    hm = torch.from_numpy(host_maps).pin_memory()
    ht = torch.empty(nz, ny, nx, dtype=torch.float32, pin_memory=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_e2e = min(args.steps, 5)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(n_e2e):
        maps.copy_(hm, non_blocking=True)
        step()
        ht.copy_(tsdf, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    ms_e2e, v_e2e = aggregate(a.elapsed_time(b), nvox * V / 1e9, n_e2e, ws, dist if ws > 1 else None,
                              device="cuda")
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    pk, pk_src = peaks()
    alu = measured_alu_peaks()
    ffma = max(alu["ffma_tflops"], alu["ffma2_tflops"]) if alu else fp32_peak_tflops(2032.0)
    # per (voxel, view): the projection (25 unfused FP32 operations) and the sdf
    # (1 sub, 1 div, 1 min, 1 add); per voxel: the centre (6 ops)
    flops = 29 * nvox * V + 6 * nvox
    alu_ach = flops / (ms_int / 1e3) / 1e12
    bytes_int = 4 * V * npix + 8 * nvox      # fused maps read once, tsdf + weight written
    bytes_fuse = 3 * 4 * V * npix             # two maps read, one written
    hbm_int = bytes_int / (ms_int / 1e3) / 1e9
    hbm_fuse = bytes_fuse / (ms_fuse / 1e3) / 1e9
    roofline = {"bound": "alu", "kernel": "k_tsdf", "achieved": alu_ach, "peak": ffma / 2, "unit": "TFLOP/s",
                "frac": alu_ach / (ffma / 2),
                "peak_source": "half the FP32 FMA throughput measured in this run (separate mul / add, no FMA)",
                "algorithmic_flops": flops, "ms_per_launch": ms_int,
                "hbm": {"achieved": hbm_int, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": hbm_int / pk["hbm_gbs"],
                        "peak_source": pk_src, "algorithmic_bytes": bytes_int},
                "fuse": {"kernel": "k_depth_fuse", "bound": "hbm", "ms_per_launch": ms_fuse, "achieved": hbm_fuse,
                         "peak": pk["hbm_gbs"], "frac": hbm_fuse / pk["hbm_gbs"], "algorithmic_bytes": bytes_fuse},
                "traffic": read_traffic("k_tsdf", "traffic_tsdf_640x640x200.txt")}
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        from oracle import tsdf_oracle as TO
        fused_o = [TO.fuse_mean([bm, gm]).astype(np.float32) for bm, gm in zip(w.building, w.background)]
        idx = np.random.default_rng(0).choice(nvox, 2_000_000, replace=False)
        t0 = time.perf_counter()
        TO.integrate(w.origin, w.voxel, w.dims, w.trunc, w.cams, fused_o, voxel_index=idx)
        t_cpu = time.perf_counter() - t0
        cpu = {"value": len(idx) * V / 1e9 / t_cpu, "unit": TSDF_UNIT, "cores": 1, "kind": "oracle",
               "sample": "2,000,000 random voxels of the grid x all 32 views (numpy, one thread; fusion excluded)",
               "s_per_step": t_cpu}
    res = {
        "metric": TSDF_METRIC, "value": value, "unit": TSDF_UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "depth fusion + TSDF: 32 building / background depth-map pairs at %dx%d of the "
                               "40-building scene, grid %dx%dx%d at %.2f m, truncation %.2f m"
                               % (W, H, nx, ny, nz, w.voxel, w.trunc),
                   "views": V, "voxels": nvox, "l2": "inputs larger than L2 (maps 1.28 GB, grids 655 MB)"},
        "roofline": roofline, "stages_ms": {"fuse": ms_fuse, "integrate": ms_int}, "cpu_baseline": cpu,
        "e2e": {"value": v_e2e, "unit": TSDF_UNIT, "h2d_bytes_per_step": int(host_maps.nbytes),
                "d2h_bytes_per_step": 4 * nvox, "ms_per_step": ms_e2e / n_e2e},
        "gpu_launches": 2 * args.steps, "clocks": ck,
    }
    print(json.dumps(res))
    if ws > 1:
        dist.destroy_process_group()


TRAIN_METRIC = "group training iterations/s (8 sub-regions, 10.5M Gaussians, one view per group per iteration)"


def train_bench(args):
    """Densification-free parallel group training (Sec. 5.1): the 8 sub-regions of
    the batched workload (200k..3M Gaussians, 4 views each at mixed resolutions);
    each iteration renders one view of every group in one batched plan, back-
    propagates and applies the fused multi-tensor Adam to all 10.5M Gaussians;
    the 4 view slots are visited in a random order per epoch, each slot's
    iteration a replayed CUDA graph.  Warm-up covers every slot once (eager run +
    capture)."""
    import numpy as np
    import torch
    import pgsag_synth as syn
    from paper_2501_01677_b300 import raster, train

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    g, ranges, views, owner = syn.config3(scale=args.scale)
    by_group = [[vw for vw, o in zip(views, owner) if o == s_] for s_ in range(len(ranges))]
    P = raster.GaussianParams.from_numpy(g)
    n_gauss = g.n
    del g
    t0 = time.perf_counter()
    tr = train.GroupTrainer(P, by_group, ranges)
    t_setup = time.perf_counter() - t0
    warm = max(args.warmup, tr.n_slots)
    tr.run(warm, seed=1, record_losses=False)
    torch.cuda.synchronize()
    tr.check_status()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    losses = tr.run(args.steps, seed=2)
    b.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    tr.check_status()
    ms = a.elapsed_time(b) / args.steps
    lo = losses.cpu().numpy()
    assert np.isfinite(lo).all()
    # the optimiser alone: 59 floats per Gaussian, read p, g, m, v and write p, m, v
    n_el = sum(t.numel() for t in P.tensors())
    adam_bytes = 28 * n_el
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        tr._adam()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_adam = e0.elapsed_time(e1) / 5
    pk, pk_src = peaks()
    mpix = tr.mask_pixels_per_iteration()
    out = {
        "metric": TRAIN_METRIC, "value": 1e3 / ms, "unit": "iterations/s", "n_gpus": 1, "steps": args.steps,
        "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "8 sub-regions (200k..3M Gaussians, %d total) x 4 views at 1920x1080 / 4000x3000 / "
                               "5472x3648; one view slot (8 views, one per group) per iteration" % n_gauss,
                   "slots": tr.n_slots, "mask_pixels_per_iteration": mpix, "scale": args.scale,
                   "l2": "inputs larger than L2 (parameters and Adam state 2.5 GB)"},
        "mask_mpix_per_s": mpix / 1e6 / (ms / 1e3),
        "roofline": {"bound": "hbm", "kernel": "k_adam_multi", "ms_per_launch": ms_adam,
                     "achieved": adam_bytes / (ms_adam / 1e3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": adam_bytes / (ms_adam / 1e3) / 1e9 / pk["hbm_gbs"], "peak_source": pk_src,
                     "algorithmic_bytes": adam_bytes},
        "loss_first_last": [float(lo[0]), float(lo[-1])],
        "setup_s": t_setup, "gpu_launches": int(round(tr.launches_per_iteration() * args.steps)), "clocks": ck,
    }
    print(json.dumps(out))


def reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    g, views = workload()
    cv, sample = cpu_crop_sample(views)
    run_oracle_steps(g, cv, args.warmup)
    times, cores = run_oracle_steps(g, cv, args.steps)
    t = sum(times)
    value = float(cv.mask.sum()) * args.steps / 1e6 / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference(a)
    elif a.workload == "batched":
        batched(a)
    elif a.workload == "capacity":
        capacity(a)
    elif a.workload == "vote":
        vote_bench(a)
    elif a.workload == "tsdf":
        tsdf_bench(a)
    elif a.workload == "train":
        train_bench(a)
    else:
        ours(a)
