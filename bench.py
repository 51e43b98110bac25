"""Benchmark: pixel-segment pairs per second of the full-sky string ISW map.

Workload (default): Nside=512 RING sky (3,145,728 pixels) and one box of 200,000 light-cone
samples -- 234 Burden loops x 512 nodes (BURDEN light-cone solve) plus 8 random-walk long
strings of 10,024 nodes at box time 0.6 (LINEAR solve) -- seeded synthetic inputs.

One step = the whole hot path on that input, one isw_map_batched call: light-cone solve of
every node, pixel table (RING pix2vec), sample records, the all-pairs map in the FP32-
compensated precision (FP64 near field; kernel variant picked by the library's autotuner in
the warm-up), written as a float64 RING map.  Also reported, outside the timed region: one
step of the plain FP64 path, the batched workload (Nside=1024, 64 shells, graph replay) and
the adjoint workload (Nside=256, 50,176 samples).  Inputs are resident in HBM before the timed
region; L2 (129 MB) is flushed between steps by writing a 256 MiB buffer outside the timed
events.  `e2e` repeats the step through the public Python API with the nodes copied from
pinned host memory and the map copied back every step.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
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

import synth  # noqa: E402

METRIC = "pixel\u00b7segment pairs/s (FP32 vs FP64 GPU) and % FP32 peak, at stated max err"
UNIT = "pairs/s"
FLOPS_PER_PAIR = 36          # algorithmic flops of one Eq. (1)-(2) pair term, FMA = 2
# algorithmic flops of one pair of the adjoint (dL/dX, dL/dXdot: the derivative sums of
# isw_map_adjoint in textbook form, FMA = 2, the two reciprocals not counted)
ADJ_FLOPS_PER_PAIR = 66
FP32_LANES = 128             # FP32 FMA lanes per SM (Blackwell)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp32_peak_tflops(sm_count: int):
    """Dense FP32 peak from unit counts and the maximum SM clock: SMs x 128 lanes x 2 flop x clock."""
    mhz = _peaks().get("sm_max_mhz", 2070.0)
    return sm_count * FP32_LANES * 2 * mhz * 1e6 / 1e12, mhz


def workload_config(w):
    return {
        "workload": f"{w.name}: Nside={w.nside} RING ({w.npix:,} pixels), {w.n:,} light-cone samples "
                    f"(234 Burden loops x 512 + 8 random-walk strings), {w.nshell} shells",
        "nside": w.nside, "npix": w.npix, "samples": w.n, "pairs_per_step": w.npix * w.n,
        "precision": "FP32 pairs, compensated per-pixel sums, FP64 near field",
        "l2": "flushed between steps (256 MiB write outside the timed events)",
        "inputs": "seeded synthetic string network (synth.config(1)) standing in for the paper's simulations",
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def weak_scaling_value(pairs_per_rank_step: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job pairs/s: every rank maps its own network; the slowest rank sets the time."""
    return world * pairs_per_rank_step * steps / (max_ms / 1e3)


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """Largest timed-region duration over all ranks (identity without a process group)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def kernel_sources_sha1() -> str:
    import hashlib

    h = hashlib.sha1()
    for f in ("map.cu", "pipeline.cuh", "isw_internal.cuh", "pack.cu", "api.cu", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_1204_5041_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _profile_record(name: str, pattern: str, variant: int):
    """A machine-readable figure of a committed ncu summary, when it was taken on the current
    kernel sources and the same variant; else None."""
    import re

    try:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    sha = kernel_sources_sha1()
    for val, v, s in re.findall(pattern + r" variant=(-?\d+) csrc_sha1=([0-9a-f]+)", txt):
        if int(v) == variant and s == sha:
            return val
    return None


def profiled_traffic(variant: int):
    """DRAM bytes per step of the pair kernels (ncu launch list of the bench step)."""
    v = _profile_record("launches_nside512_200k_seg.md", r"traffic_bytes_per_step=(\d+)", variant)
    return int(v) if v is not None else None


def profiled_fma_busy(variant: int):
    """FMA-pipe busy fraction of the far-field pass (ncu capture of the bench's samples on a smaller sky)."""
    v = _profile_record("pair_kernel_far_nside128_200k_seg.md", r"fma_pipe_busy=([0-9.]+)", variant)
    return float(v) if v is not None else None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1204_5041_gb300 as isw

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    # weak scaling: every rank maps its own independent string network (seed + rank)
    w = synth.config(1, seed=args.seed + rank)
    if args.nside is not None:
        w.nside = args.nside
    ctx = isw.default_context(local)
    ctx.set_param(isw.PARAM_VARIANT, args.variant)
    ctx.set_param(isw.PARAM_SPLIT, args.split)
    if args.d_far is not None:
        ctx.set_param(isw.PARAM_D_FAR, args.d_far)
    if args.b_min is not None:
        ctx.set_param(isw.PARAM_B_MIN, args.b_min)
    if args.near_k is not None:
        ctx.set_param(isw.PARAM_NEAR_K, args.near_k)
    nodes_h = torch.from_numpy(np.ascontiguousarray(w.nodes)).pin_memory()
    loops_h = torch.from_numpy(np.ascontiguousarray(w.loop_params)).pin_memory()
    loops_d = loops_h.to(dev)
    nodes_d = nodes_h.to(dev)
    theta_d = torch.empty(w.npix, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    flags = isw.AUTOTUNE if args.variant < 0 else 0

    def step(nodes, loops, theta, prec="f32c", fl=flags):
        # light-cone solve of every shell + pixel table + records + pair kernel (+ chunk reduce)
        isw.isw_map_batched(w.nside, nodes, w.shell_off, w.t_box, w.mode, loops, x_obs=w.x_obs, t_obs=w.t_obs,
                            GU=w.GU, prec=prec, flags=fl, out=theta)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(nodes_d, loops_d, theta_d)
    r, counts = ctx.check_status()
    if r != isw.OK:
        raise RuntimeError(f"device status {r} during warm-up: {ctx.last_error()}")

    # ---- timed region: K steps, per-step events, L2 flushed between steps (not timed)
    ctx.set_param(isw.PARAM_TIMING, 1)
    ctx.timing(reset=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    t_wall = time.perf_counter()
    with ClockSampler(local) as clk:
        for e0, e1 in evs:
            flush.fill_(1.0)
            e0.record(stream)
            step(nodes_d, loops_d, theta_d)
            e1.record(stream)
        barrier()
    t_wall = time.perf_counter() - t_wall
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    map_ms, map_launches, all_launches = ctx.timing(reset=True)
    ctx.set_param(isw.PARAM_TIMING, 0)
    variant_used = int(ctx.get_param(isw.PARAM_VARIANT))
    r, counts = ctx.check_status()
    if r != isw.OK:
        raise RuntimeError(f"device status {r} in the timed region: {ctx.last_error()}")
    total_ms = max_over_ranks(float(sum(ms)), dist if ws > 1 else None, dev)
    pairs_step = w.npix * w.n
    value = weak_scaling_value(pairs_step, args.steps, ws, total_ms)

    # ---- end to end through the public API: pinned host inputs in, map out, every step
    theta_h = torch.empty(w.npix, dtype=torch.float64).pin_memory()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(e2e_steps):
        nd = nodes_h.to(dev, non_blocking=True)
        ld = loops_h.to(dev, non_blocking=True)
        step(nd, ld, theta_d)
        theta_h.copy_(theta_d, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_value = ws * pairs_step / (e2e_ms / 1e3)

    def timed(fn):
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        fn()
        a1.record(stream)
        barrier()
        return a0.elapsed_time(a1)

    # ---- plain FP64 GPU path, one step (outside the timed region), for the FP32/FP64 ratio
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    # measured FMA-pipe peaks of this GPU (calibration kernels, outside the timed region)
    fma32 = ctx.fma_rate("f32c") / 1e12
    fma64 = ctx.fma_rate("f64") / 1e12

    def timed_kernel(fn):
        """(event time of fn on the stream, device time of its pair-kernel launches as recorded by the
        library on the launching stream, number of those launches)."""
        ctx.set_param(isw.PARAM_TIMING, 1)
        ctx.timing(reset=True)
        t = timed(fn)
        k_ms, k_n, _ = ctx.timing(reset=True)
        ctx.set_param(isw.PARAM_TIMING, 0)
        return t, k_ms / max(k_n, 1)

    fp64 = None
    theta64 = None
    if not args.skip_fp64:
        theta64 = torch.empty_like(theta_d)
        ms64, k64 = timed_kernel(lambda: step(nodes_d, loops_d, theta64, prec="f64", fl=0))
        ach64 = FLOPS_PER_PAIR * pairs_step / (k64 / 1e3) / 1e12
        fp64 = {"value": pairs_step / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                "roofline": {"bound": "alu", "achieved": ach64, "peak": fma64, "unit": "TFLOP/s",
                             "frac": ach64 / fma64, "frac_kind": "algorithmic (36 flop/pair) of measured",
                             "traffic": None, "kernel": "isw::k_map_f64 (+ chunk reduce)",
                             "kernel_ms": k64, "flops_per_pair": FLOPS_PER_PAIR,
                             "peak_note": "measured: FP64 FMA-chain calibration kernel on every SM "
                                          "(isw_fma_rate), this run"}}

    extra = {}
    if not args.skip_extra and rank == 0:
        # batched workload: Nside=1024, 64 cube shells, graph-captured + autotuned
        w2 = synth.config(2, seed=args.seed)
        n2 = torch.from_numpy(np.ascontiguousarray(w2.nodes)).to(dev)
        l2 = torch.from_numpy(np.ascontiguousarray(w2.loop_params)).to(dev)
        th2 = torch.empty(w2.npix, dtype=torch.float64, device=dev)
        run2 = lambda: isw.isw_map_batched(w2.nside, n2, w2.shell_off, w2.t_box, w2.mode, l2, prec="f32c",
                                           flags=isw.GRAPH | isw.AUTOTUNE, out=th2)
        run2()                                      # autotune + eager run + capture
        ms2 = timed(run2)                           # graph replay
        extra["batched"] = {"workload": f"{w2.name}: Nside={w2.nside}, {w2.nshell} light-cone groups "
                                        f"(64 cube shells), {w2.n:,} samples; one CUDA-graph replay",
                            "value": w2.npix * w2.n / (ms2 / 1e3), "unit": UNIT, "ms": ms2}
        del n2, th2
        # adjoint workload: Nside=256, 98 loops x 512 samples, loss sum (Theta - Theta_t)^2
        w3 = synth.config(3, seed=args.seed)
        n3 = torch.from_numpy(np.ascontiguousarray(w3.nodes)).to(dev)
        l3 = torch.from_numpy(np.ascontiguousarray(w3.loop_params)).to(dev)
        s3 = isw.lightcone_intersect(isw.BURDEN, n3, l3)
        th3 = isw.isw_map(w3.nside, s3, prec="f32c")
        tgt = torch.randn(w3.npix, dtype=torch.float64, device=dev,
                          generator=torch.Generator(device=dev).manual_seed(args.seed + 1)) * th3.std()
        g3 = 2 * (th3 - tgt)
        gout = torch.empty((6, w3.n), dtype=torch.float64, device=dev)
        adj32 = lambda: isw.isw_map_adjoint(w3.nside, s3, g3, prec="f32c", out=gout)
        adj64 = lambda: isw.isw_map_adjoint(w3.nside, s3, g3, prec="f64", out=gout)
        adj32()
        ms3, ka32 = timed_kernel(adj32)
        ms3_64, ka64 = timed_kernel(adj64)
        p3 = w3.npix * w3.n
        peak32, _ = fp32_peak_tflops(sm_count)
        a32 = ADJ_FLOPS_PER_PAIR * p3 / (ka32 / 1e3) / 1e12
        a64 = ADJ_FLOPS_PER_PAIR * p3 / (ka64 / 1e3) / 1e12
        extra["adjoint"] = {"workload": f"{w3.name}: Nside={w3.nside}, {w3.n:,} samples, dL/dX and dL/dXdot",
                            "value": p3 / (ms3 / 1e3), "unit": UNIT, "ms": ms3,
                            "fp64_value": p3 / (ms3_64 / 1e3), "fp64_ms": ms3_64,
                            "roofline": {"bound": "alu", "achieved": a32, "peak": peak32, "unit": "TFLOP/s",
                                         "frac": a32 / peak32, "flops_per_pair": ADJ_FLOPS_PER_PAIR,
                                         "frac_kind": "algorithmic (66 flop/pair) of the derived FP32 peak",
                                         "kernel": "isw::k_adj_f32c (+ chunk reduce)",
                                         "kernel_ms": ka32, "traffic": None},
                            "fp64_roofline": {"bound": "alu", "achieved": a64, "peak": fma64, "unit": "TFLOP/s",
                                              "frac": a64 / fma64, "flops_per_pair": ADJ_FLOPS_PER_PAIR,
                                              "frac_kind": "algorithmic (66 flop/pair) of the measured FP64 peak",
                                              "kernel": "isw::k_adj_f64 (+ chunk reduce)",
                                              "kernel_ms": ka64, "traffic": None}}
        # gradient through the light-cone solve: map adjoint with the dsigma row, then the
        # loop-parameter chain (98 Burden loops)
        tau3 = torch.empty(w3.n, dtype=torch.float64, device=dev)
        s3 = isw.lightcone_intersect(isw.BURDEN, n3, l3, tau=tau3)
        g10 = torch.empty((10, w3.n), dtype=torch.float64, device=dev)
        ms_m10 = timed(lambda: isw.isw_map_adjoint(w3.nside, s3, g3, prec="f32c", ngrad=10, out=g10))
        ms_lc = timed(lambda: isw.lightcone_adjoint(isw.BURDEN, n3, tau3, g10, loop_params=l3))
        extra["adjoint"].update({"lightcone_adjoint_ms": ms_lc, "map_adjoint_10rows_ms": ms_m10,
                                 "note": "lightcone_adjoint chains dL/d(samples) to the 98 loops' parameters"})
        del n3, s3, g3, gout, g10
        # stacking with HEALPix cones: 12 base-pixel cones from 4 boxes used 3 times each
        wst = synth.stack_config(seed=args.seed, nside=512)
        nb = torch.from_numpy(np.ascontiguousarray(wst.nodes_box)).to(dev)
        plc = torch.from_numpy(np.ascontiguousarray(wst.place)).to(dev)
        cpx = torch.from_numpy(wst.cone_pix).to(dev)
        rlo, rhi = torch.from_numpy(wst.r_lo).to(dev), torch.from_numpy(wst.r_hi).to(dev)
        run_st = lambda: isw.isw_map_stacked(wst.nside, nb, wst.box_off, wst.shell_box, plc, wst.t_box, wst.nside_hz,
                                             cpx, rlo, rhi, prec="f32c")
        _, kept = run_st()
        ms_st = timed(run_st)
        extra["stacked"] = {"workload": f"{wst.name}: 12 HEALPix cones (N_side^hz = 1) filled from 4 boxes used 3 "
                                        f"times, {wst.n_placed:,} placed nodes, {kept.shape[1]:,} kept; Nside={wst.nside}",
                            "value": wst.npix * kept.shape[1] / (ms_st / 1e3), "unit": UNIT, "ms": ms_st,
                            "note": "box_place + light-cone solve + cone cut (one host sync) + map; pairs of kept samples"}
        del nb, kept
        # full sky vs flat sky on a 7.2-degree gnomonic patch of the bench network (Fig. 3)
        lin_mean = w.nodes[0:3, w.shell_off[1]:].mean(axis=1)
        e3 = lin_mean / np.linalg.norm(lin_mean)
        e1 = np.cross([0.0, 0.0, 1.0], e3)
        e1 /= np.linalg.norm(e1)
        frame = np.stack([e1, np.cross(e3, e1), e3])
        s1 = torch.empty((10, w.n), dtype=torch.float64, device=dev)
        for k in range(w.nshell):
            a0, a1 = int(w.shell_off[k]), int(w.shell_off[k + 1])
            isw.lightcone_intersect(int(w.mode[k]), nodes_d[:, a0:a1], loops_d, t_box=float(w.t_box[k]),
                                    x_obs=w.x_obs, t_obs=w.t_obs, out=s1[:, a0:a1])
        Mp, wp = 1024, float(np.deg2rad(7.2))
        full = isw.isw_map_patch(frame, Mp, wp, s1, approx=isw.FULLSKY)
        flat = isw.isw_map_patch(frame, Mp, wp, s1, approx=isw.FLATSKY)
        ms_full = timed(lambda: isw.isw_map_patch(frame, Mp, wp, s1, approx=isw.FULLSKY, out=full))
        ms_flat = timed(lambda: isw.isw_map_patch(frame, Mp, wp, s1, approx=isw.FLATSKY, out=flat))
        fh, fl = full.cpu().numpy(), flat.cpu().numpy()
        fh, fl = fh - fh.mean(), fl - fl.mean()
        yy, xx = np.mgrid[0:Mp, 0:Mp]
        rad = np.hypot(xx - (Mp - 1) / 2, yy - (Mp - 1) / 2) / (Mp / 2)
        rms_full = float(np.sqrt(np.mean(fh ** 2)))
        diff = lambda m: float(np.sqrt(np.mean((fh[m] - fl[m]) ** 2)) / rms_full)
        nf = int(s1.shape[1])
        extra["patch"] = {"workload": f"7.2-degree gnomonic patch, {Mp}x{Mp} pixels, {nf:,} samples of {w.name}; "
                                      f"full sky vs flat sky, each map's mean removed for the comparison",
                          "full_value": Mp * Mp * nf / (ms_full / 1e3), "full_ms": ms_full,
                          "flat_value": Mp * Mp * nf / (ms_flat / 1e3), "flat_ms": ms_flat, "unit": UNIT,
                          "rms_full_minus_flat_over_rms": {"centre_r<0.25": diff(rad < 0.25),
                                                           "ring_0.75<r<1": diff((rad > 0.75) & (rad < 1.0)),
                                                           "all": diff(rad >= 0)}}
        del s1, full, flat
        # angular power spectrum of the bench map (Fig. 4): l_max = 3 N_side
        lmax_cl = 3 * w.nside
        cl_t = isw.isw_map_cl(w.nside, theta_d, lmax_cl)
        ms_cl = timed(lambda: isw.isw_map_cl(w.nside, theta_d, lmax_cl))
        clv = cl_t.cpu().numpy()
        # aliasing of centroid sampling (the paper's reading of its high-l excess): the same strings
        # mapped at twice the resolution, whose spectrum over the same l range is not folded
        theta_2 = isw.isw_map_batched(2 * w.nside, nodes_d, w.shell_off, w.t_box, w.mode, loops_d, x_obs=w.x_obs,
                                      t_obs=w.t_obs, GU=w.GU, prec="f32c")
        cl_2 = isw.isw_map_cl(2 * w.nside, theta_2, lmax_cl).cpu().numpy()
        del theta_2
        ls = [l for l in (10, 100, 300, 600, 1000, 1500) if l <= lmax_cl]
        extra["cl"] = {"workload": f"C_l of the {w.name} map, l_max = {lmax_cl} (RING analysis, uniform weights)",
                       "ms": ms_cl,
                       "l(l+1)C_l/2pi": {str(l): float(l * (l + 1) * clv[l] / (2 * np.pi)) for l in ls},
                       "C_l(Nside) / C_l(2 Nside)": {str(l): float(clv[l] / cl_2[l]) for l in ls},
                       "note": "ratio > 1 towards l_max: power of sub-pixel structure folded in by centroid sampling"}
        r, _ = ctx.check_status()
        if r != isw.OK:
            raise RuntimeError(f"device status {r} in the extra measurements: {ctx.last_error()}")

    peak, mhz = fp32_peak_tflops(sm_count)
    map_avg_ms = map_ms / max(map_launches, 1)
    achieved = FLOPS_PER_PAIR * pairs_step / (map_avg_ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "frac_kind": "algorithmic: 36 textbook flops per pair (the far-field form executes ~15 FP32 "
                         "lane operations per pair) of the derived FP32 peak",
            "fma_pipe_busy_far_pass": (profiled_fma_busy(variant_used) if args.nside is None else None),
            "traffic": (profiled_traffic(variant_used) if args.nside is None else None),
            "kernel": f"pair kernels: isw::k_map_f32c (far field) + k_map_f32c_near + chunk reduce, variant {variant_used}",
            "flops_per_pair": FLOPS_PER_PAIR, "kernel_ms": map_avg_ms, "kernel_launches": map_launches,
            "peak_note": f"derived: {sm_count} SMs (device) x {FP32_LANES} FP32 lanes x 2 flop x {mhz:.0f} MHz "
                         f"(max SM clock); measured FP32 FMA calibration kernel: {fma32:.1f} TFLOP/s"}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": workload_config(w),
        "clocks": clk.summary(), "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int((nodes_h.numel() + loops_h.numel()) * 8),
                "d2h_bytes_per_step": int(theta_h.numel() * 8), "ms_per_step": e2e_ms},
        "gpu_launches": int(all_launches),
        "fp64": fp64, "speedup_fp32c_vs_fp64": (value / ws) / fp64["value"] if fp64 else None,
        "measured_fma_peaks": {"fp32_tflops": fma32, "fp64_tflops": fma64, "sm_count": sm_count},
        "counts_per_step": {k: v / args.steps for k, v in counts.items()},
        "wall_s_timed_region": t_wall,
    }
    out.update(extra)
    if rank == 0 and not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline(w, theta_d, theta64, args)
        cb = out["cpu_baseline"]
        # the error the rates are stated at: GPU maps against the oracle on the sampled pixels
        out["max_err"] = {k: cb[k] for k in ("max_err_fp32c_rel_rms", "rms_err_fp32c_rel_rms", "max_err_fp64_rel_rms")
                          if k in cb}
        out["max_err"]["pixels"] = cb.get("sample")
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def _oracle_sample(w, samples, npix_sample, seed=0):
    import oracle

    rng = np.random.default_rng(seed)
    pix = np.sort(rng.choice(w.npix, npix_sample, replace=False)).astype(np.int64)
    threads = os.cpu_count() or 1
    t = time.perf_counter()
    ref, _ = oracle.isw_map(w.nside, samples, pix=pix, x_obs=w.x_obs, GU=w.GU, threads=threads)
    dt = time.perf_counter() - t
    return pix, ref, dt, threads


def cpu_baseline(w, theta32_d, theta64_d, args):
    """The oracle as it stands, on this host's cores, on a bounded pixel sample of the same
    workload (all samples, light-cone solved by the oracle), sized to ~15 s; also the GPU
    maps' error on those pixels."""
    import oracle

    samples, _, _ = oracle.lightcone_workload(w)
    probe = 1024
    _, _, dt, _ = _oracle_sample(w, samples, probe, seed=1)
    npix_sample = int(min(w.npix, max(probe, probe * args.cpu_seconds / max(dt, 1e-3))))
    pix, ref, dt, threads = _oracle_sample(w, samples, npix_sample)
    rms = float(np.sqrt(np.mean(ref ** 2)))
    res = {"value": npix_sample * w.n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{npix_sample} random pixels x all {w.n} samples ({npix_sample * w.n:.3e} pairs, {dt:.1f} s)"}
    g32 = theta32_d.cpu().numpy()[pix]
    res["max_err_fp32c_rel_rms"] = float(np.max(np.abs(g32 - ref)) / rms)
    res["rms_err_fp32c_rel_rms"] = float(np.sqrt(np.mean((g32 - ref) ** 2)) / rms)
    if theta64_d is not None:
        g64 = theta64_d.cpu().numpy()[pix]
        res["max_err_fp64_rel_rms"] = float(np.max(np.abs(g64 - ref)) / rms)
    res["map_rms"] = rms
    return res


def run_reference(args):
    """Reference arm: the oracle (plain single-threaded C per thread) on the host cores."""
    import oracle

    ws, rank, _ = _dist()
    if rank != 0:
        return
    w = synth.config(1, seed=args.seed)
    samples, _, st = oracle.lightcone_workload(w)
    threads = os.cpu_count() or 1
    probe = 32
    _, _, dt, _ = _oracle_sample(w, samples, probe, seed=1)
    per_step = int(max(probe, probe * args.ref_step_seconds / max(dt, 1e-3)))
    for k in range(args.warmup):
        _oracle_sample(w, samples, max(probe, per_step // 8), seed=100 + k)
    t = time.perf_counter()
    tot_pairs = 0
    for k in range(args.steps):
        s, _, _ = oracle.lightcone_workload(w)  # the light-cone solve is part of the step
        _oracle_sample(w, s, per_step, seed=200 + k)
        tot_pairs += per_step * w.n
    dt = time.perf_counter() - t
    value = tot_pairs / dt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(w),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": f"each step: light-cone solve of all nodes + {per_step} random pixels x "
                                      f"all {w.n} samples"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_case(args):
    """One small, self-contained invocation of a single pair kernel, for profiling with ncu (it
    prints one line of timing, not the bench line):
      map_f64       the plain FP64 map of synth.config(0): Nside 64, 10,240 Burden-loop samples
      adjoint_f32c  the FP32-compensated adjoint of synth.config(3) (50,176 samples) at Nside 128
      adjoint_f64   the FP64 adjoint of the same
      map_f32c      the FP32-compensated map of synth.config(1) (200,000 samples) at Nside 128
                    (kernel variant --variant, default the library's first)
    Each runs --warmup untimed calls and then --steps timed ones."""
    import torch

    import paper_1204_5041_gb300 as isw

    dev = torch.device("cuda", 0)
    cfg = {"map_f64": 0, "adjoint_f32c": 3, "adjoint_f64": 3, "map_f32c": 1}[args.case]
    w = synth.config(cfg, seed=args.seed)
    nside = args.nside or {0: 64, 3: 128, 1: 128}[cfg]
    ctx = isw.default_context(0)
    if args.d_far is not None:
        ctx.set_param(isw.PARAM_D_FAR, args.d_far)
    ctx.set_param(isw.PARAM_VARIANT, args.variant)
    nodes = torch.from_numpy(np.ascontiguousarray(w.nodes)).to(dev)
    loops = torch.from_numpy(np.ascontiguousarray(w.loop_params)).to(dev)
    samples = isw.lightcone_intersect_shells(nodes, w.shell_off, w.t_box, w.mode, loops, x_obs=w.x_obs,
                                             t_obs=w.t_obs)
    npix = 12 * nside * nside
    if args.case.startswith("map"):
        prec = args.case[4:]
        out = torch.empty(npix, dtype=torch.float64, device=dev)
        fn = lambda: isw.isw_map(nside, samples, x_obs=w.x_obs, GU=w.GU, prec=prec, out=out)
    else:
        prec = args.case[8:]
        g = torch.randn(npix, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(7))
        out = torch.empty((6, w.n), dtype=torch.float64, device=dev)
        fn = lambda: isw.isw_map_adjoint(nside, samples, g, x_obs=w.x_obs, GU=w.GU, prec=prec, out=out)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    r, counts = ctx.check_status()
    if r != isw.OK:
        raise RuntimeError(f"device status {r}")
    print(f"case {args.case}: Nside={nside} ({npix} pixels) x {w.n} samples = {npix * w.n:.3e} pairs, "
          f"{ms:.3f} ms per call, {npix * w.n / (ms / 1e3):.3e} pairs/s, d_far {ctx.get_param(isw.PARAM_D_FAR)}, "
          f"near pairs per call {counts['near_pairs'] / max(args.warmup + args.steps, 1):.3e}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-extra", action="store_true", help="skip the batched and adjoint sub-measurements")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=6.0)
    ap.add_argument("--variant", type=int, default=-1, help="FP32 pair-kernel variant (-1 = automatic)")
    ap.add_argument("--split", type=int, default=0, help="segment chunks (0 = automatic)")
    ap.add_argument("--d-far", type=float, default=None, help="far-field chord threshold (library default 0.25)")
    ap.add_argument("--b-min", type=float, default=None, help="FP64 routing threshold on 1 + n.Xdot (default 0.01)")
    ap.add_argument("--near-k", type=float, default=None, help="near-field radius factor (default 2)")
    ap.add_argument("--nside", type=int, default=None,
                    help="override the sky resolution (smaller skies for profiling; the bench line uses 512)")
    ap.add_argument("--case", choices=["map_f64", "map_f32c", "adjoint_f32c", "adjoint_f64"], default=None,
                    help="run one small pair-kernel case for profiling instead of the benchmark")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference" and args.case is None:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.case is not None:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
