"""Benchmark of the GB300 augmentation hot path (arXiv 1809.06839).

Headline workload (one step): the per-transform suite -- 2000 uint8 RGB images,
H, W ~ U_int[333, 500], value-noise content; every one of the 15 transforms of
the suite (parameters sampled on the device, then the transform applied to the
whole ragged batch in one plain launch) reads the same resident input and writes
its own output.  value = image-transforms per second (2000 x 15 / step time),
summed over ranks.

The same run also measures, as sub-results: the fused ragged-batch pipeline
(4096 images, H, W ~ U[256, 1024], RandomResizedCrop 224 -> flip -> jitter ->
Normalize bf16 NCHW) in fused and plain modes; the detection targets workload
(256 x 1024^2 images + masks + boxes through ShiftScaleRotate, Resize 512,
HFlip); the differentiable float32 warp + photometric forward/backward
(256 x 3 x 512 x 512).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "images/s per transform & fused ragged-batch pipeline; HBM GB/s vs GB300 peak"
UNIT = "images/s"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per image of a
# transform's kernel, from one ncu --set full capture of 256 images of the
# suite workload (same H, W distribution), scaled per image; the roofline's
# traffic figure is this times the images of one launch.  Only kernels whose
# code is unchanged since that capture are listed.
NCU_DRAM_BYTES_PER_IMAGE = {"Rotate": 1048317.0, "ShiftHSV": 849437.0, "PadToSize512": 1172000.0}
SUITE_N, SUITE_LO, SUITE_HI = 2000, 333, 500
FUSED_N, FUSED_LO, FUSED_HI = 4096, 256, 1024
DET_N, DET_HW = 256, 1024
LARGE_N = 512
DIFF_B, DIFF_HW = 256, 512
SEED = 1809


def suite_table():
    """(name, tid, cfg kwargs) of the 15-transform suite, ranges of the workload."""
    from paper_1809_06839_gb300 import alb as A
    return [
        ("HorizontalFlip", A.HFLIP, dict(p=1.0)),
        ("VerticalFlip", A.VFLIP, dict(p=1.0)),
        ("Rotate", A.ROTATE, dict(lo=(-90.0,), hi=(90.0,))),
        ("ShiftScaleRotate", A.SHIFT_SCALE_ROTATE, dict(lo=(-0.0625, 0.9, -45.0), hi=(0.0625, 1.1, 45.0))),
        ("Brightness", A.BRIGHTNESS, dict(lo=(-20.0,), hi=(20.0,))),
        ("Contrast", A.CONTRAST, dict(lo=(0.8,), hi=(1.2,))),
        ("Gamma", A.GAMMA, dict(lo=(0.8,), hi=(1.2,))),
        ("ShiftRGB", A.SHIFT_RGB, dict(lo=(-20.0,) * 3, hi=(20.0,) * 3)),
        ("ShiftHSV", A.SHIFT_HSV, dict(lo=(-20.0, -30.0, -20.0), hi=(20.0, 30.0, 20.0))),
        ("Grayscale", A.GRAYSCALE, dict(p=1.0)),
        ("RandomCrop64", A.RANDOM_CROP, dict(out_h=64, out_w=64)),
        ("PadToSize512", A.PAD_TO_SIZE, dict(out_h=512, out_w=512)),
        ("Resize512", A.RESIZE, dict(out_h=512, out_w=512)),
        ("RandomSizedCrop512", A.RANDOM_SIZED_CROP, dict(out_h=512, out_w=512, lo=(0.25,), hi=(1.0,))),
        ("Equalize", A.EQUALIZE, dict(p=1.0)),
    ]


# launches per op inside libalb (plan kernel + the op's kernels), for gpu_launches
def launches_per_op(tid):
    from paper_1809_06839_gb300 import alb as A
    if tid in (A.BRIGHTNESS, A.CONTRAST, A.BRIGHTNESS_CONTRAST, A.GAMMA, A.SHIFT_RGB):
        return 1 + 2
    if tid == A.EQUALIZE:
        return 1 + 3          # plan, histogram, tables, apply (the memset is a copy-engine op)
    if tid in (A.RESIZE, A.RANDOM_SIZED_CROP, A.RANDOM_RESIZED_CROP):
        return 1 + 6          # row plan, and a tile plan and a tile kernel per scale class (three)
    if tid in (A.ROTATE, A.SHIFT_SCALE_ROTATE, A.GRID_DISTORTION, A.ELASTIC):
        return 1 + 2          # row plan, tile plan, tile kernel
    return 1 + 1


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        """Start sampling every 50 ms and return once the first sample has
        arrived (at most 3 s), so that the samples cover the timed region that
        follows rather than nvidia-smi's own start-up."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
            return
        t0 = time.time()
        while not self.samples and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.first = list(self.samples)      # taken before the timed region
        self.samples.clear()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        if not self.samples:                 # a region shorter than one interval: the sample just before it
            self.samples = list(getattr(self, "first", []))
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for s in self.samples for j in range(4) if s[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------ helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def ev_time(fn, stream, reps=1):
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(reps):
        fn()
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e) / 1000.0 / reps


class Suite:
    """The per-transform suite on one GPU: resident inputs, per-op params/outputs."""

    def __init__(self, dev, rank=0, n=SUITE_N, only=None, lo=None, hi=None):
        from paper_1809_06839_gb300 import alb as A, synth
        from paper_1809_06839_gb300.ragged import DeviceBatch, output_batch
        self.A = A
        self.dev = dev
        self.n = n
        self.seed = SEED + rank
        self.sizes = synth.uniform_sizes(n, SUITE_LO if lo is None else lo, SUITE_HI if hi is None else hi,
                                         seed=SEED + rank)
        self.inp = DeviceBatch(synth.ragged_noise(self.sizes, seed=SEED + rank, device=dev))
        self.ops = []
        for name, tid, kw in suite_table():
            if only and name not in only:
                continue
            cfg = A.sample_cfg(tid, **kw)
            pdev = torch.zeros(n * 232, dtype=torch.uint8, device=dev)
            A.alb_sample_params_batch(cfg, SEED + rank, tid, 0, n, self.inp.dev, pdev)
            params = A.params_from_device(pdev)
            out = output_batch(params, self.inp.rb.shapes, dev)
            ws = A.workspace(A.alb_workspace_size(tid, n), dev)
            alg = 0
            for p, (h, w, c) in zip(params, self.inp.rb.shapes):
                oh, ow = A.alb_output_shape(p, h, w)
                if tid == A.RANDOM_CROP:
                    alg += 2 * oh * ow * 3
                elif tid == A.RANDOM_SIZED_CROP:
                    alg += p.ch * p.cw * 3 + oh * ow * 3
                else:
                    alg += h * w * 3 + oh * ow * 3
            self.ops.append(dict(name=name, tid=tid, cfg=cfg, pdev=pdev, out=out, ws=ws, alg_bytes=alg))
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()

    def run_op(self, op, stream, sample=True):
        A = self.A
        if sample:
            A.alb_sample_params_batch(op["cfg"], self.seed, op["tid"], 0, self.n, self.inp.dev, op["pdev"],
                                      self.status, stream)
        A.alb_apply_ragged(op["tid"], self.n, op["pdev"], self.inp.dev, op["out"].dev, ws=op["ws"],
                           dev_status=self.status, stream=stream)

    def step(self, stream):
        for op in self.ops:
            self.run_op(op, stream)

    def launches_per_step(self):
        return sum(1 + launches_per_op(op["tid"]) for op in self.ops)


def time_steps(step, stream, steps, warmup, barrier):
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(steps):
        step()
    e.record(stream)
    torch.cuda.synchronize()
    barrier()
    return s.elapsed_time(e) / 1000.0


def per_op_times(suite, stream, reps=5):
    """CUDA-event time of each op's launches (inputs > L2: no flush needed)."""
    res = {}
    for op in suite.ops:
        suite.run_op(op, stream, sample=False)
        t = ev_time(lambda: suite.run_op(op, stream, sample=False), stream, reps)
        res[op["name"]] = t
    return res


def suite_e2e(suite, stream, steps, copy_streams=2):
    """Host->host: pinned host input copied in, all 15 transforms, every output
    copied back to pinned host memory, per step.  Each output's copy to the
    host runs on a side stream (alternating between `copy_streams`) as soon as
    its transform is done, so it overlaps the next transforms; a step ends
    when every copy has landed."""
    A = suite.A
    host_in = torch.empty_like(suite.inp.rb.flat, device="cpu").pin_memory()
    host_in.copy_(suite.inp.rb.flat.cpu())
    host_out = [torch.empty(op["out"].rb.flat.numel(), dtype=torch.uint8).pin_memory() for op in suite.ops]
    bi = host_in.numel()
    bo = sum(h.numel() for h in host_out)
    side = [torch.cuda.Stream(device=suite.dev) for _ in range(copy_streams)]

    def step():
        suite.inp.rb.flat.copy_(host_in, non_blocking=True)
        for k, (op, ho) in enumerate(zip(suite.ops, host_out)):
            suite.run_op(op, stream)
            done = torch.cuda.Event()
            done.record(stream)
            cs = side[k % copy_streams]
            cs.wait_event(done)
            with torch.cuda.stream(cs):
                ho.copy_(op["out"].rb.flat, non_blocking=True)
        for cs in side:                      # the next step rewrites the outputs
            stream.wait_stream(cs)

    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(steps):
        step()
    e.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    t = max(s.elapsed_time(e) / 1000.0, 0.0)
    del A
    return dict(t=t, wall=wall, bi=bi, bo=bo)


_PROFILER_READY = False


def kernel_times(fn, reps=3):
    """Average device time per launch of each kernel that `fn` launches, from
    the profiler's CUDA activity trace (seconds, keyed by kernel name)."""
    from torch.profiler import ProfilerActivity, profile
    fn()
    torch.cuda.synchronize()
    global _PROFILER_READY
    if not _PROFILER_READY:          # the first session of a process records no kernels
        with profile(activities=[ProfilerActivity.CUDA]):
            fn()
            torch.cuda.synchronize()
        _PROFILER_READY = True
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
    out = {}
    for e in prof.key_averages():
        tot = getattr(e, "device_time_total", None)
        if tot is None:
            tot = getattr(e, "cuda_time_total", 0.0)
        if e.count and tot:
            out[e.key] = tot / 1e6 / reps
    return out


# ------------------------------------------------------------------ algorithmic bytes of the chain
def _q5_taps(n_in, n_out):
    """Source samples the half-pixel Q5 resize of n_in -> n_out reads with a
    nonzero weight: ix, and ix + 1 where the fraction is nonzero."""
    d = np.arange(n_out, dtype=np.int64)
    num = 32 * ((2 * d + 1) * n_in - n_out) + n_out
    xq = np.floor_divide(num, 2 * n_out)
    xq = np.maximum(xq, 0)
    xq = np.where((xq >> 5) >= n_in - 1, 32 * (n_in - 1), xq)
    ix, fx = xq >> 5, xq & 31
    return np.unique(np.concatenate([ix, (ix + 1)[fx > 0]]))


def _nearest_taps(n_in, n_out):
    d = np.arange(n_out, dtype=np.int64)
    return np.unique(np.minimum(((2 * d + 1) * n_in) // (2 * n_out), n_in - 1))


def _distinct_sectors(base, stride, rows, byte_cols):
    """Distinct 32-byte sectors of the bytes base + r * stride + b, r in rows
    (sorted), b in byte_cols (sorted): per row the sector set depends only on
    the row start's phase within a sector; consecutive rows can share at most
    their boundary sector (their spans are at most one row apart)."""
    starts = base + rows * stride
    phase = starts & 31
    per_phase = {}
    total = 0
    lo = np.empty(len(rows), np.int64)
    hi = np.empty(len(rows), np.int64)
    for k, (s, ph) in enumerate(zip(starts.tolist(), phase.tolist())):
        sec = per_phase.get(ph)
        if sec is None:
            sec = np.unique((ph + byte_cols) >> 5)
            per_phase[ph] = sec
        total += len(sec)
        lo[k] = (s >> 5) + sec[0]
        hi[k] = (s >> 5) + sec[-1]
    if len(rows) > 1:
        total -= int(np.maximum(hi[:-1] - lo[1:] + 1, 0).sum())
    return total


def chain_read_bytes(params, shapes, offsets, out_h=224, out_w=224, mask_planes=None, mask_offsets=None):
    """Algorithmic read bytes of the chain over the batch: the distinct 32-byte
    sectors holding the source bytes that the crop's bilinear taps (nonzero
    weight) touch, per image (and, with masks, the sectors of the nearest
    taps of every plane)."""
    total = 0
    for i, (p, (h, w, c)) in enumerate(zip(params, shapes)):
        rows = p.y0 + _q5_taps(p.ch, out_h)
        cols = p.x0 + _q5_taps(p.cw, out_w)
        bcols = (3 * cols[:, None] + np.arange(3)[None, :]).ravel()
        total += 32 * _distinct_sectors(int(offsets[i]), 3 * w, rows.astype(np.int64), bcols.astype(np.int64))
        if mask_planes is not None:
            npl = mask_planes[i]
            mr = p.y0 + _nearest_taps(p.ch, out_h)
            mc = p.x0 + _nearest_taps(p.cw, out_w)
            mb = (npl * mc[:, None] + np.arange(npl)[None, :]).ravel()
            total += 32 * _distinct_sectors(int(mask_offsets[i]), npl * w, mr.astype(np.int64), mb.astype(np.int64))
    return total


# ------------------------------------------------------------------ sub-workloads
def fused_pipeline(dev, stream, steps=3, warmup=2, n=FUSED_N, schedule=None):
    from paper_1809_06839_gb300 import alb as A, synth
    from paper_1809_06839_gb300.ragged import DeviceBatch
    FUSED_N = n
    sizes = synth.uniform_sizes(FUSED_N, FUSED_LO, FUSED_HI, seed=SEED)
    din = DeviceBatch(synth.ragged_noise(sizes, seed=SEED, device=dev))
    cfg = A.sample_cfg(A.CHAIN, out_h=224, out_w=224, lo=(0.08, 3 / 4, 0.6), hi=(1.0, 4 / 3, 1.4))
    pdev = torch.zeros(FUSED_N * 232, dtype=torch.uint8, device=dev)
    ccfg = A.chain_cfg()
    out = torch.empty((FUSED_N, 3, 224, 224), dtype=torch.bfloat16, device=dev)
    wsf = A.workspace(A.alb_batch_workspace_size(ccfg, FUSED_N, A.MODE_FUSED), dev)
    wsp = A.workspace(A.alb_batch_workspace_size(ccfg, FUSED_N, A.MODE_PLAIN), dev)
    A.alb_sample_params_batch(cfg, SEED, 20, 0, FUSED_N, din.dev, pdev, stream=stream)
    params = A.params_from_device(pdev)
    # algorithmic bytes: the distinct 32-byte sectors the crops' bilinear taps
    # read, and the bf16 NCHW output written once
    rd = chain_read_bytes(params, din.rb.shapes, din.rb.offsets)
    wr = FUSED_N * 3 * 224 * 224 * 2
    hbm = peaks()[0]

    def run(mode, ws):
        A.alb_sample_params_batch(cfg, SEED, 20, 0, FUSED_N, din.dev, pdev, stream=stream)
        A.alb_apply_batch(ccfg, FUSED_N, pdev, din.dev, out, mode, ws, stream=stream)

    # schedule chosen by the library's autotuner on this batch (outside the
    # timed region); ccfg keeps zero fields, so the fused runs use the cached pick
    if schedule:     # a fixed schedule (profiling runs): no autotuner launches before the measured ones
        ccfg = A.chain_cfg(tile_h=schedule[0], ctas_per_sm=schedule[1])
        res = {"schedule": {"rows_per_item": schedule[0], "ctas_per_sm": schedule[1], "by": "--fused-schedule"}}
    else:
        best = A.alb_autotune_batch(ccfg, FUSED_N, pdev, din.dev, out, wsf, reps=3, stream=stream)
        res = {"schedule": {"rows_per_item": best.tile_h, "ctas_per_sm": best.ctas_per_sm, "by": "alb_autotune_batch"}}
    # the schedule cache persisted to JSON and read back (the next process can
    # start from it with alb_autotune_load)
    cache = os.path.join(ROOT, "paper_1809_06839_gb300", "_build", "autotune.json")
    try:
        A.alb_autotune_save(cache)
        res["autotune_cache"] = {"path": os.path.relpath(cache, ROOT), "entries_reloaded": A.alb_autotune_load(cache)}
    except Exception as ex:  # persistence is reported, not required for the timing
        res["autotune_cache"] = {"error": str(ex)[:160]}
    for name, mode, ws in (("fused", A.MODE_FUSED, wsf), ("plain", A.MODE_PLAIN, wsp)):
        for _ in range(warmup):
            run(mode, ws)
        t = ev_time(lambda: run(mode, ws), stream, steps)
        res[name] = dict(images_per_s=FUSED_N / t, ms=t * 1e3)
    # graph-captured fused step (sampler + memset + table kernel + fused kernel)
    try:
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                A.alb_sample_params_batch(cfg, SEED, 20, 0, FUSED_N, din.dev, pdev, stream=side)
                A.alb_apply_batch(ccfg, FUSED_N, pdev, din.dev, out, A.MODE_FUSED, wsf, stream=side)
        stream.wait_stream(side)
        g.replay()
        t = ev_time(g.replay, stream, steps)
        res["fused_graph"] = dict(images_per_s=FUSED_N / t, ms=t * 1e3)
    except Exception as ex:  # graph capture is an optimisation, not a requirement
        res["fused_graph"] = dict(error=str(ex)[:160])
    tf = res["fused"]["ms"] / 1e3
    res["fused_gbs"] = (rd + wr) / tf / 1e9
    res["roofline"] = {"bound": "hbm", "algorithmic_bytes": rd + wr, "read_bytes": rd, "write_bytes": wr,
                       "achieved": round((rd + wr) / tf / 1e9, 1), "peak": hbm, "unit": "GB/s",
                       "frac": round((rd + wr) / tf / 1e9 / hbm, 4),
                       "read": "distinct 32-byte sectors of the crops' nonzero-weight bilinear taps (exact count)"}
    res["speedup_vs_plain"] = res["plain"]["ms"] / res["fused"]["ms"]
    # the plain path's materialised bytes (each step reads and writes its
    # intermediate: uint8 224^2 x 3 after the resize, the flip and the table,
    # float32 after the saturation, bf16 out) and, per step, its kernel time
    P3 = 3 * 224 * 224
    plain_alg = rd + FUSED_N * (P3 + 2 * P3 + 2 * P3 + (P3 + 4 * P3) + (4 * P3 + 2 * P3))
    tp = res["plain"]["ms"] / 1e3
    res["plain_roofline"] = {"algorithmic_bytes": plain_alg, "achieved": round(plain_alg / tp / 1e9, 1),
                             "frac": round(plain_alg / tp / 1e9 / hbm, 4)}
    steps_bytes = {"k_resize_rows": rd + FUSED_N * P3, "k_pixmap3": FUSED_N * 2 * P3, "k_lut_bulk": FUSED_N * 2 * P3,
                   "k_plain_saturate": FUSED_N * 5 * P3, "k_plain_normalize": FUSED_N * 6 * P3,
                   "k_chain_fused": rd + wr}
    try:
        kt = kernel_times(lambda: run(A.MODE_PLAIN, wsp), reps=3)
        kt.update({k: v for k, v in kernel_times(lambda: run(A.MODE_FUSED, wsf), reps=3).items() if "k_chain_fused" in k})
        tsum = {}
        for name, t in kt.items():   # a step may run as several kernel instantiations: their times add
            base = next((b for b in steps_bytes if b in name), None)
            if base is not None and t > 0:
                tsum[base] = tsum.get(base, 0.0) + t
        step_res = {}
        for base, t in tsum.items():
            step_res[base] = {"ms": round(t * 1e3, 4), "gbs": round(steps_bytes[base] / t / 1e9, 1),
                              "frac": round(steps_bytes[base] / t / 1e9 / hbm, 4)}
        res["steps"] = step_res
    except Exception as ex:  # the per-kernel breakdown needs the profiler's CUDA activity trace
        res["steps"] = {"error": str(ex)[:160]}
    # jitter mode 1: per-image random order and image-mean contrast pivot (a
    # per-image reduction between the ops before contrast and the rest), fused
    # vs plain; the fused path runs one CTA per image with the resized image in
    # shared memory, so the band schedule does not apply
    jcfg = A.chain_cfg(jitter=1)
    wsj = A.workspace(A.alb_batch_workspace_size(jcfg, FUSED_N, A.MODE_PLAIN), dev)
    jres = {"kernel": "k_chain_jitter_img: one CTA per image, the 224x224 image held in shared memory"}
    for name, mode in (("fused", A.MODE_FUSED), ("plain", A.MODE_PLAIN)):
        def runj(mode=mode):
            A.alb_sample_params_batch(cfg, SEED, 20, 0, FUSED_N, din.dev, pdev, stream=stream)
            A.alb_apply_batch(jcfg, FUSED_N, pdev, din.dev, out, mode, wsj, stream=stream)
        runj()
        t = ev_time(runj, stream, steps)
        jres[name] = dict(images_per_s=FUSED_N / t, ms=t * 1e3)
    jres["speedup_vs_plain"] = jres["plain"]["ms"] / jres["fused"]["ms"]
    tj = jres["fused"]["ms"] / 1e3
    # every sampled source sector is read once, the output written once
    jres["roofline"] = {"bound": "hbm", "algorithmic_bytes": rd + wr, "achieved": round((rd + wr) / tj / 1e9, 1),
                        "peak": hbm, "unit": "GB/s", "frac": round((rd + wr) / tj / 1e9 / hbm, 4)}
    res["jitter_random_order_mean_pivot"] = jres
    res["workload"] = "4096 ragged u8 RGB images H,W~U[256,1024] -> RRC 224 + flip + jitter + Normalize bf16 NCHW"
    del din, out, wsf, wsp, wsj
    torch.cuda.empty_cache()
    return res


def fused_detection(dev, stream, steps=3, warmup=2, n=FUSED_N):
    """The fused chain with its targets: the ragged batch of the fused
    pipeline plus a 1-8 plane instance stack and 1-50 boxes per image, box-safe
    crop windows from the device sampler; fused vs plain (images, masks, boxes)."""
    from paper_1809_06839_gb300 import alb as A, synth
    from paper_1809_06839_gb300.ragged import DeviceBatch
    sizes = synth.uniform_sizes(n, FUSED_LO, FUSED_HI, seed=SEED)
    din = DeviceBatch(synth.ragged_noise(sizes, seed=SEED, device=dev))
    planes = [1 + (i * 7) % 8 for i in range(n)]
    mi = DeviceBatch(synth.instance_stacks(sizes, planes, seed=SEED, device=dev))
    mo = DeviceBatch(synth.empty_ragged([(224, 224, c) for c in planes], device=dev))
    cap = 50
    boxes = torch.zeros((n, cap, 4), dtype=torch.float32)
    nb = torch.zeros(n, dtype=torch.int32)
    for i, (h, w) in enumerate(sizes):
        b = torch.from_numpy(synth.random_boxes(h, w, i, SEED)[:cap])
        boxes[i, :len(b)] = b
        nb[i] = len(b)
    bd, nbd = boxes.to(dev), nb.to(dev)
    bo, nbo = torch.zeros_like(bd), torch.zeros_like(nbd)
    cfg = A.sample_cfg(A.CHAIN, out_h=224, out_w=224, lo=(0.08, 3 / 4, 0.6), hi=(1.0, 4 / 3, 1.4))
    pdev = torch.zeros(n * 232, dtype=torch.uint8, device=dev)
    ccfg = A.chain_cfg()
    out = torch.empty((n, 3, 224, 224), dtype=torch.bfloat16, device=dev)
    ws = A.workspace(A.alb_batch_workspace_size(ccfg, n, A.MODE_PLAIN), dev)
    res = {}
    for name, mode in (("fused", A.MODE_FUSED), ("plain", A.MODE_PLAIN)):
        def run(mode=mode):
            A.alb_sample_chain_box_safe_batch(cfg, SEED, 20, 0, n, din.dev, bd, nbd, cap, pdev, stream=stream)
            A.alb_apply_batch_targets(ccfg, n, pdev, din.dev, out, mi.dev, mo.dev, bd, nbd, cap, bo, nbo, mode, ws,
                                      stream=stream)
        for _ in range(warmup):
            run()
        t = ev_time(run, stream, steps)
        res[name] = dict(images_per_s=n / t, ms=t * 1e3)
    res["speedup_vs_plain"] = res["plain"]["ms"] / res["fused"]["ms"]
    params = A.params_from_device(pdev)
    rd = chain_read_bytes(params, din.rb.shapes, din.rb.offsets, mask_planes=planes, mask_offsets=mi.rb.offsets)
    rd += int(nb.sum()) * 16 + 4 * n
    wr = n * 3 * 224 * 224 * 2 + sum(224 * 224 * c for c in planes) + int(nbo.cpu().sum()) * 16 + 4 * n
    hbm = peaks()[0]
    tf = res["fused"]["ms"] / 1e3
    res["roofline"] = {"bound": "hbm", "algorithmic_bytes": rd + wr, "achieved": round((rd + wr) / tf / 1e9, 1),
                       "peak": hbm, "unit": "GB/s", "frac": round((rd + wr) / tf / 1e9 / hbm, 4)}
    res["workload"] = (f"{n} ragged u8 RGB images H,W~U[{FUSED_LO},{FUSED_HI}] + 1-8 instance planes + 1-50 boxes: "
                       "box-safe crop -> 224 + flip + jitter + Normalize bf16 NCHW, masks nearest, boxes mapped")
    del din, mi, mo, out, ws
    torch.cuda.empty_cache()
    return res


def small_plain(dev, stream, hbm, n=64, reps=20):
    """The plain single-op path at small size: 64 images of 256 x 256 + their
    20-class label masks; HFlip -> Brightness/Contrast LUT -> RandomCrop 224
    (masks through the flip and the crop), each step a device-sampled ragged
    launch.  Its 12.6 MB working set fits in L2, so it is timed both hot
    (back to back) and with L2 flushed before every step (a 512 MB write that
    is not timed)."""
    from paper_1809_06839_gb300 import alb as A, synth
    from paper_1809_06839_gb300.ragged import DeviceBatch, mask_output_batch, output_batch
    sizes = [(256, 256)] * n
    img = DeviceBatch(synth.ragged_noise(sizes, seed=SEED, device=dev))
    msk = DeviceBatch(synth.ragged_masks(sizes, seed=SEED, device=dev))
    steps_cfg = [(A.HFLIP, dict(p=1.0), True), (A.BRIGHTNESS_CONTRAST, dict(lo=(0.8, -20.0), hi=(1.2, 20.0)), False),
                 (A.RANDOM_CROP, dict(out_h=224, out_w=224), True)]
    stages, cur, curm, alg = [], img, msk, 0
    for k, (tid, kw, with_mask) in enumerate(steps_cfg):
        cfg = A.sample_cfg(tid, **kw)
        pdev = torch.zeros(n * 232, dtype=torch.uint8, device=dev)
        A.alb_sample_params_batch(cfg, SEED, 100 + k, 0, n, cur.dev, pdev)
        params = A.params_from_device(pdev)
        nxt = output_batch(params, cur.rb.shapes, dev)
        nxtm = mask_output_batch(params, curm.rb.shapes, dev) if with_mask else curm
        ws = A.workspace(A.alb_workspace_size(tid, n), dev)
        stages.append((tid, cfg, pdev, cur, nxt, curm if with_mask else None, nxtm if with_mask else None, ws, k))
        alg += cur.nbytes + nxt.nbytes + ((curm.nbytes + nxtm.nbytes) if with_mask else 0)
        cur, curm = nxt, nxtm

    def step():
        for tid, cfg, pdev, a, b, ma, mb, ws, k in stages:
            A.alb_sample_params_batch(cfg, SEED, 100 + k, 0, n, a.dev, pdev, stream=stream)
            A.alb_apply_ragged(tid, n, pdev, a.dev, b.dev, ma.dev if ma else None, mb.dev if mb else None,
                               ws=ws, stream=stream)

    for _ in range(3):
        step()
    hot = ev_time(step, stream, reps)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    t = 0.0
    for _ in range(reps):
        flush.fill_(1)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        step()
        e.record(stream)
        e.synchronize()
        t += s.elapsed_time(e) / 1000.0
    cold = t / reps
    res = {}
    for name, tt in (("l2_flushed", cold), ("hot", hot)):
        res[name] = dict(images_per_s=round(n / tt, 1), ms=round(tt * 1e3, 4), gbs=round(alg / tt / 1e9, 1),
                         frac=round(alg / tt / 1e9 / hbm, 4))
    res["algorithmic_bytes"] = alg
    res["launches"] = 6
    res["workload"] = ("64 u8 RGB 256x256 + 20-class masks: HFlip -> Brightness/Contrast -> RandomCrop 224 "
                       "(plain path, three ragged launches + their device samplers)")
    del stages, img, msk, flush
    torch.cuda.empty_cache()
    return res


def distortions(dev, stream, hbm, n=SUITE_N):
    """Grid distortion (5 cells per axis, factors 1 +- 0.3) and the elastic
    transform (amplitude 8 px, lattice every 16 px) on the suite's images,
    each one ragged launch, with masks off (images only)."""
    from paper_1809_06839_gb300 import alb as A, synth
    from paper_1809_06839_gb300.ragged import DeviceBatch, output_batch
    sizes = synth.uniform_sizes(n, SUITE_LO, SUITE_HI, seed=SEED)
    inp = DeviceBatch(synth.ragged_noise(sizes, seed=SEED, device=dev))
    res = {}
    for name, tid, lo, hi in (("GridDistortion", A.GRID_DISTORTION, (-0.3, 5), (0.3, 5)),
                              ("ElasticTransform", A.ELASTIC, (8.0, 4), (8.0, 4))):
        cfg = A.sample_cfg(tid, lo=lo, hi=hi)
        pdev = torch.zeros(n * 232, dtype=torch.uint8, device=dev)
        A.alb_sample_params_batch(cfg, SEED, tid, 0, n, inp.dev, pdev)
        params = A.params_from_device(pdev)
        out = output_batch(params, inp.rb.shapes, dev)
        ws = A.workspace(A.alb_workspace_size(tid, n), dev)

        def run():
            A.alb_apply_ragged(tid, n, pdev, inp.dev, out.dev, ws=ws, stream=stream)
        run()
        t = ev_time(run, stream, 5)
        alg = sum(2 * h * w * 3 for h, w in sizes)
        res[name] = dict(images_per_s=round(n / t, 1), ms=round(t * 1e3, 4), gbs=round(alg / t / 1e9, 1),
                         frac=round(alg / t / 1e9 / hbm, 4))
        del out, ws
    res["workload"] = f"{n} u8 RGB images H,W~U[{SUITE_LO},{SUITE_HI}], each distortion alone (one ragged launch)"
    del inp
    torch.cuda.empty_cache()
    return res


def large_suite(dev, stream, hbm, n=LARGE_N, only=None):
    """The same 15 transforms on images of at least 512 x 512 (H, W ~ U[512, 1024]),
    the size class the HBM-fraction target refers to."""
    s = Suite(dev, 0, n=n, only=only, lo=512, hi=1024)
    t = per_op_times(s, stream, reps=5)
    res = {}
    for op in s.ops:
        to = t[op["name"]]
        gbs = op["alg_bytes"] / to / 1e9
        res[op["name"]] = dict(images_per_s=round(n / to, 1), ms=round(to * 1e3, 4), gbs=round(gbs, 1),
                               frac=round(gbs / hbm, 4))
    res["workload"] = f"{n} u8 RGB images H,W~U[512,1024], each transform alone (one ragged launch)"
    del s
    torch.cuda.empty_cache()
    return res


def detection(dev, stream, steps=3, warmup=2):
    from paper_1809_06839_gb300 import alb as A, synth
    from paper_1809_06839_gb300.ragged import DeviceBatch, mask_output_batch, output_batch
    n = DET_N
    sizes = [(DET_HW, DET_HW)] * n
    img = DeviceBatch(synth.ragged_noise(sizes, seed=SEED, device=dev))
    msk = DeviceBatch(synth.ragged_masks(sizes, seed=SEED, device=dev))
    cap = 50
    boxes = np.zeros((n, cap, 4), np.float32)
    nb = np.zeros(n, np.int32)
    for i in range(n):
        b = synth.random_boxes(DET_HW, DET_HW, i, SEED)
        boxes[i, :len(b)] = b
        nb[i] = len(b)
    steps_cfg = [(A.SHIFT_SCALE_ROTATE, dict(lo=(-0.0625, 0.9, -45.0), hi=(0.0625, 1.1, 45.0))),
                 (A.RESIZE, dict(out_h=512, out_w=512)), (A.HFLIP, dict(p=0.5))]
    stages = []
    cur, curm = img, msk
    bcur = torch.from_numpy(boxes).to(dev)
    ncur = torch.from_numpy(nb).to(dev)
    alg = 0
    for k, (tid, kw) in enumerate(steps_cfg):
        cfg = A.sample_cfg(tid, **kw)
        pdev = torch.zeros(n * 232, dtype=torch.uint8, device=dev)
        A.alb_sample_params_batch(cfg, SEED, 300 + k, 0, n, cur.dev, pdev)
        params = A.params_from_device(pdev)
        nxt = output_batch(params, cur.rb.shapes, dev)
        nxtm = mask_output_batch(params, curm.rb.shapes, dev)
        bo, no = torch.zeros_like(bcur), torch.zeros_like(ncur)
        ws = A.workspace(A.alb_workspace_size(tid, n), dev)
        stages.append((tid, cfg, pdev, cur, nxt, curm, nxtm, bcur, ncur, bo, no, ws, k))
        alg += cur.nbytes + nxt.nbytes + curm.nbytes + nxtm.nbytes
        cur, curm, bcur, ncur = nxt, nxtm, bo, no

    def step():
        for tid, cfg, pdev, a, b, ma, mb, bi, ni, bo, no, ws, k in stages:
            A.alb_sample_params_batch(cfg, SEED, 300 + k, 0, n, a.dev, pdev, stream=stream)
            A.alb_apply_ragged(tid, n, pdev, a.dev, b.dev, ma.dev, mb.dev, bi, ni, cap, bo, no, ws, stream=stream)

    for _ in range(warmup):
        step()
    t = ev_time(step, stream, steps)
    res = dict(images_per_s=n / t, ms=t * 1e3, gbs=alg / t / 1e9,
               workload="256 u8 RGB 1024^2 + 20-class masks + 1-50 boxes: SSR -> Resize 512 -> HFlip p=.5")
    del stages, img, msk
    torch.cuda.empty_cache()
    return res


def differentiable(dev, stream, steps=3, warmup=2, n=DIFF_B):
    from paper_1809_06839_gb300 import alb as A
    B, Cc, H, W = n, 3, DIFF_HW, DIFF_HW
    g = torch.Generator(device=dev).manual_seed(SEED)
    x = torch.rand((B, Cc, H, W), device=dev, generator=g)
    gy = torch.randn((B, Cc, H, W), device=dev, generator=g)
    r = np.random.default_rng(SEED)
    wp = torch.tensor(np.stack([r.uniform(-30, 30, B), r.uniform(0.9, 1.1, B), r.uniform(-0.0625, 0.0625, B),
                                r.uniform(-0.0625, 0.0625, B)], 1), dtype=torch.float32, device=dev)
    pp = torch.tensor(np.stack([r.uniform(0.8, 1.2, B), r.uniform(-0.1, 0.1, B), r.uniform(0.8, 1.2, B)], 1),
                      dtype=torch.float32, device=dev)
    w = torch.empty_like(x)
    y = torch.empty_like(x)
    gw = torch.empty_like(x)
    gx = torch.empty_like(x)
    gwp = torch.empty((B, 4), device=dev)
    gpp = torch.empty((B, 3), device=dev)
    ws = A.workspace(A.alb_f32_workspace_size(B, Cc, H, W), dev)

    def fwd():
        A.alb_warp_affine_f32_fwd(x, wp, w, stream=stream)
        A.alb_photometric_f32_fwd(w, pp, y, stream=stream)

    def bwd():
        A.alb_photometric_f32_bwd(w, pp, gy, gw, gpp, ws, stream=stream)
        A.alb_warp_affine_f32_bwd(x, wp, gw, gx, gwp, ws, stream=stream)

    for _ in range(warmup):
        fwd()
        bwd()
    tf = ev_time(fwd, stream, steps)
    tb = ev_time(bwd, stream, steps)
    nb = x.numel() * 4
    res = dict(fwd_images_per_s=B / tf, bwd_images_per_s=B / tb, fwd_ms=tf * 1e3, bwd_ms=tb * 1e3,
               fwd_gbs=4 * nb / tf / 1e9, bwd_gbs=(3 * nb + 3 * nb) / tb / 1e9,
               workload=f"f32 {B}x3x512x512 warp (bilinear, zero border) + photometric, fwd and bwd")
    del x, gy, w, y, gw, gx
    torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------------ CPU oracle
def oracle_suite_sample(n_images, seed=SEED, threads=None, imgs=None):
    """Time the oracle on n_images of the suite workload (all 15 transforms) on
    the host cores; returns (image-transforms/s, threads, images done, seconds).
    `imgs` (host uint8 arrays) may be passed in; otherwise they are generated."""
    import concurrent.futures as cf

    import oracle as O
    from paper_1809_06839_gb300 import synth
    sizes = synth.uniform_sizes(n_images, SUITE_LO, SUITE_HI, seed=seed)
    if imgs is None:
        imgs = [synth.value_noise_image(h, w, i, seed).numpy() for i, (h, w) in enumerate(sizes)]
    table = suite_table()
    cfgs = []
    for name, tid, kw in table:
        c = O.make_cfg(tid, p=kw.get("p", 1.0), out_h=kw.get("out_h", 0), out_w=kw.get("out_w", 0),
                       lo=kw.get("lo", ()), hi=kw.get("hi", ()))
        cfgs.append(c)
    threads = threads or os.cpu_count() or 1

    def work(i):
        h, w = sizes[i]
        for c in cfgs:
            p = O.sample_params(c, seed, c.tid, i, h, w)
            O.apply_image(p, imgs[i])
        return i

    O.lib()
    t0 = time.perf_counter()
    done = 0
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = [ex.submit(work, i) for i in range(n_images)]
        for f in cf.as_completed(futs):
            f.result()
            done += 1
    dt = time.perf_counter() - t0
    return done * len(cfgs) / dt, threads, done, dt


def summary(extra):
    """Headline figures of the sub-workloads, last in the JSON line so that a
    reader of the output's tail sees them."""
    out = {}
    fp = extra.get("fused_pipeline")
    if fp:
        out["fused_pipeline"] = {"fused_images_per_s": round(fp["fused"]["images_per_s"]),
                                 "plain_images_per_s": round(fp["plain"]["images_per_s"]),
                                 "speedup_vs_plain": round(fp["speedup_vs_plain"], 2),
                                 "fused_frac": fp["roofline"]["frac"], "fused_gbs": fp["roofline"]["achieved"]}
        j = fp.get("jitter_random_order_mean_pivot")
        if j:
            out["jitter_mode1"] = {"fused_images_per_s": round(j["fused"]["images_per_s"]),
                                   "speedup_vs_plain": round(j["speedup_vs_plain"], 2),
                                   "fused_frac": j["roofline"]["frac"]}
    fd = extra.get("fused_detection")
    if fd:
        out["fused_detection"] = {"fused_images_per_s": round(fd["fused"]["images_per_s"]),
                                  "speedup_vs_plain": round(fd["speedup_vs_plain"], 2),
                                  "fused_frac": fd["roofline"]["frac"]}
    if extra.get("detection"):
        out["detection_images_per_s"] = round(extra["detection"]["images_per_s"])
    d = extra.get("differentiable")
    if d:
        out["differentiable"] = {"fwd_ms": round(d["fwd_ms"], 3), "bwd_ms": round(d["bwd_ms"], 3)}
    sp = extra.get("small_plain")
    if sp:
        out["small_plain"] = {k: sp[k]["images_per_s"] for k in ("l2_flushed", "hot")}
    lg = extra.get("per_transform_large")
    if lg:
        out["large_frac"] = {k: v["frac"] for k, v in lg.items() if isinstance(v, dict)}
    return out


# ------------------------------------------------------------------ main
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if (torch.cuda.is_available() and args.impl != "reference") else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        return ws, rank, local, dist
    return 1, 0, 0, None


def reference_arm(args, ws, rank, dist):
    if rank != 0:
        return
    n_img = max(4, args.ref_images)
    vals = []
    thr = None
    for _ in range(args.warmup if args.warmup < 2 else 1):
        oracle_suite_sample(4)
    t_all = 0.0
    for _ in range(args.steps):
        v, thr, done, dt = oracle_suite_sample(n_img)
        vals.append(v)
        t_all += dt
    value = float(np.median(vals))
    sample = f"{n_img} images of the suite workload x 15 transforms per step (H,W~U[333,500])"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_all / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "per-transform suite: 2000 u8 RGB images H,W~U[333,500], 15 transforms",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="alb", choices=["alb", "reference"])
    ap.add_argument("--ref-images", type=int, default=400)
    ap.add_argument("--skip-extra", action="store_true", help="headline suite only")
    ap.add_argument("--cpu-images", type=int, default=2000)
    ap.add_argument("--cpu-images-1core", type=int, default=120)
    ap.add_argument("--only", default="", help="comma-separated suite transforms (profiling runs)")
    ap.add_argument("--n", type=int, default=SUITE_N, help="suite images (profiling runs)")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--extras", default="fused,detection,differentiable,large,distort,targets,small",
                    help="sub-workloads to run after the suite (comma-separated)")
    ap.add_argument("--fused-n", type=int, default=FUSED_N, help="images of the fused workload (profiling runs)")
    ap.add_argument("--diff-b", type=int, default=DIFF_B, help="batch of the differentiable workload (profiling runs)")
    ap.add_argument("--large-n", type=int, default=LARGE_N, help="images of the 512-1024 px leg (profiling runs)")
    ap.add_argument("--fused-schedule", default="", help="rows per item,CTAs per SM of the fused kernel instead of "
                    "the autotuner's pick (profiling runs)")
    args = ap.parse_args()
    ws, rank, local, dist = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, ws, rank, dist)
        return
    from paper_1809_06839_gb300 import alb as A
    from paper_1809_06839_gb300.replicas import max_over_ranks
    A.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    suite = Suite(dev, rank, n=args.n, only=set(args.only.split(",")) if args.only else None)
    hbm, peak_kind = peaks()
    clk = ClockSampler(local)
    clk.start()
    t = time_steps(lambda: suite.step(stream), stream, args.steps, args.warmup, barrier)
    clocks = clk.stop()
    t = max_over_ranks(t, dist, dev)          # the slowest rank's time (replicas: no data exchange)
    per_step = t / args.steps
    value = ws * suite.n * len(suite.ops) / per_step
    ops_t = per_op_times(suite, stream)
    per_transform = {}
    for op in suite.ops:
        to = ops_t[op["name"]]
        gbs = op["alg_bytes"] / to / 1e9
        per_transform[op["name"]] = dict(images_per_s=round(suite.n / to, 1), ms=round(to * 1e3, 4),
                                         gbs=round(gbs, 1), frac=round(gbs / hbm, 4))
    dom = max(suite.ops, key=lambda o: ops_t[o["name"]])
    achieved = dom["alg_bytes"] / ops_t[dom["name"]] / 1e9
    traffic = NCU_DRAM_BYTES_PER_IMAGE.get(dom["name"])
    traffic = None if traffic is None else round(traffic * suite.n)
    status = int(suite.status.item())
    host_images = [suite.inp.rb.image(i).cpu().numpy() for i in range(min(args.cpu_images, suite.n))]
    if args.skip_e2e:
        e2e = dict(t=float("nan"), wall=float("nan"), bi=0, bo=0)
        e2e_val = None
    else:
        e2e = suite_e2e(suite, stream, max(2, args.steps // 3))
        e2e_val = ws * suite.n * len(suite.ops) * max(2, args.steps // 3) / e2e["t"]
    launches = args.steps * suite.launches_per_step()
    n_ops = len(suite.ops)
    extra = {}
    if not args.skip_extra:
        del suite
        torch.cuda.empty_cache()
        which = set(args.extras.split(","))
        if "fused" in which:
            sched = tuple(int(v) for v in args.fused_schedule.split(",")) if args.fused_schedule else None
            extra["fused_pipeline"] = fused_pipeline(dev, stream, n=args.fused_n, schedule=sched)
        if "detection" in which:
            extra["detection"] = detection(dev, stream)
        if "differentiable" in which:
            extra["differentiable"] = differentiable(dev, stream, n=args.diff_b)
        if "large" in which:
            extra["per_transform_large"] = large_suite(dev, stream, hbm, n=args.large_n,
                                                       only=set(args.only.split(",")) if args.only else None)
        if "distort" in which:
            extra["distortions"] = distortions(dev, stream, hbm)
        if "targets" in which:
            extra["fused_detection"] = fused_detection(dev, stream)
        if "small" in which:
            extra["small_plain"] = small_plain(dev, stream, hbm)
    cpu = None
    if rank == 0 and ws == 1 and args.cpu_images > 0:
        # the oracle on the same resident workload, copied to the host
        host = host_images
        v, thr, done, dt = oracle_suite_sample(min(args.cpu_images, len(host)), imgs=host)
        cpu = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"{done} images of the suite workload x 15 transforms ({dt:.1f} s)"}
        n1 = min(args.cpu_images_1core, len(host))
        if n1 > 0:
            v1, _, done1, dt1 = oracle_suite_sample(n1, threads=1, imgs=host[:n1])
            cpu["value_1core"] = v1
            cpu["sample_1core"] = f"{done1} images of the suite workload x 15 transforms on one core ({dt1:.1f} s)"
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": {"workload": "per-transform suite: 2000 u8 RGB images H,W~U[333,500], 15 transforms "
                                       "(device-sampled params + one ragged launch each)",
                           "l2": "inputs larger than L2 (1.04 GB per step), no flush",
                           "parallelism": f"replicas x{ws}, no collective"},
                "roofline": {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1),
                             "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                             "traffic": traffic},
                "per_transform": per_transform,
                "clocks": clocks,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": e2e["bi"],
                        "d2h_bytes_per_step": e2e["bo"], "wall_s": round(e2e["wall"], 3)},
                "gpu_launches": None,
                "device_status": status,
                "cpu_baseline": cpu, **extra}
        line["gpu_launches"] = launches
        line["summary"] = summary(extra)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
