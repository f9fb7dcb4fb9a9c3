"""Benchmark of the neural six-way lightmap hot path on GB300.

One step = one frame of the whole hot path on the 128^3 FP32 smoke grid with a
radius-20 sphere obstacle, perspective camera, 512x512 billboard, step 2
voxels: grid staging -> guide march -> lightmap network -> six-way shading.
Metric: Mpix/s of completed (guide + lightmaps) frames.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f32|bf16|f16|fp8|bf16x3]
  python bench.py --impl reference ...   # the FP64 CPU oracle, timed on host cores

N > 1 (torchrun): independent replicas, one frame stream per GPU (the path has
no exchange step); value = frames of all ranks / max-over-ranks time.
The grid (10 MiB) fits in L2, so L2 is flushed (a 256 MiB write) before every
timed step, outside the timed events.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "plume128_sphere20_persp512_h2"
METRIC = "Mpix/s guide+lightmaps"
# FP32 operations charged per density evaluation of the march (algorithmic):
# sample position 7 (3 mul, 3 add, 1 mul for k*h), trilinear 30 (3 sub, 3 floor,
# 3 sub, 7 lerps x (1 sub + 1 FMA)), optical-depth accumulation 2.
FLOP_PER_SAMPLE = 39
GATHER_BYTES = 32                 # 8 FP32 voxels per trilinear density sample


def net_flop_per_pixel(c0=16):
    """Algorithmic FLOP of the lightmap network per full-resolution pixel (2 per
    multiply-add): 3x3 convolutions 2*9*cin*cout per output pixel of their
    level, transposed convolutions 2*4*cin*cout per input pixel, and per
    adapter pw1 (c->2c), depthwise 3x3 on 2c, pw2 (c->c), ffn1 (c->2c), ffn2
    (c->c), head (c->2); 85,600 at C0 = 16."""
    c = c0
    conv = [(3, c, 0), (c, c, 0), (c, 2 * c, 1), (2 * c, 2 * c, 1), (2 * c, 4 * c, 2), (4 * c, 4 * c, 2),
            (4 * c, 8 * c, 3), (8 * c, 8 * c, 3), (8 * c, 4 * c, 2), (4 * c, 4 * c, 2), (4 * c, 2 * c, 1),
            (2 * c, 2 * c, 1), (2 * c, c, 0), (c, c, 0)]
    convt = [(8 * c, 4 * c, 3), (4 * c, 2 * c, 2), (2 * c, c, 1)]
    f = sum(2 * 9 * ci * co / 4 ** lv for ci, co, lv in conv)
    f += sum(2 * 4 * ci * co / 4 ** lv for ci, co, lv in convt)
    f += 4 * (2 * (2 * c * c) + 2 * 9 * 2 * c + 2 * c * c + 2 * (2 * c * c) + 2 * c * c + 2 * 2 * c)
    return f
# DRAM bytes (read + write) of the three march passes of one frame of this
# workload: ncu dram__bytes_read.sum + dram__bytes_write.sum with
# --cache-control none on the current march kernels (octo-staged grid, in L2
# when the view pass starts; the writes are the segment scratch, the guide and
# write-backs of staged cells).
MARCH_DRAM_BYTES = 24_114_688 + 46_593_280


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def range_errs(got, ref):
    """max |got - ref| / max |ref| per plane (the oracle's range)."""
    return [float(np.abs(got[c].astype(np.float64) - ref[c]).max() / max(np.abs(ref[c]).max(), 1e-30))
            for c in range(ref.shape[0])]


def cpu_oracle_frame(pf, rows, blob_params, c0=16, keep=False):
    """The FP64 oracle on a band of `rows` image rows: guide, network on the band, shade."""
    import oracle
    r0 = (pf.camera.height - rows) // 2
    t0 = time.perf_counter()
    g, _, _ = oracle.guide(pf.density, pf.mask, pf.camera, pf.step, rows=(r0, r0 + rows))
    band = np.ascontiguousarray(g[:, r0:r0 + rows, :])
    diag = math.sqrt(sum(float(v) ** 2 for v in pf.density.shape))
    lm = oracle.net_forward(band, blob_params, c0, 1.0 / diag)
    cam = pf.camera
    import dataclasses
    cam_band = dataclasses.replace(cam, height=rows)
    oracle.shade(lm, cam_band, [pf.light])
    t = time.perf_counter() - t0
    if keep:
        return t, rows * pf.camera.width, (band, lm)
    return t, rows * pf.camera.width


REPLICA_TIMEOUT_S = 600.0   # a replica that dies ends the others' next collective with an error


def oracle_guide_full(pf):
    import oracle
    return oracle.guide(pf.density, pf.mask, pf.camera, pf.step)


def oracle_net(guide, flat, pf, c0=16):
    import oracle
    return oracle.net_forward(guide, flat, c0, 1.0 / math.sqrt(sum(float(v) ** 2 for v in pf.density.shape)))


def init_replicas(backend, timeout_s=REPLICA_TIMEOUT_S):
    """Process group of the independent replicas (one per GPU).  Its only
    collectives are the barriers around the timed region and the max-over-ranks
    reduction; the finite timeout turns a replica that died or never arrives
    into an error on the others instead of a hang."""
    import datetime
    import torch.distributed as dist
    dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s))


def max_over_ranks(local_ms, dev, ws):
    """The slowest rank's time (every rank gets it); a no-op for one process."""
    if ws <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix(frames_all_ranks, pixels_per_frame, max_ms):
    """Whole-job throughput: the frames every rank completed over the slowest rank's time."""
    return frames_all_ranks * pixels_per_frame / (max_ms / 1e3) / 1e6


def single_core_oracle(rows=8):
    """The oracle on one host core: the same band measurement in a child process
    with OpenMP held to one thread.  Returns (Mpix/s, None) or (None, reason)."""
    code = ("import sys, json; sys.path.insert(0, %r); import numpy as np; import bench, oracle; "
            "from paper_2604_03748_gb300 import inputs as I; oracle.build(); pf = I.config_obstacle_128(); "
            "flat = I.flat_params(I.make_params(16, 0)).astype(np.float64); "
            "print(json.dumps(bench.cpu_oracle_frame(pf, %d, flat)))" % (ROOT, rows))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    except subprocess.TimeoutExpired:
        return None, "timed out"
    if r.returncode != 0:
        return None, (r.stderr.strip().splitlines() or ["failed"])[-1][:200]
    t, px = json.loads(r.stdout.strip().splitlines()[-1])
    return px / t / 1e6, None


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2604_03748_gb300 import inputs as I
    oracle.build()
    pf = I.config_obstacle_128()
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    # size the per-step band so the whole run stays within --ref-seconds (150 s
    # by default): one probe band measures the per-pixel cost on this host
    probe_t, probe_px = cpu_oracle_frame(pf, 16, flat)
    per_px = probe_t / probe_px
    budget = args.ref_seconds / max(1, args.steps + args.warmup)
    rows = int(max(8, min(pf.camera.height, budget / per_px / pf.camera.width)) // 8 * 8)
    for _ in range(args.warmup):
        cpu_oracle_frame(pf, 8, flat)
    total_t, total_px = 0.0, 0
    for _ in range(args.steps):
        t, px = cpu_oracle_frame(pf, rows, flat)
        total_t += t
        total_px += px
    value = total_px / total_t / 1e6
    cores = os.cpu_count()
    one, why = single_core_oracle()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [128, 128, 128], "billboard": [512, 512],
                                        "step_voxels": 2.0, "obstacle": "sphere r=20",
                                        "sample_rows_per_step": rows},
        "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows}x512 pixel band of the 512x512 frame per step: guide march, "
                                   f"network on the band, shade",
                         "single_core": {"value": one, "unit": "Mpix/s", "cores": 1,
                                         "sample": "8x512 pixel band, OMP_NUM_THREADS=1",
                                         **({"unavailable": why} if why else {})}},
        "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="nsl", choices=["nsl", "reference"])
    ap.add_argument("--precision", default="f16", choices=["f32", "bf16", "f16", "fp8", "bf16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--forms", default="animated,batched,serving,training",
                    help="comma list of further workloads measured after the primary line's "
                         "('animated', 'batched', 'serving', 'training', or 'none')")
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="CPU time the reference arm (the FP64 oracle) spends on its timed and warm-up steps")
    ap.add_argument("--anim-frames", type=int, default=300,
                    help="frames of the animated form (300; fewer keep a profiler capture small)")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="length of each Poisson arrival run of the serving form")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        init_replicas("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2604_03748_gb300 import build as B, inputs as I, nsl
    if rank == 0 or ws == 1:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    nsl.load()

    prec = {"f32": nsl.NSL_PREC_F32, "bf16": nsl.NSL_PREC_BF16, "f16": nsl.NSL_PREC_F16,
            "fp8": nsl.NSL_PREC_FP8, "bf16x3": nsl.NSL_PREC_BF16X3}[args.precision]
    pf = I.config_obstacle_128()
    H, W = pf.camera.height, pf.camera.width
    blob = I.pack_blob(I.make_params(16, 0), 16)
    ctx = nsl.Context(pf.density.shape, nsl.NSL_F32, blob, W, H)
    stream = torch.cuda.current_stream()
    dens = torch.from_numpy(pf.density).to(dev)
    mask = torch.from_numpy(pf.mask).to(dev)
    guide = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    lm = torch.empty((8, H, W), dtype=torch.float32, device=dev)
    rgba = torch.empty((4, H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    opts = nsl.march_opts()

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        nsl.nsl_stage_grid(ctx.ctx, dens, mask, stream=stream)
        if evs:
            evs[1].record(stream)
        nsl.nsl_guiding_map(ctx.ctx, None, None, pf.camera, pf.step, guide, opts=opts, stream=stream)
        if evs:
            evs[2].record(stream)
        nsl.nsl_predict_lightmaps(ctx.ctx, guide, W, H, prec, lm, stream=stream)
        if evs:
            evs[3].record(stream)
        nsl.nsl_shade(ctx.ctx, lm, W, H, pf.camera, [pf.light], rgba, stream=stream)
        if evs:
            evs[4].record(stream)

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    samples = ctx.guide_sample_count(pf.camera, pf.step, opts)
    # the march's roofline denominators, measured on this device
    mpk = nsl.nsl_measure_peaks(stream=stream)

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    t_host0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        step(events[k])
    torch.cuda.synchronize()
    t_host = time.perf_counter() - t_host0
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[4]) for e in events]
    stage_ms = [e[0].elapsed_time(e[1]) for e in events]
    march_ms = [e[1].elapsed_time(e[2]) for e in events]
    net_ms = [e[2].elapsed_time(e[3]) for e in events]
    shade_ms = [e[3].elapsed_time(e[4]) for e in events]
    total_ms = float(sum(step_ms))
    total_ms = max_over_ranks(total_ms, dev, ws)
    frames = args.steps * ws
    value = whole_job_mpix(frames, H * W, total_ms)

    # end to end through the host entry points: H2D of the grid + mask, D2H of
    # guide, lightmaps and rgba, every frame; frames alternate between two
    # contexts on two streams (nsl_render_frame_host_async), so one frame's
    # copies overlap the other's kernels; a context's next frame waits for its
    # previous one
    pin = lambda a: torch.from_numpy(a).pin_memory()
    h_dens, h_mask = pin(pf.density), pin(pf.mask)
    ctx2 = nsl.Context(pf.density.shape, nsl.NSL_F32, blob, W, H)
    ctxs = [ctx, ctx2]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [[torch.empty((c, H, W), dtype=torch.float32).pin_memory() for c in (3, 8, 4)] for _ in range(2)]
    e2e_val = None
    if args.e2e_steps > 0:
        def e2e_frame(i):
            k = i % 2
            nsl.nsl_render_frame_host_async(ctxs[k].ctx, h_dens.numpy(), h_mask.numpy(), pf.camera, [pf.light],
                                            pf.step, prec, outs[k][0].numpy(), outs[k][1].numpy(),
                                            outs[k][2].numpy(), opts=opts, stream=streams[k])
        for i in range(4):                              # warm-up (both contexts)
            e2e_frame(i)
        torch.cuda.synchronize()
        nf = 2 * max(1, args.e2e_steps)
        t0 = time.perf_counter()
        for i in range(nf):
            if i >= 2:
                streams[i % 2].synchronize()            # this context's previous frame is done
            e2e_frame(i)
        for st_ in streams:
            st_.synchronize()
        e2e_val = nf * H * W / (time.perf_counter() - t0) / 1e6 * ws
    # the end-to-end figure of the line: one frame at a time through the
    # synchronous host entry point from page-locked host buffers (grid and
    # mask in, guide, lightmaps and rgba out), L2 flushed before each frame
    # outside the timed call, as the device-timed figure is
    e2e_sync = None
    if args.e2e_steps > 0:
        ho = [torch.empty((c, H, W), dtype=torch.float32).pin_memory() for c in (3, 8, 4)]

        def sync_frame():
            nsl.nsl_render_frame_host(ctx.ctx, h_dens.numpy(), h_mask.numpy(), pf.camera, [pf.light], pf.step, prec,
                                      ho[0].numpy(), ho[1].numpy(), ho[2].numpy(), opts=opts, stream=stream)
        for _ in range(3):
            sync_frame()
        dts = []
        for _ in range(max(10, 4 * args.e2e_steps)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sync_frame()
            dts.append(time.perf_counter() - t0)
        e2e_sync = len(dts) * H * W / sum(dts) / 1e6 * ws
    # device-resident inputs, two frames in flight on two streams (what the
    # pipelined end-to-end loop overlaps, without its copies)
    pipe_val = None
    if args.e2e_steps > 0:
        outs_d = [[torch.empty((c, H, W), dtype=torch.float32, device=dev) for c in (3, 8, 4)] for _ in range(2)]

        def dev_frame(i):
            k = i % 2
            with torch.cuda.stream(streams[k]):
                nsl.nsl_stage_grid(ctxs[k].ctx, dens, mask, stream=streams[k])
                nsl.nsl_guiding_map(ctxs[k].ctx, None, None, pf.camera, pf.step, outs_d[k][0], opts=opts,
                                    stream=streams[k])
                nsl.nsl_predict_lightmaps(ctxs[k].ctx, outs_d[k][0], W, H, prec, outs_d[k][1], stream=streams[k])
                nsl.nsl_shade(ctxs[k].ctx, outs_d[k][1], W, H, pf.camera, [pf.light], outs_d[k][2],
                              stream=streams[k])
        for i in range(4):
            dev_frame(i)
        torch.cuda.synchronize()
        nf = 2 * max(1, min(args.steps, 200))
        t0 = time.perf_counter()
        for i in range(nf):
            if i >= 2:
                streams[i % 2].synchronize()
            dev_frame(i)
        for st_ in streams:
            st_.synchronize()
        pipe_val = nf * H * W / (time.perf_counter() - t0) / 1e6 * ws
    ctx2.close()

    pk, pk_kind = peaks()
    march_avg_s = float(np.mean(march_ms)) / 1e3
    achieved = samples * FLOP_PER_SAMPLE / march_avg_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "bf16": "f32 march + bf16 net", "f16": "f32 march + f16 net",
                  "fp8": "f32 march + fp8 net", "bf16x3": "f32 march + split-bf16 net"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [128, 128, 128], "grid_dtype": "f32", "billboard": [512, 512],
                   "camera": "perspective fov 40", "step_voxels": 2.0, "obstacle": "sphere r=20",
                   "network": f"UNet C0=16 + 4 NAFBlock adapters, {args.precision}", "lights": 1,
                   "l2": "flushed (256 MiB write) before every timed step, outside the timed events"},
        "stage_ms": {"stage": float(np.mean(stage_ms)), "march": float(np.mean(march_ms)),
                     "net": float(np.mean(net_ms)), "shade": float(np.mean(shade_ms))},
        "roofline": {"kernel": "guide march (view pass + segment pass + finish pass)", "bound": "alu",
                     "achieved": achieved, "peak": mpk["fp32_tflops"], "unit": "TFLOP/s",
                     "frac": achieved / mpk["fp32_tflops"], "traffic": MARCH_DRAM_BYTES,
                     "work": {"density_samples": samples, "flop_per_sample": FLOP_PER_SAMPLE},
                     "peak_kind": f"measured in this run: FP32 FMA loop on {mpk['sms']} SMs (nsl_measure_peaks)",
                     # the march's closer limit: the trilinear gathers through L1 (8 FP32
                     # voxels = 32 B per density sample) against the L1 data path
                     "gather": {"bytes_per_sample": GATHER_BYTES,
                                "achieved": samples * GATHER_BYTES / march_avg_s / 1e9,
                                "peak": mpk["l1_gbps"], "unit": "GB/s",
                                "frac": samples * GATHER_BYTES / march_avg_s / 1e9 / mpk["l1_gbps"],
                                "peak_kind": "measured in this run: L1-resident coalesced 16-byte loads "
                                             "(nsl_measure_peaks)",
                                "l2_random_gather_gbps": mpk["l2_gather_gbps"]},
                     "network": {"kernel": "lightmap network (21 launches)", "bound": "tensor",
                                 "flop_per_pixel": net_flop_per_pixel(16),
                                 "achieved": net_flop_per_pixel(16) * H * W / (float(np.mean(net_ms)) / 1e3) / 1e12,
                                 "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                                 "frac": net_flop_per_pixel(16) * H * W / (float(np.mean(net_ms)) / 1e3) / 1e12
                                 / pk["bf16_tflops"],
                                 "peak_kind": f"{pk_kind} cuBLAS bf16 burst (FP16 has the same nominal "
                                              "tensor rate)" if args.precision in ("bf16", "f16", "bf16x3") else
                                              f"{pk_kind} cuBLAS bf16 burst (reference only: this run's "
                                              f"network is {args.precision})"}},
        "e2e": {"value": e2e_sync, "unit": "Mpix/s",
                "h2d_bytes_per_step": int(pf.density.nbytes + pf.mask.nbytes),
                "d2h_bytes_per_step": int((3 + 8 + 4) * H * W * 4),
                "mode": "one frame at a time through nsl_render_frame_host from page-locked host buffers, "
                        "L2 flushed before each frame outside the timed call"},
        "e2e_pipelined": {"value": e2e_val, "unit": "Mpix/s",
                          "note": "nsl_render_frame_host_async, two frames in flight on two streams and "
                                  "contexts (one frame's copies overlap the other's kernels), no L2 flush"},
        "pipelined": {"value": pipe_val, "unit": "Mpix/s",
                      "note": "inputs resident, two frames in flight on two streams and contexts, no L2 flush"},
        "gpu_launches": args.steps * launches_per_step(args.precision),
        "clocks": clk,
        "host_wall_s": t_host,
    }
    # the paper's own sampling distance, h = 10 voxels, on the same workload
    step10 = None
    if args.e2e_steps > 0:
        ctx10 = nsl.Context(pf.density.shape, nsl.NSL_F32, blob, W, H)
        g10 = torch.empty((3, H, W), dtype=torch.float32, device=dev)
        lm10 = torch.empty((8, H, W), dtype=torch.float32, device=dev)
        rgba10 = torch.empty((4, H, W), dtype=torch.float32, device=dev)

        def frame10():
            nsl.nsl_stage_grid(ctx10.ctx, dens, mask, stream=stream)
            nsl.nsl_guiding_map(ctx10.ctx, None, None, pf.camera, 10.0, g10, opts=opts, stream=stream)
            nsl.nsl_predict_lightmaps(ctx10.ctx, g10, W, H, prec, lm10, stream=stream)
            nsl.nsl_shade(ctx10.ctx, lm10, W, H, pf.camera, [pf.light], rgba10, stream=stream)
        for _ in range(3):
            frame10()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(5, min(args.steps, 100))):
            flush.zero_()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            frame10()
            b_.record(stream)
            ts.append((a_, b_))
        torch.cuda.synchronize()
        ms10 = float(np.mean([a_.elapsed_time(b_) for a_, b_ in ts]))
        step10 = {"value": H * W / (ms10 / 1e3) / 1e6, "unit": "Mpix/s", "ms_per_step": ms10,
                  "samples": ctx10.guide_sample_count(pf.camera, 10.0, opts)}
        ctx10.close()
    line["step_10_voxels"] = step10
    # the transmittance-volume approximation of the side lights' shadows
    # (one shadow march per voxel centre instead of per view sample)
    vol_row, g_vol = None, None
    if args.e2e_steps > 0:
        ctxv = nsl.Context(pf.density.shape, nsl.NSL_F32, blob, W, H)
        optsv = nsl.march_opts(shadow_volume=1)
        g_vol = torch.empty((3, H, W), dtype=torch.float32, device=dev)
        lmv = torch.empty((8, H, W), dtype=torch.float32, device=dev)
        rgbav = torch.empty((4, H, W), dtype=torch.float32, device=dev)

        def framev():
            nsl.nsl_guiding_map(ctxv.ctx, dens, mask, pf.camera, pf.step, g_vol, opts=optsv, stream=stream)
            nsl.nsl_predict_lightmaps(ctxv.ctx, g_vol, W, H, prec, lmv, stream=stream)
            nsl.nsl_shade(ctxv.ctx, lmv, W, H, pf.camera, [pf.light], rgbav, stream=stream)
        for _ in range(3):
            framev()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(5, min(args.steps, 100))):
            flush.zero_()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            framev()
            b_.record(stream)
            ts.append((a_, b_))
        torch.cuda.synchronize()
        msv = float(np.mean([a_.elapsed_time(b_) for a_, b_ in ts]))
        vol_row = {"value": H * W / (msv / 1e3) / 1e6, "unit": "Mpix/s", "ms_per_step": msv,
                   "note": "approximation (shadow_volume=1): side-light transmittances from 128^3 "
                           "voxel-centre volumes; error against the exact guide reported below"}
        ctxv.close()
    line["shadow_volume"] = vol_row
    # the other rows the workload configurations name: this 512^2 scene with
    # each network precision (FP32 is the plain single-plume path), the 64^3
    # orthographic 128^2 scene with the FP32 network, and one frame at a time
    # through the synchronous host entry point (copies in and out included)
    rows, lm_rows = {}, {}
    if args.e2e_steps > 0:
        gr = torch.empty((3, H, W), dtype=torch.float32, device=dev)
        nrep = max(5, min(args.steps, 50))
        for name, pr in (("f32", nsl.NSL_PREC_F32), ("bf16", nsl.NSL_PREC_BF16), ("f16", nsl.NSL_PREC_F16),
                         ("fp8", nsl.NSL_PREC_FP8), ("bf16x3", nsl.NSL_PREC_BF16X3)):
            lmr = torch.empty((8, H, W), dtype=torch.float32, device=dev)

            def frame_p(evs=None):
                if evs:
                    evs[0].record(stream)
                nsl.nsl_stage_grid(ctx.ctx, dens, mask, stream=stream)
                nsl.nsl_guiding_map(ctx.ctx, None, None, pf.camera, pf.step, gr, opts=opts, stream=stream)
                if evs:
                    evs[1].record(stream)
                nsl.nsl_predict_lightmaps(ctx.ctx, gr, W, H, pr, lmr, stream=stream)
                if evs:
                    evs[2].record(stream)
                nsl.nsl_shade(ctx.ctx, lmr, W, H, pf.camera, [pf.light], rgba, stream=stream)
                if evs:
                    evs[3].record(stream)
            for _ in range(3):
                frame_p()
            torch.cuda.synchronize()
            evl = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(nrep)]
            for k in range(nrep):
                flush.zero_()
                frame_p(evl[k])
            torch.cuda.synchronize()
            fms = float(np.mean([e[0].elapsed_time(e[3]) for e in evl]))
            nms = float(np.mean([e[1].elapsed_time(e[2]) for e in evl]))
            rows[f"{WORKLOAD}_{name}"] = {"value": H * W / (fms / 1e3) / 1e6, "unit": "Mpix/s", "ms_per_step": fms,
                                          "net_ms": nms,
                                          "net_tflops": net_flop_per_pixel(16) * H * W / (nms / 1e3) / 1e12}
            lm_rows[name] = lmr
        # the same frames with the FP32 network at base width C0 = 32
        blob32 = I.pack_blob(I.make_params(32, 0), 32)
        ctx32 = nsl.Context(pf.density.shape, nsl.NSL_F32, blob32, W, H)
        lm32 = torch.empty((8, H, W), dtype=torch.float32, device=dev)

        def frame32(evs=None):
            if evs:
                evs[0].record(stream)
            nsl.nsl_stage_grid(ctx32.ctx, dens, mask, stream=stream)
            nsl.nsl_guiding_map(ctx32.ctx, None, None, pf.camera, pf.step, gr, opts=opts, stream=stream)
            if evs:
                evs[1].record(stream)
            nsl.nsl_predict_lightmaps(ctx32.ctx, gr, W, H, nsl.NSL_PREC_F32, lm32, stream=stream)
            if evs:
                evs[2].record(stream)
            nsl.nsl_shade(ctx32.ctx, lm32, W, H, pf.camera, [pf.light], rgba, stream=stream)
            if evs:
                evs[3].record(stream)
        for _ in range(3):
            frame32()
        torch.cuda.synchronize()
        evl = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(max(5, min(args.steps, 20)))]
        for e in evl:
            flush.zero_()
            frame32(e)
        torch.cuda.synchronize()
        fms = float(np.mean([e[0].elapsed_time(e[3]) for e in evl]))
        nms = float(np.mean([e[1].elapsed_time(e[2]) for e in evl]))
        rows[f"{WORKLOAD}_f32_c0_32"] = {"value": H * W / (fms / 1e3) / 1e6, "unit": "Mpix/s", "ms_per_step": fms,
                                         "net_ms": nms,
                                         "net_tflops": net_flop_per_pixel(32) * H * W / (nms / 1e3) / 1e12}
        ctx32.close()
        # the 64^3 scene, orthographic 128^2, step 4, FP32 network
        pf1 = I.config_plain_64()
        H1, W1 = pf1.camera.height, pf1.camera.width
        ctx1 = nsl.Context(pf1.density.shape, nsl.NSL_F32, blob, W1, H1)
        d1 = torch.from_numpy(pf1.density).to(dev)
        g1 = torch.empty((3, H1, W1), dtype=torch.float32, device=dev)
        lm1 = torch.empty((8, H1, W1), dtype=torch.float32, device=dev)
        rgba1 = torch.empty((4, H1, W1), dtype=torch.float32, device=dev)

        def frame1():
            nsl.nsl_stage_grid(ctx1.ctx, d1, None, stream=stream)
            nsl.nsl_guiding_map(ctx1.ctx, None, None, pf1.camera, pf1.step, g1, opts=opts, stream=stream)
            nsl.nsl_predict_lightmaps(ctx1.ctx, g1, W1, H1, nsl.NSL_PREC_F32, lm1, stream=stream)
            nsl.nsl_shade(ctx1.ctx, lm1, W1, H1, pf1.camera, [pf1.light], rgba1, stream=stream)
        for _ in range(3):
            frame1()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(5, min(args.steps, 100))):
            flush.zero_()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            frame1()
            b_.record(stream)
            ts.append((a_, b_))
        torch.cuda.synchronize()
        ms1 = float(np.mean([a_.elapsed_time(b_) for a_, b_ in ts]))
        rows["plume64_ortho128_h4_f32"] = {"value": H1 * W1 / (ms1 / 1e3) / 1e6, "unit": "Mpix/s",
                                           "ms_per_step": ms1}
        ctx1.close()
        # synchronous frames from host buffers: nsl_render_frame_host copies the
        # grid and mask in, runs the frame and copies guide, lightmaps and rgba
        # out before returning
        hg, hl, hr = (np.empty((c, H, W), np.float32) for c in (3, 8, 4))
        for _ in range(2):
            nsl.nsl_render_frame_host(ctx.ctx, pf.density, pf.mask, pf.camera, [pf.light], pf.step, prec,
                                      hg, hl, hr, opts=opts, stream=stream)
        lat = []
        for _ in range(max(5, min(args.steps, 30))):
            t0 = time.perf_counter()
            nsl.nsl_render_frame_host(ctx.ctx, pf.density, pf.mask, pf.camera, [pf.light], pf.step, prec,
                                      hg, hl, hr, opts=opts, stream=stream)
            lat.append((time.perf_counter() - t0) * 1e3)
        rows["sync_host_frame"] = {"value": H * W / (float(np.median(lat)) / 1e3) / 1e6, "unit": "Mpix/s",
                                   "p50_ms": float(np.median(lat)), "p99_ms": float(np.percentile(lat, 99)),
                                   "precision": args.precision,
                                   "note": "one frame at a time through nsl_render_frame_host from pageable "
                                           "host buffers: 10.5 MB in, 15.7 MB out, synchronised"}
    line["rows"] = rows
    ctx.close()
    forms = [f for f in args.forms.split(",") if f and f != "none"]
    if "animated" in forms:
        line["animated"] = bench_animated(nsl, I, dev, args, rank == 0 and ws == 1 and not args.no_cpu_baseline)
    if "serving" in forms:
        line["serving"] = bench_serving(nsl, I, dev, args)
    trained_blob = None
    if "training" in forms:
        line["training"] = bench_training(nsl, I, dev, args)
        trained_blob = line["training"].pop("blob")
    if "batched" in forms:
        line["batched"] = bench_batched(nsl, I, dev, stream, flush, args, rank == 0 and ws == 1
                                        and not args.no_cpu_baseline)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
        # whole 512x512 frames until about 10 s of CPU work (at least one)
        t, px, ref = cpu_oracle_frame(pf, 512, flat, keep=True)
        nfr = 1
        while t < 10.0 and nfr < 20:
            t2, px2 = cpu_oracle_frame(pf, 512, flat)
            t += t2
            px += px2
            nfr += 1
        line["cpu_baseline"] = {"value": px / t / 1e6, "unit": "Mpix/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"{nfr} whole 512x512 frames ({t:.1f} s): FP64 guide march, "
                                          "FP64 network, shade"}
        # error of this run's last frame against that oracle frame, per channel,
        # relative to the oracle's range (guide: march; lightmaps: end to end,
        # i.e. the network's precision on top of the march)
        line["err_vs_oracle"] = {
            "guide": range_errs(guide.cpu().numpy(), ref[0]),
            "lightmaps": range_errs(lm.cpu().numpy(), ref[1]),
        }
        for name, lmr in lm_rows.items():
            rows[f"{WORKLOAD}_{name}"]["lightmaps_err_vs_oracle"] = max(range_errs(lmr.cpu().numpy(), ref[1]))
        if f"{WORKLOAD}_f32_c0_32" in rows:
            # the C0 = 32 network on this frame's guide against the oracle's
            # network at C0 = 32 on the oracle's guide, every output value
            flat32 = I.flat_params(I.make_params(32, 0)).astype(np.float64)
            ref32 = oracle_net(ref[0], flat32, pf, c0=32)
            l32 = lm32.cpu().numpy()
            rows[f"{WORKLOAD}_f32_c0_32"]["lightmaps_err_vs_oracle"] = max(range_errs(l32, ref32))
            rows[f"{WORKLOAD}_f32_c0_32"]["lightmaps_max_abs_vs_oracle"] = float(np.abs(l32 - ref32).max())
        if "plume64_ortho128_h4_f32" in rows:
            o1, _, _ = oracle_guide_full(pf1)
            ref1 = oracle_net(o1, flat, pf1)
            rows["plume64_ortho128_h4_f32"]["err_vs_oracle"] = {
                "guide": max(range_errs(g1.cpu().numpy(), o1)),
                "lightmaps_max_abs": float(np.abs(lm1.cpu().numpy() - ref1).max())}
        if vol_row is not None:
            vol_row["guide_err_vs_exact_oracle"] = range_errs(g_vol.cpu().numpy(), ref[0])
        # reported only: the fine-step (0.25 voxel) six-light reference on the
        # middle row against the coarse guide's transmittance and the lightmaps
        # of the untrained network (the physical target of a trained one)
        import oracle
        t0 = time.perf_counter()
        o7 = oracle.reference_lightmaps(pf.density, pf.mask, pf.camera, hf=0.25, rows=(H // 2, H // 2 + 1))
        r = H // 2
        g_np, lm_np = guide.cpu().numpy(), lm.cpu().numpy()
        rng7 = lambda a, b: float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))
        line["vs_fine_reference"] = {
            "row": r, "oracle_s": time.perf_counter() - t0,
            "guide_T": rng7(g_np[1, r], o7[6, r]),
            "lightmaps_six_planes": [rng7(lm_np[c, r], o7[c, r]) for c in range(6)],
            "lightmaps_T": rng7(lm_np[6, r], o7[6, r]),
            "note": "untrained network: reported, not a pass criterion",
        }
        if trained_blob is not None:
            # the network trained by the training form (32^3 volumes at 64 x 64)
            # on this 512^2 workload's guide
            ctxt = nsl.Context(pf.density.shape, nsl.NSL_F32, trained_blob, W, H)
            lmt = torch.empty((8, H, W), dtype=torch.float32, device=dev)
            ctxt.predict_lightmaps(guide, W, H, nsl.NSL_PREC_F32, lmt)
            torch.cuda.synchronize()
            ctxt.close()
            lt = lmt.cpu().numpy()
            line["vs_fine_reference"]["trained_lightmaps_six_planes"] = [rng7(lt[c, r], o7[c, r]) for c in range(6)]
            line["vs_fine_reference"]["trained_lightmaps_T"] = rng7(lt[6, r], o7[6, r])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_animated(nsl, I, dev, args, with_oracle):
    """Animated form: 300 frames (--anim-frames) of a 256^3 FP16 plume advected along a seeded
    curl-noise velocity (generated on the GPU before timing), camera on a
    seeded spline, light turning 1 degree per frame; 1024x1024 billboard, step
    4 voxels, FP8 network (and FP16 beside it).  Every frame stages its own
    grid, marches the guide, runs the network and shades, timed with CUDA
    events per frame."""
    import torch
    t0 = time.perf_counter()
    nf = max(4, args.anim_frames)
    mid = nf // 2
    seq = I.animated_sequence(256, nf, seed=3, width=1024, height=1024, step=4.0, device=dev)
    gen_s = time.perf_counter() - t0
    W = H = 1024
    blob = I.pack_blob(I.make_params(16, 0), 16)
    ctx = nsl.Context((256, 256, 256), nsl.NSL_F16, blob, W, H)
    stream = torch.cuda.current_stream()
    guide = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    lm = torch.empty((8, H, W), dtype=torch.float32, device=dev)
    rgba = torch.empty((4, H, W), dtype=torch.float32, device=dev)
    opts = nsl.march_opts()
    out = {"workload": f"256^3 f16 plume, {nf} frames (curl-noise advection, seed 3), perspective 1024x1024 "
                       "on a spline, light turning 1 deg/frame, step 4 voxels",
           "generation_s": gen_s, "frames": nf}
    for name, prec in (("fp8", nsl.NSL_PREC_FP8), ("f16", nsl.NSL_PREC_F16)):
        def frame(t, evs=None):
            if evs:
                evs[0].record(stream)
            nsl.nsl_stage_grid(ctx.ctx, seq.frames[t], None, stream=stream)
            nsl.nsl_guiding_map(ctx.ctx, None, None, seq.cameras[t], seq.step, guide, opts=opts, stream=stream)
            nsl.nsl_predict_lightmaps(ctx.ctx, guide, W, H, prec, lm, stream=stream)
            nsl.nsl_shade(ctx.ctx, lm, W, H, seq.cameras[t], [seq.lights[t]], rgba, stream=stream)
            if evs:
                evs[1].record(stream)
        for t in range(3):
            frame(t)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nf)]
        for t in range(nf):
            frame(t, evs[t])
        torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in evs])
        out[name] = {"value": nf * W * H / (ms.sum() / 1e3) / 1e6, "unit": "Mpix/s",
                     "ms_per_frame": float(ms.mean()), "p50_ms": float(np.percentile(ms, 50)),
                     "p99_ms": float(np.percentile(ms, 99)), "max_ms": float(ms.max())}
    if with_oracle:
        # FP64 oracle guide on a 64-row band of the first, middle and last
        # frames against this run's guides (the middle frame's guide then feeds
        # the network comparison below)
        import oracle
        out["err_vs_oracle"] = {}
        for t in (0, nf - 1, mid):
            frame(t)
            torch.cuda.synchronize()
            g = guide.cpu().numpy()
            host = seq.frames[t].cpu().numpy()
            t1 = time.perf_counter()
            o, _, _ = oracle.guide(host, None, seq.cameras[t], seq.step, rows=(480, 544))
            dt = time.perf_counter() - t1
            out["err_vs_oracle"][f"guide_band_frame{t}"] = range_errs(g[:, 480:544], o[:, 480:544])
        # the FP8 and FP16 networks on this frame's guide against the oracle's
        # emulation of the FP8 form and the FP64 network on the same guide
        flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
        ds = 1.0 / math.sqrt(3.0 * 256 * 256)
        gg = torch.from_numpy(g).to(dev)
        lms = {}
        for name, prec in (("fp8", nsl.NSL_PREC_FP8), ("f16", nsl.NSL_PREC_F16)):
            nsl.nsl_predict_lightmaps(ctx.ctx, gg, W, H, prec, lm, stream=stream)
            torch.cuda.synchronize()
            lms[name] = lm.cpu().numpy()
        g64 = g.astype(np.float64)
        t2 = time.perf_counter()
        full = oracle.net_forward(g64, flat, 16, ds)
        emu8 = oracle.net_forward_prec(g64, flat, 16, ds, oracle.PREC_FP8)
        out["err_vs_oracle"][f"lightmaps_frame{mid}"] = {
            "fp8_vs_fp8_emulation": max(range_errs(lms["fp8"], emu8)),
            "fp8_vs_fp64": max(range_errs(lms["fp8"], full)),
            "fp8_emulation_vs_fp64": max(range_errs(emu8, full)),
            "f16_vs_fp64": max(range_errs(lms["f16"], full)),
            "oracle_s": time.perf_counter() - t2,
            "note": "all on the GPU's guide of the frame; the FP8 form itself is far from FP64 on these "
                    "random weights (its emulation shows it), the per-layer tests hold the kernels to it"}
        out["cpu_baseline"] = {"value": 64 * W / dt / 1e6, "unit": "Mpix/s (guide only)", "cores": os.cpu_count(),
                               "kind": "oracle", "sample": f"FP64 guide march of rows 480..543 of frame {mid}"}
    ctx.close()
    del seq
    torch.cuda.empty_cache()
    return out


def bench_serving(nsl, I, dev, args):
    """Serving form: 256 plumes (seed 5) with grids from {32..256}^3 FP32 and
    billboards from {64..1024}^2 registered with the server (40 GiB HBM budget,
    2 batch streams, batches of up to 64, BF16 network), all admitted by one
    warm-up request each, then seeded Poisson arrivals at 2000 req/s (and at
    lower rates) for a fixed time, each request a new camera and light for a
    uniformly drawn plume.  Latency = submit -> lightmaps ready.  Two step
    conventions (the workload states none): 2 voxels for every grid, and n/64
    voxels (the ratio of the 128^3 and 256^3 workloads)."""
    import torch
    spec = I.serving_plumes_spec(256, seed=5)
    blob = I.pack_blob(I.make_params(16, 0), 16)
    t0 = time.perf_counter()
    hosts = [I.blob_fbm_volume_fast(p.n, p.seed, device=dev).cpu().numpy() for p in spec]
    gen_s = time.perf_counter() - t0
    mean_px = float(np.mean([p.width * p.height for p in spec]))
    out = {"workload": "256 resident plumes, grids U{32,48,64,96,128,192,256}^3 f32, billboards "
                       "U{64,128,256,512,1024}^2, perspective fov 40, seed 5; Poisson arrivals, plume "
                       "uniform, new camera and light per request",
           "budget_bytes": 40 << 30, "streams": 2, "max_batch": 64, "max_batch_pixels": 1 << 20,
           "precision": "bf16",
           "generation_s": gen_s, "frame_budgets_ms": [11.1, 16.7], "steps": {}}
    hosts16 = None
    # the last configuration serves the split-BF16 network (the BF16 form
    # within 2e-2 of range of FP64)
    for step_name, step_of, f16, sprec in (
            ("2 voxels", lambda n: 2.0, False, nsl.NSL_PREC_BF16),
            ("n/64 voxels", lambda n: n / 64.0, False, nsl.NSL_PREC_BF16),
            ("n/64 voxels, f16 grids", lambda n: n / 64.0, True, nsl.NSL_PREC_BF16),
            ("n/64 voxels, split bf16", lambda n: n / 64.0, False, nsl.NSL_PREC_BF16X3)):
        if f16 and hosts16 is None:
            hosts16 = [h.astype(np.float16) for h in hosts]
        srv = nsl.Server(blob, nsl.server_opts(hbm_budget_bytes=40 << 30, streams=2, max_batch=64,
                                               precision=sprec))
        ids = [srv.add_plume(h, None, step_of(p.n), p.width, p.height)
               for h, p in zip(hosts16 if f16 else hosts, spec)]
        for pid, p in zip(ids, spec):                 # warm-up: admit every plume once
            srv.submit(pid, p.camera, p.light)
        srv.drain()
        warm = srv.stats()
        res = {"resident_after_warmup": {"plumes": warm["resident_plumes"], "bytes": warm["resident_bytes"]},
               "runs": []}
        for rate in (2000.0, 1500.0, 1000.0, 750.0, 500.0, 350.0, 250.0):
            reqs = I.poisson_requests(len(spec), rate, args.serve_seconds, seed=5)
            cams = [(I.perspective_camera(spec[k].n, cs, spec[k].width, spec[k].height), I.random_light(ls))
                    for _, k, cs, ls in reqs]
            srv.reset_stats()
            clocks = ClockSampler(torch.cuda.current_device())
            clocks.start()
            start = time.perf_counter()
            for (t, k, _, _), (cam, light) in zip(reqs, cams):
                while time.perf_counter() - start < t:
                    pass
                srv.submit(ids[k], cam, light)
            submit_s = time.perf_counter() - start
            srv.drain(600000.0)
            st = srv.stats()
            clk = clocks.stop()
            res["runs"].append({
                "rate_req_s": rate, "requests": len(reqs), "offered_mpix_s": rate * mean_px / 1e6,
                "submit_s": submit_s, "value": st["pixels_completed"] / max(st["busy_s"], 1e-9) / 1e6,
                "unit": "Mpix/s", "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                "completed": st["completed"], "failed": st["failed"], "batches": st["batches"],
                "mean_batch": st["mean_batch"], "evictions": st["evictions"], "clocks": clk})
        srv.close()
        # the highest offered rate of the ladder whose 99th-percentile latency
        # meets each frame budget
        for budget in (16.7, 11.1):
            ok = [r["rate_req_s"] for r in res["runs"] if r["p99_ms"] <= budget and r["failed"] == 0]
            res[f"max_rate_p99_le_{budget}ms"] = max(ok) if ok else None
        out["steps"][step_name] = res
    return out


def training_dataset(nsl, I, count, n, size, seed, step=2.0, hf=0.5):
    """Synthetic (guide, fine-step reference) pairs: seeded blob x fBm volumes of
    n^3 voxels under seeded perspective cameras, size x size; the guide march
    at `step` voxels and the six-light reference at hf (emissive plane 0)."""
    import torch
    blob = I.pack_blob(I.make_params(16, 0), 16)
    ctx = nsl.Context((n, n, n), nsl.NSL_F32, blob, size, size)
    g = torch.empty((count, 3, size, size), device="cuda")
    t = torch.zeros((count, 8, size, size), device="cuda")
    ref = torch.empty((7, size, size), device="cuda")
    for k in range(count):
        d = torch.from_numpy(I.blob_fbm_volume(n, seed + k)).cuda()
        cam = I.perspective_camera(n, seed + k, size, size)
        ctx.guiding_map(d, None, cam, step, g[k])
        nsl.nsl_reference_lightmaps(ctx.ctx, None, None, cam, hf, ref)
        t[k, :7] = ref
    torch.cuda.synchronize()
    ctx.close()
    return g, t


def bench_training(nsl, I, dev, args):
    """Training slice (Sec. 4.4, MSE term): Adam on 96 synthetic pairs of 32^3
    volumes at 64 x 64 (guide march h = 2, six-light reference h_f = 0.5),
    batches of 8; steps per second, the loss, and the error of 16 held-out
    frames before and after, relative to each plane's range (max over the
    seven physical planes, median over frames)."""
    import torch
    n, S, B = 32, 64, 8
    ds = 1.0 / math.sqrt(3.0 * n * n)
    t0 = time.perf_counter()
    g_tr, t_tr = training_dataset(nsl, I, 96, n, S, seed=100)
    g_te, t_te = training_dataset(nsl, I, 16, n, S, seed=900)
    gen_s = time.perf_counter() - t0
    blob0 = I.pack_blob(I.make_params(16, 0), 16)
    tt = t_tr.cpu().numpy()
    rng6 = [float(np.mean(np.abs(tt[:, c]).max(axis=(1, 2)))) for c in range(6)]
    weights = [1.0 / max(r, 1e-3) ** 2 for r in rng6] + [1.0, 1.0]
    steps, lr0 = 1500, 2e-3
    tr = nsl.Trainer(blob0, nsl.train_opts(batch=B, width=S, height=S, lr=lr0, plane_weight=weights))
    rng = np.random.default_rng(53)
    losses = []
    t1 = time.perf_counter()
    for it in range(steps):
        tr.set_lr(lr0 * 0.5 * (1.0 + math.cos(math.pi * it / steps)) + 1e-6)
        idx = torch.from_numpy(rng.choice(96, B, replace=False)).cuda()
        losses.append(tr.step(g_tr[idx].contiguous(), t_tr[idx].contiguous(), ds))
    train_s = time.perf_counter() - t1
    trained = tr.blob()
    tr.close()

    def held_out(blob):
        ctx = nsl.Context((n, n, n), nsl.NSL_F32, blob, S, S)
        out = torch.empty((8, S, S), device="cuda")
        mx, rms = [], []
        for k in range(g_te.shape[0]):
            ctx.predict_lightmaps(g_te[k].contiguous(), S, S, nsl.NSL_PREC_F32, out)
            torch.cuda.synchronize()
            o, t = out.cpu().numpy()[:7], t_te[k].cpu().numpy()[:7]
            r = [max(np.abs(t[c]).max(), 1e-30) for c in range(7)]
            mx.append(max(float(np.abs(o[c] - t[c]).max() / r[c]) for c in range(7)))
            rms.append(max(float(np.sqrt(((o[c] - t[c]) ** 2).mean()) / r[c]) for c in range(7)))
        ctx.close()
        return {"max_abs": float(np.median(mx)), "rms": float(np.median(rms))}
    return {"workload": "96 training + 16 held-out pairs: 32^3 blob x fBm volumes, perspective 64x64, guide h=2, "
                        "reference h_f=0.5; Adam lr 2e-3 with cosine decay, batch 8, lightmap planes weighted "
                        "by 1/range^2",
            "generation_s": gen_s, "steps": steps, "steps_per_s": steps / train_s,
            "loss_first": losses[0], "loss_last_mean10": float(np.mean(losses[-10:])),
            "held_out_err_untrained": held_out(blob0), "held_out_err_trained": held_out(trained),
            "note": "error of the seven physical planes relative to each plane's range: median over "
                    "frames of the largest plane's max-abs and RMS error",
            "blob": trained}


def launches_per_step(precision):
    """Kernels of one single-plume step: staging 1, guide march 3 (view pass,
    segment pass, finish pass), network, shading 1.  Tensor-core network: SIMT
    first convolution 1 + 13 tensor-core convolutions + 3 transposed
    convolutions + adapters 4 (pass 1, the two-launch channel-attention
    reduction, pass 2) = 21; FP32 network: 14 convolutions + 3 transposed
    convolutions + adapters 3 = 20."""
    return 1 + 3 + (20 if precision == "f32" else 21) + 1


def bench_batched(nsl, I, dev, stream, flush, args, with_oracle):
    """Batched form: 64 plumes (seed 4) with grids drawn from {32..192}^3 FP32 and
    billboards from {64..512}^2, each with its own perspective camera and light,
    rendered by one captured CUDA graph per step (staging, guide march, grouped
    BF16 network, shading over all plumes), tuning from the autotuner.  The same
    64 plumes through the plain single-plume path with the FP32 network give
    the comparison figure."""
    import torch
    stream = torch.cuda.Stream()          # graph capture needs a non-default stream
    with torch.cuda.stream(stream):
        return _bench_batched(nsl, I, dev, stream, flush, args, with_oracle)


def _bench_batched(nsl, I, dev, stream, flush, args, with_oracle):
    import torch
    spec = I.batch_plumes_spec(64, seed=4)
    blob = I.pack_blob(I.make_params(16, 0), 16)
    items = []
    for p in spec:
        H, W = p.camera.height, p.camera.width
        items.append(dict(
            density=I.blob_fbm_volume_fast(p.n, p.seed, device=dev).contiguous(), mask=None,
            sigma_scale=1.0, camera=p.camera, step=p.step, light=p.light,
            guide=torch.empty((3, H, W), dtype=torch.float32, device=dev),
            lightmaps=torch.empty((8, H, W), dtype=torch.float32, device=dev),
            rgba=torch.empty((4, H, W), dtype=torch.float32, device=dev)))
    pixels = sum(p.camera.width * p.camera.height for p in spec)
    out = {"workload": "64 plumes, grids U{32,48,64,96,128,192}^3 f32, billboards U{64,128,256,512}^2, "
                       "perspective fov 40, step 2 voxels, seed 4",
           "pixels_per_step": pixels, "voxels": int(sum(p.n ** 3 for p in spec))}
    b = nsl.Batch(blob, 64)
    # bf16x3: the split-BF16 network (three BF16 tensor-core products per
    # multiply, binary32 activations), the BF16 form that meets 2e-2 of range
    for name, prec in (("bf16", nsl.NSL_PREC_BF16), ("f16", nsl.NSL_PREC_F16), ("bf16x3", nsl.NSL_PREC_BF16X3)):
        tune_ms = b.autotune(items, prec, stream=stream)
        tuning = b.get_tuning()
        b.capture_graph(items, prec, stream)
        for _ in range(max(3, args.warmup)):
            flush.zero_()
            b.launch_graph(stream)
        torch.cuda.synchronize()
        nsteps = min(args.steps, 30)                  # a batch is ~16 ms of work
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        for k in range(nsteps):
            flush.zero_()
            ev[k][0].record(stream)
            b.launch_graph(stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(c) for a, c in ev]))
        # the march form the tuner did not pick, timed the same way
        form = b.get_march_form()
        b.set_march_form(1 - form)
        b.capture_graph(items, prec, stream)
        for _ in range(3):
            b.launch_graph(stream)
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        for k in range(nsteps):
            flush.zero_()
            ev2[k][0].record(stream)
            b.launch_graph(stream)
            ev2[k][1].record(stream)
        torch.cuda.synchronize()
        ms_other = float(np.mean([a.elapsed_time(c) for a, c in ev2]))
        b.set_march_form(form)
        b.capture_graph(items, prec, stream)
        out[name] = {"value": pixels / (ms / 1e3) / 1e6, "unit": "Mpix/s", "ms_per_step": ms,
                     "ms_per_step_other_march_form": ms_other,
                     "tuning": {"seg_len": tuning[0], "march_blocks_per_sm": tuning[1],
                                "conv_ctas_per_sm": tuning[2], "march_tile_width": b.get_march_tile(),
                                "persistent_march": b.get_march_form(), "autotune_ms": tune_ms},
                     "launches_per_step": 1 + (1 if b.get_march_form() else 3) + 21 + 1}
    b.close()

    # the plain single-plume path with the FP32 network on the same plumes
    ctxs = {}
    for p in spec:
        if p.n not in ctxs:
            ctxs[p.n] = nsl.Context((p.n, p.n, p.n), nsl.NSL_F32, blob, 512, 512)
    opts = nsl.march_opts()

    def plain_pass():
        for p, it in zip(spec, items):
            c = ctxs[p.n].ctx
            nsl.nsl_stage_grid(c, it["density"], None, stream=stream)
            nsl.nsl_guiding_map(c, None, None, p.camera, p.step, it["guide"], opts=opts, stream=stream)
            nsl.nsl_predict_lightmaps(c, it["guide"], p.camera.width, p.camera.height, nsl.NSL_PREC_F32,
                                      it["lightmaps"], stream=stream)
            nsl.nsl_shade(c, it["lightmaps"], p.camera.width, p.camera.height, p.camera, [p.light],
                          it["rgba"], stream=stream)

    for _ in range(2):
        flush.zero_()
        plain_pass()
    torch.cuda.synchronize()
    reps = max(1, min(5, args.steps))
    tms = []
    for _ in range(reps):
        flush.zero_()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plain_pass()
        c.record(stream)
        torch.cuda.synchronize()
        tms.append(a.elapsed_time(c))
    ms = float(np.mean(tms))
    out["plain_f32_single_plume"] = {"value": pixels / (ms / 1e3) / 1e6, "unit": "Mpix/s", "ms_per_step": ms,
                                     "launches_per_step": 64 * (1 + 3 + 20 + 1)}
    out["speedup_bf16_vs_plain_f32"] = out["bf16"]["value"] / out["plain_f32_single_plume"]["value"]
    out["speedup_bf16x3_vs_plain_f32"] = out["bf16x3"]["value"] / out["plain_f32_single_plume"]["value"]
    for c in ctxs.values():
        c.close()

    if with_oracle:
        # FP64 oracle on 8 plumes of the batch drawn with a seeded generator:
        # timed (CPU baseline of this form) and compared with the batch's BF16,
        # F16 and split-BF16 output
        import oracle
        flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
        order = sorted(np.random.default_rng(4).choice(len(spec), size=8, replace=False).tolist())
        b = nsl.Batch(blob, 64)
        res = {}
        for name, prec in (("bf16", nsl.NSL_PREC_BF16), ("f16", nsl.NSL_PREC_F16), ("bf16x3", nsl.NSL_PREC_BF16X3)):
            b.render(items, prec, stream=stream)
            torch.cuda.synchronize()
            res[name] = [(items[k]["guide"].cpu().numpy(), items[k]["lightmaps"].cpu().numpy()) for k in order]
        b.close()
        t0 = time.perf_counter()
        px = 0
        errs = {"plumes": [f"n={spec[k].n} {spec[k].camera.width}x{spec[k].camera.height}" for k in order]}
        for j, k in enumerate(order):
            p = spec[k]
            dens = items[k]["density"].cpu().numpy()
            g, _, _ = oracle.guide(dens, None, p.camera, p.step)
            lm = oracle.net_forward(g, flat, 16, 1.0 / math.sqrt(3.0 * p.n * p.n))
            px += p.camera.width * p.camera.height
            for name in ("bf16", "f16", "bf16x3"):
                e = errs.setdefault(name, {"guide": [], "lightmaps": []})
                e["guide"].append(max(range_errs(res[name][j][0], g)))
                e["lightmaps"].append(max(range_errs(res[name][j][1], lm)))
        t = time.perf_counter() - t0
        out["err_vs_oracle"] = errs
        out["cpu_baseline"] = {"value": px / t / 1e6, "unit": "Mpix/s", "cores": os.cpu_count(),
                               "kind": "oracle", "sample": "8 seeded plumes of the batch, whole "
                                                           "frames: FP64 guide march and network"}
    return out

if __name__ == "__main__":
    sys.exit(main())
