#!/usr/bin/env python
"""fwd+bwd throughput of the FHGS feature-splatting hot path on GB300.

Workload (one step = the whole hot path on one synthetic view):
  1M Gaussians (means N(0, 0.6^2) clipped to [-2,2]^3, log-scales U[-5,-2],
  SH degree 3, opacity sigmoid(N(0,1))), 512-dim BF16 features ~N(0,1),
  one 1920x1080 pinhole camera at distance 4 (60 deg horizontal FoV),
  upstream gradients N(0,1) on the RGB and feature images.
  step = project (EWA + SH) -> bin + sort -> render forward (RGB + feature
  blend) -> render backward -> projection backward.

Prints one JSON line.  `value` is device-resident fwd+bwd Mpix/s of the
tensor-core path (the FP32 CUDA-core path is reported beside it), `e2e` the
same through the C ABI with host buffers and every copy inside the timed
region, `roofline` the dominant kernel against the measured HBM peak, and
`cpu_baseline` the FP64 oracle on the host cores on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpix/s at 1M Gaussians, D=512, BF16-TC vs FP32 path; % of roofline"
UNIT = "Mpix/s"
WORKLOAD = "1M Gaussians, 1920x1080 view, SH degree 3, D=512 BF16 features, fwd+bwd"
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--D", type=int, default=512)
    ap.add_argument("--width", type=int, default=1920, help="profiling only: smaller view, same scene")
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--path", choices=["tc", "fp32", "auto"], default="auto")
    ap.add_argument("--d-split", type=int, default=0, help="feature columns per CTA (0 = auto)")
    ap.add_argument("--fp32-steps", type=int, default=3, help="timed steps of the FP32 comparison path (0 = skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time eager launches instead of the captured step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="warm-up + one step, no JSON (for ncu)")
    ap.add_argument("--workload", choices=["render", "fusion", "ndfd", "points", "train", "batched", "surfel"],
                    default="render",
                    help="render: fwd+bwd of the 1080p view (the headline); fusion: 3M Gaussians x 64 views; "
                         "ndfd: the NDFD losses L_gt, L_cf and their backward on the 1080p view; "
                         "points: the paper's point-to-feature assignment, 3M points x 64 views; "
                         "train: one training iteration (render, L1, NDFD, Adam) on the 1080p view; "
                         "batched: 16 uneven cameras, 500k Gaussians, D=256, one CUDA graph per step; "
                         "surfel: the 2DGS surfel geometry on the 1080p view (FP32 path)")
    ap.add_argument("--views", type=int, default=64, help="fusion: number of views")
    ap.add_argument("--list-cut", type=int, choices=[0, 1], default=1,
                    help="cut the tile lists where every pixel has stopped (identical outputs); 0 = full lists")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]),
                    bf16_sus=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------- workload
def make_workload(seed, n, D, dev, width=1920, height=1080):
    import numpy as np
    import torch
    from paper_2505_19154_gb300 import synth
    scene, cams = synth.config3(seed, n=n, D=D)
    if (width, height) != (1920, 1080):  # centre crop of the same view: same focal length
        cams = [dict(cams[0], width=width, height=height, cx=width / 2.0, cy=height / 2.0)]
    t = {k: torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev)
         for k in ("means", "scales", "quats", "opacities", "sh")}
    t["features"] = torch.from_numpy(scene["features"]).to(dev).to(torch.bfloat16)
    P = cams[0]["width"] * cams[0]["height"]
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000 + seed)
    t["dC"] = torch.randn((P, 3), generator=gen, device=dev)
    t["dF"] = torch.randn((P, D), generator=gen, device=dev)
    return scene, cams, t, P


def composited_pairs(st, cams, tile=16):
    """Q = sum over tiles of (pixels in the tile) x (Gaussians the tile walks
    before its last pixel saturates), the per-pixel count sum_p last_p, and
    U = how many distinct Gaussians some tile walks (their records and
    feature rows are the ones a render pass must read).  `last` is the
    forward output: (position of the last contributor in the tile's list)
    + 1 per pixel."""
    import torch
    last, ranges, gids = st["last"], st["ranges"].to(torch.int64), st["gids"]
    q_tile, q_pix, off, toff = 0, 0, 0, 0
    walked = []
    for c in cams:
        w, h = c["width"], c["height"]
        L = last[off:off + w * h].view(h, w).to(torch.int64)
        off += w * h
        ty, tx = (h + tile - 1) // tile, (w + tile - 1) // tile
        pad = torch.zeros((ty * tile, tx * tile), dtype=torch.int64, device=L.device)
        ones = torch.zeros_like(pad)
        pad[:h, :w] = L
        ones[:h, :w] = 1
        mx = pad.view(ty, tile, tx, tile).amax(dim=(1, 3)).reshape(-1)
        cnt = ones.view(ty, tile, tx, tile).sum(dim=(1, 3)).reshape(-1)
        q_tile += int((mx * cnt).sum().item())
        q_pix += int(L.sum().item())
        start = ranges[toff:toff + ty * tx, 0]
        toff += ty * tx
        idx = torch.repeat_interleave(start, mx) + (
            torch.arange(int(mx.sum().item()), device=L.device) -
            torch.repeat_interleave(torch.cumsum(mx, 0) - mx, mx))
        walked.append(gids[idx].to(torch.int64) + (len(walked) << 40))
    U = int(torch.unique(torch.cat(walked)).numel()) if walked else 0
    return q_tile, q_pix, U


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# a kernel at 1920x1080, from an ncu capture of the 960x544 centre crop scaled
# by the pixel count (the traffic of both render kernels is the per-pixel
# image: dF read, feature image written), with the SHA-256 of the kernel's
# source file: a changed source reports null.  The hash is moved to a new
# source only when the edit leaves both render kernels untouched.
_CROP_SCALE = (1920 * 1080) / (960 * 544)
TRAFFIC = {
    "render_bwd_tc": {"bytes": int((1102.9e6 + 4.4e6) * _CROP_SCALE), "file": "render_tc.cu",
                      "sha256": "d8559e1bb2dc7cd157224a8ba80955e01e7602c18515ad362570788f18889f62"},
    "render_fwd_tc": {"bytes": int((7.6e6 + 1021.6e6) * _CROP_SCALE), "file": "render_tc.cu",
                      "sha256": "d8559e1bb2dc7cd157224a8ba80955e01e7602c18515ad362570788f18889f62"},
}


def traffic_for(kernel):
    import hashlib
    rec = TRAFFIC.get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2505_19154_gb300", "csrc", rec["file"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["sha256"]:
        return None
    return rec["bytes"]


def algorithmic_flops(N, D, Q):
    """Tensor-core FLOPs of the feature contractions: the blend W(PxB).Fe(BxD)
    forward (2DQ), dL/dw = dF.Fe^T and grad_Fe = W^T.dF backward (4DQ)."""
    return {"render_fwd": 2 * D * Q, "render_bwd": 4 * D * Q}


def algorithmic_bytes(P, N, D, I, U):
    """Bytes each kernel group must move at minimum: images once, the
    records and feature rows of the U Gaussians the tiles walk once per
    pass, their feature and footprint gradients written once, per-Gaussian
    inputs and outputs once, tile instances written and read once (4 B
    index + 8 B key each way)."""
    return {
        "project": N * (12 + 12 + 16 + 4 + 192) + N * (48 + 16 + 8),
        "bin_sort": 24 * I,
        "render_fwd": P * (4 * D + 20) + U * (2 * D + 48),
        "render_bwd": P * (4 * D + 20) + U * (2 * D + 48) + U * (4 * D + 48),
        "project_bwd": N * (236 + 48) + N * (48 + 236),
    }


def copy_rates(dev, nbytes=1 << 30, reps=3):
    """Pinned host <-> device copy rates (GB/s, best of `reps`, CUDA events):
    host to device alone, device to host alone, and both at once on two
    streams (bytes of both directions over the time of both)."""
    import torch
    h_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d_a = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d_b = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def timed(fn):
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    def both():
        cur = torch.cuda.current_stream(dev)
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        with torch.cuda.stream(s1):
            d_a.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s2):
            h_out.copy_(d_b, non_blocking=True)
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    t_h2d = timed(lambda: d_a.copy_(h_in, non_blocking=True))
    t_d2h = timed(lambda: h_out.copy_(d_b, non_blocking=True))
    t_both = timed(both)
    del h_in, h_out, d_a, d_b
    return {"h2d_gbs": round(nbytes / (t_h2d * 1e-3) / 1e9, 1), "d2h_gbs": round(nbytes / (t_d2h * 1e-3) / 1e9, 1),
            "both_gbs": round(2 * nbytes / (t_both * 1e-3) / 1e9, 1), "bytes_each": nbytes,
            "how": "pinned host <-> device copies of 1 GiB, best of 3, CUDA events"}


def run_ours(args):
    import torch
    from paper_2505_19154_gb300 import api

    rank, world, local = dist_env()
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, cams, t, P = make_workload(rank, args.n, args.D, dev, args.width, args.height)
    path = {"tc": api.PATH_TC, "fp32": api.PATH_FP32, "auto": api.PATH_AUTO}[args.path]
    rast = api.Rasterizer(local, sh_degree=3, path=path, d_split=args.d_split, list_cut=args.list_cut)
    g = (t["means"], t["scales"], t["quats"], t["opacities"], t["sh"])
    st0 = rast.prepare(*g, cams)                      # sizes the instance buffer
    I = st0["n_instances"]
    rast.capacity = int(I * 1.05) + 1024
    del st0
    I_full = I
    if args.list_cut:  # the instance count of the full lists, for the record
        rf = api.Rasterizer(local, sh_degree=3, path=path, d_split=args.d_split, list_cut=0)
        I_full = rf.prepare(*g, cams)["n_instances"]
        del rf

    def step(rr):
        st = rr.prepare(*g, cams, check=False)
        rgb, feat = rr.forward(st, t["features"])
        grads = rr.backward(st, t["dC"], t["dF"])
        return st, rgb, feat, grads

    for _ in range(max(args.warmup, 1)):
        st_w, _, _, _ = step(rast)
    torch.cuda.synchronize()
    status = rast.ctx.sync_status()
    if status != api.OK:
        raise RuntimeError(f"device status {status} after warm-up")
    if args.profile_only:
        step(rast)
        torch.cuda.synchronize()
        return
    Q, Qpix, U = composited_pairs(st_w, cams)
    del st_w

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(rr, K, with_profile):
        clocks = ClockSampler(local)
        if with_profile:
            rr.ctx.profile(True)
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        n0 = api.Context.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            step(rr)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        launches = api.Context.launch_count() - n0
        ck = clocks.stop()
        ms = e0.elapsed_time(e1) / K
        prof = rr.ctx.profile_read() if with_profile else {}
        if with_profile:
            rr.ctx.profile(False)
        if world > 1:
            x = torch.tensor([ms], device=dev)
            torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
            ms = float(x.item())
        return ms, prof, launches, ck

    K = args.steps
    # per-kernel times from an eager, event-bracketed pass (the same kernels)
    ms_eager, prof, launches, clocks = timed(rast, K, True)
    if rast.ctx.sync_status() != api.OK:
        raise RuntimeError("device status after timed region")
    ms = ms_eager
    graph_note = "eager launches"
    if not args.no_graph:
        # the step as one CUDA graph (api.CapturedStep): projection, binning,
        # forward, backward and projection backward, replayed K times
        cstep = api.CapturedStep(rast, *g, t["features"], t["dC"], t["dF"], cams)
        for _ in range(max(args.warmup, 3)):
            cstep.replay()
        torch.cuda.synchronize()
        if rast.ctx.sync_status() != api.OK:
            raise RuntimeError("device status after the graph warm-up")
        gclk = ClockSampler(local)
        barrier()
        torch.cuda.synchronize()
        gclk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            cstep.replay()
        e1.record()
        torch.cuda.synchronize()
        barrier()
        clocks = gclk.stop()
        ms = e0.elapsed_time(e1) / K
        if world > 1:
            x = torch.tensor([ms], device=dev)
            torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
            ms = float(x.item())
        if rast.ctx.sync_status() != api.OK:
            raise RuntimeError("device status after the timed graph replays")
        del cstep
        graph_note = "one CUDA graph per step (api.CapturedStep); per-kernel times from the eager pass"
    value = P * world / (ms * 1e-3) / 1e6
    used_tc = any(k.endswith("_tc") for k in prof)

    # kernel-level roofline: the dominant kernel group, algorithmic bytes / its mean duration
    peaks = load_peaks()
    N, D = args.n, args.D
    algo = algorithmic_bytes(P, N, D, I, U)
    per = {}
    for name, (cnt, tot) in prof.items():
        base = name.replace("_tc", "").replace("_fp32", "")
        per[name] = dict(launches=cnt, ms=tot / max(cnt, 1), share=tot / max(1e-9, sum(v[1] for v in prof.values())),
                         bytes=algo.get(base))
    flops = algorithmic_flops(N, D, Q)
    for name, rec in per.items():
        base = name.replace("_tc", "").replace("_fp32", "")
        sec = rec["ms"] * 1e-3
        if rec["bytes"]:
            rec["hbm_frac"] = round(rec["bytes"] / sec / 1e9 / peaks["hbm"], 4)
        if base in flops and name.endswith("_tc"):
            rec["tensor_flops"] = flops[base]
            rec["tensor_frac"] = round(flops[base] / sec / 1e12 / peaks["bf16_sus"], 4)
    dom = max(per, key=lambda k: per[k]["ms"] * per[k]["launches"]) if per else None
    roof = None
    if dom and per[dom]["bytes"]:
        # the bound is the resource whose time at peak is longer for this
        # kernel's algorithmic work (HBM bytes vs tensor-core FLOPs)
        t_hbm = per[dom]["bytes"] / (peaks["hbm"] * 1e9)
        t_tc = per[dom].get("tensor_flops", 0) / (peaks["bf16_sus"] * 1e12)
        sec = per[dom]["ms"] * 1e-3
        src = "of measured" if peaks["src"] == "measured" else "of fallback"
        if t_tc > t_hbm:
            ach = per[dom]["tensor_flops"] / sec / 1e12
            roof = {"bound": "tensor", "kernel": dom, "achieved": round(ach, 1), "peak": peaks["bf16_sus"],
                    "unit": "TFLOP/s", "frac": round(ach / peaks["bf16_sus"], 4),
                    "peak_source": src + " (bf16_tflops_sustained)"}
        else:
            ach = per[dom]["bytes"] / sec / 1e9
            roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": peaks["hbm"], "unit": "GB/s",
                    "frac": round(ach / peaks["hbm"], 4), "peak_source": src + " (hbm_gbs)"}
        roof["traffic"] = traffic_for(dom)
        roof["algorithmic_bytes"] = per[dom]["bytes"]

    # FP32 CUDA-core path on the same inputs (the baseline the TC path must beat)
    fp32 = None
    if args.fp32_steps > 0 and used_tc:
        r32 = api.Rasterizer(local, sh_degree=3, path=api.PATH_FP32, list_cut=args.list_cut)
        r32.capacity = rast.capacity
        step(r32)
        torch.cuda.synchronize()
        ms32, prof32, _, _ = timed(r32, args.fp32_steps, True)
        fp32 = {"value": round(P * world / (ms32 * 1e-3) / 1e6, 2), "ms_per_step": round(ms32, 3),
                "kernels_ms": {k: round(v[1] / max(v[0], 1), 3) for k, v in prof32.items()}}
        del r32
        # the same algorithmic contraction FLOPs, on the CUDA cores, against
        # the measured FP32 FMA peak
        fpk = fp32_peak(dev, local)
        fl = algorithmic_flops(N, D, Q)
        fp32["fp32_peak"] = fpk
        fp32["alu_frac"] = {k: round(fl[k.replace("_fp32", "")] / (fp32["kernels_ms"][k] * 1e-3) / 1e12 /
                                     fpk["tflops"], 4)
                            for k in ("render_fwd_fp32", "render_bwd_fp32") if k in fp32["kernels_ms"]}

    # end to end through the C ABI with host buffers: H2D of every input and
    # D2H of every output inside the timed region
    e2e = None
    if not args.no_e2e:
        # host-resident inputs (pinned): every step copies all of them in and
        # all outputs out, overlapped with the neighbouring steps' compute
        h_in = {"means": t["means"], "scales": t["scales"], "quats": t["quats"], "opacities": t["opacities"],
                "sh": t["sh"], "features": t["features"], "grad_rgb": t["dC"], "grad_feat": t["dF"]}
        h_in = {k: v.cpu().pin_memory() for k, v in h_in.items()}
        pipe = api.HostPipeline(rast, cams, h_in)
        pipe.start()
        for _ in range(2):
            pipe.step()
        pipe.finish()
        torch.cuda.synchronize()
        bi, bo = pipe.bytes_per_step()
        Ke = max(3, min(K, 10))
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pipe.start()
        for _ in range(Ke):
            pipe.step()
        pipe.finish()
        e1.record()
        torch.cuda.synchronize()
        barrier()
        mse = e0.elapsed_time(e1) / Ke
        if world > 1:
            x = torch.tensor([mse], device=dev)
            torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
            mse = float(x.item())
        del pipe
        e2e = {"value": round(P * world / (mse * 1e-3) / 1e6, 2), "unit": UNIT, "ms_per_step": round(mse, 3),
               "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo)}
        # the link the end-to-end number is bound by: plain pinned copies of
        # 1 GiB alone in each direction and both directions together
        link = copy_rates(dev)
        e2e["link"] = link
        e2e["copy_floor_ms"] = round(max(bi / link["h2d_gbs"], bo / link["d2h_gbs"],
                                         (bi + bo) / link["both_gbs"]) / 1e6, 3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.n, args.D)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if used_tc else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if (args.width, args.height) == (1920, 1080) else
                       WORKLOAD.replace("1920x1080 view", f"{args.width}x{args.height} centre crop"),
                       "gaussians": N, "width": args.width, "height": args.height, "feature_dim": D,
                       "sh_degree": 3, "path": "tc" if used_tc else "fp32", "tile_instances": I,
                       "tile_instances_full_lists": I_full, "list_cut": bool(args.list_cut),
                       "composited_pairs_tile": Q, "composited_pairs_pixel": Qpix,
                       "gaussians_walked": U,
                       "l2": "inputs larger than L2 (features 1 GB, dL/dfeat 4.2 GB)",
                       "parallelism": f"independent views, {world} GPU(s)", "launch": graph_note,
                       "eager_ms_per_step": round(ms_eager, 3)},
            "roofline": roof, "kernels": per, "fp32_path": fp32, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clocks, "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- fusion
def device_feature_map(seed, view, height, width, D, dev, sigma=8.0):
    """The smooth feature map recipe (N(0,1) noise, separable Gaussian blur
    with a reflected border, per-pixel L2 normalisation) generated on the
    device with torch, for the fusion workload whose 64 maps (60 GB) are too
    large to make on the host.  [H*W, D] float32."""
    import math
    import torch
    import torch.nn.functional as Fn
    gen = torch.Generator(device=dev)
    gen.manual_seed(1_000_003 * (seed + 1) + view)
    x = torch.randn((D, height, width), generator=gen, device=dev)
    r = int(math.ceil(3 * sigma))
    k = torch.exp(-0.5 * (torch.arange(-r, r + 1, device=dev, dtype=torch.float32) / sigma) ** 2)
    k = k / k.sum()
    x = Fn.pad(x[None], (r, r, r, r), mode="reflect")[0]
    x = Fn.conv2d(x[:, None], k.view(1, 1, 1, -1))[:, 0]
    x = Fn.conv2d(x[:, None], k.view(1, 1, -1, 1))[:, 0]
    x = x.permute(1, 2, 0).reshape(height * width, D)
    return (x / x.norm(dim=1, keepdim=True).clamp_min(1e-12)).contiguous()


def run_fusion(args):
    import torch
    from paper_2505_19154_gb300 import api, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, views = synth.config5(rank)
    views = views[:args.views]
    D = 256
    g = tuple(torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev)
              for k in ("means", "scales", "quats", "opacities", "sh"))
    maps = [device_feature_map(rank, v, views[v]["height"], views[v]["width"], D, dev) for v in range(len(views))]
    path = {"tc": api.PATH_TC, "fp32": api.PATH_FP32, "auto": api.PATH_AUTO}[args.path]
    rast = api.Rasterizer(local, sh_degree=3, path=path, list_cut=args.list_cut)
    for _ in range(max(1, args.warmup)):
        rast.fuse(*g, views, maps)
    torch.cuda.synchronize()
    if rast.ctx.sync_status() != api.OK:
        raise RuntimeError("device status after warm-up")
    clocks = ClockSampler(local)
    rast.ctx.profile(True)
    clocks.start()
    n0 = api.Context.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = max(1, min(args.steps, 5))
    e0.record()
    for _ in range(K):
        out, num, den = rast.fuse(*g, views, maps)
    e1.record()
    torch.cuda.synchronize()
    launches = api.Context.launch_count() - n0
    ck = clocks.stop()
    prof = rast.ctx.profile_read()
    ms = e0.elapsed_time(e1) / K
    P = sum(v["width"] * v["height"] for v in views)
    N = len(scene["means"])
    algo = P * 4 * D + 2 * N * (4 * D + 4)  # maps read once, accumulators written once
    line = {"metric": f"feature fusion Mpix/s (3M Gaussians, {len(views)} views 1280x720, D=256 FP32 maps)",
            "value": round(P / (ms * 1e-3) / 1e6, 2), "unit": "Mpix/s", "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (maps generated on the device)",
            "config": {"workload": f"fusion: 3M Gaussians, {len(views)} views 1280x720, D=256", "views": len(views), "list_cut": bool(args.list_cut),
                       "gaussians": N, "seen": int((den > 0).sum().item())},
            "roofline": {"bound": "hbm", "achieved": round(algo / (ms * 1e-3) / 1e9, 1),
                         "peak": load_peaks()["hbm"], "unit": "GB/s",
                         "frac": round(algo / (ms * 1e-3) / 1e9 / load_peaks()["hbm"], 4),
                         "algorithmic_bytes": algo, "scope": "whole fusion call"},
            "kernels": {k: {"launches": c, "ms": round(t / max(c, 1), 4), "share": round(t / max(
                1e-9, sum(v[1] for v in prof.values())), 4)} for k, (c, t) in prof.items()},
            "clocks": ck, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- CPU oracle
def oracle_sample(scene, cams, D, seed=0):
    """One bounded oracle sample of the same workload: projection and FP32
    binning of every Gaussian, per-tile lists of the 64x64 crop's tiles,
    FP64 forward + backward of the crop's 4096 pixels."""
    import numpy as np
    import oracle
    from paper_2505_19154_gb300 import synth
    x0, y0, x1, y1 = synth.CROP3
    prm = dict(sh_degree=3)
    dC, dF = synth.upstream(seed, (x1 - x0) * (y1 - y0), D)
    prep = oracle.prepare(scene, cams, prm, tile_rect=(x0 // 16, y0 // 16, (x1 - 1) // 16, (y1 - 1) // 16))
    oracle.forward(scene, cams, prm, scene["features"], region=synth.CROP3, prep=prep)
    oracle.backward(scene, cams, prm, scene["features"], [dC], [dF], region=synth.CROP3, prep=prep)
    return (x1 - x0) * (y1 - y0)


def cpu_baseline(n, D, steps=3, warmup=1):
    """The oracle timed as `--impl reference` times it, in a fresh process
    (no CUDA context, no second OpenMP runtime, no sampler beside it): one
    untimed sample (which also loads the oracle's library), then `steps`
    timed ones of the same workload."""
    import subprocess
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", str(steps),
           "--warmup", str(warmup), "--n", str(n), "--D", str(D)]
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    t0 = time.time()
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"value": None, "unit": UNIT, "kind": "oracle", "error": (r.stderr or r.stdout)[-300:]}
    ref = lines[-1]
    return {"value": ref["value"], "unit": UNIT, "cores": ref["cpu_baseline"]["cores"], "kind": "oracle",
            "sample": f"{steps} x (project + FP32-spec binning of all {n} Gaussians, lists of the 64x64 crop's "
                      f"tiles, FP64 fwd+bwd of its 4096 pixels, D={D}), after {warmup} untimed sample(s), "
                      f"in a fresh process",
            "seconds": round(steps * ref["ms_per_step"] / 1e3, 2), "wall_s": round(time.time() - t0, 1)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2505_19154_gb300 import synth
    scene, cams = synth.config3(0, n=args.n, D=args.D)
    import oracle
    for _ in range(args.warmup):
        oracle_sample(scene, cams, args.D)
    t0 = time.time()
    px = 0
    for _ in range(args.steps):
        px += oracle_sample(scene, cams, args.D)
    dt = time.time() - t0
    v = px / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / max(args.steps, 1), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "gaussians": args.n, "width": 1920, "height": 1080,
                       "feature_dim": args.D, "sample": "64x64 crop per step"},
            "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(), "value": round(v, 6),
                             "sample": "each step: project + FP32-spec binning of all Gaussians, lists of the "
                                       "64x64 crop's tiles, FP64 fwd+bwd of its 4096 pixels"},
            "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------- point features
def run_points(args):
    """The paper's point-to-feature assignment over the fusion workload's
    3M points and 64 views (maps generated on the device), one call per step."""
    import torch
    from paper_2505_19154_gb300 import api, synth
    rank, world, local = dist_env()
    if world > 1 and rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, views = synth.config5(rank)
    views = views[:args.views]
    D = 256
    means = torch.from_numpy(np.ascontiguousarray(scene["means"], np.float32)).to(dev)
    N = means.shape[0]
    maps = [device_feature_map(rank, v, views[v]["height"], views[v]["width"], D, dev) for v in range(len(views))]
    gen = torch.Generator(device=dev)
    gen.manual_seed(5_000_011 + rank)
    u = torch.rand(N, generator=gen, device=dev)
    ctx = api.Context(local)
    params = api.make_params()
    W_ = max(3, args.warmup)
    for _ in range(W_):
        out, view, pixel = api.point_features(ctx, means, views, maps, u, params)
    torch.cuda.synchronize()
    if ctx.sync_status() != api.OK:
        raise RuntimeError("device status after warm-up")
    seen = int((view >= 0).sum().item())
    clocks = ClockSampler(local)
    ctx.profile(True)
    clocks.start()
    n0 = api.Context.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = max(1, args.steps)
    e0.record()
    for _ in range(K):
        api.point_features(ctx, means, views, maps, u, params)
    e1.record()
    torch.cuda.synchronize()
    launches = api.Context.launch_count() - n0
    ck = clocks.stop()
    prof = ctx.profile_read()
    ms = e0.elapsed_time(e1) / K
    kms = prof["point_features"][1] / max(prof["point_features"][0], 1)
    # means and u read, view and pixel and the feature rows written, the seen
    # points' map rows read: each once
    algo = N * (12 + 4 + 8 + 4 * D) + seen * 4 * D
    peaks = load_peaks()
    ach = algo / (kms * 1e-3) / 1e9
    line = {"metric": "point feature assignment Mpoints/s (3M points, 64 views 1280x720, D=256 FP32 maps)",
            "value": round(N / (ms * 1e-3) / 1e6, 2), "unit": "Mpoints/s", "n_gpus": 1, "steps": K, "warmup": W_,
            "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (maps generated on the device)",
            "config": {"workload": "point features: 3M points, 64 views 1280x720, D=256", "views": len(views),
                       "points": N, "seen": seen},
            "roofline": {"bound": "hbm", "kernel": "point_features", "achieved": round(ach, 1),
                         "peak": peaks["hbm"], "unit": "GB/s", "frac": round(ach / peaks["hbm"], 4),
                         "peak_source": ("of measured" if peaks["src"] == "measured" else "of fallback") +
                                        " (hbm_gbs)", "traffic": None, "algorithmic_bytes": algo},
            "kernels": {k: {"launches": c, "ms": round(t / max(c, 1), 4)} for k, (c, t) in prof.items()},
            "e2e": None, "cpu_baseline": None if args.no_cpu_baseline else points_cpu_baseline(means, views, maps, u),
            "clocks": ck, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


def points_cpu_baseline(means, views, maps, u, n_sample=3_000_000):
    """The oracle on the workload (the first n_sample points, all of them at
    3M) against all views (binary32 projection spec, one host thread), then
    their feature rows gathered from the maps by the oracle's own (view, pixel)."""
    import oracle
    m = means[:n_sample].cpu().numpy()
    uu = u[:n_sample].cpu().numpy()
    t0 = time.time()
    r = oracle.point_views(m, views, uu)
    rows = []
    for v in range(len(views)):
        sel = np.nonzero(r["view"] == v)[0]
        if len(sel):
            rows.append(maps[v][np.ascontiguousarray(r["pixel"][sel], np.int64)].cpu().numpy())
    dt = time.time() - t0
    return {"value": round(len(m) / dt / 1e6, 4), "unit": "Mpoints/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {len(m)} points against all {len(views)} views, rows gathered by the oracle's "
                      f"(view, pixel)", "seconds": round(dt, 2)}


# ------------------------------------------------------------------ NDFD
NDFD_METRIC = "NDFD L_gt+L_cf fwd+bwd Mpix/s at 1M Gaussians, D=512 BF16; % of roofline"
NDFD_WORKLOAD = "1M Gaussians, 1920x1080 view, D=512 BF16 unit features and ground-truth map, NDFD fwd+bwd"
def fp32_peak(dev, index=0, seconds=0.6):
    """Measured FP32 FMA peak: fhgs_ffma_probe (2 x 1024 threads per SM, eight
    independent FMA chains per thread) timed with CUDA events on the launch
    stream, best launch over about `seconds`, with the SM clock sampled
    meanwhile.  Also reports FLOP per clock per SM at the sampled clock (256
    when all 128 FP32 lanes of an SM retire an FMA every clock)."""
    import ctypes
    import torch
    from paper_2505_19154_gb300 import api
    L = api.lib()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    st = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(st.cuda_stream)
    blocks, iters = 2 * sms, 4000
    flops = L.fhgs_ffma_probe(blocks, iters, sp)
    if flops <= 0:
        raise RuntimeError("fhgs_ffma_probe failed")
    torch.cuda.synchronize()
    clk = ClockSampler(index)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best, n, t_end = float("inf"), 0, time.time() + seconds
    while n < 5 or time.time() < t_end:
        e0.record(st)
        L.fhgs_ffma_probe(blocks, iters, sp)
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
        n += 1
    ck = clk.stop()
    tf = flops / (best * 1e-3) / 1e12
    mhz = ck["sm_mhz"]
    return {"tflops": round(tf, 2), "launches": n, "ms": round(best, 4), "sm_mhz": mhz,
            "flop_per_clk_per_sm": round(tf * 1e12 / (mhz * 1e6) / sms, 1) if mhz else None,
            "source": "measured: fhgs_ffma_probe, best of the timed launches (CUDA events)"}


def ndfd_cpu_baseline(scene, cams, feats, fgt, dLgt, dLcf, max_seconds=25.0, reps_max=3):
    """The oracle on a bounded sample of the NDFD workload: projection and
    FP32 binning of every Gaussian, lists of the 64x64 crop's tiles, FP64
    NDFD forward and backward of its 4096 pixels (the features of the
    Gaussians those lists hold are gathered from the device each time)."""
    import torch
    import oracle
    from paper_2505_19154_gb300 import synth
    x0, y0, x1, y1 = synth.CROP3
    W = cams[0]["width"]
    pix = torch.tensor([y * W + x for y in range(y0, y1) for x in range(x0, x1)], device=fgt.device)
    fg = fgt[pix].float().cpu().numpy()
    a, b = dLgt[pix].cpu().numpy(), dLcf[pix].cpu().numpy()
    prm = dict(sh_degree=3)
    t0 = time.time()
    reps = 0
    while reps < reps_max and (reps == 0 or time.time() - t0 < max_seconds / 2):
        prep = oracle.prepare(scene, cams, prm, tile_rect=(x0 // 16, y0 // 16, (x1 - 1) // 16, (y1 - 1) // 16))
        uniq, inv = np.unique(prep["lists"]["gids"], return_inverse=True)
        idx = torch.from_numpy(np.ascontiguousarray(uniq, np.int64)).to(feats.device)
        fc = feats[idx].float().cpu().numpy()
        rec = prep["recs"][0][uniq]
        lists = inv.astype(np.uint32)
        ranges = oracle._cam_ranges(prep["lists"], 0)
        oracle.ndfd(rec, fc, lists, ranges, cams[0], prm, fg, region=synth.CROP3)
        oracle.ndfd_bwd(rec, fc, lists, ranges, cams[0], prm, synth.CROP3, fg, a, b)
        reps += 1
    dt = time.time() - t0
    return {"value": round(reps * (x1 - x0) * (y1 - y0) / dt / 1e6, 6), "unit": UNIT,
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{reps} x (project + FP32-spec binning of all {len(scene['means'])} Gaussians, lists of "
                      f"the 64x64 crop's tiles, FP64 NDFD fwd+bwd of its 4096 pixels)",
            "seconds": round(dt, 2)}


def run_ndfd(args):
    import torch
    from paper_2505_19154_gb300 import api, synth
    rank, world, local = dist_env()
    if world > 1 and rank != 0:
        return   # one view: the NDFD line is a single-GPU measurement
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, cams = synth.config3(rank, n=args.n, D=0)
    if (args.width, args.height) != (1920, 1080):
        cams = [dict(cams[0], width=args.width, height=args.height, cx=args.width / 2.0, cy=args.height / 2.0)]
    D = args.D
    g = tuple(torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev)
              for k in ("means", "scales", "quats", "opacities", "sh"))
    feats, fgt = synth.ndfd_inputs_device(rank, args.n, cams, D, dev)
    P = fgt.shape[0]
    gen = torch.Generator(device=dev)
    gen.manual_seed(9_000_011 + rank)
    dLgt = torch.randn(P, generator=gen, device=dev)
    dLcf = torch.randn(P, generator=gen, device=dev)
    rast = api.Rasterizer(local, sh_degree=3, list_cut=args.list_cut)
    st0 = rast.prepare(*g, cams)
    I = st0["n_instances"]
    rast.capacity = int(I * 1.05) + 1024
    nc = torch.empty(P, dtype=torch.int32, device=dev)
    rast.ndfd_forward(st0, feats, fgt, ncontrib=nc)
    C = int(nc.to(torch.int64).sum().item())   # (pixel, contributor) pairs
    del st0

    def step():
        st = rast.prepare(*g, cams, check=False)
        rast.ndfd_forward(st, feats, fgt, save_state=True)  # the backward reads the walk's end state
        rast.ndfd_backward(st, feats, fgt, dLgt, dLcf)

    W_ = max(3, args.warmup)
    for _ in range(W_):
        step()
    torch.cuda.synchronize()
    if rast.ctx.sync_status() != api.OK:
        raise RuntimeError("device status after warm-up")
    if args.profile_only:
        step()
        torch.cuda.synchronize()
        return
    clocks = ClockSampler(local)
    rast.ctx.profile(True)
    clocks.start()
    n0 = api.Context.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = max(1, args.steps)
    e0.record()
    for _ in range(K):
        step()
    e1.record()
    torch.cuda.synchronize()
    launches = api.Context.launch_count() - n0
    ck = clocks.stop()
    prof = rast.ctx.profile_read()
    if rast.ctx.sync_status() != api.OK:
        raise RuntimeError("device status after timed region")
    ms = e0.elapsed_time(e1) / K
    # algorithmic FLOPs per (pixel, contributor) pair: forward f_gt.f, F.f and
    # F += w f (3 x 2D); backward f_gt.f, F.f, G.f, F -= w f, G += s w f
    # (5 x 2D); the backward's front-to-back rebuild of F_N is not counted
    fk = "ndfd_fwd_tc" if "ndfd_fwd_tc" in prof else "ndfd_fwd"
    bk = "ndfd_bwd_tc" if "ndfd_bwd_tc" in prof else "ndfd_bwd"
    flops = {fk: 6 * D * C, bk: 10 * D * C}
    tot = sum(v[1] for v in prof.values())
    per = {k: {"launches": c, "ms": round(t / max(c, 1), 4), "share": round(t / max(tot, 1e-9), 4)}
           for k, (c, t) in prof.items()}
    for k, f in flops.items():
        if k in per:
            per[k]["algorithmic_tflops"] = round(f / (per[k]["ms"] * 1e-3) / 1e12, 2)
    dom = max((fk, bk), key=lambda k: prof.get(k, (0, 0))[1])
    ach = flops[dom] / (per[dom]["ms"] * 1e-3) / 1e12
    fpk = fp32_peak(dev)
    if dom.endswith("_tc"):
        pk = load_peaks()
        roof = {"bound": "tensor", "kernel": dom, "achieved": round(ach, 2), "peak": pk["bf16_sus"],
                "unit": "TFLOP/s", "frac": round(ach / pk["bf16_sus"], 4),
                "peak_source": f"of {pk['src']} (bf16_tflops_sustained)", "traffic": None,
                "algorithmic_flops": flops[dom], "fp32_alu_frac": round(ach / fpk["tflops"], 4), "fp32_peak": fpk,
                "note": "algorithmic dot-product FLOPs of the method; the kernel issues its per-chunk products "
                        "densely on tcgen05 and is bound by its CUDA-core weight passes and the cluster exchange"}
    else:
        roof = {"bound": "alu", "kernel": dom, "achieved": round(ach, 2), "peak": fpk["tflops"],
                "unit": "TFLOP/s", "frac": round(ach / fpk["tflops"], 4),
                "peak_source": "of measured FP32 FMA peak (fhgs_ffma_probe, this run)", "traffic": None,
                "algorithmic_flops": flops[dom], "fp32_peak": fpk}
    # the FP32 CUDA-core kernels on the same inputs, for comparison
    fp32_path = None
    if dom.endswith("_tc"):
        rast.set_path(api.PATH_FP32)
        step()
        torch.cuda.synchronize()
        rast.ctx.profile(True)
        rast.ctx.profile_read()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        for _ in range(2):
            step()
        f1.record()
        torch.cuda.synchronize()
        pf = rast.ctx.profile_read()
        rast.set_path(api.PATH_AUTO)
        fms = f0.elapsed_time(f1) / 2
        fp32_path = {"value": round(P / (fms * 1e-3) / 1e6, 2), "ms_per_step": round(fms, 3),
                     "kernels_ms": {k: round(t / max(c, 1), 3) for k, (c, t) in pf.items()}}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = ndfd_cpu_baseline(scene, cams, feats, fgt, dLgt, dLcf)
    line = {"metric": NDFD_METRIC, "value": round(P / (ms * 1e-3) / 1e6, 2), "unit": UNIT, "n_gpus": 1,
            "steps": K, "warmup": W_, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (NDFD inputs on the device)",
            "config": {"workload": NDFD_WORKLOAD, "gaussians": args.n, "width": args.width, "height": args.height, "list_cut": bool(args.list_cut),
                       "feature_dim": D, "tile_instances": I, "contributor_pairs": C,
                       "l2": "inputs larger than L2 (features 1 GB, ground-truth map 2.1 GB)",
                       "step": "project + bin/sort + NDFD forward + NDFD backward + projection backward"},
            "roofline": roof, "kernels": per, "fp32_path": fp32_path, "e2e": None, "cpu_baseline": cpu,
            "clocks": ck, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


BATCH_METRIC = "fwd+bwd Mpix/s, 16 cameras of uneven size in one captured CUDA graph, 500k Gaussians, D=256 BF16"
BATCH_WORKLOAD = ("500k Gaussians, 16 cameras W~U{640..1600} x H~U{480..900} on a ring, SH degree 3, "
                  "D=256 BF16 features, fwd+bwd replayed as one CUDA graph, autotuned D split")


def batched_cpu_baseline(scene, cams, D, ci=0, steps=3):
    """The oracle on a bounded sample of the batched workload: projection and
    FP32 binning of every Gaussian for camera ci, lists of the tiles of its
    64x64 centre crop, FP64 forward + backward of those 4096 pixels, after
    one untimed sample."""
    import oracle
    from paper_2505_19154_gb300 import synth
    cam = cams[ci]
    x0, y0 = (cam["width"] // 2 - 32) // 16 * 16, (cam["height"] // 2 - 32) // 16 * 16
    reg = (x0, y0, x0 + 64, y0 + 64)
    prm = dict(sh_degree=3)
    dC, dF = synth.upstream(ci, 64 * 64, D)

    def one():
        prep = oracle.prepare(scene, [cam], prm, tile_rect=(x0 // 16, y0 // 16, (x0 + 63) // 16, (y0 + 63) // 16))
        oracle.forward(scene, [cam], prm, scene["features"], region=reg, prep=prep)
        oracle.backward(scene, [cam], prm, scene["features"], [dC], [dF], region=reg, prep=prep)

    one()
    t0 = time.time()
    for _ in range(steps):
        one()
    dt = time.time() - t0
    return {"value": round(steps * 4096 / dt / 1e6, 6), "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": round(dt, 2),
            "sample": f"{steps} x (project + FP32-spec binning of all {len(scene['means'])} Gaussians for camera "
                      f"{ci}, lists of its 64x64 centre crop's tiles, FP64 fwd+bwd of the 4096 pixels, D={D}), "
                      f"after one untimed sample"}


def run_batched(args):
    """Config 4: the whole fwd+bwd step over 16 cameras of uneven size,
    captured once in a CUDA graph (api.CapturedStep) and replayed; the D
    split is chosen by the autotuner on this scene."""
    import torch
    from paper_2505_19154_gb300 import api, autotune, synth
    rank, world, local = dist_env()
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    D = 256
    scene, cams = synth.config4(rank, n=args.n if args.n != 1_000_000 else 500_000, D=D)
    t = {k: torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev)
         for k in ("means", "scales", "quats", "opacities", "sh")}
    t["features"] = torch.from_numpy(scene["features"]).to(dev).to(torch.bfloat16)
    P = sum(c["width"] * c["height"] for c in cams)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4000 + rank)
    dC = torch.randn((P, 3), generator=gen, device=dev)
    dF = torch.randn((P, D), generator=gen, device=dev)
    rast = api.Rasterizer(local, sh_degree=3, path=api.PATH_TC, list_cut=args.list_cut)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    rast.forward(st, t["features"])
    tuned = autotune.tune_splits(rast, st, t["features"], dC, dF, cams, use_cache=False)
    Q, Qpix, U = composited_pairs(st, cams)
    I = st["n_instances"]
    del st
    step = api.CapturedStep(rast, t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], t["features"],
                            dC, dF, cams)
    for _ in range(max(args.warmup, 3)):
        step.replay()
    torch.cuda.synchronize()
    if rast.ctx.sync_status() != api.OK:
        raise RuntimeError("device status after warm-up")
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    n0 = api.Context.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = max(1, args.steps)
    e0.record()
    for _ in range(K):
        step.replay()
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    per_replay = None  # kernels inside a graph are not counted by the library's host counter
    ms = e0.elapsed_time(e1) / K
    if world > 1:
        x = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
        ms = float(x.item())
    if rast.ctx.sync_status() != api.OK:
        raise RuntimeError("device status after timed region")
    # kernel split: one eager step with the same splits, timed per kernel group
    rast.ctx.profile(True)
    n1 = api.Context.launch_count()
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    rast.forward(st, t["features"])
    rast.backward(st, dC, dF)
    torch.cuda.synchronize()
    per_replay = api.Context.launch_count() - n1
    prof = rast.ctx.profile_read()
    rast.ctx.profile(False)
    tot = sum(v[1] for v in prof.values())
    peaks = load_peaks()
    N = len(scene["means"])
    algo = algorithmic_bytes(P, N, D, I, U)
    per = {}
    for k, (c, tm) in prof.items():
        sec = tm / max(c, 1) * 1e-3
        per[k] = {"launches": c, "ms": round(sec * 1e3, 4), "share": round(tm / max(tot, 1e-9), 4)}
        base = k.replace("_tc", "").replace("_fp32", "")
        if base in algo:
            per[k]["bytes"] = algo[base]
            per[k]["hbm_frac"] = round(algo[base] / sec / 1e9 / peaks["hbm"], 4)
    dom = max(prof, key=lambda k: prof[k][1])
    base = dom.replace("_tc", "")
    roof = None
    if base in algo:
        ach = algo[base] / (per[dom]["ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": peaks["hbm"], "unit": "GB/s",
                "frac": round(ach / peaks["hbm"], 4),
                "peak_source": ("of measured" if peaks["src"] == "measured" else "of fallback") + " (hbm_gbs)",
                "traffic": None, "algorithmic_bytes": algo[base]}
    e2e = None
    if not args.no_e2e and world == 1:
        h_in = {"means": t["means"], "scales": t["scales"], "quats": t["quats"], "opacities": t["opacities"],
                "sh": t["sh"], "features": t["features"], "grad_rgb": dC, "grad_feat": dF}
        h_in = {k: v.cpu().pin_memory() for k, v in h_in.items()}
        pipe = api.HostPipeline(rast, cams, h_in)
        pipe.start()
        for _ in range(2):
            pipe.step()
        pipe.finish()
        torch.cuda.synchronize()
        bi, bo = pipe.bytes_per_step()
        Ke = 3
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        pipe.start()
        for _ in range(Ke):
            pipe.step()
        pipe.finish()
        f1.record()
        torch.cuda.synchronize()
        mse = f0.elapsed_time(f1) / Ke
        del pipe, h_in
        e2e = {"value": round(P / (mse * 1e-3) / 1e6, 2), "unit": UNIT, "ms_per_step": round(mse, 3),
               "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo), "api": "api.HostPipeline (eager)"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = batched_cpu_baseline(scene, cams, D)
    if rank == 0:
        line = {"metric": BATCH_METRIC, "value": round(P * world / (ms * 1e-3) / 1e6, 2), "unit": UNIT,
                "n_gpus": world, "steps": K, "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                "data": "synthetic",
                "config": {"workload": BATCH_WORKLOAD, "gaussians": N, "cameras": len(cams), "pixels": P, "list_cut": bool(args.list_cut),
                           "feature_dim": D, "d_split": {"fwd": tuned["fwd"], "bwd": tuned["bwd"]},
                           "tile_instances": I, "composited_pairs_tile": Q, "composited_pairs_pixel": Qpix,
                           "gaussians_walked": U, "graph": "one CUDA graph per step (api.CapturedStep)",
                           "l2": "inputs larger than L2 (dL/dfeat 12.7 GB)",
                           "parallelism": f"independent view sets, {world} GPU(s)"},
                "roofline": roof, "kernels": per, "e2e": e2e, "cpu_baseline": cpu, "clocks": ck,
                "gpu_launches": int(per_replay) * K}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


SURFEL_METRIC = "fwd+bwd Mpix/s at 1M 2DGS surfels, 1080p, D=512 BF16 features, BF16-TC path; % of roofline"
SURFEL_WORKLOAD = ("1M 2DGS surfels (config-3 distributions, s_u, s_v the first two scales), 1920x1080 view, "
                   "SH degree 3, D=512 BF16 features, fwd+bwd")


def surfel_cpu_baseline(scene, cam, D, steps=2):
    """The oracle on a bounded sample of the surfel workload: binary32
    binning of every surfel, lists of the 64x64 crop's tiles, FP64 surfel
    forward + backward of its 4096 pixels with SH colour and features,
    after one untimed sample."""
    import oracle
    from paper_2505_19154_gb300 import synth
    x0, y0, x1, y1 = synth.CROP3
    prm = dict(sh_degree=3)
    sc = dict(scene, scales2=np.asarray(scene["scales"])[:, :2])
    dC, dF = synth.upstream(0, (x1 - x0) * (y1 - y0), D)

    def one():
        oracle.surfel_forward(sc, cam, prm, feats=scene["features"], region=synth.CROP3)
        oracle.surfel_backward(sc, cam, prm, dC, feats=scene["features"], dF=dF, region=synth.CROP3)

    one()
    t0 = time.time()
    for _ in range(steps):
        one()
    dt = time.time() - t0
    return {"value": round(steps * 4096 / dt / 1e6, 6), "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": round(dt, 2),
            "sample": f"{steps} x (binary32 binning of all {len(scene['means'])} surfels, lists of the 64x64 "
                      f"crop's tiles, FP64 surfel fwd+bwd of its 4096 pixels, D={D}), after one untimed sample"}


def run_surfel(args):
    """The 2DGS surfel geometry (Sec. 3.1) on the headline scene and view:
    projection, binning, forward and backward with the D-dim feature blend
    on the FP32 CUDA-core kernels."""
    import torch
    from paper_2505_19154_gb300 import api, synth
    rank, world, local = dist_env()
    if world > 1 and rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, cams, t, P = make_workload(rank, args.n, args.D, dev, args.width, args.height)
    D = args.D
    rast = api.Rasterizer(local, sh_degree=3, geometry=api.GEOM_SURFEL, list_cut=args.list_cut)
    g = (t["means"], t["scales"], t["quats"], t["opacities"], t["sh"])
    st0 = rast.prepare(*g, cams)
    I = st0["n_instances"]
    rast.capacity = int(I * 1.05) + 1024
    rast.forward(st0, t["features"])
    Q, Qpix, U = composited_pairs(st0, cams)
    del st0

    def step():
        st = rast.prepare(*g, cams, check=False)
        rast.forward(st, t["features"])
        rast.backward(st, t["dC"], t["dF"])

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if rast.ctx.sync_status() != api.OK:
        raise RuntimeError("device status after warm-up")
    if args.profile_only:
        step()
        torch.cuda.synchronize()
        return
    K = max(1, args.steps)
    rast.ctx.profile(True)
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    n0 = api.Context.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        step()
    e1.record()
    torch.cuda.synchronize()
    launches = api.Context.launch_count() - n0
    ck = clocks.stop()
    prof = rast.ctx.profile_read()
    if rast.ctx.sync_status() != api.OK:
        raise RuntimeError("device status after timed region")
    ms = e0.elapsed_time(e1) / K
    tot = sum(v[1] for v in prof.values())
    per = {k: {"launches": c, "ms": round(tm / max(c, 1), 4), "share": round(tm / max(tot, 1e-9), 4)}
           for k, (c, tm) in prof.items()}
    fl = algorithmic_flops(args.n, D, Q)
    fpk = fp32_peak(dev, local)
    fk = "render_fwd_tc_surfel" if "render_fwd_tc_surfel" in per else "render_fwd_surfel"
    bk = "render_bwd_tc_surfel" if "render_bwd_tc_surfel" in per else "render_bwd_surfel"
    by = algorithmic_bytes(P, args.n, D, I, U)
    pk = load_peaks()
    for k, base in ((fk, "render_fwd"), (bk, "render_bwd")):
        if k in per:
            per[k]["algorithmic_tflops"] = round(fl[base] / (per[k]["ms"] * 1e-3) / 1e12, 2)
            per[k]["bytes"] = by[base]
            per[k]["hbm_frac"] = round(by[base] / (per[k]["ms"] * 1e-3) / 1e9 / pk["hbm"], 4)
    dom = max((fk, bk), key=lambda k: prof.get(k, (0, 0))[1])
    base = "render_fwd" if dom == fk else "render_bwd"
    if "_tc_" in dom:  # the tensor-core kernels: HBM-bound by the image I/O, as for EWA
        achb = by[base] / (per[dom]["ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(achb, 1), "peak": pk["hbm"], "unit": "GB/s",
                "frac": round(achb / pk["hbm"], 4), "peak_source": f"of {pk['src']} (hbm_gbs)", "traffic": None,
                "algorithmic_bytes": by[base]}
    else:
        ach = fl[base] / (per[dom]["ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": round(ach, 2), "peak": fpk["tflops"], "unit": "TFLOP/s",
                "frac": round(ach / fpk["tflops"], 4),
                "peak_source": "of measured FP32 FMA peak (fhgs_ffma_probe, this run)", "traffic": None,
                "algorithmic_flops": fl[base], "fp32_peak": fpk}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = surfel_cpu_baseline(scene, cams[0], D)
    line = {"metric": SURFEL_METRIC, "value": round(P / (ms * 1e-3) / 1e6, 2), "unit": UNIT, "n_gpus": 1,
            "steps": K, "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": SURFEL_WORKLOAD, "gaussians": args.n, "width": cams[0]["width"], "list_cut": bool(args.list_cut),
                       "height": cams[0]["height"], "feature_dim": D, "tile_instances": I,
                       "composited_pairs_tile": Q, "composited_pairs_pixel": Qpix, "gaussians_walked": U,
                       "l2": "inputs larger than L2 (features 1 GB, dL/dfeat 4.2 GB)"},
            "roofline": roof, "kernels": per, "e2e": None, "cpu_baseline": cpu, "clocks": ck,
            "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


TRAIN_METRIC = "training iteration Mpix/s at 1M Gaussians, 1080p, NDFD D=512 BF16 (render + L1 + NDFD + Adam)"
TRAIN_WORKLOAD = ("1M Gaussians, 1920x1080 view, SH degree 3, D=512 BF16 frozen features and ground-truth map: "
                  "one Adam iteration of L = L_rgb + L_gt + L_cf")


def run_train(args):
    """One training iteration per step (App. A, Alg. 1 loop body; Sec. 3.3):
    projection, binning, RGB forward, L1, NDFD forward, render backward,
    NDFD backward, projection backward, Adam over both gradient sets -- the
    composed TrainStep over the library backend."""
    import torch
    from paper_2505_19154_gb300 import api, synth
    from paper_2505_19154_gb300.train import LibraryBackend, TrainStep
    rank, world, local = dist_env()
    if world > 1 and rank != 0:
        return   # one view: a single-GPU measurement
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, cams = synth.config3(rank, n=args.n, D=0)
    if (args.width, args.height) != (1920, 1080):  # centre crop of the same view: same focal length
        cams = [dict(cams[0], width=args.width, height=args.height, cx=args.width / 2.0, cy=args.height / 2.0)]
    cam = cams[0]
    D = args.D
    # raw parameters of the 3DGS family (host-side input preparation)
    raw = {"means": scene["means"], "log_scales": np.log(scene["scales"]), "quats": scene["quats"],
           "logit_opacities": np.log(scene["opacities"] / (1.0 - scene["opacities"])), "sh": scene["sh"]}
    raw = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev) for k, v in raw.items()}
    feats, fgt = synth.ndfd_inputs_device(rank, args.n, cams, D, dev)
    P = fgt.shape[0]
    gen = torch.Generator(device=dev)
    gen.manual_seed(9_100_003 + rank)
    target = torch.rand((P, 3), generator=gen, device=dev)
    be = LibraryBackend(local, sh_degree=3, list_cut=args.list_cut)
    act = be.activate(raw)
    st0 = be.rast.prepare(raw["means"], act["scales"], raw["quats"], act["opacities"], raw["sh"], [cam])
    be.rast.capacity = int(st0["n_instances"] * 1.2) + 1024   # room for the instances to grow as Adam moves them
    I = st0["n_instances"]
    del st0
    step = TrainStep(be, raw, 3, feats)
    W_ = max(args.warmup, 3)
    for _ in range(W_):
        step(cam, target, fgt)
    torch.cuda.synchronize()
    if be.rast.ctx.sync_status() != api.OK:
        raise RuntimeError("device status after warm-up")
    be.rast.ctx.profile(True)
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    n0 = api.Context.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = max(1, args.steps)
    e0.record()
    for _ in range(K):
        out = step(cam, target, fgt)
    e1.record()
    torch.cuda.synchronize()
    launches = api.Context.launch_count() - n0
    ck = clocks.stop()
    prof = be.rast.ctx.profile_read()
    if be.rast.ctx.sync_status() != api.OK:
        raise RuntimeError("device status after timed region")
    ms = e0.elapsed_time(e1) / K
    tot = sum(v[1] for v in prof.values())
    per = {k: {"launches": c, "ms": round(t / max(c, 1), 4), "share": round(t / max(tot, 1e-9), 4)}
           for k, (c, t) in prof.items()}
    dom = max(prof, key=lambda k: prof[k][1])
    losses = {k: round(float(out[k].item()), 6) for k in ("total", "rgb", "gt", "cf")}
    line = {"metric": TRAIN_METRIC, "value": round(P / (ms * 1e-3) / 1e6, 2), "unit": UNIT, "n_gpus": 1,
            "steps": K, "warmup": W_, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (NDFD inputs on the device)",
            "config": {"workload": TRAIN_WORKLOAD, "gaussians": args.n, "width": cam["width"], "list_cut": bool(args.list_cut),
                       "height": cam["height"], "feature_dim": D, "tile_instances_at_start": I,
                       "l2": "inputs larger than L2 (features 1 GB, ground-truth map 2.1 GB)",
                       "step": "activation + project + bin/sort + render fwd (RGB) + L1 + NDFD fwd + render bwd + "
                               "NDFD bwd + projection bwd (x2) + Adam"},
            "dominant_kernel": dom, "kernels": per, "losses_last_step": losses, "roofline": None,
            "e2e": None, "cpu_baseline": None, "clocks": ck, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "fusion":
        run_fusion(args)
    elif args.workload == "ndfd":
        run_ndfd(args)
    elif args.workload == "points":
        run_points(args)
    elif args.workload == "train":
        run_train(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "surfel":
        run_surfel(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
