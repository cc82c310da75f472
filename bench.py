#!/usr/bin/env python
"""Benchmark of the HEALPix Gaussian rasterizer training step on one B300.

Workload (the paper's training-step shape, Sec. 4): Nside 512 (3,145,728 px)
masked to a 190-degree equidistant fisheye (1,709,948 in-mask px), 300,000
Gaussians with SH degree 3, loss = (1 - 0.2) L1 + 0.2 (1 - HSSIM) against a
target map rendered from a perturbed copy of the scene. One step = forward
render + loss forward + loss backward + render backward (all §8 hot-path
stages). Metric: in-mask Mpix/s of fwd+bwd (higher is better).

`value` times the device path with inputs resident in HBM (CUDA events per
step, L2 flushed between steps). `e2e` times the same step through the public
API with the step's input, the 8-bit fisheye camera image of the target, copied
from pinned host memory and resampled onto the HEALPix grid inside the step,
and the loss read back every step. `--impl reference` (and `cpu_baseline`)
time the FP64 CPU oracle: the per-Gaussian work of a step in full, the
per-pixel work on a sample. `--oracle-full` times the oracle's whole step.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P_GAUSS = 300_000
K_ORDER = 9
FOV = 190.0
SEED = 20261205
WORKLOAD = "train_step_nside512_fisheye190_P300k_sh3"
IMG_SIDE = 1472          # the fisheye camera image of the end-to-end step (about the same pixel count as the mask)

SM_COUNT, FP32_LANES = 148, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # order-5 lists blended by 16 x 16 quarters: the same maps bit for bit as order 4, with about
    # half the pairs to list and sort
    ap.add_argument("--tile-level", type=int, default=5)
    ap.add_argument("--fwd-ppt", type=int, default=0)
    ap.add_argument("--bwd-ppt", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--no-multiview", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-resample", action="store_true")
    ap.add_argument("--no-query-compare", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=12000)
    ap.add_argument("--serve-sweep-s", type=float, default=10.0)
    ap.add_argument("--oracle-full", action="store_true",
                    help="time the FP64 oracle in full (all cores and one thread) and exit")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- ours
# The source file that defines each timed stage's kernel; a stage's recorded DRAM traffic stays
# valid while that file and the shared headers are unchanged.
STAGE_SOURCE = {"hssim_fwd": "hssim.cu", "hssim_bwd": "hssim.cu", "mask": "geometry.cu"}


def csrc_sha(stage=None):
    """Hash of the sources of a stage's kernel: its .cu file (raster.cu unless listed in
    STAGE_SOURCE), every header under csrc/ and the ABI header."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2606_29794_b300", "csrc")
    files = sorted(f for f in os.listdir(d) if f.endswith(".cuh"))
    files.append(STAGE_SOURCE.get(stage, "raster.cu"))
    for f in files:
        h.update(open(os.path.join(d, f), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "hpxgs.h"), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_stage):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, if the
    kernel's sources have not changed since it was taken (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(kernel_stage)
    if not e or e.get("csrc_sha") != csrc_sha(kernel_stage):
        return None
    return e.get("bytes_per_launch")


def run_ours(args, ws_n, rank, local):
    import numpy as np
    import torch

    from paper_2606_29794_b300 import _lib as L
    from paper_2606_29794_b300 import raster as R
    from paper_2606_29794_b300 import replicas as RP
    from paper_2606_29794_b300 import synth as S

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = L.lib()
    # ---------------- inputs (synthetic, seeded; each rank its own camera pose)
    sc = S.make_scene(P_GAUSS, 3, seed=SEED)
    tgt = S.perturb_scene(sc, SEED + 1)
    rot = RP.rank_rotation(rank, SEED)
    view = S.make_view(K_ORDER, S.CAM_FISHEYE, FOV, R=rot)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev)
    K = 16
    params = [t(sc["means"]), t(sc["scales"]), t(sc["rotations"]), t(sc["opacities"]), t(np.asarray(sc["sh"]).reshape(P_GAUSS, K, 3))]
    tparams = [t(tgt["means"]), t(tgt["scales"]), t(tgt["rotations"]), t(tgt["opacities"]), t(np.asarray(tgt["sh"]).reshape(P_GAUSS, K, 3))]
    rast = R.Rasterizer(tile_level=args.tile_level, fwd_ppt=args.fwd_ppt, bwd_ppt=args.bwd_ppt,
                        blocks_per_sm=args.blocks_per_sm)
    rast.prepare([view])
    stream = torch.cuda.current_stream(dev)
    with torch.no_grad():
        tout, _ = R.Rasterizer(tile_level=args.tile_level).forward_raw(*tparams, 3, [view])
    G = tout["maps"].clone()
    del tout
    # ---------------- one training step (forward, L1 + HSSIM forward and backward, backward) as a
    # CUDA graph; every stage's start and stop events are recorded inside the graph. Two instances
    # alternate, so one's stage events are read while the other runs: the host never idles the GPU.
    def new_pairs():
        pairs = {}
        for s in L.STAGES:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream); b.record(stream)              # torch creates the CUDA event on first record
            pairs[s] = (a, b)
        return pairs

    def arm(pairs):
        for i, s in enumerate(L.STAGES):
            a, b = pairs[s]
            L.check(lib.hpxgs_profile_arm(i, ctypes.c_void_p(a.cuda_event), ctypes.c_void_p(b.cuda_event)), "arm")

    stage_pairs = [new_pairs(), new_pairs()]
    gsteps = []
    for j in range(2):
        gsteps.append(R.GraphStep(params, 3, [view], G, rast, before_capture=lambda j=j: arm(stage_pairs[j])))
        # stages the captured step does not run are still armed: drop them and disarm, so that
        # later eager steps cannot record into this instance's events
        for i, s in enumerate(L.STAGES):
            if lib.hpxgs_profile_armed(i) == 1:
                stage_pairs[j].pop(s)
                L.check(lib.hpxgs_profile_arm(i, None, None), "disarm")
    gstep = gsteps[0]
    # ---------------- measured ALU peaks (FMA and MUFU probes at the current clocks), before the
    # warm-up so that the timed steps follow the warm-up steps directly
    fma_tf, ex2_t = ctypes.c_double(), ctypes.c_double()
    L.check(lib.hpxgs_probe_alu_peak(ctypes.byref(fma_tf), ctypes.byref(ex2_t), ctypes.c_void_p(stream.cuda_stream)),
            "alu probe")
    # ---------------- warm-up and capacity check
    for i in range(max(1, args.warmup)):
        gsteps[i % 2].replay()
    torch.cuda.synchronize()
    if any(int(g.status.item()) & L.F_CAPACITY for g in gsteps):
        raise RuntimeError("pair capacity exceeded after warm-up")
    n_mask = int(np.unpackbits(gstep.out["mask"].cpu().numpy().view(np.uint8)).sum())
    wv = R.workspace_view(rast, gstep.state)
    n_pairs = int(R.device_array(wv.n_pairs, 1, torch.int32).item())
    # ---------------- timed region (device path: graph replays, L2 flushed before each)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)     # > 126 MB L2
    stage_vals = {s: [] for s in L.STAGES}
    step_ms = []
    if ws_n > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    step_ev = []

    def read_stages(j):
        for s, (a, b) in stage_pairs[j].items():
            try:
                stage_vals[s].append(a.elapsed_time(b))
            except RuntimeError:
                pass

    for k in range(args.steps):
        j = k % 2
        if k >= 2:                      # step k-2 used this instance: read its stage events before it runs again
            step_ev[k - 2][1].synchronize()
            read_stages(j)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gsteps[j].replay()
        e1.record(stream)
        step_ev.append((e0, e1))
    torch.cuda.synchronize()
    for k in range(max(0, args.steps - 2), args.steps):
        read_stages(k % 2)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    launches = gstep.launches_per_replay * args.steps
    ms = RP.job_time_ms(sum(step_ms) / len(step_ms))          # slowest rank
    if ws_n > 1:
        torch.distributed.barrier()
    stage_ms = {s: sum(v) / len(v) for s, v in stage_vals.items() if v and sum(v) > 0}
    stage_source = "events recorded by the timed graph replays"
    if not any(s in stage_ms for s in ("blend_fwd", "blend_bwd")):
        # the graph did not record the stage events: time the stages in eager steps instead
        stage_source = "eager steps after the timed region"
        vals = {s: [] for s in L.STAGES}
        for _ in range(3):
            flush.zero_()
            evs = {}
            for i, s in enumerate(L.STAGES):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream); b.record(stream)
                L.check(lib.hpxgs_profile_arm(i, ctypes.c_void_p(a.cuda_event), ctypes.c_void_p(b.cuda_event)), "arm")
                evs[s] = (a, b)
            gsteps[0]._step()
            torch.cuda.synchronize()
            for i, (s, (a, b)) in enumerate(evs.items()):
                if lib.hpxgs_profile_armed(i) == 1:           # the step does not run this stage
                    L.check(lib.hpxgs_profile_arm(i, None, None), "disarm")
                    continue
                vals[s].append(a.elapsed_time(b))
        stage_ms = {s: sum(v) / len(v) for s, v in vals.items() if v and sum(v) > 0}
    n_eval = int(R.device_array(wv.n_eval, 1, torch.int64).item())
    n_contrib = int(R.device_array(wv.n_contrib, 1, torch.int64).item())
    n_job = RP.job_units(n_mask)                               # in-mask pixels of all ranks
    value = n_job / (ms * 1e-3) / 1e6
    # ---------------- roofline of the dominant kernel
    pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2032.0))
    alu_peak = SM_COUNT * FP32_LANES * 2 * sm_max * 1e6 / 1e12        # TFLOP/s FP32 at max SM clock
    hbm = float(pk.get("hbm_gbs", 6400.0))
    # ALU unit: a contributing (pixel, entry) pair (m <= cutoff, processed before termination)
    f_fwd = L.FLOPS_EVAL + L.FLOPS_FWD_CONTRIB
    f_bwd = L.FLOPS_EVAL + L.FLOPS_BWD_CONTRIB
    work = {
        "blend_fwd": ("alu", f_fwd * n_contrib / 1e12, "TFLOP/s", alu_peak),
        "blend_bwd": ("alu", f_bwd * n_contrib / 1e12, "TFLOP/s", alu_peak),
        "pair_sort": ("hbm", 20.0 * n_pairs * math.ceil(math.log2(12 * 4 ** (K_ORDER - args.tile_level)) / 8) / 1e9, "GB/s", hbm),
        "depth_sort": ("hbm", 20.0 * P_GAUSS * 4 / 1e9, "GB/s", hbm),
        "preprocess": ("hbm", (236 + 64 + 16) * P_GAUSS / 1e9, "GB/s", hbm),
        "hssim_fwd": ("hbm", 60.0 * n_mask / 1e9, "GB/s", hbm),
        # parameters and partials in, parameter gradients out, per Gaussian
        "preprocess_bwd": ("hbm", (236 + 36 + 4 + 236) * P_GAUSS / 1e9, "GB/s", hbm),
        # staged member list read (4 B) and (tile, id) written (8 B) per pair; count, offset, slot per Gaussian
        "tile_emit": ("hbm", (12.0 * n_pairs + 16.0 * P_GAUSS) / 1e9, "GB/s", hbm),
        # sorted tile ids read per pair, [start, end) written per tile
        "ranges": ("hbm", (4.0 * n_pairs + 8.0 * 12 * 4 ** (K_ORDER - args.tile_level)) / 1e9, "GB/s", hbm),
        "hssim_bwd": ("hbm", 72.0 * n_mask / 1e9, "GB/s", hbm),
    }
    if not any(s in work for s in stage_ms):
        raise RuntimeError(f"no stage timings recorded: {stage_ms}")
    # every HBM-bound stage against the measured copy bandwidth (algorithmic bytes / stage time)
    hbm_stages = {}
    for st_name, (bnd, amount, unit, pk_) in work.items():
        if bnd == "hbm" and st_name in stage_ms:
            gbs = amount / (stage_ms[st_name] * 1e-3)
            hbm_stages[st_name] = {"ms": round(stage_ms[st_name], 4), "algorithmic_bytes": int(round(amount * 1e9)),
                                   "gbs": round(gbs, 1), "frac_of_hbm": round(gbs / pk_, 3)}
    dom = max((s for s in stage_ms if s in work), key=lambda s: stage_ms[s])
    bound, amount, unit, peak = work[dom]
    achieved = amount / (stage_ms[dom] * 1e-3)
    traffic = ncu_traffic(dom)
    roofline = {"kernel": dom, "bound": bound, "achieved": round(achieved, 3), "peak": round(peak, 1), "unit": unit,
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": ("derived: 148 SM x 128 FP32 lanes x 2 x max SM clock" if bound == "alu"
                                else "measured (MEASURED_PEAKS.json hbm_gbs)")}
    if bound == "alu":
        roofline.update({
            "unit_of_work": f"contributing (pixel, entry) pair, {f_fwd if dom == 'blend_fwd' else f_bwd} FP32 flops each",
            "peak_measured_fma": round(fma_tf.value, 1), "frac_of_measured_fma": round(achieved / fma_tf.value, 4),
            "mufu_measured_tops": round(ex2_t.value, 2)})
    # ---------------- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        from paper_2606_29794_b300 import resample as RS
        # the step's input as a camera delivers it: the 8-bit fisheye image of the target (the
        # perturbed scene's render resampled to 1472 x 1472 and quantised), in pinned host memory.
        # Every replay copies it in on a forked stream (overlapping the forward render) and
        # resamples it onto the HEALPix grid as the target (Eq. supp_image_to_healpix); the loss
        # is read back to pinned host memory.
        img, _ = RS.sphere_to_image_raw(G, K_ORDER, view, IMG_SIDE, IMG_SIDE)
        img8 = torch.round(img.clamp(0.0, 1.0) * 255.0).to(torch.uint8)
        host_img = torch.empty(img8.shape, dtype=torch.uint8, pin_memory=True)
        host_img.copy_(img8.cpu())
        hloss = torch.empty(1, dtype=torch.float32, pin_memory=True)
        estep = R.GraphStep(params, 3, [view], torch.empty_like(G), R.Rasterizer(tile_level=args.tile_level),
                            host_images=[host_img])
        # the same step fed the float image v / 255 already on the device: the loss must agree
        fimg = img8.float() / 255.0
        Gf = torch.empty_like(G)
        RS.image_to_sphere_into(fimg, view, K_ORDER, Gf)
        fstep = R.GraphStep(params, 3, [view], Gf, R.Rasterizer(tile_level=args.tile_level))
        fstep.replay()
        for _ in range(2):
            estep.replay(); hloss.copy_(estep.losses[0, :1], non_blocking=True)
        torch.cuda.synchronize()
        loss_f = float(fstep.losses[0, 0].item())
        del fstep
        ev = []
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            estep.replay()
            hloss.copy_(estep.losses[0, :1], non_blocking=True)
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        e_ms = RP.job_time_ms(sum(a.elapsed_time(b) for a, b in ev) / len(ev))
        e2e = {"value": round(n_job / (e_ms * 1e-3) / 1e6, 2), "unit": "Mpix/s",
               "h2d_bytes_per_step": int(host_img.numel()), "d2h_bytes_per_step": 4, "ms_per_step": round(e_ms, 4),
               "input": f"8-bit fisheye camera image {IMG_SIDE} x {IMG_SIDE} x 3 (pinned host), resampled onto the "
                        f"HEALPix grid inside the step",
               "loss": float(hloss.item()), "loss_float_image_path": loss_f,
               "loss_matches_float_image_path": bool(abs(float(hloss.item()) - loss_f) <= 2e-6)}
        del estep
    npix_full = 12 * 4 ** K_ORDER
    res = {
        "metric": "Mpix/s fwd+bwd at Nside 512/300k Gaussians (L1+HSSIM training step)",
        "value": round(value, 2), "unit": "Mpix/s", "n_gpus": ws_n, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "step_ms_min_median_max": [round(min(step_ms), 4), round(sorted(step_ms)[len(step_ms) // 2], 4),
                                   round(max(step_ms), 4)],
        "dtype": "f32", "data": "synthetic (seeded Gaussians shaped like the paper's scenes)",
        "config": {"workload": WORKLOAD, "nside": 512, "camera": "fisheye 190 deg", "in_mask_px": n_mask,
                   "gaussians": P_GAUSS, "sh_degree": 3, "tile_level": args.tile_level,
                   "blend_unit_px": 256 if args.tile_level == 5 else 4 ** args.tile_level, "loss": "0.8 L1 + 0.2 (1-HSSIM)",
                   "l2": "flushed (256 MB write) before every timed step", "step": "CUDA graph replay",
                   "parallelism": f"replicas x{ws_n}, no collective",
                   "pairs": n_pairs, "pairs_up_to_termination": n_eval, "contrib": n_contrib},
        "full_grid_mpix_s": round(RP.job_units(npix_full) / (ms * 1e-3) / 1e6, 2),
        "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "stage_timing": stage_source,
        "roofline": roofline,
        "hbm_stages": hbm_stages,
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": e2e,
    }
    return res


# ----------------------------------------------------------------------------- other workloads
def _tensors(sc, dev):
    import numpy as np
    import torch
    P = sc["means"].shape[0]
    K = (sc["sh_degree"] + 1) ** 2
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev)
    return [t(sc["means"]), t(sc["scales"]), t(sc["rotations"]), t(sc["opacities"]), t(np.asarray(sc["sh"]).reshape(P, K, 3))]


def _time_replays(run, steps, dev, flush):
    import torch
    evs = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(); run(); b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / len(evs)


def run_multiview(args, dev):
    """16 views of uneven size (6 pinhole 90 deg @ Nside 1024, 6 fisheye 180 deg @ 512, 4 full @ 256),
    1M SH3 Gaussians, fwd + per-view L1/HSSIM + bwd in one batched call per stage, captured in a CUDA
    graph after autotuning the launch parameters."""
    import numpy as np
    import torch
    from paper_2606_29794_b300 import raster as R
    from paper_2606_29794_b300 import synth as S
    sc = S.make_scene(1_000_000, 3, seed=SEED + 1)
    tgt = S.perturb_scene(sc, SEED + 2)
    views = S.multiview_set(SEED + 3)
    params = _tensors(sc, dev)
    with torch.no_grad():
        tout, _ = R.Rasterizer().forward_raw(*_tensors(tgt, dev), 3, views)
    targets = tout["maps"].clone()
    n_mask = int(np.unpackbits(tout["mask"].cpu().numpy().view(np.uint8)).sum())
    del tout
    torch.cuda.empty_cache()
    cands = [dict(tile_level=4), dict(tile_level=3), dict(tile_level=5), dict(tile_level=4, blocks_per_sm=2),
             dict(tile_level=4, fwd_ppt=2)]
    built = {}

    def make(kw):
        built.clear()
        torch.cuda.empty_cache()
        st = R.GraphStep(params, 3, views, targets, R.Rasterizer(**kw))
        built["s"] = st
        return st.replay
    best, timings = R.autotune(make, cands, reps=3, warmup=1)
    built.clear()
    torch.cuda.empty_cache()
    step = R.GraphStep(params, 3, views, targets, R.Rasterizer(**best))
    for _ in range(args.warmup):
        step.replay()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ms = _time_replays(step.replay, args.steps, dev, flush)
    st = int(step.status.item())
    res = {"workload": "16 views (6 pinhole 90@1024, 6 fisheye 180@512, 4 full@256), 1M SH3, fwd+L1/HSSIM+bwd",
           "in_mask_px": n_mask, "ms_per_step": round(ms, 3), "mpix_per_s": round(n_mask / (ms * 1e-3) / 1e6, 1),
           "autotuned": best, "candidates_ms": {k: round(v, 3) for k, v in timings.items()},
           "cuda_graph": True, "status": st}
    del step
    torch.cuda.empty_cache()
    return res


def run_serving(args, dev):
    """Poisson request streams against a resident 3M SH3 scene: continuous batching against one
    request at a time (plain), p50/p99 latency, throughput and mean batch. The saturation run is
    the 400 req/s stream (12,000 requests, 30 s, by default); the sweep offers both modes the
    same rates from 80 to 160 req/s, where the highest rate each sustains with p99 < 250 ms is
    read off."""
    import torch
    from paper_2606_29794_b300 import serve as SV
    from paper_2606_29794_b300 import synth as S
    sc = S.make_scene(3_000_000, 3, seed=SEED + 4)
    params = _tensors(sc, dev)
    reqs = S.request_stream(args.serve_requests, 400.0, seed=SEED + 5)
    srv = SV.RenderServer(params, 3, budget_bytes=32 << 30, slots=3, max_views=8)
    warm = S.request_stream(16, 400.0, seed=SEED + 6)
    srv.run(warm)
    limit = max(60.0, 4.0 * len(reqs) / 400.0)
    batched, _ = srv.run(reqs, time_limit_s=limit)
    torch.cuda.empty_cache()
    plain, _ = srv.run(reqs, plain=True, time_limit_s=limit)
    torch.cuda.empty_cache()
    out = {"workload": f"{len(reqs)} requests, Poisson 400 req/s, Nside 128-2048, pinhole 60-100 / fisheye 180-220 / full, "
                       "3M SH3 Gaussians resident",
           "batched": batched.summary(), "plain": plain.summary()}
    # the same offered rates for both modes (10 s streams)
    sweep = {"batched": {}, "plain": {}}
    rates = (80.0, 100.0, 120.0, 140.0, 160.0)
    for rate in rates:
        n = int(rate * args.serve_sweep_s)
        rq = S.request_stream(n, rate, seed=SEED + 7)
        for mode in ("batched", "plain"):
            st, _ = srv.run(rq, plain=(mode == "plain"), time_limit_s=3.0 * args.serve_sweep_s)
            sweep[mode][str(int(rate))] = st.summary()
            torch.cuda.empty_cache()
    out["rate_sweep"] = sweep
    for mode in ("batched", "plain"):
        ok = [r for r in rates if sweep[mode][str(int(r))]["p99_ms"] < 250.0
              and sweep[mode][str(int(r))]["served"] == int(r * args.serve_sweep_s)]
        out[f"max_sustainable_rps_p99_lt_250ms_{mode}"] = max(ok) if ok else None
    return out


def run_large(args, dev):
    """Nside 2048 full sphere, 6M SH3 Gaussians (log-scales N(-3.5, 0.7)), fwd + L1/HSSIM + bwd with
    recomputation from T_final and the last index (no blend history)."""
    import numpy as np
    import torch
    from paper_2606_29794_b300 import raster as R
    from paper_2606_29794_b300 import synth as S
    sc = S.make_scene(6_000_000, 3, seed=SEED + 8, logscale_mu=-3.5, logscale_sd=0.7)
    tgt = S.perturb_scene(sc, SEED + 9)
    view = S.make_view(11)
    params = _tensors(sc, dev)
    with torch.no_grad():
        tparams = _tensors(tgt, dev)
        tout, tstate = R.Rasterizer(tile_level=args.tile_level).forward_raw(*tparams, 3, [view])
    targets = tout["maps"].clone()
    del tout, tstate, tparams
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats(dev)
    base = torch.cuda.memory_allocated(dev)                     # scene parameters and targets
    step = R.GraphStep(params, 3, [view], targets, R.Rasterizer(tile_level=args.tile_level))
    for _ in range(max(1, args.warmup)):
        step.replay()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ms = _time_replays(step.replay, max(3, args.steps // 2), dev, flush)
    npx = 12 * 4 ** 11
    peak = torch.cuda.max_memory_allocated(dev)
    wv = R.workspace_view(step.rast, step.state)
    n_eval = int(R.device_array(wv.n_eval, 1, torch.int64).item())
    n_pairs = int(R.device_array(wv.n_pairs, 1, torch.int32).item()) & 0xffffffff
    res = {"workload": "Nside 2048 full sphere (50,331,648 px), 6M SH3 Gaussians, fwd+L1/HSSIM+bwd",
           "ms_per_step": round(ms, 3), "mpix_per_s": round(npx / (ms * 1e-3) / 1e6, 1),
           "pairs": n_pairs, "pair_capacity": int(step.rast.capacity), "pairs_up_to_termination": n_eval,
           "step_workspace_bytes": int(step.state["nb"]),
           "peak_gpu_bytes_above_inputs": int(peak - base),
           "peak_note": "includes the eager warm-up steps GraphStep runs before capture and the graph's own pool",
           "per_pixel_state_bytes": 8, "per_pixel_state_total_bytes": 8 * npx,
           "blend_history_estimate_bytes": 8 * n_eval,
           "blend_history_note": "alpha and T per processed (pixel, entry) pair, the least a backward without "
                                 "recomputation would keep",
           "status": int(step.status.item())}
    del step
    torch.cuda.empty_cache()
    return res


def run_resample(args, dev):
    """Sphere <-> image resampling (Eq. camera_synthesis; Eq. supp_image_to_healpix) at matched resolutions:
    fisheye 190 deg 1472^2 at Nside 512, pinhole 90 deg 2048^2 and a 4096 x 2048 panorama at Nside 1024.
    Algorithmic bytes: sphere -> image writes the image (12 B/px) and validity (1 B/px) and reads the map
    region it covers once (12 B per in-mask map pixel); the adjoint reads the image gradient and writes the
    whole map gradient (zero fill + accumulation of the covered region); image -> sphere reads the image
    once and writes the whole map (12 B/px) and its mask bits."""
    import numpy as np
    import torch
    from paper_2606_29794_b300 import _lib as L
    from paper_2606_29794_b300 import resample as RS
    from paper_2606_29794_b300 import synth as S
    hbm = float(peaks().get("hbm_gbs", 6400.0))
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    cases = [("fisheye190_1472x1472_nside512", {"cam": S.CAM_FISHEYE, "fov_x": 190.0, "fov_y": 190.0}, 9, 1472, 1472),
             ("pinhole90_2048x2048_nside1024", {"cam": S.CAM_PINHOLE, "fov_x": 90.0, "fov_y": 90.0}, 10, 2048, 2048),
             ("panorama_4096x2048_nside1024", {"cam": S.CAM_FULL, "fov_x": 360.0, "fov_y": 180.0}, 10, 4096, 2048)]
    out = {}
    g = torch.Generator(device=dev).manual_seed(SEED + 20)
    for name, cam, k, W, H in cases:
        npix = 12 * 4 ** k
        hmap = torch.rand((npix, 3), device=dev, generator=g)
        img = torch.rand((H, W, 3), device=dev, generator=g)
        _, words = RS.image_to_sphere(img, cam, k)
        n_in = int(np.unpackbits(words.cpu().numpy().view(np.uint8)).sum())
        ops = {
            "sphere_to_image": (lambda: RS.sphere_to_image_raw(hmap, k, cam, W, H), 13 * W * H + 12 * n_in),
            "sphere_to_image_backward": (lambda: RS.sphere_to_image_backward(img, k, cam, W, H), 12 * W * H + 12 * npix + 12 * n_in),
            "image_to_sphere": (lambda: RS.image_to_sphere(img, cam, k), 12 * W * H + 12 * npix + npix // 8),
        }
        # the same through resampling plans (the taps built once per camera): the taps an application
        # reads (32 B per output pixel with taps, plus the validity or mask) count as its bytes
        ps = RS.Plan(L.PLAN_SPHERE_TO_IMAGE, cam, k, W, H)
        pi = RS.Plan(L.PLAN_IMAGE_TO_SPHERE, cam, k, W, H)
        pimg, pval = torch.empty_like(img), torch.empty((H, W), dtype=torch.uint8, device=dev)
        pmap, pwords = torch.empty_like(hmap), torch.empty(npix // 32, dtype=torch.int32, device=dev)
        ps.sphere_to_image(hmap, pimg, pval)
        n_val = int(pval.sum().item())                    # image pixels inside D_C: the ones with taps
        ops["sphere_to_image_planned"] = (lambda: ps.sphere_to_image(hmap, pimg, pval),
                                          13 * W * H + 12 * n_in + W * H + 32 * n_val)
        ops["sphere_to_image_backward_planned"] = (lambda: ps.sphere_to_image_backward(img),
                                                   12 * W * H + 12 * npix + 12 * n_in + W * H + 32 * n_val)
        ops["image_to_sphere_planned"] = (lambda: pi.image_to_sphere(img, pmap, pwords),
                                          12 * W * H + 12 * npix + npix // 4 + 32 * n_in)
        res = {"in_mask_map_px": n_in, "image_px": W * H, "valid_image_px": n_val,
               "plan_bytes": {"sphere_to_image": ps.nbytes, "image_to_sphere": pi.nbytes}}
        for op, (fn, nbytes) in ops.items():
            for _ in range(3):
                fn()
            ms = _time_replays(fn, max(5, args.steps), dev, flush)
            gbs = nbytes / (ms * 1e-3) / 1e9
            res[op] = {"ms": round(ms, 4), "bytes": int(nbytes), "gbs": round(gbs, 1), "frac_of_hbm": round(gbs / hbm, 3)}
        out[name] = res
    return out


def run_query_compare(args, dev):
    """Tile query variants on the training-step workload (Sec. 3.3): RING (Algorithm 3) at the tile
    order (the default) and at search resolution x2 and x4 (Sec. D.2), against the NESTED quadtree
    search (Algorithm 2) refined x1, x2, x4. All list every tile the cutoff ellipse reaches, so the
    step computes the same maps; reported:
    the query stages (count + emit, CUDA events), the whole step (graph replays), and the whole
    step under the literal tile semantics (infinite cutoff), where the maps depend on the query."""
    import numpy as np
    import torch
    from paper_2606_29794_b300 import _lib as L
    from paper_2606_29794_b300 import raster as R
    from paper_2606_29794_b300 import synth as S
    lib = L.lib()
    sc = S.make_scene(P_GAUSS, 3, seed=SEED)
    view = S.make_view(K_ORDER, S.CAM_FISHEYE, FOV)
    params = _tensors(sc, dev)
    with torch.no_grad():
        G = R.Rasterizer(tile_level=4).forward_raw(*_tensors(S.perturb_scene(sc, SEED + 1), dev), 3, [view])[0]["maps"].clone()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    modes = [("ring", dict(query=L.QUERY_RING)), ("ring_x2", dict(query=L.QUERY_RING, query_log2f=1)),
             ("ring_x4", dict(query=L.QUERY_RING, query_log2f=2)),
             ("nested_x1", dict(query=L.QUERY_NESTED, query_log2f=0)),
             ("nested_x2", dict(query=L.QUERY_NESTED, query_log2f=1)), ("nested_x4", dict(query=L.QUERY_NESTED, query_log2f=2))]
    out = {}
    for name, kw in modes:
        rast = R.Rasterizer(tile_level=4, **kw)
        rast.prepare([view])
        qs = []
        for rep in range(6):
            flush.zero_()
            ev = {}
            for st in ("tile_count", "tile_emit"):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream); b.record(stream)
                L.check(lib.hpxgs_profile_arm(L.STAGES.index(st), ctypes.c_void_p(a.cuda_event), ctypes.c_void_p(b.cuda_event)), "arm")
                ev[st] = (a, b)
            o, _ = rast.forward_raw(*params, 3, [view])
            torch.cuda.synchronize()
            if rep:
                qs.append(sum(a.elapsed_time(b) for a, b in ev.values()))
        wv_pairs = None
        step = R.GraphStep(params, 3, [view], G, rast)
        for _ in range(3):
            step.replay()
        ms = _time_replays(step.replay, max(5, args.steps // 2), dev, flush)
        wv = R.workspace_view(rast, step.state)
        wv_pairs = int(R.device_array(wv.n_pairs, 1, torch.int32).item())
        del step
        torch.cuda.empty_cache()
        # the paper's literal tile semantics (no m <= 9 cutoff: every listed pixel receives a
        # contribution, so the image depends on the query), the setting of its ablation
        lstep = R.GraphStep(params, 3, [view], G, R.Rasterizer(tile_level=4, cutoff=math.inf, **kw))
        for _ in range(3):
            lstep.replay()
        ms_lit = _time_replays(lstep.replay, max(5, args.steps // 2), dev, flush)
        del lstep
        torch.cuda.empty_cache()
        out[name] = {"query_ms": round(float(np.mean(qs)), 4), "step_ms": round(ms, 4), "pairs": wv_pairs,
                     "step_ms_literal": round(ms_lit, 4)}
    for name in out:
        if name != "ring":
            out[name]["query_time_vs_ring"] = round(out[name]["query_ms"] / out["ring"]["query_ms"], 2)
            out[name]["literal_step_vs_ring"] = round(out[name]["step_ms_literal"] / out["ring"]["step_ms_literal"], 2)
    # the ablation's pairing: both queries at the x4 search resolution, literal tile semantics
    out["nested_x4_over_ring_x4_literal_step"] = round(out["nested_x4"]["step_ms_literal"] / out["ring_x4"]["step_ms_literal"], 2)
    out["nested_x4_over_ring_x4_query"] = round(out["nested_x4"]["query_ms"] / out["ring_x4"]["query_ms"], 2)
    out["paper_claim"] = ("RING about 1.7x faster than NESTED (Sec. 3.3, Table ablation: R(x4) 28.2 min vs D(x4) 49.1 min "
                          "of end-to-end training, ratio 1.74)")
    return out


# ----------------------------------------------------------------------------- oracle
def cpu_info():
    model = None
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model}


_ORACLE_WL = {}


def oracle_workload():
    """The training-step workload as the oracle takes it (built once per process)."""
    if not _ORACLE_WL:
        import numpy as np

        import oracle as O
        from paper_2606_29794_b300 import synth as S
        sc = S.make_scene(P_GAUSS, 3, seed=SEED)
        view = S.make_view(K_ORDER, S.CAM_FISHEYE, FOV)
        cfg = O.Config(tile_level=4)
        m, _ = O.mask(2 ** K_ORDER, view["cam"], FOV)
        _ORACLE_WL.update(
            sc=sc, tgt=S.perturb_scene(sc, SEED + 1), cfg=cfg, mask=m,
            v64=dict(view, W=np.asarray(view["W"], np.float64), b=np.asarray(view["b"], np.float64)),
            active=O.active_tiles(K_ORDER, cfg.tile_level, m), rho=O.tile_rho(K_ORDER, cfg.tile_level),
            pix=np.nonzero(m)[0].astype(np.int64))
    return _ORACLE_WL


# Share of the active tiles on which the reference arm's sampled oracle step runs its
# per-pixel work (cpu_baseline times the whole step).
ORACLE_FRAC = 0.2


def oracle_step(frac, seed=0):
    """One L1 + HSSIM training step of the FP64 oracle on the training-step workload.

    Work that does not scale with the pixels runs in full: preprocess of the scene and of the
    target scene, their tile lists over every active tile (Algorithm 3), and the backward's
    per-Gaussian chain (its preprocess and the chain to the parameters, timed as a backward over
    one pixel). The per-pixel work (compositing of both scenes, the HSSIM loss and gradient, the
    backward blend) runs on the in-mask pixels of a random `frac` of the active tiles, taken as
    runs of 16 neighbouring tiles (so that the sample keeps the full run's locality: a tile's
    pixels share one list, neighbouring tiles share Gaussians) and is scaled by the in-mask pixels of the step over those of the sample; frac = 1 is the
    whole step, timed as it runs. Returns the seconds of each part and the step estimate."""
    import numpy as np

    import oracle as O
    W = oracle_workload()
    sc, tgt, cfg, v64, m, act, rho, pix = (W[k] for k in ("sc", "tgt", "cfg", "v64", "mask", "active", "rho", "pix"))
    b = cfg.tile_level
    rng = np.random.default_rng(seed)
    if frac >= 1.0:
        sel = pix
    else:
        # runs of 16 consecutive active tiles (NESTED order: 4 x 4 squares of tiles), so that the
        # sample also keeps the sharing of Gaussians between neighbouring tiles
        tiles = np.nonzero(act)[0]
        nrun = max(1, int(round(frac * tiles.size / 16)))
        starts = rng.choice(tiles.size // 16, nrun, replace=False) * 16
        pick = tiles[(starts[:, None] + np.arange(16)[None, :]).ravel()]
        sel = pix[np.isin(pix >> (2 * cfg.tile_level), pick)]
    msel = m
    if frac < 1.0:
        msel = np.zeros_like(m)
        msel[sel] = 1
    t0 = time.perf_counter()
    pre = O.preprocess(sc, v64, cfg)
    pre_t = O.preprocess(tgt, v64, cfg)
    st, ids = O.tile_lists(K_ORDER, b, pre["g"], pre["rs"], pre["valid"], O.depth_bits(pre["r"]), rho, act)
    st_t, ids_t = O.tile_lists(K_ORDER, b, pre_t["g"], pre_t["rs"], pre_t["valid"], O.depth_bits(pre_t["r"]), rho, act)
    t1 = time.perf_counter()
    img = O.composite(K_ORDER, b, pre, sc["opacities"], st, ids, sel, cfg)[0]
    timg = O.composite(K_ORDER, b, pre_t, tgt["opacities"], st_t, ids_t, sel, cfg)[0]
    t2 = time.perf_counter()
    N = O.npix(2 ** K_ORDER)
    I = np.zeros((N, 3)); G = np.zeros((N, 3))
    I[sel] = img; G[sel] = timg
    # the loss over the sampled pixels' windows: the same work per pixel as over the whole mask
    _, _, _, dI = O.hssim_loss(2 ** K_ORDER, I, G, msel, cfg.lam)
    t3 = time.perf_counter()
    O.backward(sc, v64, cfg, dI[sel], st, ids, sel)
    t4 = time.perf_counter()
    parts = {"fixed_fwd_s": t1 - t0, "composite_s": t2 - t1, "hssim_s": t3 - t2, "backward_s": t4 - t3}
    if frac >= 1.0:
        est = t4 - t0
    else:
        O.backward(sc, v64, cfg, dI[sel[:1]], st, ids, sel[:1])
        b0 = time.perf_counter() - t4                       # the backward's per-Gaussian part
        parts["backward_fixed_s"] = b0
        est = (t1 - t0) + b0 + ((t2 - t1) + (t3 - t2) + max(0.0, (t4 - t3) - b0)) / (sel.size / pix.size)
    parts.update(step_s=est, sampled_px=int(sel.size), in_mask_px=int(pix.size))
    return parts


def _oracle_record(parts_list, frac):
    import oracle as O
    est = sum(p["step_s"] for p in parts_list) / len(parts_list)
    nmask = parts_list[0]["in_mask_px"]
    mean = lambda k: round(sum(p.get(k, 0.0) for p in parts_list) / len(parts_list), 3)
    return est, {"value": round(nmask / est / 1e6, 6), "unit": "Mpix/s", "cores": O.num_threads(), "kind": "oracle",
                 "cpu": cpu_info(),
                 "sample": (f"FP64 oracle (C++/OpenMP), one training step per sample: preprocess of both scenes, "
                            f"tile lists over every active tile and the backward's per-Gaussian chain in full; "
                            f"compositing of both scenes, HSSIM loss + gradient and the backward blend on the "
                            f"in-mask px of a random {frac:.4f} of the active tiles (runs of 16 neighbouring tiles), "
                            f"scaled to the {nmask} in-mask px"),
                 "parts_s": {k: mean(k) for k in ("fixed_fwd_s", "composite_s", "hssim_s", "backward_s",
                                                  "backward_fixed_s")},
                 "step_s": round(est, 3)}


def cpu_baseline():
    """One whole training step of the FP64 oracle, timed in full (no sampling)."""
    oracle_workload()
    _, rec = _oracle_record([oracle_step(1.0)], 1.0)
    rec["sample"] = ("the whole training step of the FP64 oracle (C++/OpenMP), timed in full: preprocess and tile "
                     "lists of both scenes, compositing of both scenes over every in-mask pixel, the HSSIM loss and "
                     "gradient, the backward")
    return rec


def run_reference(args):
    oracle_workload()
    frac = ORACLE_FRAC
    for i in range(args.warmup):
        oracle_step(frac, seed=1000 + i)
    parts = [oracle_step(frac, seed=i) for i in range(args.steps)]
    est, cb = _oracle_record(parts, frac)
    value = cb["value"]
    return {"impl": "reference", "metric": "Mpix/s fwd+bwd at Nside 512/300k Gaussians (L1+HSSIM training step)",
            "value": value, "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(est * 1e3, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_oracle_full(args):
    """The FP64 oracle timed in full: the plain forward render of Nside 64 with 2,000 SH0
    Gaussians, and the whole training step at Nside 512 (fisheye 190 deg, 300k SH3), each at
    every core and at one thread; beside them the sampled model of the same step."""
    import numpy as np

    import oracle as O
    from paper_2606_29794_b300 import synth as S
    ncore = O.num_threads()
    out = {"cpu": cpu_info(), "threads_all": ncore}
    sc1 = S.make_scene(2000, 0, seed=20261204)
    v1 = S.make_view(6)
    v1 = dict(v1, W=np.asarray(v1["W"], np.float64), b=np.asarray(v1["b"], np.float64))
    oracle_workload()
    frac = ORACLE_FRAC
    for th in (ncore, 1):
        O.set_threads(th)
        t = time.perf_counter()
        O.render(sc1, v1, O.Config())
        c1 = time.perf_counter() - t
        full = oracle_step(1.0)
        model = oracle_step(frac, seed=7)
        out[f"threads_{th}"] = {
            "forward_nside64_p2k_s": round(c1, 4), "forward_nside64_p2k_mpix_s": round(49152 / c1 / 1e6, 4),
            "train_step_full_s": round(full["step_s"], 2), "train_step_full_mpix_s": round(full["in_mask_px"] / full["step_s"] / 1e6, 6),
            "train_step_full_parts_s": {k: round(v, 3) for k, v in full.items() if k.endswith("_s") and k != "step_s"},
            "train_step_model_s": round(model["step_s"], 2), "model_frac": round(frac, 4),
            "model_over_full": round(model["step_s"] / full["step_s"], 3)}
    O.set_threads(ncore)
    return out


def main():
    args = parse()
    ws_n, rank, local = dist_env()
    if args.oracle_full:
        if rank == 0:
            print(json.dumps(run_oracle_full(args)))
        return 0
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)))
        return 0
    if ws_n > 1:
        import torch
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, ws_n, rank, local)
    if rank == 0 and ws_n == 1:
        import torch
        dev = torch.device("cuda", local)
        if not args.no_resample:
            res["resample"] = run_resample(args, dev)
        if not args.no_query_compare:
            res["tile_query"] = run_query_compare(args, dev)
        if not args.no_multiview:
            res["multiview"] = run_multiview(args, dev)
        if not args.no_large:
            res["large"] = run_large(args, dev)
        if not args.no_serving:
            res["serving"] = run_serving(args, dev)
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(res))
    if ws_n > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
