"""Benchmark of the time-domain Lienard-Wiechert path on GB300.

One step = one pass of the whole path over the synthetic workload:
trajectory relayout (lw_trajectories_upload, device-resident FP64 inputs),
time map + field + interpolated deposit (lw_deposit_time_domain) and the
per-pixel FFT spectrum (lw_spectrum).  The headline is the mixed path
(FP64-exact bin coordinates, FP32 field and accumulation); the FP64 path is
timed beside it and the mixed spectrum is compared with the FP64 one.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  For N > 1 (torchrun) the detector's pixels are
split into one contiguous block per rank (the paper's detector parallelization,
strong scaling: the whole job is one detector); every rank holds all
trajectories and the same observer grid, and no collective touches the data
path -- a barrier and a MAX over ranks bracket the timing.  ``--shard detectors``
gives every rank a detector of its own instead (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LW deposits/s (electron·step·pixel), mixed vs FP64 at ≤1e-4 spectrum error"
UNIT = "deposits/s"
WORKLOAD = ("c2_paper: 10,000 electrons (Gaussian bunch 5x5x10 um, gamma 60 +-0.1%, "
            "eps_n 0.5 mm mrad) x 10,000 Boris steps in a Gaussian laser (0.8 um, a0 0.5, "
            "w0 20 um, 30 fs) x 64x64 pixels over +-1.5/gamma; 65,536 observer bins")


# ----------------------------------------------------------------------------- helpers

def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in a thread."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _source_hash(path):
    """Hash of a CUDA source's code: comments removed and whitespace collapsed, so that a
    profile keyed to it stays valid across comment edits and goes stale on code edits."""
    with open(path) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = " ".join(src.split())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def _traffic_from_profile(kernel_src):
    """Per-launch DRAM bytes of the deposit kernel from the committed ncu summary,
    valid only if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "deposit_mixed_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_sha256_16") != _source_hash(kernel_src):
        return None
    return d.get("bytes_per_launch_full_size")


def grid_points_reached(t, r, det, grid, chunk=256):
    """Grid points deposited by the whole workload: per (pixel, electron), the points of
    (floor(u_first), floor(u_last)] inside [0, n_bins), u = (t_a - t_min)/dt_u of the
    trajectory's first and last sample (FP64, torch on the device; bookkeeping only)."""
    import torch
    c0 = 299792458.0
    t0 = t[0] if t.dim() == 1 else t[:, 0]
    t1 = t[-1] if t.dim() == 1 else t[:, -1]
    r0, r1 = r[:, 0, :], r[:, -1, :]
    total = 0
    for m0 in range(0, det.n_pix, chunk):
        n = det.n_hat[m0:m0 + chunk]
        u0 = ((t0 - (r0 @ n.T).T / c0) - grid.t_min) / grid.dt_u
        u1 = ((t1 - (r1 @ n.T).T / c0) - grid.t_min) / grid.dt_u
        j0 = torch.clamp(torch.floor(u0) + 1, min=0)
        j1 = torch.clamp(torch.floor(u1), max=grid.n_bins - 1)
        total += int(torch.clamp(j1 - j0 + 1, min=0).sum().item())
    return total


# Work of one mixed deposit launch (Algorithm 2 as the kernel evaluates it), per unit:
#   per grid point reached: two FP32 fields (29 flops each), the interpolation of three
#   components (9), its weight (5) and the two sample coordinates that bracket the step
#   (7 each): 86 flops; the two staged samples it reads: 2 x (16 B coordinate data + 24 B
#   field data) = 80 B of shared memory; its update of the record: one L2 reduction
#   (LW_MIXED_F32X4: x, y, z in one 16-byte vector) or three (the other records);
#   per pixel and block of samples: the double-FP32 anchor, 47 flops;
#   per launch from HBM: the mixed trajectory section once (40 B per sample, 32 B per
#   anchor) and the record once (three components per pixel and grid point).
FLOPS_PER_POINT = 86
FLOPS_PER_PIXEL_BLOCK = 47
SMEM_BYTES_PER_POINT = 80


def deposit_work(n_e, n_s, n_pix, n_bins, block, n_points, precision):
    """Algorithmic work of one mixed deposit launch (see the model above)."""
    from paper_2206_03015_gb300 import lw
    ns1 = n_s + 1
    n_blocks = -(-ns1 // block)
    step_blocks = -(-(ns1 - 1) // block)          # blocks that hold steps
    rec_word = 8 if precision in (lw.LW_MIXED, lw.LW_MIXED_KAHAN) else 4
    return {
        "grid_points": n_points,
        "pixel_blocks": n_pix * n_e * step_blocks,
        "hbm_bytes": n_e * (ns1 * (16 + 24) + n_blocks * 32) + n_pix * 3 * n_bins * rec_word,
        "l2_ops": n_points * (1 if precision == lw.LW_MIXED_F32X4 else 3),
        "fp32_flops": n_points * FLOPS_PER_POINT + n_pix * n_e * step_blocks * FLOPS_PER_PIXEL_BLOCK,
        "smem_bytes": n_points * SMEM_BYTES_PER_POINT,
    }


def deposit_roofline(work, kernel_ms, pipe_peaks, hbm_gbs, traffic=None):
    """Each bound's achieved rate (work / kernel time), peak and fraction; the binding one
    (largest fraction) is the headline."""
    t = kernel_ms * 1e-3
    l2 = pipe_peaks["red_v4f32_lines"]["ops_per_s"]
    bounds = {
        "hbm": {"achieved": work["hbm_bytes"] / t / 1e9, "peak": hbm_gbs, "unit": "GB/s"},
        "l2_red": {"achieved": work["l2_ops"] / t / 1e9, "peak": l2 / 1e9, "unit": "Gop/s"},
        "fp32": {"achieved": work["fp32_flops"] / t / 1e12,
                 "peak": pipe_peaks["fma_f32"]["flops"] / 1e12, "unit": "TFLOP/s"},
        "smem": {"achieved": work["smem_bytes"] / t / 1e9,
                 "peak": pipe_peaks["lds_v4"]["bytes_per_s"] / 1e9, "unit": "GB/s"},
    }
    for b in bounds.values():
        b["frac"] = b["achieved"] / b["peak"]
    bound = max(bounds, key=lambda k: bounds[k]["frac"])
    out = {"bound": bound, "achieved": bounds[bound]["achieved"], "peak": bounds[bound]["peak"],
           "unit": bounds[bound]["unit"], "frac": bounds[bound]["frac"],
           "traffic": traffic, "kernel": "deposit_mixed_kernel", "kernel_ms": kernel_ms,
           "bounds": bounds, "work": work}
    return out


# ----------------------------------------------------------------------------- workload

def shard_pixels(n_pix, rank, world, shard="pixels"):
    """[lo, hi) of the detector's pixels this rank deposits: one contiguous block of the
    detector per rank (Sec. 4.2, detector parallelization), or all of them when every
    rank observes a detector of its own (``shard == "detectors"``)."""
    from paper_2206_03015_gb300 import parallel
    if world == 1 or shard == "detectors":
        return 0, n_pix
    return parallel.pixel_shard(n_pix, rank, world)


def job_deposits(n_e, n_s, n_pix, world, shard="pixels"):
    """Deposits of the whole job (all ranks): one detector, or one per rank."""
    return n_e * n_s * n_pix * (world if shard == "detectors" else 1)


def make_workload(args, rank):
    from workloads import configs
    w = configs.c2_paper(n_e=args.n_e, n_s=args.n_s, nx=args.nx, n_bins=args.n_bins)
    if rank > 0 and args.shard == "detectors":
        # weak scaling: rank r observes its own detector, rotated about the beam axis
        ang = rank * 2.0 * math.pi / max(args.world, 1) * 0.5
        c, s = math.cos(ang), math.sin(ang)
        n = w.n_hat.copy()
        w.n_hat = np.stack([c * n[:, 0] - s * n[:, 1], s * n[:, 0] + c * n[:, 1], n[:, 2]], -1)
    return w


# ----------------------------------------------------------------------------- our arm

def run_ours(args, rank, world, dist):
    import torch

    from paper_2206_03015_gb300 import lw

    dev = torch.device("cuda", _env_int("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    t_gen = time.time()
    w = make_workload(args, rank)
    t_gen = time.time() - t_gen
    tr = w.traj
    # device-resident FP64 inputs
    t_d = torch.from_numpy(tr.t).to(dev)
    r_d = torch.from_numpy(tr.r).to(dev)
    b_d = torch.from_numpy(tr.beta).to(dev)
    a_d = torch.from_numpy(tr.beta_dot).to(dev)
    # grid (Eqs. tu_min, tu_max) once, from the whole detector, so that every rank's
    # pixel block shares it; it is fixed for the workload
    traj0 = lw.lw_trajectories_upload(t_d, r_d, b_d, a_d, sections=lw.LW_SECTION_MIXED,
                                      block=args.block, device=dev)
    bnd = lw.lw_grid_bounds(traj0, lw.Detector(w.n_hat, device=dev)).cpu().numpy()
    grid = lw.grid_from_bounds(bnd[0], bnd[1], w.n_bins)
    p_lo, p_hi = shard_pixels(w.n_pix, rank, world, args.shard)
    w.n_hat = np.ascontiguousarray(w.n_hat[p_lo:p_hi])
    w.theta_x, w.theta_y = w.theta_x[p_lo:p_hi], w.theta_y[p_lo:p_hi]
    det = lw.Detector(w.n_hat, device=dev)
    n_dep = w.deposits                                     # this rank's deposits
    n_job = job_deposits(tr.n_e, tr.n_s, w.n_pix if args.shard == "detectors" else
                         args.nx * args.nx, world, args.shard)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    # the timed mixed path: FP32 record (LW_MIXED_F32) by default, FP64 record with --mixed f64
    MIX = {"f32": lw.LW_MIXED_F32, "x4": lw.LW_MIXED_F32X4, "f64": lw.LW_MIXED}[args.mixed]
    shp, dt = lw.record_shape(det, grid, MIX)
    rec_m = torch.empty(shp, dtype=dt, device=dev)
    S_m = torch.empty((det.n_pix, grid.n_bins // 2 + 1), dtype=torch.float32, device=dev)
    ws_s = lw.workspace(lw.spectrum_workspace_bytes(MIX, det.n_pix, grid), dev)
    ws_t = traj0.ws
    ev_dep = []

    def step_mixed(timed=False):
        traj = lw.lw_trajectories_upload(t_d, r_d, b_d, a_d, sections=lw.LW_SECTION_MIXED,
                                         block=args.block, device=dev, ws=ws_t)
        if timed:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
        lw.lw_deposit_time_domain(traj, det, grid, MIX, record=rec_m, status=status)
        if timed:
            e1.record()
            ev_dep.append((e0, e1))
        lw.lw_spectrum(rec_m, MIX, det.n_pix, grid, ws=ws_s, out=S_m)

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed_loop(fn, steps, warmup, sampler=None, streams=()):
        for _ in range(warmup):
            fn(False)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record()
        cur = torch.cuda.current_stream(dev)
        for s in streams:   # side streams start after s0 ...
            s.wait_stream(cur)
        for _ in range(steps):
            fn(True)
        for s in streams:   # ... and s1 follows all of their work
            cur.wait_stream(s)
        s1.record()
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        barrier()
        ms = s0.elapsed_time(s1)
        if dist is not None:
            x = torch.tensor([ms], dtype=torch.float64, device=dev)
            dist.all_reduce(x, op=dist.ReduceOp.MAX)
            ms = float(x.item())
        return ms, clocks

    from paper_2206_03015_gb300 import peaks
    pipe_peaks = peaks.measure(dev)   # rates of the deposit's pipes on this GPU
    sampler = ClockSampler(dev.index)
    ms_m, clocks = timed_loop(step_mixed, args.steps, args.warmup, sampler)
    ms_step = ms_m / args.steps
    dep_ms = statistics.mean(a.elapsed_time(b) for a, b in ev_dep)
    value = n_job / (ms_step * 1e-3)
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak" if args.shard == "detectors" else "strong", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.full else f"c2_paper reduced: {args.n_e} e x "
                   f"{args.n_s} steps x {args.nx}x{args.nx} px, {args.n_bins} bins",
                   "n_e": tr.n_e, "n_s": tr.n_s, "n_pix": w.n_pix, "n_bins": w.n_bins,
                   "deposits_per_step_per_gpu": n_dep, "block": args.block,
                   "precision": {lw.LW_MIXED_F32: "LW_MIXED_F32 (FP32 record)",
                                 lw.LW_MIXED_F32X4: "LW_MIXED_F32X4 (FP32 record, x/y/z "
                                                    "interleaved per grid point)",
                                 lw.LW_MIXED: "LW_MIXED (FP64 record)"}[MIX],
                   "l2": "inputs larger than L2 (mixed trajectory section %.1f GB)"
                         % (traj0.ws.numel() / 1e9),
                   "parallelism": (f"detector parallelization: one detector per GPU x{world}"
                                   if args.shard == "detectors" else
                                   f"detector parallelization: pixels {p_lo}..{p_hi - 1} of "
                                   f"one detector on each of {world} GPU(s)"),
                   "deposits_per_step_job": n_job,
                   "generation_s": round(t_gen, 1)},
    }
    # roofline of the dominant kernel (the mixed deposit): the work of one launch by the
    # model in deposit_work(), against pipe peaks measured on this GPU just before the
    # timed region (HBM: the copy bandwidth recorded in MEASURED_PEAKS.json)
    hbm_peak, peak_src = 6800.0, "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak, peak_src = float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        pass
    n_points = grid_points_reached(t_d, r_d, det, grid)
    work = deposit_work(tr.n_e, tr.n_s, w.n_pix, w.n_bins, args.block, n_points, MIX)
    traffic = _traffic_from_profile(os.path.join(ROOT, "paper_2206_03015_gb300", "csrc",
                                                 "lw_deposit.cu"))
    result["roofline"] = deposit_roofline(work, dep_ms, pipe_peaks, hbm_peak, traffic)
    result["roofline"]["peak_source"] = (f"{peak_src} HBM copy (MEASURED_PEAKS.json hbm_gbs); "
                                         "L2 reductions, FP32 FMA and shared loads measured "
                                         "in this run (paper_2206_03015_gb300/peaks)")
    result["clocks"] = clocks
    # the other records beside it: FP64 (LW_MIXED) and compensated FP32 pairs
    # (LW_MIXED_KAHAN), each the same step with that record
    for prec2, key in ((lw.LW_MIXED, "mixed_fp64_record"), (lw.LW_MIXED_KAHAN, "mixed_kahan_record")):
        if prec2 == MIX:
            continue
        shp2, dt2 = lw.record_shape(det, grid, prec2)
        rec_2 = torch.empty(shp2, dtype=dt2, device=dev)
        S_2 = torch.empty_like(S_m)

        def step_mixed2(timed=False, prec2=prec2, rec_2=rec_2, S_2=S_2):
            traj = lw.lw_trajectories_upload(t_d, r_d, b_d, a_d, sections=lw.LW_SECTION_MIXED,
                                             block=args.block, device=dev, ws=ws_t)
            lw.lw_deposit_time_domain(traj, det, grid, prec2, record=rec_2, status=status)
            lw.lw_spectrum(rec_2, prec2, det.n_pix, grid, ws=ws_s, out=S_2)

        ms_2, _ = timed_loop(step_mixed2, args.steps, args.warmup)
        result[key] = {"ms_per_step": ms_2 / args.steps,
                       "value": n_job / (ms_2 / args.steps * 1e-3)}
        del rec_2, S_2
    torch.cuda.synchronize()
    st_m = int(status.item())

    # end to end through the C ABI from pinned host buffers, spectrum read back. The
    # electrons are streamed in chunks over four streams: host-to-device copies of a
    # chunk's FP64 inputs into one of two device staging slots (the host link, about
    # 211 GB/s on this machine, is the bound: 7.2 GB per step), the relayout of the
    # previous chunk into one of two mixed workspaces, the deposit of the one before
    # (accumulated into the step's record), and per step the spectrum and its copy back
    # to pinned host memory. Records and spectra alternate between steps, so a step's
    # spectrum and read-back overlap the next step's copies; every step's inputs cross
    # the link and its spectrum comes back inside the timed region.
    if not args.no_e2e:
        h = [torch.from_numpy(x).pin_memory() for x in (tr.t, tr.r, tr.beta, tr.beta_dot)]
        n_ch = max(1, min(args.e2e_chunks, tr.n_e))
        bounds_e = [tr.n_e * c // n_ch for c in range(n_ch + 1)]
        big = max(bounds_e[c + 1] - bounds_e[c] for c in range(n_ch))
        t_shared = h[0].dim() == 1
        stage = []
        for _ in range(2):
            d_t = torch.empty((big,) + tuple(h[0].shape[1:]) if not t_shared else h[0].shape,
                              dtype=torch.float64, device=dev)
            stage.append([d_t] + [torch.empty((big,) + tuple(x.shape[1:]), dtype=torch.float64,
                                              device=dev) for x in h[1:]])
        # workspaces sized for the largest chunk (filled once from the first electrons)
        for q in range(2):
            for dd, ss in zip(stage[q], [h[0] if t_shared else h[0][:big]] +
                              [x[:big] for x in h[1:]]):
                dd.copy_(ss)
        ws_up = [lw.lw_trajectories_upload(*(stage[q][0] if t_shared else stage[q][0][:big],
                                             stage[q][1][:big], stage[q][2][:big],
                                             stage[q][3][:big]),
                                           sections=lw.LW_SECTION_MIXED, block=args.block,
                                           device=dev).ws for q in range(2)]
        rec2 = [rec_m, torch.empty_like(rec_m)]
        S2 = [S_m, torch.empty_like(S_m)]
        S_host = [torch.empty(S_m.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        s_cp, s_pr = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        s_dp, s_bk = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev_cp = [torch.cuda.Event() for _ in range(2)]     # chunk copied into slot q
        ev_pr = [torch.cuda.Event() for _ in range(2)]     # slot q relayout done
        ev_dp = [torch.cuda.Event() for _ in range(2)]     # deposit from slot q done
        ev_sp = [torch.cuda.Event() for _ in range(2)]     # spectrum b written
        ev_bk = [torch.cuda.Event() for _ in range(2)]     # spectrum b read back
        st_e = {"g": 0, "i": 0}

        def step_e2e(timed=False):
            b = st_e["i"] % 2
            first_b = st_e["i"] < 2
            st_e["i"] += 1
            for c in range(n_ch):
                k0, k1 = bounds_e[c], bounds_e[c + 1]
                n = k1 - k0
                g = st_e["g"]
                q = g % 2
                st_e["g"] += 1
                with torch.cuda.stream(s_cp):
                    if g >= 2:
                        s_cp.wait_event(ev_pr[q])          # relayout g-2 read slot q
                    src = [h[0] if t_shared else h[0][k0:k1], h[1][k0:k1], h[2][k0:k1],
                           h[3][k0:k1]]
                    dst = [stage[q][0] if t_shared else stage[q][0][:n], stage[q][1][:n],
                           stage[q][2][:n], stage[q][3][:n]]
                    for dd, ss in zip(dst, src):
                        dd.copy_(ss, non_blocking=True)
                    ev_cp[q].record(s_cp)
                with torch.cuda.stream(s_pr):
                    s_pr.wait_event(ev_cp[q])
                    if g >= 2:
                        s_pr.wait_event(ev_dp[q])          # deposit g-2 read workspace q
                    tj = lw.lw_trajectories_upload(dst[0], dst[1], dst[2], dst[3],
                                                   sections=lw.LW_SECTION_MIXED,
                                                   block=args.block, device=dev, ws=ws_up[q])
                    ev_pr[q].record(s_pr)
                with torch.cuda.stream(s_dp):
                    if c == 0:
                        rec2[b].zero_()   # the spectrum two steps back (same stream) is done
                    s_dp.wait_event(ev_pr[q])
                    lw.lw_deposit_time_domain(tj, det, grid, MIX, record=rec2[b],
                                              accumulate=True, status=status)
                    ev_dp[q].record(s_dp)
            with torch.cuda.stream(s_dp):
                if not first_b:
                    s_dp.wait_event(ev_bk[b])              # read-back two steps back is done
                lw.lw_spectrum(rec2[b], MIX, det.n_pix, grid, ws=ws_s, out=S2[b])
                ev_sp[b].record(s_dp)
            with torch.cuda.stream(s_bk):
                s_bk.wait_event(ev_sp[b])
                S_host[b].copy_(S2[b], non_blocking=True)
                ev_bk[b].record(s_bk)

        ms_e, _ = timed_loop(step_e2e, args.steps, min(args.warmup, 3), None,
                             (s_cp, s_pr, s_dp, s_bk))
        h2d = sum(x.numel() * x.element_size() for x in h)
        result["e2e"] = {"value": n_job / (ms_e / args.steps * 1e-3), "unit": UNIT,
                         "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": S_host[0].numel() * S_host[0].element_size(),
                         "ms_per_step": ms_e / args.steps,
                         "pipeline": f"{n_ch} electron chunks; copy, relayout, deposit and "
                                     "read-back streams; records and spectra alternate "
                                     "between steps"}
        del ws_up, h, stage, rec2, S2
    # FP64 path beside it (fewer steps: GB300's FP64 pipe is 1/70 of its FP32 rate); timed
    # after the end-to-end steps, whose timing its memory use was seen to disturb
    fp64 = None
    S_64 = None
    if not args.no_fp64:
        del traj0
        rec_d = torch.empty(lw.record_shape(det, grid, lw.LW_FP64)[0], dtype=torch.float64,
                            device=dev)
        S_d = torch.empty((det.n_pix, grid.n_bins // 2 + 1), dtype=torch.float64, device=dev)
        ws_sd = lw.workspace(lw.spectrum_workspace_bytes(lw.LW_FP64, det.n_pix, grid), dev)
        trajd = lw.lw_trajectories_upload(t_d, r_d, b_d, a_d, sections=lw.LW_SECTION_FP64,
                                          device=dev)
        ws_d = trajd.ws

        def step_fp64(timed=False):
            tj = lw.lw_trajectories_upload(t_d, r_d, b_d, a_d, sections=lw.LW_SECTION_FP64,
                                           device=dev, ws=ws_d)
            lw.lw_deposit_time_domain(tj, det, grid, lw.LW_FP64, record=rec_d, status=status)
            lw.lw_spectrum(rec_d, lw.LW_FP64, det.n_pix, grid, ws=ws_sd, out=S_d)

        k64 = max(1, min(args.steps, args.fp64_steps))
        ms_d, _ = timed_loop(step_fp64, k64, 1)
        fp64 = {"value": n_job / (ms_d / k64 * 1e-3), "ms_per_step": ms_d / k64,
                "steps": k64, "warmup": 1}
        S_64 = S_d
    # accuracy of the mixed spectrum against the FP64 GPU spectrum (parity-tested vs oracle)
    acc = {}
    if S_64 is not None:
        a = S_m.double()
        b = S_64
        acc["spectrum_rel_l2_mixed_vs_fp64"] = float(torch.linalg.norm(a - b) /
                                                     torch.linalg.norm(b))
        # per band, on-axis-like fundamental omega_1(theta) +-20% and its 2nd harmonic
        from workloads.planewave import doppler_fundamental
        om = grid.omega.to(dev)
        th2 = torch.from_numpy(w.theta_x**2 + w.theta_y**2).to(dev)
        w1 = doppler_fundamental(w.gamma, w.lam, w.a0) / (1.0 + (w.gamma**2) * th2 /
                                                          (1 + 0.5 * w.a0**2))
        for name, h in (("fundamental", 1.0), ("harmonic2", 2.0)):
            mask = (om[None, :] > 0.8 * h * w1[:, None]) & (om[None, :] < 1.2 * h * w1[:, None])
            if bool(mask.any()):
                acc[f"rel_l2_{name}"] = float(torch.linalg.norm((a - b)[mask]) /
                                              torch.linalg.norm(b[mask]))
            else:
                acc[f"rel_l2_{name}"] = None
                acc[f"{name}_note"] = "band above Nyquist of this grid (aliased record)"
    result["fp64"] = fp64
    result["accuracy"] = acc
    result["status"] = {"mixed": st_m, "note": "8 = last arrival on grid point n_bins (clipped)"}

    # launches of our kernels per timed step: upload (ends, prepare, and the electron
    # order: key init, range, count, scan, scatter), deposit (1), spectrum (twiddle, then
    # pass 1 + pass 2, or the direct kernel up to 4096 bins)
    spec_k = 2 if grid.n_bins <= 4096 else 3
    result["gpu_launches"] = args.steps * (7 + 1 + spec_k)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w, grid, S_m, args)
    return result


def cpu_baseline(w, grid, S_gpu, args):
    """The FP64 oracle (as it stands) on a bounded sample of the same workload:
    all electrons and steps for a subset of pixels, timed on the host cores."""
    import oracle
    tr = w.traj
    n_threads = oracle.num_threads()
    # calibrate on one pixel, then size the sample for ~args.cpu_seconds
    t0 = time.time()
    oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, w.n_hat[:1], grid.t_min, grid.dt_u,
                       grid.n_bins)
    one = max(time.time() - t0, 1e-3)
    n_pix = int(max(1, min(w.n_pix, args.cpu_seconds / one * n_threads)))
    n_pix = max(n_threads, (n_pix // n_threads) * n_threads) if n_pix >= n_threads else n_pix
    idx = np.linspace(0, w.n_pix - 1, n_pix).astype(np.int64)
    t0 = time.time()
    rec, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, w.n_hat[idx], grid.t_min,
                                grid.dt_u, grid.n_bins)
    S = oracle.spectrum(rec, grid.dt_u)
    dt = time.time() - t0
    dep = tr.n_e * tr.n_s * n_pix
    S_g = S_gpu[idx.tolist()].double().cpu().numpy()
    err = float(np.linalg.norm(S_g - S) / np.linalg.norm(S))
    return {"value": dep / dt, "unit": UNIT, "cores": n_threads, "kind": "oracle",
            "sample": f"{n_pix} of {w.n_pix} pixels (all {tr.n_e} electrons x {tr.n_s} steps), "
                      f"deposit + FFT spectrum, {dt:.1f} s",
            "mixed_spectrum_rel_l2_vs_oracle_on_sample": err}


# ----------------------------------------------------------------------------- C5 sweep

def run_c5(args):
    """Batched design sweep (config 5): every variant's trajectories pushed on the GPU
    (lw_boris_push from its bunch), uploaded, tile shapes from the autotuner; then, wave by
    wave (as many variants as the memory budget holds), one persistent deposit launch and
    the variants' spectra captured in one CUDA graph and replayed as the timed step, against
    the same work launched variant by variant.  A step is every wave once."""
    import torch

    from paper_2206_03015_gb300 import lw
    from paper_2206_03015_gb300.autotune import Autotuner
    from workloads import configs

    dev = torch.device("cuda", 0)
    PREC = {"f32": lw.LW_MIXED_F32, "x4": lw.LW_MIXED_F32X4, "f64": lw.LW_MIXED}[args.c5_record]
    vs = configs.c5_batch(n_variants=args.c5_variants, n_e=(args.c5_ne[0], args.c5_ne[1]),
                          n_s=(args.c5_ns[0], args.c5_ns[1]), nx=(args.c5_nx[0], args.c5_nx[1]),
                          log2_bins=(args.c5_bins[0], args.c5_bins[1]))
    tuner = Autotuner(reps=1)
    rec_word = {lw.LW_MIXED_F32: 12, lw.LW_MIXED_F32X4: 16, lw.LW_MIXED: 24}[PREC]

    def resident_bytes(v):   # mixed section + record + spectrum of one variant
        return (v.n_e * (v.n_s + 1) * 40 + v.nx * v.nx * v.n_bins * rec_word
                + v.nx * v.nx * (v.n_bins // 2 + 1) * 4)

    # waves: variants by decreasing work, each wave filled up to the budget
    order = sorted(range(len(vs)), key=lambda i: -vs[i].deposits)
    budget = args.c5_budget_gb * 1e9
    waves, cur, used = [], [], 0.0
    for i in order:
        b = resident_bytes(vs[i])
        if cur and used + b > budget:
            waves.append(cur)
            cur, used = [], 0.0
        cur.append(i)
        used += b
    if cur:
        waves.append(cur)

    def build(v):
        r0, u0, t0, t1, n_hat = v.initial_state()
        dt = (t1 - t0) / v.n_s
        t = torch.empty(v.n_s + 1, dtype=torch.float64, device=dev)
        R, B, A = (torch.empty((v.n_e, v.n_s + 1, 3), dtype=torch.float64, device=dev)
                   for _ in range(3))
        L = (v.laser.lam, v.laser.a0, v.laser.w0, v.laser.fwhm)
        lw.lw_boris_push(torch.from_numpy(r0).to(dev), torch.from_numpy(u0).to(dev), t0, dt,
                         v.n_s, L, t, R, B, A)
        det = lw.Detector(n_hat, device=dev)
        traj = lw.lw_trajectories_upload(t, R, B, A, sections=lw.LW_SECTION_MIXED, device=dev)
        bnd = lw.lw_grid_bounds(traj, det).cpu().numpy()
        grid = lw.grid_from_bounds(bnd[0], bnd[1], v.n_bins)
        choice = tuner.tune((t, R, B, A), det, grid, blocks=tuple(args.c5_tune_blocks),
                            chunks=tuple(args.c5_tune_chunks), precision=PREC)
        traj = lw.lw_trajectories_upload(t, R, B, A, sections=lw.LW_SECTION_MIXED,
                                         block=choice.block, device=dev)
        del t, R, B, A
        return dict(traj=traj, det=det, grid=grid, choice=choice, v=v)

    def timed(fn, reps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_setup = time.time()
    ms_graph = ms_seq = 0.0
    units, tiles, dep = 0, [], 0
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    for wave in waves:
        items = [build(vs[i]) for i in wave]
        for it in items:
            shp, dt_ = lw.record_shape(it["det"], it["grid"], PREC)
            it["rec"] = torch.empty(shp, dtype=dt_, device=dev)
            it["S"] = torch.empty((it["det"].n_pix, it["grid"].n_bins // 2 + 1),
                                  dtype=torch.float32, device=dev)
        ws = lw.workspace(max(lw.spectrum_workspace_bytes(PREC, it["det"].n_pix, it["grid"])
                              for it in items), dev)
        bp = lw.lw_batch_plan([i["traj"] for i in items], [i["det"] for i in items],
                              [i["grid"] for i in items], [i["rec"] for i in items],
                              precision=PREC, statuses=[status] * len(items),
                              e_chunks=[i["choice"].e_chunk for i in items])

        def batched():
            lw.lw_batch_deposit(bp)
            for i in items:
                lw.lw_spectrum(i["rec"], PREC, i["det"].n_pix, i["grid"], ws=ws, out=i["S"])

        def sequential():
            for i in items:
                lw.lw_deposit_time_domain(i["traj"], i["det"], i["grid"], PREC, record=i["rec"],
                                          status=status)
                lw.lw_spectrum(i["rec"], PREC, i["det"].n_pix, i["grid"], ws=ws, out=i["S"])

        batched()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            with torch.cuda.graph(g, stream=st):
                batched()
        torch.cuda.current_stream().wait_stream(st)
        ms_graph += timed(g.replay, args.steps, args.warmup)
        ms_seq += timed(sequential, args.steps, min(args.warmup, 1))
        units += bp.plan.n_units
        tiles += [[i["choice"].block, i["choice"].e_chunk] for i in items]
        dep += sum(i["v"].deposits for i in items)
        del items, bp, g, ws
        torch.cuda.empty_cache()
    t_setup = time.time() - t_setup
    torch.cuda.synchronize()
    return {"metric": METRIC, "value": dep / (ms_graph * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"c5 sweep: {len(vs)} variants (gamma log-uniform 20-200, a0 "
                                   f"0.05-1, {args.c5_ne[0]}-{args.c5_ne[1]} electrons, "
                                   f"{args.c5_ns[0]}-{args.c5_ns[1]} steps, "
                                   f"{args.c5_nx[0]}^2-{args.c5_nx[1]}^2 pixels, "
                                   f"2^{args.c5_bins[0]}-2^{args.c5_bins[1]} bins), per wave one "
                                   "persistent deposit launch + spectra in one CUDA graph",
                       "deposits_per_step": dep, "units": units, "waves": len(waves),
                       "wave_sizes": [len(w) for w in waves], "budget_gb": args.c5_budget_gb,
                       "record": args.c5_record, "setup_s": round(t_setup, 1),
                       "tiles": tiles},
            "sequential": {"value": dep / (ms_seq * 1e-3), "ms_per_step": ms_seq},
            "status": int(status.item())}


# ----------------------------------------------------------------------------- C4 gradient

def run_c4(args):
    """Config 4: gradient of the band-integrated spectral energy (+-5 % of the on-axis
    fundamental) with respect to every electron's initial momentum and the laser's a0 and
    w0, through the library's kernels only: GPU Boris push, mixed-precision deposit and
    spectrum (the loss is FP32), the mixed-precision lw_spectrum_grad and the forward-mode
    lw_boris_push_grad; each part timed with CUDA events.  Beside it the same chain in
    FP64 and, once, the FP64 gradient with the torch-written checkpointed pusher."""
    import torch

    from paper_2206_03015_gb300 import lw
    from paper_2206_03015_gb300.autograd import (LWSpectrum, PushSpectrum, band_energy,
                                                 band_mask, boris_push)
    from workloads import configs
    from workloads.planewave import doppler_fundamental

    dev = torch.device("cuda", 0)
    r0n, u0n, laser, t0, t1, n_s, n_hat, n_bins, gamma = configs.c4_setup(
        n_e=args.c4_ne, n_s=args.c4_ns, nx=args.c4_nx, n_bins=args.c4_bins)
    n_e = r0n.shape[0]
    det = lw.Detector(n_hat, device=dev)
    r0 = torch.from_numpy(r0n).to(dev)
    L4 = (laser.lam, laser.a0, laser.w0, laser.fwhm)
    dt = (t1 - t0) / n_s
    MIX = lw.LW_MIXED_F32X4
    # the grid from one forward push (Eqs. tu_min / tu_max)
    t = torch.empty(n_s + 1, dtype=torch.float64, device=dev)
    R, B, A = (torch.empty((n_e, n_s + 1, 3), dtype=torch.float64, device=dev) for _ in range(3))
    lw.lw_boris_push(r0.clone(), torch.from_numpy(u0n).to(dev), t0, dt, n_s, L4, t, R, B, A)
    traj = lw.lw_trajectories_upload(t, R, B, A, sections=lw.LW_SECTION_FP64, device=dev)
    bnd = lw.lw_grid_bounds(traj, det).cpu().numpy()
    grid = lw.grid_from_bounds(bnd[0], bnd[1], n_bins)
    mask = band_mask(grid, doppler_fundamental(gamma, laser.lam, laser.a0), 0.05)
    del traj, t, R, B, A

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    def grad_step(prec):
        u = torch.from_numpy(u0n).to(dev).requires_grad_(True)
        a0 = torch.tensor(laser.a0, dtype=torch.float64, device=dev, requires_grad=True)
        w0 = torch.tensor(laser.w0, dtype=torch.float64, device=dev, requires_grad=True)
        S = PushSpectrum.apply(u, a0, w0, r0, laser.lam, laser.fwhm, t0, t1, n_s, det, grid,
                               lw.Q_E, prec)
        L = band_energy(S.to(torch.float64), grid, mask)
        L.backward()
        return L, u.grad, a0.grad, w0.grad

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            grad_step(prec)
        torch.cuda.synchronize()
        s0 = ev()
        for _ in range(steps):
            L, gu, ga, gw = grad_step(prec)
        s1 = ev()
        torch.cuda.synchronize()
        return s0.elapsed_time(s1) / steps, (L, gu, ga, gw)

    ms, (L, gu, ga, gw) = timed(MIX, args.steps, args.warmup)
    ms64, (L64, gu64, ga64, gw64) = timed(lw.LW_FP64, 1, 1)

    def parts_of(prec):
        # the parts, once more, each bracketed by events
        u0d = torch.from_numpy(u0n).to(dev)
        t = torch.empty(n_s + 1, dtype=torch.float64, device=dev)
        R, B, A = (torch.empty((n_e, n_s + 1, 3), dtype=torch.float64, device=dev)
                   for _ in range(3))
        sec = lw.LW_SECTION_FP64 if prec == lw.LW_FP64 else \
            lw.LW_SECTION_FP64 | lw.LW_SECTION_MIXED
        marks = [ev()]
        lw.lw_boris_push(r0.clone(), u0d.clone(), t0, dt, n_s, L4, t, R, B, A)
        marks.append(ev())
        traj = lw.lw_trajectories_upload(t, R, B, A, sections=sec, device=dev)
        marks.append(ev())
        rec = lw.lw_deposit_time_domain(traj, det, grid, prec)
        marks.append(ev())
        S, X = lw.lw_spectrum(rec, prec, det.n_pix, grid, want_X=True)
        marks.append(ev())
        gS = (mask.to(dev) * (2.0 * math.pi / (grid.n_bins * grid.dt_u)))[None, :].expand(
            S.shape).to(torch.float64)
        g_r, g_b, g_a = lw.lw_spectrum_grad(traj, det, grid, X, gS.contiguous(), precision=prec)
        marks.append(ev())
        lw.lw_boris_push_grad(r0, u0d, t0, dt, n_s, L4, g_r, g_b, g_a)
        marks.append(ev())
        torch.cuda.synchronize()
        return {name: a.elapsed_time(b) for name, a, b in zip(
            ("push", "upload", "deposit", "spectrum", "spectrum_grad", "push_grad"),
            marks[:-1], marks[1:])}

    parts = parts_of(MIX)
    parts64 = parts_of(lw.LW_FP64)
    # the torch-written checkpointed pusher (autograd) with the library's FP64 adjoint
    ref = None
    if not args.no_torch_pusher:
        u = torch.from_numpy(u0n).to(dev).requires_grad_(True)
        a0 = torch.tensor(laser.a0, dtype=torch.float64, device=dev, requires_grad=True)
        w0 = torch.tensor(laser.w0, dtype=torch.float64, device=dev, requires_grad=True)
        torch.cuda.synchronize()
        e0 = ev()
        tt, rr, bb, aa = boris_push(r0, u, a0, w0, laser.lam, laser.fwhm, t0, t1, n_s,
                                    checkpoint_every=256)
        L2 = band_energy(LWSpectrum.apply(tt, rr, bb, aa, det, grid), grid, mask)
        L2.backward()
        e1 = ev()
        torch.cuda.synchronize()
        ref = {"ms": e0.elapsed_time(e1),
               "grad_rel_diff_u0": float(torch.linalg.norm(u.grad - gu64) /
                                         torch.linalg.norm(gu64)),
               "grad_rel_diff_a0": float(abs(a0.grad - ga64) / abs(ga64)),
               "grad_rel_diff_w0": float(abs(w0.grad - gw64) / abs(gw64))}
    dep = n_e * n_s * det.n_pix
    return {"metric": METRIC, "value": dep / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"c4 gradient: {n_e} co-located electrons (gamma 60 +-0.1%) x "
                                   f"{n_s} Boris steps in a 1 um, a0 = 1, 10 fs, w0 = 20 um laser, "
                                   f"{int(round(det.n_pix ** 0.5))}^2 pixels over +-1/gamma, "
                                   f"{n_bins} bins; loss = spectral energy within +-5% of the "
                                   f"on-axis fundamental; gradient w.r.t. u0 (all electrons), a0, w0",
                       "deposits_per_step": dep,
                       "step": "forward (push, upload, mixed deposit, FP32 spectrum) + backward "
                               "(mixed lw_spectrum_grad, lw_boris_push_grad)"},
            "parts_ms": parts, "loss": float(L), "grad_a0": float(ga), "grad_w0": float(gw),
            "fp64_chain": {"ms_per_step": ms64, "parts_ms": parts64, "loss": float(L64),
                           "grad_a0": float(ga64), "grad_w0": float(gw64),
                           "mixed_vs_fp64": {
                               "loss": abs(float(L) / float(L64) - 1.0),
                               "grad_u0_rel_l2": float(torch.linalg.norm(gu - gu64) /
                                                       torch.linalg.norm(gu64)),
                               "grad_a0": float(abs(ga - ga64) / abs(ga64)),
                               "grad_w0": float(abs(gw - gw64) / abs(gw64))}},
            "torch_pusher": ref}


# ----------------------------------------------------------------------------- TDM vs FDM

def run_fdm(args):
    """The time-domain path against the frequency-domain direct sum (Eq. inty_dft,
    Algorithm 1) on a Nyquist-resolved C2 bunch at the C2 electron and step counts
    (10,000 electrons x 10,000 Boris steps; sigma_z = 0.1 um, sigma_x = sigma_y = 0.5 um so
    that 2^17 bins resolve the second harmonic) on 256 pixels over +-1.5/gamma and 2,048
    frequencies over 0.2 .. 2.5 omega_1: the normalised error of Eq. spectra_error (mean,
    max) of the mixed and FP64 time-domain spectra against the FDM, the FDM against the CPU
    oracle's FDM on sampled pixels and frequencies, and the FDM's throughput in terms
    N_s N_p N_obs N_omega per second."""
    import torch

    import oracle
    from paper_2206_03015_gb300 import lw
    from workloads import configs
    from workloads.planewave import doppler_fundamental

    dev = torch.device("cuda", 0)
    w = configs.c2x(n_e=args.fdm_ne, n_s=args.fdm_ns, nx=16, n_bins=1 << 17)
    tr = w.traj
    ins = [torch.from_numpy(x).to(dev) for x in (tr.t, tr.r, tr.beta, tr.beta_dot)]
    det = lw.Detector(w.n_hat, device=dev)
    traj = lw.lw_trajectories_upload(*ins, sections=lw.LW_SECTION_FP64 | lw.LW_SECTION_MIXED,
                                     device=dev)
    bnd = lw.lw_grid_bounds(traj, det).cpu().numpy()
    grid = lw.grid_from_bounds(bnd[0], bnd[1], w.n_bins)
    d_omega = 2 * math.pi / (grid.n_bins * grid.dt_u)
    w1 = doppler_fundamental(w.gamma, w.lam, w.a0)
    n_om = args.fdm_nomega
    l0 = int(round(0.2 * w1 / d_omega))
    step = max(1, int(round(2.3 * w1 / d_omega / n_om)))   # FDM frequencies on TDM bins
    om0, dom = l0 * d_omega, step * d_omega
    dt = float(tr.t[1] - tr.t[0])

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    S_f, ms_f = timed(lambda: lw.lw_spectrum_fdm(traj, det, om0, dom, n_om, dt))
    cols = torch.arange(n_om, device=dev) * step + l0
    res = {}
    for name, prec in (("tdm_mixed", lw.LW_MIXED_F32X4), ("tdm_fp64", lw.LW_FP64)):
        def tdm():
            rec = lw.lw_deposit_time_domain(traj, det, grid, prec)
            return lw.lw_spectrum(rec, prec, det.n_pix, grid)
        S_t, ms_t = timed(tdm)
        err = (S_t.double()[:, cols] - S_f).abs() / S_f.max()
        res[name] = {"ms": ms_t, "deposits_per_s": tr.n_e * tr.n_s * det.n_pix / (ms_t * 1e-3),
                     "spectra_error_mean": float(err.mean()), "spectra_error_max": float(err.max())}
    # the GPU FDM against the oracle's FDM: 2 pixels x 8 frequencies, all electrons and samples
    pix = [0, det.n_pix // 2 + 8]
    fi = np.linspace(0, n_om - 1, 8).astype(np.int64)
    om = om0 + dom * fi
    t0 = time.time()
    S_o, _ = oracle.fdm(tr.t, tr.r, tr.beta, tr.beta_dot, w.n_hat[pix], om, dt)
    cpu_s = time.time() - t0
    S_g = S_f[pix][:, fi.tolist()].cpu().numpy()
    terms = tr.n_e * (tr.n_s + 1) * det.n_pix * n_om
    return {"metric": "FDM terms/s (electron.sample.pixel.frequency), Eq. inty_dft",
            "value": terms / (ms_f * 1e-3), "unit": "terms/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": ms_f, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": f"c2x at C2 counts: {tr.n_e} electrons x {tr.n_s} Boris steps "
                                   f"(sigma_z 0.1 um, sigma_x,y 0.5 um), {det.n_pix} pixels over "
                                   f"+-1.5/gamma, {w.n_bins} bins; FDM on {n_om} frequencies "
                                   f"{om0 / w1:.2f} .. {(om0 + dom * (n_om - 1)) / w1:.2f} omega_1",
                       "omega_1": w1},
            "tdm_vs_fdm": res,
            "fdm_vs_oracle_rel_l2": float(np.linalg.norm(S_g - S_o) / np.linalg.norm(S_o)),
            "oracle_sample": {"pixels": pix, "frequencies": len(fi), "cpu_s": cpu_s,
                              "cores": oracle.num_threads()}}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """The CPU oracle timed as the reference arm: each step is a bounded sample
    (a subset of pixels, all electrons and steps) of the same workload."""
    if rank != 0:
        return None
    import oracle
    w = make_workload(args, 0)
    tr = w.traj
    lo, hi = oracle.grid_bounds(tr.t, tr.r, w.n_hat)
    dt_u = (hi - lo) / w.n_bins
    n_threads = oracle.num_threads()
    t0 = time.time()
    oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, w.n_hat[:1], lo, dt_u, w.n_bins)
    one = max(time.time() - t0, 1e-3)
    budget = max(1.0, args.ref_seconds / max(1, args.steps + args.warmup))
    n_pix = int(max(1, min(w.n_pix, budget / one * n_threads)))
    idx = np.linspace(0, w.n_pix - 1, n_pix).astype(np.int64)

    def step():
        rec, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, w.n_hat[idx], lo, dt_u,
                                    w.n_bins)
        oracle.spectrum(rec, dt_u)

    for _ in range(args.warmup):
        step()
    t0 = time.time()
    for _ in range(args.steps):
        step()
    dt = (time.time() - t0) / args.steps
    dep = tr.n_e * tr.n_s * n_pix
    v = dep / dt
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_pixels_per_step": n_pix},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": n_threads, "kind": "oracle",
                             "sample": f"{n_pix} of {w.n_pix} pixels per step, all electrons "
                                       f"and steps, deposit + FFT"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-e", type=int, default=10_000)
    ap.add_argument("--n-s", type=int, default=10_000)
    ap.add_argument("--nx", type=int, default=64)
    ap.add_argument("--n-bins", type=int, default=65_536)
    ap.add_argument("--block", type=int, default=512)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mixed", default="x4", choices=["f32", "x4", "f64"],
                    help="record of the timed mixed path: FP32 (LW_MIXED_F32), FP32 interleaved "
                         "(LW_MIXED_F32X4) or FP64 (LW_MIXED)")
    ap.add_argument("--e2e-chunks", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=120.0)
    ap.add_argument("--shard", default="pixels", choices=["pixels", "detectors"],
                    help="N > 1: split one detector's pixels (strong scaling) or give each "
                         "rank a detector of its own (weak scaling)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c4", "c5", "fdm"])
    ap.add_argument("--fdm-ne", type=int, default=10_000)
    ap.add_argument("--fdm-ns", type=int, default=10_000)
    ap.add_argument("--fdm-nomega", type=int, default=2048)
    ap.add_argument("--c4-ne", type=int, default=2048)
    ap.add_argument("--c4-ns", type=int, default=4096)
    ap.add_argument("--c4-nx", type=int, default=32)
    ap.add_argument("--c4-bins", type=int, default=16_384)
    ap.add_argument("--no-torch-pusher", action="store_true")
    ap.add_argument("--c5-variants", type=int, default=64)
    ap.add_argument("--c5-ne", type=int, nargs=2, default=(512, 8192))
    ap.add_argument("--c5-ns", type=int, nargs=2, default=(2000, 40000))
    ap.add_argument("--c5-nx", type=int, nargs=2, default=(16, 128))
    ap.add_argument("--c5-bins", type=int, nargs=2, default=(12, 17))
    ap.add_argument("--c5-record", default="f32", choices=["f32", "x4", "f64"])
    # resident data of a wave; building a variant also holds its FP64 trajectories and a
    # tuning record, so the budget stays well below the device memory (150 of 277 GB)
    ap.add_argument("--c5-budget-gb", type=float, default=150.0)
    ap.add_argument("--c5-tune-blocks", type=int, nargs="+", default=(256, 512))
    ap.add_argument("--c5-tune-chunks", type=int, nargs="+", default=(1, 4))
    args = ap.parse_args()
    args.full = (args.n_e, args.n_s, args.nx, args.n_bins) == (10_000, 10_000, 64, 65_536)
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    args.world = world
    dist = None
    if world > 1 and args.impl == "ours":
        import torch.distributed as tdist
        import torch
        torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
        tdist.init_process_group(backend="nccl")
        dist = tdist
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    elif args.workload == "c5":
        res = run_c5(args)
    elif args.workload == "c4":
        res = run_c4(args)
    elif args.workload == "fdm":
        res = run_fdm(args)
    else:
        res = run_ours(args, rank, world, dist)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
