"""Measured pipe peaks of the GPU (L2 reductions, FP32 / FP64 FMA, shared-memory loads).

The deposit of the time-domain method is made of a handful of operation kinds (grid-point
updates added by the L2, FP32 field arithmetic, FP64 anchors, reads of staged samples);
its roofline needs the rate of each on this GPU.  ``measure()`` times one kernel per kind
(``pipe_peaks.cu``, built into ``_build/libpeaks.so``) with CUDA events on the current
stream and returns the best of a few launches.  HBM bandwidth is not measured here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pipe_peaks.cu")
OUT_DIR = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(OUT_DIR, "libpeaks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

_lib = None


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run(["nvcc"] + ARCH + ["-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
                                      "-o", tmp, SRC], check=True)
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.lwp_red.argtypes = [I, P, I64, I, I, I, I, P]
        lib.lwp_fma.argtypes = [I, P, I, I, I, P]
        lib.lwp_lds.argtypes = [P, I, I, I, P]
        for f in (lib.lwp_red, lib.lwp_fma, lib.lwp_lds):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _best_ms(launch, reps=5):
    import torch
    launch()   # warm-up
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        launch()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def measure(device=None) -> dict:
    """Rates on the current GPU: reductions per second, FLOP/s, shared bytes per second."""
    import torch
    lib = load()
    dev = torch.device(device or "cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    blocks, threads = sms * 8, 256
    out = {"sms": sms}

    def check(rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} launch failed ({rc})")

    # L2 reductions on a 32 MiB buffer (inside the 129 MB L2 of a GB300)
    buf = torch.zeros(8 << 20, dtype=torch.float32, device=dev)
    iters = 400
    for name, kind, stride, per in (("red_f32_lines", 0, 32, 1), ("red_f32_coalesced", 0, 1, 1),
                                    ("red_f64_lines", 1, 32, 1), ("red_v4f32_lines", 2, 32, 4)):
        n = buf.numel() // (2 if kind == 1 else 1)
        ms = _best_ms(lambda: check(lib.lwp_red(kind, ctypes.c_void_p(buf.data_ptr()), n,
                                                stride, blocks, threads, iters, st), name))
        ops = blocks * threads * iters
        out[name] = {"ops_per_s": ops / (ms * 1e-3), "values_per_s": ops * per / (ms * 1e-3),
                     "ms": ms}
    del buf
    # FMA throughput (2 flops each)
    o32 = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    for name, kind, it in (("fma_f32", 0, 8192), ("fma_f64", 1, 256)):
        ms = _best_ms(lambda: check(lib.lwp_fma(kind, ctypes.c_void_p(o32.data_ptr()), blocks,
                                                threads, it, st), name))
        out[name] = {"flops": blocks * threads * it * 8 * 2 / (ms * 1e-3), "ms": ms}
    # conflict-free 16-byte shared loads
    it = 8192
    lb = sms * 4
    ms = _best_ms(lambda: check(lib.lwp_lds(ctypes.c_void_p(o32.data_ptr()), lb, threads, it, st),
                                "lds"))
    bps = lb * threads * it * 16 / (ms * 1e-3)
    out["lds_v4"] = {"bytes_per_s": bps, "wavefronts_per_s": bps / 128.0, "ms": ms}
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    import json
    print(json.dumps(measure(), indent=1))
