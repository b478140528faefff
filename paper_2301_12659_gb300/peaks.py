"""Measured peaks of the pipes the hot path runs on (the roofline
denominators): FP64 FMA, 32-bit integer multiply-add (IMAD), three-input
logic (LOP3) and an even IMAD/LOP3 mix, each in thread operations per clock
per SM and per second, from the microbenchmarks of peaks/peak_probe.cu.

The multiple double kernels run on these pipes (FP64 md algorithms, or md
values carried in integer limbs), not on HBM or the tensor cores, so their
roofline is the issue rate of these instructions.  ``measure()`` builds the
probe on first use (nvcc, sm_103a) and runs it on the current device.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "peaks", "peak_probe.cu")
SO = os.path.join(HERE, "_build", f"peak_probe-{platform.machine()}.so")
KINDS = {"fp64_fma": 0, "int_imad": 1, "int_lop3": 2, "int_mix": 3}


def build() -> str:
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    if not os.path.exists(SO) or os.path.getmtime(SO) < os.path.getmtime(SRC):
        tmp = SO + f".tmp{os.getpid()}"
        subprocess.run([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                        "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-o", tmp, SRC], check=True,
                       capture_output=True, text=True)
        os.replace(tmp, SO)
    return SO


def measure(num_sms: int = 0, blocks_per_sm: int = 8, iters: int = 4096) -> dict:
    """Each probe over the whole GPU: per kind, thread operations per second
    (`ops_per_s`), per clock per SM (`per_clk_per_sm`, with the SM clock of
    the run from the cycle counter and the nanosecond timer) and that clock."""
    import torch
    lib = ctypes.CDLL(build())
    lib.peak_probe.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p]
    lib.peak_probe.restype = ctypes.c_int
    if num_sms <= 0:
        num_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {"num_sms": num_sms, "source": "paper_2301_12659_gb300/peaks/peak_probe.cu"}
    for name, kind in KINDS.items():
        res = (ctypes.c_double * 4)()
        n_iter = iters // 16 if kind == 0 else iters  # FP64 runs ~40x slower
        rc = lib.peak_probe(kind, num_sms, blocks_per_sm, n_iter, res)
        if rc != 0:
            raise RuntimeError(f"peak_probe({name}) failed with CUDA error {rc}")
        ms, cycles, ns, ops = res[0], res[1], res[2], res[3]
        mhz = cycles / ns * 1e3 if ns > 0 else float("nan")
        ops_s = ops / (ms * 1e-3)
        out[name] = {"ops_per_s": ops_s, "per_clk_per_sm": ops_s / (num_sms * mhz * 1e6), "sm_mhz": mhz,
                     "ms": ms}
    return out


if __name__ == "__main__":
    import json
    print(json.dumps(measure(), indent=1))
