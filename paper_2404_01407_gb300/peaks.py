"""Arithmetic peaks of the GPU this process runs on, measured by the
multiply-add probe in libfnlh_probe.so (include/fnlh_probe.h).

The FP64 sweep is bound by FP64 multiply-add throughput, a figure the
measured copy/GEMM peaks do not give; this probe measures it (and the FP32
figure) with independent multiply-add accumulators on every SM, including
the sweeps' operand pattern (one operand feeding two or four multiply-adds):
on GB300 the FP64 rate ranges from about 1.06 TFLOP/s (a bare dependent
chain) to 1.23 (8 chains x 2, every operand in a register).
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def probe_lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "libfnlh_probe.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_2404_01407_gb300.build first")
        lib = ctypes.CDLL(path)
        lib.fnlh_probe_fma.restype = ctypes.c_int
        lib.fnlh_probe_fma.argtypes = [ctypes.c_int32] * 6 + [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                                               ctypes.c_void_p]
        _LIB = lib
    return _LIB


def fma_tflops(torch, device, precision: int, iters: int = 2048, reps: int = 2):
    """Multiply-add throughput in TFLOP/s (precision 0: FP64, 1: FP32): the
    best over chain counts, operand reuse (1, 2, 4 multiply-adds per loaded
    operand: the sweeps feed each block entry to a real and an imaginary
    part) and block shapes, of `reps` timed runs each after one untimed run,
    on a grid of 8 waves of resident blocks.  Returns
    (tflops, {"chains": c, "reuse": r, "threads": t, "ms": ms})."""
    lib = probe_lib()
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    stream = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    sink = torch.empty(sms * 2048 * 8, dtype=torch.float64, device=device)
    ms = ctypes.c_float(0.0)
    best, shape = 0.0, None
    for chains, reuse in ((8, 1), (16, 1), (4, 2), (8, 2), (16, 2), (4, 4), (8, 4)):
        for threads in (256, 1024):
            blocks = sms * (2048 // threads) * 8
            for r in range(reps + 1):
                rc = lib.fnlh_probe_fma(precision, chains, reuse, blocks, threads, iters,
                                        ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ms), stream)
                if rc != 0:
                    raise RuntimeError(f"fnlh_probe_fma failed ({rc})")
                if r == 0:
                    continue
                tf = 2.0 * chains * reuse * iters * threads * blocks / (ms.value * 1e-3) / 1e12
                if tf > best:
                    best, shape = tf, {"chains": chains, "reuse": reuse, "threads": threads, "ms": ms.value}
    return best, shape
