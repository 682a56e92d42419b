"""Build libfnlh.so (the CUDA library) in-tree with nvcc for sm_103a, and
beside it libfnlh_probe.so (the arithmetic peak probe the benchmark reports
its FP64 roofline against).

Each translation unit is compiled in parallel, then linked against the shared
CUDA runtime (the same libcudart the host process already uses).
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfnlh.so")
PROBE_DIR = os.path.join(PKG, "probe")
PROBE_LIB = os.path.join(PKG, "libfnlh_probe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _newest(paths):
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def _compile(src: str, extra) -> str:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if res.stderr.strip():
        sys.stderr.write(res.stderr)
    return obj


def _link(objs, out):
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-ldl"]  # -ldl: NVTX loads its tool
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, out)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile and link libfnlh.so and libfnlh_probe.so if any source or header is newer."""
    srcs = sources()
    probe_srcs = sorted(os.path.join(PROBE_DIR, f) for f in os.listdir(PROBE_DIR) if f.endswith(".cu"))
    deps = headers() + [__file__]
    need_lib = force or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(srcs + deps)
    need_probe = (force or not os.path.exists(PROBE_LIB)
                  or os.path.getmtime(PROBE_LIB) < _newest(probe_srcs + deps))
    if not (need_lib or need_probe):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra) + (["-Xptxas", "-v"] if verbose else [])
    todo = (srcs if need_lib else []) + (probe_srcs if need_probe else [])
    with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
        objs = dict(zip(todo, ex.map(lambda s_: _compile(s_, extra), todo)))
    if need_lib:
        _link([objs[s_] for s_ in srcs], LIB)
    if need_probe:
        _link([objs[s_] for s_ in probe_srcs], PROBE_LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
