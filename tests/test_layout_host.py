"""The sweeps' internal vector layout (csrc/common.cuh), compiled as host code
and checked against the properties the kernels rely on (CPU only):

* FP64 vectors, and FP32 vectors of K >= 3 systems: complex slices of 2b
  values, system k at 2bk, node stride 2bK;
* FP32 vectors of K <= 2 (mean flow alone, or with one harmonic): the mean
  flow real in a padded slot, the slices tiling the node without overlap,
  every slice and node start on the alignment of the kernels' vector loads
  (16 bytes for b = 6, 8 for b = 5), never longer than the complex layout the
  workspace is sized for;
* mean_pos maps the mean flow's b values one to one onto the slot's non-pad
  positions, the first half on the even positions a harmonic's real parts
  use.
"""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("layout") / "layout_check")
    subprocess.run([nvcc, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(HERE, "layout_check.cu")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines()
    strides, means = {}, {}
    for line in out:
        f = line.split()
        if f[0] == "S":
            b, elem, K, real, stride = (int(v) for v in f[1:6])
            rest = [int(v) for v in f[6:]]
            strides[(b, elem, K)] = (bool(real), stride, [(rest[2 * k], rest[2 * k + 1]) for k in range(K)])
        else:
            b, slot = int(f[1]), int(f[2])
            means[b] = (slot, [int(v) for v in f[3:3 + b]], [bool(int(v)) for v in f[3 + b:]])
    return strides, means


def test_complex_layout(layout):
    strides, _ = layout
    for (b, elem, K), (real, stride, sl) in strides.items():
        if elem == 8 or K >= 3:
            assert not real
            assert stride == 2 * b * K
            assert sl == [(2 * b * k, 2 * b) for k in range(K)]


def test_real_mean_layout_tiles_and_aligns(layout):
    strides, means = layout
    for (b, elem, K), (real, stride, sl) in strides.items():
        if elem != 4 or K >= 3:
            continue
        assert real
        slot = means[b][0]
        assert slot >= b and stride == slot + 2 * b * (K - 1) <= 2 * b * K
        covered = []
        for off, ln in sl:
            covered += list(range(off, off + ln))
        assert sorted(covered) == list(range(stride))  # slices tile the node, no overlap
        align = 16 if (2 * b) % 4 == 0 else 8
        assert (stride * elem) % align == 0
        assert all((off * elem) % align == 0 for off, _ in sl)


def test_mean_positions(layout):
    _, means = layout
    for b, (slot, pos, pad) in means.items():
        assert len(pad) == slot
        assert sorted(pos + [e for e in range(slot) if pad[e]]) == list(range(slot))
        assert all(pos[t] == 2 * t for t in range(slot // 2))
        assert all(pos[t] % 2 == 1 for t in range(slot // 2, b))
