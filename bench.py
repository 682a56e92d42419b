#!/usr/bin/env python
"""Benchmark of the shared-Jacobian FNLH relaxation on GB300.

The metric has two halves, both on the one JSON line:

* value -- node-system updates per second per Jacobi sweep on the FP64 GPU
  baseline: a 128x64x48 perturbed hex passage (393,216 nodes, 1,162,240
  edges), 6x6 blocks (Euler + one turbulence equation), mean flow + 4
  harmonics at omega_n = n, CFL 20.  One step = assemble J and D (+ the
  per-node Schur prep) -> 50 FP64 block-Jacobi sweeps over all 5 systems ->
  FP64 residual norms; value = n K sweeps / step time, whole job.  Its
  roofline is the FP64 sweep kernel against the FP64 multiply-add peak that
  the probe in libfnlh_probe.so measures in the same run.
* time_to_1e8 -- mixed vs FP64 time to a 1e-8 relative FP64 residual on the
  2.1M-node passage with 8 harmonics (FP64 Jacobi; FP64 defect correction
  with FP32 and BF16 blocks), device-resident and end to end through the
  public API, each solution's residual and error against the oracle's
  solution, and the oracle's own time on the host cores.

Extra sections: the batched multi-row form (three blade rows of 200k/600k/
1.1M nodes with 2/8/4 harmonics) against per-row launches, five RK(5,3)
stages with the paper's linear-solve rule, phase-lagged periodic edges, the
partitioned (domain-truncated) solve, ILU(0) against Jacobi, a randomly
renumbered mesh, and an 8M-node passage with 16 harmonics.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fnlh|reference]
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
sys.path.insert(0, ROOT)

METRIC = "node·harmonic updates/s per Jacobi sweep; mixed vs FP64 time-to-1e-8 residual"
UNIT = "updates/s"
SWEEPS = 50
WORKLOAD = "c2"
BF16_INNER = 21  # BF16-block inner sweeps per correction (FP32 blocks: 30)

# FP64 peak from unit counts and clocks (152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz): context only; the
# roofline is taken against the FP64 peak the multiply-add probe measures on the same GPU in the same run
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.07e9
# DRAM bytes (read + write) per launch of the top kernel from an ncu capture (profiles/k_sweep_f64_c2.md),
# valid only while the kernel's sources hash to the value they had when it was taken
NCU_TRAFFIC = {"k_sweep_f64_c2": {"bytes": 1363062784 + 177632768,
                                  "sources_sha256": "144813b06f193bafef69f33c1fdd03e149971173103c471efb3cfa73f5c171bd"}}
KERNEL_SOURCES = ("paper_2404_01407_gb300/csrc/sweep.cu", "paper_2404_01407_gb300/csrc/sweep_kernel.cuh",
                  "paper_2404_01407_gb300/csrc/common.cuh", "include/fnlh.h")


def kernel_sources_sha256():
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(key):
    """(bytes per launch, note): the captured DRAM bytes, or None once the sources changed."""
    rec = NCU_TRAFFIC.get(key)
    if not rec or rec["bytes"] is None:
        return None, "no capture on record"
    if rec["sources_sha256"] != kernel_sources_sha256():
        return None, "kernel sources changed since the capture"
    return rec["bytes"], "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch (profiles/k_sweep_f64_c2.md)"


def measure_arith_peaks(torch, dev, index):
    """FP64 and FP32 multiply-add peaks of this GPU from the probe in libfnlh_probe.so, with the SM clock
    sampled while it runs (outside every timed region)."""
    from paper_2404_01407_gb300 import peaks

    ck = ClockSampler(index)
    ck.start()
    f64, s64 = peaks.fma_tflops(torch, dev, 0)
    f32, s32 = peaks.fma_tflops(torch, dev, 1)
    torch.cuda.synchronize()
    clocks = ck.stop()
    return {"fp64_tflops": f64, "fp32_tflops": f32, "fp64_shape": s64, "fp32_shape": s32, "clocks": clocks,
            "source": "measured: multiply-add accumulators on every SM (libfnlh_probe.so, include/fnlh_probe.h), "
                      "best over chain counts, operand reuse 1/2/4 (the sweeps' pattern is 2) and 256/1024-thread "
                      "blocks, SM clock sampled meanwhile"}


def tri_solve_flops(b: int, real: bool) -> int:
    """Flops of one shifted back-substitution (T + i s I) y = r with the per-node
    real Schur factor T and the pivot factors computed once per call: 4 per
    off-diagonal term and 6 per row for the scaling by (d - i s) / (d^2 + s^2)
    of a complex system; 2 and 1 for the real (mean-flow) system."""
    if real:
        return b * (b - 1) + b
    return 2 * b * (b - 1) + 6 * b


def sweep_flops(n, nnz, b, n_harm, block_entries=None):
    """block_entries: structurally nonzero entries per off-diagonal block the
    kernel multiplies (b^2, or 31 for b = 6 with the frozen-turbulence pattern)."""
    C = 1 + 2 * n_harm
    e = b * b if block_entries is None else block_entries
    return 2.0 * nnz * e * C + n * (n_harm * tri_solve_flops(b, False) + tri_solve_flops(b, True))


def sweep_bytes(n, nnz, b, n_harm, s_j, s_d, s_x, s_b):
    """Algorithmic bytes of one sweep: each block once, X gathered once, X written once, B once."""
    C = 1 + 2 * n_harm
    return nnz * (b * b * s_j + 4) + n * (4 + b * b * s_d + 16) + n * b * C * (2 * s_x + s_b)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.file.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    """Largest value over the ranks (the job time is the slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- CPU oracle

def cpu_oracle_rate(p, budget_s=15.0, max_sweeps=100):
    """The oracle as it stands on the host cores: one build, S sweeps, one residual."""
    import oracle

    m = p.mesh
    t0 = time.perf_counter()
    oj = oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    X = oracle.jacobi(oj, m.vol, p.omega, p.b, 1)
    t1 = time.perf_counter() - t0
    S = int(max(1, min(max_sweeps, (budget_s - t_build) / max(t1, 1e-3))))
    t0 = time.perf_counter()
    X = oracle.jacobi(oj, m.vol, p.omega, p.b, S, X0=X)
    oracle.residual(oj, m.vol, p.omega, p.b, X)
    t = time.perf_counter() - t0
    K = 1 + p.n_harm
    cores = oracle.num_threads()
    # the same on one thread, over fewer sweeps
    oracle.set_num_threads(1)
    try:
        S1 = max(1, min(3, S))
        t0 = time.perf_counter()
        oracle.jacobi(oj, m.vol, p.omega, p.b, S1, X0=X)
        t_1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    return {"value": m.n_nodes * K * S / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{p.name} full mesh, {S} FP64 Jacobi sweeps + 1 residual after 1 warm sweep "
                      f"(build {t_build:.1f} s excluded), {t:.1f} s",
            "single_thread": {"value": m.n_nodes * K * S1 / t_1, "unit": UNIT, "cores": 1,
                              "sample": f"{S1} FP64 Jacobi sweeps, {t_1:.1f} s"}}


def cpu_oracle_large(max_sweeps=3):
    """The oracle on the 8M-node passage (256x200x156, b = 6), a bounded sample: Jacobian build and
    `max_sweeps` FP64 Jacobi sweeps with the mean flow and one harmonic; its cost is linear in the number
    of systems, so the per-sweep time of the 17-system case is extrapolated from the update rate."""
    import oracle
    from paper_2404_01407_gb300 import inputs

    c = inputs.CONFIGS["c5"]
    p = inputs.config_problem("c5", n_harm=1)
    m = p.mesh
    t0 = time.perf_counter()
    oj = oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.jacobi(oj, m.vol, p.omega, p.b, max_sweeps)
    t = time.perf_counter() - t0
    rate = m.n_nodes * 2 * max_sweeps / t
    return {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"c5 full mesh ({m.n_nodes} nodes), mean + 1 harmonic, {max_sweeps} FP64 Jacobi sweeps, "
                      f"{t:.1f} s (build {t_build:.1f} s excluded)",
            "build_seconds": t_build,
            "extrapolated_seconds_per_sweep_N16": m.n_nodes * (1 + c["n_harm"]) / rate,
            "note": "per-sweep time at 16 harmonics extrapolated from the update rate at 1 (linear in systems)"}


def stress_permuted_section(torch, fnlh, inputs, dev):
    """Locality stress: the measured passage with its nodes randomly renumbered (seed 4) against the
    lexicographic numbering -- sweep times per precision."""
    p = inputs.config_problem(WORKLOAD)
    mesh, perm = inputs.permute_mesh(p.mesh, seed=4)
    out = {"workload": f"{WORKLOAD}: lexicographic vs randomly renumbered (seed 4) nodes, sweep time"}
    for tag, m, q, b in (("lexicographic", p.mesh, p.q, p.b), ("permuted", mesh, p.q[perm], p.b[perm])):
        dm = fnlh.DeviceMesh.from_mesh(m, dev)
        J = fnlh.DeviceJacobian(dm, p.block, fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_BF16, dev)
        fnlh.fnlh_build_jacobian(dm, torch.from_numpy(q).to(dev), fnlh.make_params(p.cfl), J)
        B = torch.from_numpy(b).to(dev)
        X = torch.zeros_like(B)
        ws = fnlh.workspace(m.n_nodes, p.block, p.n_harm, dev)
        out[tag] = {name + "_sweep_ms": sweep_time_ms(torch, fnlh, dm, J, p, B, X, ws, prec)
                    for name, prec in (("f64", fnlh.FNLH_F64), ("f32", fnlh.FNLH_F32), ("bf16", fnlh.FNLH_BF16))}
        del dm, J, B, X, ws
        torch.cuda.empty_cache()
    for name in ("f64", "f32", "bf16"):
        out[f"{name}_slowdown"] = out["permuted"][f"{name}_sweep_ms"] / out["lexicographic"][f"{name}_sweep_ms"]
    return out


def run_reference(args):
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    import oracle
    from paper_2404_01407_gb300 import inputs

    p = inputs.config_problem(args.workload)
    m = p.mesh
    K = 1 + p.n_harm

    def step():  # the GPU arm's step: assemble J and D, SWEEPS FP64 block-Jacobi sweeps, residual
        oj = oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl)
        X = oracle.jacobi(oj, m.vol, p.omega, p.b, SWEEPS)
        oracle.residual(oj, m.vol, p.omega, p.b, X)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    t = time.perf_counter() - t0
    value = m.n_nodes * K * SWEEPS * args.steps / t
    sample = (f"{args.workload} full mesh; each step the GPU arm's step: Jacobian build + {SWEEPS} FP64 "
              f"Jacobi sweeps + 1 residual")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(p),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_config(p, sweeps=SWEEPS):
    return {"workload": f"{p.name}: {p.mesh.dims[0]}x{p.mesh.dims[1]}x{p.mesh.dims[2]} perturbed hex passage, "
                        f"{p.mesh.n_nodes} nodes, {p.mesh.n_edges} edges, b={p.block}, mean + {p.n_harm} harmonics, "
                        f"CFL {p.cfl:g}, {sweeps} FP64 block-Jacobi sweeps per step (+ Jacobian build + residual)",
            "nodes": p.mesh.n_nodes, "edges": p.mesh.n_edges, "block": p.block, "harmonics": p.n_harm,
            "sweeps_per_step": sweeps, "l2": "inputs larger than L2 (J alone 0.67 GB FP64)"}


# ------------------------------------------------------------------ GPU arm

def run_fnlh(args):
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2404_01407_gb300 import fnlh, inputs

    fnlh.lib()
    peaks, peaks_kind = load_peaks()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    p = inputs.config_problem(args.workload)
    n, E, b, N = p.mesh.n_nodes, p.mesh.n_edges, p.block, p.n_harm
    K, nnz = 1 + N, 2 * E
    dm = fnlh.DeviceMesh.from_mesh(p.mesh, dev)
    J = fnlh.DeviceJacobian(dm, b, fnlh.FNLH_PREP_F64, dev)
    params = fnlh.make_params(p.cfl)
    Q = torch.from_numpy(p.q).to(dev)
    B = torch.from_numpy(p.b).to(dev)
    X = torch.zeros_like(B)
    ws = fnlh.workspace(n, b, N, dev)
    norms = torch.empty((K, 2), dtype=torch.float64, device=dev)

    def step():
        fnlh.fnlh_build_jacobian(dm, Q, params, J)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, SWEEPS, fnlh.FNLH_F64, ws)
        fnlh.fnlh_residual(dm, J, p.omega, B, X, norms=norms, ws=ws)

    # kernels launched per step: build, basis, pattern check (b = 6), block rotation; rotate B and X in; the
    # reciprocal-pivot table; the sweeps; rotate out; residual + its reduction (the ncu launch list shows the
    # same count)
    launches_per_step = (4 if p.block == 6 else 3) + 2 + 1 + SWEEPS + 1 + 2
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sweep_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
    for a, z in sweep_ev:  # torch creates the CUDA event on its first record
        a.record(stream)
        z.record(stream)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.steps):
        fnlh.fnlh_set_sweep_events(*sweep_ev[s])
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    fnlh.fnlh_set_sweep_events(None, None)
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world)
    sweep_ms = sum(a.elapsed_time(z) for a, z in sweep_ev) / (args.steps * SWEEPS)
    rel = np.sqrt(norms[:, 0].cpu().numpy() / norms[:, 1].cpu().numpy())

    updates = n * K * SWEEPS
    value = world * updates / (ms * 1e-3)
    structured = fnlh.fnlh_prep_structured(J)
    flops = sweep_flops(n, nnz, b, N, block_entries=(b * b - (b - 1)) if structured else None)
    achieved = flops / (sweep_ms * 1e-3)
    bytes_alg = sweep_bytes(n, nnz, b, N, 8, 8, 8, 8)
    traffic, traffic_note = ncu_traffic(f"k_sweep_f64_{args.workload}")

    # end to end through the public API with host buffers (pinned), copies inside the timed region.  The
    # copies run on a second stream, double-buffered: step s+1's inputs go up while step s computes, and
    # step s's result (a device snapshot of X and the norms) comes down while step s+1 computes.
    Qh = torch.from_numpy(p.q).pin_memory()
    Bh = torch.from_numpy(p.b).pin_memory()
    Xh = torch.empty_like(Bh).pin_memory()
    nh = torch.empty((K, 2), dtype=torch.float64).pin_memory()
    cs = torch.cuda.Stream(device=dev)
    Qb, Bb = [Q, torch.empty_like(Q)], [B, torch.empty_like(B)]
    Xs, ns = [torch.empty_like(X) for _ in range(2)], [torch.empty_like(norms) for _ in range(2)]
    in_ready, used, out_done = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))
    for ev in used + out_done:  # recorded once, so that the first waits on them are satisfied
        ev.record(stream)

    def h2d(k):
        with torch.cuda.stream(cs):
            cs.wait_event(used[k])  # the step that last read buffer k has finished
            Qb[k].copy_(Qh, non_blocking=True)
            Bb[k].copy_(Bh, non_blocking=True)
            in_ready[k].record(cs)

    def compute(k):
        stream.wait_event(in_ready[k])
        stream.wait_event(out_done[k])  # snapshot buffer k has gone down
        fnlh.fnlh_build_jacobian(dm, Qb[k], params, J)
        fnlh.fnlh_relax(dm, J, p.omega, Bb[k], X, SWEEPS, fnlh.FNLH_F64, ws)
        fnlh.fnlh_residual(dm, J, p.omega, Bb[k], X, norms=norms, ws=ws)
        Xs[k].copy_(X, non_blocking=True)
        ns[k].copy_(norms, non_blocking=True)
        used[k].record(stream)

    def d2h(k):
        with torch.cuda.stream(cs):
            cs.wait_event(used[k])
            Xh.copy_(Xs[k], non_blocking=True)
            nh.copy_(ns[k], non_blocking=True)
            out_done[k].record(cs)

    def pipeline(n_steps):
        h2d(0)
        for s_ in range(n_steps):
            k = s_ % 2
            compute(k)
            if s_ + 1 < n_steps:
                h2d(1 - k)
            d2h(k)
        stream.wait_stream(cs)

    e2e_steps = max(2, min(args.steps, 5))
    pipeline(1)  # warm-up
    barrier(world)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    pipeline(e2e_steps)
    a1 = torch.cuda.Event(enable_timing=True)
    a1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(a0.elapsed_time(a1) / e2e_steps, world)
    e2e = {"value": world * updates / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": Qh.numel() * 8 + Bh.numel() * 8,
           "d2h_bytes_per_step": Xh.numel() * 8 + nh.numel() * 8, "ms_per_step": e2e_ms}

    # the FP64 peak the sweep is bound by, measured now (after the timed regions)
    arith = measure_arith_peaks(torch, dev, local)
    peak = arith["fp64_tflops"] * 1e12
    roofline = {"bound": "alu", "kernel": "k_sweep_f64<6> (FP64 fused sweep)",
                "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_note": traffic_note,
                "peak_source": arith["source"], "peak_probe": {k: arith[k] for k in ("fp64_shape", "clocks")},
                "peak_note": f"derived from unit counts and clocks: {FP64_PEAK_DERIVED / 1e12:.3f} TFLOP/s "
                             "(152 SMs x 2 FP64 FMA/clk x 2.07 GHz); MEASURED_PEAKS.json has no FP64 figure",
                "frac_of_derived": achieved / FP64_PEAK_DERIVED,
                "sweep_ms": sweep_ms, "flops_per_launch": flops, "alg_bytes_per_launch": bytes_alg,
                "hbm_gbs_alg": bytes_alg / (sweep_ms * 1e-3) / 1e9,
                "hbm_frac_alg": bytes_alg / (sweep_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded perturbed hex passage, flow state and right-hand sides)",
            "config": workload_config(p), "roofline": roofline, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": ck,
            "final_rel_residual": [float(x) for x in rel],
            "final_rel_residual_Rz": float(np.sqrt(np.mean(np.square(rel)))), "peaks_source": peaks_kind}

    if rank == 0 and world == 1:
        del J, ws
        torch.cuda.empty_cache()
        line["time_to_1e8"] = time_to_1e8_section(torch, fnlh, inputs, dev, with_oracle=not args.no_cpu)
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_extras:
        line["batched"] = batched_section(torch, fnlh, inputs, dev, args)
        torch.cuda.empty_cache()
        line["batched_small_rows"] = batched_small_section(torch, fnlh, inputs, dev)
        torch.cuda.empty_cache()
        line["rk_stages"] = rk_section(torch, fnlh, inputs, dev)
        torch.cuda.empty_cache()
        line["periodic"] = periodic_section(torch, fnlh, inputs, dev)
        torch.cuda.empty_cache()
        line["partitions"] = partition_section(torch, fnlh, inputs, dev)
        torch.cuda.empty_cache()
        line["ilu_vs_jacobi"] = ilu_section(torch, fnlh, inputs, dev, arith)
        torch.cuda.empty_cache()
        line["stress_permuted"] = stress_permuted_section(torch, fnlh, inputs, dev)
        if not args.no_large:
            torch.cuda.empty_cache()
            line["large"] = large_section(torch, fnlh, inputs, dev)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate(p)
        if not args.no_large:
            line["cpu_baseline"]["large"] = cpu_oracle_large()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def time_to_1e8_section(torch, fnlh, inputs, dev, with_oracle=True, tol=1e-8):
    """The metric's second half on the mixed-precision workload (160x128x102, 2.1M nodes, mean + 8
    harmonics): time to a 1e-8 relative FP64 residual for plain FP64 Jacobi (residual every 10 sweeps)
    and FP64 defect correction with FP32 and BF16 blocks.  Per precision: device-resident time, the
    same through the public API with B copied in from pinned host memory and x copied out, the residual
    the library reports per system, the oracle's FP64 residual of the returned x per system, and each
    system's error against the oracle's own solution (plain FP64 Jacobi to the same tolerance and check
    cadence on the host cores, whose time is reported too)."""
    p = inputs.config_problem("c3")
    n, b, N = p.mesh.n_nodes, p.block, p.n_harm
    dm = fnlh.DeviceMesh.from_mesh(p.mesh, dev)
    flags = fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_BF16 | fnlh.FNLH_PREP_FF
    J = fnlh.DeviceJacobian(dm, b, flags, dev)
    fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).to(dev), fnlh.make_params(p.cfl), J)
    Bh = torch.from_numpy(p.b).pin_memory()
    Xh = torch.empty_like(Bh).pin_memory()
    B = Bh.to(dev)
    X = torch.zeros_like(B)
    # the mixed solves' workspace holds the float-float shadows: their intermediate checks run on the FP32
    # units, the certifying one in FP64 (fnlh_solve); the FP64 workspace (the largest) serves the FP64 solve
    ws = fnlh.solve_workspace(n, b, N, flags, dev, fnlh.FNLH_F64)
    ws_ff = {prec: fnlh.solve_workspace(n, b, N, flags, dev, prec) for prec in (fnlh.FNLH_F32, fnlh.FNLH_BF16)}
    out = {"workload": f"c3: 160x128x102 hex passage, {n} nodes, {p.mesh.n_edges} edges, b=6, mean + {N} "
                       f"harmonics, CFL 20, to a {tol:g} relative FP64 residual per system, from zero; mixed "
                       f"solves with float-float intermediate checks and an FP64 certifying check",
           "unit": "s", "higher_is_better": False}
    # inner sweeps per FP64 residual: the best of a scan of 10..40 on this workload (every run needs
    # ~60 sweeps; each extra check costs one FP64 residual)
    # inner sweeps per correction: the fewest that keep the fewest corrections (scanned on GB300: FP32 29
    # and BF16 20 each need one more check on every workload here)
    cases = [("f64", fnlh.FNLH_F64, 10), ("f32", fnlh.FNLH_F32, 30), ("bf16", fnlh.FNLH_BF16, BF16_INNER)]
    zg = fnlh.FNLH_SOLVE_ZERO_GUESS
    sols = {}
    for name, prec, inner in cases:
        w = ws_ff.get(prec, ws)
        fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, tol, inner, 2, ws=w, raise_on_error=False, flags=zg)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, tol, inner, 200, ws=w,
                                                  raise_on_error=False, flags=zg)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        # end to end through the public API: B up from pinned host memory, the solve, x down
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        B.copy_(Bh, non_blocking=True)
        ev[1].record()
        fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, tol, inner, 200, ws=w, raise_on_error=False, flags=zg)
        ev[2].record()
        Xh.copy_(X, non_blocking=True)
        ev[3].record()
        torch.cuda.synchronize()
        e0, e1 = ev[0], ev[3]
        sols[name] = Xh.numpy().copy()
        out[name] = {"status": fnlh.fnlh_strerror(st), "seconds": t, "checks": checks, "sweeps": sweeps,
                     "inner_sweeps": inner, "max_rel_residual": float(np.max(rel)),
                     "rel_residual_per_system": [float(v) for v in rel],
                     "e2e": {"seconds": e0.elapsed_time(e1) * 1e-3, "h2d_bytes": Bh.numel() * 8,
                             "d2h_bytes": Xh.numel() * 8, "h2d_ms": ev[0].elapsed_time(ev[1]),
                             "solve_ms": ev[1].elapsed_time(ev[2]), "d2h_ms": ev[2].elapsed_time(ev[3])}}
    # the same mixed solves with every check in FP64 (the plain-size workspace has no float-float shadows)
    for name, prec, inner in cases[1:]:
        w = fnlh.workspace(n, b, N, dev, precision=prec)
        t0 = time.perf_counter()
        st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, tol, inner, 200, ws=w,
                                                  raise_on_error=False, flags=zg)
        torch.cuda.synchronize()
        out[name]["fp64_checks"] = {"seconds": time.perf_counter() - t0, "checks": checks, "sweeps": sweeps,
                                    "status": fnlh.fnlh_strerror(st), "max_rel_residual": float(np.max(rel))}
        del w
    if out["f64"]["status"] == "success":
        for name in ("f32", "bf16"):
            out[name]["speedup_vs_f64"] = out["f64"]["seconds"] / out[name]["seconds"]
            out[name]["e2e_speedup_vs_f64"] = out["f64"]["e2e"]["seconds"] / out[name]["e2e"]["seconds"]
    # the inner sweep alone: HBM roofline (algorithmic bytes, FP32 iterate)
    peaks, _ = load_peaks()
    nnz = 2 * p.mesh.n_edges
    for name, prec, sj in (("f32", fnlh.FNLH_F32, 4), ("bf16", fnlh.FNLH_BF16, 2)):
        ms = sweep_time_ms(torch, fnlh, dm, J, p, B, X, ws, prec)
        alg = sweep_bytes(n, nnz, b, N, sj, 4, 4, 4)
        out[name]["inner_sweep"] = {"ms": ms, "alg_bytes": alg, "gbs": alg / (ms * 1e-3) / 1e9,
                                    "frac_hbm": alg / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                                    "frac_hbm_nominal_7900": alg / (ms * 1e-3) / 1e9 / 7900.0}
    del dm, J, B, X, ws, ws_ff
    torch.cuda.empty_cache()
    if with_oracle:
        import oracle

        m = p.mesh
        t0 = time.perf_counter()
        oj = oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl)
        t_build = time.perf_counter() - t0
        t0 = time.perf_counter()
        xo, osw = oracle.solve_to_tol(oj, m.vol, p.omega, p.b, tol=tol, chunk=10)
        t_solve = time.perf_counter() - t0
        orel = oracle.rel_residuals(oj, m.vol, p.omega, p.b, xo)
        out["oracle"] = {"seconds": t_solve, "build_seconds": t_build, "sweeps": osw, "checks_every": 10,
                         "cores": oracle.num_threads(), "kind": "oracle (plain FP64 block Jacobi, C, OpenMP)",
                         "rel_residual_per_system": [float(v) for v in orel]}
        cols = [[0]] + [[2 * k - 1, 2 * k] for k in range(1, N + 1)]
        for name in ("f64", "f32", "bf16"):
            x = sols[name]
            out[name]["oracle_rel_residual_per_system"] = [
                float(v) for v in oracle.rel_residuals(oj, m.vol, p.omega, p.b, x)]
            out[name]["rel_error_vs_oracle_per_system"] = [
                float(np.linalg.norm(x[:, c] - xo[:, c]) / np.linalg.norm(xo[:, c])) for c in cols]
            out[name]["speedup_vs_oracle"] = t_solve / out[name]["seconds"]
        del oj, xo
    return out


def sweep_time_ms(torch, fnlh, dm, J, p, B, X, ws, prec, sweeps=10, reps=3, sigma=None):
    """Average duration of one sweep launch (CUDA events recorded by the library around its sweep launches)."""
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 2, prec, ws, sigma=sigma)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, z in ev:
        a.record()
        z.record()
    for a, z in ev:
        fnlh.fnlh_set_sweep_events(a, z)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, sweeps, prec, ws, sigma=sigma)
    torch.cuda.synchronize()
    fnlh.fnlh_set_sweep_events(None, None)
    return sum(a.elapsed_time(z) for a, z in ev) / (reps * sweeps)


def rk_section(torch, fnlh, inputs, dev):
    """Five implicit RK(5,3) stages on the FP64 workload with the paper's linear-solve rule
    (1e-2 drop, at most 10 iterations), with and without freezing converged systems."""
    from paper_2404_01407_gb300 import rk_stage

    p = inputs.config_problem(WORKLOAD)
    n, b, N = p.mesh.n_nodes, p.block, p.n_harm
    dm = fnlh.DeviceMesh.from_mesh(p.mesh, dev)
    J = fnlh.DeviceJacobian(dm, b, fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32, dev)
    fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).to(dev), fnlh.make_params(p.cfl), J)
    rng = np.random.default_rng(11)
    R = [torch.from_numpy(-p.b * (1.0 - 0.1 * k) + 0.05 * rng.normal(size=p.b.shape)).to(dev) for k in range(5)]
    ws = fnlh.workspace(n, b, N, dev)
    out = {"workload": f"{p.name}: 5 RK(5,3) stages (Table rk_coff alphas), stage solves from zero to a 1e-2 "
                       f"residual drop, <= 10 sweeps, residual checked every 2 sweeps"}
    for name, prec in (("f64", fnlh.FNLH_F64), ("f32", fnlh.FNLH_F32)):
        for mask in (False, True):
            rk_stage.run_stages(dm, J, p.omega, R, precision=prec, mask=mask, ws=ws)  # warm
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, recs = rk_stage.run_stages(dm, J, p.omega, R, precision=prec, mask=mask, ws=ws)
            torch.cuda.synchronize()
            out[f"{name}{'_masked' if mask else ''}"] = {
                "seconds": time.perf_counter() - t0, "sweeps": [r["sweeps"] for r in recs],
                "max_rel_residual": max(max(r["rel_residual"]) for r in recs)}
    return out


def periodic_section(torch, fnlh, inputs, dev):
    """Phase-lagged periodic edges on the measured workload: the same passage
    with its pitchwise boundary closed by 6,144 periodic edges, harmonic l at
    inter-blade phase angle 2 pi l 3/8.  Sweep time per precision against the
    same mesh without the closure, and the mixed FP32 solve to a 1e-8 FP64 residual (float-float
    intermediate checks with the phase factors; the all-FP64-checks time beside it)."""
    c = inputs.CONFIGS[WORKLOAD]
    out = {}
    prep = fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_BF16 | fnlh.FNLH_PREP_FF
    for tag, periodic in (("plain", False), ("periodic", True)):
        p = inputs.problem(c["dims"], c["block"], c["n_harm"], c["cfl"], c["omega_base"], name=WORKLOAD,
                           periodic=periodic)
        dm = fnlh.DeviceMesh.from_mesh(p.mesh, dev)
        J = fnlh.DeviceJacobian(dm, p.block, prep | (fnlh.FNLH_PREP_TAGS if periodic else 0), dev)
        fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).to(dev), fnlh.make_params(p.cfl), J)
        B = torch.from_numpy(p.b).to(dev)
        X = torch.zeros_like(B)
        ws = fnlh.workspace(p.mesh.n_nodes, p.block, p.n_harm, dev)
        rec = {"edges": p.mesh.n_edges}
        for name, prec in (("f64", fnlh.FNLH_F64), ("f32", fnlh.FNLH_F32), ("bf16", fnlh.FNLH_BF16)):
            rec[f"{name}_sweep_ms"] = sweep_time_ms(torch, fnlh, dm, J, p, B, X, ws, prec, sigma=p.phase)
        if periodic:
            out["workload"] = (f"{WORKLOAD} passage closed pitchwise by {int((p.mesh.periodic != 0).sum())} "
                               f"periodic edges, sigma_l = 2 pi l 3/8, l = 1..{p.n_harm}")
            def solve(w):
                fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F32, 1e-8, 12, 2, ws=w, raise_on_error=False,
                                flags=fnlh.FNLH_SOLVE_ZERO_GUESS, sigma=p.phase)  # warm
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F32, 1e-8, 12, 100, ws=w,
                                      raise_on_error=False, flags=fnlh.FNLH_SOLVE_ZERO_GUESS, sigma=p.phase)
                torch.cuda.synchronize()
                return time.perf_counter() - t0, res

            # the FP64-sized workspace holds the float-float shadows; the plain FP32 one does not
            t, (st, checks, sweeps, rel) = solve(ws)
            ws32 = fnlh.workspace(p.mesh.n_nodes, p.block, p.n_harm, dev, precision=fnlh.FNLH_F32)
            t64, (st64, checks64, sweeps64, rel64) = solve(ws32)
            del ws32
            rec["mixed_f32_solve"] = {"status": fnlh.fnlh_strerror(st), "seconds": t, "checks": checks,
                                      "sweeps": sweeps, "max_rel_residual": float(np.max(rel)),
                                      "fp64_checks": {"seconds": t64, "checks": checks64, "sweeps": sweeps64,
                                                      "max_rel_residual": float(np.max(rel64))}}
        out[tag] = rec
        del dm, J, B, X, ws
        torch.cuda.empty_cache()
    for name in ("f64", "f32", "bf16"):
        out[f"{name}_overhead"] = out["periodic"][f"{name}_sweep_ms"] / out["plain"][f"{name}_sweep_ms"] - 1.0
    return out


def ilu_pass_roofline(torch, fnlh, dm, J, ilu, p, B, X, ws, prec, arith, reps=3):
    """Colour passes of one ILU(0) iteration (forward + backward, all colours):
    CUDA-event time on the launching stream (the library's timing hook brackets
    the passes of the last iteration), algorithmic flops and bytes per
    iteration, and their fractions of the measured arithmetic peak of the
    passes' own precision (FP64 or FP32, from the multiply-add probe) and of
    the measured HBM peak."""
    n, b, N = p.mesh.n_nodes, p.block, p.n_harm
    K, C = 1 + N, 1 + 2 * N
    nnz = 2 * p.mesh.n_edges
    color = ilu.color_host
    rp, ci = dm.row_ptr_host, dm.col_idx_host
    owner = np.repeat(np.arange(n), np.diff(rp))
    n_upper = int(np.unique(owner[color[ci] > color[owner]]).shape[0])
    # gathers: 2 flops per structurally nonzero block entry and real column (the mean flow is one real
    # column, a harmonic two); pivots: a dense complex P^-1 per harmonic, a real one for the mean flow
    e = b * b - (b - 1) if fnlh.fnlh_prep_structured(J) else b * b
    flops = 2 * e * nnz * C + (n + n_upper) * (8 * b * b * N + 2 * b * b)
    if prec == fnlh.FNLH_F64:  # original basis: FP64 blocks, r read and x updated in the caller's layout
        bytes_ = ((n + n_upper) * K * b * b * 2 * 8 + nnz * b * b * 8 + n * C * b * 8 + 4 * n * K * 2 * b * 8
                  + 2 * n * C * b * 8 + nnz * 4 + n * 8)
    else:  # Schur basis: FP32 blocks and rotated FP32 residual; x += Q e runs after the passes
        bytes_ = ((n + n_upper) * K * b * b * 2 * 4 + nnz * b * b * 4 + n * K * 2 * b * 4 + 4 * n * K * 2 * b * 4
                  + nnz * 4 + n * 8)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, z in ev:
        a.record()
        z.record()
    for a, z in ev:
        fnlh.fnlh_set_sweep_events(a, z)
        fnlh.fnlh_solve_ilu(dm, J, ilu, p.omega, B, X, 0.0, 2, ws=ws, raise_on_error=False)
    torch.cuda.synchronize()
    fnlh.fnlh_set_sweep_events(None, None)
    ms = sum(a.elapsed_time(z) for a, z in ev) / reps
    peaks, _ = load_peaks()
    tflops = flops / (ms * 1e-3) / 1e12
    out = {"ms": ms, "flops": flops, "alg_bytes": bytes_, "tflops": tflops, "gbs": bytes_ / (ms * 1e-3) / 1e9,
           "frac_hbm": bytes_ / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
    if prec == fnlh.FNLH_F64:
        out["frac_fp64_peak"] = tflops / arith["fp64_tflops"]
    else:
        out["frac_fp32_peak"] = tflops / arith["fp32_tflops"]
    return out


def ilu_section(torch, fnlh, inputs, dev, arith, tol=1e-8):
    """The paper's smoother, block ILU(0) in red-black order, against block
    Jacobi on the measured passage: iterations and time to a 1e-8 FP64
    residual, and the paper's stage rule (1e-2 drop from zero, at most 10).  The FP32 forms (ILU(0) with
    an FP32 factor, Jacobi defect correction) take their intermediate residuals in float-float
    (FNLH_PREP_FF), the final one in FP64."""
    p = inputs.config_problem(WORKLOAD)
    n, b, N = p.mesh.n_nodes, p.block, p.n_harm
    dm = fnlh.DeviceMesh.from_mesh(p.mesh, dev)
    J = fnlh.DeviceJacobian(dm, b, fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_FF, dev)
    fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).to(dev), fnlh.make_params(p.cfl), J)
    B = torch.from_numpy(p.b).to(dev)
    X = torch.zeros_like(B)
    ws = fnlh.workspace(n, b, N, dev)
    zg = fnlh.FNLH_SOLVE_ZERO_GUESS
    out = {"workload": f"{WORKLOAD}: mean + {N} harmonics, to {tol:g} and the paper's stage rule"}

    def timed(fn):
        fn()  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, res

    for name, prec in (("ilu_f64", fnlh.FNLH_F64), ("ilu_f32", fnlh.FNLH_F32)):
        ilu = fnlh.DeviceIlu(dm, b, N, precision=prec, device=dev)
        tf, _ = timed(lambda: fnlh.fnlh_ilu_factor(dm, J, p.omega, ilu, ws=ws))
        t, (st, its, rel) = timed(lambda: fnlh.fnlh_solve_ilu(dm, J, ilu, p.omega, B, X, tol, 200, ws=ws, flags=zg,
                                                              raise_on_error=False))
        _, (st2, its2, rel2) = timed(lambda: fnlh.fnlh_solve_ilu(dm, J, ilu, p.omega, B, X, 1e-2, 10, ws=ws,
                                                                 flags=zg, raise_on_error=False))
        out[name] = {"colors": ilu.n_colors, "factor_seconds": tf, "status": fnlh.fnlh_strerror(st),
                     "iterations": its, "seconds": t, "max_rel_residual": float(np.max(rel)),
                     "stage_rule_iterations": its2, "factor_bytes": int(ilu.factor.numel()),
                     "passes": ilu_pass_roofline(torch, fnlh, dm, J, ilu, p, B, X, ws, prec, arith)}
        del ilu
        torch.cuda.empty_cache()
    # the colour passes read every array in colour order: with the nodes
    # numbered by colour each pass streams contiguous memory
    perm = np.argsort(inputs.lattice_colors(inputs.CONFIGS[WORKLOAD]["dims"]), kind="stable")
    pm, _ = inputs.permute_mesh(p.mesh, perm=perm)
    dmc = fnlh.DeviceMesh.from_mesh(pm, dev)
    Jc = fnlh.DeviceJacobian(dmc, b, fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_FF, dev)
    fnlh.fnlh_build_jacobian(dmc, torch.from_numpy(p.q[perm]).to(dev), fnlh.make_params(p.cfl), Jc)
    Bc = torch.from_numpy(p.b[perm]).to(dev)
    for name, prec in (("ilu_f64_colour_numbered", fnlh.FNLH_F64), ("ilu_f32_colour_numbered", fnlh.FNLH_F32)):
        ilu = fnlh.DeviceIlu(dmc, b, N, precision=prec, device=dev)
        fnlh.fnlh_ilu_factor(dmc, Jc, p.omega, ilu, ws=ws)
        t, (st, its, rel) = timed(lambda: fnlh.fnlh_solve_ilu(dmc, Jc, ilu, p.omega, Bc, X, tol, 200, ws=ws,
                                                              flags=zg, raise_on_error=False))
        out[name] = {"status": fnlh.fnlh_strerror(st), "iterations": its, "seconds": t,
                     "max_rel_residual": float(np.max(rel)),
                     "passes": ilu_pass_roofline(torch, fnlh, dmc, Jc, ilu, p, Bc, X, ws, prec, arith)}
        del ilu
    del dmc, Jc, Bc
    torch.cuda.empty_cache()
    for name, prec, inner in (("jacobi_f64", fnlh.FNLH_F64, 10), ("jacobi_f32", fnlh.FNLH_F32, 12)):
        t, (st, checks, sweeps, rel) = timed(lambda: fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, tol, inner, 200,
                                                                     ws=ws, flags=zg, raise_on_error=False))
        _, (st2, c2, sw2, rel2) = timed(lambda: fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F64, 1e-2, 1, 11,
                                                                ws=ws, flags=zg, raise_on_error=False))
        out[name] = {"status": fnlh.fnlh_strerror(st), "sweeps": sweeps, "seconds": t,
                     "max_rel_residual": float(np.max(rel)), "stage_rule_sweeps": sw2,
                     "stage_rule_status": fnlh.fnlh_strerror(st2)}
    return out


def partition_section(torch, fnlh, inputs, dev, tol=1e-8, inner=12):
    """Domain-truncated sweeps (the paper's parallel decomposition drops the
    couplings between partitions) on the measured passage cut into 1 to 4,096
    boxes: FP32 defect correction to a 1e-8 FP64 residual -- the full residual
    wins back what the truncated sweeps leave out -- and its cost as the
    boxes shrink."""
    c = inputs.CONFIGS[WORKLOAD]
    p = inputs.config_problem(WORKLOAD)
    n = p.mesh.n_nodes
    B = torch.from_numpy(p.b).to(dev)
    X = torch.zeros_like(B)
    ws = fnlh.workspace(n, p.block, p.n_harm, dev)
    out = {"workload": f"{WORKLOAD}: FP32 blocks, {inner} truncated inner sweeps per FP64 residual, "
                       f"to {tol:g}; boxes px x py x pz of the 128x64x48 lattice"}
    zg = fnlh.FNLH_SOLVE_ZERO_GUESS
    for parts in ((1, 1, 1), (2, 2, 2), (4, 4, 4), (8, 8, 8), (16, 16, 16)):
        part = inputs.box_partition(c["dims"], parts)
        dm = fnlh.DeviceMesh.from_mesh(p.mesh, dev, part=part)
        J = fnlh.DeviceJacobian(dm, p.block, fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_TAGS, dev)
        fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).to(dev), fnlh.make_params(p.cfl), J)
        fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F32, tol, inner, 2, ws=ws, raise_on_error=False, flags=zg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F32, tol, inner, 200, ws=ws,
                                                  raise_on_error=False, flags=zg)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        nparts = parts[0] * parts[1] * parts[2]
        out[f"parts_{nparts}"] = {"nodes_per_part": n // nparts, "status": fnlh.fnlh_strerror(st), "checks": checks,
                                  "sweeps": sweeps, "seconds": t, "max_rel_residual": float(np.max(rel))}
        del dm, J
        torch.cuda.empty_cache()
    return out


def large_section(torch, fnlh, inputs, dev, tol=1e-8):
    """c5: 256x200x156 (8M nodes), b=6, mean + 16 harmonics, BF16 blocks with FP64 defect correction
    (float-float intermediate checks, FP64 certifying check; the all-FP64-checks time beside it);
    Jacobian bytes for N=1 and N=16; peak device memory."""
    c = inputs.CONFIGS["c5"]
    mesh = inputs.hex_mesh(*c["dims"])
    q = inputs.flow_state(mesh.n_nodes, 6)
    n = mesh.n_nodes
    dm = fnlh.DeviceMesh.from_mesh(mesh, dev)
    prep = fnlh.FNLH_PREP_BF16 | fnlh.FNLH_PREP_FF
    J = fnlh.DeviceJacobian(dm, 6, prep, dev)
    fnlh.fnlh_build_jacobian(dm, torch.from_numpy(q).to(dev), fnlh.make_params(c["cfl"]), J)
    del q
    out = {"workload": f"c5: 256x200x156 hex passage, {n} nodes, {mesh.n_edges} edges, b=6, CFL {c['cfl']:g}, "
                       f"BF16 blocks, FP64 defect correction to {tol:g} ({BF16_INNER} inner sweeps per correction, "
                       f"float-float intermediate checks)",
           "jacobian_bytes": J.nbytes()}
    peaks, _ = load_peaks()
    for N in (16, 1):
        torch.cuda.reset_peak_memory_stats(dev)
        Bh = inputs.rhs(n, 6, N)
        B = torch.from_numpy(Bh).to(dev)
        del Bh
        X = torch.empty_like(B)
        ws = fnlh.solve_workspace(n, 6, N, prep, dev, fnlh.FNLH_BF16)
        om = inputs.omegas(N)
        zg = fnlh.FNLH_SOLVE_ZERO_GUESS
        fnlh.fnlh_solve(dm, J, om, B, X, fnlh.FNLH_BF16, tol, BF16_INNER, 1, ws=ws, raise_on_error=False, flags=zg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, om, B, X, fnlh.FNLH_BF16, tol, BF16_INNER, 200, ws=ws,
                                                  raise_on_error=False, flags=zg)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        peak = torch.cuda.max_memory_allocated(dev)
        # the same solve with every check in FP64 (the plain workspace holds no float-float shadows)
        ws64 = fnlh.workspace(n, 6, N, dev, precision=fnlh.FNLH_BF16)
        t0 = time.perf_counter()
        st64, checks64, sweeps64, rel64 = fnlh.fnlh_solve(dm, J, om, B, X, fnlh.FNLH_BF16, tol, BF16_INNER, 200,
                                                          ws=ws64, raise_on_error=False, flags=zg)
        torch.cuda.synchronize()
        fp64_checks = {"seconds": time.perf_counter() - t0, "checks": checks64, "sweeps": sweeps64,
                       "status": fnlh.fnlh_strerror(st64), "max_rel_residual": float(np.max(rel64))}
        del ws64

        class _P:
            omega = om
        ms = sweep_time_ms(torch, fnlh, dm, J, _P, B, X, ws, fnlh.FNLH_BF16)
        alg = sweep_bytes(n, 2 * mesh.n_edges, 6, N, 2, 4, 4, 4)
        out[f"N{N}"] = {"status": fnlh.fnlh_strerror(st), "seconds": t, "checks": checks, "sweeps": sweeps,
                        "max_rel_residual": float(np.max(rel)), "jacobian_bytes": J.nbytes(),
                        "workspace_bytes": ws.numel(), "vector_bytes": 2 * B.numel() * 8,
                        "updates_per_s": n * (1 + N) * sweeps / t,
                        "inner_sweep": {"ms": ms, "alg_bytes": alg, "gbs": alg / (ms * 1e-3) / 1e9,
                                        "frac_hbm": alg / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]},
                        "peak_device_bytes": peak, "fp64_checks": fp64_checks}
        del B, X, ws
        torch.cuda.empty_cache()
    out["jacobian_bytes_independent_of_N"] = out["N1"]["jacobian_bytes"] == out["N16"]["jacobian_bytes"]
    return out


def batched_section(torch, fnlh, inputs, dev, args, sweeps=20, prec_name="bf16"):
    """Three blade rows: one persistent launch per sweep (graph-captured) vs per-row launches."""
    prec = fnlh.PRECISIONS[prec_name]
    rows = []
    for key in ("c4_row0", "c4_row1", "c4_row2"):
        c = inputs.CONFIGS[key]
        p = inputs.problem(c["dims"], c["block"], c["n_harm"], c["cfl"], c["omega_base"], name=key)
        dm = fnlh.DeviceMesh.from_mesh(p.mesh, dev)
        J = fnlh.DeviceJacobian(dm, p.block, fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_BF16
                                | fnlh.FNLH_PREP_FF, dev)
        fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).to(dev), fnlh.make_params(p.cfl), J)
        B = torch.from_numpy(p.b).to(dev)
        rows.append((p, dm, J, B, torch.zeros_like(B),
                     fnlh.workspace(p.mesh.n_nodes, p.block, p.n_harm, dev, precision=fnlh.FNLH_F64)))
    updates = sum(p.mesh.n_nodes * (1 + p.n_harm) for p, *_ in rows) * sweeps

    def per_row():
        for p, dm, J, B, X, ws in rows:
            fnlh.fnlh_relax(dm, J, p.omega, B, X, sweeps, prec, ws)

    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for p, dm, J, B, X, ws in rows])
    bws = torch.empty(batch.workspace_bytes(6), dtype=torch.uint8, device=dev)

    def batched(tn=None):
        fnlh.fnlh_relax_batched(batch, sweeps, prec, tuning=tn, ws=bws)

    def timeit(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    from paper_2404_01407_gb300 import autotune

    best, table = autotune.tune_batched(lambda tn: timeit(lambda: batched(tn), reps=2))
    t_rows = timeit(per_row)
    t_batch = timeit(lambda: batched(best))
    # CUDA graph of the whole batched call
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        batched(best)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            batched(best)
    torch.cuda.current_stream().wait_stream(s)
    t_graph = timeit(g.replay)
    # the solve: mixed-precision batched defect correction against plain FP64 per-row solves, to 1e-8
    zg = fnlh.FNLH_SOLVE_ZERO_GUESS
    solves = {}

    def fp64_rows():
        out = 0
        for p, dm, J, B, X, ws in rows:
            st, c, sw, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F64, 1e-8, 10, 200, ws=ws, flags=zg,
                                             raise_on_error=False)
            assert st == fnlh.FNLH_OK, fnlh.fnlh_strerror(st)
            out = max(out, sw)
        return out

    for name, fn in (("fp64_per_row", fp64_rows),):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sw = fn()
        torch.cuda.synchronize()
        solves[name] = {"seconds": time.perf_counter() - t0, "max_sweeps": sw}
    for pname, pc, inner in (("f32", fnlh.FNLH_F32, 30), ("bf16", fnlh.FNLH_BF16, BF16_INNER)):
        sb = fnlh.BatchedRows([(dm, J, p.omega, B, X) for p, dm, J, B, X, ws in rows])
        entry = {}
        for ff in (True, False):  # float-float intermediate checks (the headline), then every check in FP64
            sws = torch.empty(sb.workspace_bytes(6, pc, ff=ff), dtype=torch.uint8, device=dev)
            fnlh.fnlh_solve_batched(sb, pc, 1e-8, inner, 200, ws=sws, flags=zg, raise_on_error=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, c, sw, rel = fnlh.fnlh_solve_batched(sb, pc, 1e-8, inner, 200, ws=sws, flags=zg,
                                                     raise_on_error=False)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            res = {"status": fnlh.fnlh_strerror(st), "seconds": t, "checks": c, "sweeps": sw,
                   "max_rel_residual": float(np.max(rel))}
            if ff:
                entry = dict(res, inner_sweeps=inner,
                             speedup_vs_fp64_per_row=solves["fp64_per_row"]["seconds"] / t)
            else:
                entry["fp64_checks"] = res
            del sws
        solves[f"batched_{pname}"] = entry
    return {"workload": "c4: rows 80x50x50 (N=2), 100x75x80 (N=8), 125x110x80 (N=4), b=6, "
                        f"{sweeps} {prec_name} sweeps", "per_row_ms": t_rows, "batched_ms": t_batch,
            "solve_to_1e-8": solves,
            "batched_graph_ms": t_graph, "tuning": {"threads": best.threads, "ctas_per_sm": best.ctas_per_sm},
            "updates_per_s_graph": updates / (t_graph * 1e-3), "speedup_vs_per_row": t_rows / t_graph,
            "tuning_table": table}


def batched_small_section(torch, fnlh, inputs, dev, sweeps=20):
    """Rows the size of the paper's compressor (33k nodes) and turbine (72k nodes) meshes, where a sweep
    takes microseconds: per-row launches against one batched launch per sweep, eager and captured in a
    CUDA graph."""
    specs = [("compressor-size row", (42, 28, 28), 4, 1.0, (1, 2, 3)),
             ("turbine-size row", (60, 40, 30), 4, 1.6, (4, 5, 6))]
    rows = []
    for name, dims, N, ob, seeds in specs:
        p = inputs.problem(dims, 6, N, 20.0, ob, seeds=seeds, name=name)
        dm = fnlh.DeviceMesh.from_mesh(p.mesh, dev)
        J = fnlh.DeviceJacobian(dm, 6, fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_BF16, dev)
        fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).to(dev), fnlh.make_params(p.cfl), J)
        B = torch.from_numpy(p.b).to(dev)
        rows.append((p, dm, J, B, torch.zeros_like(B),
                     fnlh.workspace(p.mesh.n_nodes, 6, N, dev, precision=fnlh.FNLH_F32)))
    updates = sum(p.mesh.n_nodes * (1 + p.n_harm) for p, *_ in rows) * sweeps

    def timeit(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def graphed(fn):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            fn()
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                fn()
        torch.cuda.current_stream().wait_stream(s)
        return g

    out = {"workload": "rows 42x28x28 (32,928 nodes) and 60x40x30 (72,000 nodes), b=6, mean + 4 harmonics, "
                       f"{sweeps} sweeps"}
    for pname in ("bf16", "f32"):
        prec = fnlh.PRECISIONS[pname]

        def per_row():
            for p, dm, J, B, X, ws in rows:
                fnlh.fnlh_relax(dm, J, p.omega, B, X, sweeps, prec, ws)

        batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for p, dm, J, B, X, ws in rows])
        bws = torch.empty(batch.workspace_bytes(6, prec), dtype=torch.uint8, device=dev)

        def batched():
            fnlh.fnlh_relax_batched(batch, sweeps, prec, ws=bws)

        g_rows, g_batch = graphed(per_row), graphed(batched)
        t = {"per_row_ms": timeit(per_row), "batched_ms": timeit(batched),
             "per_row_graph_ms": timeit(g_rows.replay), "batched_graph_ms": timeit(g_batch.replay)}
        t["updates_per_s_batched_graph"] = updates / (t["batched_graph_ms"] * 1e-3)
        t["speedup_batched_graph_vs_per_row"] = t["per_row_ms"] / t["batched_graph_ms"]
        out[pname] = t
        del g_rows, g_batch, bws
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fnlh", choices=["fnlh", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=["c1", "c2"],
                    help="c2 (128x64x48, the measured configuration) or c1 (16x8x8, a quick check)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_fnlh(args)


if __name__ == "__main__":
    main()
