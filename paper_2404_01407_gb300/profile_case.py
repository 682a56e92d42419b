"""Run one operation of one seeded workload a fixed number of times.

A driver for profilers (ncu): it sets the problem up, runs `--warm` untimed
calls, then `--reps` calls of the chosen operation, and prints their mean
time from CUDA events.

  python -m paper_2404_01407_gb300.profile_case --op relax --prec bf16 --dims 96 96 64 --harm 8
  python -m paper_2404_01407_gb300.profile_case --op batched --prec bf16 --rows 60,40,40,2 75,56,60,8 94,82,60,4
"""

from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import fnlh, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["relax", "residual", "build", "solve", "ilu", "batched"], default="relax")
    ap.add_argument("--prec", choices=list(fnlh.PRECISIONS), default="f64")
    ap.add_argument("--dims", type=int, nargs=3, default=[128, 64, 48])
    ap.add_argument("--block", type=int, default=6)
    ap.add_argument("--harm", type=int, default=4)
    ap.add_argument("--cfl", type=float, default=20.0)
    ap.add_argument("--sweeps", type=int, default=1)
    ap.add_argument("--warm", type=int, default=2)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--ff", action="store_true", help="--op solve: float-float checks (FNLH_PREP_FF, solve workspace)")
    ap.add_argument("--rows", nargs="+", default=["60,40,40,2", "75,56,60,8", "94,82,60,4"],
                    help="--op batched: blade rows as nx,ny,nz,harmonics (row r: omega base 1 + 0.65 r)")
    ap.add_argument("--threads", type=int, default=0, help="--op batched: fnlh_tuning.threads (0: default)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="--op batched: fnlh_tuning.ctas_per_sm")
    a = ap.parse_args()
    if a.op == "batched":
        return batched(a)
    prec = fnlh.PRECISIONS[a.prec]
    p = inputs.problem(tuple(a.dims), a.block, a.harm, a.cfl, name="profile")
    dev = torch.device("cuda")
    dm = fnlh.DeviceMesh.from_mesh(p.mesh, dev)
    prep = fnlh.PREP_FOR.get(prec, fnlh.FNLH_PREP_F64) | (fnlh.FNLH_PREP_FF if a.ff else 0)
    J = fnlh.DeviceJacobian(dm, a.block, prep, dev)
    Q = torch.from_numpy(p.q).to(dev)
    params = fnlh.make_params(p.cfl)
    fnlh.fnlh_build_jacobian(dm, Q, params, J)
    B = torch.from_numpy(p.b).to(dev)
    X = torch.zeros_like(B)
    ws = fnlh.workspace(p.mesh.n_nodes, a.block, a.harm, dev)
    if a.ff:
        ws = fnlh.solve_workspace(p.mesh.n_nodes, a.block, a.harm, prep, dev, prec)
    ilu = None
    if a.op == "ilu":  # factor once; each call runs `--sweeps` ILU(0) iterations
        ilu = fnlh.DeviceIlu(dm, a.block, a.harm, precision=prec, device=dev)
        fnlh.fnlh_ilu_factor(dm, J, p.omega, ilu, ws=ws)

    def op():
        if a.op == "relax":
            fnlh.fnlh_relax(dm, J, p.omega, B, X, a.sweeps, prec, ws)
        elif a.op == "residual":
            fnlh.fnlh_residual(dm, J, p.omega, B, X, ws=ws)
        elif a.op == "build":
            fnlh.fnlh_build_jacobian(dm, Q, params, J)
        elif a.op == "ilu":
            fnlh.fnlh_solve_ilu(dm, J, ilu, p.omega, B, X, 0.0, a.sweeps, ws=ws, raise_on_error=False)
        else:
            fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 1e-8, a.sweeps, 50, ws=ws, flags=fnlh.FNLH_SOLVE_ZERO_GUESS)

    for _ in range(a.warm):
        op()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sw = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.reps)]
    for b, e in sw:  # torch creates the CUDA event on its first record
        b.record()
        e.record()
    e0.record()
    for r in range(a.reps):
        if a.op in ("relax", "ilu"):
            fnlh.fnlh_set_sweep_events(*sw[r])
        op()
    e1.record()
    torch.cuda.synchronize()
    fnlh.fnlh_set_sweep_events(None, None)
    out = {"op": a.op, "prec": a.prec, "dims": a.dims, "harm": a.harm, "nodes": p.mesh.n_nodes,
           "ms_per_call": e0.elapsed_time(e1) / max(a.reps, 1),
           "finite": bool(np.isfinite(X.cpu().numpy()).all())}
    if a.op == "relax" and a.reps > 0 and a.sweeps > 0:
        out["ms_per_sweep"] = sum(b.elapsed_time(e) for b, e in sw) / (a.reps * a.sweeps)
    if a.op == "ilu" and a.reps > 0 and a.sweeps > 0:  # the hook brackets the last iteration's passes
        out["ms_passes_per_iteration"] = sum(b.elapsed_time(e) for b, e in sw) / a.reps
    print(json.dumps(out))


def batched(a):
    """Blade rows through fnlh_relax_batched: `--warm` untimed calls, then
    `--reps` timed calls of `--sweeps` sweeps each."""
    prec = fnlh.PRECISIONS[a.prec]
    dev = torch.device("cuda")
    rows, keep = [], []
    for r, spec in enumerate(a.rows):
        nx, ny, nz, N = (int(v) for v in spec.split(","))
        p = inputs.problem((nx, ny, nz), a.block, N, a.cfl, 1.0 + 0.65 * r, seeds=(1 + 3 * r, 2 + 3 * r, 3 + 3 * r))
        dm = fnlh.DeviceMesh.from_mesh(p.mesh, dev)
        J = fnlh.DeviceJacobian(dm, a.block, fnlh.PREP_FOR.get(prec, fnlh.FNLH_PREP_F64), dev)
        fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).to(dev), fnlh.make_params(p.cfl), J)
        B = torch.from_numpy(p.b).to(dev)
        X = torch.zeros_like(B)
        rows.append((dm, J, p.omega, B, X))
        keep.append(p.mesh.n_nodes)
    batch = fnlh.BatchedRows(rows)
    ws = torch.empty(batch.workspace_bytes(a.block, prec), dtype=torch.uint8, device=dev)
    tn = fnlh.fnlh_tuning(a.threads, a.ctas_per_sm)
    for _ in range(a.warm):
        fnlh.fnlh_relax_batched(batch, a.sweeps, prec, tuning=tn, ws=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        fnlh.fnlh_relax_batched(batch, a.sweeps, prec, tuning=tn, ws=ws)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"op": "batched", "prec": a.prec, "rows": a.rows, "nodes": keep,
                      "ms_per_call": e0.elapsed_time(e1) / max(a.reps, 1),
                      "finite": all(bool(torch.isfinite(r[4]).all()) for r in rows)}))


if __name__ == "__main__":
    main()
