"""GPU: batched solve over several blade rows (one launch per inner sweep
covering every row) against the per-row solves and the oracle.

With tol = 0 both run the same number of checks and sweeps: the mixed
batched solve equals the per-row mixed solves bit for bit (same tile body,
residual and update), the FP64 batched solve equals the per-row FP64 solves
to 1e-13 (the batched FP64 tile takes the complex path for the mean flow).
Solved to 1e-8, every row's true FP64 residual (oracle) is below 1e-8.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2404_01407_gb300 import fnlh, inputs
from tests import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    fnlh.lib()


def rows_problem():
    return [inputs.problem((9, 7, 5), 6, 2, 20.0, 1.0, seeds=(1, 2, 3)),
            inputs.problem((12, 8, 6), 6, 8, 20.0, 1.6, seeds=(4, 5, 6)),
            inputs.problem((10, 9, 7), 6, 4, 20.0, 2.3, seeds=(7, 8, 9))]


def device_rows(probs, part=None, prep=_gpu.ALL_PREP | fnlh.FNLH_PREP_TAGS):
    dev = []
    for q, p in enumerate(probs):
        pa = None if part is None else part[q]
        dm = fnlh.DeviceMesh.from_mesh(p.mesh, "cuda", part=pa)
        J = fnlh.DeviceJacobian(dm, p.block, prep)
        fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).cuda(), fnlh.make_params(p.cfl), J)
        dev.append((p, dm, J, torch.from_numpy(p.b).cuda()))
    return dev


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16, fnlh.FNLH_F64])
def test_batched_solve_equals_per_row_solves(prec):
    dev = device_rows(rows_problem())
    inner, checks = 6, 4
    singles = []
    for p, dm, J, B in dev:
        X = torch.zeros_like(B)
        st, c, sw, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 0.0, inner, checks, raise_on_error=False)
        assert st == fnlh.FNLH_ERR_NOT_CONVERGED and c == checks
        singles.append(X.cpu().numpy())
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6, prec), dtype=torch.uint8, device="cuda")
    st, c, sw, rel = fnlh.fnlh_solve_batched(batch, prec, 0.0, inner, checks, ws=ws, raise_on_error=False)
    assert st == fnlh.FNLH_ERR_NOT_CONVERGED and c == checks and sw == inner * (checks - 1)
    assert rel.shape == (3 + 9 + 5,)
    for X, ref, (p, *_r) in zip(Xs, singles, dev):
        if prec == fnlh.FNLH_F64:
            _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm, tol=1e-13)
        else:
            assert np.array_equal(X.cpu().numpy(), ref)


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16])
def test_batched_mixed_solve_reaches_1e8(prec):
    probs = rows_problem()
    dev = device_rows(probs)
    Xs = [torch.full_like(B, 7.0) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6, prec), dtype=torch.uint8, device="cuda")
    flags = fnlh.FNLH_SOLVE_ZERO_GUESS | fnlh.FNLH_SOLVE_MASK_CONVERGED
    st, c, sw, rel = fnlh.fnlh_solve_batched(batch, prec, 1e-8, 12, 60, ws=ws, flags=flags)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-8), (st, rel)
    for X, p in zip(Xs, probs):
        oj = _gpu.oracle_jacobian(p)
        true_rel = oracle.rel_residuals(oj, p.mesh.vol, p.omega, p.b, X.cpu().numpy())
        assert np.all(true_rel <= 1e-8), true_rel


@pytest.mark.parametrize("ff", [False, True])
def test_batched_solve_with_partitioned_and_periodic_rows(ff):
    """ff: float-float intermediate checks (with the periodic row's phase
    factors and the partitioned row's full couplings)."""
    probs = [inputs.problem((12, 8, 6), 6, 4, 20.0, 1.6, seeds=(4, 5, 6)),
             inputs.problem((10, 6, 7), 6, 3, 20.0, 2.3, seeds=(7, 8, 9), periodic=True)]
    parts = [inputs.box_partition((12, 8, 6), (2, 2, 1)), None]
    prep = _gpu.ALL_PREP | fnlh.FNLH_PREP_TAGS | (fnlh.FNLH_PREP_FF if ff else 0)
    dev = device_rows(probs, parts, prep=prep)
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X, p.phase) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6, fnlh.FNLH_F32, ff=ff), dtype=torch.uint8, device="cuda")
    st, c, sw, rel = fnlh.fnlh_solve_batched(batch, fnlh.FNLH_F32, 1e-8, 12, 60, ws=ws)
    assert st == fnlh.FNLH_OK
    for X, p in zip(Xs, probs):
        m = p.mesh
        oj = oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl, periodic=m.periodic)
        true_rel = oracle.rel_residuals(oj, m.vol, p.omega, p.b, X.cpu().numpy(), sigma=p.phase)
        assert np.all(true_rel <= 1e-8), true_rel
    ws64 = torch.empty(batch.workspace_bytes(6), dtype=torch.uint8, device="cuda")
    with pytest.raises(fnlh.FnlhError) as e:
        fnlh.fnlh_solve_batched(batch, fnlh.FNLH_F64, 1e-8, 10, 60, ws=ws64)
    assert e.value.status == fnlh.FNLH_ERR_UNSUPPORTED


def _capture(fn):
    """Capture fn() in a CUDA graph on a side stream (one warm-up call first)."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        fn(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            fn(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("tuning", [None, (64, 0), (128, 2)])
def test_batched_relax_graph_replay_matches_oracle(tuning):
    """The benchmark's timed form of the batched launch: fnlh_relax_batched
    captured once in a CUDA graph and replayed.  FP64 replays match the
    oracle's Jacobi row by row (every entry within 1e-12 of the system's
    largest); BF16 replays equal the direct call bit for bit and stay within
    the low-precision bound of the oracle; two replays give identical bits."""
    sweeps = 15
    probs = rows_problem()
    dev = device_rows(probs)
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    tn = None if tuning is None else fnlh.fnlh_tuning(*tuning)
    refs = [oracle.jacobi(_gpu.oracle_jacobian(p), p.mesh.vol, p.omega, p.b, sweeps) for p in probs]
    for prec in (fnlh.FNLH_F64, fnlh.FNLH_BF16):
        ws = torch.empty(batch.workspace_bytes(6, prec), dtype=torch.uint8, device="cuda")
        for X in Xs:
            X.zero_()
        fnlh.fnlh_relax_batched(batch, sweeps, prec, tuning=tn, ws=ws)
        direct = [X.clone() for X in Xs]
        g = _capture(lambda s: fnlh.fnlh_relax_batched(batch, sweeps, prec, tuning=tn, ws=ws, stream=s))
        replays = []
        for _ in range(2):
            for X in Xs:
                X.zero_()
            g.replay()
            torch.cuda.synchronize()
            replays.append([X.clone() for X in Xs])
        for X1, X2, Xd, ref, p in zip(replays[0], replays[1], direct, refs, probs):
            assert torch.equal(X1, X2)
            assert torch.equal(X1, Xd)
            if prec == fnlh.FNLH_F64:
                _gpu.assert_fp64_parity(X1.cpu().numpy(), ref, p.n_harm)
            else:
                err = _gpu.rel_err_per_system(X1.cpu().numpy(), ref, p.n_harm)
                assert np.all(err <= 5e-2), err
        del g, ws


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16, fnlh.FNLH_F64])
def test_per_row_mode_equals_single_row_calls(prec):
    """fnlh_tuning.ctas_per_sm = FNLH_TUNING_PER_ROW runs every row's own
    single-row sweeps: the batched relax and the batched solve then equal the
    per-row calls bit for bit in every precision (the FP64 one included,
    whose shared-launch tile takes the complex path for the mean flow), also
    when the batched relax is replayed from a CUDA graph."""
    tn = fnlh.fnlh_tuning(0, fnlh.FNLH_TUNING_PER_ROW)
    dev = device_rows(rows_problem())
    sweeps = 7
    singles = []
    for p, dm, J, B in dev:
        X = torch.zeros_like(B)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, sweeps, prec)
        singles.append(X.clone())
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6, prec), dtype=torch.uint8, device="cuda")
    fnlh.fnlh_relax_batched(batch, sweeps, prec, tuning=tn, ws=ws)
    for X, ref in zip(Xs, singles):
        assert torch.equal(X, ref)
    g = _capture(lambda s: fnlh.fnlh_relax_batched(batch, sweeps, prec, tuning=tn, ws=ws, stream=s))
    for X in Xs:
        X.zero_()
    g.replay()
    torch.cuda.synchronize()
    for X, ref in zip(Xs, singles):
        assert torch.equal(X, ref)
    del g
    # the solve: same checks, sweeps and bits as the per-row solves
    inner, checks = 6, 4
    solos = []
    for p, dm, J, B in dev:
        X = torch.zeros_like(B)
        fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 0.0, inner, checks, raise_on_error=False)
        solos.append(X.clone())
    for X in Xs:
        X.zero_()
    st, c, sw, rel = fnlh.fnlh_solve_batched(batch, prec, 0.0, inner, checks, tuning=tn, ws=ws,
                                             raise_on_error=False)
    assert st == fnlh.FNLH_ERR_NOT_CONVERGED and c == checks and sw == inner * (checks - 1)
    for X, ref in zip(Xs, solos):
        assert torch.equal(X, ref)


FF_PREP = _gpu.ALL_PREP | fnlh.FNLH_PREP_TAGS | fnlh.FNLH_PREP_FF


def device_rows_ff(probs, prep=FF_PREP):
    dev = []
    for p in probs:
        dm = fnlh.DeviceMesh.from_mesh(p.mesh, "cuda")
        J = fnlh.DeviceJacobian(dm, p.block, prep)
        fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).cuda(), fnlh.make_params(p.cfl), J)
        dev.append((p, dm, J, torch.from_numpy(p.b).cuda()))
    return dev


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16])
def test_batched_float_float_solve_equals_per_row(prec):
    """tol = 0: every check after the first is float-float in both, so the
    batched solve makes the per-row solves' corrections, bit for bit."""
    dev = device_rows_ff(rows_problem())
    inner, checks = 6, 4
    singles = []
    for p, dm, J, B in dev:
        X = torch.zeros_like(B)
        ws = fnlh.solve_workspace(p.mesh.n_nodes, 6, p.n_harm, FF_PREP, "cuda", prec)
        st, c, sw, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 0.0, inner, checks, ws=ws,
                                         raise_on_error=False)
        assert st == fnlh.FNLH_ERR_NOT_CONVERGED and c == checks
        singles.append((X, rel))
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6, prec, ff=True), dtype=torch.uint8, device="cuda")
    assert ws.numel() > batch.workspace_bytes(6, prec)
    st, c, sw, rel = fnlh.fnlh_solve_batched(batch, prec, 0.0, inner, checks, ws=ws, raise_on_error=False)
    assert st == fnlh.FNLH_ERR_NOT_CONVERGED and c == checks and sw == inner * (checks - 1)
    o = 0
    for X, (ref, rel1), (p, *_r) in zip(Xs, singles, dev):
        assert torch.equal(X, ref)
        assert np.array_equal(rel[o:o + 1 + p.n_harm], rel1)
        o += 1 + p.n_harm


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16])
@pytest.mark.parametrize("flags", [0, fnlh.FNLH_SOLVE_MASK_CONVERGED])
def test_batched_float_float_solve_certified_by_oracle(prec, flags):
    probs = rows_problem()
    dev = device_rows_ff(probs)
    Xs = [torch.full_like(B, 3.0) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6, prec, ff=True), dtype=torch.uint8, device="cuda")
    st, c, sw, rel = fnlh.fnlh_solve_batched(batch, prec, 1e-8, 12, 60, ws=ws,
                                             flags=flags | fnlh.FNLH_SOLVE_ZERO_GUESS)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-8), (st, rel)
    o = 0
    for p, X in zip(probs, Xs):
        true_rel = oracle.rel_residuals(_gpu.oracle_jacobian(p), p.mesh.vol, p.omega, p.b, X.cpu().numpy())
        assert np.all(true_rel <= 1e-8), true_rel
        # the reported residuals are the certifying FP64 check's
        assert np.allclose(rel[o:o + 1 + p.n_harm], true_rel, rtol=1e-6, atol=1e-12)
        o += 1 + p.n_harm


def test_batched_float_float_needs_every_row_split():
    """One row without FNLH_PREP_FF: the batch takes every check in FP64, as
    with the plain workspace, whatever the workspace size."""
    probs = rows_problem()
    dev = device_rows_ff(probs[:2]) + device_rows_ff(probs[2:], prep=_gpu.ALL_PREP | fnlh.FNLH_PREP_TAGS)
    out = []
    for ff in (True, False):
        Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
        batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
        ws = torch.empty(batch.workspace_bytes(6, fnlh.FNLH_F32, ff=ff), dtype=torch.uint8, device="cuda")
        st, c, sw, rel = fnlh.fnlh_solve_batched(batch, fnlh.FNLH_F32, 0.0, 6, 3, ws=ws, raise_on_error=False)
        assert st == fnlh.FNLH_ERR_NOT_CONVERGED and c == 3
        out.append((Xs, rel))
    for Xa, Xb in zip(out[0][0], out[1][0]):
        assert torch.equal(Xa, Xb)
    assert np.array_equal(out[0][1], out[1][1])
