"""GPU: FP32 / BF16 work on nodes with at most two systems -- the mean flow
alone (N = 0) or the mean flow and one harmonic (N = 1).  For so few systems
the library stores the FP32 mean flow without its zero imaginary part and
sweeps with one thread per node, each off-diagonal block loaded once for all
of the node's systems.

What pins it:
* system independence, bit for bit.  The systems of Eq. lhs_lin share J and
  nothing else, and each kernel applies the same operations in the same
  order to every system, so the mean flow and first harmonic of an N = 1 run
  equal the first three columns of an N = 2 run on the same J, B and
  frequencies (one thread per (node, system), every slice complex) -- sweeps
  on plain, periodic and partitioned passages, the mixed solve with FP64 and
  with float-float checks, the FP32 ILU(0) iterations;
* the oracle's FP64 Jacobi (plain, periodic, partitioned), within the
  low-precision bounds the other sweep tests use;
* the oracle's FP64 residual of mixed solves (masked too), at most 1e-8;
* batched rows that include N = 0 and N = 1 rows: equal to per-row sweeps
  bit for bit in every launch shape, and the batched mixed solve certified by
  the oracle.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2404_01407_gb300 import fnlh, inputs
from tests import _gpu

pytestmark = pytest.mark.gpu

PREP = _gpu.ALL_PREP | fnlh.FNLH_PREP_TAGS
FF_PREP = PREP | fnlh.FNLH_PREP_FF
LOW = [fnlh.FNLH_F32, fnlh.FNLH_BF16]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    fnlh.lib()


def oracle_jac(p):
    m = p.mesh
    return oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl, periodic=m.periodic)


def device(p, part=None, prep=PREP):
    dm = fnlh.DeviceMesh.from_mesh(p.mesh, "cuda", part=part)
    J = fnlh.DeviceJacobian(dm, p.block, prep)
    fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).cuda(), fnlh.make_params(p.cfl), J)
    return dm, J, torch.from_numpy(p.b).cuda()


def leading(p, B, n_harm):
    """The mean flow and the first n_harm harmonics of an N >= n_harm problem:
    right-hand side columns, frequencies and phase angles."""
    C = 1 + 2 * n_harm
    sig = None if p.phase is None else p.phase[:n_harm]
    return B[:, :C, :].contiguous(), p.omega[:n_harm], sig


# ragged sizes (several tiles and a tail), b = 5 and 6, plain / periodic / partitioned
CASES = {
    "b6": dict(dims=(13, 6, 5), block=6, periodic=False, parts=None),
    "b5": dict(dims=(7, 5, 3), block=5, periodic=False, parts=None),
    "b6_periodic": dict(dims=(9, 3, 4), block=6, periodic=True, parts=None),
    "b6_partitioned": dict(dims=(13, 6, 5), block=6, periodic=False, parts=(2, 2, 1)),
}


def case(key, n_harm):
    c = CASES[key]
    p = inputs.problem(c["dims"], c["block"], n_harm, 20.0, 1.3, name=key, periodic=c["periodic"])
    part = None if c["parts"] is None else inputs.box_partition(c["dims"], c["parts"])
    return p, part


@pytest.mark.parametrize("prec", LOW)
@pytest.mark.parametrize("key", sorted(CASES))
def test_few_systems_equal_leading_systems_of_more(key, prec):
    p, part = case(key, 2)
    dm, J, B = device(p, part)
    X2 = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X2, 12, prec, sigma=p.phase)
    for n in (1, 0):
        Bn, om, sig = leading(p, B, n)
        Xn = torch.zeros_like(Bn)
        fnlh.fnlh_relax(dm, J, om, Bn, Xn, 12, prec, sigma=sig)
        assert torch.equal(Xn, X2[:, :1 + 2 * n, :]), (key, n)


@pytest.mark.parametrize("prec,bound", [(fnlh.FNLH_F32, 2e-5), (fnlh.FNLH_BF16, 5e-2)])
@pytest.mark.parametrize("key", sorted(CASES))
@pytest.mark.parametrize("n_harm", [0, 1])
def test_few_systems_bounded_by_oracle(key, n_harm, prec, bound):
    p, part = case(key, n_harm)
    dm, J, B = device(p, part)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 30, prec, sigma=p.phase)
    ref = oracle.jacobi(oracle_jac(p), p.mesh.vol, p.omega, p.b, 30, sigma=p.phase, part=part)
    err = _gpu.rel_err_per_system(X.cpu().numpy(), ref, n_harm)
    assert np.all(err <= bound), err


@pytest.mark.parametrize("prec", LOW)
@pytest.mark.parametrize("ff", [False, True])
def test_few_systems_mixed_solve_equals_leading_systems(prec, ff):
    """tol = 0 and a fixed number of checks: the same corrections per system
    (FP64 or float-float checks; the residual writes the real mean flow)."""
    p = inputs.problem((16, 12, 9), 6, 2, 20.0, name="n2")
    prep = FF_PREP if ff else PREP
    dm, J, B = device(p, prep=prep)
    n = p.mesh.n_nodes

    def solve(Bx, om):
        X = torch.zeros_like(Bx)
        nh = len(om)
        ws = (fnlh.solve_workspace(n, 6, nh, prep, "cuda", prec) if ff else fnlh.workspace(n, 6, nh, "cuda", prec))
        st, c, s, rel = fnlh.fnlh_solve(dm, J, om, Bx, X, prec, 0.0, 8, 3, ws=ws,
                                        flags=fnlh.FNLH_SOLVE_ZERO_GUESS, raise_on_error=False)
        assert st == fnlh.FNLH_ERR_NOT_CONVERGED and c == 3 and s == 16
        return X, rel

    X2, rel2 = solve(B, p.omega)
    B1, om1, _ = leading(p, B, 1)
    X1, rel1 = solve(B1, om1)
    assert torch.equal(X1, X2[:, :3, :])
    B0, om0, _ = leading(p, B, 0)
    X0, rel0 = solve(B0, om0)
    assert torch.equal(X0, X2[:, :1, :])


@pytest.mark.parametrize("prec", LOW)
@pytest.mark.parametrize("flags", [0, fnlh.FNLH_SOLVE_MASK_CONVERGED])
@pytest.mark.parametrize("ff", [False, True])
def test_few_systems_solve_certified_by_oracle(prec, flags, ff):
    p = inputs.problem((24, 16, 12), 6, 1, 20.0, name="n1")
    prep = FF_PREP if ff else PREP
    dm, J, B = device(p, prep=prep)
    X = torch.full_like(B, 7.0)
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 1e-8, 12, 60,
                                              flags=flags | fnlh.FNLH_SOLVE_ZERO_GUESS)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-8), (st, rel)
    true_rel = oracle.rel_residuals(oracle_jac(p), p.mesh.vol, p.omega, p.b, X.cpu().numpy())
    assert np.all(true_rel <= 1e-8), true_rel


@pytest.mark.parametrize("ff", [False, True])
def test_few_systems_ilu_f32_equals_leading_systems(ff):
    """FP32 ILU(0): the correction vector of an N = 1 problem keeps the real
    mean flow; fixed iterations give the N = 2 problem's first columns (with
    float-float residuals too: the residual writes the real mean flow)."""
    dims = (13, 6, 5)
    p = inputs.problem(dims, 6, 2, 20.0)
    dm, J, B = device(p, prep=FF_PREP if ff else PREP)
    color = inputs.lattice_colors(dims)
    out = {}
    for nh in (2, 1, 0):
        Bn, om, _ = leading(p, B, nh)
        ilu = fnlh.DeviceIlu(dm, 6, nh, color=color, precision=fnlh.FNLH_F32)
        fnlh.fnlh_ilu_factor(dm, J, om, ilu)
        X = torch.zeros_like(Bn)
        st, its, rel = fnlh.fnlh_solve_ilu(dm, J, ilu, om, Bn, X, 0.0, 4, raise_on_error=False)
        assert st == fnlh.FNLH_ERR_NOT_CONVERGED and its == 4
        out[nh] = X
    assert torch.equal(out[1], out[2][:, :3, :])
    assert torch.equal(out[0], out[2][:, :1, :])


def batch_rows():
    return [inputs.problem((9, 7, 5), 6, 1, 20.0, 1.0, seeds=(1, 2, 3)),
            inputs.problem((12, 8, 6), 6, 4, 20.0, 1.6, seeds=(4, 5, 6)),
            inputs.problem((10, 9, 7), 6, 0, 20.0, 2.3, seeds=(7, 8, 9))]


@pytest.mark.parametrize("prec", LOW)
def test_batched_rows_with_few_systems_match_per_row(prec):
    dev = [(p, *device(p)) for p in batch_rows()]
    singles = []
    for p, dm, J, B in dev:
        X = torch.zeros_like(B)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, 11, prec)
        singles.append(X)
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6, prec), dtype=torch.uint8, device="cuda")
    for tn in (None, fnlh.fnlh_tuning(128, 2), fnlh.fnlh_tuning(256, 0),
               fnlh.fnlh_tuning(0, fnlh.FNLH_TUNING_PER_ROW)):
        for X in Xs:
            X.zero_()
        fnlh.fnlh_relax_batched(batch, 11, prec, tuning=tn, ws=ws)
        for X, ref in zip(Xs, singles):
            assert torch.equal(X, ref), tn


@pytest.mark.parametrize("prec", LOW)
@pytest.mark.parametrize("flags", [0, fnlh.FNLH_SOLVE_MASK_CONVERGED])
@pytest.mark.parametrize("ff", [False, True])
def test_batched_solve_with_few_systems_certified_by_oracle(prec, flags, ff):
    """With ff the rows' float-float shadows are in the workspace: the rows
    of K <= 2 systems, swept by their own launches, advance theirs too."""
    probs = batch_rows()
    dev = [(p, *device(p, prep=FF_PREP if ff else PREP)) for p in probs]
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6, prec, ff=ff), dtype=torch.uint8, device="cuda")
    st, c, sw, rel = fnlh.fnlh_solve_batched(batch, prec, 1e-8, 12, 60, ws=ws, flags=flags)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-8), (st, rel)
    for p, X in zip(probs, Xs):
        true_rel = oracle.rel_residuals(oracle_jac(p), p.mesh.vol, p.omega, p.b, X.cpu().numpy())
        assert np.all(true_rel <= 1e-8), true_rel
