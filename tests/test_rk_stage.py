"""RK(5,3) stage loop: coefficients against the paper's table (CPU) and the
masked inexact stage solves (GPU)."""

import os

import numpy as np
import pytest

from paper_2404_01407_gb300 import rk_stage

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rk53_coefficients.txt")


def test_coefficients_match_the_paper_table():
    alpha, beta, extra = rk_stage.read_golden(GOLDEN)
    assert alpha == rk_stage.RK53_ALPHA and beta == rk_stage.RK53_BETA
    assert extra["tol"] == rk_stage.LINEAR_TOL and extra["max_iterations"] == rk_stage.LINEAR_MAX_ITERATIONS
    assert extra["eps"] == rk_stage.EPS
    assert rk_stage.RK53_ALPHA[-1] == 1  # the last stage takes the full step


@pytest.mark.gpu
def test_masked_solve_freezes_converged_systems():
    import torch

    import oracle
    from paper_2404_01407_gb300 import fnlh, inputs
    from tests import _gpu

    p = inputs.problem((20, 12, 10), 6, 6, 20.0, 1.5)
    dm, J, B = _gpu.device_problem(p)
    oj = _gpu.oracle_jacobian(p)
    for prec in (fnlh.FNLH_F64, fnlh.FNLH_F32):
        Xa, Xb = torch.empty_like(B), torch.empty_like(B)
        zg = fnlh.FNLH_SOLVE_ZERO_GUESS
        sa = fnlh.fnlh_solve(dm, J, p.omega, B, Xa, prec, 1e-6, 3, 60, flags=zg)
        sb = fnlh.fnlh_solve(dm, J, p.omega, B, Xb, prec, 1e-6, 3, 60, flags=zg | fnlh.FNLH_SOLVE_MASK_CONVERGED)
        assert sa[0] == sb[0] == fnlh.FNLH_OK and sa[2] == sb[2]
        xa, xb = Xa.cpu().numpy(), Xb.cpu().numpy()
        rel = oracle.rel_residuals(oj, p.mesh.vol, p.omega, p.b, xb)
        cols = [[0]] + [[2 * k - 1, 2 * k] for k in range(1, p.n_harm + 1)]
        frozen = 0
        for k, c in enumerate(cols):
            if np.array_equal(xa[:, c], xb[:, c]):
                continue  # never frozen: the independent systems give identical bits
            frozen += 1
            assert rel[k] <= 1.0001e-6  # frozen once it met the tolerance
        assert frozen >= 1  # the high harmonics converge first


@pytest.mark.gpu
def test_rk_stage_loop_follows_the_linear_solve_rule():
    import torch

    from paper_2404_01407_gb300 import fnlh, inputs
    from tests import _gpu

    p = inputs.problem((24, 16, 12), 6, 4, 20.0)
    dm, J, B = _gpu.device_problem(p)
    rng = np.random.default_rng(7)
    R = [torch.from_numpy(-p.b * (1.0 - 0.1 * k) + 0.05 * rng.normal(size=p.b.shape)).cuda() for k in range(5)]
    for prec in (fnlh.FNLH_F64, fnlh.FNLH_F32):
        ups, recs = rk_stage.run_stages(dm, J, p.omega, R, precision=prec)
        assert len(ups) == 5
        for rec in recs:
            assert rec["sweeps"] <= rk_stage.LINEAR_MAX_ITERATIONS
            assert rec["status"] == "success" or rec["sweeps"] == rk_stage.LINEAR_MAX_ITERATIONS
            assert max(rec["rel_residual"]) < 0.05
        # the update scales with Gamma alpha_k: stage 5 (alpha = 1) vs a direct solve of the same RHS
        X5 = torch.empty_like(B)
        st = rk_stage.stage_solve(dm, J, p.omega, R[4] * (-1.0 / rk_stage.EPS), X5, prec)
        assert np.allclose(X5.cpu().numpy(), ups[4].cpu().numpy())
