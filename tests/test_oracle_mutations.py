"""The oracle pins catch plausible mistakes (CPU only).

Each case plants one mistake into a temporary copy of the oracle's C source
(a dropped term, a flipped sign, a transposed block, a wrong index, a wrong
state), builds it, swaps it in, and runs the pins of test_oracle_pins.py:
at least one pin must fail.  The real oracle is restored afterwards.
"""

import inspect
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "fnlh_oracle.c")

MUTATIONS = {
    "offd_sign_in_sweep": ("S[c * b + r] -= acc;", "S[c * b + r] += acc;"),
    "transposed_block_in_sweep": ("acc += Jij[r * b + t] * xs[t];",
                                  "acc += Jij[t * b + r] * xs[t];"),
    "omega_sign_in_sweep": ("cplx shift = D[i] + I * omega[k - 1] * vol[i];",
                            "cplx shift = D[i] - I * omega[k - 1] * vol[i];"),
    "re_im_swapped_in_sweep": ("yc[r] = S[(2 * k - 1) * b + r] + I * S[(2 * k) * b + r];",
                               "yc[r] = S[(2 * k) * b + r] + I * S[(2 * k - 1) * b + r];"),
    "mean_without_D": ("for (int r = 0; r < b; r++) M[r * b + r] += D[i];", ""),
    "offd_from_own_state": ("Oij[t] = 0.5 * (Aj[t] - Ab[t]);", "Oij[t] = 0.5 * (Ai[t] - Ab[t]);"),
    "offd_dissipation_sign": ("Oij[t] = 0.5 * (Aj[t] - Ab[t]);", "Oij[t] = 0.5 * (Aj[t] + Ab[t]);"),
    "no_average_state": ("qbar[m] = 0.5 * (qi[m] + qj[m]);", "qbar[m] = qi[m];"),
    "dropped_closure_face": ("for (int t = 0; t < bb; t++) Pi[t] += 0.5 * (Ai[t] + Ab[t]);\n        lsum",
                             "lsum"),
    "no_entropy_fix": ("f[k] = fabs(lam[k]) > fix ? fabs(lam[k]) : fix;", "f[k] = fabs(lam[k]);"),
    "energy_flux_without_p": ("f[4] = (q[4] + p) * un;", "f[4] = q[4] * un;"),
    "D_times_cfl": ("D[i] = lsum / cfl;", "D[i] = lsum * cfl;"),
    "no_turbulence_doubling": ("if (b == 6) Pi[5 * b + 5] *= 2.0;", ""),
    "residual_omega_sign": ("R[(2 * k) * b + rr] -= wv * Xi[(2 * k - 1) * b + rr];",
                            "R[(2 * k) * b + rr] += wv * Xi[(2 * k - 1) * b + rr];"),
    "residual_without_D": ("acc += D[i] * Xi[c * b + rr];", ""),
    "residual_transposed_diag": ("acc += Pi[rr * b + t] * Xi[c * b + t];",
                                 "acc += Pi[t * b + rr] * Xi[c * b + t];"),
    "phase_sign_flipped": ("const double ang = s * sigma[l - 1];", "const double ang = -s * sigma[l - 1];"),
    "phase_rotation_re_sign": ("xs[t] = (c % 2 == 1) ? cs * re - sn * im : sn * re + cs * im;",
                               "xs[t] = (c % 2 == 1) ? cs * re + sn * im : sn * re + cs * im;"),
    "phase_side_ignores_direction": ("side[p] = (int8_t)(nb[p].sgn * periodic[nb[p].e]);",
                                     "side[p] = (int8_t)(periodic[nb[p].e]);"),
    "phase_im_part_unrotated": (": sn * re + cs * im;", ": im;"),
    "partition_cut_ignored": ("if (part && part[col_idx[p]] != part[i]) continue;", ""),
    "partition_cut_inverted": ("if (part && part[col_idx[p]] != part[i]) continue;",
                               "if (part && part[col_idx[p]] == part[i]) continue;"),
    "ilu_multiplier_order": ("mul_cplx(b, Wo + (size_t)pik * bb, Uinv, L);", "mul_cplx(b, Uinv, Wo + (size_t)pik * bb, L);"),
    "ilu_update_sign": ("for (int t = 0; t < bb; t++) target[t] -= upd[t];",
                        "for (int t = 0; t < bb; t++) target[t] += upd[t];"),
    "ilu_update_from_lower_row_part": ("if (rank[j] <= rank[k] || (part && part[j] != part[k])) continue;",
                                       "if (part && part[j] != part[k]) continue;"),
    "ilu_forward_uses_upper": ("if (rank[k] >= rank[i] || (part && part[k] != part[i])) continue;",
                               "if (rank[k] <= rank[i] || (part && part[k] != part[i])) continue;"),
    "sylvester_wrong_index": ("double am = A[t * b + c] - ((t == c) ? lam[m] : 0.0);",
                              "double am = A[c * b + t] - ((t == c) ? lam[m] : 0.0);"),
}


def _pin_functions():
    out = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        marks = getattr(fn, "pytestmark", [])
        params = [m for m in marks if m.name == "parametrize"]
        if params:
            argname = params[0].args[0]
            for v in params[0].args[1]:
                out.append((f"{name}[{v}]", lambda fn=fn, a=argname, v=v: fn(**{a: v})))
        else:
            out.append((name, fn))
    return out


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(mutation, tmp_path):
    old, new = MUTATIONS[mutation]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor missing from the oracle source"
    mutated = src.replace(old, new, 1)
    csrc = tmp_path / "mut.c"
    csrc.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), str(csrc), "-lm"], check=True)
    prev = oracle.use_library(str(so))
    failed = []
    try:
        for name, fn in _pin_functions():
            try:
                fn()
            except Exception:  # AssertionError, or a singular / failed build
                failed.append(name)
                break
    finally:
        oracle.restore_library(prev)
    assert failed, f"no pin caught the planted mistake '{mutation}'"
