"""The pins catch plausible oracle mistakes.

Each case copies the oracle's C source, plants one mistake (a dropped term, a
wrong index or operand, an off-by-one, a strict instead of inclusive test, a
missing reset), compiles it into a temporary library and runs the pin suite
against it: at least one pin must fail.  Everything happens on the CPU.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle_gd as gdpins
import test_oracle_gppr as gpins
import test_oracle_localch as chpins
import test_oracle_series as spins
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "localgd.c")

MUTANTS = {
    "ppr_x_drops_alpha": ("x[u] = x[u] + alpha * rho[i];", "x[u] = x[u] + rho[i];"),
    "ppr_share_not_divided_by_degree": ("double w = (one_minus_alpha * rho[i]) / (double)d;",
                                        "double w = (one_minus_alpha * rho[i]);"),
    "ppr_share_uses_alpha": ("const double one_minus_alpha = 1.0 - alpha;",
                             "const double one_minus_alpha = alpha;"),
    "strict_threshold": ("fabs(r[u]) >= thr) active", "fabs(r[u]) > thr) active"),
    "threshold_without_degree": ("double thr = eps_theta * (double)deg_of(off, u);",
                                 "double thr = eps_theta;"),
    "active_not_zeroed": ("        r[u] = 0.0;\n        vol +=", "        vol +="),
    "katz_share_divided_by_degree": ("double w = beta * rho[i];",
                                     "double w = beta * rho[i] / (double)(deg_of(off, u) + 1);"),
    "hk_coef_off_by_one": ("const double coef = tau / (double)(t + 1);",
                           "const double coef = tau / (double)(t + 2);"),
    "hk_theta_without_psi": ("exp(tau) / ((double)(N + 1) * oracle_hk_psi(tau, N, t))",
                             "exp(tau) / ((double)(N + 1))"),
    "hk_terms_one_short": ("if (tail <= tol) best = N; else break;",
                           "if (tail <= tol) best = N - 1; else break;"),
    "hk_psi_wrong_factorial": ("term = term * (tau / (double)(k + j));",
                               "term = term * (tau / (double)(j));"),
    "gppr_target_exponent_sign": ("double dv = pow((double)deg_of(off, v), beta);",
                                  "double dv = pow((double)deg_of(off, v), -beta);"),
    "gppr_source_exponent": ("double du = pow((double)d, 1.0 - beta);",
                             "double du = pow((double)d, beta);"),
    "gppr_threshold_exponent": ("double thr_u = eps * pow((double)deg_of(off, u), 1.0 - beta);",
                                "double thr_u = eps * pow((double)deg_of(off, u), beta);"),
    "gppr_x_drops_alpha": ("x[u] += alpha * rho[i];", "x[u] += rho[i];"),
    "series_ratio_off_by_one": ("double ratio = t < N ? c[t + 1] / c[t] : 0.0;",
                                "double ratio = t + 1 < N ? c[t + 2] / c[t + 1] : 0.0;"),
    "series_theta_without_psi": ("return 1.0 / ((double)(N + 1) * c[0] * oracle_series_psi(c, N, t));",
                                 "return 1.0 / ((double)(N + 1) * c[0]);"),
    "series_result_unscaled": ("for (int64_t u = 0; u < n; u++) x[u] = c[0] * x[u];", ""),
    "gd_stop_without_degree": ("double q = fabs(r[u]) / (double)(d > 0 ? d : 1);", "double q = fabs(r[u]);"),
    "gd_stop_inclusive": ("if (worst < eps) break;", "if (worst <= eps * 1.5) break;"),
    "localch_delta_recursion_sign": ("dnext = 1.0 / (2.0 / c - delta);", "dnext = 1.0 / (2.0 / c + delta);"),
    "localch_residual_not_rescaled": ("r[u] = rho[i] - xh[i] / alpha;", "r[u] = rho[i] - xh[i];"),
    "localch_share_drops_keep": ("double w = (c * (xh[i] / alpha)) / (double)d;", "double w = (xh[i] / alpha) / (double)d;"),
}

PIN_CASES = [
    (pins.test_ppr_edge2_rounds, dict(alpha=0.15)),
    (pins.test_ppr_star_rounds_from_center, dict(k=3)),
    (pins.test_katz_star_closed_form, dict(k=4, beta=0.3)),
    (pins.test_hk_star_closed_form, dict(k=5, tau=3.0)),
    (pins.test_ppr_error_bound_dense, dict(gi=4, alpha=0.15, eps=1e-4)),
    (pins.test_hk_dense, dict(gi=4, tau=5.0)),
    (pins.test_ppr_round_invariants, dict(gi=4)),
    (pins.test_threshold_is_inclusive, {}),
    (pins.test_hk_terms_against_poisson_tail, {}),
    (pins.test_hk_psi_definition, {}),
    (pins.test_hk_weighted_mass_and_layer_invariant, {}),
    (gpins.test_star_by_hand, {}),
    (gpins.test_error_bound_against_dense, dict(gi=0, beta=0.5)),
    (gpins.test_round_invariant, dict(beta=0.25)),
    (spins.test_ipr_bound_against_dense, dict(gi=0, theta=1.3)),
    (spins.test_heat_kernel_coefficients_give_the_heat_kernel, {}),
    (gdpins.test_iteration_count_closed_form, dict(k=8, alpha=0.2, eps=3e-5)),
    (chpins.test_invariant_and_bound, dict(gi=0, eps=1e-5)),
    (chpins.test_fewer_rounds_than_localgd, dict(gi=2)),
]


def build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-std=c11", "-o", str(so), str(path), "-lm"])
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, monkeypatch, name):
    so = build_mutant(tmp_path, name)
    good = oracle._load()
    bad = ctypes.CDLL(so)
    # same signatures as the real library
    for sym in ("oracle_ppr_round", "oracle_katz_round", "oracle_hk_round", "oracle_hk_terms",
                "oracle_hk_psi", "oracle_hk_theta", "oracle_localgd_solve",
                "oracle_localgd_solve_many", "oracle_push_fifo", "oracle_gppr_round", "oracle_gppr_solve",
                "oracle_series_round", "oracle_series_psi", "oracle_series_theta", "oracle_series_solve",
                "oracle_gd_solve", "oracle_localch_solve"):
        f, g = getattr(bad, sym), getattr(good, sym)
        f.argtypes, f.restype = g.argtypes, g.restype
    monkeypatch.setattr(oracle, "_lib", bad)
    caught = []
    for fn, kw in PIN_CASES:
        try:
            fn(**kw)
        except AssertionError:
            caught.append(fn.__name__)
    assert caught, f"no pin caught mutant {name}"
