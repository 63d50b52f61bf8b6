"""The oracle's pins catch plausible mistakes in the oracle.

Each mutant below plants one mistake in a copy of the oracle's C source: a
flipped sign, a dropped term or factor, a transposed operand, a wrong index
or conjugate, a step of the solvers out of order.  The copy is built in a
temporary directory and the pin suite (tests/test_oracle_pins.py, without its
two slowest tests) runs against it in a subprocess, with that copy imported
as `oracle`.  Every mutant must fail at least one pin; the unmodified copy,
run the same way, must pass them all.  Nothing here touches the product.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")
FAST = "not noise_free and not kkt"

# (name, text in sl1m_oracle.c, replacement); the text occurs exactly once.
MUTANTS = [
    ("dirac_phase_sign", "return cexp(-2.0 * ORC_PI * i * (u * l + v * m + w * nm1)) / n;",
     "return cexp(2.0 * ORC_PI * i * (u * l + v * m + w * nm1)) / n;"),
    ("dirac_drops_1_over_n", "return cexp(-2.0 * ORC_PI * i * (u * l + v * m + w * nm1)) / n;",
     "return cexp(-2.0 * ORC_PI * i * (u * l + v * m + w * nm1));"),
    ("dirac_drops_w_term", "return cexp(-2.0 * ORC_PI * i * (u * l + v * m + w * nm1)) / n;",
     "return cexp(-2.0 * ORC_PI * i * (u * l + v * m)) / n;"),
    ("dirac_transposes_v_l", "return cexp(-2.0 * ORC_PI * i * (u * l + v * m + w * nm1)) / n;",
     "return cexp(-2.0 * ORC_PI * i * (u * l + v * l + w * nm1)) / n;"),
    ("n_minus_one_sign", "double nm1 = -r2 / (1.0 + n);", "double nm1 = r2 / (1.0 + n);"),
    ("gauss_q_sign", "double complex q = 1.0 / (1.0 - i * w * s2);",
     "double complex q = 1.0 / (1.0 + i * w * s2);"),
    ("gauss_drops_q_prefactor", "double complex a = q * cexp(q * c) / n;",
     "double complex a = cexp(q * c) / n;"),
    ("gauss_drops_quadratic_phase", "+ i * ORC_PI * w * r2\n", "\n"),
    ("gauss_width_factor", "- ORC_PI * s2 * (u * u + v * v);", "- 2.0 * ORC_PI * s2 * (u * u + v * v);"),
    ("wide_printed_sign", "a *= cexp(-2.0 * ORC_PI * i * w * (nm1 + 0.5 * r2));",
     "a *= cexp(-2.0 * ORC_PI * i * w * (nm1 - 0.5 * r2));"),
    ("gain_conjugate_on_a", "double complex g = (ga[0] + _Complex_I * ga[1]) * conj(gb[0] + _Complex_I * gb[1]);",
     "double complex g = conj(ga[0] + _Complex_I * ga[1]) * (gb[0] + _Complex_I * gb[1]);"),
    ("gain_second_antenna_index", "int aa = P->ant_pair[2 * k], bb = P->ant_pair[2 * k + 1];\n        const double *ga",
     "int aa = P->ant_pair[2 * k], bb = P->ant_pair[2 * k];\n        const double *ga"),
    ("forward_conjugates_entry", "acc += entry_kj(P, k, j) * x[j];", "acc += conj(entry_kj(P, k, j)) * x[j];"),
    ("adjoint_drops_conjugate", "acc += creal(conj(entry_kj(P, k, j)) * rk);", "acc += creal(entry_kj(P, k, j) * rk);"),
    ("adjoint_takes_imaginary_part", "acc += creal(conj(entry_kj(P, k, j)) * rk);",
     "acc += cimag(conj(entry_kj(P, k, j)) * rk);"),
    ("power_weights_real_part_only", "            work[2 * k + 1] *= P->weights[k];\n", ""),
    ("power_no_normalisation", "for (long j = 0; j < np; ++j) x[j] = z[j] / mu;",
     "for (long j = 0; j < np; ++j) x[j] = z[j];"),
    ("power_rayleigh_start_not_unit", "x[j] = 1.0 / sqrt((double)np);", "x[j] = 1.0;"),
    ("threshold_hard", "return x > d ? x - d : 0.0;", "return x > d ? x : 0.0;"),
    ("fista_gradient_sign", "Ik[j] = thresh_pos(y[j] - g[j] / L, lambda / L);",
     "Ik[j] = thresh_pos(y[j] + g[j] / L, lambda / L);"),
    ("fista_threshold_not_scaled", "Ik[j] = thresh_pos(y[j] - g[j] / L, lambda / L);",
     "Ik[j] = thresh_pos(y[j] - g[j] / L, lambda);"),
    ("fista_momentum_index", "double beta = (t - 1.0) / t_next;", "double beta = (t - 1.0) / t;"),
    ("fista_momentum_sign", "y[j] = Ik[j] + beta * (Ik[j] - Iprev[j]);", "y[j] = Ik[j] - beta * (Ik[j] - Iprev[j]);"),
    ("fista_ignores_weights",
     "        st = orc_forward(P, y, res);\n        if (st) break;\n        for (long q = 0; q < nv; ++q) {\n            double wk = P->weights ? P->weights[q] : 1.0;\n            res[2 * q] = wk * (res[2 * q] - vis[2 * q]);\n            res[2 * q + 1] = wk * (res[2 * q + 1] - vis[2 * q + 1]);\n        }\n        st = orc_adjoint(P, res, g);\n        if (st) break;\n        for (long j = 0; j < np; ++j)\n            Ik[j]",
     "        st = orc_forward(P, y, res);\n        if (st) break;\n        for (long q = 0; q < nv; ++q) {\n            double wk = 1.0;\n            res[2 * q] = wk * (res[2 * q] - vis[2 * q]);\n            res[2 * q + 1] = wk * (res[2 * q + 1] - vis[2 * q + 1]);\n        }\n        st = orc_adjoint(P, res, g);\n        if (st) break;\n        for (long j = 0; j < np; ++j)\n            Ik[j]"),
    ("fista_stop_on_paper_E", "            double E = 0.5 * r2 + lambda * l1;\n            if (fabs(E - E_prev)",
     "            double E = r2 + lambda * l1;\n            if (fabs(E - E_prev)"),
    ("wide_correction_on_paraxial_too", "if (kind == ORC_GAUSS_WIDE) {", "if (kind != ORC_DIRAC) {"),
    ("wide_correction_drops_r2", "a *= cexp(-2.0 * ORC_PI * i * w * (nm1 + 0.5 * r2));",
     "a *= cexp(-2.0 * ORC_PI * i * w * nm1);"),
    ("forward_skips_negative_flux", "if (x[j] == 0.0) continue;", "if (x[j] <= 0.0) continue;"),
    ("resid2_ignores_weights", "s += wk * (dr * dr + di * di);", "s += dr * dr + di * di;"),
    ("fista_ignores_x0", "        memcpy(y, x0, sizeof(double) * np);\n        memcpy(Ik, x0",
     "        memcpy(Ik, x0"),
    ("fista_nnz_counts_zeros", "for (long j = 0; j < np; ++j) { l1 += Ik[j]; nnz += Ik[j] > 0.0; }",
     "for (long j = 0; j < np; ++j) { l1 += Ik[j]; nnz += Ik[j] >= 0.0; }"),
    ("mfista_ignores_x0", "        memcpy(x, x0, sizeof(double) * np);\n        memcpy(y, x0, sizeof(double) * np);",
     "        memcpy(x, x0, sizeof(double) * np);"),
    ("gauss_exponent_without_q", "double complex a = q * cexp(q * c) / n;", "double complex a = q * cexp(c) / n;"),
    ("n_sign_inside_root", "double n = sqrt(1.0 - r2);", "double n = sqrt(1.0 + r2);"),
    ("gain_index_transposed", "const double *ga = P->gains + 2 * ((size_t)j * P->n_ant + aa);",
     "const double *ga = P->gains + 2 * ((size_t)aa * P->n_pix + j);"),
    ("fista_t_update_constant", "double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));\n        double beta",
     "double t_next = 0.5 * (1.0 + sqrt(1.0 + 2.0 * t * t));\n        double beta"),
    ("power_absolute_tolerance", "if (it > 1 && fabs(mu - mu_prev) <= tol * mu) break;",
     "if (it > 1 && fabs(mu - mu_prev) <= tol) break;"),
    ("power_returns_previous_mu", "    *L_out = mu;\n", "    *L_out = mu_prev > 0.0 ? mu_prev : mu;\n"),
    ("fista_stop_before_the_step_is_kept", "            if (fabs(E - E_prev) <= tol * E_prev) { converged = 1; break; }",
     "            if (fabs(E - E_prev) <= tol) { converged = 1; break; }"),
    ("mfista_momentum_uses_t_next_minus_one", "y[j] = xk + (t / t_next) * (z[j] - xk) + ((t - 1.0) / t_next) * (xk - x[j]);",
     "y[j] = xk + ((t - 1.0) / t_next) * (z[j] - xk) + ((t - 1.0) / t_next) * (xk - x[j]);"),
    ("stats_E_paper_halved", "            stats->E_paper = r2 + lambda * l1;\n            stats->t_final = t;\n        }\n    }\n    free(Ik);",
     "            stats->E_paper = 0.5 * r2 + lambda * l1;\n            stats->t_final = t;\n        }\n    }\n    free(Ik);"),
    ("mfista_absolute_stop", "if (tol > 0.0 && fabs(Fz - Fx_prev) <= tol * Fx_prev) { converged = 1; break; }",
     "if (tol > 0.0 && fabs(Fz - Fx_prev) <= tol) { converged = 1; break; }"),
    ("entry_accepts_pixels_off_the_sky", "    if (!(l * l + m * m < 1.0) || !out) return ORC_ERR_ARG;",
     "    if (!out) return ORC_ERR_ARG;"),
    ("mfista_drops_z_term", "y[j] = xk + (t / t_next) * (z[j] - xk) + ((t - 1.0) / t_next) * (xk - x[j]);",
     "y[j] = xk + ((t - 1.0) / t_next) * (xk - x[j]);"),
    ("mfista_always_takes_z", "const int take = Fz <= Fx;", "const int take = 1;"),
    ("mfista_objective_without_half", "    *out = 0.5 * r2 + lambda * l1;", "    *out = r2 + lambda * l1;"),
]


def _copy_oracle(dst, mutant=None):
    pkg = os.path.join(dst, "oracle")
    os.makedirs(pkg)
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), pkg)
    src = open(os.path.join(ROOT, "oracle", "sl1m_oracle.c")).read()
    if mutant is not None:
        _, old, new = mutant
        assert src.count(old) == 1, mutant[0]
        src = src.replace(old, new)
    with open(os.path.join(pkg, "sl1m_oracle.c"), "w") as f:
        f.write(src)
    # build here, so that a mutant that does not compile fails this test and
    # not the pin run
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-fno-fast-math", "-ffp-contract=off", "-pthread", "-fPIC",
                           "-shared", "-o", os.path.join(pkg, "libsl1m_oracle.so"),
                           os.path.join(pkg, "sl1m_oracle.c"), "-lm"])
    return dst


def _run_pins(under_test):
    env = dict(os.environ, SL1M_ORACLE_UNDER_TEST=under_test, PYTHONDONTWRITEBYTECODE="1")
    return subprocess.Popen([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider",
                             "-k", FAST], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                            stderr=subprocess.STDOUT)


def test_every_planted_mistake_fails_a_pin(tmp_path):
    todo = [("unmodified", None)] + [(m[0], m) for m in MUTANTS]
    width = max(2, os.cpu_count() or 2)
    codes, logs = {}, {}
    for i in range(0, len(todo), width):            # at most one pin run per core at a time
        runs = {name: _run_pins(_copy_oracle(str(tmp_path / name), m)) for name, m in todo[i:i + width]}
        for name, p in runs.items():
            out, _ = p.communicate(timeout=600)
            codes[name], logs[name] = p.returncode, out.decode(errors="replace")
    assert codes["unmodified"] == 0, logs["unmodified"][-2000:]
    survivors = [n for n, c in codes.items() if n != "unmodified" and c != 1]
    assert not survivors, {n: (codes[n], logs[n][-400:]) for n in survivors}
