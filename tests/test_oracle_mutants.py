"""Plant plausible mistakes in copies of the oracle and check that the pins
catch every one.

Each mutant is a textual edit of oracle/bfm_oracle.c (a dropped term, a wrong
sign or index, a transposed operand, a wrong constant), compiled into a
temporary library that the oracle module is pointed at; the pins of
test_oracle_pins.py must then fail.  The shipped oracle source is untouched.
"""
import os
import subprocess

import pytest

import oracle
from test_oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "bfm_oracle.c")

# (name, text in the oracle, replacement, which occurrence (0-based) or None for all)
MUTANTS = [
    ("ct_drop_half", "double v = 0.5 * d * d + f[j];", "double v = d * d + f[j];", 0),
    ("ct_sign_of_phi", "cur[i] = -phi[i];", "cur[i] = phi[i];", 0),
    ("ct_cell_centre_shift", "double y = (j + 0.5) * h;\n            double d = x - y;",
     "double y = (j + 1.5) * h;\n            double d = x - y;", 0),
    ("llt_sweep_direction", "if (slope < x) k++; else break;", "if (slope > x) k++; else break;", 0),
    ("llt_hull_test", "if (cross <= 0.0) H--; else break;", "if (cross >= 0.0) H--; else break;", 0),
    ("full_ct_drop_half", "c += 0.5 * d * d;", "c += d * d;", 0),
    ("line_base_axis", "base += c * g->stride[b];", "base += c * g->stride[a];", 0),
    ("dct2_centre", "s += x[j] * cos(M_PI * k * (j + 0.5) / n);", "s += x[j] * cos(M_PI * k * j / n);", 0),
    ("dct3_weight", "s += 2.0 * X[k] * cos", "s += X[k] * cos", 0),
    ("dct2_fft_twiddle_sign", "double ang = -M_PI * k / (2.0 * n);", "double ang = M_PI * k / (2.0 * n);", 0),
    ("fft_reorder", "buf[n - 1 - q] = x[2 * q + 1];", "buf[n - 1 - q] = x[2 * q];", 0),
    ("eig_factor", "lam += 4.0 * g.n[a] * (double)g.n[a] * s * s;", "lam += 2.0 * g.n[a] * (double)g.n[a] * s * s;", 0),
    ("eig_angle", "double s = sin(M_PI * k / (2.0 * g.n[a]));", "double s = sin(M_PI * k / g.n[a]);", 0),
    ("map_sign", "double t = x - disp;", "double t = x + disp;", 0),
    ("central_difference", "grad = (psi[p + s] - psi[p - s]) / (2.0 * h);", "grad = (psi[p + s] - psi[p - s]) / h;", 0),
    ("onesided_difference", "grad = (psi[p + s] - psi[p]) / h;", "grad = (psi[p + s] - psi[p]) / (2.0 * h);", 0),
    ("bilinear_swap", "w *= up ? w1[a] : (1.0 - w1[a]);", "w *= up ? (1.0 - w1[a]) : w1[a];", 0),
    ("deposit_floor", "int i = (int)floor(pos);", "int i = (int)floor(pos + 0.5);", 0),
    ("step_rule_inverted", "if (gain < o->beta1 * sigma * G) {", "if (gain > o->beta1 * sigma * G) {", 0),
    ("step_rule_alpha_swapped_decrease", "double s = o->alpha2 * sigma;", "double s = o->alpha1 * sigma;", 0),
    ("step_rule_alpha_swapped_increase", "return o->alpha1 * sigma;", "return o->alpha2 * sigma;", 0),
    ("step_rule_window_collapsed", "if (gain > o->beta2 * sigma * G)", "if (gain > o->beta1 * sigma * G)", 0),
    ("step_rule_beta2_doubled", "if (gain > o->beta2 * sigma * G)", "if (gain > 2.0 * o->beta2 * sigma * G)", 0),
    ("step_rule_floor_dropped", "return (s > floor_) ? s : floor_;", "return s;", 0),
    ("step_rule_no_growth", "if (gain > o->beta2 * sigma * G) return o->alpha1 * sigma;", "", 0),
    ("residual_uniform_fallback_dropped", "double r = (Gref > 0) ? sqrt(fmax(G, 0.0) / Gref) : sqrt(fmax(G, 0.0));",
     "double r = sqrt(fmax(G, 0.0) / Gref);", None),
    ("sigma0_constant", "8.0 * fmin(1.0 / mx_mu, 1.0 / mx_nu)", "4.0 * fmin(1.0 / mx_mu, 1.0 / mx_nu)", 0),
    ("w2_factor", "info_out[2] = 2.0 * Jold;", "info_out[2] = Jold;", 0),
    ("psi_half_measure", "bfm_oracle_pushforward_p(tmp, nu, rho, ndim, n, pc);",
     "bfm_oracle_pushforward_p(tmp, mu, rho, ndim, n, pc);", 0),
    ("power_cost_exponent", "return pow(fabs(z), p) / p;", "return pow(fabs(z), p) / 2.0;", 0),
    ("power_map_inverse_gradient", "pow(fabs(grad), 1.0 / (pw[a] - 1.0))", "pow(fabs(grad), pw[a] - 1.0)", 0),
    ("psi_half_residual", "f[i] = mu[i] - rho[i];", "f[i] = nu[i] - rho[i];", 0),
    ("update_sign", "phi[i] += sigma * gr[i];", "phi[i] -= sigma * gr[i];", 0),
    ("dual_uses_wrong_density", "Jold = dot_hd(&g, phi, nu) + dot_hd(&g, tmp, mu);",
     "Jold = dot_hd(&g, phi, mu) + dot_hd(&g, tmp, nu);", 0),
    ("mass_missing_hd", "mass_mu *= g.hd; mass_nu *= g.hd;", "mass_nu *= g.hd;", 0),
    ("interp_swapped", "double s = t * map[a * g.N + p] + (1.0 - t) * x;",
     "double s = (1.0 - t) * map[a * g.N + p] + t * x;", 0),
]


def _replace_nth(text, old, new, k):
    if k is None:
        return text.replace(old, new)
    pos = -1
    for _ in range(k + 1):
        pos = text.index(old, pos + 1)
    return text[:pos] + new + text[pos + len(old):]


@pytest.mark.parametrize("name,old,new,k", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new, k):
    src = open(SRC).read()
    assert old in src, f"mutation site for {name} no longer in the oracle"
    mutated = _replace_nth(src, old, new, k)
    c = tmp_path / "mutant.c"
    c.write_text(mutated)
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), str(c), "-lm"], check=True)
    oracle.use_library(str(so))
    caught = []
    try:
        for pin in ALL_PINS:
            try:
                pin()
            except (AssertionError, ValueError, FloatingPointError, IndexError):
                caught.append(pin.__name__)
                break
    finally:
        oracle.use_library(None)
    assert caught, f"no pin caught the planted mistake {name}"
