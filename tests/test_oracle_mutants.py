"""Planted mistakes: each mutant is a copy of oracle/oracle.c with one plausible
error (a dropped term, a wrong sign or index, a transposed operand, ...). It is
built on the CPU and the oracle pins are run against it; every mutant must fail
at least one pin. This shows the pins constrain each part of the oracle.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PINS = ["tests/test_oracle_bessel.py", "tests/test_oracle_propagation.py", "tests/test_oracle_haydock.py",
        "tests/test_oracle_qe.py", "tests/test_oracle_ac.py",
        "tests/test_oracle_kpm.py", "tests/test_oracle_dos.py"]

# name: [(original text, planted text)], each original must occur in oracle.c
MUTANTS = {
    "coeff_sign": [("case 1: mi_k = -I; break;", "case 1: mi_k = I; break;"),
                   ("default: mi_k = I; break;", "default: mi_k = -I; break;")],
    "coeff_factor_two": [("c[k] = (k == 0 ? 1.0 : 2.0) * mi_k * j;", "c[k] = mi_k * j;")],
    "bessel_series_sign": [("term *= -(h * h)", "term *= (h * h)")],
    "dropped_last_term": [("for (int k = 2; k < K; ++k) {", "for (int k = 2; k < K - 1; ++k) {")],
    "transposed_operand": [("acc += val[p] * x[col[p]];", "acc += conj(val[p]) * x[col[p]];")],
    "first_order_scale": [("spmv(n, rp, col, val, 1.0 / rescale, t0, t1);\n#pragma",
                           "spmv(n, rp, col, val, 2.0 / rescale, t0, t1);\n#pragma")],
    "kpm_first_order_scale": [("spmv(n, rp, col, val, 1.0 / rescale, t0, t1);\n        mu[1]",
                               "spmv(n, rp, col, val, 2.0 / rescale, t0, t1);\n        mu[1]")],
    "recurrence_sign": [("t2[i] -= t0[i];\n            out[i]", "t2[i] += t0[i];\n            out[i]")],
    "dot_without_conj": [("acc += conj(a[i]) * b[i];", "acc += a[i] * b[i];")],
    "corr_stale_state": [("if (corr) corr[s + 1] = dot(n, psi0, psi);",
                          "if (corr) corr[s + 1] = dot(n, psi0, out);")],
    "kpm_index": [("mu[m] = dot(n, psi0, t2);", "mu[m] = dot(n, psi0, t1);")],
    "kpm_recurrence_sign": [("t2[i] -= t0[i];\n        mu[m]", "t2[i] += t0[i];\n        mu[m]")],
    "hann_window_sign": [("double w = 0.5 * (1.0 + cos(PI * (double)m", "double w = 0.5 * (1.0 - cos(PI * (double)m")],
    "hann_no_conj": [("cplx cm = m < 0 ? conj(corr[a]) : corr[a];", "cplx cm = corr[a];")],
    "hann_norm": [("acc *= dt / (2.0 * PI);", "acc *= dt / PI;")],
    "hann_phase_sign": [("acc += w * cm * cexp(I * e * t);", "acc += w * cm * cexp(-I * e * t);")],
    "jackson_sin_sign": [("+ sin(q * m) / tan(q)", "- sin(q * m) / tan(q)")],
    "kpm_dos_factor_two": [("s += 2.0 * g[m] * mu_re[m]", "s += g[m] * mu_re[m]")],
    "kpm_dos_rescale": [("rho[j] = s / (PI * sqrt(1.0 - x * x)) / rescale;",
                         "rho[j] = s / (PI * sqrt(1.0 - x * x));")],
    "haydock_tail_not_squared": [("b[m] * b[m] * g;", "b[m] * g;")],
    "haydock_no_previous_term": [("w[i] -= bn * vp[i];", "w[i] -= 0.0 * vp[i];")],
    "haydock_eta_sign": [("cplx z = energies[j] + I * eta;", "cplx z = energies[j] - I * eta;")],
    "haydock_stale_vector": [("vp[i] = v[i]; v[i] = w[i] / bm;", "vp[i] = v[i]; v[i] = w[i];")],
    "qe_phase_sign": [("cplx ph = pre * w * cexp(I * energies[e] * t);",
                       "cplx ph = pre * w * cexp(-I * energies[e] * t);")],
    "qe_forward_only": [("for (int dir = 0; dir < 2; ++dir) {", "for (int dir = 0; dir < 1; ++dir) {")],
    "qe_no_window": [("double w = 0.5 * (1.0 + cos(PI * (double)s / (double)N));", "double w = 1.0;")],
    "fermi_exp_sign": [("double q = exp(-z);", "double q = exp(z);")],
    "fermi_a0_doubled": [("a[k] = (k == 0 ? 1.0 : 2.0) * s / M;", "a[k] = 2.0 * s / M;")],
    "fermi_node_offset": [("fj[j] = fermi(beta, mu, rescale * cos(PI * (j + 0.5) / M));",
                           "fj[j] = fermi(beta, mu, rescale * cos(PI * j / M));")],
    "ac_f_instead_of_one_minus_f": [("v[1 + b][i] = u[i] - out[i];", "v[1 + b][i] = out[i];")],
    "ac_current_swapped": [("spmv(n, jrp, jcol, al == 0 ? jx : jy, 1.0, v[0], u);",
                            "spmv(n, jrp, jcol, al == 0 ? jy : jx, 1.0, v[0], u);")],
    "ac_cond_sign": [("sigma[j] = (exp(-beta * w) - 1.0) / (w * s) * acc;",
                      "sigma[j] = (1.0 - exp(-beta * w)) / (w * s) * acc;")],
    "ac_cond_real_part": [("sin(w * m * dt) * 2.0 * cimag(corr[m]);", "sin(w * m * dt) * 2.0 * creal(corr[m]);")],
    "ac_cond_no_window": [("double win = 0.5 * (1.0 + cos(PI * (double)m / (double)N));", "double win = 1.0;")],
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    src = open(SRC).read()
    for old, new in MUTANTS[name]:
        assert src.count(old) == 1, f"mutation site for {name} not found once in oracle.c"
        src = src.replace(old, new)
    with tempfile.TemporaryDirectory() as tmp:
        c = os.path.join(tmp, "mutant.c")
        so = os.path.join(tmp, "libmutant.so")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", c, "-o", so, "-lm"])
        env = dict(os.environ, TBPM_ORACLE_LIB=so, OMP_NUM_THREADS="2")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 1, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
