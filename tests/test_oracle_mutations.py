"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/hh_oracle.c`` (a wrong
order, a dropped term, a flipped sign, a transposed use), compiles it on the
CPU, and runs the pin suite ``test_oracle.py`` against it in a subprocess; the
suite has to fail.  The unmodified source has to pass.
"""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hh_oracle.c")

MUTATIONS = {
    "chain_order_reversed": (
        "for (int64_t k = h - 1; k >= 0; --k) reflect(n, U + k * ldu, tau[k], z);",
        "for (int64_t k = 0; k < h; ++k) reflect(n, U + k * ldu, tau[k], z);"),
    "tau_missing_factor_2": ("tau[k] = (nn > 0.0) ? 2.0 / nn : 0.0;",
                             "tau[k] = (nn > 0.0) ? 1.0 / nn : 0.0;"),
    "reflect_wrong_sign": ("for (int64_t j = 0; j < n; ++j) z[j] -= c * v[j];",
                           "for (int64_t j = 0; j < n; ++j) z[j] += c * v[j];"),
    "sign_dropped_in_WT": ("""            } else if (mode == ORACLE_WT) {
                apply_sign(n, sigma, z);""", """            } else if (mode == ORACLE_WT) {"""),
    "sym_spectrum_dropped": ("for (int64_t j = 0; j < n; ++j) z[j] *= d[j];",
                             "for (int64_t j = 0; j < n; ++j) z[j] *= 1.0;"),
    "grad_tau2_term_dropped": ("double cv = tau * tau * va * vg;", "double cv = 0.0;"),
    "grad_swapped_operands": ("gv[j] += cv * v[j] - tau * va * G[j] - tau * vg * a[j];",
                              "gv[j] += cv * v[j] - tau * vg * G[j] - tau * va * a[j];"),
    "grad_state_off_by_one": (
        "reflect_backward(n, U + k * ldu, tau[k], sa + (k + 1) * n, G, gu_t + k * n);",
        "reflect_backward(n, U + k * ldu, tau[k], sa + k * n, G, gu_t + k * n);"),
    "grad_d_after_scaling": ("""                        gd_t[j] += sb[h * n + j] * G[j];
                        G[j] *= d[j];""", """                        G[j] *= d[j];
                        gd_t[j] += sb[h * n + j] * G[j];"""),
    "mahalanobis_unweighted": ("for (int64_t j = 0; j < n; ++j) s += d[j] * z[j] * z[j];",
                               "for (int64_t j = 0; j < n; ++j) s += z[j] * z[j];"),
    "mahalanobis_uses_W": ("""            apply_sign(n, sigma, z);
            chain_WT(n, h, U, ldu, tau, z);
            double s = 0.0;""", """            apply_sign(n, sigma, z);
            chain_W(n, h, U, ldu, tau, z);
            double s = 0.0;"""),
}


def _build(tmp_path, name, text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", str(so),
                    str(c), "-lm"], check=True)
    return str(so)


def _run_pins(lib):
    env = dict(os.environ, HH_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    return r.returncode


def test_unmodified_oracle_passes(tmp_path):
    src = open(SRC).read()
    assert _run_pins(_build(tmp_path, "orig", src)) == 0


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mutant = src.replace(old, new, 1)
    assert _run_pins(_build(tmp_path, name, mutant)) != 0, f"pins did not catch {name}"
