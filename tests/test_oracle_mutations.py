"""Plants plausible mistakes in a copy of the oracle and checks that the pins
in test_oracle_pins.py catch every one (CPU only; the copy is compiled into a
temporary directory and loaded through ACCSINK_ORACLE_LIB)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "acc_sinkhorn_oracle.c")

# (name, original text, planted mistake)
MUTATIONS = [
    ("row_sign", "s += exp(x[j] - orc_cost_entry(c, i, j) / eps - mx);\n        u[i] =",
     "s += exp(x[j] + orc_cost_entry(c, i, j) / eps - mx);\n        u[i] ="),
    ("row_drops_loga", "u[i] = loga[i] - (mx + log(s));", "u[i] = - (mx + log(s));"),
    ("no_centring", "for (long j = 0; j < m; ++j) s[j] -= mean; /* P_Nperp */", ";"),
    ("v_update_sign", "s[j] = p->logb[j] - ell[j];", "s[j] = p->logb[j] + ell[j];"),
    ("alg1_w_coef", "(w[q] + (alpha * alpha - 2.0) * x1[q] + 2.0 * s1[q])",
     "(w[q] + (alpha * alpha - 1.0) * x1[q] + 2.0 * s1[q])"),
    ("alg1_x_denominator", "x1[q] = (w[q] + s[q]) / (1.0 + alpha);",
     "x1[q] = (w[q] + s[q]) / (1.0 + 2.0 * alpha);"),
    ("stage_length", "m_stage = (long)floor(sqrt(2.0) * (double)m_stage) + 1;",
     "m_stage = (long)floor(sqrt(2.0) * (double)m_stage) + 2;"),
    ("mu_schedule", "mu = mu / 2.0;", "mu = mu / 3.0;"),
    ("alpha_rule", "double alpha = sqrt(2.0 * mu);", "double alpha = 2.0 * sqrt(mu);"),
    ("cond1_metric_index", "l1 += p0 * p0 * D1;", "l1 += p0 * p0 * D0;"),
    ("cond2_power", "out[3] = pow(alpha, 1.5) * r2;", "out[3] = pow(alpha, 0.75) * r2;"),
    ("kappa1", "double kappa1 = (4.0 - alpha * alpha - 2.0 * sqrt(alpha)) /",
     "double kappa1 = (4.0 - alpha * alpha - 1.0 * sqrt(alpha)) /"),
    ("kl_sign", "kl += b[j] * (expm1(p0) - p0);", "kl += b[j] * (expm1(p0) + p0);"),
    ("metric_D", "return bj * expm1(z) / z;", "return bj * exp(z) / z;"),
    ("v_k", "double v0 = w_k[j] / alpha - x_k[j];", "double v0 = w_k[j] * alpha - x_k[j];"),
    ("err_uses_a", "err += fabs(c[j] - p->b[j]);", "err += fabs(c[j] - p->a[j]);"),
    ("dual_sign", "return p->eps * (ua + xb - 1.0);", "return p->eps * (ua - xb - 1.0);"),
    ("gate_restart", "for (long q = 0; q < m; ++q) w1[q] = alpha * x1[q];",
     "for (long q = 0; q < m; ++q) w1[q] = x1[q];"),
    ("eval_cost", "cost += cij * pij;", "cost += pij;"),
    ("carry_ratio", "double ratio = sqrt(2.0 * (mu / 2.0)) / alpha;",
     "double ratio = alpha / sqrt(2.0 * (mu / 2.0));"),
    ("sqeuclid", "v += t * t;", "v += fabs(t);"),
    ("cosine", "v = 1.0 - dot;", "v = dot;"),
]


@pytest.mark.parametrize("name,orig,mutant", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, mutant):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation site for {name} not found exactly once"
    cfile = tmp_path / "mutant.c"
    cfile.write_text(src.replace(orig, mutant))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", str(cfile),
                    "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, ACCSINK_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} was not caught by any pin"
