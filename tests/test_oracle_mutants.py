"""Planted mistakes in the oracle: each case compiles a copy of svdup_oracle.c with
one plausible slip (a dropped term, a wrong sign or index, a transposed operand) and
runs the pins of test_oracle_pins.py against it in a child process.  Every planted
copy must fail at least one pin, and the unaltered copy, compiled the same way, must
pass them all.  CPU only; the mistakes live in temporary copies, never in the oracle.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "svdup_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, passage the altered code follows, text in the oracle, planted text)
MUTANTS = [
    ("schur2_root_sign", "Alg. 6.1 STEP 2: r1 r2 = -1",
     "r1 = 0.5 * (g + s); r2 = -1.0 / r1;", "r1 = 0.5 * (g + s); r2 = 1.0 / r1;"),
    ("schur2_unnormalised", "Alg. 6.1 STEP 2: Q orthogonal",
     "out[3] = 1.0 / n1;", "out[3] = 1.0;"),
    ("gemv_index", "RankOneUpdate STEP 1: abar = X^T a1",
     "for (int r = 0; r < rows; r++) s += col[r] * x[r];",
     "for (int r = 0; r < rows; r++) s += col[r] * x[rows - 1 - r];"),
    ("secular_dropped_term", "Sec. 3.1: the secular sum",
     "for (int i = 0; i < k; i++) {\n        double del = (d[i] - dorg) - tau;",
     "for (int i = 1; i < k; i++) {\n        double del = (d[i] - dorg) - tau;"),
    ("secular_offset_sign", "Sec. 3.1: d_i - mu = (d_i - d_org) - tau",
     "double del = (d[i] - dorg) - tau;", "double del = (d[i] - dorg) + tau;"),
    ("bisection_branch", "Sec. 3.1: w increases across each bracket",
     "if (w > 0.0) hi = mid; else lo = mid;", "if (w > 0.0) lo = mid; else hi = mid;"),
    ("reflection_sign", "Sec. 3.1: rho < 0 by reflection",
     "else { org[k - 1 - j] = k - 1 - o; tau[k - 1 - j] = -t; }",
     "else { org[k - 1 - j] = k - 1 - o; tau[k - 1 - j] = t; }"),
    ("loewner_dropped_rho", "Sec. 3.2: rho zhat_i^2 prod (d_j - d_i) = prod (mu_j - d_i)",
     "double prod = root_minus_pole(dd, oo, tt, k - 1, i) / r;",
     "double prod = root_minus_pole(dd, oo, tt, k - 1, i);"),
    ("loewner_root_index", "Sec. 3.2: the Loewner product over all roots",
     "prod *= root_minus_pole(dd, oo, tt, j - 1, i) / (dd[j] - dd[i]);",
     "prod *= root_minus_pole(dd, oo, tt, j, i) / (dd[j] - dd[i]);"),
    ("norm_without_root", "Sec. 3.2: normalised columns",
     "e->inv_norm[jj] = 1.0 / sqrt(s2);", "e->inv_norm[jj] = 1.0 / s2;"),
    ("deflation_tol_single", "Sec. 3.1 deflation: tolerance of order u",
     "return 8.0 * ORC_U * (dmax > t ? dmax : t);", "return 8.0 * 1e-8 * (dmax > t ? dmax : t);"),
    ("givens_sign", "Sec. 3.1 case (3): the rotation applied to the vectors",
     "work[b] = -s * va + c * vb;", "work[b] = s * va + c * vb;"),
    ("givens_poles_swapped", "Sec. 3.1 case (3): the rotated poles",
     "e->ds[s] = sn * sn * dj + c * c * dsv;", "e->ds[s] = c * c * dj + sn * sn * dsv;"),
    ("step1_transposed_U", "Alg. 6.1 STEP 1: btilde = U S V^T b",
     "gemv_n(m, m, U, ldu, tmp, bt);", "oracle_gemv_t(m, m, U, ldu, tmp, bt);"),
    ("step2_transposed_Q", "Alg. 6.1 STEP 2: [a btilde] Q = [a1 b1]",
     "b1[i] = qu[4] * a[i] + qu[5] * bt[i];", "b1[i] = qu[5] * a[i] + qu[4] * bt[i];"),
    ("schur_alpha_beta_swapped", "Alg. 6.1 STEPs 2-3: beta = b^T b on the left",
     "oracle_schur2(beta, qu);", "oracle_schur2(alpha, qu);"),
    ("step8_order", "Alg. 6.1 STEP 8: values with their vectors",
     "Sn[c] = Dn[m - 1 - c];", "Sn[c] = Dn[c];"),
    ("pair_sign", "u_j^T Ahat v_j >= 0 pairs the signs",
     "if (t < 0.0) for (int i = 0; i < n; i++) vj[i] = -vj[i];",
     "if (t > 0.0) for (int i = 0; i < n; i++) vj[i] = -vj[i];"),
    ("null_block_pole", "Alg. 6.1 STEP 6: D_v = diag(sigma^2, 0)",
     "Dv[i] = (i < m) ? S[i] * S[i] : 0.0;", "Dv[i] = (i < m) ? S[i] : 0.0;"),
    ("origin_far_pole", "Sec. 3.1: the offset is taken from the nearer pole",
     "if (wm >= 0.0) { o = j;     lo = 0.0;             hi = d[j + 1] - d[j]; }",
     "if (wm < 0.0)  { o = j;     lo = 0.0;             hi = d[j + 1] - d[j]; }"),
    ("root_minus_pole_sign", "Sec. 3.2: mu_j - d_i from the stored offset",
     "return (d[org[j]] - d[i]) + tau[j];", "return (d[org[j]] - d[i]) - tau[j];"),
    ("loewner_reflected_origin", "Sec. 3.2 for rho < 0, by reflection",
     "oo[i] = k - 1 - org[k - 1 - i];", "oo[i] = org[k - 1 - i];"),
    ("loewner_sign_of_z", "Sec. 3.2: zhat takes the sign of z",
     "zhat[iz] = (z[iz] < 0.0) ? -mag : mag;", "zhat[iz] = (z[iz] > 0.0) ? -mag : mag;"),
    ("norm_offset_sign", "Sec. 3.2: ||c_j||^2 = sum zhat_i^2/(d_i - mu_j)^2",
     "double del = (e->dk[i] - e->dk[e->org[jj]]) - e->tau[jj];",
     "double del = (e->dk[i] - e->dk[e->org[jj]]) + e->tau[jj];"),
    ("atilde_with_D", "Alg. 6.1 STEP 1: atilde = V S^T U^T a",
     "for (int i = 0; i < n; i++) tmp[i] = (i < m) ? S[i] * Uta[i] : 0.0;",
     "for (int i = 0; i < n; i++) tmp[i] = (i < m) ? S[i] * S[i] * Uta[i] : 0.0;"),
    ("beta_short_sum", "Alg. 6.1 STEP 1: beta = b^T b over all n entries",
     "for (int i = 0; i < n; i++) beta += b[i] * b[i];",
     "for (int i = 0; i < m; i++) beta += b[i] * b[i];"),
    ("step3_transposed_Q", "Alg. 6.1 STEP 3: [b atilde] Q = [a2 b2]",
     "a2[i] = qv[2] * b[i] + qv[3] * at[i];", "a2[i] = qv[3] * b[i] + qv[2] * at[i];"),
    ("apply_index", "Alg. 6.1 STEPs 5, 7: Q X summed over the columns of Q",
     "for (int r = 0; r < N; r++) y[r] += qv[r] * x[c];",
     "for (int r = 0; r < N; r++) y[r] += qv[r] * x[r];"),
    ("jacobi_rotation", "one-sided Jacobi: an orthogonal plane rotation",
     "wp[i] = c * x - s * y; wq[i] = s * x + c * y;",
     "wp[i] = c * x - s * y; wq[i] = s * x - c * y;"),
]


def _compile(src_text, out_dir, name):
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, "lib" + name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", so, c, "-lm"])
    return so


def _run_pins(so):
    env = dict(os.environ, SVDUP_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q",
                            "-p", "no:cacheprovider"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    except subprocess.TimeoutExpired:
        return None, "timeout"
    return r.returncode, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def verdicts(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("oracle_mutants"))
    with open(SRC) as f:
        base = f.read()
    libs = {"unaltered": _compile(base, out, "unaltered")}
    for name, _, old, new in MUTANTS:
        assert base.count(old) == 1, "planted text not found once: %s" % name
        libs[name] = _compile(base.replace(old, new), out, name)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as ex:
        futs = {name: ex.submit(_run_pins, so) for name, so in libs.items()}
        return {name: f.result() for name, f in futs.items()}


def test_unaltered_copy_passes_every_pin(verdicts):
    rc, log = verdicts["unaltered"]
    assert rc == 0, log


@pytest.mark.parametrize("name,passage", [(m[0], m[1]) for m in MUTANTS],
                         ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(verdicts, name, passage):
    rc, log = verdicts[name]
    # a failed assertion (exit 1) or a crash of the child both reject the copy
    assert rc is not None and rc != 0, "no pin caught the planted mistake (%s):\n%s" % (passage, log)
    assert rc < 0 or "failed" in log, log
