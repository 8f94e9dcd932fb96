"""The oracle's pins catch plausible mistakes: each case below plants one
mistake in a copy of the oracle (a dropped term, a flipped sign, a transposed
operand, a wrong index or constant, a bound too narrow or too wide) and runs
the pin file that should catch it against that copy; the run must fail.

The copy lives in a temporary directory and is imported ahead of the
repository's own (the working directory and PYTHONPATH put it first), so the
repository's oracle is never modified.  CPU only."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")

# (what is wrong, file in oracle/, text, replacement, pin file that must fail)
MUTATIONS = [
    ("ACA: t1 drops Q3.y (Eq. 27)", "oracle.c",
     "const double t1 = fA1 - Q3x - Q3y;", "const double t1 = fA1 - Q3x;", "test_oracle_aca.py"),
    ("ACA: H_C's third row takes c33 - c11 (Eq. 28)", "oracle.c",
     "{c11, 0, 0, 0, c22, 0, c11 - c33, c22 - c33, c33}", "{c11, 0, 0, 0, c22, 0, c33 - c11, c22 - c33, c33}",
     "test_oracle_aca.py"),
    ("ACA: H_A1 with M1P1 and M1N1 exchanged (Eq. 20)", "oracle.c",
     "c33};\n    const double L1[9] = {MP1y, -MP1x, 0, -MN1y, MN1x, 0, 0, 0, fA1};",
     "c33};\n    const double L1[9] = {-MN1y, MN1x, 0, MP1y, -MP1x, 0, 0, 0, fA1};", "test_oracle_aca.py"),
    ("DLT: the second row's y2 x1 term with the wrong sign (Eq. 2)", "oracle.c",
     "r1[6] = Y * x;", "r1[6] = -Y * x;", "test_oracle_aca.py"),
    ("SKS: Q7.y adds P5.y (Eq. 10)", "oracle.c",
     "Q7y = Q3[2] / Q3[1] - P5y;", "Q7y = Q3[2] / Q3[1] + P5y;", "test_oracle_sks_rect_jac.py"),
    ("affine: H_A2^-1 with M2N2 and M2P2 exchanged (Eq. 38)", "oracle.c",
     "mat3_mul(L1, T1, HA1);\n    const double HA2inv[9] = {MN2x, MP2x, M2x, MN2y, MP2y, M2y, 0, 0, 1};\n    mat3_mul(HA2inv, HA1, H);",
     "mat3_mul(L1, T1, HA1);\n    const double HA2inv[9] = {MP2x, MN2x, M2x, MP2y, MN2y, M2y, 0, 0, 1};\n    mat3_mul(HA2inv, HA1, H);",
     "test_oracle_aca.py"),
    ("rectangle: Eq. 42's y0 term without the aspect ratio", "oracle.c",
     "-r * Q4y * y0, t2", "-Q4y * y0, t2", "test_oracle_sks_rect_jac.py"),
    ("RANSAC argmax: a tie takes the later hypothesis", "oracle.c",
     "        for (int32_t h = 0; h < k; ++h)\n            if (cnt[h] > bc) {\n                bc = cnt[h];\n                bh = h;\n            }\n        if (bc < 0) {",
     "        for (int32_t h = 0; h < k; ++h)\n            if (cnt[h] >= bc) {\n                bc = cnt[h];\n                bh = h;\n            }\n        if (bc < 0) {",
     "test_oracle_sampling_scoring.py"),
    ("degenerate samples: the triple (N, P, Q) not tested", "oracle.c",
     "triple_degenerate(MNx, MNy, MQx, MQy) || triple_degenerate(NPx, NPy, NQx, NQy);",
     "triple_degenerate(MNx, MNy, MQx, MQy);", "test_oracle_sampling_scoring.py"),
    ("normalisation: h33 made negative", "oracle.c",
     "(H[8] > 0 ? 1.0 : -1.0)", "(H[8] > 0 ? -1.0 : 1.0)", "test_oracle_sampling_scoring.py"),
    ("Jacobian: the dual chain's t1 drops Q3.y", "oracle.c",
     "const dual t1 = dsub(dsub(fA1, Q3x), Q3y);", "const dual t1 = dsub(fA1, Q3x);", "test_oracle_sks_rect_jac.py"),
    ("rectangle Jacobian: the dual chain's y0 term without the aspect ratio", "oracle.c",
     "dneg(dmul(dmul(R, Q4y), Y0))", "dneg(dmul(Q4y, Y0))", "test_oracle_sks_rect_jac.py"),
    ("Philox: a key increment off by one", "oracle.c",
     "k0 += 0x9E3779B9u;", "k0 += 0x9E3779B8u;", "test_oracle_sampling_scoring.py"),
    ("sampling: a rank steps over strictly smaller earlier draws only", "oracle.c",
     "if (j >= sorted[a])", "if (j > sorted[a])", "test_oracle_sampling_scoring.py"),
    ("scoring: w takes h13 for h33", "oracle.c",
     "const double w = H[6] * x + H[7] * y + H[8];\n    if (w == 0) {",
     "const double w = H[6] * x + H[7] * y + H[2];\n    if (w == 0) {", "test_oracle_sampling_scoring.py"),
    ("scoring: the threshold test made strict", "oracle.c",
     "    return r <= thr;", "    return r < thr;", "test_oracle_sampling_scoring.py"),
    ("adaptive K: w^3 for w^4 (Sec. 6.2)", "oracle.c",
     "const double w4 = (w * w) * (w * w);", "const double w4 = (w * w) * w;", "test_oracle_adaptive.py"),
    ("adaptive stop: one hypothesis past K", "oracle.c",
     "if (i >= kreq) return i;", "if (i > kreq) return i;", "test_oracle_adaptive.py"),
    ("refit: Hartley scale to mean distance 2, not sqrt(2)", "inlier_refit.py",
     "SQRT2 = np.sqrt(2.0)", "SQRT2 = 2.0", "test_oracle_refit.py"),
    ("refit: the DLT's second row with the wrong sign of y2 (Eq. 2)", "inlier_refit.py",
     "A[1:2 * len(x):2, 6:9] = X[:, 1:2] * xh", "A[1:2 * len(x):2, 6:9] = -X[:, 1:2] * xh", "test_oracle_refit.py"),
    ("refit: a wrong Jacobian entry of the LM residual", "inlier_refit.py",
     "J[1::2, 6] = -v * x[:, 0] / w", "J[1::2, 6] = -u * x[:, 0] / w", "test_oracle_refit.py"),
    ("bound: the rounding of X / thr left out", "fp32_bounds.c",
     "const int Xs = mul(t, X, rt), Ys = mul(t, Y, rt);", "const int Xs = xscale(t, X, V(rt)), Ys = mul(t, Y, rt);",
     "test_oracle_fp32_bounds.py"),
    ("bound: the multiplication rule doubled", "fp32_bounds.c",
     "const double v = V(a) * V(b);\n    const int k = push(t, v, fabs(v), fabs(v));",
     "const double v = V(a) * V(b);\n    const int k = push(t, v, fabs(v), 2.0 * fabs(v));",
     "test_oracle_fp32_bounds.py"),
    ("bound: Kahan's determinant rule halved", "fp32_bounds.c",
     "const int k = push(t, v, fabs(v), 2.0 * fabs(v));\n    dep(t, k, a, V(d));",
     "const int k = push(t, v, fabs(v), fabs(v));\n    dep(t, k, a, V(d));", "test_oracle_fp32_bounds.py"),
    ("bound: negation's derivative with the wrong sign", "fp32_bounds.c",
     "dep(t, k, a, -1.0);\n    return k;\n}\n/* exact sum", "dep(t, k, a, 1.0);\n    return k;\n}\n/* exact sum",
     "test_oracle_fp32_bounds.py"),
    ("bound: the reverse sweep over absolute weights", "fp32_bounds.c",
     "adj[q->p[i]] += a * q->w[i];", "adj[q->p[i]] += a * fabs(q->w[i]);", "test_oracle_fp32_bounds.py"),
]


def _run_mutant(tmp, k, case):
    what, fname, old, new, pin = case
    d = os.path.join(tmp, f"m{k}")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    path = os.path.join(d, "oracle", fname)
    with open(path) as f:
        src = f.read()
    assert src.count(old) == 1, f"{what}: the text to replace must occur exactly once"
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([d, ROOT]), OMP_NUM_THREADS="2")
    # the copy, not the repository's oracle, is the one imported, and it
    # builds: a pin run then fails on the planted mistake, not on the build
    where = subprocess.run([sys.executable, "-c", "import oracle; oracle.build(); print(oracle.__file__)"], cwd=d,
                           env=env, capture_output=True, text=True)
    assert where.returncode == 0 and where.stdout.strip().startswith(d), where.stdout + where.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(TESTS, pin), "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider", "-p", "no:xdist"], cwd=d, env=env, capture_output=True, text=True)
    return what, pin, r.returncode, r.stdout[-1500:] + r.stderr[-1500:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda kc: _run_mutant(str(tmp_path), *kc), enumerate(MUTATIONS)))
    survived = [(w, p) for w, p, rc, _ in results if rc == 0]
    broken = [(w, p, rc, out) for w, p, rc, out in results if rc not in (0, 1)]
    assert not broken, f"pin runs that did not complete (exit code other than pass or fail): {broken}"
    assert not survived, f"planted mistakes that no pin caught: {survived}"
    print(f"{len(results)} planted mistakes, each failed its pin file")
