"""Mutation check of the oracle's pins (CPU only).

Each case plants one plausible mistake in a temporary copy of the oracle package -- a wrong sign,
a dropped term or factor, a transposed operand, an index slip, a precision slip -- and runs the
oracle's pin tests against that copy in a fresh interpreter.  Every planted mistake must make at
least one pin fail, and the unmodified copy must pass them all, so that a failure is the
mistake's and not the harness's.  The mistakes are planted in the copy only; the oracle itself is
never modified.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join(ROOT, "tests", f"test_oracle_{k}.py") for k in ("qr", "svd", "rsvd", "mlp", "h2")]

# (what the mistake is, file, exact text, replacement); each text occurs exactly once in its file.
MUTANTS = [
    # Algorithm 1: Householder QR
    ("house: reflector built with the wrong sign", "oracle.c",
     "v[0] += (x[0] >= 0.0 ? alpha : -alpha);", "v[0] += (x[0] >= 0.0 ? -alpha : alpha);"),
    ("house: sign(0) taken as -1", "oracle.c",
     "v[0] += (x[0] >= 0.0 ? alpha : -alpha);", "v[0] += (x[0] > 0.0 ? alpha : -alpha);"),
    ("house: v left unnormalised", "oracle.c",
     "for (int i = 0; i < len; ++i) v[i] /= nv;", "for (int i = 0; i < len; ++i) v[i] /= nv * nv;"),
    ("QR: factor 2 dropped from the update of R", "oracle.c",
     "for (int r = 0; r < m; ++r) AT(Rw, m, r, j) -= 2.0 * w * v[r];",
     "for (int r = 0; r < m; ++r) AT(Rw, m, r, j) -= w * v[r];"),
    ("QR: reflector applied to Q from the left (transposed operand)", "oracle.c",
     "for (int c = 0; c < m; ++c) w += AT(Qw, m, r, c) * v[c];",
     "for (int c = 0; c < m; ++c) w += AT(Qw, m, c, r) * v[c];"),
    ("QR: entries below the diagonal of R not zeroed", "oracle.c",
     "AT(R, ldr, i, j) = (i <= j) ? AT(Rw, m, i, j) : 0.0;", "AT(R, ldr, i, j) = AT(Rw, m, i, j);"),
    ("QR: diagonal of R dropped", "oracle.c",
     "AT(R, ldr, i, j) = (i <= j) ? AT(Rw, m, i, j) : 0.0;", "AT(R, ldr, i, j) = (i < j) ? AT(Rw, m, i, j) : 0.0;"),
    ("nrm2: square root dropped", "oracle.c", "return scale * sqrt(ssq);", "return scale * ssq;"),
    # Algorithm 2: one-sided Jacobi
    ("rot: zeta with the wrong sign", "oracle.c",
     "double zeta = (beta - alpha) / (2.0 * gamma);", "double zeta = (alpha - beta) / (2.0 * gamma);"),
    ("rot: factor 2 dropped from zeta", "oracle.c",
     "double zeta = (beta - alpha) / (2.0 * gamma);", "double zeta = (beta - alpha) / gamma;"),
    ("rot: sine with the wrong sign", "oracle.c", "*s = *c * t;", "*s = -*c * t;"),
    ("rot: skip test not scaled by the column norms", "oracle.c",
     "if (fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) return 0;", "if (fabs(gamma) <= tol) return 0;"),
    ("Jacobi: gamma accumulates a_i a_i", "oracle.c", "gamma += ai * aj;", "gamma += ai * ai;"),
    ("Jacobi: column j rotated with the wrong sign", "oracle.c",
     "AT(W, ldw, r, j) = s * ai + c * aj;", "AT(W, ldw, r, j) = s * ai - c * aj;"),
    ("Jacobi: rotation of V transposed", "oracle.c",
     "AT(V, ldv, r, i) = c * vi - s * vj;\n                    AT(V, ldv, r, j) = s * vi + c * vj;",
     "AT(V, ldv, r, i) = c * vi + s * vj;\n                    AT(V, ldv, r, j) = -s * vi + c * vj;"),
    ("Jacobi: last column never paired", "oracle.c",
     "for (int j = i + 1; j < n; ++j) {", "for (int j = i + 1; j < n - 1; ++j) {"),
    ("Jacobi: FP32 tolerance in the FP64 oracle", "oracle.c",
     "if (tol <= 0.0) tol = sqrt((double)mm) * ldexp(1.0, -53);",
     "if (tol <= 0.0) tol = sqrt((double)mm) * ldexp(1.0, -24);"),
    ("SVD: singular values sorted ascending", "oracle.c",
     "while (b >= 0 && sig[perm[b]] < sig[p]) {", "while (b >= 0 && sig[perm[b]] > sig[p]) {"),
    ("SVD: U columns not divided by sigma", "oracle.c",
     "AT(Ul, ldul, i, q) = (sig[j] > 0.0) ? AT(W, mm, i, j) / sig[j] : 0.0;",
     "AT(Ul, ldul, i, q) = AT(W, mm, i, j);"),
    ("SVD: wide matrix read untransposed", "oracle.c",
     "AT(W, mm, i, j) = tr ? AT(A, lda, j, i) : AT(A, lda, i, j);",
     "AT(W, mm, i, j) = tr ? AT(A, lda, i % m, j) : AT(A, lda, i, j);"),
    ("SVD: V columns not permuted with sigma", "oracle.c",
     "for (int i = 0; i < nn; ++i) AT(Vr, ldvr, i, q) = AT(Vw, nn, i, j);",
     "for (int i = 0; i < nn; ++i) AT(Vr, ldvr, i, q) = AT(Vw, nn, i, q);"),
    # Philox4x32-10 and Box-Muller
    ("Philox: second Weyl constant replaced by the first", "oracle.c",
     "k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;"),
    ("Philox: x3 instead of x1 in the first output word", "oracle.c",
     "uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;", "uint32_t y0 = (uint32_t)(p1 >> 32) ^ x3 ^ k0;"),
    ("Philox: nine rounds", "oracle.c",
     "for (int round = 0; round < 10; ++round) {", "for (int round = 0; round < 9; ++round) {"),
    ("Box-Muller: radius without the factor 2", "oracle.c",
     "double r = sqrt(-2.0 * log(ua));", "double r = sqrt(-log(ua));"),
    ("Box-Muller: both rows of a pair from one uniform", "oracle.c",
     "uint32_t wa = w[(sub >> 1) * 2], wb = w[(sub >> 1) * 2 + 1];",
     "uint32_t wa = w[(sub >> 1) * 2], wb = w[(sub >> 1) * 2];"),
    # Algorithm 4: randomized SVD
    ("RSVD: power step dropped", "oracle.c",
     "for (int it = 0; it < q && rc == 0; ++it) {", "for (int it = 0; it < 0 && rc == 0; ++it) {"),
    ("RSVD: small SVD of R_B instead of R_B^T", "oracle.c",
     "for (int i = 0; i < l; ++i) AT(RBt, l, i, j) = AT(RB, l, j, i);",
     "for (int i = 0; i < l; ++i) AT(RBt, l, i, j) = AT(RB, l, i, j);"),
    ("RSVD: V = Q_B U_R", "oracle.c",
     "orc_gemm(0, 0, n, l, l, QB, n, VR, l, V, n);", "orc_gemm(0, 0, n, l, l, QB, n, UR, l, V, n);"),
    ("RSVD: projection B = Q A instead of Q^T A", "oracle.c",
     "orc_gemm(1, 0, l, n, m, Q, m, A, lda, B, l);", "orc_gemm(0, 0, l, n, m, Q, m, A, lda, B, l);"),
    ("gemm: op(B) transposed the wrong way", "oracle.c",
     "double b = tb ? AT(B, ldb, j, l) : AT(B, ldb, l, j);", "double b = tb ? AT(B, ldb, l, j) : AT(B, ldb, j, l);"),
    ("adaptive: round accepted at eps instead of eps / 2", "oracle.c",
     "if (est2 <= 0.25 * eps * eps * norm2) {", "if (est2 <= eps * eps * norm2) {"),
    ("adaptive: probes drawn from the Omega stream", "oracle.c",
     "orc_omega(seed, index, 1, n, 0, r, W);", "orc_omega(seed, index, 0, n, 0, r, W);"),
    ("adaptive: probe residual without the singular values", "oracle.c",
     "for (int c = 0; c < l; ++c) e -= AT(U, m, i, c) * S[c] * AT(VW, l, c, j);",
     "for (int c = 0; c < l; ++c) e -= AT(U, m, i, c) * AT(VW, l, c, j);"),
    ("adaptive: estimate not averaged over the probes", "oracle.c",
     "return r > 0 ? sum / r : 0.0;", "return sum;"),
    ("adaptive: sample grows by one column per round", "oracle.c", "            l += p;\n", "            l += 1;\n"),
    ("adaptive: fallback only past min(m, n)", "oracle.c",
     "} else if (l + p >= k || l + p > lcap) {", "} else if (l + p > k || l + p > lcap) {"),
    ("budget: estimate added to the truncation budget", "oracle.c",
     "double thr = 0.95 * 0.95 * eps * eps * normA2 - 4.0 * est2;",
     "double thr = 0.95 * 0.95 * eps * eps * normA2 + 4.0 * est2;"),
    ("fixed rank: full SVD only past min(m, n)", "oracle.c",
     "    if (l >= kk || l > lcap) {", "    if (l > kk || l > lcap) {"),
    ("truncation: threshold not squared", "oracle.c", "double thr2 = thr * thr;", "double thr2 = thr;"),
    ("truncation: rank one too high", "oracle.c", "if (t > thr2) break;\n        tail = t;\n        k = i;\n",
     "if (t > thr2) break;\n        tail = t;\n        k = i + 1;\n"),
    ("budget: rank one too high", "oracle.c", "if (t > thr) break;\n        tail = t;\n        k = i;\n",
     "if (t > thr) break;\n        tail = t;\n        k = i + 1;\n"),
    # rank predictor (FP64 reference of the network and its features)
    ("MLP: loss without the factor 1/2", "mlp.py",
     "L = 0.5 * float(r @ r) / B", "L = float(r @ r) / B"),
    ("MLP: second ReLU gated by the first layer", "mlp.py",
     'd2 = np.outer(dy, q["w3"]) * (z2 > 0)', 'd2 = np.outer(dy, q["w3"]) * (z1 > 0)'),
    ("MLP: W2 transposed in backpropagation", "mlp.py",
     'd1 = (d2 @ q["W2"]) * (z1 > 0)', 'd1 = (d2 @ q["W2"].T) * (z1 > 0)'),
    ("MLP: bias b3 gradient from the unscaled residual", "mlp.py",
     "g_b3 = np.array([dy.sum()])", "g_b3 = np.array([r.sum()])"),
    ("MLP: output bias dropped from the forward pass", "mlp.py",
     'y = h2 @ q["w3"] + q["b3"][0]', 'y = h2 @ q["w3"]'),
    ("features: column norms unsquare-rooted", "mlp.py",
     "r = np.sqrt(cn) / fro", "r = cn / fro"),
    ("features: power ratio divided by ||A||_F", "mlp.py",
     "w = ww / (yy * fro2)", "w = ww / (yy * fro)"),
    ("features: stable rank from rmax, not rmax^2", "mlp.py",
     "l10(fro2 / rmax ** 2)", "l10(fro2 / rmax)"),
    ("features: top-energy share over all columns", "mlp.py",
     "etop = np.sort(cn)[::-1][:top].sum()", "etop = np.sort(cn)[:top].sum()"),
    ("features: log-norm spread without the mean", "mlp.py",
     "math.sqrt(max((lr * lr).mean() - lr.mean() ** 2, 0.0))", "math.sqrt(max((lr * lr).mean(), 0.0))"),
    ("features: sketch from the wrong Gaussian stream", "mlp.py",
     "G = omega(seed, index, 2, n, 0, 8)", "G = omega(seed, index, 1, n, 0, 8)"),
    # H^2 basis-tree truncation (Section 8.2)
    ("H2: parent projection without the singular values", "h2.py",
     "T[l - 1].append(st[:, None] * wt.T)", "T[l - 1].append(wt.T)"),
    ("H2: new transfers split at the second child's rank", "h2.py",
     "r1 = ranks[l][c1]", "r1 = ranks[l][c2]"),
    ("H2: threshold against the squared norm", "h2.py",
     "trunc_rank(s, float(np.sqrt((s * s).sum())), eps)", "trunc_rank(s, float((s * s).sum()), eps)"),
    ("H2: children swapped in TE", "h2.py",
     "np.vstack([T[l][c1] @ transfers[l][c1], T[l][c2] @ transfers[l][c2]])",
     "np.vstack([T[l][c2] @ transfers[l][c2], T[l][c1] @ transfers[l][c1]])"),
    ("H2: TE from the transfers without the children's projections", "h2.py",
     "np.vstack([T[l][c1] @ transfers[l][c1], T[l][c2] @ transfers[l][c2]])",
     "np.vstack([transfers[l][c1][:ranks[l][c1]], transfers[l][c2][:ranks[l][c2]]])"),
]

# Builds and imports the copy before any pin runs; a copy that does not build or import exits 97
# (a harness error, never counted as a caught mistake).
_BOOT = ("import sys; sys.path.insert(0, sys.argv[1])\n"
         "try:\n"
         "    import oracle, oracle.mlp; assert oracle.__file__.startswith(sys.argv[1]); oracle.build()\n"
         "except BaseException as e:\n"
         "    print('copy does not build:', e); sys.exit(97)\n"
         "import pytest; sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider'] + sys.argv[2:]))\n")


def _copy(dst, mutant=None):
    pkg = os.path.join(dst, "oracle")
    os.makedirs(pkg)
    for f in ("__init__.py", "mlp.py", "h2.py", "oracle.c"):
        shutil.copy(os.path.join(ROOT, "oracle", f), pkg)
    if mutant is not None:
        _, fname, old, new = mutant
        path = os.path.join(pkg, fname)
        with open(path) as fh:
            src = fh.read()
        assert src.count(old) == 1, f"{mutant[0]}: text not found exactly once in {fname}"
        with open(path, "w") as fh:
            fh.write(src.replace(old, new))


def _run(dst):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    p = subprocess.run([sys.executable, "-c", _BOOT, dst] + PINS, cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return p.returncode, p.stdout + p.stderr


def test_unmodified_copy_passes_every_pin(tmp_path):
    _copy(str(tmp_path))
    rc, out = _run(str(tmp_path))
    assert rc == 0, out[-3000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    dirs = []
    for k, mutant in enumerate(MUTANTS):
        d = os.path.join(str(tmp_path), f"m{k:02d}")
        _copy(d, mutant)
        dirs.append(d)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(_run, dirs))
    broken = [(m[0], out[-600:]) for m, (rc, out) in zip(MUTANTS, results) if rc not in (0, 1) and rc > 0]
    assert not broken, f"mutants that did not build or run: {broken}"
    # pytest exits 1 when a pin fails; a negative code is a crash of the planted mistake itself
    survived = [m[0] for m, (rc, _) in zip(MUTANTS, results) if rc == 0]
    assert not survived, f"planted mistakes that no pin caught: {survived}"
