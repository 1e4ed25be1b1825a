"""Comparison helpers for the GPU-vs-oracle parity tests (host side, FP64).

Tolerances (the arithmetic behind each bound is written beside it):
  * singular values, normwise: max_i |s_i - s_i^oracle| / s_1^oracle <= 1e-12 (FP64), 1e-5 (FP32).
    Jacobi is backward stable column by column, so the normwise error is a small multiple of
    m * u (u = 2^-53 or 2^-24); the bounds are the ones the method is specified to meet.
  * orthogonality ||U^T U - I||_max, ||V^T V - I||_max and the residual
    ||A - U S V^T||_F / ||A||_F: the same bound (columns with s = 0 excluded from U).
  * singular vectors are unique only up to sign and only for simple singular values; their
    first-order sensitivity is (perturbation) / (gap), so column j is compared after sign
    alignment within  C * u * s_1 / gap_j  with gap_j the distance to the nearest other value.
  * QR: Q and R are compared after normalising diag(R) >= 0 on both sides; the forward error of
    Householder QR is bounded by a multiple of kappa(A) * u for Q and of u * ||A|| for R.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def gate(dtype) -> float:
    return 1e-5 if np.dtype(dtype) == np.float32 else 1e-12


def unit(dtype) -> float:
    return U32 if np.dtype(dtype) == np.float32 else U64


def svd_errors(a64, u, s, v, s_ref):
    """Normwise sigma error vs the oracle, orthogonality of U (s > 0) and V, relative residual."""
    s = np.asarray(s, np.float64)
    s_ref = np.asarray(s_ref, np.float64)
    scale = s_ref[0] if s_ref.size and s_ref[0] > 0 else 1.0
    e_s = float(np.abs(s - s_ref).max() / scale) if s.size else 0.0
    out = {"sigma": e_s}
    if u is not None:
        u = np.asarray(u, np.float64)
        keep = s > 0
        uu = u[:, keep]
        out["orth_u"] = float(np.abs(uu.T @ uu - np.eye(uu.shape[1])).max()) if uu.size else 0.0
    if v is not None:
        v = np.asarray(v, np.float64)
        out["orth_v"] = float(np.abs(v.T @ v - np.eye(v.shape[1])).max()) if v.size else 0.0
    if u is not None and v is not None:
        na = np.linalg.norm(a64)
        out["resid"] = float(np.linalg.norm(a64 - (u * s) @ v.T) / na) if na > 0 else float(np.abs(u * s).max(initial=0))
    return out


def vector_errors(x, x_ref, s_ref, dtype, c: float = 64.0, s_all=None):
    """Columns of x vs x_ref after sign alignment, each within c * u * s_1 / gap_j.

    Returns the worst ratio (error / allowed); <= 1 passes.  Columns whose gap is zero (repeated
    singular values) are skipped: only their span is unique.  ``s_all`` (default s_ref) is the full
    list the gaps are measured in, when x holds only the leading columns of a factorisation.
    """
    x = np.asarray(x, np.float64)
    x_ref = np.asarray(x_ref, np.float64)
    s_ref = np.asarray(s_ref, np.float64)
    s_all = s_ref if s_all is None else np.asarray(s_all, np.float64)
    k = s_ref.size
    worst = 0.0
    u = unit(dtype)
    for j in range(k):
        others = np.delete(s_all, j)
        gap = np.abs(others - s_ref[j]).min() if others.size else s_ref[0]
        if gap <= 0 or s_ref[j] <= 0:
            continue
        sg = 1.0 if x[:, j] @ x_ref[:, j] >= 0 else -1.0
        err = np.abs(sg * x[:, j] - x_ref[:, j]).max()
        allowed = c * u * max(s_ref[0], 1e-300) / gap + 1e-300
        worst = max(worst, err / allowed)
    return worst


def qr_errors(a64, q, r, q_ref, r_ref, dtype):
    """(worst Q error / allowed, worst R error / allowed, orthogonality, residual) after sign fix."""
    q = np.asarray(q, np.float64)
    r = np.asarray(r, np.float64)
    m, n = q.shape if q is not None else (a64.shape[0], r.shape[0])
    d = np.sign(np.diag(r)) if r is not None else np.ones(n)
    d[d == 0] = 1.0
    dref = np.sign(np.diag(r_ref))
    dref[dref == 0] = 1.0
    u = unit(dtype)
    sv = np.linalg.svd(a64, compute_uv=False)
    na = sv[0] if sv.size else 0.0
    kappa = sv[0] / sv[-1] if sv.size and sv[-1] > 0 else np.inf
    out = {}
    if r is not None:
        rr = r * d[:, None]
        out["r"] = float(np.abs(rr - r_ref * dref[:, None]).max(initial=0.0) / (64 * u * max(na, 1e-300) * max(1, np.sqrt(m))))
        out["tril_zero"] = bool(np.all(np.tril(r, -1) == 0.0))
    if q is not None:
        qq = q * d
        if np.isfinite(kappa):
            out["q"] = float(np.abs(qq - q_ref * dref).max(initial=0.0) / (64 * u * kappa * max(1, np.sqrt(m))))
        out["orth_q"] = float(np.abs(q.T @ q - np.eye(n)).max(initial=0.0))
    if q is not None and r is not None and na > 0:
        out["resid"] = float(np.linalg.norm(a64 - q @ r) / np.linalg.norm(a64))
    return out
