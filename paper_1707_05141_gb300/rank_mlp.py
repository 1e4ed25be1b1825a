"""Learned rank predictor for the batched randomized SVD: training and use.

The network (16 sketch features -> 64 -> 64 -> 1, ReLU) runs in the library's own CUDA kernels
(``bsvd_mlp_forward``, ``bsvd_mlp_grad``, ``bsvd_mlp_adam``); this module only drives them.  It is
trained on the ranks the plain adaptive randomized SVD (no rank hint) finds at the requested
tolerance, and its prediction becomes the rank hint of ``batched_rsvd`` -- whose posterior
estimate still accepts or extends every result, so a poor prediction costs time, never accuracy.
The paper has no learned part; this is the project's addition.

Checkpoint format: 8-byte magic ``BSVDMLP1``, a little-endian uint32 header length, a JSON header
(feature standardisation folded in, training metadata), then 5313 little-endian float32 params.
"""
from __future__ import annotations

import json
import math
import struct

import numpy as np

from . import (MLP_PARAMS, SKETCH_FEATURES, Batch, bsvd_mlp_adam, bsvd_mlp_forward, bsvd_mlp_grad,
               bsvd_sketch_features, rsvd)

MAGIC = b"BSVDMLP1"
F, H = SKETCH_FEATURES, 64


def init_params(seed: int = 0) -> np.ndarray:
    """He initialisation of the hidden layers, small output weights, output bias 1."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, F)) * math.sqrt(2.0 / F)
    W2 = rng.standard_normal((H, H)) * math.sqrt(2.0 / H)
    w3 = rng.standard_normal(H) * math.sqrt(1.0 / H)
    p = np.concatenate([W1.reshape(-1), np.zeros(H), W2.reshape(-1), np.zeros(H), w3, [1.0]])
    return p.astype(np.float32)


def features(flat, offsets, m, n, seed: int = 0):
    """Sketch features (batch x 16 FP32 device tensor) of matrices packed in ``flat``."""
    import torch
    A = Batch.packed(flat, offsets, m, n)
    out = torch.empty((A.batch, F), dtype=torch.float32, device=flat.device)
    bsvd_sketch_features(A, out, seed)
    return out


def plain_adaptive_ranks(flat, offsets, m, n, tol: float = 1e-5, seed: int = 0, max_rounds: int = 16,
                         oversample: int = 8):
    """Labels: the ranks the adaptive randomized SVD finds without a hint."""
    res = rsvd(flat, offsets, m, n, rank_hint=None, tol=tol, oversample=oversample, max_rounds=max_rounds, seed=seed)
    return res.rank, res


def _fold_standardisation(p: np.ndarray, mu: np.ndarray, sd: np.ndarray) -> np.ndarray:
    """Parameters trained on (f - mu) / sd rewritten to act on raw features f."""
    p = p.astype(np.float64).copy()
    W1 = p[:H * F].reshape(H, F)
    b1 = p[H * F:H * F + H]
    W1n = W1 / sd
    b1n = b1 - W1n @ mu
    p[:H * F] = W1n.reshape(-1)
    p[H * F:H * F + H] = b1n
    return p.astype(np.float32)


def train(feats, ranks, steps: int = 3000, batch: int = 2048, lr: float = 3e-3, seed: int = 0, log_every: int = 0):
    """Train on device tensors ``feats`` (N x 16) and integer ``ranks`` (N); returns (params on the
    device, acting on raw features, and the loss history)."""
    import torch
    dev = feats.device
    fh = feats.double().cpu().numpy()
    mu = fh.mean(0)
    sd = fh.std(0)
    sd[sd < 1e-6] = 1.0
    Xn = torch.from_numpy(((fh - mu) / sd).astype(np.float32)).to(dev)
    target = torch.log(ranks.float() + 1.0).to(dev)
    params = torch.from_numpy(init_params(seed)).to(dev)
    grad = torch.zeros_like(params)
    mom = torch.zeros_like(params)
    vel = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    N = Xn.shape[0]
    hist = []
    for step in range(1, steps + 1):
        idx = torch.randint(0, N, (min(batch, N),), generator=gen).to(dev)
        bsvd_mlp_grad(Xn[idx].contiguous(), target[idx].contiguous(), params, grad, loss)
        bsvd_mlp_adam(params, grad, mom, vel, step, lr * (0.5 * (1 + math.cos(math.pi * step / steps))) + 1e-5)
        if log_every and (step % log_every == 0 or step == steps):
            hist.append((step, float(loss.item())))
    raw = torch.from_numpy(_fold_standardisation(params.cpu().numpy(), mu, sd)).to(dev)
    return raw, hist


def predict(feats, params, margin: float = 2.0, m=None, n=None):
    """(log(rank + 1) estimates, rank hints) for ``feats`` on the device."""
    import torch
    B = feats.shape[0]
    out = torch.empty(B, dtype=torch.float32, device=feats.device)
    hint = torch.empty(B, dtype=torch.int32, device=feats.device)
    md = None if m is None else torch.as_tensor(np.asarray(m, np.int32)).to(feats.device)
    nd = None if n is None else torch.as_tensor(np.asarray(n, np.int32)).to(feats.device)
    bsvd_mlp_forward(feats, params, out, hint, margin, md, nd)
    return out, hint


def save(path: str, params, meta: dict | None = None) -> None:
    p = params.detach().cpu().numpy().astype("<f4") if hasattr(params, "detach") else np.asarray(params, "<f4")
    if p.size != MLP_PARAMS:
        raise ValueError(f"{p.size} parameters, expected {MLP_PARAMS}")
    hdr = json.dumps(dict(meta or {}, nparams=int(p.size), features=F, hidden=H)).encode()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<I", len(hdr)))
        f.write(hdr)
        f.write(p.tobytes())


def load(path: str):
    """(params as a float32 numpy array, header dict)."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != MAGIC or len(data) < 12:
        raise ValueError(f"{path}: not a rank-predictor checkpoint")
    (hl,) = struct.unpack("<I", data[8:12])
    body = data[12 + hl:]
    try:
        hdr = json.loads(data[12:12 + hl].decode()) if 12 + hl <= len(data) else None
    except (UnicodeDecodeError, ValueError):
        hdr = None
    if not isinstance(hdr, dict):
        raise ValueError(f"{path}: damaged checkpoint header")
    if len(body) != 4 * MLP_PARAMS or hdr.get("nparams", MLP_PARAMS) != MLP_PARAMS:
        raise ValueError(f"{path}: {len(body) // 4} parameters, expected {MLP_PARAMS}")
    return np.frombuffer(body, dtype="<f4").copy(), hdr
