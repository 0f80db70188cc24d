"""Helpers shared by the tests (test-only)."""
from __future__ import annotations

import numpy as np


def rel_inf(x, ref) -> float:
    """Normwise relative error max|x - ref| / max|ref| (max-abs if ref is 0)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if x.size == 0:
        return 0.0
    d = np.max(np.abs(x - ref))
    s = np.max(np.abs(ref))
    return float(d / s) if s > 0 else float(d)


def to_np(t) -> np.ndarray:
    return t.detach().float().cpu().numpy().astype(np.float64)


def upload(x: dict, dtype, device="cuda"):
    """Move generator outputs to the GPU: tokens in ``dtype``, the rest float32."""
    import torch
    out = {}
    for n, a in x.items():
        t = torch.from_numpy(np.ascontiguousarray(a))
        if n in ("q", "k", "v", "d_o"):
            t = t.to(dtype)
        out[n] = t.to(device).contiguous()
    return out
