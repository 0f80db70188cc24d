"""Plain FP64 CPU oracle of the steps around the TTT layer in Scal3R's Global
Context Memory (GCM) module.

TEST INFRASTRUCTURE ONLY, like ``ttt_oracle``: nothing on the product path
uses it, and it shares no code with the CUDA path.

What it computes (arXiv 2604.08542):

* The GCM module projects a chunk's tokens x [T, d] to queries, keys and
  values with a standard linear layer (Sec. 4.2, first paragraph; Supp.
  "Global Context Memory module"), [q | k | v] = x Wqkv^T + bqkv, split into
  H heads of D = d / H.
* The TTT layer (``ttt_oracle.forward``) updates the fast weights with k, v
  and a token-wise learning rate "predicted from the input tokens" (Sec. 4.2,
  after Eq. 8) and applies them to q, giving o.
* An output projection o Wo^T, and the gated residual of Eq. 5,
      out = alpha (o) (o Wo^T) + x,   alpha in R^d.
* Readings where the paper is silent: q and k are scaled to unit L2 norm per
  head (the layer's inputs in the paper's references are normalised; the
  paper does not say); the learning-rate predictor is
      lr = base * sigmoid(x w_eta^T + b_eta),  w_eta [H, d], b_eta [H];
  the output projection has no bias.

The backward is written out by the chain rule through these steps and the
TTT oracle's backward; the tests pin it to central finite differences.
"""
from __future__ import annotations

import numpy as np

from .ttt_oracle import backward as ttt_backward
from .ttt_oracle import forward as ttt_forward
from .ttt_oracle import sigmoid


def gcm_forward(x, wqkv, bqkv, w_eta, b_eta, base_lr, wo, alpha, w0, layout, H: int, D: int, F: int,
                eps: float = 1e-12) -> dict:
    """out = alpha * (TTT(q, k, v, lr) Wo^T) + x for tokens x [T, d]."""
    x, wqkv, bqkv, w_eta, b_eta, wo, alpha = (np.asarray(a, dtype=np.float64)
                                               for a in (x, wqkv, bqkv, w_eta, b_eta, wo, alpha))
    T, d = x.shape
    raw = x @ wqkv.T + bqkv
    q = raw[:, :d].reshape(T, H, D)
    k = raw[:, d:2 * d].reshape(T, H, D)
    v = raw[:, 2 * d:].reshape(T, H, D)
    qn = np.sqrt((q * q).sum(-1))
    kn = np.sqrt((k * k).sum(-1))
    qh = q / np.maximum(qn, 1e-300)[..., None]
    kh = k / np.maximum(kn, 1e-300)[..., None]
    s = sigmoid(x @ w_eta.T + b_eta)
    lr = base_lr * s
    t = ttt_forward(qh, kh, v, lr, w0, layout, D, F, eps=eps)
    o = t["o"].reshape(T, d)
    y = o @ wo.T
    out = alpha * y + x
    return {"out": out, "y": y, "q": qh, "k": kh, "v": v, "qn": qn, "kn": kn, "sig": s, "lr": lr, "o": o,
            "ttt": t}


def gcm_backward(x, wqkv, bqkv, w_eta, b_eta, base_lr, wo, alpha, w0, layout, d_out, H: int, D: int, F: int,
                 eps: float = 1e-12) -> dict:
    """Gradients of sum(d_out * out) w.r.t. x, Wqkv, bqkv, w_eta, b_eta, Wo, alpha and w0."""
    f = gcm_forward(x, wqkv, bqkv, w_eta, b_eta, base_lr, wo, alpha, w0, layout, H, D, F, eps=eps)
    x, wqkv, w_eta, wo, alpha = (np.asarray(a, dtype=np.float64) for a in (x, wqkv, w_eta, wo, alpha))
    d_out = np.asarray(d_out, dtype=np.float64)
    T, d = x.shape
    # out = alpha y + x
    dalpha = (f["y"] * d_out).sum(0)
    dx = d_out.copy()
    dy = alpha * d_out
    # y = o Wo^T
    dwo = dy.T @ f["o"]
    do = (dy @ wo).reshape(T, H, D)
    tb = ttt_backward(f["q"], f["k"], f["v"], f["lr"], w0, layout, do, D, F, eps=eps)
    # unit-norm scaling of q and k: d raw = (g - u (u . g)) / |raw|, u = raw / |raw|
    dq = (tb["dq"] - f["q"] * (f["q"] * tb["dq"]).sum(-1, keepdims=True)) / f["qn"][..., None]
    dk = (tb["dk"] - f["k"] * (f["k"] * tb["dk"]).sum(-1, keepdims=True)) / f["kn"][..., None]
    dqkv = np.concatenate([dq.reshape(T, d), dk.reshape(T, d), tb["dv"].reshape(T, d)], axis=1)
    dbqkv = dqkv.sum(0)
    dwqkv = dqkv.T @ x
    dx += dqkv @ wqkv
    # lr = base * sigmoid(z), z = x w_eta^T + b_eta
    dz = tb["dlr"] * base_lr * f["sig"] * (1.0 - f["sig"])
    db_eta = dz.sum(0)
    dw_eta = dz.T @ x
    dx += dz @ w_eta
    return {"dx": dx, "dwqkv": dwqkv, "dbqkv": dbqkv, "dw_eta": dw_eta, "db_eta": db_eta, "dwo": dwo,
            "dalpha": dalpha, "dw0": tb["dw0"]}
