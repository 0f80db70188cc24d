"""torch-facing wrapper of the GCM module around the layer (scal3r_gcm.h).

The Global Context Memory module (Sec. 4.1, Eq. 5) maps a chunk's tokens
x [T, d] to ``out = alpha * (o Wo^T) + x`` where o is the test-time-training
layer applied to the projected, normalised q, k and the projected v, with a
predicted token-wise learning rate.  Every step runs in the library: the two
projections with their row work in the GEMM epilogues (``scal3r_gcm_qkv``,
``scal3r_gcm_out`` and their backward), the layer on ``scal3r_ttt_forward`` /
``_backward``.  This module only allocates outputs and passes pointers and
the current stream.

Parameter layouts: wqkv [3d, d] and wo [d, d] bfloat16 (y = x W^T); bqkv
[3d], w_eta [H, d], b_eta [H], alpha [d] float32; w0 as for :class:`TTT`.
"""
from __future__ import annotations

import torch

from . import (_check, scal3r_gcm_out, scal3r_gcm_out_backward, scal3r_gcm_qkv, scal3r_gcm_qkv_backward,
               scal3r_gcm_workspace_size)
from .layer import TTT, _ptr


class GCM:
    """One GCM module: the layer (a :class:`TTT` handle) and the steps around it."""

    def __init__(self, num_heads: int, head_dim: int, hidden_dim: int, base_lr: float = 0.1,
                 weight_norm: str = "row_w0", norm_eps: float = 1e-6):
        self.ttt = TTT(num_heads, head_dim, hidden_dim, dtype=torch.bfloat16, weight_norm=weight_norm,
                       norm_eps=norm_eps)
        self.H, self.D, self.F = num_heads, head_dim, hidden_dim
        self.d = num_heads * head_dim
        self.base_lr = float(base_lr)
        self._ws = None   # the calls' shared workspace (grown on demand)

    def _workspace(self, T, dev):
        n = max(256, scal3r_gcm_workspace_size(self.ttt.handle, T))
        if self._ws is None or self._ws.numel() < n or self._ws.device != dev:
            self._ws = torch.empty(n, dtype=torch.uint8, device=dev)
        return self._ws

    def forward(self, x, wqkv, bqkv, w_eta, b_eta, wo, alpha, w0, chunk_offsets, seq_chunk_ptr):
        """Returns (out [T, d] bf16, saved) for :meth:`backward`."""
        T, d, H, D = x.shape[0], self.d, self.H, self.D
        dev = x.device
        st = torch.cuda.current_stream(dev).cuda_stream
        ws = self._workspace(T, dev)
        q, k, v = (torch.empty((T, H, D), dtype=torch.bfloat16, device=dev) for _ in range(3))
        lr, qn, kn, sig = (torch.empty((T, H), dtype=torch.float32, device=dev) for _ in range(4))
        _check(scal3r_gcm_qkv(self.ttt.handle, _ptr(x), _ptr(wqkv), _ptr(bqkv), _ptr(w_eta), _ptr(b_eta),
                              self.base_lr, T, _ptr(q), _ptr(k), _ptr(v), _ptr(lr), _ptr(qn), _ptr(kn), _ptr(sig),
                              _ptr(ws), ws.numel(), st), "scal3r_gcm_qkv")
        o, ck, wn, _ = self.ttt.forward(q, k, v, lr, w0, chunk_offsets, seq_chunk_ptr)
        out = torch.empty((T, d), dtype=torch.bfloat16, device=dev)
        y = torch.empty((T, d), dtype=torch.bfloat16, device=dev)
        _check(scal3r_gcm_out(self.ttt.handle, _ptr(o), _ptr(wo), _ptr(x), _ptr(alpha), T, _ptr(out), _ptr(y), st),
               "scal3r_gcm_out")
        saved = {"x": x, "wqkv": wqkv, "w_eta": w_eta, "wo": wo, "alpha": alpha, "w0": w0, "q": q, "k": k, "v": v,
                 "lr": lr, "qn": qn, "kn": kn, "sig": sig, "o": o, "ck": ck, "wn": wn, "y": y,
                 "layout": (chunk_offsets, seq_chunk_ptr)}
        return out, saved

    def backward(self, saved, d_out):
        """Gradients of sum(d_out * out): (dx, dwqkv, dbqkv, dw_eta, db_eta, dwo, dalpha, dw0), float32."""
        s = saved
        x = s["x"]
        T, d, H, D = x.shape[0], self.d, self.H, self.D
        dev = x.device
        st = torch.cuda.current_stream(dev).cuda_stream
        ws = self._workspace(T, dev)
        d_out = d_out.contiguous()
        do = torch.empty((T, H, D), dtype=torch.bfloat16, device=dev)
        dwo = torch.empty((d, d), dtype=torch.float32, device=dev)
        dalpha = torch.empty(d, dtype=torch.float32, device=dev)
        _check(scal3r_gcm_out_backward(self.ttt.handle, _ptr(d_out), _ptr(s["o"]), _ptr(s["wo"]), _ptr(s["y"]),
                                       _ptr(s["alpha"]), T, _ptr(do), _ptr(dwo), _ptr(dalpha), _ptr(ws), ws.numel(),
                                       st), "scal3r_gcm_out_backward")
        off, ptr = s["layout"]
        dq, dk, dv, dlr, dw0 = self.ttt.backward(s["q"], s["k"], s["v"], s["lr"], s["w0"], off, ptr, do, s["ck"],
                                                 s["wn"])
        dx = torch.empty((T, d), dtype=torch.float32, device=dev)
        dwqkv = torch.empty((3 * d, d), dtype=torch.float32, device=dev)
        dbqkv = torch.empty(3 * d, dtype=torch.float32, device=dev)
        dw_eta = torch.empty((H, d), dtype=torch.float32, device=dev)
        db_eta = torch.empty(H, dtype=torch.float32, device=dev)
        _check(scal3r_gcm_qkv_backward(self.ttt.handle, _ptr(dq), _ptr(dk), _ptr(dv), _ptr(dlr), _ptr(s["q"]),
                                       _ptr(s["k"]), _ptr(s["qn"]), _ptr(s["kn"]), _ptr(s["sig"]), self.base_lr,
                                       _ptr(x), _ptr(s["wqkv"]), _ptr(s["w_eta"]), _ptr(d_out), T, _ptr(dx),
                                       _ptr(dwqkv), _ptr(dbqkv), _ptr(dw_eta), _ptr(db_eta), _ptr(ws), ws.numel(), st),
               "scal3r_gcm_qkv_backward")
        return dx, dwqkv, dbqkv, dw_eta, db_eta, dwo, dalpha, dw0
