"""torch-facing wrapper of the GCM module around the layer (scal3r_gcm.h).

The Global Context Memory module (Sec. 4.1, Eq. 5) maps a chunk's tokens
x [T, d] to ``out = alpha * (o Wo^T) + x`` where o is the test-time-training
layer applied to the projected, normalised q, k and the projected v, with a
predicted token-wise learning rate.  Every step runs in the library: the
projections and their gradients on ``scal3r_ttt_gemm``, the row steps on
``scal3r_gcm_*``, the layer on ``scal3r_ttt_forward`` / ``_backward``.  This
module only allocates outputs and passes pointers and the current stream.

Parameter layouts: wqkv [3d, d] and wo [d, d] bfloat16 (y = x W^T); bqkv
[3d], w_eta [H, d], b_eta [H], alpha [d] float32; w0 as for :class:`TTT`.
"""
from __future__ import annotations

import torch

from . import (_check, scal3r_gcm_gate, scal3r_gcm_gate_backward, scal3r_gcm_prep, scal3r_gcm_prep_backward,
               scal3r_gcm_workspace_size, scal3r_ttt_gemm, scal3r_ttt_gemm_workspace_size)
from .layer import TTT, _ptr

_PAD = 64   # the learning-rate predictor's rows, zero-padded for the GEMMs


class GCM:
    """One GCM module: the layer (a :class:`TTT` handle) and the steps around it."""

    def __init__(self, num_heads: int, head_dim: int, hidden_dim: int, base_lr: float = 0.1,
                 weight_norm: str = "row_w0", norm_eps: float = 1e-6):
        self.ttt = TTT(num_heads, head_dim, hidden_dim, dtype=torch.bfloat16, weight_norm=weight_norm,
                       norm_eps=norm_eps)
        self.H, self.D, self.F = num_heads, head_dim, hidden_dim
        self.d = num_heads * head_dim
        self.base_lr = float(base_lr)
        self._gws = None   # split-K partial planes of the weight-gradient GEMMs (grown on demand)

    def _gemm(self, a, lda, a_kmajor, b, ldb, b_kmajor, c, ldc, out_fp32, accumulate, M, N, K):
        st = torch.cuda.current_stream(c.device).cuda_stream
        n = scal3r_ttt_gemm_workspace_size(self.ttt.handle, M, N, K, out_fp32)
        if n and (self._gws is None or self._gws.numel() < n or self._gws.device != c.device):
            self._gws = torch.empty(n, dtype=torch.uint8, device=c.device)
        ws = self._gws if n else None
        _check(scal3r_ttt_gemm(self.ttt.handle, _ptr(a), lda, a_kmajor, _ptr(b), ldb, b_kmajor, _ptr(c), ldc,
                               out_fp32, accumulate, M, N, K, _ptr(ws), n, st), "scal3r_ttt_gemm")

    def forward(self, x, wqkv, bqkv, w_eta, b_eta, wo, alpha, w0, chunk_offsets, seq_chunk_ptr):
        """Returns (out [T, d] bf16, saved) for :meth:`backward`."""
        T, d, H, D = x.shape[0], self.d, self.H, self.D
        dev = x.device
        st = torch.cuda.current_stream(dev).cuda_stream
        raw = torch.empty((T, 3 * d), dtype=torch.float32, device=dev)
        self._gemm(x, d, 1, wqkv, d, 1, raw, 3 * d, 1, 0, T, 3 * d, d)
        q, k, v = (torch.empty((T, H, D), dtype=torch.bfloat16, device=dev) for _ in range(3))
        lr, qn, kn, sig = (torch.empty((T, H), dtype=torch.float32, device=dev) for _ in range(4))
        _check(scal3r_gcm_prep(self.ttt.handle, _ptr(raw), _ptr(bqkv), _ptr(x), _ptr(w_eta), _ptr(b_eta),
                               self.base_lr, T, _ptr(q), _ptr(k), _ptr(v), _ptr(lr), _ptr(qn), _ptr(kn), _ptr(sig),
                               st), "scal3r_gcm_prep")
        o, ck, wn, _ = self.ttt.forward(q, k, v, lr, w0, chunk_offsets, seq_chunk_ptr)
        y = torch.empty((T, d), dtype=torch.float32, device=dev)
        self._gemm(o, d, 1, wo, d, 1, y, d, 1, 0, T, d, d)
        out = torch.empty((T, d), dtype=torch.bfloat16, device=dev)
        _check(scal3r_gcm_gate(self.ttt.handle, _ptr(y), _ptr(x), _ptr(alpha), T, _ptr(out), st), "scal3r_gcm_gate")
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
        ws = torch.empty(max(256, scal3r_gcm_workspace_size(self.ttt.handle, T)), dtype=torch.uint8, device=dev)
        dy = torch.empty((T, d), dtype=torch.bfloat16, device=dev)
        dx = torch.empty((T, d), dtype=torch.float32, device=dev)
        dalpha = torch.empty(d, dtype=torch.float32, device=dev)
        _check(scal3r_gcm_gate_backward(self.ttt.handle, _ptr(d_out.contiguous()), _ptr(s["y"]), _ptr(s["alpha"]), T,
                                        _ptr(dy), _ptr(dx), _ptr(dalpha), _ptr(ws), ws.numel(), st),
               "scal3r_gcm_gate_backward")
        # y = o Wo^T:  d_o = dy Wo,  dWo = dy^T o
        do = torch.empty((T, H, D), dtype=torch.bfloat16, device=dev)
        self._gemm(dy, d, 1, s["wo"], d, 0, do, d, 0, 0, T, d, d)
        dwo = torch.empty((d, d), dtype=torch.float32, device=dev)
        self._gemm(dy, d, 0, s["o"], d, 0, dwo, d, 1, 0, d, d, T)
        off, ptr = s["layout"]
        dq, dk, dv, dlr, dw0 = self.ttt.backward(s["q"], s["k"], s["v"], s["lr"], s["w0"], off, ptr, do, s["ck"],
                                                 s["wn"])
        dqkv = torch.empty((T, 3 * d), dtype=torch.bfloat16, device=dev)
        dlogit = torch.empty((T, _PAD), dtype=torch.bfloat16, device=dev)
        dbqkv = torch.empty(3 * d, dtype=torch.float32, device=dev)
        db_eta = torch.empty(H, dtype=torch.float32, device=dev)
        _check(scal3r_gcm_prep_backward(self.ttt.handle, _ptr(dq), _ptr(dk), _ptr(dv), _ptr(dlr), _ptr(s["q"]),
                                        _ptr(s["k"]), _ptr(s["qn"]), _ptr(s["kn"]), _ptr(s["sig"]), self.base_lr, T,
                                        _ptr(dqkv), _ptr(dlogit), _ptr(dbqkv), _ptr(db_eta), _ptr(ws), ws.numel(),
                                        st), "scal3r_gcm_prep_backward")
        # [q | k | v] = x Wqkv^T + b:  dx += dqkv Wqkv,  dWqkv = dqkv^T x
        self._gemm(dqkv, 3 * d, 1, s["wqkv"], d, 0, dx, d, 1, 1, T, d, 3 * d)
        dwqkv = torch.empty((3 * d, d), dtype=torch.float32, device=dev)
        self._gemm(dqkv, 3 * d, 0, x, d, 0, dwqkv, d, 1, 0, 3 * d, d, T)
        # z = x w_eta^T + b_eta:  dx += dz w_eta,  dw_eta = dz^T x  (rows padded to 64)
        w_eta64 = torch.zeros((_PAD, d), dtype=torch.bfloat16, device=dev)
        w_eta64[:H] = s["w_eta"].to(torch.bfloat16)
        self._gemm(dlogit, _PAD, 1, w_eta64, d, 0, dx, d, 1, 1, T, d, _PAD)
        dw_eta64 = torch.empty((_PAD, d), dtype=torch.float32, device=dev)
        self._gemm(dlogit, _PAD, 0, x, d, 0, dw_eta64, d, 1, 0, _PAD, d, T)
        return dx, dwqkv, dbqkv, dw_eta64[:H].clone(), db_eta, dwo, dalpha, dw0
