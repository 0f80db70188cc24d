"""torch-facing wrapper of the C ABI: tensors in, tensors out.

Only argument marshalling happens here (shape/dtype checks, output and
workspace allocation, the current CUDA stream); the computation is the
library's.  Layouts follow the C header: q, k, v, o [T, H, D]; lr [T, H]
float32 ([T, H, 3] with per-matrix rates: W1, W3, W2); w0 [H, 3*F*D] (shared) or [S, H, 3*F*D] (per sequence) float32,
packed W1 [F, D], W3 [F, D], W2 [D, F]; chunk_offsets [C+1] int64 and
seq_chunk_ptr [S+1] int32 on the host.
"""
from __future__ import annotations

import numpy as np
import torch

import hashlib
import json
import os

from . import (SCAL3R_BF16, SCAL3R_FP32, SCAL3R_LOSS_DOT, SCAL3R_LOSS_MSE, SCAL3R_MODEL_LINEAR,
               SCAL3R_MODEL_SWIGLU, SCAL3R_NORM_NONE,
               SCAL3R_NORM_ROW_W0, SCAL3R_NORM_UNIT, Scal3rError, _check, scal3r_ttt_autotune, scal3r_ttt_backward,
               scal3r_ttt_config, scal3r_ttt_destroy, scal3r_ttt_forward, scal3r_ttt_get_schedule,
               scal3r_ttt_get_status, scal3r_ttt_init, scal3r_ttt_plan, scal3r_ttt_schedule,
               scal3r_ttt_set_graph_mode, scal3r_ttt_set_schedule, scal3r_ttt_workspace_size,
               scal3r_ttt_partial_grad, scal3r_ttt_apply_update, scal3r_ttt_apply, scal3r_ttt_ckpt_slots,
               scal3r_ttt_set_finite_check)

NORMS = {"row_w0": SCAL3R_NORM_ROW_W0, "none": SCAL3R_NORM_NONE, "unit": SCAL3R_NORM_UNIT}
LOSSES = {"dot": SCAL3R_LOSS_DOT, "mse": SCAL3R_LOSS_MSE}
MODELS = {"swiglu": SCAL3R_MODEL_SWIGLU, "linear": SCAL3R_MODEL_LINEAR}


def _ptr(t):
    return None if t is None else t.data_ptr()


class TTT:
    """One configured layer (a C-ABI handle) on the current CUDA device."""

    def __init__(self, num_heads: int, head_dim: int = 64, hidden_dim: int = 128,
                 dtype: torch.dtype = torch.bfloat16, loss: str = "dot", weight_norm: str = "row_w0",
                 norm_eps: float = 1e-6, ckpt_every: int = 1, lr_per_matrix: bool = False,
                 model: str = "swiglu", deterministic: bool = True):
        if dtype not in (torch.bfloat16, torch.float32):
            raise ValueError("dtype must be torch.bfloat16 or torch.float32")
        self.H, self.D, self.F = num_heads, head_dim, hidden_dim
        self.dtype = dtype
        self.model = model
        self.cfg = scal3r_ttt_config(num_heads, head_dim, hidden_dim,
                                     SCAL3R_BF16 if dtype == torch.bfloat16 else SCAL3R_FP32,
                                     LOSSES[loss], NORMS[weight_norm], float(norm_eps), int(ckpt_every),
                                     int(bool(lr_per_matrix)), MODELS[model], int(bool(deterministic)))
        self.lr_shape = (num_heads, 3) if lr_per_matrix else (num_heads,)
        self.handle = scal3r_ttt_init(self.cfg)
        self._ws = None

    @property
    def P(self) -> int:
        return self.D * self.D if self.model == "linear" else 3 * self.F * self.D

    @property
    def R(self) -> int:
        return self.D if self.model == "linear" else 2 * self.F + self.D

    def close(self) -> None:
        if getattr(self, "handle", None):
            scal3r_ttt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers ---------------------------------------------------------
    def plan(self, chunk_offsets, seq_chunk_ptr) -> None:
        scal3r_ttt_plan(self.handle, chunk_offsets, seq_chunk_ptr)

    def workspace(self, chunk_offsets, seq_chunk_ptr, with_backward: bool, device) -> torch.Tensor:
        n = scal3r_ttt_workspace_size(self.handle, chunk_offsets, seq_chunk_ptr, with_backward)
        if self._ws is None or self._ws.numel() < n or self._ws.device != torch.device(device):
            self._ws = torch.empty(max(n, 256), dtype=torch.uint8, device=device)
        return self._ws

    def _check_lr(self, lr, T):
        if lr.dtype != torch.float32 or tuple(lr.shape) != (T, *self.lr_shape) or not lr.is_contiguous():
            raise ValueError(f"lr must be a contiguous float32 tensor of shape {[T, *self.lr_shape]}")

    def _check_tokens(self, name, t, T):
        if t.dtype != self.dtype or t.dim() != 3 or tuple(t.shape) != (T, self.H, self.D) or not t.is_cuda \
                or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {self.dtype} tensor of shape [T, H, D]")

    def _w0_stride(self, w0, S):
        if w0.dtype != torch.float32 or not w0.is_cuda or not w0.is_contiguous():
            raise ValueError("w0 must be a contiguous CUDA float32 tensor")
        if w0.dim() == 2 and tuple(w0.shape) == (self.H, self.P):
            return 0
        if w0.dim() == 3 and tuple(w0.shape) == (S, self.H, self.P):
            return self.H * self.P
        raise ValueError("w0 must be [H, P] or [S, H, P] (P = 3*F*D, or D*D for the linear model)")

    # -- passes ------------------------------------------------------------
    def forward(self, q, k, v, lr, w0, chunk_offsets, seq_chunk_ptr, *, save_for_backward=True,
                want_final=False, workspace=None, o=None, w_ckpt=None, wnorm=None):
        """Returns (o, w_ckpt, wnorm, w_final).  o, w_ckpt and wnorm may be
        given (preallocated, e.g. to keep a captured graph's pointers)."""
        off = np.ascontiguousarray(chunk_offsets, dtype=np.int64)
        ptr = np.ascontiguousarray(seq_chunk_ptr, dtype=np.int32)
        T, C, S = int(off[-1]), len(off) - 1, len(ptr) - 1
        for n, t in (("q", q), ("k", k), ("v", v)):
            self._check_tokens(n, t, T)
        self._check_lr(lr, T)
        stride = self._w0_stride(w0, S)
        dev = q.device
        o = torch.empty_like(q) if o is None else o
        slots = C if self.cfg.ckpt_every <= 1 else scal3r_ttt_ckpt_slots(self.handle, ptr)
        if save_for_backward:
            if w_ckpt is None:
                w_ckpt = torch.empty((slots, self.H, self.P), dtype=torch.float32, device=dev)
            if wnorm is None:
                wnorm = torch.empty((C, self.H, self.R), dtype=torch.float32, device=dev)
            if tuple(w_ckpt.shape) != (slots, self.H, self.P) or tuple(wnorm.shape) != (C, self.H, self.R):
                raise ValueError("w_ckpt / wnorm have the wrong shape for this layout")
        else:
            w_ckpt = wnorm = None
        w_final = torch.empty((S, self.H, self.P), dtype=torch.float32, device=dev) if want_final else None
        ws = self.workspace(off, ptr, False, dev) if workspace is None else workspace
        st = torch.cuda.current_stream(dev).cuda_stream
        rc = scal3r_ttt_forward(self.handle, _ptr(q), _ptr(k), _ptr(v), _ptr(lr), _ptr(w0), stride, off, ptr,
                                _ptr(o), _ptr(w_ckpt), _ptr(wnorm), _ptr(w_final), _ptr(ws), ws.numel(), st)
        _check(rc, "scal3r_ttt_forward")
        return o, w_ckpt, wnorm, w_final

    def backward(self, q, k, v, lr, w0, chunk_offsets, seq_chunk_ptr, d_o, w_ckpt, wnorm, *, workspace=None,
                 out=None):
        """Returns (dq, dk, dv, dlr, dw0); ``out`` may give them preallocated."""
        off = np.ascontiguousarray(chunk_offsets, dtype=np.int64)
        ptr = np.ascontiguousarray(seq_chunk_ptr, dtype=np.int32)
        T, S = int(off[-1]), len(ptr) - 1
        for n, t in (("q", q), ("k", k), ("v", v), ("d_o", d_o)):
            self._check_tokens(n, t, T)
        self._check_lr(lr, T)
        stride = self._w0_stride(w0, S)
        if out is None:
            dq, dk, dv, dlr, dw0 = (torch.empty_like(t) for t in (q, k, v, lr, w0))
        else:
            dq, dk, dv, dlr, dw0 = out
            for a, b in zip(out, (q, k, v, lr, w0)):
                if a.shape != b.shape or a.dtype != b.dtype or not a.is_contiguous():
                    raise ValueError("out tensors must match q, k, v, lr, w0")
        ws = self.workspace(off, ptr, True, q.device) if workspace is None else workspace
        st = torch.cuda.current_stream(q.device).cuda_stream
        rc = scal3r_ttt_backward(self.handle, _ptr(q), _ptr(k), _ptr(v), _ptr(lr), _ptr(w0), stride, off, ptr,
                                 _ptr(d_o), _ptr(w_ckpt), _ptr(wnorm), _ptr(dq), _ptr(dk), _ptr(dv), _ptr(dlr),
                                 _ptr(dw0), _ptr(ws), ws.numel(), st)
        _check(rc, "scal3r_ttt_backward")
        return dq, dk, dv, dlr, dw0

    # -- Global Context Synchronisation (Eq. 10): a chunk step in local parts ----
    def partial_grad(self, k, v, lr, w, chunk_offsets, seq_chunk_ptr, *, workspace=None):
        """The inner gradient of Eq. 8 over each sequence's (single) chunk at
        the weights w ([H, P] or [S, H, P]); returns grad [S, H, P] float32."""
        off = np.ascontiguousarray(chunk_offsets, dtype=np.int64)
        ptr = np.ascontiguousarray(seq_chunk_ptr, dtype=np.int32)
        T, S = int(off[-1]), len(ptr) - 1
        for n, t in (("k", k), ("v", v)):
            self._check_tokens(n, t, T)
        self._check_lr(lr, T)
        stride = self._w0_stride(w, S)
        grad = torch.empty((S, self.H, self.P), dtype=torch.float32, device=k.device)
        ws = self.workspace(off, ptr, False, k.device) if workspace is None else workspace
        st = torch.cuda.current_stream(k.device).cuda_stream
        _check(scal3r_ttt_partial_grad(self.handle, _ptr(k), _ptr(v), _ptr(lr), _ptr(w), stride, off, ptr,
                                       _ptr(grad), _ptr(ws), ws.numel(), st), "scal3r_ttt_partial_grad")
        return grad

    def apply_update(self, w, grad, w0):
        """W - grad with the rows rescaled (targets from w0); returns
        (w_next [S, H, P], wnorm [S, H, 2F+D])."""
        if grad.dtype != torch.float32 or grad.dim() != 3 or grad.shape[1:] != (self.H, self.P) \
                or not grad.is_contiguous():
            raise ValueError("grad must be a contiguous float32 tensor [S, H, 3*F*D]")
        S = grad.shape[0]
        ws, w0s = self._w0_stride(w, S), self._w0_stride(w0, S)
        w_out = torch.empty_like(grad)
        wnorm = torch.empty((S, self.H, self.R), dtype=torch.float32, device=grad.device)
        st = torch.cuda.current_stream(grad.device).cuda_stream
        _check(scal3r_ttt_apply_update(self.handle, _ptr(w), ws, _ptr(grad), _ptr(w0), w0s, S, _ptr(w_out),
                                       _ptr(wnorm), st), "scal3r_ttt_apply_update")
        return w_out, wnorm

    def apply(self, q, w, chunk_offsets, seq_chunk_ptr, *, workspace=None):
        """o = f_W(q) for each sequence's (single) chunk with its weights w."""
        off = np.ascontiguousarray(chunk_offsets, dtype=np.int64)
        ptr = np.ascontiguousarray(seq_chunk_ptr, dtype=np.int32)
        T, S = int(off[-1]), len(ptr) - 1
        self._check_tokens("q", q, T)
        stride = self._w0_stride(w, S)
        o = torch.empty_like(q)
        ws = self.workspace(off, ptr, False, q.device) if workspace is None else workspace
        st = torch.cuda.current_stream(q.device).cuda_stream
        _check(scal3r_ttt_apply(self.handle, _ptr(q), _ptr(w), stride, off, ptr, _ptr(o), _ptr(ws), ws.numel(), st),
               "scal3r_ttt_apply")
        return o

    def status(self) -> int:
        return scal3r_ttt_get_status(self.handle, torch.cuda.current_stream().cuda_stream)

    # -- graphs and schedules ---------------------------------------------
    def set_finite_check(self, enable: bool = True) -> None:
        """Scan each call's inputs and outputs for NaN / infinity afterwards;
        a hit shows as SCAL3R_ERR_NONFINITE from status()."""
        scal3r_ttt_set_finite_check(self.handle, enable)

    def set_graph_mode(self, enable: bool = True) -> None:
        """Record forward/backward launch sequences into CUDA graphs and replay them."""
        scal3r_ttt_set_graph_mode(self.handle, enable)

    def schedule(self) -> dict:
        return scal3r_ttt_get_schedule(self.handle).as_dict()

    def set_schedule(self, **kw) -> None:
        sch = scal3r_ttt_get_schedule(self.handle)
        for k, v in kw.items():
            setattr(sch, k, v)
        scal3r_ttt_set_schedule(self.handle, sch)

    def layout_key(self, chunk_offsets, seq_chunk_ptr) -> str:
        off = np.ascontiguousarray(chunk_offsets, dtype=np.int64)
        ptr = np.ascontiguousarray(seq_chunk_ptr, dtype=np.int32)
        h = hashlib.sha1(off.tobytes() + b"|" + ptr.tobytes())
        h.update(f"{self.H},{self.D},{self.F},{self.dtype}".encode())
        return h.hexdigest()[:16]

    def autotune(self, q, k, v, lr, w0, chunk_offsets, seq_chunk_ptr, d_o=None, cache_path=None) -> dict:
        """Pick the piece schedule for this layout by timing candidates (the
        library's tuner); forward only unless d_o is given.  With cache_path,
        results are kept in a JSON file keyed by the layout."""
        key = self.layout_key(chunk_offsets, seq_chunk_ptr) + ("b" if d_o is not None else "f")
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
            if key in cache:
                self.set_schedule(**cache[key]["schedule"])
                return cache[key]
        off = np.ascontiguousarray(chunk_offsets, dtype=np.int64)
        ptr = np.ascontiguousarray(seq_chunk_ptr, dtype=np.int32)
        T, C, S = int(off[-1]), len(off) - 1, len(ptr) - 1
        stride = self._w0_stride(w0, S)
        dev = q.device
        o = torch.empty_like(q)
        ck = torch.empty((C, self.H, self.P), dtype=torch.float32, device=dev)
        wn = torch.empty((C, self.H, self.R), dtype=torch.float32, device=dev)
        grads = [None] * 6
        if d_o is not None:
            grads = [d_o, torch.empty_like(q), torch.empty_like(k), torch.empty_like(v), torch.empty_like(lr),
                     torch.empty_like(w0)]
        st = torch.cuda.current_stream(dev).cuda_stream
        best, ms = scal3r_ttt_autotune(self.handle, _ptr(q), _ptr(k), _ptr(v), _ptr(lr), _ptr(w0), stride, off, ptr,
                                       _ptr(o), _ptr(ck), _ptr(wn), *(_ptr(g) for g in grads), d_o is not None, st)
        res = {"schedule": best.as_dict(), "ms": ms}
        if cache_path:
            cache = {}
            if os.path.exists(cache_path):
                with open(cache_path) as f:
                    cache = json.load(f)
            cache[key] = res
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        return res


class TTTFunction(torch.autograd.Function):
    """o = TTT(q, k, v, lr, w0) with the library's hand-written backward.

    ``TTTFunction.apply(q, k, v, lr, w0, layer, chunk_offsets, seq_chunk_ptr)``;
    the fast weights are checkpointed at every chunk boundary in the forward
    and the chunks in between are recomputed in the backward.
    """

    @staticmethod
    def forward(ctx, q, k, v, lr, w0, layer: TTT, chunk_offsets, seq_chunk_ptr):
        o, w_ckpt, wnorm, _ = layer.forward(q, k, v, lr, w0, chunk_offsets, seq_chunk_ptr, save_for_backward=True)
        ctx.layer = layer
        ctx.layout = (np.asarray(chunk_offsets, dtype=np.int64).copy(), np.asarray(seq_chunk_ptr, dtype=np.int32).copy())
        ctx.save_for_backward(q, k, v, lr, w0, w_ckpt, wnorm)
        return o

    @staticmethod
    def backward(ctx, d_o):
        q, k, v, lr, w0, w_ckpt, wnorm = ctx.saved_tensors
        off, ptr = ctx.layout
        d_o = d_o.contiguous()
        dq, dk, dv, dlr, dw0 = ctx.layer.backward(q, k, v, lr, w0, off, ptr, d_o, w_ckpt, wnorm)
        return dq, dk, dv, dlr, dw0, None, None, None


__all__ = ["TTT", "TTTFunction", "Scal3rError"]
