"""GB300 (sm_103a) test-time-training layer of Scal3R (arXiv 2604.08542).

Thin Python binding over the C-ABI library ``libscal3r_ttt.so`` (built from
``csrc/`` by ``build.py``).  Every step of the layer runs in the library's
CUDA kernels; this package only marshals arguments (torch tensors provide
device memory and the current stream).  There is no CPU fallback: if the
library is missing, every call raises.

Public names mirror the C ABI (``scal3r_ttt_init``, ``scal3r_ttt_forward``,
``scal3r_ttt_backward``, ...), plus a convenience class :class:`TTT` and the
``torch.autograd.Function`` :class:`TTTFunction`.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SCAL3R_TTT_LIBRARY selects another build of the same ABI (the
# bounds-checking variant, libscal3r_ttt_bounds.so).
LIB_PATH = os.environ.get("SCAL3R_TTT_LIBRARY") or os.path.join(_HERE, "libscal3r_ttt.so")

SCAL3R_OK = 0
SCAL3R_ERR_INVALID_ARG = 1
SCAL3R_ERR_UNSUPPORTED = 2
SCAL3R_ERR_MISALIGNED = 3
SCAL3R_ERR_CUDA = 4
SCAL3R_ERR_TIMEOUT = 5
SCAL3R_ERR_WORKSPACE = 6
SCAL3R_ERR_NO_DEVICE = 7
SCAL3R_ERR_NONFINITE = 8
SCAL3R_ERR_BOUNDS = 9

SCAL3R_FP32 = 0
SCAL3R_BF16 = 1
SCAL3R_LOSS_DOT = 0
SCAL3R_LOSS_MSE = 1
SCAL3R_NORM_ROW_W0 = 0
SCAL3R_NORM_NONE = 1
SCAL3R_NORM_UNIT = 2
SCAL3R_MODEL_SWIGLU = 0
SCAL3R_MODEL_LINEAR = 1

SCAL3R_KERNEL_FWD_SWEEP = 0
SCAL3R_KERNEL_FWD_UPDATE = 1
SCAL3R_KERNEL_BWD_SWEEP = 2
SCAL3R_KERNEL_BWD_UPDATE = 3
SCAL3R_KERNEL_OTHER = 4
KERNEL_KINDS = {0: "fwd_sweep", 1: "fwd_update", 2: "bwd_sweep", 3: "bwd_update", 4: "other"}

EXPORTED = ("scal3r_ttt_init", "scal3r_ttt_destroy", "scal3r_ttt_error_string", "scal3r_ttt_plan",
            "scal3r_ttt_workspace_size", "scal3r_ttt_forward", "scal3r_ttt_backward",
            "scal3r_ttt_set_schedule", "scal3r_ttt_get_schedule", "scal3r_ttt_set_graph_mode",
            "scal3r_ttt_autotune", "scal3r_ttt_profile_enable", "scal3r_ttt_profile_read",
            "scal3r_ttt_get_status", "scal3r_ttt_forward_noalloc", "scal3r_ttt_noalloc_status", "scal3r_ttt_partial_grad",
            "scal3r_ttt_apply_update", "scal3r_ttt_apply", "scal3r_ttt_ckpt_slots", "scal3r_ttt_gemm", "scal3r_ttt_gemm_workspace_size", "scal3r_ttt_gemm_timeout_test", "scal3r_ttt_set_finite_check", "scal3r_ttt_debug_bounds", "scal3r_gcm_workspace_size",
            "scal3r_gcm_qkv", "scal3r_gcm_out", "scal3r_gcm_out_backward", "scal3r_gcm_qkv_backward")


class scal3r_ttt_config(ctypes.Structure):
    _fields_ = [("num_heads", ctypes.c_int32), ("head_dim", ctypes.c_int32),
                ("hidden_dim", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("loss", ctypes.c_int32), ("weight_norm", ctypes.c_int32),
                ("norm_eps", ctypes.c_float), ("ckpt_every", ctypes.c_int32),
                ("lr_per_matrix", ctypes.c_int32), ("model", ctypes.c_int32),
                ("deterministic", ctypes.c_int32)]

    def __init__(self, *args, **kw):
        if len(args) < 11:
            kw.setdefault("deterministic", 1)
        super().__init__(*args, **kw)


class scal3r_ttt_schedule(ctypes.Structure):
    _fields_ = [("fwd_waves", ctypes.c_int32), ("bwd_waves", ctypes.c_int32),
                ("min_piece_tokens", ctypes.c_int32), ("fwd_key_cost", ctypes.c_float),
                ("bwd_key_cost", ctypes.c_float), ("tail_fill", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class Scal3rError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {error_string(status)} (status {status})")


_lib_handle = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the C-ABI library (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2604_08542_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    lib.scal3r_ttt_init.argtypes = [ctypes.POINTER(scal3r_ttt_config), ctypes.POINTER(vp)]
    lib.scal3r_ttt_init.restype = ctypes.c_int
    lib.scal3r_ttt_destroy.argtypes = [vp]
    lib.scal3r_ttt_destroy.restype = None
    lib.scal3r_ttt_error_string.argtypes = [ctypes.c_int]
    lib.scal3r_ttt_error_string.restype = ctypes.c_char_p
    lib.scal3r_ttt_plan.argtypes = [vp, vp, i32, vp, i32]
    lib.scal3r_ttt_plan.restype = ctypes.c_int
    lib.scal3r_ttt_workspace_size.argtypes = [vp, vp, i32, vp, i32, i32, ctypes.POINTER(sz)]
    lib.scal3r_ttt_workspace_size.restype = ctypes.c_int
    lib.scal3r_ttt_forward.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp, i32, vp, i32,
                                       vp, vp, vp, vp, vp, sz, vp]
    lib.scal3r_ttt_forward.restype = ctypes.c_int
    lib.scal3r_ttt_backward.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp, i32, vp, i32,
                                        vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.scal3r_ttt_backward.restype = ctypes.c_int
    lib.scal3r_ttt_set_schedule.argtypes = [vp, ctypes.POINTER(scal3r_ttt_schedule)]
    lib.scal3r_ttt_set_schedule.restype = ctypes.c_int
    lib.scal3r_ttt_get_schedule.argtypes = [vp, ctypes.POINTER(scal3r_ttt_schedule)]
    lib.scal3r_ttt_get_schedule.restype = ctypes.c_int
    lib.scal3r_ttt_set_graph_mode.argtypes = [vp, i32]
    lib.scal3r_ttt_set_graph_mode.restype = ctypes.c_int
    lib.scal3r_ttt_autotune.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp, i32, vp, i32, vp, vp, vp, vp, vp, vp, vp,
                                        vp, vp, i32, vp, ctypes.POINTER(scal3r_ttt_schedule),
                                        ctypes.POINTER(ctypes.c_float)]
    lib.scal3r_ttt_autotune.restype = ctypes.c_int
    lib.scal3r_ttt_forward_noalloc.argtypes = [ctypes.POINTER(scal3r_ttt_config), vp, vp, vp, vp, vp, i64, vp,
                                               i32, vp, i32, vp, vp, vp, vp, vp]
    lib.scal3r_ttt_forward_noalloc.restype = ctypes.c_int
    lib.scal3r_ttt_noalloc_status.argtypes = [vp]
    lib.scal3r_ttt_noalloc_status.restype = ctypes.c_int
    lib.scal3r_ttt_profile_enable.argtypes = [vp, i32]
    lib.scal3r_ttt_profile_enable.restype = ctypes.c_int
    lib.scal3r_ttt_profile_read.argtypes = [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.scal3r_ttt_profile_read.restype = ctypes.c_int
    lib.scal3r_ttt_debug_bounds.argtypes = [vp, i32, i64]
    lib.scal3r_ttt_debug_bounds.restype = ctypes.c_int
    lib.scal3r_ttt_get_status.argtypes = [vp, vp]
    lib.scal3r_ttt_get_status.restype = ctypes.c_int
    lib.scal3r_ttt_partial_grad.argtypes = [vp, vp, vp, vp, vp, i64, vp, i32, vp, i32, vp, vp, sz, vp]
    lib.scal3r_ttt_partial_grad.restype = ctypes.c_int
    lib.scal3r_ttt_apply_update.argtypes = [vp, vp, i64, vp, vp, i64, i32, vp, vp, vp]
    lib.scal3r_ttt_apply_update.restype = ctypes.c_int
    lib.scal3r_ttt_apply.argtypes = [vp, vp, vp, i64, vp, i32, vp, i32, vp, vp, sz, vp]
    lib.scal3r_ttt_apply.restype = ctypes.c_int
    f32 = ctypes.c_float
    lib.scal3r_ttt_ckpt_slots.argtypes = [vp, vp, i32, ctypes.POINTER(i64)]
    lib.scal3r_ttt_ckpt_slots.restype = ctypes.c_int
    lib.scal3r_ttt_gemm.argtypes = [vp, vp, i64, i32, vp, i64, i32, vp, i64, i32, i32, i64, i64, i64, vp,
                                    ctypes.c_size_t, vp]
    lib.scal3r_ttt_gemm.restype = ctypes.c_int
    lib.scal3r_ttt_set_finite_check.argtypes = [vp, i32]
    lib.scal3r_ttt_set_finite_check.restype = ctypes.c_int
    lib.scal3r_ttt_gemm_timeout_test.argtypes = [vp, i32]
    lib.scal3r_ttt_gemm_timeout_test.restype = ctypes.c_int
    lib.scal3r_ttt_gemm_workspace_size.argtypes = [vp, i64, i64, i64, i32, ctypes.POINTER(sz)]
    lib.scal3r_ttt_gemm_workspace_size.restype = ctypes.c_int
    lib.scal3r_gcm_workspace_size.argtypes = [vp, i64, ctypes.POINTER(sz)]
    lib.scal3r_gcm_workspace_size.restype = ctypes.c_int
    lib.scal3r_gcm_qkv.argtypes = [vp, vp, vp, vp, vp, vp, f32, i64, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.scal3r_gcm_qkv.restype = ctypes.c_int
    lib.scal3r_gcm_out.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp]
    lib.scal3r_gcm_out.restype = ctypes.c_int
    lib.scal3r_gcm_out_backward.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp, sz, vp]
    lib.scal3r_gcm_out_backward.restype = ctypes.c_int
    lib.scal3r_gcm_qkv_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, f32, vp, vp, vp, vp, i64, vp, vp,
                                            vp, vp, vp, vp, sz, vp]
    lib.scal3r_gcm_qkv_backward.restype = ctypes.c_int
    _lib_handle = lib
    return lib


def error_string(status: int) -> str:
    try:
        return load_library().scal3r_ttt_error_string(status).decode()
    except RuntimeError:
        return "library not loaded"


def _check(status: int, what: str) -> None:
    if status != SCAL3R_OK:
        raise Scal3rError(status, what)


# ---------------------------------------------------------------------------
# the C ABI, one wrapper per entry point (pointers are ints or None)
# ---------------------------------------------------------------------------

def scal3r_ttt_init(cfg: scal3r_ttt_config) -> int:
    h = ctypes.c_void_p()
    _check(load_library().scal3r_ttt_init(ctypes.byref(cfg), ctypes.byref(h)), "scal3r_ttt_init")
    return h.value


def scal3r_ttt_destroy(handle: int) -> None:
    load_library().scal3r_ttt_destroy(handle)


def scal3r_ttt_error_string(status: int) -> str:
    return error_string(status)


def _host_layout(chunk_offsets, seq_chunk_ptr):
    off = np.ascontiguousarray(chunk_offsets, dtype=np.int64)
    ptr = np.ascontiguousarray(seq_chunk_ptr, dtype=np.int32)
    return off, ptr


def scal3r_ttt_plan(handle: int, chunk_offsets, seq_chunk_ptr) -> None:
    off, ptr = _host_layout(chunk_offsets, seq_chunk_ptr)
    _check(load_library().scal3r_ttt_plan(handle, off.ctypes.data, len(off) - 1, ptr.ctypes.data, len(ptr) - 1),
           "scal3r_ttt_plan")


def scal3r_ttt_workspace_size(handle: int, chunk_offsets, seq_chunk_ptr, with_backward: bool) -> int:
    off, ptr = _host_layout(chunk_offsets, seq_chunk_ptr)
    n = ctypes.c_size_t()
    _check(load_library().scal3r_ttt_workspace_size(handle, off.ctypes.data, len(off) - 1, ptr.ctypes.data,
                                                    len(ptr) - 1, int(bool(with_backward)), ctypes.byref(n)),
           "scal3r_ttt_workspace_size")
    return n.value


def scal3r_ttt_forward(handle, q, k, v, lr, w0, w0_seq_stride, chunk_offsets, seq_chunk_ptr,
                       o, w_ckpt, wnorm, w_final, workspace, workspace_bytes, stream) -> int:
    """Raw entry point: every tensor argument is a device pointer (int) or None."""
    off, ptr = _host_layout(chunk_offsets, seq_chunk_ptr)
    return load_library().scal3r_ttt_forward(handle, q, k, v, lr, w0, w0_seq_stride, off.ctypes.data,
                                             len(off) - 1, ptr.ctypes.data, len(ptr) - 1, o, w_ckpt, wnorm,
                                             w_final, workspace, workspace_bytes, stream)


def scal3r_ttt_backward(handle, q, k, v, lr, w0, w0_seq_stride, chunk_offsets, seq_chunk_ptr, d_o,
                        w_ckpt, wnorm, dq, dk, dv, dlr, dw0, workspace, workspace_bytes, stream) -> int:
    off, ptr = _host_layout(chunk_offsets, seq_chunk_ptr)
    return load_library().scal3r_ttt_backward(handle, q, k, v, lr, w0, w0_seq_stride, off.ctypes.data,
                                              len(off) - 1, ptr.ctypes.data, len(ptr) - 1, d_o, w_ckpt, wnorm,
                                              dq, dk, dv, dlr, dw0, workspace, workspace_bytes, stream)


def scal3r_ttt_partial_grad(handle, k, v, lr, w, w_seq_stride, chunk_offsets, seq_chunk_ptr, grad,
                            workspace, workspace_bytes, stream) -> int:
    off, ptr = _host_layout(chunk_offsets, seq_chunk_ptr)
    return load_library().scal3r_ttt_partial_grad(handle, k, v, lr, w, w_seq_stride, off.ctypes.data, len(off) - 1,
                                                  ptr.ctypes.data, len(ptr) - 1, grad, workspace, workspace_bytes,
                                                  stream)


def scal3r_ttt_apply_update(handle, w, w_seq_stride, grad, w0, w0_seq_stride, num_seqs, w_out, wnorm,
                            stream) -> int:
    return load_library().scal3r_ttt_apply_update(handle, w, w_seq_stride, grad, w0, w0_seq_stride, num_seqs,
                                                  w_out, wnorm, stream)


def scal3r_ttt_apply(handle, q, w, w_seq_stride, chunk_offsets, seq_chunk_ptr, o, workspace, workspace_bytes,
                     stream) -> int:
    off, ptr = _host_layout(chunk_offsets, seq_chunk_ptr)
    return load_library().scal3r_ttt_apply(handle, q, w, w_seq_stride, off.ctypes.data, len(off) - 1,
                                           ptr.ctypes.data, len(ptr) - 1, o, workspace, workspace_bytes, stream)


def scal3r_ttt_set_schedule(handle: int, sch: scal3r_ttt_schedule) -> None:
    _check(load_library().scal3r_ttt_set_schedule(handle, ctypes.byref(sch)), "scal3r_ttt_set_schedule")


def scal3r_ttt_get_schedule(handle: int) -> scal3r_ttt_schedule:
    sch = scal3r_ttt_schedule()
    _check(load_library().scal3r_ttt_get_schedule(handle, ctypes.byref(sch)), "scal3r_ttt_get_schedule")
    return sch


def scal3r_ttt_set_graph_mode(handle: int, enable: bool) -> None:
    _check(load_library().scal3r_ttt_set_graph_mode(handle, int(bool(enable))), "scal3r_ttt_set_graph_mode")


def scal3r_ttt_autotune(handle, q, k, v, lr, w0, w0_seq_stride, chunk_offsets, seq_chunk_ptr, o, w_ckpt, wnorm,
                        d_o, dq, dk, dv, dlr, dw0, with_backward, stream):
    """Raw entry point; returns (schedule, best_ms)."""
    off, ptr = _host_layout(chunk_offsets, seq_chunk_ptr)
    best = scal3r_ttt_schedule()
    ms = ctypes.c_float()
    _check(load_library().scal3r_ttt_autotune(handle, q, k, v, lr, w0, w0_seq_stride, off.ctypes.data,
                                              len(off) - 1, ptr.ctypes.data, len(ptr) - 1, o, w_ckpt, wnorm, d_o,
                                              dq, dk, dv, dlr, dw0, int(bool(with_backward)), stream,
                                              ctypes.byref(best), ctypes.byref(ms)), "scal3r_ttt_autotune")
    return best, ms.value


def scal3r_ttt_forward_noalloc(cfg: scal3r_ttt_config, q, k, v, lr, w0, w0_seq_stride, chunk_offsets,
                               seq_chunk_ptr, o, w_ckpt, wnorm, w_final, stream) -> int:
    """Forward pass for callers that cannot allocate device memory: no handle,
    no workspace; its scratch is a fixed 32 MiB device array inside the
    library (see the C header).  Pointers are device pointers (int) or None."""
    off, ptr = _host_layout(chunk_offsets, seq_chunk_ptr)
    return load_library().scal3r_ttt_forward_noalloc(ctypes.byref(cfg), q, k, v, lr, w0, w0_seq_stride,
                                                     off.ctypes.data, len(off) - 1, ptr.ctypes.data, len(ptr) - 1,
                                                     o, w_ckpt, wnorm, w_final, stream)


def scal3r_ttt_noalloc_status(stream) -> int:
    """The status word of the allocation-free forward's array (synchronises
    `stream`; SCAL3R_OK or SCAL3R_ERR_TIMEOUT), cleared after the read."""
    return load_library().scal3r_ttt_noalloc_status(stream)


def scal3r_ttt_profile_enable(handle: int, enable: bool) -> None:
    _check(load_library().scal3r_ttt_profile_enable(handle, int(bool(enable))), "scal3r_ttt_profile_enable")


def scal3r_ttt_profile_read(handle: int, kind: int) -> dict:
    n = ctypes.c_int64()
    ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load_library().scal3r_ttt_profile_read(handle, kind, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                                  ctypes.byref(by)), "scal3r_ttt_profile_read")
    return {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}


def scal3r_ttt_get_status(handle: int, stream=None) -> int:
    return load_library().scal3r_ttt_get_status(handle, stream)


def scal3r_ttt_ckpt_slots(handle: int, seq_chunk_ptr) -> int:
    ptr = np.ascontiguousarray(seq_chunk_ptr, dtype=np.int32)
    n = ctypes.c_int64()
    _check(load_library().scal3r_ttt_ckpt_slots(handle, ptr.ctypes.data, len(ptr) - 1, ctypes.byref(n)),
           "scal3r_ttt_ckpt_slots")
    return n.value


# -- the GEMM and the row steps of the GCM module around the layer (raw entry
#    points: device pointers as ints, sizes as ints) --------------------------
def scal3r_ttt_gemm(handle, a, lda, a_kmajor, b, ldb, b_kmajor, c, ldc, out_fp32, accumulate, M, N, K,
                    workspace, workspace_bytes, stream) -> int:
    return load_library().scal3r_ttt_gemm(handle, a, lda, int(a_kmajor), b, ldb, int(b_kmajor), c, ldc,
                                          int(out_fp32), int(accumulate), M, N, K, workspace, workspace_bytes,
                                          stream)


def scal3r_ttt_debug_bounds(handle: int, tensor: int, shrink_bytes: int) -> int:
    """Bounds-checking build: register tensor number `tensor` shrink_bytes
    shorter on the following calls.  Returns the status: SCAL3R_OK in that
    build, SCAL3R_ERR_UNSUPPORTED in the ordinary one."""
    return int(load_library().scal3r_ttt_debug_bounds(handle, int(tensor), int(shrink_bytes)))


def scal3r_ttt_set_finite_check(handle: int, enable: bool) -> None:
    _check(load_library().scal3r_ttt_set_finite_check(handle, int(enable)), "scal3r_ttt_set_finite_check")


def scal3r_ttt_gemm_timeout_test(handle: int, enable: bool) -> None:
    _check(load_library().scal3r_ttt_gemm_timeout_test(handle, int(enable)), "scal3r_ttt_gemm_timeout_test")


def scal3r_ttt_gemm_workspace_size(handle: int, M: int, N: int, K: int, out_fp32: bool) -> int:
    n = ctypes.c_size_t()
    _check(load_library().scal3r_ttt_gemm_workspace_size(handle, M, N, K, int(out_fp32), ctypes.byref(n)),
           "scal3r_ttt_gemm_workspace_size")
    return n.value


def scal3r_gcm_workspace_size(handle: int, T: int) -> int:
    n = ctypes.c_size_t()
    _check(load_library().scal3r_gcm_workspace_size(handle, T, ctypes.byref(n)), "scal3r_gcm_workspace_size")
    return n.value


def scal3r_gcm_qkv(handle, x, wqkv, bqkv, w_eta, b_eta, base_lr, T, q, k, v, lr, qn, kn, sig, workspace,
                   workspace_bytes, stream) -> int:
    return load_library().scal3r_gcm_qkv(handle, x, wqkv, bqkv, w_eta, b_eta, float(base_lr), T, q, k, v, lr, qn, kn,
                                         sig, workspace, workspace_bytes, stream)


def scal3r_gcm_out(handle, o, wo, x, alpha, T, out, y, stream) -> int:
    return load_library().scal3r_gcm_out(handle, o, wo, x, alpha, T, out, y, stream)


def scal3r_gcm_out_backward(handle, d_out, o, wo, y, alpha, T, d_o, dwo, dalpha, workspace, workspace_bytes,
                            stream) -> int:
    return load_library().scal3r_gcm_out_backward(handle, d_out, o, wo, y, alpha, T, d_o, dwo, dalpha, workspace,
                                                  workspace_bytes, stream)


def scal3r_gcm_qkv_backward(handle, dq, dk, dv, dlr, q, k, qn, kn, sig, base_lr, x, wqkv, w_eta, d_out, T, dx, dwqkv,
                            dbqkv, dw_eta, db_eta, workspace, workspace_bytes, stream) -> int:
    return load_library().scal3r_gcm_qkv_backward(handle, dq, dk, dv, dlr, q, k, qn, kn, sig, float(base_lr), x, wqkv,
                                                  w_eta, d_out, T, dx, dwqkv, dbqkv, dw_eta, db_eta, workspace,
                                                  workspace_bytes, stream)


from .layer import TTT, TTTFunction  # noqa: E402,F401
