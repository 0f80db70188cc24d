"""The allocation-free forward entry point against the ordinary one (GPU).

scal3r_ttt_forward_noalloc serves callers that may not call cudaMalloc (code
running while a stream is in global-mode graph capture, plugins whose host
framework owns all device memory, latency-critical paths that must not enter
the driver's allocator); its scratch is a fixed device array inside the
library.  Two calls in a row through the C ABI must both reproduce
scal3r_ttt_forward within the tolerance of the parity tests, and the array's
status word, read after each call, must be clean.  This file is collected
last so that a run stopping at the first failure has run every other test
already; it also passes alone in a fresh process.
"""
import threading

import numpy as np
import pytest

import ttt_synth as syn
from _util import rel_inf, to_np, upload

pytestmark = pytest.mark.gpu

CASES = [("bf16", "dot", False, False, 2e-2), ("fp32", "dot", False, False, 1e-5),
         ("fp32", "mse", False, False, 1e-5), ("fp32", "dot", True, False, 1e-5), ("bf16", "dot", True, True, 2e-2)]


def _setup(dtype_name, loss, per_seq_w0, per_matrix=False, seed=31):
    import torch
    import paper_2604_08542_gb300 as ttt
    dtype = torch.bfloat16 if dtype_name == "bf16" else torch.float32
    lay = syn.layout_from_lengths([[3000, 1500, 77], [1041], [2, 640]])
    H, D, F = 4, 64, 128
    T, S = lay.num_tokens, lay.num_seqs
    x = syn.make_inputs(T, H, D, F, seed=seed, dtype=dtype_name)
    if loss == "mse":
        x["lr"] = x["lr"] * 0.3   # keeps the squared-error recurrence in range
    if per_matrix:
        x["lr"] = syn.per_matrix_lr(seed + 2, T, H, lr_max=0.1)
    g = upload(x, dtype)
    if per_seq_w0:
        w = syn.make_inputs(1, S * H, D, F, seed=seed + 1)["w0"].reshape(S, H, 3 * F * D)
        g["w0"] = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    layer = ttt.TTT(H, D, F, dtype=dtype, loss=loss, lr_per_matrix=per_matrix)
    ref = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                        want_final=True)
    torch.cuda.synchronize()
    cfg = ttt.scal3r_ttt_config(H, D, F, ttt.SCAL3R_BF16 if dtype_name == "bf16" else ttt.SCAL3R_FP32,
                                ttt.SCAL3R_LOSS_MSE if loss == "mse" else ttt.SCAL3R_LOSS_DOT,
                                ttt.SCAL3R_NORM_ROW_W0, 1e-6, 0, lr_per_matrix=int(per_matrix))
    stride = H * 3 * F * D if per_seq_w0 else 0
    return lay, g, ref, cfg, stride, (H, D, F)


def _outputs(lay, shape, like):
    import torch
    H, D, F = shape
    C, S = lay.num_chunks, lay.num_seqs
    return (torch.full_like(like, float("nan")),
            torch.full((C, H, 3 * F * D), float("nan"), device="cuda"),
            torch.full((C, H, 2 * F + D), float("nan"), device="cuda"),
            torch.full((S, H, 3 * F * D), float("nan"), device="cuda"))


def _call(ttt, cfg, g, stride, lay, outs, stream):
    o, ck, wn, wf = outs
    return ttt.scal3r_ttt_forward_noalloc(cfg, g["q"].data_ptr(), g["k"].data_ptr(), g["v"].data_ptr(),
                                          g["lr"].data_ptr(), g["w0"].data_ptr(), stride, lay.chunk_offsets,
                                          lay.seq_chunk_ptr, o.data_ptr(), ck.data_ptr(), wn.data_ptr(),
                                          wf.data_ptr(), stream)


def _check(outs, ref, tol, tag):
    for name, a, b in zip(("o", "w_ckpt", "wnorm", "w_final"), outs, ref):
        err = rel_inf(to_np(a), to_np(b))
        assert np.isfinite(err) and err <= tol, (tag, name, err)


@pytest.mark.parametrize("dtype_name,loss,per_seq_w0,per_matrix,tol", CASES)
def test_noalloc_forward_matches_forward_twice(dtype_name, loss, per_seq_w0, per_matrix, tol):
    import torch
    import paper_2604_08542_gb300 as ttt
    lay, g, ref, cfg, stride, shape = _setup(dtype_name, loss, per_seq_w0, per_matrix)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        outs = _outputs(lay, shape, g["q"])
        rc = _call(ttt, cfg, g, stride, lay, outs, stream)
        assert rc == ttt.SCAL3R_OK, ttt.error_string(rc)
        assert ttt.scal3r_ttt_noalloc_status(stream) == ttt.SCAL3R_OK
        _check(outs, ref, tol, call)


def test_noalloc_forward_while_another_thread_captures_in_global_mode():
    # The first use named for this entry point: another thread holds a stream
    # in global-mode capture (where cudaMalloc would be refused) while the
    # forward runs on a stream of its own.  Neither the call nor the capture
    # may fail, and the outputs are the ordinary forward's.
    import torch
    import paper_2604_08542_gb300 as ttt
    lay, g, ref, cfg, stride, shape = _setup("bf16", "dot", False, seed=5)
    side, cap = torch.cuda.Stream(), torch.cuda.Stream()
    warm = _outputs(lay, shape, g["q"])
    assert _call(ttt, cfg, g, stride, lay, warm, side.cuda_stream) == ttt.SCAL3R_OK   # set-up outside capture
    assert ttt.scal3r_ttt_noalloc_status(side.cuda_stream) == ttt.SCAL3R_OK
    outs = _outputs(lay, shape, g["q"])
    x = torch.zeros(4096, device="cuda")
    torch.cuda.synchronize()
    started, release, errors = threading.Event(), threading.Event(), []

    def capture():
        graph = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(graph, stream=cap, capture_error_mode="global"):
                x.mul_(2.0)
                started.set()
                release.wait(60)
                x.add_(1.0)
            graph.replay()
            torch.cuda.synchronize()
        except Exception as e:   # reported below
            errors.append(e)
            started.set()

    t = threading.Thread(target=capture)
    t.start()
    try:
        assert started.wait(60)
        rc = _call(ttt, cfg, g, stride, lay, outs, side.cuda_stream)
    finally:
        release.set()
        t.join(120)
    assert not errors, errors
    assert rc == ttt.SCAL3R_OK, ttt.error_string(rc)
    assert ttt.scal3r_ttt_noalloc_status(side.cuda_stream) == ttt.SCAL3R_OK
    _check(outs, ref, 2e-2, "during capture")
    assert torch.all(x == 1.0)   # the captured graph ran once: 0 * 2 + 1


def test_noalloc_rejects_layouts_beyond_its_scratch():
    import torch
    import paper_2604_08542_gb300 as ttt
    # 400 sequences x 16 heads of master weights alone exceed the fixed scratch
    lay = syn.layout_from_lengths([[8]] * 400)
    cfg = ttt.scal3r_ttt_config(16, 64, 128, ttt.SCAL3R_BF16, ttt.SCAL3R_LOSS_DOT, ttt.SCAL3R_NORM_ROW_W0, 1e-6, 0)
    T = lay.num_tokens
    q = torch.zeros((T, 16, 64), dtype=torch.bfloat16, device="cuda")
    lr = torch.zeros((T, 16), dtype=torch.float32, device="cuda")
    w0 = torch.zeros((16, 3 * 128 * 64), dtype=torch.float32, device="cuda")
    o = torch.empty_like(q)
    rc = ttt.scal3r_ttt_forward_noalloc(cfg, q.data_ptr(), q.data_ptr(), q.data_ptr(), lr.data_ptr(),
                                        w0.data_ptr(), 0, lay.chunk_offsets, lay.seq_chunk_ptr, o.data_ptr(),
                                        None, None, None, torch.cuda.current_stream().cuda_stream)
    assert rc == ttt.SCAL3R_ERR_WORKSPACE
