"""Failure detection without a GPU fault (GPU).

Every wait in the library's kernels is bounded in time: when it runs out the
kernel raises an abort flag, every role leaves its loop, tensor memory is
freed and the handle's status word reads SCAL3R_ERR_TIMEOUT.  The test makes
one such wait run out on purpose (a barrier that no thread completes, after
all the kernel's copies and MMAs are done) and checks that the status is
reported, that the product was still stored, and that the context and the
handle keep working.
"""
import time

import pytest

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import torch
    import paper_2604_08542_gb300 as ttt
    M, N, K = 300, 512, 1024
    g = torch.Generator().manual_seed(7)
    A = torch.randn((M, K), generator=g).to(torch.bfloat16).cuda()
    B = torch.randn((N, K), generator=g).to(torch.bfloat16).cuda()
    ref = (A.double() @ B.double().T).cpu()
    layer = ttt.TTT(1, 256, 256, dtype=torch.bfloat16)
    h = layer.handle
    st = torch.cuda.current_stream().cuda_stream

    def gemm():
        c = torch.empty((M, N), dtype=torch.float32, device="cuda")
        rc = ttt.scal3r_ttt_gemm(h, A.data_ptr(), K, 1, B.data_ptr(), K, 1, c.data_ptr(), N, 1, 0, M, N, K, None, 0, st)
        assert rc == 0
        return c

    assert ttt.scal3r_ttt_get_status(h, st) == 0
    ttt.scal3r_ttt_gemm_timeout_test(h, True)
    t0 = time.perf_counter()
    c = gemm()
    status = ttt.scal3r_ttt_get_status(h, st)   # synchronises the stream
    waited = time.perf_counter() - t0
    assert status == ttt.SCAL3R_ERR_TIMEOUT
    assert waited >= 0.04                         # the 50 ms wait ran out
    scale = ref.abs().max().item()
    assert (c.cpu().double() - ref).abs().max().item() / scale < 5e-5   # stored before the wait
    # the status word was read and cleared; the context and handle still work
    ttt.scal3r_ttt_gemm_timeout_test(h, False)
    c2 = gemm()
    assert ttt.scal3r_ttt_get_status(h, st) == 0
    assert (c2.cpu().double() - ref).abs().max().item() / scale < 5e-5
    x = torch.ones(1024, device="cuda")
    assert float(x.sum().item()) == 1024.0


@pytest.mark.parametrize("dtype_name,D,F", [("bf16", 64, 128), ("fp32", 64, 128), ("bf16", 256, 512)])
def test_finite_check_reports_nonfinite_inputs(dtype_name, D, F):
    """With finite checking on, a NaN in q (forward) or an infinity in d_o
    (backward) sets SCAL3R_ERR_NONFINITE; clean calls and calls with the check
    off report 0."""
    import numpy as np
    import torch
    import paper_2604_08542_gb300 as ttt
    import ttt_synth as syn
    from _util import upload
    dtype = torch.bfloat16 if dtype_name == "bf16" else torch.float32
    H = 2
    lay = syn.layout_from_lengths([[200, 77], [130]])
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=5, dtype=dtype_name, with_grad_out=True)
    g = upload(x, dtype)
    layer = ttt.TTT(H, D, F, dtype=dtype)

    def run(q, d_o):
        o, ck, wn, _ = layer.forward(q, g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr)
        s_f = layer.status()
        layer.backward(q, g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr, d_o, ck, wn)
        return s_f, layer.status()

    layer.set_finite_check(True)
    assert run(g["q"], g["d_o"]) == (0, 0)
    q_bad = g["q"].clone()
    q_bad[17, 1, 3] = float("nan")
    s_f, _ = run(q_bad, g["d_o"])
    assert s_f == ttt.SCAL3R_ERR_NONFINITE
    d_bad = g["d_o"].clone()
    d_bad[150, 0, 5] = float("inf")
    assert run(g["q"], d_bad) == (0, ttt.SCAL3R_ERR_NONFINITE)
    layer.set_finite_check(False)
    assert run(g["q"], d_bad) == (0, 0)
    assert np.isfinite(float(g["q"].float().sum()))
