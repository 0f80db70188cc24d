"""The allocation-free forward entry point against the ordinary one (GPU).

scal3r_ttt_forward_noalloc serves callers that may not call cudaMalloc (code
running while a stream is in global-mode graph capture, plugins whose host
framework owns all device memory, latency-critical paths that must not enter
the driver's allocator); its scratch is a fixed device array inside the
library.  Two calls in a row through the C ABI must both reproduce
scal3r_ttt_forward within the tolerance of the parity tests.  This file is
collected last so that a run stopping at the first failure has run every
other test already; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import ttt_synth as syn
from _util import rel_inf, to_np, upload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype_name,tol", [("bf16", 2e-2), ("fp32", 1e-5)])
def test_noalloc_forward_matches_forward_twice(dtype_name, tol):
    import torch
    import paper_2604_08542_gb300 as ttt
    dtype = torch.bfloat16 if dtype_name == "bf16" else torch.float32
    lay = syn.layout_from_lengths([[3000, 1500, 77], [1041], [2, 640]])
    H, D, F = 4, 64, 128
    T, C, S = lay.num_tokens, lay.num_chunks, lay.num_seqs
    x = syn.make_inputs(T, H, D, F, seed=31, dtype=dtype_name)
    g = upload(x, dtype)
    layer = ttt.TTT(H, D, F, dtype=dtype)
    ref = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                        want_final=True)
    torch.cuda.synchronize()
    cfg = ttt.scal3r_ttt_config(H, D, F, ttt.SCAL3R_BF16 if dtype_name == "bf16" else ttt.SCAL3R_FP32,
                                ttt.SCAL3R_LOSS_DOT, ttt.SCAL3R_NORM_ROW_W0, 1e-6, 0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        o = torch.full_like(g["q"], float("nan"))
        ck = torch.full((C, H, 3 * F * D), float("nan"), device="cuda")
        wn = torch.full((C, H, 2 * F + D), float("nan"), device="cuda")
        wf = torch.full((S, H, 3 * F * D), float("nan"), device="cuda")
        rc = ttt.scal3r_ttt_forward_noalloc(cfg, g["q"].data_ptr(), g["k"].data_ptr(), g["v"].data_ptr(),
                                            g["lr"].data_ptr(), g["w0"].data_ptr(), 0, lay.chunk_offsets,
                                            lay.seq_chunk_ptr, o.data_ptr(), ck.data_ptr(), wn.data_ptr(),
                                            wf.data_ptr(), stream)
        assert rc == ttt.SCAL3R_OK, ttt.error_string(rc)
        torch.cuda.synchronize()
        for name, a, b in (("o", o, ref[0]), ("w_ckpt", ck, ref[1]), ("wnorm", wn, ref[2]),
                           ("w_final", wf, ref[3])):
            err = rel_inf(to_np(a), to_np(b))
            assert np.isfinite(err) and err <= tol, (call, name, err)


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
