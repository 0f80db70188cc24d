"""The ragged-batch and long-sequence workloads at full size (GPU).

Every head of the batch runs; the oracle checks sampled (sequence, head)
chains whose inputs come from the counter-based generator (chains never
interact); properties that hold at any size cover the rest.
"""
import numpy as np
import pytest

import oracle
import ttt_synth as syn
from _util import device_inputs, rel_inf, seq_layout, to_np

pytestmark = pytest.mark.gpu

TOL = 2e-2


def test_ragged24_full_size_sampled_chains():
    """24 sequences with U{8..200} frames (about 2.6 M tokens), 16 heads,
    chunk 16 frames, forward: the longest and the shortest sequence on two
    heads each against the oracle."""
    import torch
    import paper_2604_08542_gb300 as ttt
    w = syn.workload("bf16_ragged24")
    lay = w.layout()
    frames = w.frames
    s_long = int(np.argmax(frames))
    s_short = int(np.argmin(frames))
    samples = [(s_long, 3), (s_long, 12), (s_short, 0), (s_short, 9)]
    g, host = device_inputs(lay, 16, 64, 128, seed=5, samples=samples)
    layer = ttt.TTT(16, 64, 128, dtype=torch.bfloat16)
    layer.set_graph_mode(True)
    o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                                  want_final=True)
    torch.cuda.synchronize()
    assert layer.status() == 0
    o_np = o.float().cpu().numpy()
    wf_np = wf.cpu().numpy()
    for (s, h), x in host.items():
        a, b = lay.seq_range(s)
        ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], seq_layout(lay, s), 64, 128, eps=1e-6)
        e_o = rel_inf(o_np[a:b, h], ref["o"][:, 0])
        e_w = rel_inf(wf_np[s, h], ref["w_final"][0, 0])
        assert e_o <= TOL and e_w <= TOL, ((s, h), e_o, e_w)


def test_long2000_streams_and_matches_oracle_on_one_head():
    """1 sequence x 2000 frames (2.08 M tokens), chunk 32 frames, 16 heads:
    the fast-weight state streams over 63 chunks.  One head against the
    oracle; and, for all heads, running the first 992 frames, then the rest
    from the carried weights, gives the one-pass result."""
    import torch
    import paper_2604_08542_gb300 as ttt
    w = syn.workload("bf16_long2000")
    lay = w.layout()
    g, host = device_inputs(lay, 16, 64, 128, seed=6, samples=[(0, 7)])
    layer = ttt.TTT(16, 64, 128, dtype=torch.bfloat16)
    o, _, _, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                                save_for_backward=False, want_final=True)
    torch.cuda.synchronize()
    x = host[(0, 7)]
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, 64, 128, eps=1e-6)
    assert rel_inf(o[:, 7].float().cpu().numpy(), ref["o"][:, 0]) <= TOL
    assert rel_inf(wf[0, 7].cpu().numpy(), ref["w_final"][0, 0]) <= TOL
    # streaming in two windows (the cut falls on a chunk boundary)
    cut = 31 * 32 * 1041
    la = syn.layout_from_frames([992], 1041, 32)
    lb = syn.layout_from_frames([1008], 1041, 32)
    sl = lambda t, a, b: t[a:b].contiguous()
    oa, _, _, wfa = layer.forward(*(sl(g[n], 0, cut) for n in ("q", "k", "v", "lr")), g["w0"], la.chunk_offsets,
                                  la.seq_chunk_ptr, save_for_backward=False, want_final=True)
    ob, _, _, wfb = layer.forward(*(sl(g[n], cut, lay.num_tokens) for n in ("q", "k", "v", "lr")), wfa.contiguous(),
                                  lb.chunk_offsets, lb.seq_chunk_ptr, save_for_backward=False, want_final=True)
    torch.cuda.synchronize()
    assert rel_inf(to_np(oa), to_np(o[:cut])) <= 1e-6
    assert rel_inf(to_np(ob), to_np(o[cut:])) <= TOL
    assert rel_inf(wfb.cpu().numpy(), wf.cpu().numpy()) <= TOL


def test_window256_forward_backward_sampled_head():
    """256-frame window (266,496 tokens, 8 chunks of 32 frames), forward and
    backward with checkpoints at every chunk; one head against the oracle."""
    import torch
    import paper_2604_08542_gb300 as ttt
    w = syn.workload("bf16_window256")
    lay = w.layout()
    g, host = device_inputs(lay, 16, 64, 128, seed=7, samples=[(0, 4)], with_grad_out=True)
    layer = ttt.TTT(16, 64, 128, dtype=torch.bfloat16)
    o, ck, wn, _ = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr, g["d_o"],
                           ck, wn)
    torch.cuda.synchronize()
    x = host[(0, 4)]
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, 64, 128, eps=1e-6)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], 64, 128, eps=1e-6)
    assert rel_inf(o[:, 4].float().cpu().numpy(), ref["o"][:, 0]) <= TOL
    for n, t in zip(("dq", "dk", "dv", "dlr", "dw0"), grads):
        a = t[4:5].cpu().numpy() if n == "dw0" else t[:, 4:5].float().cpu().numpy()
        assert rel_inf(a, rb[n]) <= TOL, n
