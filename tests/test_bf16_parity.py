"""BF16 tensor-core path through the C ABI against the FP64 oracle (GPU).

The oracle runs on the same bfloat16-rounded q, k, v (exact in float64).
Bar: normwise relative error max|x - ref| / max|ref| <= 2e-2 for every
output (o, every checkpoint, w_final) and every gradient.  Results must be
bitwise reproducible run to run (fixed-order reductions).
"""
import numpy as np
import pytest

import oracle
import ttt_synth as syn
from _util import rel_inf, to_np, upload

pytestmark = pytest.mark.gpu

TOL = 2e-2


def _layer(H, **kw):
    import torch
    import paper_2604_08542_gb300 as ttt
    return ttt.TTT(H, 64, 128, dtype=torch.bfloat16, **kw)


def _forward(layer, g, lay):
    return layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                         want_final=True)


def _check(out, ref, tol=TOL, heads=None):
    o, ck, wn, wf = (to_np(t) for t in out)
    sel = slice(None) if heads is None else heads
    errs = {"o": rel_inf(o[:, sel], ref["o"]), "w_ckpt": rel_inf(ck[:, sel], ref["w_ckpt"]),
            "wnorm": rel_inf(wn[:, sel], ref["wnorm"]), "w_final": rel_inf(wf[:, sel], ref["w_final"])}
    bad = {n: e for n, e in errs.items() if not e <= tol}
    assert not bad, f"above {tol}: {bad}; all {errs}"
    return errs


@pytest.mark.parametrize("lengths", [
    [[300, 129, 77], [513], [1, 200, 64, 5]],      # ragged tails, 1-token chunk
    [[31], [33, 1], [127, 128, 129]],               # tile edges
    [[2000, 1041], [], [4096]],                     # empty sequence, multi-tile pieces
])
def test_bf16_ragged_matches_oracle(lengths):
    import torch
    lay = syn.layout_from_lengths(lengths)
    H = 3
    x = syn.make_inputs(lay.num_tokens, H, 64, 128, seed=21, dtype="bf16")
    g = upload(x, torch.bfloat16)
    out = _forward(_layer(H), g, lay)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, 64, 128, eps=1e-6)
    _check(out, ref)


def test_bf16_is_deterministic():
    import torch
    lay = syn.layout_from_lengths([[5000, 3000], [700]])
    H = 4
    x = syn.make_inputs(lay.num_tokens, H, 64, 128, seed=22, dtype="bf16")
    g = upload(x, torch.bfloat16)
    layer = _layer(H)
    a = [t.clone() for t in _forward(layer, g, lay)]
    b = _forward(layer, g, lay)
    for u, w in zip(a, b):
        assert torch.equal(u, w)


def test_bf16_vggt64_full_size_sampled_heads():
    """64 frames x 1041 tokens, 16 heads, chunk 16 frames, in the launch
    configuration the benchmark times; the oracle checks three whole heads."""
    import torch
    w = syn.workload("bf16_vggt64")
    lay = w.layout()
    x = syn.make_inputs(lay.num_tokens, 16, 64, 128, seed=0, dtype="bf16")
    g = upload(x, torch.bfloat16)
    out = _forward(_layer(16), g, lay)
    heads = [0, 7, 15]
    xs = {n: x[n][:, heads] for n in ("q", "k", "v", "lr")}
    ref = oracle.forward(xs["q"], xs["k"], xs["v"], xs["lr"], x["w0"][heads], lay, 64, 128, eps=1e-6)
    errs = _check(out, ref, heads=heads)
    print("vggt64 errors", errs)


def test_bf16_lr_zero_gives_plain_mlp():
    import torch
    lay = syn.layout_from_lengths([[400, 260]])
    x = syn.make_inputs(lay.num_tokens, 2, 64, 128, seed=23, dtype="bf16")
    x["lr"][:] = 0.0
    g = upload(x, torch.bfloat16)
    out = _forward(_layer(2), g, lay)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, 64, 128, eps=1e-6)
    _check(out, ref)
    # the weights do not move (up to fp32 rounding of the row rescale)
    wf = to_np(out[3])
    assert rel_inf(wf, ref["w_final"]) < 1e-6


def test_bf16_backward_matches_oracle():
    import torch
    lay = syn.layout_from_lengths([[700, 333], [129]])
    H = 2
    x = syn.make_inputs(lay.num_tokens, H, 64, 128, seed=24, dtype="bf16", with_grad_out=True)
    g = upload(x, torch.bfloat16)
    layer = _layer(H)
    o, ck, wn, _ = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], 64, 128, eps=1e-6)
    errs = {n: rel_inf(to_np(t), rb[n]) for n, t in zip(("dq", "dk", "dv", "dlr", "dw0"), grads)}
    bad = {n: e for n, e in errs.items() if not e <= TOL}
    assert not bad, f"above {TOL}: {bad}; all {errs}"


def test_bf16_backward_full_size_sampled_heads():
    """2 sequences x 32 frames x 1041 tokens, 16 heads, chunk 8 frames (the
    forward+backward workload); the oracle checks the gradients of two heads."""
    import torch
    w = syn.workload("bf16_fwdbwd_2x32")
    lay = w.layout()
    x = syn.make_inputs(lay.num_tokens, 16, 64, 128, seed=3, dtype="bf16", with_grad_out=True)
    g = upload(x, torch.bfloat16)
    layer = _layer(16)
    o, ck, wn, _ = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    heads = [2, 13]
    xs = {n: x[n][:, heads] for n in ("q", "k", "v", "lr", "d_o")}
    rb = oracle.backward(xs["q"], xs["k"], xs["v"], xs["lr"], x["w0"][heads], lay, xs["d_o"], 64, 128, eps=1e-6)
    errs = {}
    for n, t in zip(("dq", "dk", "dv", "dlr", "dw0"), grads):
        a = to_np(t)
        errs[n] = rel_inf(a[heads] if n == "dw0" else a[:, heads], rb[n])
    print("fwdbwd_2x32 gradient errors", errs)
    bad = {n: e for n, e in errs.items() if not e <= TOL}
    assert not bad, f"above {TOL}: {bad}; all {errs}"


@pytest.mark.parametrize("tail_fill", [0, 3])
def test_bf16_vggt64_backward_in_graph_mode_sampled_heads(tail_fill):
    """The benchmark's own step: 64 frames x 1041 tokens, 16 heads, 4 chunks of
    16,656 tokens, forward + backward replayed from the library's CUDA graphs
    (second call; the first captures).  The oracle checks every output and
    gradient of two whole heads.  With the tail fill on, the three steps that
    hold both roles launch extra pieces behind the first wave in each
    direction (the host planner tests show which)."""
    import torch
    w = syn.workload("bf16_vggt64")
    lay = w.layout()
    x = syn.make_inputs(lay.num_tokens, 16, 64, 128, seed=4, dtype="bf16", with_grad_out=True)
    g = upload(x, torch.bfloat16)
    layer = _layer(16)
    layer.set_schedule(tail_fill=tail_fill)
    layer.set_graph_mode(True)
    for _ in range(2):
        o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets,
                                      lay.seq_chunk_ptr, want_final=True)
        grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                               g["d_o"], ck, wn)
    torch.cuda.synchronize()
    assert layer.status() == 0
    heads = [5, 10]
    xs = {n: x[n][:, heads] for n in ("q", "k", "v", "lr", "d_o")}
    ref = oracle.forward(xs["q"], xs["k"], xs["v"], xs["lr"], x["w0"][heads], lay, 64, 128, eps=1e-6)
    errs = _check((o, ck, wn, wf), ref, heads=heads)
    rb = oracle.backward(xs["q"], xs["k"], xs["v"], xs["lr"], x["w0"][heads], lay, xs["d_o"], 64, 128, eps=1e-6)
    for n, t in zip(("dq", "dk", "dv", "dlr", "dw0"), grads):
        a = to_np(t)
        errs[n] = rel_inf(a[heads] if n == "dw0" else a[:, heads], rb[n])
    print("vggt64 graph-mode errors", errs)
    bad = {n: e for n, e in errs.items() if not e <= TOL}
    assert not bad, f"above {TOL}: {bad}; all {errs}"
