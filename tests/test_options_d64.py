"""The layer's options at head_dim 64, hidden 128 (GPU, through the C ABI):
per-matrix learning rates (reading A4b: matrix j's gradient of Eq. 8
weighted by its own rate), on the float32 path and the fused bfloat16 path,
forward and backward, against the FP64 oracle.

Bars: 1e-5 normwise for float32, 2e-2 for bfloat16 (the oracle run on the
same bfloat16-rounded inputs).
"""
import numpy as np
import pytest

import oracle
import ttt_synth as syn
from _util import rel_inf, to_np, upload

pytestmark = pytest.mark.gpu

D, F = 64, 128
TOLS = {"fp32": 1e-5, "bf16": 2e-2}


def _run(dtype_name, lay, H, seed, loss="dot", lr=None, norm="row_w0", heads=None, **cfg):
    """Forward + backward through the library and the oracle; returns the
    normwise errors of every output and gradient (on `heads` only if given)."""
    import torch
    import paper_2604_08542_gb300 as ttt
    dtype = torch.bfloat16 if dtype_name == "bf16" else torch.float32
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=seed, dtype=dtype_name, with_grad_out=True)
    if lr is not None:
        x["lr"] = lr
    g = upload(x, dtype)
    layer = ttt.TTT(H, D, F, dtype=dtype, loss=loss, weight_norm=norm, **cfg)
    o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                                  want_final=True)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    torch.cuda.synchronize()
    assert layer.status() == 0
    hs = list(range(H)) if heads is None else heads
    xs = {n: x[n][:, hs] for n in ("q", "k", "v", "lr", "d_o")}
    ref = oracle.forward(xs["q"], xs["k"], xs["v"], xs["lr"], x["w0"][hs], lay, D, F, loss=loss, norm=norm,
                         eps=1e-6)
    rb = oracle.backward(xs["q"], xs["k"], xs["v"], xs["lr"], x["w0"][hs], lay, xs["d_o"], D, F, loss=loss,
                         norm=norm, eps=1e-6)
    errs = {"o": rel_inf(to_np(o)[:, hs], ref["o"]), "w_final": rel_inf(to_np(wf)[:, hs], ref["w_final"])}
    if layer.cfg.ckpt_every <= 1:
        errs["w_ckpt"] = rel_inf(to_np(ck)[:, hs], ref["w_ckpt"])
    errs["wnorm"] = rel_inf(to_np(wn)[:, hs], ref["wnorm"])
    for n, t in zip(("dq", "dk", "dv", "dlr", "dw0"), grads):
        a = to_np(t)
        errs[n] = rel_inf(a[hs] if n == "dw0" else a[:, hs], rb[n])
    return errs, (o, ck, wn, grads)


def _assert(errs, tol, tag=""):
    bad = {n: e for n, e in errs.items() if not e <= tol}
    assert not bad, f"{tag} above {tol}: {bad}; all {errs}"


# ---- per-matrix learning rates ----------------------------------------------

@pytest.mark.parametrize("dtype_name,loss", [("fp32", "dot"), ("fp32", "mse"), ("bf16", "dot")])
def test_per_matrix_rates_match_oracle(dtype_name, loss):
    """lr [T, H, 3] (W1, W3, W2): forward outputs and every gradient, dlr
    included in the same layout; two heads, ragged chunks with tile edges."""
    lay = syn.layout_from_lengths([[300, 129], [77, 257]])
    H = 2
    lr = syn.per_matrix_lr(81, lay.num_tokens, H, lr_max=0.1)
    errs, _ = _run(dtype_name, lay, H, seed=80, loss=loss, lr=lr, lr_per_matrix=True)
    _assert(errs, TOLS[dtype_name], f"{dtype_name}/{loss}")


@pytest.mark.parametrize("dtype_name", ["fp32", "bf16"])
def test_per_matrix_rates_with_one_matrix_frozen(dtype_name):
    """W3's rates all zero: the oracle keeps W3's update at zero while W1 and
    W2 move, and the library matches it (which rate scales which matrix)."""
    lay = syn.layout_from_lengths([[200, 129]])
    H = 2
    lr = syn.per_matrix_lr(83, lay.num_tokens, H, lr_max=0.1)
    lr[:, :, 1] = 0.0
    errs, _ = _run(dtype_name, lay, H, seed=82, lr=lr, norm="none", lr_per_matrix=True)
    _assert(errs, TOLS[dtype_name])


@pytest.mark.parametrize("dtype_name", ["fp32", "bf16"])
def test_equal_per_matrix_rates_are_the_one_rate_layer(dtype_name):
    """Three equal rates per token reproduce the one-rate layer, with dlr
    split three ways (the bfloat16 forward bitwise: its gradient pieces scale
    the same products by the same rate; the float32 one applies the rate
    after the W2 product instead of before, so up to rounding)."""
    import torch
    import paper_2604_08542_gb300 as ttt
    dtype = torch.bfloat16 if dtype_name == "bf16" else torch.float32
    lay = syn.layout_from_lengths([[260, 200], [128]])
    H = 2
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=84, dtype=dtype_name, with_grad_out=True)
    g = upload(x, dtype)
    res = []
    for per in (False, True):
        layer = ttt.TTT(H, D, F, dtype=dtype, lr_per_matrix=per)
        lr = g["lr"][..., None].expand(-1, -1, 3).contiguous() if per else g["lr"]
        o, ck, wn, _ = layer.forward(g["q"], g["k"], g["v"], lr, g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr)
        grads = layer.backward(g["q"], g["k"], g["v"], lr, g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                               g["d_o"], ck, wn)
        torch.cuda.synchronize()
        assert layer.status() == 0
        res.append((o, ck, grads))
    (o1, ck1, g1), (o3, ck3, g3) = res
    if dtype_name == "bf16":
        assert torch.equal(o1, o3) and torch.equal(ck1, ck3)
    else:
        assert rel_inf(to_np(o3), to_np(o1)) < 1e-6 and rel_inf(to_np(ck3), to_np(ck1)) < 1e-6
    tol = 1e-5 if dtype_name == "fp32" else 5e-3
    for n, a, b in zip(("dq", "dk", "dv", "dw0"), (g1[0], g1[1], g1[2], g1[4]), (g3[0], g3[1], g3[2], g3[4])):
        assert rel_inf(to_np(b), to_np(a)) < tol, n
    assert rel_inf(to_np(g3[3]).sum(-1), to_np(g1[3])) < tol


def test_per_matrix_rates_full_size_sampled_heads():
    """The forward+backward workload (2 sequences x 32 frames x 1041 tokens,
    16 heads, chunk 8 frames) with a rate per matrix; the oracle checks two
    whole heads."""
    w = syn.workload("bf16_fwdbwd_2x32")
    lay = w.layout()
    lr = syn.per_matrix_lr(86, lay.num_tokens, 16, lr_max=0.1)
    errs, _ = _run("bf16", lay, 16, seed=85, lr=lr, heads=[4, 11], lr_per_matrix=True)
    print("per-matrix fwdbwd_2x32 errors", errs)
    _assert(errs, TOLS["bf16"])


# ---- sparse checkpoints -----------------------------------------------------

def _fwd_bwd(dtype_name, lay, H, seed, ckpt_every):
    import torch
    import paper_2604_08542_gb300 as ttt
    dtype = torch.bfloat16 if dtype_name == "bf16" else torch.float32
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=seed, dtype=dtype_name, with_grad_out=True)
    g = upload(x, dtype)
    layer = ttt.TTT(H, D, F, dtype=dtype, ckpt_every=ckpt_every)
    o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                                  want_final=True)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    torch.cuda.synchronize()
    assert layer.status() == 0
    return x, (o, ck, wn, wf), grads


def _slots(lay, n):
    """(global chunk index, slot) of every stored checkpoint with ckpt_every = n."""
    out, slot = [], 0
    for s in range(lay.num_seqs):
        c0, c1 = int(lay.seq_chunk_ptr[s]), int(lay.seq_chunk_ptr[s + 1])
        for i in range(c1 - c0):
            if (i + 1) % n == 0:
                out.append((c0 + i, slot))
                slot += 1
    return out


@pytest.mark.parametrize("dtype_name,n", [("fp32", 2), ("fp32", 3), ("bf16", 2), ("bf16", 4)])
def test_sparse_checkpoints_reproduce_dense_bitwise(dtype_name, n):
    """ckpt_every = n stores the weights after local chunks n-1, 2n-1, ...;
    the backward recomputes the others with the forward's own gradient
    pieces and updates, so every output and gradient equals the run with a
    checkpoint per chunk bit for bit.  Sequences of 5, 2, 3 and 1 chunks:
    segments that end at a sequence's last chunk, sequences shorter than a
    segment, a last step that is not a multiple of n."""
    import torch
    lay = syn.layout_from_lengths([[300, 129, 77, 200, 50], [130, 257], [100, 100, 100], [64]])
    H = 2
    x, (o1, ck1, wn1, wf1), g1 = _fwd_bwd(dtype_name, lay, H, 90, 1)
    _, (o2, ck2, wn2, wf2), g2 = _fwd_bwd(dtype_name, lay, H, 90, n)
    assert torch.equal(o1, o2) and torch.equal(wn1, wn2) and torch.equal(wf1, wf2)
    pairs = _slots(lay, n)
    assert ck2.shape[0] == len(pairs)
    for c, slot in pairs:
        assert torch.equal(ck2[slot], ck1[c])
    for name, a, b in zip(("dq", "dk", "dv", "dlr", "dw0"), g1, g2):
        assert torch.equal(a, b), name


def test_sparse_checkpoints_full_size_fwdbwd():
    """The forward+backward workload (2 sequences x 32 frames x 1041 tokens,
    16 heads, chunk 8 frames: 4 chunks a sequence) with a checkpoint every
    third chunk: bitwise the dense run, and the oracle on two whole heads."""
    import torch
    w = syn.workload("bf16_fwdbwd_2x32")
    lay = w.layout()
    x, (o1, _, _, _), g1 = _fwd_bwd("bf16", lay, 16, 91, 1)
    _, (o3, ck3, _, _), g3 = _fwd_bwd("bf16", lay, 16, 91, 3)
    assert ck3.shape[0] == len(_slots(lay, 3))
    assert torch.equal(o1, o3)
    for a, b in zip(g1, g3):
        assert torch.equal(a, b)
    hs = [2, 13]
    xs = {n: x[n][:, hs] for n in ("q", "k", "v", "lr", "d_o")}
    rb = oracle.backward(xs["q"], xs["k"], xs["v"], xs["lr"], x["w0"][hs], lay, xs["d_o"], D, F, eps=1e-6)
    for name, t in zip(("dq", "dk", "dv", "dlr", "dw0"), g3):
        a = to_np(t)
        assert rel_inf(a[hs] if name == "dw0" else a[:, hs], rb[name]) <= TOLS["bf16"], name


# ---- squared-error loss on the fused bfloat16 path --------------------------

@pytest.mark.parametrize("norm", ["row_w0", "none"])
def test_mse_bf16_matches_oracle(norm):
    """Eq. 9 with the squared-error loss (reading A10) on the fused kernels:
    the residual pieces write r = v - f_W(k), the gradient pieces take r as
    their values, and the backward adds the apply VJP over the keys with the
    upstream gradient -dr.  Forward outputs and every gradient against the
    oracle, ragged chunks with tile edges, two heads."""
    lay = syn.layout_from_lengths([[300, 129], [77, 257, 1]])
    x = syn.make_inputs(lay.num_tokens, 2, D, F, seed=92, dtype="bf16")
    errs, _ = _run("bf16", lay, 2, seed=92, loss="mse", lr=x["lr"] * 0.3, norm=norm)
    _assert(errs, TOLS["bf16"], f"mse/{norm}")


def test_mse_bf16_with_per_matrix_rates():
    lay = syn.layout_from_lengths([[200, 129], [64]])
    lr = syn.per_matrix_lr(94, lay.num_tokens, 2, lr_max=0.03)
    errs, _ = _run("bf16", lay, 2, seed=93, loss="mse", lr=lr, lr_per_matrix=True)
    _assert(errs, TOLS["bf16"])


def test_mse_bf16_sparse_checkpoints_reproduce_dense_bitwise():
    import torch
    import paper_2604_08542_gb300 as ttt
    lay = syn.layout_from_lengths([[300, 129, 77, 200, 50], [130, 257]])
    x = syn.make_inputs(lay.num_tokens, 2, D, F, seed=95, dtype="bf16", with_grad_out=True)
    x["lr"] = x["lr"] * 0.3
    g = upload(x, torch.bfloat16)
    res = []
    for n in (1, 2):
        layer = ttt.TTT(2, D, F, dtype=torch.bfloat16, loss="mse", ckpt_every=n)
        o, ck, wn, _ = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr)
        grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                               g["d_o"], ck, wn)
        torch.cuda.synchronize()
        assert layer.status() == 0
        res.append([o] + list(grads))
    for a, b in zip(*res):
        assert torch.equal(a, b)


def test_mse_bf16_full_size_sampled_heads():
    """The forward+backward workload (2 x 32 frames x 1041 tokens, 16 heads)
    with the squared-error loss; the oracle checks two whole heads."""
    w = syn.workload("bf16_fwdbwd_2x32")
    lay = w.layout()
    x = syn.make_inputs(lay.num_tokens, 16, D, F, seed=96, dtype="bf16")
    errs, _ = _run("bf16", lay, 16, seed=96, loss="mse", lr=x["lr"] * 0.3, heads=[1, 9])
    print("mse fwdbwd_2x32 errors", errs)
    _assert(errs, TOLS["bf16"])
