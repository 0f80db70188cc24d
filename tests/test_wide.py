"""The wide-weight BF16 forward (head_dim and hidden multiples of 256, up to the
paper's own AMU shape: one head, hd = 1024, hidden = 4 hd) through the C ABI,
against the FP64 oracle on the same bfloat16-rounded q, k, v (GPU).

Bar: normwise relative error <= 2e-2 on o, every checkpoint, the
pre-normalisation row norms and w_final, as for the head_dim-64 BF16 path.
"""
import numpy as np
import pytest

import oracle
import ttt_synth as syn
from _util import rel_inf, to_np, upload

pytestmark = pytest.mark.gpu

TOL = 2e-2


def _run(H, D, F, lengths, seed, graph=False, layer=None):
    import torch
    import paper_2604_08542_gb300 as ttt
    lay = syn.layout_from_lengths(lengths)
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=seed, dtype="bf16")
    g = upload(x, torch.bfloat16)
    if layer is None:
        layer = ttt.TTT(H, D, F, dtype=torch.bfloat16)
    layer.set_graph_mode(graph)
    out = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                        want_final=True)
    torch.cuda.synchronize()
    assert layer.status() == 0
    return layer, lay, x, out


def _check(out, ref, tol=TOL):
    o, ck, wn, wf = (to_np(t) for t in out)
    errs = {"o": rel_inf(o, ref["o"]), "w_ckpt": rel_inf(ck, ref["w_ckpt"]), "wnorm": rel_inf(wn, ref["wnorm"]),
            "w_final": rel_inf(wf, ref["w_final"])}
    bad = {n: e for n, e in errs.items() if not e <= tol}
    assert not bad, f"above {tol}: {bad}; all {errs}"
    return errs


def test_wide_two_heads_ragged_matches_oracle():
    """D = 256, F = 512, two heads, two sequences; chunk lengths off the
    128-token tile (300, 129) and a short sequence (77)."""
    H, D, F = 2, 256, 512
    _, lay, x, out = _run(H, D, F, [[300, 129], [77]], seed=41)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=1e-6)
    _check(out, ref)


def test_wide_paper_shape_matches_oracle():
    """The paper's AMU: one head, hd = 1024, hidden 4096 (k = 4); two chunks."""
    H, D, F = 1, 1024, 4096
    _, lay, x, out = _run(H, D, F, [[640, 200]], seed=42)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=1e-6)
    _check(out, ref)


@pytest.mark.parametrize("k_scale", [1, 2])
def test_wide_state_size_ablation_shapes(k_scale):
    """hd = 512 with hidden k * hd for k = 1, 2 (the state-size ablation's k)."""
    H, D = 1, 512
    F = k_scale * D
    _, lay, x, out = _run(H, D, F, [[383, 260]], seed=43 + k_scale)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=1e-6)
    _check(out, ref)


def test_wide_graph_replay_and_determinism():
    import torch
    layer, lay, x, a = _run(1, 256, 512, [[500, 300]], seed=44)
    a = [t.clone() for t in a]
    _, _, _, b = _run(1, 256, 512, [[500, 300]], seed=44, layer=layer)
    for _ in range(2):
        _, _, _, c = _run(1, 256, 512, [[500, 300]], seed=44, graph=True, layer=layer)
    for u, w, z in zip(a, b, c):
        assert torch.equal(u, w) and torch.equal(u, z)


def _fwd_bwd(H, D, F, lengths, seed, layer=None, graph=False, per_seq_w0=False):
    import torch
    import paper_2604_08542_gb300 as ttt
    lay = syn.layout_from_lengths(lengths)
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=seed, dtype="bf16", with_grad_out=True)
    if per_seq_w0:
        S = len(lengths)
        x["w0"] = np.stack([x["w0"] * (1.0 + 0.1 * s) for s in range(S)]).astype(np.float32)
    g = upload(x, torch.bfloat16)
    if layer is None:
        layer = ttt.TTT(H, D, F, dtype=torch.bfloat16)
    layer.set_graph_mode(graph)
    o, ck, wn, _ = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    torch.cuda.synchronize()
    assert layer.status() == 0
    return layer, lay, x, grads


def _check_grads(grads, rb, tol=TOL):
    errs = {n: rel_inf(to_np(t), rb[n]) for n, t in zip(("dq", "dk", "dv", "dlr", "dw0"), grads)}
    bad = {n: e for n, e in errs.items() if not e <= tol}
    assert not bad, f"above {tol}: {bad}; all {errs}"
    return errs


def test_wide_backward_two_heads_ragged_matches_oracle():
    """dq, dk, dv, d eta and dW0 (shared over two sequences) at hd 256, hidden
    512: chunks off the tile (300, 129) and a one-chunk sequence (77)."""
    H, D, F = 2, 256, 512
    _, lay, x, grads = _fwd_bwd(H, D, F, [[300, 129], [77]], seed=51)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, eps=1e-6)
    _check_grads(grads, rb)


def test_wide_backward_per_sequence_w0_matches_oracle():
    """Three chunks in one sequence and a second sequence with its own w0."""
    H, D, F = 1, 512, 1024
    _, lay, x, grads = _fwd_bwd(H, D, F, [[200, 256, 70], [140]], seed=52, per_seq_w0=True)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, eps=1e-6)
    _check_grads(grads, rb)


def test_wide_backward_paper_shape_matches_oracle():
    """The paper's AMU: one head, hd 1024, hidden 4096; two chunks."""
    H, D, F = 1, 1024, 4096
    _, lay, x, grads = _fwd_bwd(H, D, F, [[384, 200]], seed=53)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, eps=1e-6)
    _check_grads(grads, rb)


@pytest.mark.parametrize("k", [1, 2])
def test_wide_state_size_ablation_hd1024_forward_backward(k):
    """The paper's state-size ablation: one head, hd 1024, hidden k * hd with
    k = 1 and 2 (the AMU uses k = 4); forward outputs and every gradient, two
    chunks off the 128-token tile.  The first chunk is long enough (16 and
    10 K blocks of 64 tokens) for the weight-sized reductions, whose 32 and
    64 output tiles leave most SMs idle, to run split over K (4 and 2
    ranges) and be summed in a fixed order."""
    H, D, F = 1, 1024, 1024 * k
    lengths = [[1000 if k == 1 else 600, 141]]
    _, lay, x, out = _run(H, D, F, lengths, seed=56 + k)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=1e-6)
    _check(out, ref)
    _, lay, x, grads = _fwd_bwd(H, D, F, lengths, seed=58 + k)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, eps=1e-6)
    _check_grads(grads, rb)


def test_wide_backward_graph_replay_is_bitwise_equal():
    import torch
    layer, lay, x, a = _fwd_bwd(1, 256, 512, [[300, 200]], seed=54)
    a = [t.clone() for t in a]
    for _ in range(2):
        _, _, _, b = _fwd_bwd(1, 256, 512, [[300, 200]], seed=54, layer=layer, graph=True)
        for u, w in zip(a, b):
            assert torch.equal(u, w)


def test_wide_split_reductions_match_oracle():
    """Chunks of 2600 and 900 tokens at hd 256, hidden 512 (4 output tiles
    per weight-sized reduction): the reductions run in 10 and 3 K ranges
    whose partial planes are summed in a fixed order; two heads, forward
    and backward."""
    H, D, F = 2, 256, 512
    lengths = [[2600, 300], [900]]
    _, lay, x, out = _run(H, D, F, lengths, seed=63)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=1e-6)
    _check(out, ref)
    _, lay, x, grads = _fwd_bwd(H, D, F, lengths, seed=64)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, eps=1e-6)
    _check_grads(grads, rb)


@pytest.mark.parametrize("lengths", [[[200, 256, 70, 130, 90], [140, 60]], [[1100, 256, 700, 130, 90], [140, 600]]],
                         ids=["short", "split"])
@pytest.mark.parametrize("n", [2, 3])
def test_wide_sparse_checkpoints_are_bitwise_the_dense_ones(n, lengths):
    """ckpt_every = n stores the weights after local chunks n-1, 2n-1, ... of
    each sequence; the backward recomputes the rest with the forward's own
    steps, so every output equals the every-chunk run bit for bit (also
    when the chunks are long enough for the weight-sized reductions to run
    split over K)."""
    import torch
    import paper_2604_08542_gb300 as ttt
    H, D, F = 1, 256, 512
    lay = syn.layout_from_lengths(lengths)
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=55, dtype="bf16", with_grad_out=True)
    g = upload(x, torch.bfloat16)
    out = {}
    for every in (1, n):
        layer = ttt.TTT(H, D, F, dtype=torch.bfloat16, ckpt_every=every)
        o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets,
                                      lay.seq_chunk_ptr, want_final=True)
        grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                               g["d_o"], ck, wn)
        torch.cuda.synchronize()
        assert layer.status() == 0
        out[every] = (o, ck, wn, wf, grads)
    o1, ck1, wn1, wf1, g1 = out[1]
    on, ckn, wnn, wfn, gn = out[n]
    stored = [c0 + j - 1 for s, (c0, c1) in enumerate(zip(lay.seq_chunk_ptr[:-1], lay.seq_chunk_ptr[1:]))
              for j in range(n, c1 - c0 + 1, n)]
    assert ckn.shape[0] == len(stored)
    assert torch.equal(ckn, ck1[stored])
    for a, b in [(o1, on), (wn1, wnn), (wf1, wfn), *zip(g1, gn)]:
        assert torch.equal(a, b)


# ---- the squared-error loss (L = 1/2 |f_W(k) - v|^2 in Eq. 8) ----

@pytest.mark.parametrize("H,D,F,lengths", [(2, 256, 512, [[300, 129], [77]]),
                                           (1, 2048, 256, [[260, 130]])])
def test_wide_mse_forward_and_backward_match_oracle(H, D, F, lengths):
    """Forward outputs and every gradient under the squared-error loss; the
    second shape has more output-column tiles (D / 256) than hidden-unit
    groups of 64, the d eta partials' other sizing."""
    import torch
    import paper_2604_08542_gb300 as ttt
    lay = syn.layout_from_lengths(lengths)
    layer = ttt.TTT(H, D, F, dtype=torch.bfloat16, loss="mse")
    _, _, x, out = _run(H, D, F, lengths, seed=61, layer=layer)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, loss="mse", eps=1e-6)
    _check(out, ref)
    _, _, x, grads = _fwd_bwd(H, D, F, lengths, seed=62, layer=layer)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, loss="mse", eps=1e-6)
    _check_grads(grads, rb)


def test_wide_mse_paper_shape_matches_oracle():
    """The paper's AMU (hd 1024, hidden 4096) under the squared-error loss."""
    import torch
    import paper_2604_08542_gb300 as ttt
    H, D, F, lengths = 1, 1024, 4096, [[384, 200]]
    lay = syn.layout_from_lengths(lengths)
    layer = ttt.TTT(H, D, F, dtype=torch.bfloat16, loss="mse")
    _, _, x, grads = _fwd_bwd(H, D, F, lengths, seed=63, layer=layer)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, loss="mse", eps=1e-6)
    _check_grads(grads, rb)


def test_wide_mse_sparse_checkpoints_are_bitwise_the_dense_ones():
    import torch
    import paper_2604_08542_gb300 as ttt
    H, D, F = 1, 256, 512
    lengths = [[200, 256, 70, 130]]
    lay = syn.layout_from_lengths(lengths)
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=64, dtype="bf16", with_grad_out=True)
    g = upload(x, torch.bfloat16)
    res = []
    for every in (1, 2):
        layer = ttt.TTT(H, D, F, dtype=torch.bfloat16, loss="mse", ckpt_every=every)
        o, ck, wn, _ = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets,
                                     lay.seq_chunk_ptr)
        grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                               g["d_o"], ck, wn)
        torch.cuda.synchronize()
        assert layer.status() == 0
        res.append((o, wn, *grads))
    for a, b in zip(*res):
        assert torch.equal(a, b)


# ---- per-matrix learning rates (lr [T, H, 3]: W1, W3, W2) ----

@pytest.mark.parametrize("loss", ["dot", "mse"])
def test_wide_per_matrix_rates_match_oracle(loss):
    """Forward outputs and every gradient (dlr [T, H, 3]) with a rate per
    matrix, both losses, two heads and ragged chunks."""
    import torch
    import paper_2604_08542_gb300 as ttt
    H, D, F = 2, 256, 512
    lengths = [[300, 129], [77]]
    lay = syn.layout_from_lengths(lengths)
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=71, dtype="bf16", with_grad_out=True)
    x["lr"] = syn.per_matrix_lr(72, lay.num_tokens, H, lr_max=0.1)
    g = upload(x, torch.bfloat16)
    layer = ttt.TTT(H, D, F, dtype=torch.bfloat16, loss=loss, lr_per_matrix=True)
    o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                                  want_final=True)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    torch.cuda.synchronize()
    assert layer.status() == 0
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, loss=loss, eps=1e-6)
    _check((o, ck, wn, wf), ref)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, loss=loss, eps=1e-6)
    assert tuple(grads[3].shape) == x["lr"].shape
    _check_grads(grads, rb)


def test_wide_equal_per_matrix_rates_match_one_rate():
    """Three equal rates per token give the one-rate layer's outputs (up to
    the kernels' rounding order) and d eta split three ways."""
    import torch
    import paper_2604_08542_gb300 as ttt
    H, D, F = 1, 512, 1024
    lengths = [[260, 200]]
    lay = syn.layout_from_lengths(lengths)
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=73, dtype="bf16", with_grad_out=True)
    g = upload(x, torch.bfloat16)
    res = []
    for per in (False, True):
        layer = ttt.TTT(H, D, F, dtype=torch.bfloat16, lr_per_matrix=per)
        lr = g["lr"][..., None].expand(-1, -1, 3).contiguous() if per else g["lr"]
        o, ck, wn, _ = layer.forward(g["q"], g["k"], g["v"], lr, g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr)
        grads = layer.backward(g["q"], g["k"], g["v"], lr, g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                               g["d_o"], ck, wn)
        torch.cuda.synchronize()
        assert layer.status() == 0
        res.append((o, ck, grads))
    (o1, ck1, g1), (o3, ck3, g3) = res
    assert rel_inf(to_np(o3), to_np(o1)) < 5e-3
    assert rel_inf(to_np(ck3), to_np(ck1)) < 1e-4
    for n, a, b in zip(("dq", "dk", "dv", "dw0"), (g1[0], g1[1], g1[2], g1[4]), (g3[0], g3[1], g3[2], g3[4])):
        assert rel_inf(to_np(b), to_np(a)) < 5e-3, n
    assert rel_inf(to_np(g3[3]).sum(-1), to_np(g1[3])) < 5e-3


# ---- edge cases and the full-size paper workload ----

def test_wide_tiny_and_empty_chunks_match_oracle():
    """Chunks of 1, 63 and 65 tokens, an empty sequence and tile edges (127, 129)
    at the smallest wide shape (hd 256, hidden 256), forward and backward."""
    H, D, F = 2, 256, 256
    lengths = [[1, 63, 65], [], [129, 127]]
    _, lay, x, out = _run(H, D, F, lengths, seed=81)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=1e-6)
    _check(out, ref)
    _, lay, x, grads = _fwd_bwd(H, D, F, lengths, seed=82)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, eps=1e-6)
    _check_grads(grads, rb)


@pytest.mark.parametrize("D,F", [(4096, 256), (256, 4096)])
def test_wide_largest_dims_match_oracle(D, F):
    """The largest head_dim and the largest hidden size the path takes."""
    _, lay, x, grads = _fwd_bwd(1, D, F, [[200, 90]], seed=83)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, eps=1e-6)
    _check_grads(grads, rb)


def test_wide_lr_zero_gives_plain_mlp():
    """With every learning rate 0 the weights never move: o = f_W0(q) and every
    checkpoint equals W0 (exactly, the row rescale of an unchanged row aside)."""
    import torch
    import paper_2604_08542_gb300 as ttt
    H, D, F = 1, 512, 1024
    lay = syn.layout_from_lengths([[300, 212]])
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=84, dtype="bf16")
    x["lr"][:] = 0.0
    g = upload(x, torch.bfloat16)
    layer = ttt.TTT(H, D, F, dtype=torch.bfloat16)
    o, ck, _, _ = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr)
    torch.cuda.synchronize()
    assert layer.status() == 0
    W0 = oracle.unpack(x["w0"][0].astype(np.float64), D, F)
    ref = oracle.apply(W0, x["q"][:, 0].astype(np.float64))
    assert rel_inf(to_np(o)[:, 0], ref) <= TOL
    assert rel_inf(to_np(ck)[:, 0], np.stack([x["w0"][0]] * 2)) <= 1e-6


def test_wide_amu_full_size_graph_matches_oracle():
    """The paper-shape bench workload at full size (66,624 tokens, one head,
    hd 1024, hidden 4096, four chunks of 16,656 tokens) in graph mode, the
    launch configuration the benchmark times: o, every checkpoint and the
    pre-normalisation row norms against the oracle."""
    import torch
    import paper_2604_08542_gb300 as ttt
    w = syn.workload("bf16_amu1024")
    lay = w.layout()
    T, H, D, F = lay.num_tokens, w.heads, w.head_dim, w.hidden
    x = syn.make_inputs(T, H, D, F, seed=85, dtype="bf16")
    g = upload(x, torch.bfloat16)
    layer = ttt.TTT(H, D, F, dtype=torch.bfloat16)
    layer.set_graph_mode(True)
    for _ in range(2):
        out = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                            want_final=True)
    torch.cuda.synchronize()
    assert layer.status() == 0
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=1e-6)
    _check(out, ref)
