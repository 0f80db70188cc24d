"""The linear-model mode on the GPU (float32 path, through the C ABI):
f_W(x) = W x with one D x D matrix per chain (Sec. 3.2, Eq. 3-4 with a linear
map).

* P2: with the dot loss and no normalisation the outputs are chunk-causal
  linear attention, o_t = W0 q_t + sum over keys j of chunks up to t's own of
  lr_j (q_t . k_j) v_j, computed here directly from that definition.
* P3: with the squared-error loss and no normalisation the checkpoints follow
  the chunkwise delta rule W <- W (I - K^T diag(lr) K) + V^T diag(lr) K.
* Forward and backward against the FP64 oracle for every loss and
  normalisation, ragged chunks with tile edges (tiles of 32 tokens), shared and
  per-sequence w0, D in {16, 32, 64}.

Bar: 1e-5 normwise (the float32 path's).
"""
import numpy as np
import pytest

import oracle
import ttt_synth as syn
from _util import rel_inf, to_np

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _inputs(lay, H, D, seed, per_seq_w0=False, lr_scale=1.0):
    x = syn.make_inputs(lay.num_tokens, H, D, 2 * D, seed=seed, with_grad_out=True)
    x["lr"] = (x["lr"] * lr_scale).astype(np.float32)
    shape = (lay.num_seqs, H, D * D) if per_seq_w0 else (H, D * D)
    x["w0"] = (syn.random_direction(seed + 1, shape) * 0.3).astype(np.float32)
    return x


def _dev(x):
    import torch
    return {n: torch.from_numpy(np.ascontiguousarray(a)).cuda() for n, a in x.items()}


def _layer(H, D, loss="dot", norm="none"):
    import torch
    import paper_2604_08542_gb300 as ttt
    return ttt.TTT(H, D, D, dtype=torch.float32, loss=loss, weight_norm=norm, model="linear")


def _forward(layer, g, lay, want_final=True):
    import torch
    out = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                        want_final=want_final)
    torch.cuda.synchronize()
    assert layer.status() == 0
    return out


@pytest.mark.parametrize("D", [16, 64])
def test_linear_dot_is_chunk_causal_linear_attention(D):
    lay = syn.layout_from_lengths([[70, 33, 1, 96], [5, 64]])
    H = 2
    x = _inputs(lay, H, D, seed=11)
    o = to_np(_forward(_layer(H, D), _dev(x), lay)[0])
    ref = np.zeros_like(o)
    for s in range(lay.num_seqs):
        a, b = lay.seq_range(s)
        cid = np.zeros(b - a, dtype=int)
        for j, (t0, t1) in enumerate(lay.seq_chunks(s)):
            cid[t0 - a:t1 - a] = j
        mask = cid[None, :] <= cid[:, None]
        for h in range(H):
            Q, K, V = (x[n][a:b, h].astype(np.float64) for n in ("q", "k", "v"))
            eta = x["lr"][a:b, h].astype(np.float64)
            W0 = x["w0"][h].astype(np.float64).reshape(D, D)
            ref[a:b, h] = Q @ W0.T + ((Q @ K.T) * mask * eta[None, :]) @ V
    assert rel_inf(o, ref) <= TOL


def test_linear_mse_is_chunkwise_delta_rule():
    D = 32
    lay = syn.layout_from_lengths([[40, 7, 65]])
    x = _inputs(lay, 1, D, seed=12, lr_scale=0.2)
    _, ck, _, wf = _forward(_layer(1, D, loss="mse"), _dev(x), lay)
    ck = to_np(ck)
    W = x["w0"][0].astype(np.float64).reshape(D, D)
    for c, (t0, t1) in enumerate(lay.seq_chunks(0)):
        K, V = (x[n][t0:t1, 0].astype(np.float64) for n in ("k", "v"))
        eta = x["lr"][t0:t1, 0].astype(np.float64)
        W = W @ (np.eye(D) - (K.T * eta) @ K) + (V.T * eta) @ K
        assert rel_inf(ck[c, 0].reshape(D, D), W) <= TOL, c
    assert rel_inf(to_np(wf)[0, 0].reshape(D, D), W) <= TOL


CASES = [(16, "dot", "none", False), (32, "dot", "row_w0", False), (64, "dot", "unit", True),
         (64, "mse", "none", False), (32, "mse", "row_w0", True), (16, "mse", "unit", False)]


@pytest.mark.parametrize("D,loss,norm,per_seq", CASES)
def test_linear_forward_backward_match_oracle(D, loss, norm, per_seq):
    import torch
    lay = syn.layout_from_lengths([[70, 33, 1, 96], [], [5, 64, 31]])
    H = 2
    x = _inputs(lay, H, D, seed=13, per_seq_w0=per_seq, lr_scale=0.3 if loss == "mse" else 1.0)
    g = _dev(x)
    layer = _layer(H, D, loss, norm)
    o, ck, wn, wf = _forward(layer, g, lay)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    torch.cuda.synchronize()
    assert layer.status() == 0
    kw = dict(loss=loss, norm=norm, model="linear", eps=1e-6)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, D, **kw)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, D, **kw)
    errs = {"o": rel_inf(to_np(o), ref["o"]), "w_ckpt": rel_inf(to_np(ck), ref["w_ckpt"]),
            "wnorm": rel_inf(to_np(wn), ref["wnorm"]), "w_final": rel_inf(to_np(wf), ref["w_final"])}
    for n, t in zip(("dq", "dk", "dv", "dlr", "dw0"), grads):
        errs[n] = rel_inf(to_np(t), rb[n])
    bad = {n: e for n, e in errs.items() if not e <= TOL}
    assert not bad, f"above {TOL}: {bad}; all {errs}"


def test_linear_backward_is_deterministic():
    import torch
    lay = syn.layout_from_lengths([[100, 50], [77]])
    x = _inputs(lay, 3, 64, seed=14)
    g = _dev(x)
    layer = _layer(3, 64, "mse", "row_w0")
    runs = []
    for _ in range(2):
        o, ck, wn, _ = _forward(layer, g, lay, want_final=False)
        grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                               g["d_o"], ck, wn)
        torch.cuda.synchronize()
        runs.append([o.clone()] + [t.clone() for t in grads])
    for a, b in zip(*runs):
        assert torch.equal(a, b)
