"""FP32 SIMT path through the C ABI against the FP64 oracle (GPU).

Bar: normwise relative error max|x - ref| / max|ref| <= 1e-5 for every
output, every checkpoint and every gradient; gradients also agree with
central finite differences of the oracle along random directions.
"""
import numpy as np
import pytest

import oracle
import ttt_synth as syn
from _util import rel_inf, to_np, upload

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _run(lay, H, D, F, seed=0, loss="dot", norm="row_w0", lr_max=0.1, per_seq_w0=False, backward=False):
    import torch
    import paper_2604_08542_gb300 as ttt
    T = lay.num_tokens
    x = syn.make_inputs(T, H, D, F, seed=seed, lr_max=lr_max, with_grad_out=backward)
    if per_seq_w0:
        w = np.stack([syn.make_inputs(1, H, D, F, seed=seed + 100 + s)["w0"] for s in range(lay.num_seqs)])
        x["w0"] = w
    g = upload(x, torch.float32)
    layer = ttt.TTT(H, D, F, dtype=torch.float32, loss=loss, weight_norm=norm)
    o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets,
                                  lay.seq_chunk_ptr, want_final=True)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, loss=loss, norm=norm, eps=1e-6)
    out = {"o": (to_np(o), ref["o"]), "w_ckpt": (to_np(ck), ref["w_ckpt"]),
           "wnorm": (to_np(wn), ref["wnorm"]), "w_final": (to_np(wf), ref["w_final"])}
    if backward:
        dq, dk, dv, dlr, dw0 = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets,
                                              lay.seq_chunk_ptr, g["d_o"], ck, wn)
        rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, loss=loss,
                             norm=norm, eps=1e-6)
        for n, t in (("dq", dq), ("dk", dk), ("dv", dv), ("dlr", dlr), ("dw0", dw0)):
            out[n] = (to_np(t), rb[n])
    torch.cuda.synchronize()
    assert layer.status() == 0
    return out, x


def _assert_all(out, tol=TOL):
    errs = {n: rel_inf(a, b) for n, (a, b) in out.items()}
    bad = {n: e for n, e in errs.items() if not e <= tol}
    assert not bad, f"errors above {tol}: {bad} (all: {errs})"


def test_fp32_small_config_matches_oracle():
    """1 seq x 8 frames x 128 tokens, 1 head, D=64, F=128, chunk 128."""
    w = syn.workload("fp32_small")
    out, _ = _run(w.layout(), 1, 64, 128)
    _assert_all(out)


def test_fp32_ragged_multihead():
    lay = syn.layout_from_lengths([[300, 129, 77], [513], [1, 200, 64, 5], []])
    out, _ = _run(lay, 3, 64, 128, seed=4)
    _assert_all(out)


@pytest.mark.parametrize("loss,norm,lr_max", [("dot", "none", 0.05), ("dot", "unit", 0.1),
                                              ("mse", "row_w0", 0.1), ("mse", "none", 0.02)])
def test_fp32_loss_and_norm_variants(loss, norm, lr_max):
    lay = syn.layout_from_lengths([[128, 128, 96], [40, 300]])
    out, _ = _run(lay, 2, 64, 128, seed=5, loss=loss, norm=norm, lr_max=lr_max)
    _assert_all(out)


def test_fp32_small_shape_per_sequence_w0():
    lay = syn.layout_from_lengths([[50, 30], [17, 17, 17]])
    out, _ = _run(lay, 2, 16, 32, seed=6, per_seq_w0=True)
    _assert_all(out)


@pytest.mark.parametrize("loss,norm", [("dot", "row_w0"), ("dot", "none"), ("mse", "row_w0")])
def test_fp32_backward_matches_oracle(loss, norm):
    lay = syn.layout_from_lengths([[128, 200, 64], [1, 90]])
    out, _ = _run(lay, 2, 64, 128, seed=7, loss=loss, norm=norm, backward=True)
    _assert_all(out)


def test_fp32_backward_per_sequence_w0():
    lay = syn.layout_from_lengths([[40, 33], [20, 7, 9]])
    out, _ = _run(lay, 2, 16, 32, seed=8, per_seq_w0=True, backward=True)
    _assert_all(out)


def test_fp32_gradients_match_finite_differences():
    """<grad, u> against central differences of the FP64 oracle (eps 1e-6), tol 1e-4."""
    import torch
    import paper_2604_08542_gb300 as ttt
    lay = syn.layout_from_lengths([[128, 128, 128]])
    H, D, F = 2, 64, 128
    T = lay.num_tokens
    x = syn.make_inputs(T, H, D, F, seed=9, with_grad_out=True)
    g = upload(x, torch.float32)
    layer = ttt.TTT(H, D, F, dtype=torch.float32)
    o, ck, wn, _ = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    gnp = dict(zip(("q", "k", "v", "lr", "w0"), (to_np(t) for t in grads)))
    base = {n: x[n].astype(np.float64) for n in ("q", "k", "v", "lr", "w0")}
    d_o = x["d_o"].astype(np.float64)

    def objective(inp):
        r = oracle.forward(inp["q"], inp["k"], inp["v"], inp["lr"], inp["w0"], lay, D, F, eps=1e-6)
        return float(np.sum(r["o"] * d_o))

    eps = 1e-6
    for i, n in enumerate(("q", "k", "v", "lr", "w0")):
        u = syn.random_direction(100 + i, base[n].shape)
        plus = dict(base)
        minus = dict(base)
        plus[n] = base[n] + eps * u
        minus[n] = base[n] - eps * u
        fd = (objective(plus) - objective(minus)) / (2 * eps)
        an = float(np.sum(gnp[n] * u))
        assert abs(an - fd) <= 1e-4 * max(1.0, abs(fd)), (n, an, fd)


@pytest.mark.parametrize("dtype_name,D,F,tol", [("fp32", 16, 32, TOL), ("bf16", 64, 128, 2e-2)])
def test_clamped_rows_match_oracle(dtype_name, D, F, tol):
    """The clamp branch of the row rescale (reading A8: max(||row||, eps)) on
    the GPU.  Every other row of w0 is scaled down, so the rows' norms fall in
    two groups with a wide gap, and eps lies in the gap: the small rows are
    rescaled by rho / eps (and stay below eps), the others by rho / ||row||.
    Forward and backward against the oracle run with the same eps."""
    import torch
    import paper_2604_08542_gb300 as ttt
    dtype = torch.float32 if dtype_name == "fp32" else torch.bfloat16
    lay = syn.layout_from_lengths([[300, 129], [257]])
    H, T = 2, lay.num_tokens
    x = syn.make_inputs(T, H, D, F, seed=41, dtype=dtype_name, with_grad_out=True, lr_max=0.3)
    # rows of W1 and W3 hold D values, rows of W2 F values (packed W1, W3, W2)
    rows = np.concatenate([np.repeat(np.arange(2 * F), D), 2 * F + np.repeat(np.arange(D), F)])
    x["w0"] = (x["w0"] * np.where(rows % 2 == 0, 0.3, 1.0)[None, :]).astype(np.float32)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=1e-6)
    n = np.sort(ref["wnorm"].reshape(-1))
    gap = int(np.argmax(n[1:] / n[:-1]))                 # the widest gap between consecutive norms
    eps = float(np.sqrt(n[gap] * n[gap + 1]))
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=eps)
    n = ref["wnorm"].reshape(-1)
    assert np.any(n < eps) and np.any(n > eps) and np.min(np.abs(n - eps)) > 0.1 * eps
    g = upload(x, dtype)
    layer = ttt.TTT(H, D, F, dtype=dtype, norm_eps=eps)
    o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                                  want_final=True)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    torch.cuda.synchronize()
    assert layer.status() == 0
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, eps=eps)
    out = {"o": (to_np(o), ref["o"]), "w_ckpt": (to_np(ck), ref["w_ckpt"]), "wnorm": (to_np(wn), ref["wnorm"]),
           "w_final": (to_np(wf), ref["w_final"])}
    for nme, t in zip(("dq", "dk", "dv", "dlr", "dw0"), grads):
        out[nme] = (to_np(t), rb[nme])
    _assert_all(out, tol)
