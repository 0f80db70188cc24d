"""Child process of test_bounds_build.py: runs the wide-weight and the fused
head_dim-64 layers on the bounds-checking build of the library (selected by SCAL3R_TTT_LIBRARY before
the package loads it) and prints one JSON line of results."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import paper_2604_08542_gb300 as ttt  # noqa: E402
import ttt_synth as syn  # noqa: E402
from _util import rel_inf, to_np, upload  # noqa: E402

OUT_TENSOR = 5   # o, in the order of scal3r_ttt_debug_bounds


def clean_case(loss, lr_mat, seed):
    """Forward and backward with every range registered at its true size:
    no violation, and the results still match the oracle."""
    H, D, F = 2, 256, 512
    lengths = [[1100, 300], [129]]   # a 1100-token chunk runs its reductions split over K
    lay = syn.layout_from_lengths(lengths)
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=seed, dtype="bf16", with_grad_out=True)
    if lr_mat:
        x["lr"] = syn.per_matrix_lr(seed, lay.num_tokens, H)
    g = upload(x, torch.bfloat16)
    layer = ttt.TTT(H, D, F, dtype=torch.bfloat16, loss=loss, lr_per_matrix=lr_mat)
    assert ttt.scal3r_ttt_debug_bounds(layer.handle, -1, 0) == 0
    o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                                  want_final=True)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    torch.cuda.synchronize()
    status = layer.status()
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, loss=loss, eps=1e-6)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, loss=loss, eps=1e-6)
    errs = {"o": rel_inf(to_np(o), ref["o"]), "w_final": rel_inf(to_np(wf), ref["w_final"])}
    for n, t in zip(("dq", "dk", "dv", "dlr", "dw0"), grads):
        errs[n] = rel_inf(to_np(t), rb[n])
    layer.close()
    return {"status": status, "errors": errs}


def planted_case():
    """o registered 32 bytes short: the last row's last 16 outputs are one
    checked store that falls outside, so it is skipped (the sentinel stays)
    and the status reports it; every access stays inside the real buffer."""
    H, D, F = 1, 256, 512
    lay = syn.layout_from_lengths([[300, 200]])
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=71, dtype="bf16")
    g = upload(x, torch.bfloat16)
    layer = ttt.TTT(H, D, F, dtype=torch.bfloat16)
    o = torch.full_like(g["q"], 7.0)
    ttt.scal3r_ttt_debug_bounds(layer.handle, OUT_TENSOR, 32)
    layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr, o=o)
    torch.cuda.synchronize()
    status = layer.status()
    flat = o.reshape(-1).float()
    tail = flat[-16:]
    before = flat[-32:-16]
    applied = int(lay.num_tokens - lay.chunk_offsets[1])   # tokens of the applied (last) chunk
    ttt.scal3r_ttt_debug_bounds(layer.handle, OUT_TENSOR, 0)
    layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr, o=o)
    torch.cuda.synchronize()
    status_after = layer.status()
    layer.close()
    return {"status": status, "tail_untouched": bool(torch.all(tail == 7.0)),
            "before_tail_written": bool(torch.all(before != 7.0)), "applied_tokens": applied,
            "status_after_restore": status_after}


def clean_case_d64(loss, lr_mat, ckpt_every, seed):
    """The fused head_dim-64 kernels (and the update kernels between them),
    forward and backward on a ragged layout whose chunks end in partial
    tiles (the plain-store rows): no violation, and the oracle's results."""
    H, D, F = 4, 64, 128
    lay = syn.layout_from_lengths([[300, 129, 77, 200], [1100], [1]])
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=seed, dtype="bf16", with_grad_out=True)
    if lr_mat:
        x["lr"] = syn.per_matrix_lr(seed, lay.num_tokens, H)
    g = upload(x, torch.bfloat16)
    layer = ttt.TTT(H, D, F, dtype=torch.bfloat16, loss=loss, lr_per_matrix=lr_mat, ckpt_every=ckpt_every)
    o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                                  want_final=True)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    torch.cuda.synchronize()
    status = layer.status()
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, loss=loss, eps=1e-6)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, loss=loss, eps=1e-6)
    errs = {"o": rel_inf(to_np(o), ref["o"]), "w_final": rel_inf(to_np(wf), ref["w_final"])}
    for n, t in zip(("dq", "dk", "dv", "dlr", "dw0"), grads):
        errs[n] = rel_inf(to_np(t), rb[n])
    layer.close()
    return {"status": status, "errors": errs}


def planted_case_d64():
    """The same planted violation on the head_dim-64 apply role, whose o rows
    are plain 16-byte stores: o registered 32 bytes short skips the last row's
    last two stores (16 outputs) and the status reports it."""
    H, D, F = 2, 64, 128
    lay = syn.layout_from_lengths([[300, 200]])
    x = syn.make_inputs(lay.num_tokens, H, D, F, seed=72, dtype="bf16")
    g = upload(x, torch.bfloat16)
    layer = ttt.TTT(H, D, F, dtype=torch.bfloat16)
    o = torch.full_like(g["q"], 7.0)
    ttt.scal3r_ttt_debug_bounds(layer.handle, OUT_TENSOR, 32)
    layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr, o=o)
    torch.cuda.synchronize()
    status = layer.status()
    flat = o.reshape(-1).float()
    tail, before = flat[-16:], flat[-32:-16]
    ttt.scal3r_ttt_debug_bounds(layer.handle, OUT_TENSOR, 0)
    layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr, o=o)
    torch.cuda.synchronize()
    status_after = layer.status()
    layer.close()
    return {"status": status, "tail_untouched": bool(torch.all(tail == 7.0)),
            "before_tail_written": bool(torch.all(before != 7.0)), "status_after_restore": status_after}


def main():
    out = {"library": ttt.LIB_PATH,
           "dot": clean_case("dot", False, 81),
           "dot_per_matrix": clean_case("dot", True, 82),
           "mse": clean_case("mse", False, 83),
           "planted": planted_case(),
           "d64_dot": clean_case_d64("dot", False, 1, 84),
           "d64_per_matrix_ckpt2": clean_case_d64("dot", True, 2, 85),
           "d64_mse": clean_case_d64("mse", False, 1, 86),
           "d64_planted": planted_case_d64()}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
