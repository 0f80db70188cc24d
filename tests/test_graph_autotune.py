"""CUDA-graph replay and the schedule autotuner (GPU)."""
import numpy as np
import pytest

import oracle
import ttt_synth as syn
from _util import rel_inf, to_np, upload

pytestmark = pytest.mark.gpu


def _setup(H=4, lengths=((3000, 2500, 100), (1041,), (7, 900)), seed=41):
    import torch
    import paper_2604_08542_gb300 as ttt
    lay = syn.layout_from_lengths([list(x) for x in lengths])
    x = syn.make_inputs(lay.num_tokens, H, 64, 128, seed=seed, dtype="bf16", with_grad_out=True)
    g = upload(x, torch.bfloat16)
    return ttt, lay, x, g


def _fwd_bwd(layer, g, lay, outs=None):
    o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                                  want_final=True)
    grads = layer.backward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                           g["d_o"], ck, wn)
    return [o, ck, wn, wf, *grads]


def test_graph_replay_is_bitwise_equal_to_direct_launches():
    import torch
    ttt, lay, x, g = _setup()
    direct = ttt.TTT(4, 64, 128, dtype=torch.bfloat16)
    ref = [t.clone() for t in _fwd_bwd(direct, g, lay)]
    graphed = ttt.TTT(4, 64, 128, dtype=torch.bfloat16)
    graphed.set_graph_mode(True)
    for _ in range(3):                      # capture, then replays / in-place updates
        got = _fwd_bwd(graphed, g, lay)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    # new input values behind the same pointers: the replay must see them
    g["k"].mul_(-1)
    ref2 = [t.clone() for t in _fwd_bwd(direct, g, lay)]
    got2 = _fwd_bwd(graphed, g, lay)
    torch.cuda.synchronize()
    for a, b in zip(got2, ref2):
        assert torch.equal(a, b)
    assert graphed.status() == 0


def test_schedule_roundtrip_and_validation():
    import torch
    import paper_2604_08542_gb300 as ttt
    layer = ttt.TTT(2, 64, 128, dtype=torch.bfloat16)
    s = layer.schedule()
    assert s["fwd_waves"] == 1 and s["bwd_waves"] == 1
    assert s["tail_fill"] == 3 and abs(s["fwd_key_cost"] - 2.45) < 1e-6   # the BF16 head_dim-64 defaults
    layer.set_schedule(fwd_waves=3, fwd_key_cost=1.5)
    s = layer.schedule()
    assert s["fwd_waves"] == 3 and abs(s["fwd_key_cost"] - 1.5) < 1e-6
    with pytest.raises(ttt.Scal3rError):
        layer.set_schedule(fwd_waves=0)
    with pytest.raises(ttt.Scal3rError):
        layer.set_schedule(min_piece_tokens=16)
    layer.set_schedule(tail_fill=0)
    assert layer.schedule()["tail_fill"] == 0
    with pytest.raises(ttt.Scal3rError):
        layer.set_schedule(tail_fill=4)


@pytest.mark.parametrize("waves", [1, 2, 3])
def test_other_schedules_keep_parity(waves):
    """Piece splits change only the order of the sums over pieces."""
    import torch
    ttt, lay, x, g = _setup(H=2, lengths=((5000, 3000), (2100,)), seed=42)
    layer = ttt.TTT(2, 64, 128, dtype=torch.bfloat16)
    layer.set_schedule(fwd_waves=waves, bwd_waves=waves, fwd_key_cost=1.0 + waves, bwd_key_cost=1.5 * waves)
    out = _fwd_bwd(layer, g, lay)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, 64, 128, eps=1e-6)
    rb = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], 64, 128, eps=1e-6)
    pairs = [(out[0], ref["o"]), (out[1], ref["w_ckpt"]), (out[3], ref["w_final"])]
    pairs += [(t, rb[n]) for t, n in zip(out[4:], ("dq", "dk", "dv", "dlr", "dw0"))]
    for t, r in pairs:
        assert rel_inf(to_np(t), r) <= 2e-2


def test_autotune_picks_a_valid_schedule_and_caches_it(tmp_path):
    import torch
    ttt, lay, x, g = _setup(H=16, lengths=((16656, 16656, 16656),), seed=43)
    layer = ttt.TTT(16, 64, 128, dtype=torch.bfloat16)
    cache = str(tmp_path / "tune.json")
    res = layer.autotune(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                         d_o=g["d_o"], cache_path=cache)
    s = res["schedule"]
    assert 1 <= s["fwd_waves"] <= 3 and 1 <= s["bwd_waves"] <= 3 and res["ms"] > 0
    assert 0 <= s["tail_fill"] <= 3
    assert layer.schedule() == s
    again = ttt.TTT(16, 64, 128, dtype=torch.bfloat16).autotune(
        g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr, d_o=g["d_o"],
        cache_path=cache)
    assert again["schedule"] == s
    # the tuned schedule still matches the oracle on one head
    o, ck, wn, wf = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets, lay.seq_chunk_ptr,
                                  want_final=True)
    ref = oracle.forward(x["q"][:, 5:6], x["k"][:, 5:6], x["v"][:, 5:6], x["lr"][:, 5:6], x["w0"][5:6], lay, 64,
                         128, eps=1e-6)
    assert rel_inf(to_np(o)[:, 5:6], ref["o"]) <= 2e-2
