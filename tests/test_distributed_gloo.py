"""The multi-rank path on CPU: two gloo ranks (no GPU).

1. Sharding by sequence: each rank runs its sequences (the FP64 oracle
   stands in for the layer), the shards are gathered, and the result equals
   the unsharded run exactly (chains never interact).
2. Global Context Synchronization (Eq. 10): two ranks hold halves of one
   chunk; the sum of their inner gradients, all-reduced over gloo, equals the
   gradient of the whole chunk.
3. The max-over-ranks timer used by bench.py.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import ttt_synth as syn

D, F = 8, 16


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _layout():
    return syn.layout_from_lengths([[9, 4], [13], [2, 2, 7], [5], [11, 3]])


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    from paper_2604_08542_gb300 import distributed as ttd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch
        lay = _layout()
        x = syn.make_inputs(lay.num_tokens, 2, D, F, seed=3)
        shards = ttd.shard_sequences(ttd.seq_token_counts(lay.chunk_offsets, lay.seq_chunk_ptr), world)
        off, ptr, tok = ttd.sub_layout(lay.chunk_offsets, lay.seq_chunk_ptr, shards[rank])
        sub = syn.Layout(off, ptr)
        mine = oracle.forward(x["q"][tok], x["k"][tok], x["v"][tok], x["lr"][tok], x["w0"], sub, D, F)
        got = [None] * world
        dist.all_gather_object(got, (tok, mine["o"], shards[rank], mine["w_final"]))
        # Eq. 10: one chunk split across ranks, gradients summed by all-reduce
        W = oracle.unpack(x["w0"][0], D, F)
        a, b = lay.seq_range(0)
        cut = a + (b - a) // 2
        lo, hi = (a, cut) if rank == 0 else (cut, b)
        G = oracle.pack(oracle.inner_gradient(W, x["k"][lo:hi, 0].astype(np.float64),
                                              x["v"][lo:hi, 0].astype(np.float64),
                                              x["lr"][lo:hi, 0].astype(np.float64)))
        t = torch.from_numpy(G.copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        tmax = ttd.max_over_ranks(float(rank + 1))
        if rank == 0:
            q.put((got, t.numpy(), tmax))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_shard_sequences_and_sum_gradients():
    import oracle
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, gsum, tmax = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    lay = _layout()
    x = syn.make_inputs(lay.num_tokens, 2, D, F, seed=3)
    full = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F)
    o = np.zeros_like(full["o"])
    seen = []
    for tok, o_r, seqs, wf in got:
        o[tok] = o_r
        seen += seqs
        for j, s in enumerate(seqs):
            np.testing.assert_array_equal(wf[j], full["w_final"][s])
    assert sorted(seen) == list(range(lay.num_seqs))
    np.testing.assert_array_equal(o, full["o"])
    W = oracle.unpack(x["w0"][0], D, F)
    a, b = lay.seq_range(0)
    G = oracle.pack(oracle.inner_gradient(W, x["k"][a:b, 0].astype(np.float64), x["v"][a:b, 0].astype(np.float64),
                                          x["lr"][a:b, 0].astype(np.float64)))
    np.testing.assert_allclose(gsum, G, rtol=1e-12, atol=1e-15)
    assert tmax == 2.0


def test_sharding_balances_and_covers():
    from paper_2604_08542_gb300 import distributed as ttd
    counts = [100, 7, 55, 55, 3, 80, 20]
    sh = ttd.shard_sequences(counts, 3)
    assert sorted(s for r in sh for s in r) == list(range(len(counts)))
    loads = [sum(counts[s] for s in r) for r in sh]
    assert max(loads) - min(loads) <= max(counts)
    assert ttd.shard_sequences(counts, 1) == [list(range(len(counts)))]
