"""Global Context Synchronisation (Sec. 4.2, Eq. 10): a chunk step split into
partial_grad (per token shard) -> sum over shards -> apply_update -> apply.

CPU: two gloo ranks run the chunk loop of distributed.gcs_forward with the
FP64 oracle's pieces, each holding a shard of every chunk; the gathered
result equals the oracle's forward of the unsharded sequence.

GPU (through the C ABI): the same loop with the library's three calls, two
shards per chunk summed on one device, equals the library's own forward of
the unsharded sequence (the chunk sums group the tokens differently, so up to
rounding) and the oracle within each path's bar.
"""
import os
import time
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import ttt_synth as syn
from _util import rel_inf, to_np, upload

D_CPU, F_CPU = 8, 16
CHUNKS = [9, 13, 6]          # one sequence, three chunks
CUTS = [4, 7, 6]             # rank 0 holds the first CUTS[j] tokens of chunk j (all of the last one)


def _oracle_pieces(H, D, F, eps=1e-6):
    """partial_grad / apply_update / apply of one sequence with all heads, in FP64."""
    def partial_grad(k, v, lr, w):
        out = np.zeros((H, 3 * F * D))
        for h in range(H):
            if len(k):
                out[h] = oracle.pack(oracle.inner_gradient(oracle.unpack(w[h], D, F), k[:, h].astype(np.float64),
                                                           v[:, h].astype(np.float64), lr[:, h].astype(np.float64)))
        return out

    def apply_update(w, g, w0):
        out = np.zeros_like(w)
        for h in range(H):
            Wt = [a - b for a, b in zip(oracle.unpack(w[h], D, F), oracle.unpack(g[h], D, F))]
            rho = oracle.row_targets(oracle.unpack(w0[h].astype(np.float64), D, F), "row_w0")
            out[h] = oracle.pack(oracle.normalise(Wt, rho, eps)[0])
        return out

    def apply(q, w):
        return np.stack([oracle.apply(oracle.unpack(w[h], D, F), q[:, h].astype(np.float64)) for h in range(H)],
                        axis=1) if len(q) else np.zeros((0, H, D))

    return partial_grad, apply_update, apply


def _shards(x, rank):
    """This rank's rows of every chunk, and their bounds in its local arrays."""
    idx, bounds, base = [], [], 0
    for n, c in zip(CHUNKS, CUTS):
        lo, hi = (0, c) if rank == 0 else (c, n)
        idx.append(np.arange(base + lo, base + hi))
        base += n
    local = {}
    for name in ("q", "k", "v", "lr"):
        local[name] = np.concatenate([x[name][i] for i in idx])
    a = 0
    for i in idx:
        bounds.append((a, a + len(i)))
        a += len(i)
    return local, bounds, idx


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    from paper_2604_08542_gb300 import distributed as ttd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        H = 2
        x = syn.make_inputs(sum(CHUNKS), H, D_CPU, F_CPU, seed=5)
        loc, bounds, idx = _shards(x, rank)
        pg, au, ap = _oracle_pieces(H, D_CPU, F_CPU)

        def all_reduce(g):
            t = torch.from_numpy(np.ascontiguousarray(g))
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            return t.numpy()

        outs, w = ttd.gcs_forward(loc["q"], loc["k"], loc["v"], loc["lr"], x["w0"].astype(np.float64), bounds,
                                  partial_grad=pg, apply_update=au, apply=ap, all_reduce=all_reduce)
        got = [None] * world
        dist.all_gather_object(got, (idx, outs, w))
        if rank == 0:
            q.put(got)
    finally:
        dist.destroy_process_group()


def _collect(q, procs, timeout):
    """Rank 0's gathered result; fails as soon as a rank has died instead of
    waiting out the whole timeout."""
    import queue as _queue
    deadline = time.monotonic() + timeout
    while True:
        try:
            got = q.get(timeout=2)
            break
        except _queue.Empty:
            dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
            if dead or time.monotonic() > deadline:
                for p in procs:
                    if p.is_alive():
                        p.terminate()
                pytest.fail(f"a rank failed (exit codes {[p.exitcode for p in procs]})" if dead
                            else "ranks timed out")
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return got


@pytest.mark.timeout(300)
def test_gcs_two_gloo_ranks_equal_unsharded_oracle():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = _collect(q, procs, 240)
    H = 2
    x = syn.make_inputs(sum(CHUNKS), H, D_CPU, F_CPU, seed=5)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], syn.layout_from_lengths([CHUNKS]), D_CPU, F_CPU)
    o = np.full_like(ref["o"], np.nan)
    for idx, outs, w in got:
        for i, part in zip(idx, outs):
            o[i] = part
        np.testing.assert_allclose(w, ref["w_final"][0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(o, ref["o"], rtol=1e-10, atol=1e-13)


def test_gcs_one_rank_is_the_forward():
    """World of one: the loop with an identity all-reduce is the forward."""
    from paper_2604_08542_gb300 import distributed as ttd
    H = 3
    x = syn.make_inputs(sum(CHUNKS), H, D_CPU, F_CPU, seed=6)
    pg, au, ap = _oracle_pieces(H, D_CPU, F_CPU)
    bounds = [(a, b) for a, b in syn.layout_from_lengths([CHUNKS]).seq_chunks(0)]
    outs, w = ttd.gcs_forward(x["q"], x["k"], x["v"], x["lr"], x["w0"].astype(np.float64), bounds,
                              partial_grad=pg, apply_update=au, apply=ap, all_reduce=lambda g: g)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], syn.layout_from_lengths([CHUNKS]), D_CPU, F_CPU)
    np.testing.assert_allclose(np.concatenate(outs), ref["o"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(w, ref["w_final"][0], rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------
# GPU: the library's three calls
# ---------------------------------------------------------------------------

def _gpu_gcs(dtype, H, D, F, chunks, cuts, seed, per_matrix=False, loss="dot"):
    """Two shards per chunk on one device, in the order of
    distributed.gcs_forward: returns (outputs of the loop, its weights after
    every chunk, the library's forward of the unsharded sequence (o, w_ckpt),
    the oracle's forward).  per_matrix: rates [T, H, 3]."""
    import torch

    import paper_2604_08542_gb300 as ttt
    lay = syn.layout_from_lengths([chunks])
    T = lay.num_tokens
    x = syn.make_inputs(T, H, D, F, seed=seed, dtype="bf16" if dtype == torch.bfloat16 else "fp32")
    if per_matrix:
        x["lr"] = syn.per_matrix_lr(seed + 1, T, H, lr_max=0.1)
    if loss == "mse":
        x["lr"] = x["lr"] * 0.3
    g = upload(x, dtype)
    layer = ttt.TTT(H, D, F, dtype=dtype, lr_per_matrix=per_matrix, loss=loss)
    o_ref, ck_ref, _, _ = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets,
                                        lay.seq_chunk_ptr)
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=1e-6, loss=loss)

    def one_chunk(n):
        return syn.layout_from_lengths([[n]] if n > 0 else [[]])

    o = torch.empty_like(g["q"])
    w = g["w0"]
    ckpts = []
    base = 0
    for n, c in zip(chunks, cuts):
        shards = [(base, base + c), (base + c, base + n)]
        grads = []
        for a, b in shards:   # each shard in its own allocation, as its own caller would hold it
            lo = one_chunk(b - a)
            grads.append(layer.partial_grad(g["k"][a:b].clone(), g["v"][a:b].clone(),
                                            g["lr"][a:b].clone(), w, lo.chunk_offsets, lo.seq_chunk_ptr))
        w_next, _ = layer.apply_update(w, grads[0] + grads[1], g["w0"])
        for a, b in shards:
            if b > a:
                lo = one_chunk(b - a)
                o[a:b] = layer.apply(g["q"][a:b].clone(), w_next, lo.chunk_offsets, lo.seq_chunk_ptr)
        w = w_next
        ckpts.append(w_next[0])
        base += n
    torch.cuda.synchronize()
    assert layer.status() == 0
    return to_np(o), np.stack([to_np(c) for c in ckpts]), to_np(o_ref), to_np(ck_ref), ref


@pytest.mark.gpu
def test_gpu_gcs_fp32_equals_forward():
    """FP32 path, 2 heads, chunks 300/129/77 tokens cut at 137/0/40: one shard empty."""
    import torch
    o, ck, o_ref, ck_ref, ref = _gpu_gcs(torch.float32, 2, 64, 128, [300, 129, 77], [137, 0, 40], seed=3)
    assert rel_inf(o, o_ref) <= 1e-5 and rel_inf(ck, ck_ref) <= 1e-5
    assert rel_inf(o, ref["o"]) <= 1e-5 and rel_inf(ck, ref["w_ckpt"]) <= 1e-5


@pytest.mark.gpu
def test_gpu_gcs_bf16_equals_forward():
    """BF16 path, 4 heads, chunks 2,000/1,041/333 tokens, ragged cuts."""
    import torch
    o, ck, o_ref, ck_ref, ref = _gpu_gcs(torch.bfloat16, 4, 64, 128, [2000, 1041, 333], [1000, 513, 129], seed=4)
    assert rel_inf(o, o_ref) <= 5e-3 and rel_inf(ck, ck_ref) <= 1e-4
    assert rel_inf(o, ref["o"]) <= 2e-2 and rel_inf(ck, ref["w_ckpt"]) <= 2e-2


@pytest.mark.gpu
@pytest.mark.parametrize("dtype_name", ["fp32", "bf16"])
def test_gpu_gcs_per_matrix_rates_equals_forward(dtype_name):
    """Rates [T, H, 3] at head_dim 64: each shard's gradient carries its own
    three rates, so the split loop still equals the unsharded forward."""
    import torch
    dtype = torch.bfloat16 if dtype_name == "bf16" else torch.float32
    o, ck, o_ref, ck_ref, ref = _gpu_gcs(dtype, 2, 64, 128, [300, 129, 77], [137, 0, 40], 7, per_matrix=True)
    tol = 1e-5 if dtype_name == "fp32" else 5e-3
    assert rel_inf(o, o_ref) <= tol
    assert rel_inf(ck, ck_ref) <= (tol if dtype_name == "fp32" else 1e-4)
    assert rel_inf(o, ref["o"]) <= (1e-5 if dtype_name == "fp32" else 2e-2)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype_name", ["fp32", "bf16"])
def test_gpu_gcs_mse_equals_forward(dtype_name):
    """The squared-error loss: each shard's partial gradient takes its own
    residuals v - f_W(k) at the shared weights, so the split loop still
    equals the unsharded forward."""
    import torch
    dtype = torch.bfloat16 if dtype_name == "bf16" else torch.float32
    o, ck, o_ref, ck_ref, ref = _gpu_gcs(dtype, 2, 64, 128, [300, 129, 77], [137, 0, 40], 8, loss="mse")
    tol = 1e-5 if dtype_name == "fp32" else 5e-3
    assert rel_inf(o, o_ref) <= tol
    assert rel_inf(ck, ck_ref) <= (tol if dtype_name == "fp32" else 1e-4)
    assert rel_inf(o, ref["o"]) <= (1e-5 if dtype_name == "fp32" else 2e-2)


@pytest.mark.gpu
def test_gpu_partial_grad_sums_to_the_chunk_gradient():
    """Eq. 10 on the device: the gradients of two token shards at the same
    weights add up to the oracle's gradient of the whole chunk (FP32 path)."""
    import torch

    import paper_2604_08542_gb300 as ttt
    H, D, F, n, c = 2, 64, 128, 257, 100
    x = syn.make_inputs(n, H, D, F, seed=9)
    g = upload(x, torch.float32)
    layer = ttt.TTT(H, D, F, dtype=torch.float32)
    tot = 0
    for a, b in ((0, c), (c, n)):
        lo = syn.layout_from_lengths([[b - a]])
        tot = tot + layer.partial_grad(g["k"][a:b].clone(), g["v"][a:b].clone(),
                                       g["lr"][a:b].clone(), g["w0"], lo.chunk_offsets, lo.seq_chunk_ptr)
    torch.cuda.synchronize()
    ref = np.stack([oracle.pack(oracle.inner_gradient(oracle.unpack(x["w0"][h].astype(np.float64), D, F),
                                                      x["k"][:, h].astype(np.float64), x["v"][:, h].astype(np.float64),
                                                      x["lr"][:, h].astype(np.float64))) for h in range(H)])
    assert rel_inf(to_np(tot)[0], ref) <= 1e-5


@pytest.mark.gpu
def test_gpu_gcs_rejects_two_chunks_per_sequence():
    import torch

    import paper_2604_08542_gb300 as ttt
    layer = ttt.TTT(1, 64, 128, dtype=torch.float32)
    k = torch.zeros((20, 1, 64), device="cuda")
    lr = torch.zeros((20, 1), device="cuda")
    w = torch.zeros((1, 3 * 128 * 64), device="cuda")
    with pytest.raises(ttt.Scal3rError):
        layer.partial_grad(k, k, lr, w, [0, 10, 20], [0, 2])


@pytest.mark.gpu
def test_gpu_gcs_wide_equals_forward():
    """The split chunk step on the wide-weight path (2 heads x 256, hidden 512):
    chunks 600/257/130 tokens cut at 300/128/64."""
    import torch
    o, ck, o_ref, ck_ref, ref = _gpu_gcs(torch.bfloat16, 2, 256, 512, [600, 257, 130], [300, 128, 64], seed=7)
    assert rel_inf(o, o_ref) <= 5e-3 and rel_inf(ck, ck_ref) <= 1e-4
    assert rel_inf(o, ref["o"]) <= 2e-2 and rel_inf(ck, ref["w_ckpt"]) <= 2e-2


@pytest.mark.gpu
def test_gpu_partial_grad_wide_sums_to_the_chunk_gradient():
    """Eq. 10 at the paper's AMU shape (one head, hd 1024, hidden 4096): two
    token shards' gradients at the same weights add up to the oracle's."""
    import torch

    import paper_2604_08542_gb300 as ttt
    H, D, F, n, c = 1, 1024, 4096, 300, 129
    x = syn.make_inputs(n, H, D, F, seed=10, dtype="bf16")
    g = upload(x, torch.bfloat16)
    layer = ttt.TTT(H, D, F, dtype=torch.bfloat16)
    tot = 0
    for a, b in ((0, c), (c, n)):
        lo = syn.layout_from_lengths([[b - a]])
        tot = tot + layer.partial_grad(g["k"][a:b].clone(), g["v"][a:b].clone(),
                                       g["lr"][a:b].clone(), g["w0"], lo.chunk_offsets, lo.seq_chunk_ptr)
    torch.cuda.synchronize()
    assert layer.status() == 0
    ref = oracle.pack(oracle.inner_gradient(oracle.unpack(x["w0"][0].astype(np.float64), D, F),
                                            x["k"][:, 0].astype(np.float64), x["v"][:, 0].astype(np.float64),
                                            x["lr"][:, 0].astype(np.float64)))
    assert rel_inf(to_np(tot)[0, 0], ref) <= 2e-2


# ---------------------------------------------------------------------------
# GPU: two processes, the library's calls on each, the sum over gloo
# ---------------------------------------------------------------------------

GPU_CASES = {"fp32": (2, [300, 129, 77], [137, 0, 40], 3), "bf16": (4, [2000, 1041, 333], [1000, 513, 129], 4)}


def _gpu_worker(rank, world, port, q, dtype_name):
    import torch
    import torch.distributed as dist

    import paper_2604_08542_gb300 as ttt
    from paper_2604_08542_gb300 import distributed as ttd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        H, chunks, cuts, seed = GPU_CASES[dtype_name]
        D, F = 64, 128
        dtype = torch.bfloat16 if dtype_name == "bf16" else torch.float32
        x = syn.make_inputs(sum(chunks), H, D, F, seed=seed, dtype=dtype_name)
        # this rank's rows of every chunk: rank 0 the first cuts[j], rank 1 the rest
        idx, bounds, base, a = [], [], 0, 0
        for n, c in zip(chunks, cuts):
            lo, hi = (0, c) if rank == 0 else (c, n)
            idx.append(np.arange(base + lo, base + hi))
            bounds.append((a, a + hi - lo))
            a += hi - lo
            base += n
        loc = upload({n: np.concatenate([x[n][i] for i in idx]) for n in ("q", "k", "v", "lr")}, dtype)
        w0 = torch.from_numpy(x["w0"]).cuda()
        layer = ttt.TTT(H, D, F, dtype=dtype)

        def one_chunk(n):
            return syn.layout_from_lengths([[n]] if n > 0 else [[]])

        def partial_grad(k, v, lr, w):
            lo = one_chunk(k.shape[0])
            # row slices of [T, H] rates start at any 4-byte offset; the C ABI
            # wants 16-byte aligned tensors, so each shard piece is a fresh copy
            return layer.partial_grad(k.clone(), v.clone(), lr.clone(), w, lo.chunk_offsets, lo.seq_chunk_ptr)

        def all_reduce(g):
            t = g.float().cpu()
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            return t.cuda()

        def apply_update(w, g, w0_):
            return layer.apply_update(w, g, w0_)[0]

        def apply(qs, w):
            if qs.shape[0] == 0:
                return qs.clone()
            lo = one_chunk(qs.shape[0])
            return layer.apply(qs.clone(), w, lo.chunk_offsets, lo.seq_chunk_ptr)

        outs, w = ttd.gcs_forward(loc["q"], loc["k"], loc["v"], loc["lr"], w0, bounds, partial_grad=partial_grad,
                                  apply_update=apply_update, apply=apply, all_reduce=all_reduce)
        torch.cuda.synchronize()
        assert layer.status() == 0
        got = [None] * world
        dist.all_gather_object(got, (idx, [to_np(o) for o in outs], to_np(w)))
        if rank == 0:
            q.put(got)
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
@pytest.mark.timeout(600)
@pytest.mark.parametrize("dtype_name", ["fp32", "bf16"])
def test_gpu_gcs_two_processes_over_gloo(dtype_name):
    """Sec. 4.2, Eq. 10 across processes: two gloo ranks on the one GPU, each
    holding part of every chunk's tokens, run partial_grad on their shard,
    sum the partials over gloo on the host, then apply_update and apply.  The
    gathered outputs and weights equal the library's forward of the unsharded
    sequence (the chunk sums group the tokens differently, so up to rounding)
    and the oracle within the path's bar.  No kernel of one rank waits for the
    other: the exchange is the host all-reduce between launches."""
    import torch

    import paper_2604_08542_gb300 as ttt
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gpu_worker, args=(r, world, port, q, dtype_name)) for r in range(world)]
    for p in procs:
        p.start()
    got = _collect(q, procs, 500)
    H, chunks, cuts, seed = GPU_CASES[dtype_name]
    D, F = 64, 128
    dtype = torch.bfloat16 if dtype_name == "bf16" else torch.float32
    lay = syn.layout_from_lengths([chunks])
    x = syn.make_inputs(sum(chunks), H, D, F, seed=seed, dtype=dtype_name)
    g = upload(x, dtype)
    layer = ttt.TTT(H, D, F, dtype=dtype)
    o_ref, _, _, wf_ref = layer.forward(g["q"], g["k"], g["v"], g["lr"], g["w0"], lay.chunk_offsets,
                                        lay.seq_chunk_ptr, want_final=True)
    torch.cuda.synchronize()
    ref = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, eps=1e-6)
    o = np.full(ref["o"].shape, np.nan)
    for idx, outs, w in got:
        for i, part in zip(idx, outs):
            o[i] = part
        tol_lib, tol_w = (1e-5, 1e-5) if dtype_name == "fp32" else (5e-3, 1e-4)
        assert rel_inf(w, to_np(wf_ref)[0]) <= tol_w
        assert rel_inf(w, ref["w_final"][0]) <= (1e-5 if dtype_name == "fp32" else 2e-2)
    assert np.all(np.isfinite(o))
    tol_lib = 1e-5 if dtype_name == "fp32" else 5e-3
    assert rel_inf(o, to_np(o_ref)) <= tol_lib
    assert rel_inf(o, ref["o"]) <= (1e-5 if dtype_name == "fp32" else 2e-2)
