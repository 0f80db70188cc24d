"""Host-side logic for running the layer on several GPUs (one process each).

The layer's chains (sequence, head) are independent, so a batch of
sequences shards across ranks with no exchange on the data path: every rank
runs its own sequences (longest first onto the least-loaded rank) and the
results are gathered only if the caller needs them.  Throughput timing takes
the maximum over ranks.

torch.distributed is the transport (NCCL on GPUs, gloo on CPU); this module
holds no arithmetic of the method.
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_sequences(seq_tokens, world: int) -> list[list[int]]:
    """Assign sequences to ranks, longest first onto the least-loaded rank.

    Returns, for every rank, the sorted list of its sequence indices.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(seq_tokens)), key=lambda s: (-int(seq_tokens[s]), s))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for s in order:
        load, r = heapq.heappop(heap)
        out[r].append(s)
        heapq.heappush(heap, (load + int(seq_tokens[s]), r))
    return [sorted(x) for x in out]


def sub_layout(chunk_offsets, seq_chunk_ptr, seqs):
    """The layout of the given sequences alone, and the global token index
    of each of its tokens (so that shard results can be scattered back)."""
    off = np.asarray(chunk_offsets, dtype=np.int64)
    ptr = np.asarray(seq_chunk_ptr, dtype=np.int32)
    new_off = [0]
    new_ptr = [0]
    idx = []
    for s in seqs:
        for c in range(int(ptr[s]), int(ptr[s + 1])):
            n = int(off[c + 1] - off[c])
            new_off.append(new_off[-1] + n)
            idx.append(np.arange(off[c], off[c + 1], dtype=np.int64))
        new_ptr.append(len(new_off) - 1)
    tokens = np.concatenate(idx) if idx else np.zeros(0, dtype=np.int64)
    return np.asarray(new_off, dtype=np.int64), np.asarray(new_ptr, dtype=np.int32), tokens


def seq_token_counts(chunk_offsets, seq_chunk_ptr) -> list[int]:
    off = np.asarray(chunk_offsets, dtype=np.int64)
    ptr = np.asarray(seq_chunk_ptr, dtype=np.int32)
    return [int(off[ptr[s + 1]] - off[ptr[s]]) for s in range(len(ptr) - 1)]


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of a per-rank float over all ranks (the value itself when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gcs_forward(q, k, v, lr, w0, chunk_bounds, *, partial_grad, apply_update, apply, all_reduce):
    """One sequence under Global Context Synchronisation (Sec. 4.2, Eq. 10):
    the tokens of every chunk are spread over the ranks, and this rank holds
    rows [a, b) of its own q, k, v, lr arrays for chunk j
    (chunk_bounds[j] = (a, b); an empty range is allowed).

    For each chunk, in order:
      G_local = partial_grad(k[a:b], v[a:b], lr[a:b], W)   this rank's tokens
      G = all_reduce(G_local)                              the sum over ranks
      W = apply_update(W, G, w0)                           the same on every rank
      o[a:b] = apply(q[a:b], W)                            this rank's queries
    and W starts at w0.  The callables are whatever computes those pieces for
    this rank (the library's calls on a GPU, or a reference); this function
    only orders them.  Returns (the list of per-chunk outputs, the final W).
    """
    w = w0
    outs = []
    for a, b in chunk_bounds:
        g = all_reduce(partial_grad(k[a:b], v[a:b], lr[a:b], w))
        w = apply_update(w, g, w0)
        outs.append(apply(q[a:b], w))
    return outs, w
