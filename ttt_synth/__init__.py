"""Seeded synthetic inputs for the test-time-training layer.

This module is the only code shared by the FP64 oracle side and the CUDA side
of the tests and the benchmark.  It holds no arithmetic of the method itself:
it draws random tensors, lays out ragged sequences and chunks, and rounds
values to bfloat16 bit patterns.

Random numbers come from a counter-based generator written here from its
published definitions, so that a value depends only on (seed, stream,
element index) and never on the numpy or torch version:

* SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
  number generators", OOPSLA 2014): the i-th output of a stream whose state
  starts at ``key`` is ``mix64(key + (i + 1) * 0x9E3779B97F4A7C15)``.
* Uniform doubles in (0, 1) from the top 53 bits.
* Box-Muller (G. Box, M. Muller, 1958): ``sqrt(-2 ln u1) * cos(2 pi u2)``.

Workload shapes follow the synthetic VGGT-shaped token streams that stand in
for the paper's video sequences (Sec. 5, Table 1, Table S2): a 518x392 image
at patch 14 gives 37x28 = 1036 patch tokens plus 5 special tokens, so 1041
tokens per frame; frames are grouped into chunks of a fixed frame count
(Sec. 4.1), the last chunk of a sequence may be partial.
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np

TOKENS_PER_FRAME = 1041

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids, one per drawn tensor
S_Q, S_K, S_V, S_LR, S_W0, S_DO, S_FRAMES, S_DIR, S_LR3 = range(9)


def _stream_key(seed: int, stream: int, sub: int) -> np.uint64:
    """64-bit key of one random stream: (seed, tensor stream, sub-stream)."""
    x = (int(seed) * 0x100000001B3 + int(stream) * 0x10001 + int(sub) * 0x9E37) & (2**64 - 1)
    return np.uint64(x)


def splitmix64(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream with state ``key``."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = key + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Doubles in the open interval (0, 1): (top 53 bits + 0.5) / 2^53."""
    z = splitmix64(key, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(key: np.uint64, count: int, start: int = 0) -> np.ndarray:
    """Standard normals start .. start+count-1 of the stream: Box-Muller on
    consecutive uniform pairs (normals 2i and 2i+1 come from uniforms 2i, 2i+1)."""
    p0 = start // 2
    p1 = (start + count + 1) // 2
    u = uniform01(key, 2 * p0, 2 * (p1 - p0))
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * np.pi * u[1::2]
    out = np.empty(2 * (p1 - p0), dtype=np.float64)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    o = start - 2 * p0
    return out[o:o + count]


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even).

    Returns the bfloat16 values widened back to float32 (exactly
    representable).  NaN is kept as NaN.
    """
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (b >> np.uint32(16)) & np.uint32(1)
    with np.errstate(over="ignore"):
        r = (b + np.uint32(0x7FFF) + lsb) & np.uint32(0xFFFF0000)
    nan = np.isnan(x)
    out = r.view(np.float32).copy()
    out[nan] = np.nan
    return out


def bf16_bits(x32: np.ndarray) -> np.ndarray:
    """The upper 16 bits of float32 values that are already bfloat16-exact."""
    return (np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32) >> np.uint32(16)).astype(np.uint16)


# ---------------------------------------------------------------------------
# ragged layouts
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Layout:
    """Ragged token layout of a batch of sequences cut into chunks.

    ``chunk_offsets`` [C+1] int64: token boundaries of every chunk, all
    sequences concatenated (chunk_offsets[0] = 0, chunk_offsets[C] = T).
    ``seq_chunk_ptr`` [S+1] int32: the chunks of sequence s are
    seq_chunk_ptr[s] .. seq_chunk_ptr[s+1]-1.
    """
    chunk_offsets: np.ndarray
    seq_chunk_ptr: np.ndarray

    @property
    def num_tokens(self) -> int:
        return int(self.chunk_offsets[-1])

    @property
    def num_chunks(self) -> int:
        return len(self.chunk_offsets) - 1

    @property
    def num_seqs(self) -> int:
        return len(self.seq_chunk_ptr) - 1

    def seq_range(self, s: int) -> tuple[int, int]:
        return (int(self.chunk_offsets[self.seq_chunk_ptr[s]]),
                int(self.chunk_offsets[self.seq_chunk_ptr[s + 1]]))

    def seq_chunks(self, s: int) -> list[tuple[int, int]]:
        c0, c1 = int(self.seq_chunk_ptr[s]), int(self.seq_chunk_ptr[s + 1])
        return [(int(self.chunk_offsets[c]), int(self.chunk_offsets[c + 1])) for c in range(c0, c1)]


def layout_from_lengths(seq_chunk_lengths: list[list[int]]) -> Layout:
    """Layout from explicit per-sequence chunk token counts."""
    offs = [0]
    ptr = [0]
    for chunks in seq_chunk_lengths:
        for n in chunks:
            offs.append(offs[-1] + int(n))
        ptr.append(len(offs) - 1)
    return Layout(np.asarray(offs, dtype=np.int64), np.asarray(ptr, dtype=np.int32))


def layout_from_frames(frames_per_seq: list[int], tokens_per_frame: int, chunk_frames: int) -> Layout:
    """Each sequence of f frames is cut into ceil(f / chunk_frames) chunks of
    chunk_frames frames (the last one partial)."""
    seqs = []
    for f in frames_per_seq:
        full, rem = divmod(int(f), chunk_frames)
        chunks = [chunk_frames * tokens_per_frame] * full
        if rem:
            chunks.append(rem * tokens_per_frame)
        seqs.append(chunks)
    return layout_from_lengths(seqs)


def ragged_frames(seed: int, num_seqs: int, lo: int, hi: int) -> list[int]:
    """Frame counts drawn uniformly from the integers lo..hi (inclusive)."""
    u = uniform01(_stream_key(seed, S_FRAMES, 0), 0, num_seqs)
    return [int(lo + min(hi - lo, int(x * (hi - lo + 1)))) for x in u]


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    frames: list[int]
    tokens_per_frame: int
    chunk_frames: int
    heads: int
    head_dim: int
    hidden: int
    dtype: str            # "fp32" or "bf16" (dtype of q, k, v, o)
    backward: bool
    description: str

    def layout(self) -> Layout:
        return layout_from_frames(self.frames, self.tokens_per_frame, self.chunk_frames)


def workload(name: str, seed: int = 0) -> Workload:
    """The workloads of the layer's benchmark suite, by name."""
    if name == "fp32_small":
        return Workload(name, [8], 128, 1, 1, 64, 128, "fp32", False,
                        "1 seq x 8 frames x 128 tokens, 1 head, D=64, F=128, chunk 128 tokens, FP32")
    if name == "bf16_vggt64":
        return Workload(name, [64], TOKENS_PER_FRAME, 16, 16, 64, 128, "bf16", False,
                        "1 seq x 64 frames x 1041 tokens, 16 heads x 64, F=128, chunk 16 frames, BF16 q/k/v, float32 "
                        "fast weights")
    if name == "bf16_fwdbwd_2x32":
        return Workload(name, [32, 32], TOKENS_PER_FRAME, 8, 16, 64, 128, "bf16", True,
                        "2 seqs x 32 frames x 1041 tokens, 16 heads x 64, F=128, chunk 8 frames, BF16 fwd+bwd")
    if name == "bf16_ragged24":
        return Workload(name, ragged_frames(seed, 24, 8, 200), TOKENS_PER_FRAME, 16, 16, 64, 128, "bf16", False,
                        "24 seqs, frames ~ U{8..200}, 1041 tokens/frame, 16 heads x 64, F=128, chunk 16 frames, BF16")
    if name == "bf16_long2000":
        return Workload(name, [2000], TOKENS_PER_FRAME, 32, 16, 64, 128, "bf16", False,
                        "1 seq x 2000 frames x 1041 tokens, 16 heads x 64, F=128, chunk 32 frames, BF16 forward")
    if name == "bf16_window256":
        return Workload(name, [256], TOKENS_PER_FRAME, 32, 16, 64, 128, "bf16", True,
                        "1 seq x 256 frames x 1041 tokens, 16 heads x 64, F=128, chunk 32 frames, BF16 fwd+bwd")
    if name == "bf16_amu1024":
        return Workload(name, [64], TOKENS_PER_FRAME, 16, 1, 1024, 4096, "bf16", False,
                        "1 seq x 64 frames x 1041 tokens, 1 head x 1024 (the paper's AMU), F=4096 (k=4), "
                        "chunk 16 frames, BF16 forward")
    raise KeyError(name)


WORKLOADS = ["fp32_small", "bf16_vggt64", "bf16_fwdbwd_2x32", "bf16_ragged24", "bf16_long2000", "bf16_window256",
             "bf16_amu1024"]


# ---------------------------------------------------------------------------
# tensors
# ---------------------------------------------------------------------------

def _per_head_normals(seed: int, stream: int, T: int, H: int, D: int, heads, t0: int = 0) -> np.ndarray:
    """[T, len(heads), D] normals of tokens t0 .. t0+T-1; head h draws from its
    own sub-stream, so a single head (or token range) can be regenerated
    without the others.  Heads are drawn on a thread pool (numpy releases the
    GIL in its array loops)."""
    out = np.empty((T, len(heads), D), dtype=np.float32)

    def one(j_h):
        j, h = j_h
        out[:, j, :] = normal(_stream_key(seed, stream, h), T * D, start=t0 * D).reshape(T, D)

    if len(heads) > 1 and T * D > 65536:
        import concurrent.futures as cf
        with cf.ThreadPoolExecutor(max_workers=min(len(heads), os.cpu_count() or 1)) as ex:
            list(ex.map(one, enumerate(heads)))
    else:
        for jh in enumerate(heads):
            one(jh)
    return out


def _l2_rows(x: np.ndarray) -> np.ndarray:
    """Normalise the last axis to unit L2 norm (per token and head)."""
    n = np.sqrt(np.sum(x.astype(np.float64) ** 2, axis=-1, keepdims=True))
    return (x / np.maximum(n, 1e-30)).astype(np.float32)


def make_inputs(T: int, H: int, D: int, F: int, seed: int = 0, dtype: str = "fp32",
                heads=None, lr_max: float = 0.1, with_grad_out: bool = False,
                w0_std: float = 0.125, tokens=None) -> dict:
    """Seeded inputs of one batch.

    q, k, v: [T, H', D] float32, N(0,1) per element then L2-normalised per
    (token, head) over D; rounded to bfloat16 when dtype == "bf16" (the
    float32 arrays then hold the exact bfloat16 values).
    lr:      [T, H'] float32, U[0, lr_max].
    w0:      [H', 2*F*D + D*F] float32, N(0, w0_std^2), packed W1 [F,D], W3 [F,D], W2 [D,F].
    d_o:     [T, H', D] float32 N(0,1) (bfloat16-rounded for "bf16") if with_grad_out.
    ``heads`` selects a subset of heads (default: all H); values for head h
    do not depend on which other heads are generated.  ``tokens`` = (a, b)
    draws only tokens a .. b-1 of the T-token batch (the same values as the
    full draw); T is then the batch size and the arrays have b - a rows.
    """
    heads = list(range(H)) if heads is None else list(heads)
    a, b = (0, T) if tokens is None else (int(tokens[0]), int(tokens[1]))
    n = b - a
    out = {}
    for name, st in (("q", S_Q), ("k", S_K), ("v", S_V)):
        x = _l2_rows(_per_head_normals(seed, st, n, H, D, heads, t0=a))
        out[name] = round_bf16(x) if dtype == "bf16" else x
    lr = np.empty((n, len(heads)), dtype=np.float32)
    for j, h in enumerate(heads):
        lr[:, j] = (uniform01(_stream_key(seed, S_LR, h), a, n) * lr_max).astype(np.float32)
    out["lr"] = lr
    P = 3 * F * D
    w0 = np.empty((len(heads), P), dtype=np.float32)
    for j, h in enumerate(heads):
        w0[j] = (normal(_stream_key(seed, S_W0, h), P) * w0_std).astype(np.float32)
    out["w0"] = w0
    if with_grad_out:
        g = _per_head_normals(seed, S_DO, n, H, D, heads, t0=a)
        out["d_o"] = round_bf16(g) if dtype == "bf16" else g
    return out


def per_matrix_lr(seed: int, T: int, H: int, lr_max: float = 0.1) -> np.ndarray:
    """Seeded per-matrix learning rates [T, H, 3] float32, U[0, lr_max]; the
    three rates of a (token, head) are those of W1, W3, W2, drawn from their
    own streams (one per head and matrix)."""
    lr = np.empty((T, H, 3), dtype=np.float32)
    for h in range(H):
        for j in range(3):
            lr[:, h, j] = (uniform01(_stream_key(seed, S_LR3, 3 * h + j), 0, T) * lr_max).astype(np.float32)
    return lr


def random_direction(seed: int, shape, sub: int = 0) -> np.ndarray:
    """A seeded N(0,1) array of the given shape (finite-difference directions)."""
    n = int(np.prod(shape))
    return normal(_stream_key(seed, S_DIR, sub), n).reshape(shape)
