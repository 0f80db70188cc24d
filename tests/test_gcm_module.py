"""The GCM module around the layer (Sec. 4.1, Eq. 5) through the C ABI: the
projections on the tcgen05 GEMM with the row work in their epilogues, the
remaining row steps, and the layer, forward and backward, against the FP64
oracle on the same bf16-rounded tensors (GPU).

Bar: normwise relative error <= 2e-2 (the BF16 bar) on out and on every
gradient (x, Wqkv, bqkv, w_eta, b_eta, Wo, alpha, w0)."""
import numpy as np
import pytest

import oracle
import ttt_synth as syn
from _util import rel_inf, to_np

pytestmark = pytest.mark.gpu

TOL = 2e-2
BASE = 0.1


def _bf(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


def _case(H, D, F, lengths, seed):
    import torch
    from paper_2604_08542_gb300.gcm import GCM
    rng = np.random.default_rng(seed)
    lay = syn.layout_from_lengths(lengths)
    T, d = lay.num_tokens, H * D
    host = {"x": _bf(rng.normal(size=(T, d))), "wqkv": _bf(rng.normal(size=(3 * d, d)) / np.sqrt(d)),
            "wo": _bf(rng.normal(size=(d, d)) / np.sqrt(d)), "d_out": _bf(rng.normal(size=(T, d)))}
    f32 = {"bqkv": 0.1 * rng.normal(size=3 * d), "w_eta": 0.3 / np.sqrt(d) * rng.normal(size=(H, d)),
           "b_eta": -1.0 + 0.1 * rng.normal(size=H), "alpha": 0.5 * rng.normal(size=d),
           "w0": 0.125 * rng.normal(size=(H, 3 * F * D))}
    g = {n: t.cuda() for n, t in host.items()}
    g.update({n: torch.from_numpy(a.astype(np.float32)).cuda() for n, a in f32.items()})
    m = GCM(H, D, F, base_lr=BASE)
    out, saved = m.forward(g["x"], g["wqkv"], g["bqkv"], g["w_eta"], g["b_eta"], g["wo"], g["alpha"], g["w0"],
                           lay.chunk_offsets, lay.seq_chunk_ptr)
    grads = m.backward(saved, g["d_out"])
    torch.cuda.synchronize()
    assert m.ttt.status() == 0
    ref = {n: host[n].float().numpy().astype(np.float64) for n in host}
    ref.update({n: f32[n].astype(np.float32).astype(np.float64) for n in f32})
    args = (ref["x"], ref["wqkv"], ref["bqkv"], ref["w_eta"], ref["b_eta"], BASE, ref["wo"], ref["alpha"], ref["w0"],
            lay)
    fo = oracle.gcm_forward(*args, H, D, F, eps=1e-6)
    bo = oracle.gcm_backward(*args, ref["d_out"], H, D, F, eps=1e-6)
    errs = {"out": rel_inf(to_np(out), fo["out"])}
    for n, t in zip(("dx", "dwqkv", "dbqkv", "dw_eta", "db_eta", "dwo", "dalpha", "dw0"), grads):
        errs[n] = rel_inf(to_np(t), bo[n])
    bad = {n: e for n, e in errs.items() if not e <= TOL}
    assert not bad, f"above {TOL}: {bad}; all {errs}"
    return errs


def test_gcm_module_sixteen_heads_of_64():
    """d = 1024 as 16 heads x 64 (the fused per-head layer), two sequences."""
    _case(16, 64, 128, [[300, 129], [77]], seed=61)


def test_gcm_module_wide_heads():
    """d = 512 as 2 heads x 256 (the wide-weight layer), one sequence of two chunks."""
    _case(2, 256, 512, [[300, 200]], seed=62)


def test_gcm_module_four_heads_one_token_chunk():
    """d = 256 as 4 heads x 64, a one-token chunk and a ragged tail."""
    _case(4, 64, 128, [[1], [200, 3]], seed=63)


@pytest.mark.parametrize("M,N,K,a_kmajor,b_kmajor", [(64, 1024, 8192, 0, 0), (1024, 512, 4100, 0, 0),
                                                      (300, 256, 2048, 1, 1), (2560, 1024, 16384, 0, 0)])
def test_gemm_split_k_matches_reference(M, N, K, a_kmajor, b_kmajor):
    """The GEMM entry point on weight-gradient shapes (few output tiles, long K),
    where it runs in K ranges with a fixed-order sum: against an FP64 product of
    the same bf16 operands, against the unsplit run, accumulating into C, and
    bitwise equal run to run.  2560 x 1024 has 80 output tiles, more than half
    the SMs: the range count comes from the estimate of rounds of work and
    plane traffic, which splits it (one wave of 80 tiles leaves 72 SMs idle
    for the whole K loop)."""
    import torch
    import paper_2604_08542_gb300 as ttt
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn((M, K), generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), generator=g).to(torch.bfloat16)
    ref = A.double() @ B.double().T
    a_dev = (A if a_kmajor else A.T.contiguous()).cuda()
    b_dev = (B if b_kmajor else B.T.contiguous()).cuda()
    lda = K if a_kmajor else M
    ldb = K if b_kmajor else N
    layer = ttt.TTT(1, 256, 256, dtype=torch.bfloat16)
    h = layer.handle
    st = torch.cuda.current_stream().cuda_stream
    nbytes = ttt.scal3r_ttt_gemm_workspace_size(h, M, N, K, True)
    if M <= 128 or M * N <= 512 * 1024 or (M, N) == (2560, 1024):
        assert nbytes > 0          # these shapes take the split path
    ws = torch.empty(max(nbytes, 16), dtype=torch.uint8, device="cuda")

    def run(c, accumulate, use_ws):
        rc = ttt.scal3r_ttt_gemm(h, a_dev.data_ptr(), lda, a_kmajor, b_dev.data_ptr(), ldb, b_kmajor, c.data_ptr(), N,
                                 1, accumulate, M, N, K, ws.data_ptr() if use_ws else None,
                                 nbytes if use_ws else 0, st)
        assert rc == 0

    c1 = torch.empty((M, N), dtype=torch.float32, device="cuda")
    c2 = torch.empty_like(c1)
    c3 = torch.empty_like(c1)
    run(c1, 0, True)
    run(c2, 0, True)
    run(c3, 0, False)
    base = torch.full((M, N), 0.5, dtype=torch.float32, device="cuda")
    run(base, 1, True)
    torch.cuda.synchronize()
    assert layer.status() == 0
    # float32 accumulation on the tensor cores over up to 8,192 K steps: within
    # 5e-5 of the largest entry (bf16 rounding of the operands is not involved:
    # the reference multiplies the same bf16 values)
    scale = ref.abs().max().item()
    for c in (c1, c3):
        err = (c.cpu().double() - ref).abs().max().item() / scale
        assert err < 5e-5, err
    assert torch.equal(c1, c2)
    assert (base.cpu().double() - 0.5 - ref).abs().max().item() / scale < 5e-5
