"""Helpers shared by the tests (test-only)."""
from __future__ import annotations

import numpy as np


def rel_inf(x, ref) -> float:
    """Normwise relative error max|x - ref| / max|ref| (max-abs if ref is 0)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if x.size == 0:
        return 0.0
    d = np.max(np.abs(x - ref))
    s = np.max(np.abs(ref))
    return float(d / s) if s > 0 else float(d)


def to_np(t) -> np.ndarray:
    return t.detach().float().cpu().numpy().astype(np.float64)


def upload(x: dict, dtype, device="cuda"):
    """Move generator outputs to the GPU: tokens in ``dtype``, the rest float32."""
    import torch
    out = {}
    for n, a in x.items():
        t = torch.from_numpy(np.ascontiguousarray(a))
        if n in ("q", "k", "v", "d_o"):
            t = t.to(dtype)
        out[n] = t.to(device).contiguous()
    return out


def device_inputs(lay, H, D, F, seed, samples=(), with_grad_out=False, lr_max=0.1):
    """Inputs of a large batch built on the GPU: seeded torch draws with the
    generator's distributions for every head, except the chains in
    ``samples`` ((sequence, head) pairs), whose token ranges hold the
    counter-based generator's values (returned per chain for the oracle).
    Chains never interact, so the sampled chains see exactly those inputs."""
    import torch
    import ttt_synth as syn
    T = lay.num_tokens
    g = torch.Generator(device="cuda")
    g.manual_seed(1000 + seed)

    def tok():
        x = torch.randn((T, H, D), generator=g, device="cuda")
        x = x / x.norm(dim=-1, keepdim=True)
        return x.to(torch.bfloat16)

    out = {"q": tok(), "k": tok(), "v": tok(),
           "lr": torch.rand((T, H), generator=g, device="cuda") * lr_max,
           "w0": torch.from_numpy(syn.make_inputs(1, H, D, F, seed=seed)["w0"]).cuda()}
    if with_grad_out:
        out["d_o"] = torch.randn((T, H, D), generator=g, device="cuda").to(torch.bfloat16)
    host = {}
    for s, h in samples:
        a, b = lay.seq_range(s)
        x = syn.make_inputs(T, H, D, F, seed=seed, dtype="bf16", heads=[h], tokens=(a, b),
                            with_grad_out=with_grad_out, lr_max=lr_max)
        for n in ("q", "k", "v", "d_o"):
            if n in x:
                out[n][a:b, h] = torch.from_numpy(x[n][:, 0]).to(torch.bfloat16).cuda()
        out["lr"][a:b, h] = torch.from_numpy(x["lr"][:, 0]).cuda()
        x["w0"] = out["w0"][h:h + 1].cpu().numpy()
        host[(s, h)] = x
    return out, host


def seq_layout(lay, s):
    """Single-sequence layout of sequence s of a batch layout."""
    import ttt_synth as syn
    return syn.layout_from_lengths([[t1 - t0 for t0, t1 in lay.seq_chunks(s)]])
