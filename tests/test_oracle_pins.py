"""Pins of the FP64 oracle to facts other than itself (CPU only).

Each test checks the oracle against something the paper or mathematics
fixes independently of the oracle's own code: library routines (torch
float64 SiLU / matmul), closed forms (linear attention, the delta rule),
central finite differences of a loss written here from Eq. 9, and
invariants of the method (Eq. 8, Eq. 10, Sec. 4.4).
"""
import numpy as np
import pytest
import torch

import oracle
import ttt_synth as syn

D, F = 4, 8


def _tiny(seed, T=15, H=1, lr_max=0.3, dtype="fp32"):
    x = syn.make_inputs(T, H, D, F, seed=seed, lr_max=lr_max, with_grad_out=True, w0_std=0.5)
    return x


def _layout_2seq():
    # two sequences, 3 chunks each, ragged (5,4,6) and (3,5,2) tokens
    return syn.layout_from_lengths([[5, 4, 6], [3, 5, 2]])


def _torch_f(W1, W3, W2, X):
    """SwiGLU f_W(x) = W2 (SiLU(W1 x) o (W3 x)) with torch float64 routines."""
    return torch.nn.functional.silu(X @ W1.T) * (X @ W3.T) @ W2.T


# ---------------------------------------------------------------------------
# elementwise pieces against a library routine
# ---------------------------------------------------------------------------

def test_silu_and_derivatives_against_torch():
    z = np.linspace(-30, 30, 2001)
    zt = torch.tensor(z, dtype=torch.float64, requires_grad=True)
    y = torch.nn.functional.silu(zt)
    np.testing.assert_allclose(oracle.silu(z), y.detach().numpy(), rtol=1e-14, atol=1e-300)
    (g,) = torch.autograd.grad(y.sum(), zt, create_graph=True)
    np.testing.assert_allclose(oracle.silu_prime(z), g.detach().numpy(), rtol=1e-12, atol=1e-14)
    (g2,) = torch.autograd.grad(g.sum(), zt)
    np.testing.assert_allclose(oracle.silu_second(z), g2.numpy(), rtol=1e-10, atol=1e-13)


# ---------------------------------------------------------------------------
# P1: learning rate 0 -> plain MLP, weights unchanged
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("norm", ["row_w0", "none"])
def test_lr_zero_is_plain_mlp(norm):
    lay = _layout_2seq()
    T = lay.num_tokens
    x = syn.make_inputs(T, 2, D, F, seed=1)
    lr = np.zeros_like(x["lr"])
    out = oracle.forward(x["q"], x["k"], x["v"], lr, x["w0"], lay, D, F, norm=norm)
    for h in range(2):
        w = torch.tensor(x["w0"][h], dtype=torch.float64)
        W1, W3, W2 = w[:F * D].view(F, D), w[F * D:2 * F * D].view(F, D), w[2 * F * D:].view(D, F)
        ref = _torch_f(W1, W3, W2, torch.tensor(x["q"][:, h], dtype=torch.float64)).numpy()
        np.testing.assert_allclose(out["o"][:, h], ref, rtol=1e-13, atol=1e-15)
        for s in range(2):
            assert np.array_equal(out["w_final"][s, h], x["w0"][h].astype(np.float64))


# ---------------------------------------------------------------------------
# P2: linear model + dot loss + no norm == chunk-causal linear attention
# ---------------------------------------------------------------------------

def test_linear_dot_is_chunk_causal_linear_attention():
    lay = syn.layout_from_lengths([[7, 3, 9, 1], [4, 4]])
    T = lay.num_tokens
    H = 2
    x = syn.make_inputs(T, H, D, F, seed=2)
    w0 = (syn.random_direction(5, (H, D * D)) * 0.3).astype(np.float32)
    out = oracle.forward(x["q"], x["k"], x["v"], x["lr"], w0, lay, D, F,
                         norm="none", model="linear")
    for s in range(lay.num_seqs):
        a, b = lay.seq_range(s)
        cid = np.zeros(b - a, dtype=int)
        for j, (t0, t1) in enumerate(lay.seq_chunks(s)):
            cid[t0 - a:t1 - a] = j
        mask = (cid[None, :] <= cid[:, None]).astype(np.float64)   # key chunk <= query chunk
        for h in range(H):
            Q = x["q"][a:b, h].astype(np.float64)
            K = x["k"][a:b, h].astype(np.float64)
            V = x["v"][a:b, h].astype(np.float64)
            eta = x["lr"][a:b, h].astype(np.float64)
            W0 = w0[h].astype(np.float64).reshape(D, D)
            scores = (Q @ K.T) * mask * eta[None, :]
            ref = Q @ W0.T + scores @ V
            np.testing.assert_allclose(out["o"][a:b, h], ref, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------------------
# P3: linear model + MSE + no norm == chunkwise delta rule
# ---------------------------------------------------------------------------

def test_linear_mse_is_chunkwise_delta_rule():
    lay = syn.layout_from_lengths([[6, 5, 8]])
    T = lay.num_tokens
    x = syn.make_inputs(T, 1, D, F, seed=3)
    w0 = (syn.random_direction(6, (1, D * D)) * 0.3).astype(np.float32)
    out = oracle.forward(x["q"], x["k"], x["v"], x["lr"], w0, lay, D, F,
                         loss="mse", norm="none", model="linear")
    W = w0[0].astype(np.float64).reshape(D, D)
    for c, (t0, t1) in enumerate(lay.seq_chunks(0)):
        K = x["k"][t0:t1, 0].astype(np.float64)
        V = x["v"][t0:t1, 0].astype(np.float64)
        eta = x["lr"][t0:t1, 0].astype(np.float64)
        W = W @ (np.eye(D) - (K.T * eta) @ K) + (V.T * eta) @ K
        np.testing.assert_allclose(out["w_ckpt"][c, 0].reshape(D, D), W, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------
# P4: inner gradient == central finite differences of the Eq. 9 loss
# ---------------------------------------------------------------------------

def _loss_torch(w, K, V, eta, loss):
    W1, W3, W2 = w[:F * D].view(F, D), w[F * D:2 * F * D].view(F, D), w[2 * F * D:].view(D, F)
    Y = _torch_f(W1, W3, W2, K)
    if loss == "dot":
        per = -(Y * V).sum(1)                 # Eq. 9: -f_W(k)^T v
    else:
        per = 0.5 * ((Y - V) ** 2).sum(1)
    return float((eta * per).sum())


@pytest.mark.parametrize("loss", ["dot", "mse"])
def test_inner_gradient_matches_finite_differences(loss):
    x = syn.make_inputs(5, 1, D, F, seed=4, w0_std=0.5)
    K = torch.tensor(x["k"][:, 0], dtype=torch.float64)
    V = torch.tensor(x["v"][:, 0], dtype=torch.float64)
    eta = torch.tensor(x["lr"][:, 0], dtype=torch.float64)
    w = torch.tensor(x["w0"][0], dtype=torch.float64)
    G = oracle.pack(oracle.inner_gradient(oracle.unpack(w.numpy(), D, F), K.numpy(), V.numpy(),
                                          eta.numpy(), loss))
    h = 1e-6
    fd = np.zeros_like(G)
    for i in range(w.numel()):
        wp = w.clone(); wp[i] += h
        wm = w.clone(); wm[i] -= h
        fd[i] = (_loss_torch(wp, K, V, eta, loss) - _loss_torch(wm, K, V, eta, loss)) / (2 * h)
    np.testing.assert_allclose(G, fd, rtol=1e-6, atol=1e-9)


def test_update_descends_the_dot_loss():
    """Eq. 8 subtracts the gradient: a small step lowers the chunk's loss (sign pin)."""
    x = syn.make_inputs(9, 1, D, F, seed=7, lr_max=0.01, w0_std=0.5)
    lay = syn.layout_from_lengths([[9]])
    out = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, norm="none")
    K = torch.tensor(x["k"][:, 0], dtype=torch.float64)
    V = torch.tensor(x["v"][:, 0], dtype=torch.float64)
    eta = torch.tensor(x["lr"][:, 0], dtype=torch.float64)
    before = _loss_torch(torch.tensor(x["w0"][0], dtype=torch.float64), K, V, eta, "dot")
    after = _loss_torch(torch.tensor(out["w_final"][0, 0]), K, V, eta, "dot")
    assert after < before


# ---------------------------------------------------------------------------
# P5: full backward == central finite differences of <dO, o>
# ---------------------------------------------------------------------------

def _objective(inp, lay, d_o, loss, norm, model):
    out = oracle.forward(inp["q"], inp["k"], inp["v"], inp["lr"], inp["w0"], lay, D, F,
                         loss=loss, norm=norm, model=model)
    return float(np.sum(out["o"] * d_o))


@pytest.mark.parametrize("loss,norm,model,lr_max", [
    ("dot", "row_w0", "swiglu", 0.3),
    ("dot", "none", "swiglu", 0.3),
    ("mse", "row_w0", "swiglu", 0.3),
    ("mse", "none", "swiglu", 0.03),
    ("dot", "unit", "swiglu", 0.3),
    ("dot", "none", "linear", 0.3),
    ("mse", "none", "linear", 0.1),
])
def test_backward_matches_finite_differences(loss, norm, model, lr_max):
    lay = _layout_2seq()
    T = lay.num_tokens
    H = 1
    x = _tiny(11, T=T, H=H, lr_max=lr_max)
    inp = {n: x[n].astype(np.float64) for n in ("q", "k", "v", "lr")}
    if model == "linear":
        inp["w0"] = syn.random_direction(12, (H, D * D)) * 0.3
    else:
        inp["w0"] = x["w0"].astype(np.float64)
    d_o = x["d_o"].astype(np.float64)
    g = oracle.backward(inp["q"], inp["k"], inp["v"], inp["lr"], inp["w0"], lay, d_o, D, F,
                        loss=loss, norm=norm, model=model)
    names = {"q": "dq", "k": "dk", "v": "dv", "lr": "dlr", "w0": "dw0"}
    h = 1e-6
    for n, gn in names.items():
        base = inp[n]
        fd = np.zeros_like(base)
        flat = base.reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            fp = _objective(inp, lay, d_o, loss, norm, model)
            flat[i] = old - h
            fm = _objective(inp, lay, d_o, loss, norm, model)
            flat[i] = old
            fd.reshape(-1)[i] = (fp - fm) / (2 * h)
        scale = max(1.0, np.max(np.abs(fd)))
        err = np.max(np.abs(g[gn] - fd)) / scale
        assert err < 2e-7, (n, err)


# ---------------------------------------------------------------------------
# P5b: the clamp branch of the row rescale (reading A8: max(||row||, eps))
# ---------------------------------------------------------------------------

def clamp_eps(inp, lay, loss, norm, margin=1e-3):
    """An eps that some pre-rescale row norms of the run fall below and others
    above, every norm at least `margin` (relative) away from it.  The run is
    redone with each candidate, since clamping changes the later chunks."""
    base = oracle.forward(inp["q"], inp["k"], inp["v"], inp["lr"], inp["w0"], lay, D, F, loss=loss, norm=norm)
    qs = np.quantile(base["wnorm"], np.linspace(0.2, 0.8, 25))
    for eps in qs * (1.0 + margin * 3):
        out = oracle.forward(inp["q"], inp["k"], inp["v"], inp["lr"], inp["w0"], lay, D, F, loss=loss,
                             norm=norm, eps=eps)
        n = out["wnorm"].reshape(-1)
        if np.any(n < eps) and np.any(n > eps) and np.min(np.abs(n - eps)) > margin * eps:
            return float(eps)
    raise AssertionError("no eps with a margin")


def _fd_check(inp, lay, d_o, loss, norm, eps, h=1e-6, tol=2e-7, kink=()):
    """The oracle's backward against central differences of <dO, o> for all
    five inputs.  Entries of w0 listed in `kink` sit at a zero row, where
    the target norm is |h| on either side: there the difference has an O(h)
    term, so those entries are checked to converge to the backward's value
    linearly in h instead."""
    g = oracle.backward(inp["q"], inp["k"], inp["v"], inp["lr"], inp["w0"], lay, d_o, D, F,
                        loss=loss, norm=norm, eps=eps)

    def obj():
        out = oracle.forward(inp["q"], inp["k"], inp["v"], inp["lr"], inp["w0"], lay, D, F, loss=loss,
                             norm=norm, eps=eps)
        return float(np.sum(out["o"] * d_o))

    def cdiff(flat, i, step):
        old = flat[i]
        flat[i] = old + step
        fp = obj()
        flat[i] = old - step
        fm = obj()
        flat[i] = old
        return (fp - fm) / (2 * step)
    names = {"q": "dq", "k": "dk", "v": "dv", "lr": "dlr", "w0": "dw0"}
    for n, gn in names.items():
        flat = inp[n].reshape(-1)
        ref = g[gn].reshape(-1)
        skip = set(kink) if n == "w0" else set()
        fd = np.array([cdiff(flat, i, h) if i not in skip else ref[i] for i in range(flat.size)])
        scale = max(1.0, np.max(np.abs(fd)))
        err = np.max(np.abs(ref - fd)) / scale
        assert err < tol, (n, err)
        for i in sorted(skip):
            e7, e8 = abs(cdiff(flat, i, 1e-7) - ref[i]), abs(cdiff(flat, i, 1e-8) - ref[i])
            assert e8 < 2e-6 * scale and e8 < 0.3 * e7 + 1e-7 * scale, (i, e7, e8)


@pytest.mark.parametrize("loss,norm", [("dot", "row_w0"), ("mse", "row_w0"), ("dot", "unit")])
def test_backward_with_clamped_rows_matches_finite_differences(loss, norm):
    """Rows whose norm after the gradient step is below eps are rescaled by
    rho / eps (R = (rho / eps) lambda, drho = w~ . lambda / eps); rows above it
    by rho / ||row||.  A run with both kinds of rows, every norm away from
    eps, against central differences of <dO, o> for all five inputs."""
    lay = _layout_2seq()
    x = _tiny(21, T=lay.num_tokens, H=1, lr_max=0.3)
    inp = {n: x[n].astype(np.float64) for n in ("q", "k", "v", "lr", "w0")}
    eps = clamp_eps(inp, lay, loss, norm)
    out = oracle.forward(inp["q"], inp["k"], inp["v"], inp["lr"], inp["w0"], lay, D, F, loss=loss, norm=norm,
                         eps=eps)
    # the clamped rows' norm is rho * ||w~|| / eps, not rho
    n = out["wnorm"][0, 0]
    W = oracle.unpack(out["w_ckpt"][0, 0], D, F)
    rows = np.concatenate([np.sqrt(np.sum(m * m, axis=1)) for m in W])
    rho = (np.concatenate([np.sqrt(np.sum(m * m, axis=1)) for m in oracle.unpack(inp["w0"][0], D, F)])
           if norm == "row_w0" else np.ones_like(n))
    np.testing.assert_allclose(rows, rho * np.minimum(n / eps, 1.0), rtol=1e-12)
    _fd_check(inp, lay, x["d_o"].astype(np.float64), loss, norm, eps)


def test_backward_with_a_zero_initial_row_matches_finite_differences():
    """A row of W0 that is zero has target 0: the row stays zero, and its
    target contributes nothing to dW0 (the central difference of |h| is 0)."""
    lay = _layout_2seq()
    x = _tiny(23, T=lay.num_tokens, H=1, lr_max=0.3)
    inp = {n: x[n].astype(np.float64) for n in ("q", "k", "v", "lr", "w0")}
    inp["w0"][0, 3 * D:4 * D] = 0.0          # row 3 of W1
    inp["w0"][0, 2 * F * D + F:2 * F * D + 2 * F] = 0.0           # row 1 of W2
    out = oracle.forward(inp["q"], inp["k"], inp["v"], inp["lr"], inp["w0"], lay, D, F)
    for c in range(lay.num_chunks):
        W = oracle.unpack(out["w_ckpt"][c, 0], D, F)
        assert np.all(W[0][3] == 0.0) and np.all(W[2][1] == 0.0)
    kink = list(range(3 * D, 4 * D)) + list(range(2 * F * D + F, 2 * F * D + 2 * F))
    _fd_check(inp, lay, x["d_o"].astype(np.float64), "dot", "row_w0", 1e-12, kink=kink)


# ---------------------------------------------------------------------------
# per-matrix learning rates: G_j = d/dW_j sum_i eta_{j,i} L_i
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("loss", ["dot", "mse"])
def test_per_matrix_inner_gradient_matches_finite_differences(loss):
    """Each matrix's block is the central difference of the loss weighted by
    that matrix's own rates (W1: eta[:, 0], W3: eta[:, 1], W2: eta[:, 2])."""
    x = syn.make_inputs(5, 1, D, F, seed=4, w0_std=0.5)
    K = torch.tensor(x["k"][:, 0], dtype=torch.float64)
    V = torch.tensor(x["v"][:, 0], dtype=torch.float64)
    eta3 = syn.per_matrix_lr(21, 5, 1, lr_max=0.5)[:, 0].astype(np.float64)
    w = torch.tensor(x["w0"][0], dtype=torch.float64)
    G = oracle.pack(oracle.inner_gradient(oracle.unpack(w.numpy(), D, F), K.numpy(), V.numpy(), eta3, loss))
    h = 1e-6
    fd = np.zeros_like(G)
    for i in range(w.numel()):
        j = min(i // (F * D), 2)            # packed W1, W3, W2 blocks of F*D each
        eta = torch.tensor(eta3[:, j])
        wp = w.clone(); wp[i] += h
        wm = w.clone(); wm[i] -= h
        fd[i] = (_loss_torch(wp, K, V, eta, loss) - _loss_torch(wm, K, V, eta, loss)) / (2 * h)
    np.testing.assert_allclose(G, fd, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("loss", ["dot", "mse"])
def test_equal_per_matrix_rates_reduce_to_one_rate(loss):
    lay = _layout_2seq()
    x = _tiny(31, T=lay.num_tokens, H=2)
    lr3 = np.repeat(x["lr"][..., None], 3, axis=2)
    a = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, loss=loss)
    b = oracle.forward(x["q"], x["k"], x["v"], lr3, x["w0"], lay, D, F, loss=loss)
    for n in ("o", "w_ckpt", "wnorm", "w_final"):
        np.testing.assert_allclose(b[n], a[n], rtol=1e-12, atol=1e-14)
    ga = oracle.backward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, x["d_o"], D, F, loss=loss)
    gb = oracle.backward(x["q"], x["k"], x["v"], lr3, x["w0"], lay, x["d_o"], D, F, loss=loss)
    for n in ("dq", "dk", "dv", "dw0"):
        np.testing.assert_allclose(gb[n], ga[n], rtol=1e-10, atol=1e-13)
    assert gb["dlr"].shape == lr3.shape
    np.testing.assert_allclose(gb["dlr"].sum(-1), ga["dlr"], rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("zero", [0, 1, 2])
def test_zero_rate_leaves_its_matrix(zero):
    """With no row normalisation, a matrix whose rates are all zero keeps its
    weights through every update while the others move (index pin)."""
    lay = syn.layout_from_lengths([[6, 5]])
    x = _tiny(32, T=lay.num_tokens)
    lr3 = syn.per_matrix_lr(33, lay.num_tokens, 1, lr_max=0.3)
    lr3[:, :, zero] = 0.0
    out = oracle.forward(x["q"], x["k"], x["v"], lr3, x["w0"], lay, D, F, norm="none")
    before = oracle.unpack(x["w0"][0].astype(np.float64), D, F)
    after = oracle.unpack(out["w_final"][0, 0], D, F)
    for j in range(3):
        same = np.array_equal(after[j], before[j])
        assert same == (j == zero), j


@pytest.mark.parametrize("loss,norm,lr_max", [("dot", "row_w0", 0.3), ("mse", "none", 0.03)])
def test_per_matrix_backward_matches_finite_differences(loss, norm, lr_max):
    lay = _layout_2seq()
    T = lay.num_tokens
    x = _tiny(34, T=T, H=1, lr_max=lr_max)
    inp = {n: x[n].astype(np.float64) for n in ("q", "k", "v", "w0")}
    inp["lr"] = syn.per_matrix_lr(35, T, 1, lr_max=lr_max).astype(np.float64)
    d_o = x["d_o"].astype(np.float64)
    g = oracle.backward(inp["q"], inp["k"], inp["v"], inp["lr"], inp["w0"], lay, d_o, D, F, loss=loss, norm=norm)
    h = 1e-6
    for n, gn in {"q": "dq", "k": "dk", "v": "dv", "lr": "dlr", "w0": "dw0"}.items():
        flat = inp[n].reshape(-1)
        fd = np.zeros(flat.size)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            fp = _objective(inp, lay, d_o, loss, norm, "swiglu")
            flat[i] = old - h
            fm = _objective(inp, lay, d_o, loss, norm, "swiglu")
            flat[i] = old
            fd[i] = (fp - fm) / (2 * h)
        scale = max(1.0, np.max(np.abs(fd)))
        err = np.max(np.abs(g[gn].reshape(-1) - fd)) / scale
        assert err < 2e-7, (n, err)


# ---------------------------------------------------------------------------
# invariants (P6 - P12)
# ---------------------------------------------------------------------------

def test_rows_keep_their_initial_norm():
    lay = _layout_2seq()
    x = _tiny(13, T=lay.num_tokens, H=2)
    out = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F)
    for h in range(2):
        W0 = oracle.unpack(x["w0"][h], D, F)
        rho = [np.sqrt((m.astype(np.float64) ** 2).sum(1)) for m in W0]
        for c in range(lay.num_chunks):
            Wc = oracle.unpack(out["w_ckpt"][c, h], D, F)
            for m, r in zip(Wc, rho):
                np.testing.assert_allclose(np.sqrt((m ** 2).sum(1)), r, rtol=1e-12)


def test_permuting_tokens_inside_a_chunk():
    lay = syn.layout_from_lengths([[6, 7, 5]])
    x = _tiny(14, T=18, H=1)
    perm = np.arange(18)
    rng = np.random.default_rng(0)
    perm[6:13] = 6 + rng.permutation(7)
    out = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F)
    xp = {n: x[n][perm] for n in ("q", "k", "v", "lr")}
    outp = oracle.forward(xp["q"], xp["k"], xp["v"], xp["lr"], x["w0"], lay, D, F)
    np.testing.assert_allclose(outp["o"], out["o"][perm], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(outp["w_final"], out["w_final"], rtol=1e-12, atol=1e-14)


def test_ragged_batch_equals_separate_chains():
    lay = _layout_2seq()
    x = _tiny(15, T=lay.num_tokens, H=3)
    out = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F)
    for s in range(lay.num_seqs):
        a, b = lay.seq_range(s)
        sub = syn.layout_from_lengths([[t1 - t0 for t0, t1 in lay.seq_chunks(s)]])
        for h in range(3):
            one = oracle.forward(x["q"][a:b, h:h + 1], x["k"][a:b, h:h + 1], x["v"][a:b, h:h + 1],
                                 x["lr"][a:b, h:h + 1], x["w0"][h:h + 1], sub, D, F)
            np.testing.assert_array_equal(one["o"][:, 0], out["o"][a:b, h])


def test_gcs_gradient_sum_over_shards():
    """Eq. 10: the chunk gradient equals the sum of the gradients of any token split."""
    x = _tiny(16, T=20, H=1)
    W = oracle.unpack(x["w0"][0], D, F)
    K, V, eta = (x[n][:, 0].astype(np.float64) for n in ("k", "v", "lr"))
    full = oracle.inner_gradient(W, K, V, eta)
    parts = [oracle.inner_gradient(W, K[a:b], V[a:b], eta[a:b]) for a, b in ((0, 3), (3, 11), (11, 20))]
    for j in range(3):
        np.testing.assert_allclose(sum(p[j] for p in parts), full[j], rtol=1e-12, atol=1e-15)


def test_streaming_resume_equals_one_pass():
    lay = syn.layout_from_lengths([[5, 4, 6, 3]])
    x = _tiny(17, T=18, H=2)
    out = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, norm="none")
    la = syn.layout_from_lengths([[5, 4]])
    lb = syn.layout_from_lengths([[6, 3]])
    a = oracle.forward(*(x[n][:9] for n in ("q", "k", "v", "lr")), x["w0"], la, D, F, norm="none")
    b = oracle.forward(*(x[n][9:] for n in ("q", "k", "v", "lr")), x["w0"], lb, D, F, norm="none",
                       w_init=a["w_final"])
    np.testing.assert_array_equal(np.concatenate([a["o"], b["o"]]), out["o"])
    np.testing.assert_array_equal(b["w_final"], out["w_final"])


@pytest.mark.parametrize("norm", ["row_w0", "unit"])
def test_streaming_resume_with_row_rescale_equals_one_pass(norm):
    # With the row rescale the resumed run takes its targets from the rows of
    # w_init: every row of w_final already has its target norm (rho for
    # row_w0, 1 for unit), so the resumed targets are the original ones up to
    # rounding and the two runs agree to rounding.
    lay = syn.layout_from_lengths([[5, 4, 6, 3]])
    x = _tiny(19, T=18, H=2)
    out = oracle.forward(x["q"], x["k"], x["v"], x["lr"], x["w0"], lay, D, F, norm=norm)
    la = syn.layout_from_lengths([[5, 4]])
    lb = syn.layout_from_lengths([[6, 3]])
    a = oracle.forward(*(x[n][:9] for n in ("q", "k", "v", "lr")), x["w0"], la, D, F, norm=norm)
    if norm == "unit":
        w_init = a["w_final"]
    else:
        # resuming under row_w0 with the original rows' norms: w_final rows
        # have exactly those norms
        w_init = a["w_final"]
        rho = [np.sqrt(np.sum(m * m, axis=1)) for m in oracle.unpack(x["w0"][0].astype(np.float64), D, F)]
        got = [np.sqrt(np.sum(m * m, axis=1)) for m in oracle.unpack(w_init[0, 0], D, F)]
        for r, g in zip(rho, got):
            np.testing.assert_allclose(g, r, rtol=1e-13)
    b = oracle.forward(*(x[n][9:] for n in ("q", "k", "v", "lr")), x["w0"], lb, D, F, norm=norm,
                       w_init=w_init)
    np.testing.assert_allclose(np.concatenate([a["o"], b["o"]]), out["o"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b["w_final"], out["w_final"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b["wnorm"], out["wnorm"][2:], rtol=1e-12)


def test_zero_lr_chunk_keeps_weights():
    lay = syn.layout_from_lengths([[5, 4, 6]])
    x = _tiny(18, T=15, H=1)
    lr = x["lr"].copy()
    lr[5:9] = 0.0
    out = oracle.forward(x["q"], x["k"], x["v"], lr, x["w0"], lay, D, F)
    # the rows of W_1 already have their target norm, so the rescale is 1 up to rounding
    np.testing.assert_allclose(out["w_ckpt"][1], out["w_ckpt"][0], rtol=1e-15, atol=1e-16)


# ---------------------------------------------------------------------------
# the input generator
# ---------------------------------------------------------------------------

def test_generator_is_deterministic_and_headwise():
    a = syn.make_inputs(50, 4, 64, 128, seed=3)
    b = syn.make_inputs(50, 4, 64, 128, seed=3, heads=[2])
    np.testing.assert_array_equal(a["k"][:, 2], b["k"][:, 0])
    np.testing.assert_array_equal(a["w0"][2], b["w0"][0])
    n = np.sqrt((a["q"].astype(np.float64) ** 2).sum(-1))
    np.testing.assert_allclose(n, 1.0, rtol=1e-6)
    assert a["lr"].min() >= 0 and a["lr"].max() <= 0.1
    z = syn.normal(syn._stream_key(0, 0, 0), 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_bf16_rounding_matches_torch():
    x = (syn.normal(syn._stream_key(1, 0, 0), 100000) * 3).astype(np.float32)
    x[:4] = [1.00390625, 1.01171875, -2.00781250, 0.0]           # ties to even cases
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(syn.round_bf16(x), ref)


def test_workload_layouts():
    w = syn.workload("bf16_vggt64")
    lay = w.layout()
    assert lay.num_tokens == 64 * 1041 and lay.num_chunks == 4
    assert int(lay.chunk_offsets[1]) == 16 * 1041
    w4 = syn.workload("bf16_long2000").layout()
    assert w4.num_chunks == 63 and int(w4.chunk_offsets[-1] - w4.chunk_offsets[-2]) == 16 * 1041
    w3 = syn.workload("bf16_ragged24")
    assert len(w3.frames) == 24 and min(w3.frames) >= 8 and max(w3.frames) <= 200


def test_generator_token_ranges_match_the_full_draw():
    full = syn.make_inputs(37, 3, 8, 16, seed=9, with_grad_out=True)
    part = syn.make_inputs(37, 3, 8, 16, seed=9, with_grad_out=True, heads=[1, 2], tokens=(11, 30))
    for n in ("q", "k", "v", "lr", "d_o"):
        np.testing.assert_array_equal(part[n], full[n][11:30, 1:3])
    z = syn.normal(syn._stream_key(2, 1, 1), 101)
    np.testing.assert_array_equal(syn.normal(syn._stream_key(2, 1, 1), 40, start=33), z[33:73])
