"""Plain FP64 CPU oracle of the Scal3R test-time-training (TTT) layer.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
links this module: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may use it.  It shares no
code with the CUDA path.

What it computes (paper sections and equations of arXiv 2604.08542):

* The fast-weight network of one head is the SwiGLU MLP of Supp. Sec. A,
      f_W(x) = W2 ( SiLU(W1 x) o (W3 x) ),  SiLU(z) = z * sigmoid(z),
  with W1, W3 in R^{F x D} and W2 in R^{D x F} (y = W x orientation).
* A long token stream is cut into chunks (Sec. 4.1, 4.2).  Each chunk is
  one update unit: the gradient of the learning-rate-weighted loss over all
  tokens of the chunk, taken at the pre-chunk weights, is subtracted once
  (Eq. 8); the loss is the negative dot product of f_W(k) and v (Eq. 9).
  The TTT update / apply pair is Eq. 3 / Eq. 4.
* After the update the chunk's queries are transformed by the updated
  weights (Sec. 4.2, last sentence before "Global Context Synchronization").
* The fast weights carry over from chunk to chunk; a single GPU processes
  the chunks sequentially (Sec. 4.4, last sentence).  Each sequence starts
  from the initial weights.
* Readings where the paper is silent: every row of W1, W3, W2 is rescaled
  after each update to the L2 norm it had in the initial weights
  ("row_w0"; "unit" rescales to 1, "none" skips it) with the clamp
  max(||row||, eps); the MSE loss is 1/2 ||f_W(k) - v||^2; the learning rate
  is one scalar per (token, head) shared by W1, W3, W2, or, as an option,
  one per matrix: lr [T, H, 3] with lr[..., 0], [..., 1], [..., 2] the rates
  of W1, W3, W2, and G_j = d/dW_j sum_i eta_{j,i} L_i (Eq. 8 with the rate
  of the matrix being updated).
* ``model="linear"`` replaces f_W by the linear map f_W(x) = W x (W in
  R^{D x D}); with the dot loss and no normalisation the layer is then
  chunk-causal linear attention, a closed form the tests check.

The backward pass is written out by reverse-mode differentiation of the
forward recurrence (the paper gives none); the tests pin it to central
finite differences.

Arrays: q, k, v, d_o [T, H, D]; lr [T, H] (or [T, H, 3], one rate per matrix); w0 [H, P] (shared by all
sequences) or [S, H, P] (per sequence), P = 3*F*D packed as W1, W3, W2
row-major (linear model: P = D*D).  All arithmetic is float64.
"""
from __future__ import annotations

import numpy as np

LOSSES = ("dot", "mse")
NORMS = ("row_w0", "unit", "none")
MODELS = ("swiglu", "linear")


# ---------------------------------------------------------------------------
# elementwise pieces of the SwiGLU network (Supp. Sec. A)
# ---------------------------------------------------------------------------

def sigmoid(z):
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_prime(z):
    """d/dz [z sigmoid(z)] = sigmoid(z) (1 + z (1 - sigmoid(z)))."""
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def silu_second(z):
    """d^2/dz^2 [z sigmoid(z)] = s (1 - s) (2 + z (1 - 2 s))."""
    s = sigmoid(z)
    return s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s))


# ---------------------------------------------------------------------------
# packing
# ---------------------------------------------------------------------------

def param_count(D: int, F: int, model: str = "swiglu") -> int:
    return D * D if model == "linear" else 3 * F * D


def unpack(w: np.ndarray, D: int, F: int, model: str = "swiglu") -> list:
    """Packed vector -> list of weight matrices ([W1, W3, W2] or [W])."""
    w = np.asarray(w, dtype=np.float64)
    if model == "linear":
        return [w.reshape(D, D).copy()]
    return [w[:F * D].reshape(F, D).copy(),
            w[F * D:2 * F * D].reshape(F, D).copy(),
            w[2 * F * D:].reshape(D, F).copy()]


def pack(mats: list) -> np.ndarray:
    return np.concatenate([m.reshape(-1) for m in mats])


def row_norm_count(D: int, F: int, model: str = "swiglu") -> int:
    """Number of rows whose norm is stored per chunk (F + F + D for SwiGLU)."""
    return D if model == "linear" else 2 * F + D


# ---------------------------------------------------------------------------
# one chunk: the inner gradient (Eq. 8 with the loss of Eq. 9) and apply (Eq. 4)
# ---------------------------------------------------------------------------

def apply(W: list, X: np.ndarray, model: str = "swiglu") -> np.ndarray:
    """f_W applied to every row of X [M, D] (Eq. 4, Supp. Sec. A)."""
    if model == "linear":
        return X @ W[0].T
    W1, W3, W2 = W
    return (silu(X @ W1.T) * (X @ W3.T)) @ W2.T


def inner_gradient(W: list, K: np.ndarray, V: np.ndarray, eta: np.ndarray,
                   loss: str = "dot", model: str = "swiglu") -> list:
    """G_j = d/dW_j sum_i eta_i L(f_W(k_i), v_i) at fixed W (Eq. 8, 9).

    Rows of K, V [M, D] are the chunk's keys and values, eta [M] their
    learning rates (or [M, 3]: one rate per matrix W1, W3, W2).  Returned in
    the order of W.
    """
    if eta.ndim == 2:
        return _inner_gradient_per_matrix(W, K, V, eta, loss, model)
    eta = eta[:, None]
    if model == "linear":
        (Wl,) = W
        Y = K @ Wl.T
        E = -eta * V if loss == "dot" else eta * (Y - V)      # dL/df per token, times eta
        return [E.T @ K]
    W1, W3, W2 = W
    Z1 = K @ W1.T
    Z3 = K @ W3.T
    A = silu(Z1)
    U = A * Z3
    if loss == "dot":
        E = -eta * V                                        # d(-eta f.v)/df
    else:
        E = eta * (U @ W2.T - V)                            # d(eta/2 ||f - v||^2)/df
    P = E @ W2                                              # p_i = W2^T e_i
    G3 = P * A
    G1 = P * Z3 * silu_prime(Z1)
    return [G1.T @ K, G3.T @ K, E.T @ U]                    # dW1, dW3, dW2


def _inner_gradient_per_matrix(W, K, V, eta, loss, model):
    """G_j = d/dW_j sum_i eta_{j,i} L_i: each matrix's gradient with its own
    per-token rate, all at the same W."""
    if model != "swiglu":
        raise ValueError("per-matrix rates need the SwiGLU network's three matrices")
    W1, W3, W2 = W
    Z1 = K @ W1.T
    Z3 = K @ W3.T
    A = silu(Z1)
    U = A * Z3
    Eh = -V if loss == "dot" else U @ W2.T - V              # dL_i/df, without a rate
    Ph = Eh @ W2                                            # W2^T e_i
    e1, e3, e2 = eta[:, 0:1], eta[:, 1:2], eta[:, 2:3]
    G1 = e1 * Ph * Z3 * silu_prime(Z1)
    G3 = e3 * Ph * A
    return [G1.T @ K, G3.T @ K, (e2 * Eh).T @ U]


def row_targets(W0: list, norm: str) -> list:
    """Target L2 norm of every row: its norm in the initial weights ("row_w0"),
    1 ("unit"), or None ("none")."""
    if norm == "none":
        return [None for _ in W0]
    if norm == "unit":
        return [np.ones(m.shape[0]) for m in W0]
    return [np.sqrt(np.sum(m * m, axis=1)) for m in W0]


def normalise(Wt: list, rho: list, eps: float) -> tuple:
    """Rescale every row of every matrix to its target norm:
    row <- row * rho / max(||row||, eps).  Returns (weights, pre-norm row norms)."""
    out, norms = [], []
    for m, r in zip(Wt, rho):
        n = np.sqrt(np.sum(m * m, axis=1))
        norms.append(n)
        if r is None:
            out.append(m.copy())
        else:
            out.append(m * (r / np.maximum(n, eps))[:, None])
    return out, np.concatenate(norms)


# ---------------------------------------------------------------------------
# forward over a ragged batch
# ---------------------------------------------------------------------------

def _chain_w0(w0: np.ndarray, s: int, h: int) -> np.ndarray:
    return w0[s, h] if w0.ndim == 3 else w0[h]


def chain_forward(Q, K, V, eta, W0: list, chunks, loss="dot", norm="row_w0",
                  model="swiglu", eps=1e-12, keep_history=False):
    """Forward of one chain (one sequence, one head).

    Q, K, V [L, D], eta [L] are the chain's tokens; ``chunks`` lists the
    (start, end) token ranges of its chunks relative to the chain.
    Returns (O [L, D], list of W after each chunk, list of pre-norm row
    norms per chunk, history) where history (if requested) holds, per
    chunk, (W before, W after the gradient step, W after normalisation).
    """
    W = [m.copy() for m in W0]
    rho = row_targets(W0, norm)
    O = np.zeros_like(Q)
    ckpts, norms, hist = [], [], []
    for (t0, t1) in chunks:
        G = inner_gradient(W, K[t0:t1], V[t0:t1], eta[t0:t1], loss, model)   # Eq. 8 at pre-chunk W
        Wt = [m - g for m, g in zip(W, G)]
        Wn, n = normalise(Wt, rho, eps)
        if keep_history:
            hist.append((W, Wt, Wn))
        W = Wn
        ckpts.append([m.copy() for m in W])
        norms.append(n)
        O[t0:t1] = apply(W, Q[t0:t1], model)                                  # apply after update
    return O, ckpts, norms, hist


def forward(q, k, v, lr, w0, layout, D: int, F: int, loss="dot", norm="row_w0",
            model="swiglu", eps=1e-12, w_init=None) -> dict:
    """Forward of the whole ragged batch.

    ``layout`` has ``chunk_offsets`` [C+1] and ``seq_chunk_ptr`` [S+1].
    ``w_init`` [S, H, P], if given, replaces w0 as the starting weights of
    each sequence (streaming resume); the normalisation targets are the
    row norms of the starting weights.
    Returns o [T,H,D], w_ckpt [C,H,P] (weights after each chunk's update),
    wnorm [C,H,R] (pre-normalisation row norms), w_final [S,H,P].
    """
    q, k, v = (np.asarray(x, dtype=np.float64) for x in (q, k, v))
    lr = np.asarray(lr, dtype=np.float64)
    w0 = np.asarray(w0, dtype=np.float64)
    T, H, _ = q.shape
    C = len(layout.chunk_offsets) - 1
    S = len(layout.seq_chunk_ptr) - 1
    P = param_count(D, F, model)
    o = np.zeros((T, H, D))
    w_ckpt = np.zeros((C, H, P))
    wnorm = np.zeros((C, H, row_norm_count(D, F, model)))
    w_final = np.zeros((S, H, P))
    for s in range(S):
        c0, c1 = int(layout.seq_chunk_ptr[s]), int(layout.seq_chunk_ptr[s + 1])
        base = int(layout.chunk_offsets[c0])
        end = int(layout.chunk_offsets[c1])
        chunks = [(int(layout.chunk_offsets[c]) - base, int(layout.chunk_offsets[c + 1]) - base)
                  for c in range(c0, c1)]
        for h in range(H):
            start = w_init[s, h] if w_init is not None else _chain_w0(w0, s, h)
            W0 = unpack(start, D, F, model)
            O, ck, nr, _ = chain_forward(q[base:end, h], k[base:end, h], v[base:end, h],
                                         lr[base:end, h], W0, chunks, loss, norm, model, eps)
            o[base:end, h] = O
            for j, c in enumerate(range(c0, c1)):
                w_ckpt[c, h] = pack(ck[j])
                wnorm[c, h] = nr[j]
            w_final[s, h] = pack(ck[-1]) if ck else pack(W0)
    return {"o": o, "w_ckpt": w_ckpt, "wnorm": wnorm, "w_final": w_final}


# ---------------------------------------------------------------------------
# backward: reverse-mode differentiation of the forward recurrence
# ---------------------------------------------------------------------------

def _apply_vjp(W, Q, dO, model):
    """VJP of O = f_W(Q): returns (dW list, dQ)."""
    if model == "linear":
        (Wl,) = W
        return [dO.T @ Q], dO @ Wl
    W1, W3, W2 = W
    Z1 = Q @ W1.T
    Z3 = Q @ W3.T
    A = silu(Z1)
    U = A * Z3
    dW2 = dO.T @ U
    dU = dO @ W2
    dZ3 = dU * A
    dZ1 = dU * Z3 * silu_prime(Z1)
    return [dZ1.T @ Q, dZ3.T @ Q, dW2], dZ1 @ W1 + dZ3 @ W3


def _normalise_vjp(Wt, rho, Lam, eps):
    """VJP of W = normalise(Wt): returns (dWt list, drho list)."""
    dWt, drho = [], []
    for m, r, lam in zip(Wt, rho, Lam):
        if r is None:
            dWt.append(lam.copy())
            drho.append(None)
            continue
        n = np.sqrt(np.sum(m * m, axis=1))
        big = n >= eps
        nn = np.where(big, n, 1.0)
        what = m / nn[:, None]                                # unit rows where unclamped
        proj = np.sum(what * lam, axis=1)
        R_big = (r / nn)[:, None] * (lam - what * proj[:, None])
        R_small = (r / eps)[:, None] * lam
        dWt.append(np.where(big[:, None], R_big, R_small))
        drho.append(np.where(big, proj, np.sum(m * lam, axis=1) / eps))
    return dWt, drho


def _update_vjp(W, K, V, eta, R, loss, model):
    """VJP of Wt = W - G(W; K, V, eta) given R = dL/dWt.

    Returns (dL/dW list, dK, dV, deta).  dG = -R."""
    if eta.ndim == 2:
        return _update_vjp_per_matrix(W, K, V, eta, R, loss, model)
    etac = eta[:, None]
    if model == "linear":
        (Wl,) = W
        (Rl,) = R
        Y = K @ Wl.T
        E = -etac * V if loss == "dot" else etac * (Y - V)
        # G = E^T K
        dE = -(K @ Rl.T)                      # dL/de_t = dG k_t = -R k_t
        dK = -(E @ Rl)                        # dG^T e_t = -R^T e_t
        dW = [Rl.copy()]
        if loss == "dot":
            dV = -etac * dE
            deta = -np.sum(V * dE, axis=1)
        else:
            dY = etac * dE
            dV = -etac * dE
            deta = np.sum((Y - V) * dE, axis=1)
            dW[0] += dY.T @ K
            dK += dY @ Wl
        return dW, dK, dV, deta
    W1, W3, W2 = W
    R1, R3, R2 = R
    Z1 = K @ W1.T
    Z3 = K @ W3.T
    sp = silu_prime(Z1)
    spp = silu_second(Z1)
    A = silu(Z1)
    U = A * Z3
    if loss == "dot":
        Y = None
        E = -etac * V
    else:
        Y = U @ W2.T
        E = etac * (Y - V)
    P = E @ W2
    G3 = P * A
    G1 = P * Z3 * sp
    # G2 = E^T U, G1 = G1^T K, G3 = G3^T K enter Wt with a minus sign
    dE = -(U @ R2.T)
    dU = -(E @ R2)
    dG1 = -(K @ R1.T)
    dG3 = -(K @ R3.T)
    dK = -(G1 @ R1 + G3 @ R3)
    # g3 = p a ; g1 = p z3 s'
    dP = dG3 * A + dG1 * Z3 * sp
    dA = dG3 * P
    dZ3 = dG1 * P * sp
    dZ1 = dG1 * P * Z3 * spp
    # p = W2^T e
    dE = dE + dP @ W2.T
    dW2 = R2 + E.T @ dP
    # loss head
    if loss == "dot":
        dV = -etac * dE
        deta = -np.sum(V * dE, axis=1)
    else:
        dY = etac * dE
        dV = -etac * dE
        deta = np.sum((Y - V) * dE, axis=1)
        dU = dU + dY @ W2
        dW2 = dW2 + dY.T @ U
    # u = a z3 ; a = silu(z1)
    dA = dA + dU * Z3
    dZ3 = dZ3 + dU * A
    dZ1 = dZ1 + dA * sp
    dW1 = R1 + dZ1.T @ K
    dW3 = R3 + dZ3.T @ K
    dK = dK + dZ1 @ W1 + dZ3 @ W3
    return [dW1, dW3, dW2], dK, dV, deta


def _update_vjp_per_matrix(W, K, V, eta, R, loss, model):
    """``_update_vjp`` with one rate per matrix (eta [M, 3]; deta [M, 3])."""
    if model != "swiglu":
        raise ValueError("per-matrix rates need the SwiGLU network's three matrices")
    W1, W3, W2 = W
    R1, R3, R2 = R
    e1, e3, e2 = eta[:, 0:1], eta[:, 1:2], eta[:, 2:3]
    Z1 = K @ W1.T
    Z3 = K @ W3.T
    sp = silu_prime(Z1)
    spp = silu_second(Z1)
    A = silu(Z1)
    U = A * Z3
    Eh = -V if loss == "dot" else U @ W2.T - V
    Ph = Eh @ W2
    H1 = Ph * Z3 * sp                     # G1 = (e1 H1)^T K
    H3 = Ph * A                           # G3 = (e3 H3)^T K
    # G2 = (e2 Eh)^T U; all three enter Wt with a minus sign
    dS1 = -(K @ R1.T)                     # dL/d(e1 H1)
    dS3 = -(K @ R3.T)                     # dL/d(e3 H3)
    dS2 = -(U @ R2.T)                     # dL/d(e2 Eh)
    deta = np.stack([np.sum(H1 * dS1, axis=1), np.sum(H3 * dS3, axis=1), np.sum(Eh * dS2, axis=1)], axis=1)
    dK = -((e1 * H1) @ R1 + (e3 * H3) @ R3)
    dU = -((e2 * Eh) @ R2)
    dH1 = e1 * dS1
    dH3 = e3 * dS3
    dEh = e2 * dS2
    # H1 = ph z3 s' ; H3 = ph a
    dPh = dH1 * Z3 * sp + dH3 * A
    dA = dH3 * Ph
    dZ3 = dH1 * Ph * sp
    dZ1 = dH1 * Ph * Z3 * spp
    # ph = W2^T e
    dEh = dEh + dPh @ W2.T
    dW2 = R2 + Eh.T @ dPh
    dV = -dEh
    if loss != "dot":                     # e = W2 u - v
        dU = dU + dEh @ W2
        dW2 = dW2 + dEh.T @ U
    dA = dA + dU * Z3
    dZ3 = dZ3 + dU * A
    dZ1 = dZ1 + dA * sp
    dW1 = R1 + dZ1.T @ K
    dW3 = R3 + dZ3.T @ K
    dK = dK + dZ1 @ W1 + dZ3 @ W3
    return [dW1, dW3, dW2], dK, dV, deta


def chain_backward(Q, K, V, eta, W0, chunks, dO, loss="dot", norm="row_w0",
                   model="swiglu", eps=1e-12):
    """Gradients of sum(dO * O) for one chain: (dQ, dK, dV, deta, dW0 list)."""
    _, _, _, hist = chain_forward(Q, K, V, eta, W0, chunks, loss, norm, model, eps, keep_history=True)
    rho = row_targets(W0, norm)
    dQ = np.zeros_like(Q)
    dK = np.zeros_like(K)
    dV = np.zeros_like(V)
    deta = np.zeros_like(eta)
    Lam = [np.zeros_like(m) for m in W0]                  # dL/dW_c, carried backwards
    drho = [None if r is None else np.zeros_like(r) for r in rho]
    for idx in range(len(chunks) - 1, -1, -1):
        t0, t1 = chunks[idx]
        Wprev, Wt, Wc = hist[idx]
        # 1. apply part: O_c = f_{W_c}(Q_c)
        dWa, dQ[t0:t1] = _apply_vjp(Wc, Q[t0:t1], dO[t0:t1], model)
        Lam = [a + b for a, b in zip(Lam, dWa)]
        # 2. normalisation
        R, dr = _normalise_vjp(Wt, rho, Lam, eps)
        if norm == "row_w0":
            drho = [a + b for a, b in zip(drho, dr)]
        # 3. gradient step Wt = Wprev - G(Wprev)
        Lam, dK[t0:t1], dV[t0:t1], deta[t0:t1] = _update_vjp(Wprev, K[t0:t1], V[t0:t1],
                                                            eta[t0:t1], R, loss, model)
    dW0 = [l.copy() for l in Lam]
    if norm == "row_w0":
        # rho = ||W0 row|| contributes drho * W0_row / ||W0_row||
        for j, (m, r) in enumerate(zip(W0, rho)):
            dW0[j] += (drho[j] / np.where(r > 0, r, 1.0))[:, None] * m
    return dQ, dK, dV, deta, dW0


def backward(q, k, v, lr, w0, layout, d_o, D: int, F: int, loss="dot", norm="row_w0",
             model="swiglu", eps=1e-12) -> dict:
    """Gradients of sum(d_o * o) w.r.t. q, k, v, lr and w0.

    dw0 has the shape of w0: summed over sequences when w0 is shared [H, P].
    """
    q, k, v, d_o = (np.asarray(x, dtype=np.float64) for x in (q, k, v, d_o))
    lr = np.asarray(lr, dtype=np.float64)
    w0 = np.asarray(w0, dtype=np.float64)
    T, H, _ = q.shape
    S = len(layout.seq_chunk_ptr) - 1
    dq = np.zeros_like(q)
    dk = np.zeros_like(k)
    dv = np.zeros_like(v)
    dlr = np.zeros_like(lr)
    dw0 = np.zeros_like(w0)
    for s in range(S):
        c0, c1 = int(layout.seq_chunk_ptr[s]), int(layout.seq_chunk_ptr[s + 1])
        base = int(layout.chunk_offsets[c0])
        end = int(layout.chunk_offsets[c1])
        chunks = [(int(layout.chunk_offsets[c]) - base, int(layout.chunk_offsets[c + 1]) - base)
                  for c in range(c0, c1)]
        for h in range(H):
            W0 = unpack(_chain_w0(w0, s, h), D, F, model)
            gq, gk, gv, ge, gW = chain_backward(q[base:end, h], k[base:end, h], v[base:end, h],
                                                lr[base:end, h], W0, chunks, d_o[base:end, h],
                                                loss, norm, model, eps)
            dq[base:end, h] = gq
            dk[base:end, h] = gk
            dv[base:end, h] = gv
            dlr[base:end, h] = ge
            if w0.ndim == 3:
                dw0[s, h] += pack(gW)
            else:
                dw0[h] += pack(gW)
    return {"dq": dq, "dk": dk, "dv": dv, "dlr": dlr, "dw0": dw0}
