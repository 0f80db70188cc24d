"""Pins of the GCM-module oracle (CPU): the gated residual of Eq. 5 and the
chain rule through the projections, the per-head normalisation and the
learning-rate predictor, against central finite differences in float64."""
import numpy as np
import pytest

import oracle
import ttt_synth as syn

H, D, F = 2, 4, 8
d = H * D


def _problem(seed=0, T_chunks=((5, 4), (3,))):
    rng = np.random.default_rng(seed)
    lay = syn.layout_from_lengths([list(c) for c in T_chunks])
    T = lay.num_tokens
    p = {
        "x": rng.normal(size=(T, d)),
        "wqkv": rng.normal(size=(3 * d, d)) / np.sqrt(d),
        "bqkv": 0.1 * rng.normal(size=3 * d),
        "w_eta": 0.3 * rng.normal(size=(H, d)),
        "b_eta": 0.1 * rng.normal(size=H),
        "wo": rng.normal(size=(d, d)) / np.sqrt(d),
        "alpha": rng.normal(size=d),
        "w0": 0.3 * rng.normal(size=(H, 3 * F * D)),
    }
    return lay, p, rng


def _out(lay, p, base=0.5):
    return oracle.gcm_forward(p["x"], p["wqkv"], p["bqkv"], p["w_eta"], p["b_eta"], base, p["wo"], p["alpha"],
                              p["w0"], lay, H, D, F)["out"]


def test_zero_gate_is_the_identity():
    lay, p, _ = _problem(1)
    p["alpha"] = np.zeros(d)
    np.testing.assert_array_equal(_out(lay, p), p["x"])


def test_constant_learning_rate_without_predictor_weights():
    lay, p, _ = _problem(2)
    p["w_eta"] = np.zeros((H, d))
    p["b_eta"] = np.zeros(H)
    f = oracle.gcm_forward(p["x"], p["wqkv"], p["bqkv"], p["w_eta"], p["b_eta"], 0.5, p["wo"], p["alpha"], p["w0"],
                           lay, H, D, F)
    np.testing.assert_allclose(f["lr"], 0.25)
    np.testing.assert_allclose(np.linalg.norm(f["q"], axis=-1), 1.0)
    np.testing.assert_allclose(np.linalg.norm(f["k"], axis=-1), 1.0)


@pytest.mark.parametrize("name", ["x", "wqkv", "bqkv", "w_eta", "b_eta", "wo", "alpha", "w0"])
def test_backward_matches_finite_differences(name):
    lay, p, rng = _problem(3)
    d_out = rng.normal(size=p["x"].shape)
    g = oracle.gcm_backward(p["x"], p["wqkv"], p["bqkv"], p["w_eta"], p["b_eta"], 0.5, p["wo"], p["alpha"],
                            p["w0"], lay, d_out, H, D, F)
    u = rng.normal(size=p[name].shape)
    h = 1e-5

    def loss(sign):
        q = dict(p)
        q[name] = p[name] + sign * h * u
        return float((d_out * _out(lay, q)).sum())

    fd = (loss(1) - loss(-1)) / (2 * h)
    an = float((g["d" + name] * u).sum())
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, fd, an)
