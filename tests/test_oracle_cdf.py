"""Pins of the float64 learned-model oracle (oracle/cdf.py).

The model is not in the paper; its oracle is pinned by mathematics: central
finite differences of the loss, closed forms of special parameter settings,
the exact piecewise-linear interpolation of a linear base, a linear scan for
the segment lookup, and Adam's first step.
"""
import numpy as np
import pytest

import oracle
from oracle import cdf


def params_random(rng, H=8):
    return {"W1": rng.normal(size=(H, 2)), "b1": rng.normal(size=H) * 0.3,
            "w2": rng.normal(size=H), "b2": np.float64(rng.normal())}


def base_and_labels(rng, N=5000, S=16, Q=300):
    X = np.sort(np.exp(rng.normal(size=N) * 0.5 + rng.choice([0.0, 2.0], size=N))).astype(np.float32)
    q = np.sort(np.exp(rng.normal(size=Q) * 0.5 + 1.0)).astype(np.float32)
    L = np.array([oracle.rank_high(v, X) for v in q], dtype=np.int64)
    K, R = cdf.knots(X, S)
    return X, q, L, K, R


def test_segment_lookup_against_linear_scan():
    rng = np.random.default_rng(0)
    X, q, L, K, R = base_and_labels(rng)
    S = len(K) - 1
    for v in np.concatenate([q, K, [K[0] - 1, K[-1] + 1]]).astype(np.float32):
        s = cdf.segment_of(v, K)
        assert s == sum(1 for k in range(1, S) if K[k] <= v)
        if s >= 1:
            assert K[s] <= v
        if s < S - 1:
            assert v < K[s + 1]


def test_knots_definition():
    X = np.arange(100, dtype=np.float32) * 2
    K, R = cdf.knots(X, 8)
    assert R.tolist() == [(s * 100) // 8 for s in range(9)]
    assert K[:-1].tolist() == [float(X[r]) for r in R[:-1]] and K[-1] == X[-1]


def test_pla_exact_on_linear_base():
    # X[k] = k: knots sit at (k, k), so linear interpolation reproduces q.
    N, S = 4096, 64
    X = np.arange(N, dtype=np.float32)
    K, R = cdf.knots(X, S)
    q = np.arange(0, N - N // S, 7, dtype=np.float32) + 0.25
    fw = cdf.forward(cdf_zero(), q, K, R)
    assert np.allclose(fw["pla"], q.astype(np.float64), atol=1e-9)


def cdf_zero(H=4):
    return {"W1": np.zeros((H, 2)), "b1": np.zeros(H), "w2": np.zeros(H), "b2": np.float64(0)}


def test_closed_form_constant_hidden():
    # W1 = 0: h = relu(b1) for every key, y = w2 . relu(b1) + b2 constant.
    rng = np.random.default_rng(1)
    X, q, L, K, R = base_and_labels(rng)
    H = 6
    b1 = np.array([0.5, -1.0, 2.0, 0.0, 1.5, -0.2])
    w2 = rng.normal(size=H)
    P = {"W1": np.zeros((H, 2)), "b1": b1, "w2": w2, "b2": np.float64(0.3)}
    loss, g, fw, tau = cdf.loss_and_grads(P, q, L, K, R)
    y0 = float(w2 @ np.maximum(b1, 0) + 0.3)
    assert np.allclose(fw["y"], y0)
    mean_r = float(np.mean(y0 - tau))
    assert np.isclose(g["b2"], mean_r)
    assert np.allclose(g["w2"], mean_r * np.maximum(b1, 0))
    assert np.allclose(g["b1"], mean_r * w2 * (b1 > 0))
    assert np.isclose(loss, 0.5 * np.mean((y0 - tau) ** 2))


def test_gradients_against_finite_differences():
    rng = np.random.default_rng(2)
    X, q, L, K, R = base_and_labels(rng)
    P = params_random(rng)
    loss, g, _, _ = cdf.loss_and_grads(P, q, L, K, R)
    h = 1e-6
    for name in ("W1", "b1", "w2", "b2"):
        base = np.array(P[name], dtype=np.float64)
        flat = base.reshape(-1)
        gflat = np.asarray(g[name], dtype=np.float64).reshape(-1)
        for idx in range(flat.size):
            plus, minus = flat.copy(), flat.copy()
            plus[idx] += h
            minus[idx] -= h
            Pp = dict(P); Pp[name] = plus.reshape(base.shape)
            Pm = dict(P); Pm[name] = minus.reshape(base.shape)
            fd = (cdf.loss_and_grads(Pp, q, L, K, R)[0] - cdf.loss_and_grads(Pm, q, L, K, R)[0]) / (2 * h)
            assert abs(fd - gflat[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, gflat[idx])


def test_adam_first_step_is_signed_lr():
    # After one step m_hat = g and v_hat = g^2, so the update is lr * g / (|g| + eps).
    rng = np.random.default_rng(3)
    P = params_random(rng)
    G = {k: np.asarray(rng.normal(size=np.shape(v))) for k, v in P.items()}
    st = cdf.adam_init(P)
    new = cdf.adam_step(P, G, st, lr=0.01)
    for k in P:
        g = np.asarray(G[k])
        assert np.allclose(new[k], np.asarray(P[k]) - 0.01 * g / (np.abs(g) + cdf.ADAM_EPS))


def test_training_reduces_loss_and_bounds_error():
    rng = np.random.default_rng(4)
    X, q, L, K, R = base_and_labels(rng, N=20000, S=32, Q=2000)
    P = params_random(rng, H=16)
    P["w2"] *= 0.01
    st = cdf.adam_init(P)
    first = cdf.loss_and_grads(P, q, L, K, R)[0]
    for _ in range(200):
        loss, g, _, _ = cdf.loss_and_grads(P, q, L, K, R)
        P = cdf.adam_step(P, g, st, lr=3e-3)
    assert loss < first
    eps = cdf.error_bound_frac(P, q, L, K, R)
    fw = cdf.forward(P, q, K, R)
    # every label lies within eps segment units of the prediction
    assert np.all(np.abs(fw["pred"] - L) <= eps * fw["scale"] + 1e-6)


def test_pla_exact_outside_the_base():
    # Below X[0] the exact rank_high is 0 and from X[N-1] up it is N (the
    # definition of rank_high, Section 2); the piecewise-linear part must
    # give exactly these, whatever the knots.
    rng = np.random.default_rng(5)
    X, _, _, K, R = base_and_labels(rng)
    q = np.array([X[0] - 3.0, X[0] - 1e-3, X[-1], X[-1] + 1e-3, X[-1] + 50.0], dtype=np.float32)
    fw = cdf.forward(cdf_zero(), q, K, R)
    exact = [oracle.rank_high(v, X) for v in q]
    assert exact == [0, 0, len(X), len(X), len(X)]
    assert fw["pla"].tolist() == [float(e) for e in exact]
    assert np.all((fw["t"] >= 0.0) & (fw["t"] <= 1.0))


def test_segment_feature_is_the_segment_midpoint():
    # f1 places segment s at the midpoint of the s-th of S equal parts of
    # [-1, 1]; f0 maps the position in the segment onto [-1, 1].
    rng = np.random.default_rng(6)
    X, _, _, K, R = base_and_labels(rng, S=16)
    S = len(K) - 1
    q = np.sort(rng.uniform(float(X[0]), float(X[-1]), size=4000)).astype(np.float32)
    s, t, f0, f1 = cdf.features(q, K)
    mids = np.linspace(-1.0, 1.0, 2 * S + 1)[1::2]
    assert len(np.unique(s)) > S // 2
    assert np.allclose(f1, mids[s], atol=1e-15)
    assert np.allclose(f0, -1.0 + 2.0 * t, atol=1e-15)
    assert np.all(np.abs(f0) <= 1.0)


def test_loss_is_half_squared_error_of_the_predicted_rank():
    # Independent of the target's algebra: with pred the model's rank
    # estimate, the loss is the mean of ((pred - L) / scale)^2 / 2.
    rng = np.random.default_rng(7)
    X, q, L, K, R = base_and_labels(rng)
    P = params_random(rng)
    loss, _, fw, _ = cdf.loss_and_grads(P, q, L, K, R)
    err = (fw["pred"] - L) / fw["scale"]
    assert np.isclose(loss, 0.5 * np.mean(err * err), rtol=1e-12)


def test_error_bound_covers_underestimates():
    # A model that predicts below every label: the bound is the largest
    # distance, not the largest signed residual.
    rng = np.random.default_rng(8)
    X, q, L, K, R = base_and_labels(rng)
    P = params_random(rng)
    P["b2"] = np.float64(-50.0)
    fw = cdf.forward(P, q, K, R)
    assert np.all(fw["pred"] < L)
    eps = cdf.error_bound_frac(P, q, L, K, R)
    assert np.isclose(eps, np.max(np.abs(fw["pred"] - L) / fw["scale"]), rtol=1e-12)
