"""Float64 oracle of the learned cross-rank model.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper has no learned component: its cross ranks come from plain binary
search (Steps 1 and 2).  The GPU library adds a model that *proposes* the
high cross rank ``rank_high(q, X)`` of a key q in a large sorted base array X,
so that the exact search only scans a short window; a bracket check
X[r-1] <= q < X[r] (the definition of rank_high, Section 2) verifies every
answer and a full binary search replaces any that fails.  The merged output
therefore never depends on the model; only speed does.

Model (all arithmetic in this file is float64):

* Piecewise-linear part, S segments.  Knot ranks R[s] = floor(s*N/S) for
  s = 0..S (R[S] = N); knot keys K[s] = X[R[s]] for s < S, K[S] = X[N-1].
  Segment of q: s = number of knots K[1..S-1] that are <= q (0..S-1).
  Position in segment t = (q - K[s]) / (K[s+1] - K[s]) clamped to [0, 1]
  (t = 0 when the two knots are equal).  pla = R[s] + t * (R[s+1] - R[s]).
* MLP on the features f0 = 2t - 1, f1 = (2s + 1)/S - 1:
  z = W1 @ [f0, f1] + b1 (H units), h = relu(z), y = w2 . h + b2.
  y is the residual in units of the segment's size:
  scale = max(R[s+1] - R[s], 1), pred = pla + y * scale.
* Loss over a batch of labelled keys (q_b, L_b), L_b the exact rank:
  target tau_b = (L_b - pla_b) / scale_b, loss = mean(0.5 * (y_b - tau_b)^2).
* Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8) with bias correction.
* Error bound in segment units: eps_frac = max_b |y_b - tau_b|.
"""
from __future__ import annotations

import numpy as np

BETA1 = 0.9
BETA2 = 0.999
ADAM_EPS = 1e-8


def knots(X: np.ndarray, S: int):
    """Knot keys K[0..S] (the base's own float32 values) and knot ranks R[0..S]."""
    N = len(X)
    if N == 0:
        raise ValueError("empty base array")
    R = np.array([(s * N) // S for s in range(S + 1)], dtype=np.int64)
    K = np.empty(S + 1, dtype=X.dtype)
    for s in range(S):
        K[s] = X[R[s]]
    K[S] = X[N - 1]
    return K, R


def segment_of(q, K: np.ndarray) -> int:
    """Number of interior knots K[1..S-1] that are <= q."""
    S = len(K) - 1
    lo, hi = 1, S            # count knots <= q among K[1..S-1] by bisection
    while lo < hi:
        mid = (lo + hi) // 2
        if K[mid] <= q:
            lo = mid + 1
        else:
            hi = mid
    return lo - 1


def features(q: np.ndarray, K: np.ndarray):
    """Per key: segment s (int64), t, f0, f1 (float64)."""
    S = len(K) - 1
    q = np.asarray(q)
    s = np.array([segment_of(v, K) for v in q], dtype=np.int64)
    k0 = K[s].astype(np.float64)
    k1 = K[s + 1].astype(np.float64)
    width = k1 - k0
    num = q.astype(np.float64) - k0
    t = np.where(width > 0, num / np.where(width > 0, width, 1.0), 0.0)
    t = np.clip(t, 0.0, 1.0)
    f0 = 2.0 * t - 1.0
    f1 = (2.0 * s + 1.0) / S - 1.0
    return s, t, f0, f1


def forward(params: dict, q: np.ndarray, K: np.ndarray, R: np.ndarray):
    """Returns a dict with s, t, pla, scale, z, h, y, pred (float64 arrays)."""
    s, t, f0, f1 = features(q, K)
    Rs = R[s].astype(np.float64)
    seg = (R[s + 1] - R[s]).astype(np.float64)
    pla = Rs + t * seg
    scale = np.maximum(seg, 1.0)
    F = np.stack([f0, f1], axis=1)                     # (B, 2)
    z = F @ params["W1"].T + params["b1"]              # (B, H)
    h = np.maximum(z, 0.0)
    y = h @ params["w2"] + params["b2"]                # (B,)
    return {"s": s, "t": t, "f0": f0, "f1": f1, "pla": pla, "scale": scale,
            "z": z, "h": h, "y": y, "pred": pla + y * scale}


def loss_and_grads(params: dict, q: np.ndarray, L: np.ndarray,
                   K: np.ndarray, R: np.ndarray):
    """Mean half-squared residual loss and its exact gradients."""
    fw = forward(params, q, K, R)
    tau = (np.asarray(L, dtype=np.float64) - fw["pla"]) / fw["scale"]
    r = fw["y"] - tau
    B = len(r)
    loss = 0.5 * float(np.mean(r * r))
    dy = r / B                                          # dloss/dy_b
    dw2 = fw["h"].T @ dy
    db2 = np.sum(dy)
    dz = np.outer(dy, params["w2"]) * (fw["z"] > 0)     # (B, H)
    F = np.stack([fw["f0"], fw["f1"]], axis=1)
    dW1 = dz.T @ F                                      # (H, 2)
    db1 = dz.sum(axis=0)
    grads = {"W1": dW1, "b1": db1, "w2": dw2, "b2": np.float64(db2)}
    return loss, grads, fw, tau


def adam_init(params: dict) -> dict:
    return {"m": {k: np.zeros_like(np.asarray(v, dtype=np.float64)) for k, v in params.items()},
            "v": {k: np.zeros_like(np.asarray(v, dtype=np.float64)) for k, v in params.items()},
            "step": 0}


def adam_step(params: dict, grads: dict, state: dict, lr: float) -> dict:
    """One Adam update; returns new params (float64)."""
    state["step"] += 1
    k = state["step"]
    out = {}
    for name, p in params.items():
        g = np.asarray(grads[name], dtype=np.float64)
        m = BETA1 * state["m"][name] + (1.0 - BETA1) * g
        v = BETA2 * state["v"][name] + (1.0 - BETA2) * g * g
        state["m"][name], state["v"][name] = m, v
        mhat = m / (1.0 - BETA1 ** k)
        vhat = v / (1.0 - BETA2 ** k)
        out[name] = np.asarray(p, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + ADAM_EPS)
    return out


def error_bound_frac(params: dict, q: np.ndarray, L: np.ndarray,
                     K: np.ndarray, R: np.ndarray) -> float:
    """eps_frac = max |y - tau| over the labelled keys (segment units)."""
    fw = forward(params, q, K, R)
    tau = (np.asarray(L, dtype=np.float64) - fw["pla"]) / fw["scale"]
    return float(np.max(np.abs(fw["y"] - tau))) if len(tau) else 0.0
