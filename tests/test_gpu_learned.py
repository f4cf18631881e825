"""GPU tests of the learned cross-rank proposal: training kernels against the
float64 oracle (gradients, Adam steps, knots), and the learned merge against
the oracle merge (bit-exact) over consecutive LSM-style merges."""
import numpy as np
import pytest
import torch

import oracle
from oracle import cdf as ocdf
from paper_1202_6575_gb300 import tm, workloads as W
from tests.helpers import first_mismatch, vals_np

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def setup_model(N, S, H, Q, seed=0):
    X, Xv = W.lsm_base("cpu", n=N, seed=W.SEED_BASE + 50 + seed)
    q = W.lsm_label_keys("cpu", count=Q, seed=W.SEED_BASE + 60 + seed)
    Xn, qn = X.numpy(), q.numpy()
    L = np.array([oracle.rank_high(v, Xn) for v in qn], dtype=np.int64) if Q <= 4096 else None
    init = W.cdf_init(hidden=H, seed=W.SEED_BASE + 70 + seed)
    flat = torch.cat([init["W1"].reshape(-1), init["b1"], init["w2"], init["b2"].reshape(1)])
    model = tm.CdfModel(S, H, DEV).init(X.to(DEV), flat)
    return X, Xv, q, L, init, model


def params_of(model):
    p = model.params().cpu().numpy().astype(np.float64)
    H = model.H
    return {"W1": p[:2 * H].reshape(H, 2), "b1": p[2 * H:3 * H], "w2": p[3 * H:4 * H], "b2": np.float64(p[4 * H])}


def test_knots_match_oracle():
    X, Xv, q, L, init, model = setup_model(100003, 64, 8, 16)
    K, R = ocdf.knots(X.numpy(), 64)
    assert np.array_equal(model.knots().cpu().numpy(), K)
    assert np.array_equal(model.ranks(0).cpu().numpy(), R)
    h = model.header()
    assert (h["S"], h["H"], h["N"], h["cur"], h["adam_steps"]) == (64, 8, 100003, 0, 0)


def test_labels_from_plain_search_match_oracle():
    X = W.lsm_base("cpu", n=50000)[0]
    q = W.lsm_label_keys("cpu", count=3000)
    lab = tm.tm_rank_search("f32", "high", q.to(DEV), X.to(DEV)).cpu().numpy()
    assert lab.tolist() == [oracle.rank_high(v, X.numpy()) for v in q.numpy()]


@pytest.mark.parametrize("S,H", [(16, 8), (256, 64)])
def test_gradients_against_oracle(S, H):
    X, Xv, q, L, init, model = setup_model(20000, S, H, 3000, seed=S)
    g, loss = model.grad(q.to(DEV), torch.from_numpy(L).to(DEV))
    K, R = ocdf.knots(X.numpy(), S)
    P0 = {k: v.numpy() for k, v in init.items()}
    P0 = {k: v.astype(np.float32).astype(np.float64) for k, v in P0.items()}   # the float32 parameters
    oloss, og, _, _ = ocdf.loss_and_grads(P0, q.numpy(), L, K, R)
    flat = np.concatenate([og["W1"].reshape(-1), og["b1"], og["w2"], [og["b2"]]])
    gg = g.cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(flat))
    assert np.max(np.abs(gg - flat)) <= 2e-4 * scale + 1e-7, (np.max(np.abs(gg - flat)), scale)
    assert abs(loss.item() - oloss) <= 1e-4 * abs(oloss) + 1e-7


def test_adam_steps_against_oracle():
    S, H = 32, 16
    X, Xv, q, L, init, model = setup_model(30000, S, H, 2000, seed=3)
    K, R = ocdf.knots(X.numpy(), S)
    P = {k: v.numpy().astype(np.float32).astype(np.float64) for k, v in init.items()}
    st = ocdf.adam_init(P)
    for _ in range(5):
        _, g, _, _ = ocdf.loss_and_grads(P, q.numpy(), L, K, R)
        P = ocdf.adam_step(P, g, st, lr=1e-3)
    model.train(q.to(DEV), torch.from_numpy(L).to(DEV), steps=5, lr=1e-3)
    got = params_of(model)
    # Adam moves each parameter by about lr * sign(g); components whose
    # gradient is too small for its float32 sign to be determined are skipped
    for k in ("W1", "b1", "w2", "b2"):
        sure = np.abs(np.asarray(st["m"][k])) > 1e-5
        assert np.allclose(np.asarray(got[k])[sure], np.asarray(P[k])[sure], rtol=1e-4, atol=3e-5), k
        assert np.mean(sure) > 0.5
    assert model.header()["adam_steps"] == 5


def train_lsm_model(N, S=4096, H=64, Q=1 << 16, steps=300, lr=3e-3, seed=0):
    X, Xv = W.lsm_base(DEV, n=N)
    q = W.lsm_label_keys(DEV, count=Q)
    labels = tm.tm_rank_search("f32", "high", q, X)               # exact ranks from the plain search
    init = W.cdf_init(hidden=H)
    flat = torch.cat([init["W1"].reshape(-1), init["b1"], init["w2"], init["b2"].reshape(1)])
    model = tm.CdfModel(S, H, DEV).init(X, flat)
    model.train(q, labels, steps=steps, lr=lr)
    model.calibrate(q, labels)
    return X, Xv, q, labels, model, flat


def test_trained_model_predictions_within_bound():
    X, Xv, q, labels, model, flat = train_lsm_model(1 << 20, S=1024, H=32, Q=1 << 14, steps=200)
    h = model.header()
    assert h["eps"] > 0 and h["loss"] >= 0
    pred = model.predict(q).cpu().numpy().astype(np.float64)
    lab = labels.cpu().numpy()
    # every label within eps segment units of its prediction (float32 prediction: + a few ranks)
    Kn, Rn = model.knots().cpu().numpy(), model.ranks(0).cpu().numpy()
    s = np.array([ocdf.segment_of(v, Kn) for v in q.cpu().numpy()])
    scale = np.maximum(Rn[s + 1] - Rn[s], 1)
    assert np.all(np.abs(pred - lab) <= h["eps"] * scale + 4 + 1e-3 * np.abs(lab))


def check_merge_equal(C, Cv, A, Av, B, Bv):
    K, V = oracle.merge_two_pointer(A.cpu().numpy(), vals_np(Av), B.cpu().numpy(), vals_np(Bv))
    assert first_mismatch(C.cpu().numpy(), K) is None
    assert first_mismatch(vals_np(Cv), V) is None


def test_learned_lsm_merges_exact_and_knots_advance():
    N0, m, merges = 1 << 22, 1 << 16, 6
    X, Xv, q, labels, model, flat = train_lsm_model(N0, S=4096, H=64, Q=1 << 15, steps=150)
    A, Av = X, Xv
    for k in range(merges):
        B, Bv = W.lsm_batch(k, DEV, size=m, base_n=N0)
        n = A.numel()
        p = tm.tm_merge_blocks(n, m)
        xb_plain, yb_plain = tm.tm_cross_ranks("f32", A, B, p)
        cur = model.header()["cur"]
        R_before = model.ranks(cur).clone()
        C, Cv, ws = tm.tm_merge_learned(model, A, Av, B, Bv, flags=tm.LEARNED_ADVANCE)
        assert tm.tm_read_status(ws) == 0
        check_merge_equal(C, Cv, A, Av, B, Bv)
        # the learned Steps 1-2 return exactly the plain cross ranks (xbar
        # after the 256-byte control block, ybar on the next 256-byte boundary)
        xl = ws[256:256 + 8 * (p + 1)].view(torch.int64)
        y_off = 256 + (8 * (p + 1) + 255) // 256 * 256
        yl = ws[y_off:y_off + 8 * (p + 1)].view(torch.int64)
        assert torch.equal(xl, xb_plain) and torch.equal(yl, yb_plain)
        h = model.header()
        assert h["cur"] == 1 - cur and h["N"] == n + m
        # knot ranks now locate the knot keys in the merged base
        R_after = model.ranks(h["cur"])
        Kn = model.knots()
        assert torch.equal(C[R_after[:-1]], Kn[:-1])
        assert int(R_after[-1]) == n + m
        assert torch.all(R_after >= R_before)
        A, Av = C, Cv
    h = model.header()
    assert h["learned"] > 0


def test_forced_fallback_still_exact():
    X, Xv, q, labels, model, flat = train_lsm_model(1 << 20, S=256, H=16, Q=4096, steps=20)
    params = model.params()
    params[-1] = 1e6                                          # b2: every prediction far off
    B, Bv = W.lsm_batch(0, DEV, size=1 << 14, base_n=1 << 20)
    before = model.header()["fallbacks"]
    C, Cv, ws = tm.tm_merge_learned(model, X, Xv, B, Bv)
    assert tm.tm_read_status(ws) == 0
    check_merge_equal(C, Cv, X, Xv, B, Bv)
    h = model.header()
    assert h["fallbacks"] - before > 0


def test_gain_of_the_trained_network():
    """What the trained network gains over the method without it.  Plain
    Steps 1-2 bisect the whole base: log2 N probes per search.  The trained
    model proposes each rank and leaves a window of 3 eps_s segment units
    (eps_s its calibrated error in the key's segment): far fewer probes,
    every answer still exact.  Against its own piecewise-linear part alone
    (MLP output 0, calibrated the same way), training lowers the objective
    (mean squared residual) but not the windows: the residual that sets a
    segment's maximum error is the sampling noise of the base inside the
    segment, which a smooth function of (position in segment, segment
    index) cannot predict.  Asserted: the network's mean window is within a
    quarter probe of the piecewise-linear part's (it gains no probes, and
    costs none), and both answer every search of a merge exactly."""
    N = 1 << 24
    X, Xv, q, labels, model, flat = train_lsm_model(N, S=4096, H=64, Q=1 << 18, steps=400)
    zero = torch.zeros(model.P, dtype=torch.float32, device=DEV)
    pla = tm.CdfModel(4096, 64, DEV).init(X, zero)
    pla.calibrate(q, labels)
    _, loss_mlp = model.grad(q, labels)
    _, loss_pla = pla.grad(q, labels)
    seg = N / 4096
    e_mlp = model.eps_segments().cpu().numpy()
    e_pla = pla.eps_segments().cpu().numpy()
    w_mlp = np.log2(2 * (3 * e_mlp * seg + 32) + 1)
    w_pla = np.log2(2 * (3 * e_pla * seg + 32) + 1)
    print(f"loss: pla {loss_pla.item():.3e} mlp {loss_mlp.item():.3e}; median eps_s: pla {np.median(e_pla):.4f} "
          f"mlp {np.median(e_mlp):.4f}; mean window probes: plain {np.log2(N):.1f} pla {w_pla.mean():.2f} "
          f"mlp {w_mlp.mean():.2f}")
    assert loss_mlp.item() < loss_pla.item()
    assert w_mlp.mean() < np.log2(N) - 10
    assert abs(w_mlp.mean() - w_pla.mean()) < 0.25
    # both answer every query of a merge exactly, with few fallbacks
    B, Bv = W.lsm_batch(0, DEV, size=1 << 20, base_n=N)
    p = tm.tm_merge_blocks(N, B.numel())
    xp, yp = tm.tm_cross_ranks("f32", X, B, p)
    for m_ in (model, pla):
        xl, yl = tm.tm_cross_ranks_learned(m_, X, B, p)
        assert torch.equal(xl, xp) and torch.equal(yl, yp)
        h = m_.header()
        print(f"fallbacks {h['fallbacks']} of {h['learned']} learned searches")
        assert h["fallbacks"] <= 0.01 * h["learned"]
