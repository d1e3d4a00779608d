"""Pins of the oracle's learned min-sum gradient: central finite differences of the loss,
agreement of its forward pass with the layered decoder, and structural zeros."""
import numpy as np
import pytest

import oracle
from synth import make_workload


def _loss_from_post(post, cw, N):
    L = post.astype(np.float64)
    c = cw[:, :N].astype(np.float64)
    sp = np.where(L > 0, np.log1p(np.exp(-L)), -L + np.log1p(np.exp(L)))
    return float((sp + c * L).mean())


def _setup(kind="BG2", Z=4, B=3, T=3, seed=0, ebn0=1.0):
    wl = make_workload(kind, Z, B, ebn0, modulation="BPSK", seed=seed)
    rng = np.random.default_rng(seed)
    params = np.zeros((T, wl.n_rows, 2), np.float32)
    params[..., 0] = rng.uniform(0.6, 1.0, size=(T, wl.n_rows))
    params[..., 1] = rng.uniform(0.0, 0.3, size=(T, wl.n_rows))
    return wl, params


def test_forward_matches_layered_decoder():
    wl, params = _setup(kind="BG1", Z=8, B=4, T=4, seed=1)
    loss, gp, _, post = oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, params,
                                            wl.codewords, want_post=True)
    ref = oracle.decode_layered(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, algo=oracle.LEARNED,
                                learned=params, max_iter=4, early_stop=False, want_post=True)
    assert np.array_equal(post, ref.post)
    assert abs(loss - _loss_from_post(post, wl.codewords, post.shape[1])) < 1e-9


def _fd_agreement(f, x0, grad, idx_iter, h=1e-4):
    """Central differences of f around x0 along the given coordinates.  Coordinates where
    the two one-sided differences disagree (an argmin or max(., 0) kink inside +-h) are
    skipped.  Returns (agreeing, disagreeing) counts at a 2 % tolerance."""
    l0 = f(x0)
    ok = bad = 0
    for ix in idx_iter:
        x1 = x0.copy()
        x1[ix] += h
        x2 = x0.copy()
        x2[ix] -= h
        a, b = f(x1), f(x2)
        d1, d2 = a - l0, l0 - b
        if abs(d1 - d2) > 0.05 * max(abs(d1), abs(d2)) + 1e-10:
            continue
        fd = (a - b) / (2 * h)
        if abs(fd - grad[ix]) <= 0.02 * max(abs(fd), 1e-4) + 1e-6:
            ok += 1
        else:
            bad += 1
    return ok, bad


@pytest.mark.parametrize("kind,Z,punct,seed", [("TINY", 3, 0, 3), ("TINY", 3, 0, 4),
                                               ("BG2", 2, 2, 3)])
def test_param_gradient_finite_differences(kind, Z, punct, seed):
    """Reverse-mode gradient of the unrolled decoder against central differences of the
    loss in (beta, gamma), on small codes where the forward pass is piecewise linear."""
    T = 2
    wl = make_workload(kind, Z, 4, 2.0, modulation="BPSK", seed=seed, punct_cols=punct)
    rng = np.random.default_rng(seed)
    params = np.zeros((T, wl.n_rows, 2), np.float32)
    params[..., 0] = rng.uniform(0.6, 1.0, size=(T, wl.n_rows))
    params[..., 1] = rng.uniform(0.0, 0.3, size=(T, wl.n_rows))

    def f(p):
        return oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, p, wl.codewords,
                                   punct=punct)[0]

    _, gp, _, _ = oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, params,
                                      wl.codewords, punct=punct)
    idx = [(t, r, k) for t in range(T) for r in range(wl.n_rows) for k in range(2)]
    ok, bad = _fd_agreement(f, params, gp, idx)
    assert ok >= 8 and bad <= 0.1 * (ok + bad), (ok, bad)


def test_llr_gradient_finite_differences():
    T = 2
    wl = make_workload("TINY", 3, 3, 2.0, modulation="BPSK", seed=9, punct_cols=0)
    rng = np.random.default_rng(9)
    params = np.zeros((T, wl.n_rows, 2), np.float32)
    params[..., 0] = rng.uniform(0.6, 1.0, size=(T, wl.n_rows))
    params[..., 1] = rng.uniform(0.0, 0.3, size=(T, wl.n_rows))

    def f(l):
        return oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, l, params, wl.codewords,
                                   punct=0)[0]

    _, _, gl, _ = oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, params,
                                      wl.codewords, punct=0, want_grad_llr=True)
    idx = [(b, j) for b in range(wl.llr.shape[0]) for j in range(wl.llr.shape[1])]
    ok, bad = _fd_agreement(f, wl.llr, gl, idx)
    assert ok >= 30 and bad <= 0.1 * (ok + bad), (ok, bad)


def test_structural_zeros():
    wl, params = _setup(seed=6)
    params[..., 0] = 0.0                  # beta = 0: no messages, L stays the channel LLR
    _, gp, gl, post = oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, params,
                                          wl.codewords, want_grad_llr=True, want_post=True)
    assert np.all(gp[..., 1] == 0.0)      # gamma has no effect when beta = 0
    N = post.shape[1]
    Z = wl.Z
    # posteriors are the channel LLRs, and dLoss/dLLR is the BCE derivative itself
    assert np.array_equal(post[:, 2 * Z:2 * Z + wl.n_tx], wl.llr)
    L = wl.llr.astype(np.float64)
    c = wl.codewords[:, 2 * Z:2 * Z + wl.n_tx].astype(np.float64)
    want = (c - 1.0 / (1.0 + np.exp(L))) / (wl.llr.shape[0] * N)
    assert np.allclose(gl, want, rtol=1e-6, atol=1e-12)


# ------------------------------------------------------- loss over every iteration's output

def test_iteration_weighted_loss_value_and_split():
    """loss(w) = sum_t w_t * BCE(posteriors after iteration t): the value equals the BCE of
    layered decodes stopped after t + 1 iterations, and the gradient of the term of
    iteration t equals the final-loss gradient of the table cut after iteration t (later
    iterations have no influence on it)."""
    T = 3
    wl, params = _setup(kind="BG2", Z=4, B=3, T=T, seed=12)
    w = np.array([0.5, 0.25, 1.0])
    loss, gp, _, _ = oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, params,
                                         wl.codewords, iter_weights=w)
    want = 0.0
    for t in range(T):
        r = oracle.decode_layered(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr,
                                  algo=oracle.LEARNED, learned=params[:t + 1],
                                  max_iter=t + 1, early_stop=False, want_post=True)
        want += w[t] * _loss_from_post(r.post, wl.codewords, r.post.shape[1])
    assert abs(loss - want) < 1e-9
    total = np.zeros_like(gp)
    for t in range(T):
        e = np.zeros(T)
        e[t] = 1.0
        _, g_t, _, _ = oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, params,
                                           wl.codewords, iter_weights=e)
        _, g_cut, _, _ = oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr,
                                             params[:t + 1], wl.codewords)
        assert np.all(g_t[t + 1:] == 0.0)
        assert np.allclose(g_t[:t + 1], g_cut, rtol=1e-12, atol=1e-15)
        total += w[t] * g_t
    assert np.allclose(gp, total, rtol=1e-9, atol=1e-15)


def test_iteration_weighted_gradient_finite_differences():
    T = 3
    wl = make_workload("TINY", 3, 4, 2.0, modulation="BPSK", seed=13, punct_cols=0)
    rng = np.random.default_rng(13)
    params = np.zeros((T, wl.n_rows, 2), np.float32)
    params[..., 0] = rng.uniform(0.6, 1.0, size=(T, wl.n_rows))
    params[..., 1] = rng.uniform(0.0, 0.3, size=(T, wl.n_rows))
    w = np.array([1.0, 0.5, 2.0])

    def f(p):
        return oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, p, wl.codewords,
                                   punct=0, iter_weights=w)[0]

    _, gp, _, _ = oracle.learned_grad(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, params,
                                      wl.codewords, punct=0, iter_weights=w)
    idx = [(t, r, k) for t in range(T) for r in range(wl.n_rows) for k in range(2)]
    ok, bad = _fd_agreement(f, params, gp, idx)
    assert ok >= 8 and bad <= 0.1 * (ok + bad), (ok, bad)
