"""Learned min-sum on the GPU: forward identical to the oracle's fp32 learned decoder, the
hand-written backward against the oracle gradient, the autograd wrapper against finite
differences, and the regular decode path with a learned table."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ldpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05534_gb300 import build
    build.build()
    import paper_2009_05534_gb300 as pkg
    return pkg


def _params(T, n_rows, seed):
    rng = np.random.default_rng(seed)
    p = np.zeros((T, n_rows, 2), np.float32)
    p[..., 0] = rng.uniform(0.6, 1.0, size=(T, n_rows))
    p[..., 1] = rng.uniform(0.0, 0.3, size=(T, n_rows))
    return p


@pytest.mark.parametrize("kind,Z,T", [("BG2", 16, 4), ("BG1", 32, 3), ("BG2", 128, 2)])
def test_forward_and_gradient_match_oracle(ldpc, kind, Z, T):
    from paper_2009_05534_gb300 import learned
    wl = make_workload(kind, Z, 6, 1.5, modulation="BPSK", seed=Z)
    prm = _params(T, wl.n_rows, Z)
    g = ldpc.Graph(wl.base, wl.K_b, Z)
    llr = torch.from_numpy(wl.llr).cuda()
    pt = torch.from_numpy(prm).cuda()
    post, ws = learned.forward(g, llr, pt)
    loss_o, gp_o, gl_o, post_o = oracle.learned_grad(wl.base, wl.K_b, Z, wl.n_rows, wl.llr, prm,
                                                     wl.codewords, want_post=True,
                                                     want_grad_llr=True)
    assert np.array_equal(post.cpu().numpy(), post_o)          # same fp32 operations
    N = post.shape[1]
    c = torch.from_numpy(wl.codewords[:, :N]).cuda().float()
    gpost = (c - torch.sigmoid(-post)) / post.numel()           # dLoss/dL of the mean BCE
    gp, gl = learned.backward(g, gpost, pt, ws, n_tx=wl.n_tx, want_grad_llr=True)
    torch.cuda.synchronize()
    gp = gp.sum(0).cpu().numpy().astype(np.float64)
    for t in range(T):                  # each iteration at its own scale
        scale = np.abs(gp_o[t]).max()
        assert np.allclose(gp[t], gp_o[t], rtol=1e-3, atol=1e-4 * scale), t
    assert np.allclose(gl.cpu().numpy(), gl_o, rtol=1e-3, atol=1e-4 * np.abs(gl_o).max())
    g.close()


@pytest.mark.parametrize("kind,Z,T", [("BG2", 16, 4), ("BG1", 32, 3)])
def test_every_iteration_loss_matches_oracle(ldpc, kind, Z, T):
    """Per-iteration posteriors equal the oracle's decodes stopped after t + 1 iterations,
    and the gradient of the iteration-weighted BCE (through the autograd wrapper) matches
    the oracle's."""
    from paper_2009_05534_gb300 import learned
    wl = make_workload(kind, Z, 5, 1.5, modulation="BPSK", seed=Z + 1)
    prm = _params(T, wl.n_rows, Z + 1)
    w = np.linspace(0.5, 1.5, T)
    g = ldpc.Graph(wl.base, wl.K_b, Z)
    llr = torch.from_numpy(wl.llr).cuda()
    pt = torch.from_numpy(prm).cuda().requires_grad_(True)
    post = learned.learned_decode(pt, llr, g, 0, wl.n_tx, every_iteration=True)
    for t in range(T):
        ref = oracle.decode_layered(wl.base, wl.K_b, Z, wl.n_rows, wl.llr, algo=oracle.LEARNED,
                                    learned=prm[:t + 1], max_iter=t + 1, early_stop=False,
                                    want_post=True)
        assert np.array_equal(post[t].detach().cpu().numpy(), ref.post)
    cw = torch.from_numpy(wl.codewords).cuda()
    loss = learned.bce_loss(post, cw, torch.tensor(w, dtype=torch.float32, device="cuda"))
    loss.backward()
    loss_o, gp_o, _, _ = oracle.learned_grad(wl.base, wl.K_b, Z, wl.n_rows, wl.llr, prm,
                                             wl.codewords, iter_weights=w)
    assert abs(float(loss.detach()) - loss_o) < 1e-4 * abs(loss_o)
    gp = pt.grad.cpu().numpy().astype(np.float64)
    for t in range(T):
        assert np.allclose(gp[t], gp_o[t], rtol=1e-3, atol=1e-4 * np.abs(gp_o[t]).max()), t
    g.close()


def test_detached_gradient_is_each_iterations_own_partial(ldpc):
    """With adjoints reset at iteration boundaries, the parameters of iteration t get
    w_t * dBCE_t/dtheta_t: the oracle's gradient of the single term t (iteration t's inputs
    do not depend on theta_t, so that slice is exact)."""
    from paper_2009_05534_gb300 import learned
    T = 4
    wl = make_workload("BG2", 16, 5, 2.0, modulation="BPSK", seed=23)
    prm = _params(T, wl.n_rows, 23)
    w = np.array([0.4, 0.3, 0.2, 1.0])
    g = ldpc.Graph(wl.base, wl.K_b, 16)
    pt = torch.from_numpy(prm).cuda().requires_grad_(True)
    post = learned.learned_decode(pt, torch.from_numpy(wl.llr).cuda(), g, 0, wl.n_tx,
                                  every_iteration=True, detach=True)
    learned.bce_loss(post, torch.from_numpy(wl.codewords).cuda(),
                     torch.tensor(w, dtype=torch.float32, device="cuda")).backward()
    gp = pt.grad.cpu().numpy().astype(np.float64)
    for t in range(T):
        e = np.zeros(T)
        e[t] = w[t]
        _, g_t, _, _ = oracle.learned_grad(wl.base, wl.K_b, 16, wl.n_rows, wl.llr, prm,
                                           wl.codewords, iter_weights=e)
        assert np.allclose(gp[t], g_t[t], rtol=1e-3, atol=1e-4 * np.abs(g_t[t]).max()), t
    g.close()


def test_autograd_matches_finite_differences(ldpc):
    from paper_2009_05534_gb300 import learned
    wl = make_workload("TINY", 3, 4, 2.0, modulation="BPSK", seed=3, punct_cols=0)
    # the TINY code is unpunctured: decode through a graph whose first two columns carry
    # LLRs, i.e. pass all N bits as transmitted and compare against the oracle gradient
    g = ldpc.Graph(wl.base, wl.K_b, 3)
    T = 2
    prm = _params(T, wl.n_rows, 4)
    # the CUDA learned path punctures two columns; use the BG2-shaped code instead
    g.close()
    wl = make_workload("BG2", 2, 4, 2.0, modulation="BPSK", seed=3)
    g = ldpc.Graph(wl.base, wl.K_b, 2)
    prm = _params(T, wl.n_rows, 4)
    p = torch.from_numpy(prm).cuda().requires_grad_(True)
    llr = torch.from_numpy(wl.llr).cuda()
    cw = torch.from_numpy(wl.codewords).cuda()
    loss = learned.bce_loss(learned.learned_decode(p, llr, g, 0, wl.n_tx), cw)
    loss.backward()
    grad = p.grad.cpu().numpy()

    def f(x):
        with torch.no_grad():
            return float(learned.bce_loss(learned.learned_decode(
                torch.from_numpy(x).cuda(), llr, g, 0, wl.n_tx), cw).double().item())

    h, ok, bad = 1e-3, 0, 0
    l0 = f(prm)
    for t in range(T):
        for r in range(wl.n_rows):
            for k in range(2):
                x1, x2 = prm.copy(), prm.copy()
                x1[t, r, k] += h
                x2[t, r, k] -= h
                a, b = f(x1), f(x2)
                if abs((a - l0) - (l0 - b)) > 0.05 * max(abs(a - l0), abs(l0 - b)) + 1e-7:
                    continue
                fd = (a - b) / (2 * h)
                if abs(fd - grad[t, r, k]) <= 0.03 * max(abs(fd), 1e-3) + 2e-5:
                    ok += 1
                else:
                    bad += 1
    assert ok >= 20 and bad <= 0.1 * (ok + bad), (ok, bad)
    g.close()


def test_learned_table_through_decode_path(ldpc):
    """A trained-style table decodes identically through the regular fp32 decode entry."""
    wl = make_workload("BG2", 16, 20, 2.0, modulation="BPSK", seed=8)
    T = 6
    prm = _params(T, wl.n_rows, 9)
    g = ldpc.Graph(wl.base, wl.K_b, 16)
    tab = torch.from_numpy(prm).cuda()
    bits, it, post, _ = ldpc.decode(g, torch.from_numpy(wl.llr).cuda(), T,
                                    algo=ldpc.LEARNED, learned=tab, early_stop=False, debug=True)
    torch.cuda.synchronize()
    ref = oracle.decode_layered(wl.base, wl.K_b, 16, wl.n_rows, wl.llr, algo=oracle.LEARNED,
                                learned=prm, max_iter=T, early_stop=False, want_post=True)
    assert np.array_equal(post.cpu().numpy(), ref.post)
    g.close()


def test_training_reduces_loss(ldpc):
    from paper_2009_05534_gb300 import learned
    wl = make_workload("BG2", 16, 512, 1.5, modulation="BPSK", seed=21)
    g = ldpc.Graph(wl.base, wl.K_b, 16)
    llr = torch.from_numpy(wl.llr).cuda()
    cw = torch.from_numpy(wl.codewords).cuda()
    batches = [(llr, cw)] * 60
    p, hist = learned.train(g, wl.n_rows, 5, batches, lr=1e-2)
    assert hist[-1] < hist[0]
    assert np.isfinite(hist).all()
    g.close()


def test_trained_table_gains_over_plain_min_sum(ldpc):
    """The committed table (trained by the hand-written kernels on 2^20 synthetic codewords)
    against plain normalised min-sum on the same fresh codewords at 2.75 dB, 10 iterations,
    binary16: plain fails on almost every codeword there, the learned decoder on almost none."""
    import os

    from paper_2009_05534_gb300.train_learned import TABLE_DIR, load_table
    path = os.path.join(TABLE_DIR, "learned_bg2_z128_t10.json")
    table, meta = load_table(path)
    wl = make_workload("BG2", 128, 2048, 2.75, seed=31337, graph_seed=0)
    g = ldpc.Graph(wl.base, wl.K_b, 128)
    h = torch.from_numpy(wl.llr_fp16()).cuda()
    bits_p, _ = ldpc.decode(g, h, meta["T"], algo=ldpc.NORMALISED, alpha=0.75, early_stop=False)
    bits_l, _ = ldpc.decode(g, h, meta["T"], algo=ldpc.LEARNED,
                            learned=torch.from_numpy(table).cuda(), early_stop=False)
    torch.cuda.synchronize()
    bler_p = (ldpc.unpack_bits(bits_p.cpu().numpy(), wl.K) != wl.info).any(1).mean()
    bler_l = (ldpc.unpack_bits(bits_l.cpu().numpy(), wl.K) != wl.info).any(1).mean()
    assert bler_p > 0.5 and bler_l < 0.02, (bler_p, bler_l)
    g.close()


def test_checkpoint_resume_equals_uninterrupted(ldpc, tmp_path):
    """Training 3 steps, stopping, and resuming from the checkpoint to 6 steps gives the same
    table as 6 uninterrupted steps (deterministic kernels, Adam state restored)."""
    from paper_2009_05534_gb300 import learned
    wl = make_workload("BG2", 16, 256, 1.5, modulation="BPSK", seed=44)
    g = ldpc.Graph(wl.base, wl.K_b, 16)
    llr = torch.from_numpy(wl.llr).cuda()
    cw = torch.from_numpy(wl.codewords).cuda()

    def batch(k):
        sl = slice((k % 4) * 64, (k % 4) * 64 + 64)
        return llr[sl], cw[sl]

    w = np.full(4, 0.25)
    ref, _ = learned.train(g, wl.n_rows, 4, batch, n_steps=6, lr=1e-2, iter_weights=w,
                           detach=True)
    ck = tmp_path / "ck.pt"
    learned.train(g, wl.n_rows, 4, batch, n_steps=3, lr=1e-2, iter_weights=w, detach=True,
                  checkpoint=ck)
    res, hist = learned.train(g, wl.n_rows, 4, batch, n_steps=6, lr=1e-2, iter_weights=w,
                              detach=True, checkpoint=ck)
    assert len(hist) == 6
    assert torch.equal(res, ref)
    g.close()


def test_training_recipe_end_to_end(ldpc, tmp_path):
    """The training command on a tiny budget: generates, trains, evaluates, writes a table
    that loads back with its recipe."""
    from paper_2009_05534_gb300 import train_learned
    out = tmp_path / "t.json"
    train_learned.main(["--Z", "16", "--T", "4", "--codewords", "2048", "--batch", "512",
                        "--epochs", "1", "--lr", "0.01", "--eval-codewords", "512",
                        "--eval-grid", "2.0:3.0:0.5", "--out", str(out)])
    table, meta = train_learned.load_table(out)
    assert table.shape == (4, 42, 2) and np.isfinite(table).all()
    assert meta["training"]["steps"] == 4 and len(meta["eval"]["bler_plain"]) == 3
