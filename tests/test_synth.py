"""Pins of the seeded input generators (Philox, graphs, encoders, channel, quantiser)."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from synth import (SHAPES, encode_gaussian, encode_structured, expand_H, generate_base_graph,
                   info_bits, make_workload, modulate_llr, philox4x32, quantize_int8,
                   rate_params, std_normals)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _h(x):
    return int(x, 16) if isinstance(x, str) else int(x)


def test_philox_known_answers():
    kat = json.load(open(os.path.join(GOLDEN, "philox_kat.json")))
    for v in kat["vectors"]:
        c = [_h(x) for x in v["ctr"]]
        k = [_h(x) for x in v["key"]]
        out = philox4x32(*c, *k)
        assert [int(o) for o in out] == [_h(x) for x in v["out"]]


@pytest.mark.parametrize("kind", ["BG1", "BG2", "TINY"])
@pytest.mark.parametrize("seed", [0, 1, 7])
def test_graph_shape(kind, seed):
    """Sec. II structure: K_b systematic columns, dual-diagonal core, degree-1 extensions."""
    sh = SHAPES[kind]
    H = generate_base_graph(kind, seed)
    assert H.shape == (sh.M, sh.N) and H.dtype == np.int16
    assert ((H == -1) | ((H >= 0) & (H < 384))).all()
    Kb = sh.K_b
    nz = H >= 0
    # core parity pattern
    assert [tuple(nz[r, Kb:Kb + 4]) for r in range(4)] == [
        (True, True, False, False), (True, True, True, False),
        (False, False, True, True), (True, False, False, True)]
    assert H[0, Kb] == H[3, Kb] and H[1, Kb] == 0
    assert H[0, Kb + 1] == H[1, Kb + 1] == H[1, Kb + 2] == H[2, Kb + 2] == 0
    assert H[2, Kb + 3] == H[3, Kb + 3] == 0
    assert nz[0, 0] and not nz[0, 1] and nz[1:4, 0:2].all()
    assert not nz[:4, Kb + 4:].any()
    if sh.core_deg is not None:
        assert (nz[:4].sum(axis=1) == sh.core_deg).all()
    for r in range(4, sh.M):
        row = nz[r]
        assert H[r, Kb + r] == 0                       # identity on own parity column
        assert row[Kb + 4:].sum() == 1                 # only its own extension column
        assert row[0] != row[1]                        # exactly one of columns 0, 1
        assert sh.ext_deg_lo <= row.sum() <= sh.ext_deg_hi
    assert (nz[:, :Kb + 4].sum(axis=0) >= 2).all()
    assert (nz[:, Kb + 4:].sum(axis=0) == 1).all()


def test_graph_deterministic_and_seeded():
    a = generate_base_graph("BG1", 0)
    assert (a == generate_base_graph("BG1", 0)).all()
    assert not (a == generate_base_graph("BG1", 1)).all()


def test_bg1_edge_count_near_paper():
    """Sec. IV: BG1 row weights run 3..19 and S_c->v = 121 kB at eps=1, Z=384 (E ~ 315)."""
    E = [(generate_base_graph("BG1", s) >= 0).sum() for s in range(8)]
    assert 280 <= np.mean(E) <= 340


@pytest.mark.parametrize("kind,rate,m", [
    ("BG1", "1/3", 46), ("BG1", "1/2", 24), ("BG1", "2/3", 13), ("BG1", "5/6", 7), ("BG1", "8/9", 5),
    ("BG2", "1/5", 42), ("BG2", "1/3", 22), ("BG2", "1/2", 12), ("BG2", "2/3", 7), ("BG2", "5/6", 4),
    ("BG2", "8/9", 4)])
def test_rate_rows(kind, rate, m):
    """Sec. II: R = K/N and rate set by the number of rows used."""
    sh = SHAPES[kind]
    for Z in (16, 384):
        mm, n_tx = rate_params(kind, Z, Fraction(rate))
        assert mm == m
        assert n_tx == int(Fraction(sh.K_b * Z) / Fraction(rate) + Fraction(1, 2))
        assert Z * (sh.K_b + mm - 2) >= n_tx > Z * (sh.K_b + mm - 3) or mm == 4


@pytest.mark.parametrize("kind,Z", [("BG1", 8), ("BG1", 16), ("BG2", 16), ("BG2", 13), ("TINY", 3)])
def test_encoders_parity_and_agree(kind, Z):
    """P1: H c = 0 over GF(2) for every encoded word; the two encoders agree bit for bit."""
    sh = SHAPES[kind]
    base = generate_base_graph(kind, 3)
    u = info_bits(5, 24, sh.K_b * Z)
    c1 = encode_structured(base, sh.K_b, Z, u)
    c2 = encode_gaussian(base, sh.K_b, Z, u)
    assert (c1 == c2).all()
    assert (c1[:, : sh.K_b * Z] == u).all()
    H = expand_H(base, Z).astype(np.int64)
    assert ((H @ c1.T.astype(np.int64)) % 2 == 0).all()


def _syndrome_rolls(base, Z, n_rows, cw):
    """GF(2) syndrome of codewords [B][cols*Z] written with circulant rolls."""
    B = cw.shape[0]
    x = cw.reshape(B, -1, Z)
    bad = 0
    for r in range(n_rows):
        acc = np.zeros((B, Z), np.uint8)
        for c in range(x.shape[1]):
            v = int(base[r, c])
            if v >= 0:
                acc ^= np.roll(x[:, c, :], -(v % Z), axis=1)
        bad += int(acc.sum())
    return bad


@pytest.mark.parametrize("kind,Z,rate", [("BG1", 384, None), ("BG1", 384, "8/9"), ("BG2", 128, "1/3")])
def test_encoder_large_lifting(kind, Z, rate):
    sh = SHAPES[kind]
    wl = make_workload(kind, Z, 4, 2.0, rate=None if rate is None else Fraction(rate))
    assert _syndrome_rolls(wl.base, Z, wl.n_rows, wl.codewords) == 0
    c2 = encode_gaussian(wl.base, sh.K_b, Z, wl.info, wl.n_rows)
    assert (c2 == wl.codewords).all()


def test_info_bits_balanced():
    u = info_bits(0, 64, 8448)
    assert abs(u.mean() - 0.5) < 0.01
    assert not (u[0] == u[1]).all()


def test_normals_moments():
    z = std_normals(0, 64, 4096)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    # same normals at every first_cw offset slice (common random numbers across calls)
    z2 = std_normals(0, 8, 4096, first_cw=3)
    assert np.array_equal(z2[0], z[3])


@pytest.mark.parametrize("mod", ["BPSK", "QPSK"])
def test_llr_consistency(mod):
    """An AWGN bit LLR with bit 0 sent is Gaussian with mean mu and variance 2 mu."""
    bits = np.zeros((32, 8192), np.uint8)
    L = modulate_llr(bits, 1.0, 1 / 3, mod, seed=11).astype(np.float64)
    mu, var = L.mean(), L.var()
    m = 1 if mod == "BPSK" else 2
    n0 = 1.0 / ((1 / 3) * m * 10 ** 0.1)
    A2 = 1.0 if mod == "BPSK" else 0.5
    assert abs(mu - 4 * A2 / n0) / mu < 0.02
    assert abs(var - 2 * mu) / (2 * mu) < 0.03
    # sign convention: LLR = ln P(0)/P(1), bit 1 -> negative mean
    L1 = modulate_llr(np.ones((4, 4096), np.uint8), 1.0, 1 / 3, mod, seed=11)
    assert L1.mean() < 0


@pytest.mark.parametrize("m", [4, 6])
def test_qam_maxlog_against_2d_enumeration(m):
    """Max-log LLR of bit k = (min over constellation points with bit k = 1 of |y-x|^2
    - min over points with bit k = 0) / N0, enumerated over the full 2-D constellation and
    compared with the per-axis implementation; unit average symbol energy; Gray labels."""
    from synth.channel import pam_map, pam_maxlog_llr
    mh = m // 2
    L = 1 << mh
    # every m-bit label, first mh bits on I, next mh on Q
    labels = np.array(list(itertools.product([0, 1], repeat=m)), np.uint8)
    xi = pam_map(labels[:, :mh], mh)
    xq = pam_map(labels[:, mh:], mh)
    assert abs(np.mean(xi ** 2 + xq ** 2) - 1.0) < 1e-12
    assert len(set(zip(xi.round(9), xq.round(9)))) == 1 << m
    # Gray property: neighbouring levels on an axis differ in exactly one label bit
    pts1 = np.unique(xi.round(12))
    for a_, b_ in zip(pts1[:-1], pts1[1:]):
        la = labels[np.isclose(xi, a_)][0, :mh]
        lb = labels[np.isclose(xi, b_)][0, :mh]
        assert (la != lb).sum() == 1
    rng = np.random.default_rng(m)
    n0 = 0.3
    for _ in range(200):
        y = rng.standard_normal(2) * 0.8
        d2 = (y[0] - xi) ** 2 + (y[1] - xq) ** 2
        want = [(d2[labels[:, k] == 1].min() - d2[labels[:, k] == 0].min()) / n0 for k in range(m)]
        got = np.concatenate([pam_maxlog_llr(np.array([y[0]]), mh, n0)[0],
                              pam_maxlog_llr(np.array([y[1]]), mh, n0)[0]])
        assert np.allclose(got, want, atol=1e-12)


@pytest.mark.parametrize("mod", ["16QAM", "64QAM"])
def test_qam_high_snr_hard_decisions(mod):
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2, size=(3, 600)).astype(np.uint8)
    L = modulate_llr(bits, 30.0, 0.5, mod, seed=4)
    assert ((L < 0).astype(np.uint8) == bits).all()


def test_quantize_int8():
    x = np.array([0.125, 0.375, -0.125, -0.375, 31.875, 40.0, -40.0, 0.0, 2.6], np.float32)
    q = quantize_int8(x, 4.0)
    # 4x = 0.5 -> 0 (half to even), 1.5 -> 2, -0.5 -> 0, -1.5 -> -2, 127.5 -> 127 (clamp),
    # 160 -> 127, -160 -> -127 (never -128), 0, 10.4 -> 10
    assert q.tolist() == [0, 2, 0, -2, 127, 127, -127, 0, 10]
    big = quantize_int8(np.linspace(-1000, 1000, 10001, dtype=np.float32))
    assert big.min() == -127 and big.max() == 127


@pytest.mark.parametrize("mod", ["BPSK", "QPSK", "16QAM", "64QAM"])
def test_per_codeword_ebn0_matches_scalar(mod):
    """A batch with one Eb/N0 per codeword equals each codeword generated alone."""
    e = np.array([0.5, 1.0, 2.5, 1.0, 0.7])
    w = make_workload("BG2", 16, 5, e, modulation=mod, seed=3, graph_seed=0)
    assert np.array_equal(w.meta["ebn0_db"], e)
    for b in range(5):
        w1 = make_workload("BG2", 16, 1, float(e[b]), modulation=mod, seed=3, graph_seed=0,
                           first_cw=b)
        assert np.array_equal(w1.llr[0], w.llr[b])


def test_threaded_normals_match_single_range():
    from synth.channel import _std_normals, std_normals
    a = std_normals(11, 700, 6001, first_cw=5)          # large enough to take the pool
    assert np.array_equal(a, _std_normals(11, 700, 6001, 5))
    assert np.array_equal(a[123], _std_normals(11, 1, 6001, 5 + 123)[0])


@pytest.mark.parametrize("mod", ["QPSK", "16QAM", "64QAM"])
def test_llr_sweep_equals_one_point_at_a_time(mod):
    """The Eb/N0 sweep helper reuses symbols and normals; each of its LLR arrays equals the
    single-point channel, also when the max-log demapper splits rows over threads."""
    from fractions import Fraction

    from synth.channel import modulate_llr, modulate_llr_sweep
    wl = make_workload("BG1", 64, 300, 3.0, rate=Fraction(2, 3), modulation=mod, seed=4)
    tx = wl.codewords[:, wl.punct_cols * 64: wl.punct_cols * 64 + wl.n_tx]
    grid = [2.5, 3.0, 4.25]
    for e, got in zip(grid, modulate_llr_sweep(tx, grid, wl.meta["rate"], mod, 4)):
        assert np.array_equal(got, modulate_llr(tx, e, wl.meta["rate"], mod, 4))
    assert np.array_equal(
        next(modulate_llr_sweep(tx, [3.0], wl.meta["rate"], mod, 4)), wl.llr)


def test_threaded_maxlog_equals_serial():
    from synth.channel import _pam_maxlog, pam_maxlog_llr
    y = np.random.default_rng(3).normal(size=(256, 5000))
    for mh in (2, 3):
        assert np.array_equal(pam_maxlog_llr(y, mh, 0.37), _pam_maxlog(y, mh, 0.37))
