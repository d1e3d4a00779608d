"""Identities the binary16x2 decode kernels rely on, checked exhaustively in IEEE binary16
(numpy float16 arithmetic rounds every operation to binary16, like the f16x2 instructions).

* 8-bit saturation through two relu FMAs: for every v = L - c with L, c in [-127, 127],
  127 - max(254 - max(v + 127, 0), 0) == clamp(v, -127, 127), and with posteriors stored as
  L + 1279 and messages as c + 1152 the first relu argument is one exact subtraction.
* Posterior and message biases: L + 1279 and c + 1152 are exact and order-preserving.
* Message magnitude without an argmin index: max(m1', (m1 + m2 - 1) - |v|) equals m2' on an
  edge attaining m1 and m1' elsewhere, for the offset-1 correction m' = max(m - 1, 0).
* Second minimum from plain min / max of magnitudes equals the sorted second smallest.
"""
import itertools

import numpy as np

f16 = np.float16


def relu(x):
    return np.maximum(x, f16(0))


def test_relu_saturation_exhaustive():
    L = np.arange(-127, 128).astype(f16)
    c = np.arange(-127, 128).astype(f16)
    LL, CC = np.meshgrid(L, c, indexing="ij")
    Xb = (LL + f16(1279)).astype(f16)              # stored posterior
    Mb = (CC + f16(1152)).astype(f16)              # unpacked message
    y = relu((Xb - Mb).astype(f16))                # fma.relu(M, -1, X)
    z = relu((f16(254) - y).astype(f16))           # fma.relu(y, -1, 254)
    sat = (f16(127) - z).astype(f16)
    want = np.clip(LL.astype(np.int32) - CC.astype(np.int32), -127, 127)
    assert np.array_equal(sat.astype(np.int32), want)
    # every intermediate is an exactly represented integer
    assert np.array_equal((Xb - Mb).astype(np.int32), LL.astype(np.int32) - CC.astype(np.int32) + 127)


def test_biases_exact_and_monotone():
    v = np.arange(-127, 128)
    for bias in (1279, 1152):
        b = (v.astype(f16) + f16(bias)).astype(f16)
        assert np.array_equal(b.astype(np.int32), v + bias)
        assert np.all(np.diff(b.view(np.uint16).astype(np.int64)) == 1)   # pattern = 0x6400 + n
    # the posterior update and its clamp stay inside the exact range [1152, 1406]
    x = np.arange(-127, 128)
    cn = np.arange(-126, 127)
    X, C = np.meshgrid(x, cn, indexing="ij")
    s = ((C + 1152).astype(f16) + (X + 127).astype(f16)).astype(f16).astype(np.int32)
    assert np.array_equal(np.clip(s, 1152, 1406), np.clip(X + C, -127, 127) + 1279)


def test_sigma_trick_offset_one():
    rng = np.random.default_rng(0)
    for d in range(2, 20):
        for _ in range(200):
            a = rng.integers(0, 128, size=d)
            if rng.random() < 0.3:
                a[rng.integers(d)] = a.min()                            # ties
            s = np.sort(a)
            m1, m2 = s[0], s[1]
            m1c, m2c = max(m1 - 1, 0), max(m2 - 1, 0)
            T1 = f16(m1) + f16(m2) + f16(-1)
            for k in range(d):
                ex = max(f16(m1c), f16(T1 - f16(a[k])))
                others = np.delete(a, k)
                assert int(ex) == max(int(others.min()) - 1, 0)


def test_second_minimum_from_plain_min_max():
    rng = np.random.default_rng(1)
    for d in range(2, 21):
        for _ in range(100):
            x = rng.integers(-127, 128, size=d).astype(f16)
            m1, m2 = f16(np.inf), f16(np.inf)
            for v in x:
                m2 = min(m2, max(abs(m1), abs(v)))
                m1 = min(abs(m1), abs(v))
            s = np.sort(np.abs(x.astype(np.float64)))
            assert float(m1) == s[0] and float(m2) == s[1]
