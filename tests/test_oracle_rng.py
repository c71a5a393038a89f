"""Pins for the oracle's random-number layer (not GPU).

* Philox4x32-10 is pinned against cuRAND's host-side Philox4_32_10 generator,
  a library routine: its output block b for seed s equals Philox with key
  (s mod 2^32, s div 2^32) and counter (b div 65536, 0, b mod 65536, 0).
* Uniforms are pinned by exactness and range identities.
* Box-Muller normals are pinned by a Kolmogorov-Smirnov test against N(0,1)
  and by their first two moments.
* Gumbel-max sampling is pinned by a chi-square test of action frequencies
  against softmax(logits) (Sec. 3.3: actions are sampled from a softmax).
* Bernoulli thresholds are pinned by the closed form floor(p * 2^32) computed
  with exact rationals.
"""
import ctypes
import ctypes.util
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import inputs


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if not cand:
            continue
        try:
            return ctypes.CDLL(cand)
        except OSError:
            continue
    return None


def _curand_host_philox(seed, n):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    PHILOX4_32_10 = 161  # curandRngType_t value of CURAND_RNG_PSEUDO_PHILOX4_32_10
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(n, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 7, 0x0123456789ABCDEF])
def test_philox_matches_curand_host_generator(seed):
    n_blocks = 65536 + 512  # crosses into counter word 0 = 1
    ref = _curand_host_philox(seed, 4 * n_blocks).reshape(-1, 4)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    picks = list(range(0, 64)) + list(range(65536 - 32, 65536 + 512)) + \
        list(inputs.rng(seed & 0xFFFF).integers(0, n_blocks, 200))
    for b in picks:
        got = oracle.philox((b >> 16, 0, b & 0xFFFF, 0), key)
        assert got == [int(v) for v in ref[b]], (seed, b)


def test_philox_depends_on_every_counter_and_key_word():
    base = oracle.philox((1, 2, 3, 4), (5, 6))
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert oracle.philox(c, (5, 6)) != base
    assert oracle.philox((1, 2, 3, 4), (4, 6)) != base
    assert oracle.philox((1, 2, 3, 4), (5, 7)) != base


def test_uniform_exact_open_interval():
    words = list(inputs.random_words(2000, seed=1)) + [0, 1, 255, 256, 0xFFFFFFFF, 0xFFFFFF00]
    for r in words:
        u = oracle.uniform(int(r))
        assert 0.0 < u < 1.0
        k = u * 2**24
        assert k == int(k) and int(k) % 2 == 1          # an odd multiple of 2^-24
        assert float(np.float32(u)) == u                  # exact in binary32
        assert int(k) >> 1 == int(r) >> 9                 # the draw's top 23 bits
    assert oracle.uniform(0) == 2.0**-24
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 2.0**-24


def test_box_muller_normals_are_standard_normal():
    from scipy import stats
    w = inputs.random_words(4 * 60000, seed=2).reshape(-1, 4)
    n = np.array([oracle.normals4(row) for row in w]).ravel()
    assert abs(n.mean()) < 0.01
    assert abs(n.var() - 1.0) < 0.01
    assert stats.kstest(n, "norm").pvalue > 1e-3
    # the two members of a pair are uncorrelated
    assert abs(np.corrcoef(n[0::4], n[1::4])[0, 1]) < 0.02


def test_gumbel_max_frequencies_match_softmax():
    from scipy import stats
    logits = np.array([0.3, -1.0, 1.2, 0.0, 0.7, -0.4])
    p = np.exp(logits - logits.max())
    p /= p.sum()
    draws = 40000
    w = inputs.random_words(draws * len(logits), seed=3).reshape(draws, len(logits))
    counts = np.zeros(len(logits))
    for row in w:
        g = [oracle.gumbel(int(r)) for r in row]
        counts[int(np.argmax(logits + np.array(g)))] += 1
    chi2 = stats.chisquare(counts, p * draws)
    assert chi2.pvalue > 1e-3, (counts, p * draws)


def test_gumbel_closed_form_values():
    # u = 2^-24 * odd; G(u) = -ln(-ln u): check two exact points by rationals
    r = (0x800000 << 8)  # top 24 bits = 2^23 -> u = (2^23 | 1) / 2^24 ~ 0.5
    u = (2**23 | 1) / 2**24
    assert abs(oracle.gumbel(r) - (-np.log(-np.log(u)))) < 1e-15


@pytest.mark.parametrize("p", [0.0, 0.005, 0.01, 0.02, 0.05, 0.1, 0.5, 0.999])
def test_threshold_closed_form(p):
    exact = Fraction(float(np.float32(p))) * 2**32
    want = min(int(exact), 2**32 - 1)  # floor of a non-negative rational
    assert oracle.threshold(p) == want


def test_threshold_rate():
    thr = oracle.threshold(0.05)
    w = inputs.random_words(400000, seed=4)
    rate = float(np.mean(w < thr))
    assert abs(rate - 0.05) < 0.002
