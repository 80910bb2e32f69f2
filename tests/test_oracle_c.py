"""Pins of the C restatement of Algorithm 1 (oracle/alg1.c) against the paper
(brute force) and the pinned numpy oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import rel_l2
from oracle import alg1


def test_brute_force_n16_k4():
    # c = (Ff)_J for f = F^{-1} c by a library inverse FFT (N = 16, k = 4)
    rng = np.random.default_rng(16)
    for _ in range(5):
        piv = W.random_pivots(4, 2, rng)
        J = W.homogeneous_support(4, piv, rng)
        Jc = O.canonical_support_by_key(J, piv)
        c = W.complex_gaussian(4, rng)
        x = np.zeros(16, dtype=np.complex128)
        x[Jc.astype(np.int64)] = c
        f = np.fft.ifft(x)[O.sample_set(4, piv).astype(np.int64)]
        got, _ = alg1.alg1_batch(4, piv, Jc, f)
        assert rel_l2(got, c) < 1e-14


@pytest.mark.parametrize("s", [0, 1, 3, 7, 12, 14])
def test_matches_numpy_oracle(s):
    rng = np.random.default_rng(100 + s)
    M = s + 6
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    Jc = O.canonical_support_by_key(J, piv)
    F = W.complex_gaussian((5, 1 << s), rng)
    got, used = alg1.alg1_batch(M, piv, Jc, F, threads=2)
    ref = O.transform_levels(M, piv, Jc, F)
    assert used >= 1
    assert rel_l2(got, ref) < 1e-13


def test_large_pivots():
    # pivots near the top of a 60-bit index space (reduction of Jc mod 2^r)
    rng = np.random.default_rng(7)
    M, s = 60, 6
    piv = np.sort(rng.choice(np.arange(50, 60), size=s, replace=False))
    J = W.homogeneous_support(M, piv, rng)
    Jc = O.canonical_support_by_key(J, piv)
    F = W.complex_gaussian((2, 1 << s), rng)
    got, _ = alg1.alg1_batch(M, piv, Jc, F)
    assert rel_l2(got, O.transform_levels(M, piv, Jc, F)) < 1e-12


@pytest.mark.parametrize("M,s", [(30, 10), (40, 6), (62, 8)])
def test_large_N_against_closed_form(M, s):
    # at large N the C oracle's twiddles (angles 2 pi rho / 2^(r+1) with r up to
    # 61) must still give c_j = (N/k) sum_i f(i) exp(-2 pi i (i j mod N) / N)
    rng = np.random.default_rng(500 + M)
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    Jc = O.canonical_support_by_key(J, piv)
    F = W.complex_gaussian((2, 1 << s), rng)
    got, _ = alg1.alg1_batch(M, piv, Jc, F, threads=2)
    I = O.sample_set(M, piv)
    pick = rng.choice(1 << s, size=8, replace=False)
    for b in range(2):
        ref = O.coefficients_at(M, Jc[pick], I, F[b])
        assert rel_l2(got[b][pick], ref) < 1e-12
