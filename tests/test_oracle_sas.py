"""Pins of the Shift-and-Sample oracle (oracle/sas.py) against the paper and
the mathematics, CPU only."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import rel_l2


def _full_signal(M, J, c):
    """f = F^{-1} c by a library inverse FFT of the zero-filled spectrum."""
    N = 1 << M
    x = np.zeros(N, dtype=np.complex128)
    x[np.asarray(J, dtype=np.int64)] = c
    return np.fft.ifft(x)          # (1/N) sum_k x_k exp(+2 pi i k n / N)


def _run(M, J, R, c):
    r = O.sas_pivots(J, M, R)
    mu = O.sas_mu(J, r)
    idx = O.sas_sample_sets(M, r, max(mu.values()))
    f = _full_signal(M, J, c)
    return r, mu, idx, O.sas_transform(M, J, r, f[idx.astype(np.int64)])


def test_paper_example_two_aliased_coefficients():
    # Section "preliminary observations": N = 1024, J = {0, 512, 1, 6, 7} at
    # level 2: 1, 6, 7 isolated, 0 and 512 aliased, a 2 x 2 Vandermonde
    # system, 8 time-domain samples in all.
    M, J = 10, [0, 512, 1, 6, 7]
    rng = np.random.default_rng(1)
    c = W.complex_gaussian(len(J), rng)
    r, mu, idx, got = _run(M, J, 2, c)
    assert r == [0, 1]
    assert O.sas_nodes(J, r) == {0: [0, 512], 1: [1], 2: [6], 3: [7]}
    assert max(mu.values()) == 2 and idx.size == 8
    assert rel_l2(got, c) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_arbitrary_sets(seed):
    # any set is part-homogeneous for its first R split levels; recovery is
    # exact up to the conditioning of the per-class Vandermonde systems
    rng = np.random.default_rng(100 + seed)
    M = 6 + seed % 3
    k = int(rng.integers(3, 24))
    J = sorted(int(x) for x in rng.choice(1 << M, size=k, replace=False))
    c = W.complex_gaussian(k, rng)
    levels = O.split_levels(J, M)
    for R in range(max(0, len(levels) - 3), len(levels) + 1):
        r, mu, idx, got = _run(M, J, R, c)
        conds = []
        for t, members in O.sas_nodes(J, r).items():
            A = O.sas.__dict__["_z_powers"](M, members, len(members))
            conds.append(np.linalg.cond(A))
        assert rel_l2(got, c) < 1e-13 * max(conds) + 1e-13, (R, max(conds))


def test_homogeneous_sets_reduce_to_algorithm_1():
    rng = np.random.default_rng(7)
    for s in (0, 1, 3, 5):
        M = s + 4
        piv = W.random_pivots(M, s, rng)
        J = W.homogeneous_support(M, piv, rng)
        c = W.complex_gaussian(1 << s, rng)
        r, mu, idx, got = _run(M, J, s, c)
        assert r == [int(p) for p in piv] and max(mu.values()) == 1
        assert idx.shape == (1, 1 << s)
        Jc = O.canonical_support_by_key(J, r)
        f = _full_signal(M, J, c)
        ref = O.transform_levels(M, r, Jc, f[idx[0].astype(np.int64)])
        # SAS returns J's order, Algorithm 1 the canonical order
        pos = {int(j): i for i, j in enumerate(Jc)}
        assert rel_l2(got, np.asarray([ref[pos[int(j)]] for j in J])) < 1e-12
        assert rel_l2(got, c) < 1e-12


@pytest.mark.parametrize("k,d", [(100, 1), (100, 37), (300, 5)])
def test_arithmetic_progressions_are_balanced(k, d):
    # Corollary "AP" / universal sets: class sizes at any level differ by at
    # most one, so R = ceil(log2 k) split levels isolate every coefficient
    M = 12
    rng = np.random.default_rng(k + d)
    a = int(rng.integers(0, 1 << M))
    J = [(a + n * d) % (1 << M) for n in range(k)]
    c = W.complex_gaussian(k, rng)
    Rk = int(np.ceil(np.log2(k)))
    for R in (Rk - 1, Rk):
        r = O.sas_pivots(J, M, R)
        assert r == list(range(R))                   # odd d: consecutive split levels
        mu = list(O.sas_mu(J, r).values())
        assert max(mu) - min(mu) <= 1
    r, mu, idx, got = _run(M, J, Rk, c)
    assert max(mu.values()) == 1
    assert rel_l2(got, c) < 1e-12
    r, mu, idx, got = _run(M, J, Rk - 1, c)
    assert max(mu.values()) == 2
    assert rel_l2(got, c) < 1e-9


def test_node_values_are_modulated_class_sums():
    # Lemma "shift-mod-Hi-DFT" / eq. "alg1_system": the Hi-DFT of the a-th
    # shifted sample set at class v is sum_{j in v} c_j exp(2 pi i a j / N)
    M = 8
    rng = np.random.default_rng(3)
    J = sorted(int(x) for x in rng.choice(1 << M, size=20, replace=False))
    c = W.complex_gaussian(20, rng)
    R = 3
    r = O.sas_pivots(J, M, R)
    nodes = O.sas_nodes(J, r)
    mu_star = max(len(m) for m in nodes.values())
    idx = O.sas_sample_sets(M, r, mu_star)
    f = _full_signal(M, J, c)
    Y = O.sas_node_values(M, J, r, f[idx.astype(np.int64)])
    cj = dict(zip(J, c))
    for t in range(1 << R):
        for a in range(mu_star):
            want = sum(cj[j] * np.exp(2j * np.pi * ((a * j) % (1 << M)) / (1 << M)) for j in nodes.get(t, []))
            assert abs(Y[a, t] - want) < 1e-11 * (1 + abs(want)), (t, a)


def test_virtual_support_is_homogeneous_with_the_chosen_pivots():
    rng = np.random.default_rng(11)
    for _ in range(40):
        M = int(rng.integers(5, 10))
        k = int(rng.integers(2, 30))
        J = sorted(int(x) for x in rng.choice(1 << M, size=k, replace=False))
        levels = O.split_levels(J, M)
        R = int(rng.integers(0, len(levels) + 1))
        r = levels[:R]
        V = O.virtual_support(J, M, r)
        assert O.is_homogeneous(V, M) and O.pivots_by_tree(V, M) == r
        assert [O.node_key(v, r) for v in V] == list(range(1 << R))
        rho = (r[-1] + 1) if R else 0
        for t, members in O.sas_nodes(J, r).items():
            assert all(j % (1 << rho) == int(V[t]) for j in members)


def test_planted_shift_sign_fails():
    # samples at I_r - a instead of I_r + a conjugate the Vandermonde nodes
    # (0 and 256 alias at level 2 with z = 1 and z = i)
    M, J = 10, [0, 256, 1, 6, 7]
    rng = np.random.default_rng(2)
    c = W.complex_gaussian(len(J), rng)
    r = O.sas_pivots(J, M, 2)
    I = O.sample_set(M, r).astype(np.int64)
    f = _full_signal(M, J, c)
    wrong = np.stack([f[(I - a) % (1 << M)] for a in range(2)])
    assert rel_l2(O.sas_transform(M, J, r, wrong), c) > 1e-3


def test_sample_complexity_is_mu_star_times_2R():
    # Lemma "computation_shift_sample": mu* shifted Hi-DFTs of 2^R samples
    M = 12
    rng = np.random.default_rng(5)
    J = sorted(int(x) for x in rng.choice(1 << M, size=50, replace=False))
    for R in range(0, 7):
        r = O.sas_pivots(J, M, R)
        mu = O.sas_mu(J, r)
        idx = O.sas_sample_sets(M, r, max(mu.values()))
        assert idx.shape == (max(mu.values()), 1 << R)
        assert sum(mu.values()) == len(J)


@pytest.mark.parametrize("log2k", [8, 10, 12])
def test_random_subsets_alias_at_most_c_log_k(log2k):
    # Lemma "bound_mu_r_star" / Theorem "hom_rand_subset": keep every element of
    # a homogeneous K independently with probability k/|K|; with the first n
    # pivots of K, n = floor(log2 k - log2 log2 k), the largest class stays
    # below c log2 k, c = 4 + 3 ln 2, and SAS recovers the coefficients
    k = 1 << log2k
    c_const = 4 + 3 * np.log(2)
    for seed in range(3):
        rng = W.rng_for(0, 900 + 10 * log2k + seed)
        M = log2k + 8
        J, piv = W.bernoulli_subset_of_homogeneous(M, log2k + 3, k, rng)
        J = [int(j) for j in J]
        n = int(np.floor(log2k - np.log2(log2k)))
        r = O.sas_pivots(J, M, n)
        assert r == [int(p) for p in piv[:n]]            # J splits where K does, w.h.p.
        mu = O.sas_mu(J, r)
        assert max(mu.values()) < c_const * log2k
        if log2k <= 10:
            c = W.complex_gaussian(len(J), rng)
            idx = O.sas_sample_sets(M, r, max(mu.values()))
            F = O.sas_samples_direct(M, J, c, idx)
            got = O.sas_transform(M, J, r, F)
            conds = [np.linalg.cond(O.sas.__dict__["_z_powers"](M, m, len(m))) for m in O.sas_nodes(J, r).values()]
            assert rel_l2(got, c) < 1e-14 * max(conds) + 1e-12


def test_union_of_elementary_example():
    # Lemma "UoE1" example: {31, 22}, {3, 4, 9, 10} and {1, 2, 3, 4, 8, 13, 22, 23}
    # are elementary (one element per class mod 2, 4, 8) and, with {0}, their
    # union keeps the pivots 0, 1, 2. (The printed J omits the 0 of the
    # printed union; the union is taken as the set.)
    parts = [[0], [31, 22], [3, 4, 9, 10], [1, 2, 3, 4, 8, 13, 22, 23]]
    for i, p in enumerate(parts):
        assert O.is_homogeneous(p, 5) and O.pivots_by_tree(p, 5) == list(range(i))
    J = sorted(set().union(*map(set, parts)))
    assert O.split_levels(J, 5)[:3] == [0, 1, 2]
    rng = np.random.default_rng(12)
    c = W.complex_gaussian(len(J), rng)
    for R in (2, 3):
        r, mu, idx, got = _run(5, J, R, c)
        assert rel_l2(got, c) < 1e-11


@pytest.mark.parametrize("base", ["elementary", "homogeneous"])
def test_union_of_homogeneous_alias_bound(base):
    # Proposition "UoE-mu-r-star-bound" (and its homogeneous analogue under
    # Theorem "UoE2"): at the s-th pivot level, s <= a, every class holds at most
    # C (s + 2^(a-s+1) - 1) members, C = max eta_i; the union keeps the parts' pivots
    for seed in range(4):
        rng = W.rng_for(0, 5000 + seed)
        M, a = 14, 6
        l = list(range(M)) if base == "elementary" else [int(x) for x in W.random_pivots(M, a + 3, rng)]
        etas = [int(x) for x in rng.integers(1, 4, size=a + 1)]
        J, parts = W.union_of_homogeneous(M, l, etas, rng, rng)
        J = [int(j) for j in J]
        C = max(etas)
        assert O.split_levels(J, M)[:a] == l[:a]
        for s in range(1, a + 1):
            mu = O.sas_mu(J, l[:s])
            assert max(mu.values()) <= C * (s + 2 ** (a - s + 1) - 1), (s, max(mu.values()))
        c = W.complex_gaussian(len(J), rng)
        r, mu, idx, got = _run(M, J, a, c)
        conds = [np.linalg.cond(O.sas.__dict__["_z_powers"](M, m, len(m))) for m in O.sas_nodes(J, r).values()]
        assert rel_l2(got, c) < 1e-14 * max(conds) + 1e-12


@pytest.mark.parametrize("sizes", [(8, 8), (5, 6, 7), (16, 3)])
def test_generalized_progressions_have_few_pivots(sizes):
    # Lemma "gap-complexity", eq. "gap-pivot-bound": a proper GAP of dimension d
    # with n split levels satisfies 2^n <= n^d 2^d |J|; SAS recovers its coefficients
    d = len(sizes)
    for seed in range(4):
        rng = W.rng_for(0, 7000 + 17 * seed + sum(sizes))
        M = 20
        J = [int(j) for j in W.generalized_arithmetic_progression(M, sizes, rng)]
        n = len(O.split_levels(J, M))
        assert 2 ** n <= n ** d * 2 ** d * len(J), (n, len(J))
    c = W.complex_gaussian(len(J), rng)
    levels = O.split_levels(J, M)
    R = min(len(levels), int(np.ceil(np.log2(len(J)))) + 1)
    r = O.sas_pivots(J, M, R)
    mu = O.sas_mu(J, r)
    idx = O.sas_sample_sets(M, r, max(mu.values()))
    F = O.sas_samples_direct(M, J, c, idx)
    got = O.sas_transform(M, J, r, F)
    conds = [np.linalg.cond(O.sas.__dict__["_z_powers"](M, m, len(m))) for m in O.sas_nodes(J, r).values()]
    assert rel_l2(got, c) < 1e-14 * max(conds) + 1e-12
