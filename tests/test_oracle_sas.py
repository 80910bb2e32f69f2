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


# ---- operation counts: Lemma "computation_shift_sample" and the worked example ----

def _golden_opcount():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "sas_example_sec9_opcount.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = [x.strip() for x in line.split("|")]
            rows.append((int(f[0]), [int(x) for x in f[1].split()], int(f[2]), int(f[3]), int(f[4]),
                         int(f[5]), int(f[6])))
    return rows


def _counted(M, J, R, c):
    r = O.sas_pivots(J, M, R)
    mu = O.sas_mu(J, r)
    idx = O.sas_sample_sets(M, r, max(mu.values()))
    f = _full_signal(M, J, c)
    cnt = {}
    got = O.sas_transform(M, J, r, f[idx.astype(np.int64)], counter=cnt)
    return r, mu, idx, got, cnt


def test_worked_example_operation_count_is_the_papers():
    # Section IX: two size-4 Hi-DFTs at 12 operations each, one 2 x 2 system at
    # 5 operations: 29 operations, 8 samples (tests/golden/sas_example_sec9_opcount.txt)
    for M, J, R, t_ops, s_ops, total, samples in _golden_opcount():
        c = W.complex_gaussian(len(J), np.random.default_rng(5))
        r, mu, idx, got, cnt = _counted(M, J, R, c)
        assert cnt["transform_ops"] == t_ops
        assert cnt["solve_ops"] == s_ops
        assert cnt["transform_ops"] + cnt["solve_ops"] == total
        assert idx.size == samples
        assert rel_l2(got, c) < 1e-12


def test_vandermonde_solve_against_a_library_solve():
    # the O(mu^2) class solve equals an LU solve of the same system and leaves
    # no residual; 5 mu (mu - 1) / 2 operations
    rng = np.random.default_rng(17)
    for mu in range(1, 9):
        for _ in range(5):
            M = int(rng.integers(mu.bit_length() + 2, 14))
            members = sorted(int(x) for x in rng.choice(1 << M, size=mu, replace=False))
            A = O.sas.__dict__["_z_powers"](M, members, mu)
            y = W.complex_gaussian(mu, rng)
            cnt = {}
            z = O.sas.__dict__["_z_powers"](M, members, 2)[1]       # z_u = exp(2 pi i l_u / N)
            x = O.vandermonde_solve(z, y, cnt)
            ref = np.linalg.solve(A, y)
            cond = np.linalg.cond(A)
            assert rel_l2(x, ref) < 1e-12 * cond + 1e-14, (mu, cond)
            assert rel_l2(A @ x, y) < 1e-12 * cond + 1e-14
            assert cnt["solve_ops"] == 5 * mu * (mu - 1) // 2


@pytest.mark.parametrize("seed", range(5))
def test_lemma_count_matches_the_instrumented_run(seed):
    # Lemma "computation_shift_sample": the mu* transforms of 2^R values cost
    # c1 R 2^R mu* (c1 = 3/2, counted butterfly by butterfly), the class solves
    # at most c2 sum mu(v)^2 (c2 = 6; the O(mu^2) solver needs 5 mu (mu - 1) / 2);
    # sas_cost adds exactly these two terms for the classes the run solved
    rng = np.random.default_rng(300 + seed)
    M = int(rng.integers(7, 12))
    k = int(rng.integers(4, 60))
    J = sorted(int(x) for x in rng.choice(1 << M, size=k, replace=False))
    c = W.complex_gaussian(k, rng)
    levels = O.split_levels(J, M)
    for R in range(max(1, len(levels) - 3), len(levels) + 1):
        r, mu, idx, got, cnt = _counted(M, J, R, c)
        mu_star = max(mu.values())
        assert cnt["transforms"] == mu_star
        assert cnt["transform_ops"] == 1.5 * R * (1 << R) * mu_star
        assert cnt["solve_mu2"] == sum(m * m for m in mu.values())
        assert cnt["solve_ops"] <= 6 * cnt["solve_mu2"]
        assert O.sas_cost(R, mu) == cnt["transform_ops"] + 6 * cnt["solve_mu2"]
        # the instrumented run computes the same coefficients as the plain one
        plain = O.sas_transform(M, J, r, _full_signal(M, J, c)[idx.astype(np.int64)])
        conds = [np.linalg.cond(O.sas.__dict__["_z_powers"](M, m, len(m))) for m in O.sas_nodes(J, r).values()]
        assert rel_l2(got, plain) < 1e-12 * max(conds) + 1e-13


def test_planted_constant_mistake_fails_the_worked_example():
    # c1 = 2 (the alternative the lemma's proof mentions) would give 16 operations
    # per size-4 transform and 37 in all, not the paper's 29
    M, J, R, t_ops, s_ops, total, samples = _golden_opcount()[0]
    mu = O.sas_mu(J, O.sas_pivots(J, M, R))
    mu_star = max(mu.values())
    wrong = 2.0 * R * (1 << R) * mu_star + s_ops
    assert wrong != total
    assert 1.5 * R * (1 << R) * mu_star + s_ops == total
