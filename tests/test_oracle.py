"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each check is independent of the oracle's own formulas: the paper's printed
values (tests/golden), a library FFT on the zero-filled full spectrum, closed
forms, invariants the paper proves, and brute force on small inputs.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import read_golden, rel_l2


def _random_instance(rng, M_max=10):
    M = int(rng.integers(1, M_max + 1))
    s = int(rng.integers(0, M + 1))
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    return M, piv, J


# --------------------------------------------------------------------------
# Paper values
# --------------------------------------------------------------------------

def _parse_matrix_fixture():
    lines = read_golden("printed_matrix_sec7.txt")
    d = {"row": []}
    for ln in lines:
        key, *vals = ln.split()
        if key == "row":
            v = [float(x) for x in vals]
            d["row"].append([complex(v[2 * q], v[2 * q + 1]) for q in range(4)])
        else:
            d[key] = [int(x) for x in vals]
    return d


def test_printed_matrix_section7():
    d = _parse_matrix_fixture()
    M = d["M"][0]
    J = d["J"]
    piv = O.pivots_by_tree(J, M)
    assert piv == d["pivots"]
    I = O.sample_set(M, piv)
    assert [int(x) for x in I] == d["I"]
    Jc = O.canonical_support(J, piv)
    assert [int(x) for x in Jc] == d["cols"]
    got = O.Finv_sub(M, I, Jc) * 2.0 ** 8
    want = np.array(d["row"])
    assert np.max(np.abs(got - want)) < 1e-4


@pytest.mark.parametrize("line", read_golden("pivot_examples.txt"))
def test_pivot_examples(line):
    name, M, J, expect = [x.strip() for x in line.split("|")]
    M = int(M)
    J = [int(x) for x in J.split()]
    by_tree = O.pivots_by_tree(J, M)
    assert by_tree == O.pivots_by_pairs(J), name
    if expect == "NOT_HOMOGENEOUS":
        assert not O.is_homogeneous(J, M), name
    else:
        assert by_tree == [int(x) for x in expect.split()], name
        assert O.is_homogeneous(J, M), name


def test_spectral_example_section2():
    # Section II: rows {1, 292, 641, 932} give a unitary (up to scale) submatrix.
    M = 10
    J = np.array([316, 384, 828, 896], dtype=np.uint64)
    rows = np.array([1, 292, 641, 932], dtype=np.uint64)
    A = O.F_sub(M, rows, J)
    assert np.allclose(A.conj().T @ A, 4 * np.eye(4), atol=1e-12)
    # our own sample set for the same J is also a spectrum (Proposition 3)
    I = O.sample_set(M, O.pivots_by_tree(J, M))
    B = O.F_sub(M, J, I)
    assert np.allclose(B.conj().T @ B, 4 * np.eye(4), atol=1e-12)


def test_butterfly_example_section8_brute_force():
    M = 10
    J = [23, 187, 190, 247, 386, 731, 990, 994]
    piv = O.pivots_by_tree(J, M)
    assert piv == [0, 2, 5]
    rng = np.random.default_rng(7)
    Jc = O.canonical_support(J, piv)
    c = W.complex_gaussian(8, rng)
    I = O.sample_set(M, piv)
    f = O.brute_force_samples(M, Jc, c, I)
    _, got = O.transform(M, J, f, piv, Jc)
    assert rel_l2(got, c) < 1e-13


# --------------------------------------------------------------------------
# Brute force: library inverse FFT of the zero-filled spectrum
# --------------------------------------------------------------------------

def test_brute_force_n16_k4():
    rng = W.rng_for(1, 99)
    M, s = 4, 2
    for trial in range(20):
        piv = W.random_pivots(M, s, rng)
        J = W.homogeneous_support(M, piv, rng)
        Jc = O.canonical_support(J, piv)
        I = O.sample_set(M, piv)
        c = W.complex_gaussian(4, rng)
        f = O.brute_force_samples(M, Jc, c, I)
        assert rel_l2(O.transform(M, J, f, piv, Jc)[1], c) < 1e-14
        assert rel_l2(O.solve(M, Jc, I, f), c) < 1e-14
        assert rel_l2(O.adjoint_transform(M, Jc, I, f), c) < 1e-14


def test_brute_force_random_supports():
    rng = np.random.default_rng(2024)
    for trial in range(150):
        M, piv, J = _random_instance(rng)
        Jc = O.canonical_support(J, piv)
        I = O.sample_set(M, piv)
        c = W.complex_gaussian(J.size, rng)
        f = O.brute_force_samples(M, Jc, c, I)
        assert rel_l2(O.synthesize(M, Jc, c, I), f) < 1e-13
        assert rel_l2(O.synthesize_fast(M, piv, Jc, c), f) < 1e-13
        assert rel_l2(O.transform(M, J, f, piv, Jc)[1], c) < 1e-12
        assert rel_l2(O.solve(M, Jc, I, f), c) < 1e-12
        assert rel_l2(O.adjoint_transform(M, Jc, I, f), c) < 1e-12


def test_config1_single_instance_brute_force():
    inst = W.workload_single()
    piv = O.pivots_by_tree(inst.J, inst.M)
    assert piv == list(inst.pivots)
    Jc = O.canonical_support(inst.J, piv)
    # coefficients are drawn aligned with the user's order of J
    c_user = dict(zip([int(j) for j in inst.J], inst.coeffs))
    c = np.array([c_user[int(j)] for j in Jc])
    I = O.sample_set(inst.M, piv)
    f = O.brute_force_samples(inst.M, Jc, c, I)
    assert rel_l2(O.transform(inst.M, inst.J, f, piv, Jc)[1], c) < 1e-13


# --------------------------------------------------------------------------
# Special cases that reduce to a library FFT (Section VII examples 1-3)
# --------------------------------------------------------------------------

def test_full_support_is_the_dft():
    rng = np.random.default_rng(5)
    M = 7
    N = 1 << M
    J = np.arange(N, dtype=np.uint64)
    piv = list(range(M))
    x = W.complex_gaussian(N, rng)                  # any signal: supp(Fx) is in Z_N
    I = O.sample_set(M, piv)
    Jc, c = O.transform(M, J, x[I.astype(np.int64)], piv)
    ref = np.fft.fft(x)
    assert rel_l2(c, ref[Jc.astype(np.int64)]) < 1e-13


def test_elementary_set_uniform_downsampling():
    rng = np.random.default_rng(6)
    M, s = 9, 4
    N, k = 1 << M, 1 << s
    piv = list(range(s))
    J = W.homogeneous_support(M, piv, rng)
    I = O.sample_set(M, piv)
    assert sorted(int(i) for i in I) == [b * (N // k) for b in range(k)]
    Jc = O.canonical_support(J, piv)
    c = W.complex_gaussian(k, rng)
    f = O.synthesize(M, Jc, c, I)
    # uniform samples in natural order, then a k-point library FFT
    order = np.argsort(I.astype(np.int64))
    fdown = f[order]
    X = np.fft.fft(fdown) * (N / k)
    assert rel_l2(X[(Jc % np.uint64(k)).astype(np.int64)], c) < 1e-12


def test_bottom_pivots_take_first_samples():
    rng = np.random.default_rng(8)
    M, s = 10, 5
    piv = list(range(M - s, M))
    I = O.sample_set(M, piv)
    assert sorted(int(i) for i in I) == list(range(1 << s))
    J = W.homogeneous_support(M, piv, rng)
    Jc = O.canonical_support(J, piv)
    c = W.complex_gaussian(1 << s, rng)
    f = O.brute_force_samples(M, Jc, c, I)
    assert rel_l2(O.transform(M, J, f, piv, Jc)[1], c) < 1e-12


# --------------------------------------------------------------------------
# Invariants the paper proves
# --------------------------------------------------------------------------

def test_aliasing_lemma_and_product_formula():
    rng = np.random.default_rng(9)
    for trial in range(40):
        M, piv, J = _random_instance(rng)
        k = J.size
        m = rng.integers(0, 1 << M, size=16)
        assert np.allclose(O.aliasing_pattern_product(M, piv, m),
                           O.aliasing_pattern_direct(M, piv, m), atol=1e-9)
        Ji = J.astype(np.int64)
        diff = (Ji[:, None] - Ji[None, :]).ravel()
        h = O.aliasing_pattern_direct(M, piv, diff).reshape(k, k)
        assert np.allclose(h, k * np.eye(k), atol=1e-9)


def test_scaled_unitarity():
    rng = np.random.default_rng(10)
    for trial in range(40):
        M, piv, J = _random_instance(rng)
        k, N = J.size, 1 << M
        I = O.sample_set(M, piv)
        A = O.F_sub(M, J, I)
        assert np.allclose(A.conj().T @ A, k * np.eye(k), atol=1e-10)
        assert np.allclose(A @ O.Finv_sub(M, I, J), (k / N) * np.eye(k), atol=1e-12)


def test_block_structure_corollary():
    rng = np.random.default_rng(11)
    for trial in range(40):
        M, piv, J = _random_instance(rng)
        if J.size < 2:
            continue
        k = J.size
        Jc = O.canonical_support(J, piv)
        I = O.sample_set(M, piv)
        Ih = O.sample_set(M, piv[:-1])
        F1 = O.F_sub(M, Jc[: k // 2], Ih)
        a = 1 << (M - 1 - int(piv[-1]))
        d = np.exp(-2j * np.pi * ((a * Jc[: k // 2].astype(object)) % (1 << M)).astype(np.float64) / (1 << M))
        D = np.diag(d)
        Id = np.eye(k // 2)
        left = np.block([[Id, D], [Id, -D]])
        right = np.block([[F1, np.zeros_like(F1)], [np.zeros_like(F1), F1]])
        assert np.allclose(O.F_sub(M, Jc, I), left @ right, atol=1e-10)
        # eq. "Hi-DFT-dynamic-programming": both halves see the same height-1 values
        F2 = O.F_sub(M, Jc[k // 2:], Ih)
        assert np.allclose(F1, F2, atol=1e-10)


def test_opcount_theorem1():
    rng = np.random.default_rng(12)
    for s in range(0, 9):
        M = s + 3
        piv = W.random_pivots(M, s, rng)
        J = W.homogeneous_support(M, piv, rng)
        Jc = O.canonical_support(J, piv)
        cnt = {}
        O.hidft(np.ones(1 << s, dtype=np.complex128), piv, Jc, M, cnt)
        assert cnt.get("ops", 0) == O.theorem1_opcount(s)
        assert cnt.get("butterflies", 0) == s * (1 << s) // 2


def test_prop1_and_prop2_on_random_sets():
    rng = np.random.default_rng(13)
    for trial in range(200):
        M = int(rng.integers(2, 8))
        k = int(rng.integers(1, min(1 << M, 16) + 1))
        J = rng.choice(1 << M, size=k, replace=False)
        npiv = len(O.pivots_by_tree(J, M))
        assert npiv >= int(np.ceil(np.log2(k)))          # Proposition 1
        hom = O.is_homogeneous(J, M)
        # Proposition 2: (1) <=> (2) <=> (4)
        eq2 = O.splits_are_even_and_levelwise(J, M) and O.is_pow2(k)
        eq4 = O.is_pow2(k) and len(O.pivots_by_pairs(J)) == (k.bit_length() - 1)
        assert hom == eq2 == eq4
    for trial in range(50):
        M, piv, J = _random_instance(rng, 8)
        assert O.is_homogeneous(J, M) and O.splits_are_even_and_levelwise(J, M)


def test_sample_set_forms_and_its_own_homogeneity():
    rng = np.random.default_rng(14)
    for trial in range(50):
        M = int(rng.integers(1, 12))
        s = int(rng.integers(0, M + 1))
        piv = W.random_pivots(M, s, rng)
        I = O.sample_set(M, piv)
        assert np.array_equal(I, O.sample_set_closed_form(M, piv))
        assert len(set(int(i) for i in I)) == 1 << s
        if s:
            # I_r is (M-1-r)-homogeneous (Section VII)
            assert O.pivots_by_tree(I, M) == sorted(M - 1 - int(p) for p in piv)


def test_roundtrip_large_sparse_check():
    # N = 2^30, k = 2^12: fast synthesis checked by direct sums at sampled points,
    # then the transform inverts it.
    rng = np.random.default_rng(15)
    M, s = 30, 12
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    Jc = O.canonical_support(J, piv)
    I = O.sample_set(M, piv)
    c = W.complex_gaussian(1 << s, rng)
    f = O.synthesize_fast(M, piv, Jc, c)
    pick = rng.choice(1 << s, size=32, replace=False)
    direct = O.synthesize(M, Jc, c, I[pick])
    assert rel_l2(f[pick], direct) < 1e-12
    _, back = O.transform(M, J, f, piv, Jc)
    assert rel_l2(back, c) < 1e-12
    spot = O.coefficients_at(M, Jc[pick], I, f)
    assert rel_l2(spot, c[pick]) < 1e-12


# --------------------------------------------------------------------------
# Planted mistakes: the pins above must catch them
# --------------------------------------------------------------------------

def _brute_force_error(M, piv, J, rng):
    Jc = O.canonical_support(J, piv)
    I = O.sample_set(M, piv)
    c = W.complex_gaussian(J.size, rng)
    f = O.brute_force_samples(M, Jc, c, I)
    return rel_l2(O.transform(M, J, f, piv, Jc)[1], c)


def test_planted_twiddle_sign_is_caught(monkeypatch):
    import oracle.fp64 as H
    rng = np.random.default_rng(16)
    M, piv = 8, [1, 3, 6]
    J = W.homogeneous_support(M, piv, rng)
    good = _brute_force_error(M, piv, J, rng)
    real = H._omega
    monkeypatch.setattr(H, "_omega", lambda M_, a, Jh: np.conj(real(M_, a, Jh)))
    bad = _brute_force_error(M, piv, J, rng)
    assert good < 1e-12 and bad > 0.1


def test_planted_wrong_support_half_is_caught():
    # Algorithm 1 must take the twiddles from the first half of the canonical
    # support; taking them from the second half (or misordering J) must fail.
    rng = np.random.default_rng(17)
    M, piv = 8, [0, 4, 5]
    J = W.homogeneous_support(M, piv, rng)
    Jc = O.canonical_support(J, piv)
    I = O.sample_set(M, piv)
    c = W.complex_gaussian(J.size, rng)
    f = O.brute_force_samples(M, Jc, c, I)
    h = Jc.size // 2
    wrong = np.concatenate([Jc[h:], Jc[:h]])
    _, got = O.transform(M, J, f, piv, wrong)
    assert rel_l2(got, c) > 0.1


def test_planted_dropped_normalisation_is_caught():
    rng = np.random.default_rng(18)
    M, piv = 9, [2, 3, 7]
    J = W.homogeneous_support(M, piv, rng)
    Jc = O.canonical_support(J, piv)
    I = O.sample_set(M, piv)
    c = W.complex_gaussian(J.size, rng)
    f = O.brute_force_samples(M, Jc, c, I)
    y = O.hidft(f, piv, Jc, M)                      # height-0 Hi-DFT, no N/k
    assert rel_l2(y * (1 << M) / J.size, c) < 1e-12
    assert rel_l2(y * J.size, c) > 0.1              # the paper's "|J| (Ff)_J" as printed


def test_level_forms_match_recursions():
    rng = np.random.default_rng(19)
    for trial in range(60):
        M, piv, J = _random_instance(rng, 12)
        Jc = O.canonical_support(J, piv)
        assert np.array_equal(O.canonical_support_by_key(J, piv), Jc)
        I = O.sample_set(M, piv)
        C = W.complex_gaussian((3, J.size), rng)
        F = O.synthesize(M, Jc, C, I)
        assert rel_l2(O.synthesize_levels(M, piv, Jc, C), F) < 1e-13
        assert rel_l2(O.hidft_levels(F, piv, Jc, M), np.stack([O.hidft(f, piv, Jc, M) for f in F])) < 1e-13
        assert rel_l2(O.transform_levels(M, piv, Jc, F), C) < 1e-12
