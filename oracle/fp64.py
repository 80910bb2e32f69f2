"""Plain FP64 CPU oracle for the generalized radix-2 transform (Hi-DFT).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this module:
only the tests, the smoke check and the bench's CPU-baseline leg may call it.
It shares no code with the CUDA path; both receive inputs from `workloads`.

Notation follows arxiv 2211.15299 ("Fast DFT Computation for Signals with
Structured Support"): N = 2^M, F(m, n) = exp(-2 pi i m n / N) (Section II),
F^{-1}(m, n) = exp(+2 pi i m n / N) / N (Section IV, item 1); J is the frequency
support, k = |J| = 2^s, r = (r_1 < ... < r_s) the pivots, I_r the pivoted
sampling pattern (Section VII, Definition "r_sampling_pattern").

Every function is written for clarity, not speed: dense matrices, explicit
recursion, Python loops where sets are small. Products i*j are reduced modulo
N exactly in integer arithmetic before any exponential is taken.

Readings of the paper that this file takes (each is pinned by a test):
  * Normalisation: F(J, I_r) F^{-1}(I_r, J) = (k/N) Id, so the coefficients are
    (N/k) times the height-0 Hi-DFT (the paper drops F^{-1}'s 1/N around
    eq. "hom-implies-spectral").
  * Twiddle sign: exp(-2 pi i a j / N), as in Lemma "rec-hom-tree-split" and the
    definition of omega_M; Algorithm 1 prints the opposite sign.
  * Algorithm 1's second half is f_I(n/2 : n-1) (printed with an off-by-one).
  * Canonical order: samples in the order the recursive definition of I_r
    lists them; coefficients with the bit r_max = 0 half first and the other
    half paired element-by-element (same residue mod 2^{r_max}), recursively
    (Corollary "block-structure"). This is the order of the paper's printed
    4x4 example in Section VII.
  * Lemma "rec-hom-tree-split" carries no factor 2 and the right descendant
    uses -omega^{j_1}; the lemma's own proof gives these.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

# ---------------------------------------------------------------------------
# Integer helpers
# ---------------------------------------------------------------------------


def ctz(x: int) -> int:
    """Largest e with 2^e | x (x != 0): the 2-adic valuation."""
    x = int(x)
    if x == 0:
        raise ValueError("ctz(0) undefined")
    return (x & -x).bit_length() - 1


def is_pow2(k: int) -> bool:
    return k > 0 and (k & (k - 1)) == 0


def log2_exact(k: int) -> int:
    if not is_pow2(k):
        raise ValueError("not a power of two")
    return k.bit_length() - 1


# ---------------------------------------------------------------------------
# Congruence trees, pivots, homogeneity (Section VI)
# ---------------------------------------------------------------------------


def congruence_tree(J: Sequence[int], M: int) -> List[Dict[int, List[int]]]:
    """T(J): level l holds the nonempty classes of J modulo 2^l (Section VI).

    Returns a list of M+1 dicts, level -> {residue mod 2^l: sorted members}.
    """
    J = [int(j) for j in J]
    levels = []
    for level in range(M + 1):
        mod = 1 << level
        nodes: Dict[int, List[int]] = {}
        for j in J:
            nodes.setdefault(j % mod, []).append(j)
        levels.append({v: sorted(m) for v, m in nodes.items()})
    return levels


def pivots_by_tree(J: Sequence[int], M: int) -> List[int]:
    """Definition 8: level l is a pivot when some node at level l has two
    children, i.e. its members disagree on bit l."""
    tree = congruence_tree(J, M)
    out = []
    for level in range(M):
        for members in tree[level].values():
            if len({(j >> level) & 1 for j in members}) == 2:
                out.append(level)
                break
    return out


def pivots_by_pairs(J: Sequence[int]) -> List[int]:
    """Remark "pivot-as-gcd": e is a pivot iff 2^e exactly divides j_a - j_b for
    some pair j_a != j_b (all pairs; quadratic)."""
    J = [int(j) for j in J]
    piv = set()
    for a in range(len(J)):
        for b in range(a + 1, len(J)):
            piv.add(ctz(J[a] - J[b]))
    return sorted(piv)


def is_homogeneous(J: Sequence[int], M: int) -> bool:
    """Definition 9: T(J) has exactly log|J| pivots (|J| a power of two and the
    elements distinct in Z_N)."""
    J = [int(j) for j in J]
    if not is_pow2(len(J)) or len(set(J)) != len(J):
        return False
    if any(j < 0 or j >= (1 << M) for j in J):
        return False
    return len(pivots_by_tree(J, M)) == log2_exact(len(J))


def splits_are_even_and_levelwise(J: Sequence[int], M: int) -> bool:
    """Proposition "hom-tree-prop" item 2: at every split the two children have
    equal weight, and if one node of a level splits then all nodes of it do."""
    tree = congruence_tree(J, M)
    for level in range(M):
        split_flags = []
        for members in tree[level].values():
            ones = sum((j >> level) & 1 for j in members)
            zeros = len(members) - ones
            split = ones > 0 and zeros > 0
            if split and ones != zeros:
                return False
            split_flags.append(split)
        if any(split_flags) and not all(split_flags):
            return False
    return True


# ---------------------------------------------------------------------------
# Pivoted sampling pattern (Section VII, Definition "r_sampling_pattern")
# ---------------------------------------------------------------------------


def sample_set(M: int, r: Sequence[int]) -> np.ndarray:
    """I_r by its recursive definition, in the order the recursion lists it:
    I_() = {0}; I_r = I_{r^-} followed by I_{r^-} + 2^{M-1-r_max}."""
    r = [int(x) for x in r]
    if not r:
        return np.zeros(1, dtype=np.uint64)
    prev = sample_set(M, r[:-1])
    shift = np.uint64(1) << np.uint64(M - 1 - r[-1])
    return np.concatenate([prev, prev + shift]).astype(np.uint64)


def sample_set_closed_form(M: int, r: Sequence[int]) -> np.ndarray:
    """I_r = { sum_k b_k 2^{M-1-r_k} : b in {0,1}^s } (the non-recursive form),
    listed with b_1 as the least significant selector bit."""
    r = [int(x) for x in r]
    out = []
    for t in range(1 << len(r)):
        out.append(sum(((t >> (q)) & 1) << (M - 1 - r[q]) for q in range(len(r))))
    return np.array(out, dtype=np.uint64)


# ---------------------------------------------------------------------------
# Canonical order of the support (Corollary "block-structure")
# ---------------------------------------------------------------------------


def canonical_support(J: Sequence[int], r: Sequence[int]) -> np.ndarray:
    """Order J so that F(J, I_r) has the block form of Corollary
    "block-structure": split on the deepest pivot r_max; the half with bit
    r_max = 0 (J_1) comes first, ordered recursively for r^-; the other half
    follows, element u paired with J_1[u] (same residue mod 2^{r_max})."""
    J = [int(j) for j in J]
    r = [int(x) for x in r]
    if len(J) == 1:
        return np.array(J, dtype=np.uint64)
    rmax = r[-1]
    J1 = [j for j in J if not (j >> rmax) & 1]
    J2 = [j for j in J if (j >> rmax) & 1]
    if len(J1) != len(J2):
        raise ValueError("support is not homogeneous for these pivots")
    J1c = [int(x) for x in canonical_support(J1, r[:-1])]
    by_residue = {j % (1 << rmax): j for j in J2}
    J2c = [by_residue[j % (1 << rmax)] for j in J1c]
    return np.array(J1c + J2c, dtype=np.uint64)


# ---------------------------------------------------------------------------
# DFT submatrices (Sections II, IV, V)
# ---------------------------------------------------------------------------


def _phase(M: int, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """(rows x cols) mod N as float fraction of a turn: exact integer reduction
    (uint64 wraps mod 2^64, and 2^M divides 2^64), then one division."""
    rows = np.asarray(rows, dtype=np.uint64).reshape(-1, 1)
    cols = np.asarray(cols, dtype=np.uint64).reshape(1, -1)
    mask = np.uint64((1 << M) - 1) if M < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        p = (rows * cols) & mask
    return p.astype(np.float64) / float(1 << M)


def F_sub(M: int, rows, cols) -> np.ndarray:
    """F(rows, cols) with entries exp(-2 pi i m n / N)."""
    return np.exp(-2j * np.pi * _phase(M, rows, cols))


def Finv_sub(M: int, rows, cols) -> np.ndarray:
    """F^{-1}(rows, cols) with entries exp(+2 pi i m n / N) / N."""
    return np.exp(2j * np.pi * _phase(M, rows, cols)) / float(1 << M)


def synthesize(M: int, J, c, I) -> np.ndarray:
    """Samples of f in B^J at I: f_I = F^{-1}(I, J) (Ff)_J (eq.
    "submatrix-method"). `c` is (k,) or (B, k); returns the same leading shape."""
    A = Finv_sub(M, I, J)
    c = np.asarray(c, dtype=np.complex128)
    return (A @ c.T).T if c.ndim == 2 else A @ c


def solve(M: int, J, I, f) -> np.ndarray:
    """The plain definition: solve F^{-1}(I, J) c = f_I for c by LU (eq.
    "submatrix-method"). `f` is (k,) or (B, k); one factorisation serves all."""
    A = Finv_sub(M, I, J)
    f = np.asarray(f, dtype=np.complex128)
    if f.ndim == 2:
        return np.linalg.solve(A, f.T).T
    return np.linalg.solve(A, f)


def adjoint_transform(M: int, J, I, f) -> np.ndarray:
    """Closed form for a homogeneous J: c = (N/k) F(J, I_r) f_I, because
    F(J, I_r) F^{-1}(I_r, J) = (k/N) Id (eq. "hom-implies-spectral" with the
    1/N of F^{-1} kept). O(k) per coefficient."""
    J = np.asarray(J, dtype=np.uint64)
    k = J.size
    A = F_sub(M, J, I)
    f = np.asarray(f, dtype=np.complex128)
    scale = float(1 << M) / k
    return scale * ((A @ f.T).T if f.ndim == 2 else A @ f)


def coefficients_at(M: int, J_sel, I, f) -> np.ndarray:
    """Closed form evaluated one coefficient at a time for selected support
    elements (used for spot checks at sizes where a dense k x k is too big)."""
    I = np.asarray(I, dtype=np.uint64)
    f = np.asarray(f, dtype=np.complex128)
    out = np.empty(len(J_sel), dtype=np.complex128)
    k = I.size
    for q, j in enumerate(J_sel):
        row = F_sub(M, np.array([j], dtype=np.uint64), I)[0]
        out[q] = row @ f
    return out * (float(1 << M) / k)


# ---------------------------------------------------------------------------
# Algorithm 1 (Section VIII), with the readings listed in the module docstring
# ---------------------------------------------------------------------------


def _omega(M: int, a: int, J_half: np.ndarray) -> np.ndarray:
    """exp(-2 pi i a J / N) for the first half of the canonical support."""
    return F_sub(M, np.array([a], dtype=np.uint64), J_half)[0]


def hidft(f_I, r: Sequence[int], Jc, M: int, counter: Dict[str, int] = None) -> np.ndarray:
    """Height-0 Hi-DFT F(J, I_r) f_I by the recursion of Lemma
    "rec-hom-tree-split" / Algorithm 1. `f_I` in the order of `sample_set`,
    `Jc` in the order of `canonical_support`; output in the order of `Jc`.
    `counter` (optional) accumulates butterflies and arithmetic operations."""
    f_I = np.asarray(f_I, dtype=np.complex128)
    Jc = np.asarray(Jc, dtype=np.uint64)
    n = f_I.shape[-1]
    if n == 1:
        if counter is not None:                    # T(s) = 1 in Theorem 1's proof
            counter["ops"] = counter.get("ops", 0) + 1
        return f_I.copy()
    half = n // 2
    r = [int(x) for x in r]
    f1 = hidft(f_I[..., :half], r[:-1], Jc[:half], M, counter)
    f2 = hidft(f_I[..., half:], r[:-1], Jc[:half], M, counter)
    a = 1 << (M - 1 - r[-1])                       # a = N / 2^{r_max + 1}
    w = _omega(M, a, Jc[:half])
    t = w * f2
    if counter is not None:
        counter["butterflies"] = counter.get("butterflies", 0) + half
        # Proof of Theorem 1: combining two halves of n/2 values costs
        # 3 x n/2 operations (T(n) = 2 T(n+1) + 3 * 2^{s-n-1}).
        counter["ops"] = counter.get("ops", 0) + 3 * half
    return np.concatenate([f1 + t, f1 - t], axis=-1)


def transform(M: int, J, f_I, r: Sequence[int] = None, Jc=None) -> Tuple[np.ndarray, np.ndarray]:
    """Coefficients (Ff)_J by Algorithm 1: returns (Jc, c) with c aligned to the
    canonical support Jc; c = (N/k) x height-0 Hi-DFT."""
    J = np.asarray(J, dtype=np.uint64)
    if r is None:
        r = pivots_by_tree(J, M)
    if Jc is None:
        Jc = canonical_support(J, r)
    k = J.size
    y = hidft(f_I, r, Jc, M)
    return Jc, y * (float(1 << M) / k)


def hidft_adjoint(y, r: Sequence[int], Jc, M: int) -> np.ndarray:
    """F(J, I_r)^H y by transposing the block factorisation of Corollary
    "block-structure": F(J, I_r)^H = diag(F_1^H, F_1^H) [[I, I], [D^*, -D^*]]."""
    y = np.asarray(y, dtype=np.complex128)
    Jc = np.asarray(Jc, dtype=np.uint64)
    n = y.shape[-1]
    if n == 1:
        return y.copy()
    half = n // 2
    r = [int(x) for x in r]
    a = 1 << (M - 1 - r[-1])
    w = _omega(M, a, Jc[:half])
    y1, y2 = y[..., :half], y[..., half:]
    z1 = y1 + y2
    z2 = np.conj(w) * (y1 - y2)
    return np.concatenate([hidft_adjoint(z1, r[:-1], Jc[:half], M),
                           hidft_adjoint(z2, r[:-1], Jc[:half], M)], axis=-1)


def synthesize_fast(M: int, r: Sequence[int], Jc, c) -> np.ndarray:
    """f_I = F^{-1}(I_r, J) c = (1/N) F(J, I_r)^H c in O(k log k): the inverse of
    `transform`, for sizes where a dense k x k is infeasible. `c` aligned with
    Jc; result in the order of `sample_set`."""
    return hidft_adjoint(c, r, Jc, M) / float(1 << M)


# ---------------------------------------------------------------------------
# Independent checks (used to pin the functions above)
# ---------------------------------------------------------------------------


def brute_force_samples(M: int, J, c, I) -> np.ndarray:
    """Zero-fill the spectrum outside J, inverse-DFT the full N-point vector with
    a library FFT, and read the samples at I (small N only)."""
    N = 1 << M
    X = np.zeros(N, dtype=np.complex128)
    X[np.asarray(J, dtype=np.int64)] = c
    f = np.fft.ifft(X)          # includes the 1/N of F^{-1}
    return f[np.asarray(I, dtype=np.int64)]


def aliasing_pattern_product(M: int, r: Sequence[int], m) -> np.ndarray:
    """h_r(m) = prod_i (1 + exp(-2 pi i m / 2^{r_i + 1}))  (eq.
    "pivoted-aliasing-pattern")."""
    m = np.asarray(m, dtype=np.float64)
    h = np.ones(m.shape, dtype=np.complex128)
    for ri in r:
        h = h * (1.0 + np.exp(-2j * np.pi * m / float(1 << (int(ri) + 1))))
    return h


def aliasing_pattern_direct(M: int, r: Sequence[int], m) -> np.ndarray:
    """h_r = F 1_{I_r} evaluated at m (direct sum over the sample set)."""
    I = sample_set(M, r)
    m = np.asarray(m, dtype=np.int64) % (1 << M)
    return F_sub(M, m.astype(np.uint64), I).sum(axis=1)


def theorem1_opcount(s: int) -> int:
    """T(0) = 1.5 A log A + A with A = 2^s (Theorem "computation_Hi-DFT")."""
    A = 1 << s
    return int(1.5 * A * s + A)


# ---------------------------------------------------------------------------
# Level-by-level forms for large k (same arithmetic as the recursions above,
# vectorised over a batch; pinned against them in the tests)
# ---------------------------------------------------------------------------


def canonical_support_by_key(J, r: Sequence[int]) -> np.ndarray:
    """The canonical order of `canonical_support`, computed directly: element j
    goes to position sum_q bit_{r_q}(j) 2^{q-1} (its pivot bits read as a
    binary number, r_1 least significant). Raises if two elements collide."""
    J = np.asarray(J, dtype=np.uint64)
    key = np.zeros(J.size, dtype=np.int64)
    for q, rq in enumerate(r):
        key |= (((J >> np.uint64(int(rq))) & np.uint64(1)).astype(np.int64)) << q
    out = np.zeros(J.size, dtype=np.uint64)
    if np.unique(key).size != J.size:
        raise ValueError("support is not homogeneous for these pivots")
    out[key] = J
    return out


def _omegas(M: int, r: Sequence[int], Jc: np.ndarray) -> List[np.ndarray]:
    """omega vector of each recursion depth m = 1..s: exp(-2 pi i a_m J(0:2^{m-1}-1)/N),
    a_m = 2^{M-1-r_m}."""
    return [_omega(M, 1 << (M - 1 - int(r[m - 1])), Jc[: 1 << (m - 1)]) for m in range(1, len(r) + 1)]


def hidft_levels(f_I, r: Sequence[int], Jc, M: int) -> np.ndarray:
    """F(J, I_r) f_I with Algorithm 1's recursion unrolled bottom-up: at depth m
    every block of 2^m samples is [f1 + w f2, f1 - w f2] of its two halves.
    `f_I` is (k,) or (B, k)."""
    x = np.array(f_I, dtype=np.complex128, copy=True)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[None, :]
    B, k = x.shape
    Jc = np.asarray(Jc, dtype=np.uint64)
    for m, w in enumerate(_omegas(M, r, Jc), start=1):
        half = 1 << (m - 1)
        x = x.reshape(B, k // (2 * half), 2, half)
        t = x[:, :, 1, :] * w
        a = x[:, :, 0, :]
        x = np.stack([a + t, a - t], axis=2).reshape(B, k)
    return x[0] if squeeze else x


def transform_levels(M: int, r: Sequence[int], Jc, f_I) -> np.ndarray:
    """c = (N/k) F(J, I_r) f_I aligned with Jc, via `hidft_levels`."""
    Jc = np.asarray(Jc, dtype=np.uint64)
    return hidft_levels(f_I, r, Jc, M) * (float(1 << M) / Jc.size)


def synthesize_levels(M: int, r: Sequence[int], Jc, c) -> np.ndarray:
    """f_I = (1/N) F(J, I_r)^H c with `hidft_adjoint` unrolled top-down.
    `c` is (k,) or (B, k) aligned with Jc; result in sample order."""
    y = np.array(c, dtype=np.complex128, copy=True)
    squeeze = y.ndim == 1
    if squeeze:
        y = y[None, :]
    B, k = y.shape
    Jc = np.asarray(Jc, dtype=np.uint64)
    ws = _omegas(M, r, Jc)
    nblk = 1
    for m in range(len(r), 0, -1):
        half = 1 << (m - 1)
        y = y.reshape(B, nblk, 2, half)
        a, b = y[:, :, 0, :], y[:, :, 1, :]
        y = np.stack([a + b, np.conj(ws[m - 1]) * (a - b)], axis=2).reshape(B, 2 * nblk, half)
        nblk *= 2
    y = y.reshape(B, k) / float(1 << M)
    return y[0] if squeeze else y
