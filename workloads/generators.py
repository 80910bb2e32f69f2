"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module draws supports, pivot sets and coefficient vectors. It performs none
of the transform's arithmetic: it never forms a sample set, a twiddle, a DFT
entry or a sample value. Both the CPU oracle and the GPU path receive what is
drawn here as plain integer / complex arrays.

Support construction follows the tree characterisation of homogeneous sets
(Section VI, Proposition "hom-tree-prop", item 2): walk the complete binary
tree T_N from the root (level 0) downwards; at a pivot level every node keeps
both children (bit l = 0 and bit l = 1); at any other level every node keeps
exactly one child, whose bit l is drawn at random.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 20221115


def rng_for(config: int, salt: int = 0) -> np.random.Generator:
    """PCG64 generator for a numbered workload (seed = 20221115 + config)."""
    return np.random.Generator(np.random.PCG64([BASE_SEED + config, salt]))


def random_pivots(M: int, s: int, rng: np.random.Generator) -> np.ndarray:
    """s distinct levels drawn uniformly from {0..M-1}, ascending."""
    if not 0 <= s <= M:
        raise ValueError("need 0 <= s <= M")
    return np.sort(rng.choice(M, size=s, replace=False)).astype(np.int64)


def contiguous_pivots(M: int, s: int, rng: np.random.Generator) -> np.ndarray:
    """A block of s consecutive levels o..o+s-1 with o uniform on {0..M-s}."""
    o = int(rng.integers(0, M - s + 1))
    return np.arange(o, o + s, dtype=np.int64)


def homogeneous_support(M: int, pivots: Sequence[int], rng: np.random.Generator,
                        shuffle: bool = True) -> np.ndarray:
    """Draw a support in Z_{2^M} whose split levels are exactly `pivots`.

    Returns k = 2^len(pivots) distinct uint64 values (in random order when
    `shuffle`, to exercise the planner's sorting).
    """
    piv = set(int(p) for p in pivots)
    if any(p < 0 or p >= M for p in piv) or len(piv) != len(pivots):
        raise ValueError("pivots must be distinct levels in [0, M)")
    nodes = np.zeros(1, dtype=np.uint64)            # residues mod 2^l
    for level in range(M):
        bit = np.uint64(1) << np.uint64(level)
        if level in piv:
            nodes = np.concatenate([nodes, nodes | bit])
        else:
            pick = rng.integers(0, 2, size=nodes.size, dtype=np.uint64).astype(bool)
            nodes = np.where(pick, nodes | bit, nodes)
    if shuffle:
        nodes = nodes[rng.permutation(nodes.size)]
    return nodes.astype(np.uint64)


def complex_gaussian(shape, rng: np.random.Generator) -> np.ndarray:
    """i.i.d. CN(0,1): real and imaginary parts N(0, 1/2), E|z|^2 = 1."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return ((re + 1j * im) * np.sqrt(0.5)).astype(np.complex128)


def log_uniform_coeffs(shape, rng: np.random.Generator, lo: float = 1e-3,
                       hi: float = 1e3) -> np.ndarray:
    """Uniform phase, magnitude 10^U(log10 lo, log10 hi)."""
    z = complex_gaussian(shape, rng)
    mag = 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size=shape)
    return (z / np.abs(z) * mag).astype(np.complex128)


def log_uniform_exponent(lo: int, hi: int, rng: np.random.Generator) -> int:
    """Integer exponent uniform on {lo..hi} ("log-uniform" sizes 2^lo..2^hi)."""
    return int(rng.integers(lo, hi + 1))


@dataclasses.dataclass
class Instance:
    M: int
    pivots: np.ndarray          # ascending levels
    J: np.ndarray               # uint64 support, user order
    coeffs: Optional[np.ndarray] = None   # complex128, aligned with J (user order)

    @property
    def s(self) -> int:
        return int(len(self.pivots))

    @property
    def k(self) -> int:
        return 1 << self.s

    @property
    def N(self) -> int:
        return 1 << self.M


# ---------------------------------------------------------------------------
# The five workloads (seed 20221115 + number). Sizes are parameters so tests can
# draw reduced versions with the same recipe.
# ---------------------------------------------------------------------------

def workload_single(M: int = 10, s: int = 5, config: int = 1, salt: int = 0) -> Instance:
    """One instance: s of M levels are pivots, CN(0,1) coefficients."""
    rng = rng_for(config, salt)
    piv = random_pivots(M, s, rng)
    J = homogeneous_support(M, piv, rng)
    return Instance(M, piv, J, complex_gaussian(J.size, rng))


def workload_shared(M: int = 20, s: int = 12, batch: int = 4096, config: int = 2,
                    salt: int = 0, coeffs: bool = True):
    """One shared support, `batch` coefficient vectors with log-uniform
    magnitudes over 1e-3..1e3. Returns (Instance without coeffs, coeffs[batch, k])."""
    rng = rng_for(config, salt)
    piv = random_pivots(M, s, rng)
    J = homogeneous_support(M, piv, rng)
    C = log_uniform_coeffs((batch, J.size), rng) if coeffs else None
    return Instance(M, piv, J), C


def workload_large(M: int = 30, s: int = 20, batch: int = 64, contiguous: bool = True,
                   config: int = 3, salt: int = 0, coeffs: bool = True):
    """One shared large support; pivots either one contiguous block or spread.
    Returns (Instance, coeffs[batch, k] CN(0,1) or None)."""
    rng = rng_for(config, salt + (0 if contiguous else 1))
    piv = contiguous_pivots(M, s, rng) if contiguous else random_pivots(M, s, rng)
    J = homogeneous_support(M, piv, rng)
    C = complex_gaussian((batch, J.size), rng) if coeffs else None
    return Instance(M, piv, J), C


def workload_uneven(count: int = 10000, M_range=(12, 24), s_range=(4, 16), config: int = 4,
                    salt: int = 0, coeffs: bool = False) -> List[Instance]:
    """`count` instances, each with its own support; M and s integer-uniform on
    the ranges, s redrawn until s <= M."""
    rng = rng_for(config, salt)
    out = []
    for _ in range(count):
        M = log_uniform_exponent(*M_range, rng)
        s = log_uniform_exponent(*s_range, rng)
        while s > M:
            s = log_uniform_exponent(*s_range, rng)
        piv = random_pivots(M, s, rng)
        J = homogeneous_support(M, piv, rng)
        c = complex_gaussian(J.size, rng) if coeffs else None
        out.append(Instance(M, piv, J, c))
    return out


@dataclasses.dataclass
class ServingTrace:
    arrivals: np.ndarray        # seconds, ascending
    plan_ids: np.ndarray        # index into `plans` (resident pool) or >= len(pool) for new
    plans: List[Instance]       # resident pool followed by the fresh supports


def workload_serving(rate: float = 20000.0, duration: float = 10.0, pool: int = 256,
                     reuse: float = 0.8, M_range=(10, 26), s_range=(4, 18), config: int = 5,
                     salt: int = 0) -> ServingTrace:
    """Poisson arrivals; each request either reuses one of `pool` resident supports
    (probability `reuse`) or brings a fresh one."""
    rng = rng_for(config, salt)

    def draw():
        M = log_uniform_exponent(*M_range, rng)
        s = log_uniform_exponent(*s_range, rng)
        while s > M:
            s = log_uniform_exponent(*s_range, rng)
        piv = random_pivots(M, s, rng)
        return Instance(M, piv, homogeneous_support(M, piv, rng))

    n = int(rng.poisson(rate * duration))
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps)
    plans = [draw() for _ in range(pool)]
    ids = np.empty(n, dtype=np.int64)
    for r in range(n):
        if rng.random() < reuse:
            ids[r] = int(rng.integers(0, pool))
        else:
            plans.append(draw())
            ids[r] = len(plans) - 1
    return ServingTrace(arrivals, ids, plans)


# ---------------------------------------------------------------------------
# Supports that are not homogeneous (Shift-and-Sample)
# ---------------------------------------------------------------------------


def arithmetic_progression(M: int, k: int, d: int, rng: np.random.Generator) -> np.ndarray:
    """{a + n d mod N : 0 <= n < k} with a uniform start a (Corollary "AP")."""
    N = 1 << M
    a = int(rng.integers(0, N))
    J = (a + np.arange(k, dtype=np.uint64) * np.uint64(d)) % np.uint64(N)
    if np.unique(J).size != k:
        raise ValueError("progression wraps onto itself")
    return J


def random_subset_of_homogeneous(M: int, s_h: int, k: int, rng: np.random.Generator) -> np.ndarray:
    """k elements drawn without replacement from a homogeneous set with s_h
    random pivots (the random-subset family, Theorem "hom_rand_subset")."""
    piv = random_pivots(M, s_h, rng)
    H = homogeneous_support(M, piv, rng)
    return np.sort(rng.choice(H, size=k, replace=False)).astype(np.uint64)


def bernoulli_subset_of_homogeneous(M: int, s_h: int, k: int, rng: np.random.Generator):
    """Every element of a homogeneous set K (s_h random pivots) kept
    independently with probability k / |K| (the model of Theorem
    "hom_rand_subset"); returns (J sorted, K's pivots)."""
    piv = random_pivots(M, s_h, rng)
    K = homogeneous_support(M, piv, rng)
    keep = rng.random(K.size) < (k / K.size)
    return np.sort(K[keep]).astype(np.uint64), piv


def workload_sas(kind: str = "subset", M: int = 20, k: int = 3000, batch: int = 1024, config: int = 6,
                 salt: int = 0) -> np.ndarray:
    """Supports for the Shift-and-Sample path: an arithmetic progression with
    odd difference ("ap"), a Bernoulli subset of expected size k of a
    homogeneous set with ceil(log2 k) + 2 pivots ("subset"), or a union of
    homogeneous sets ("uoh", Theorem "UoE2")."""
    rng = rng_for(config, salt)
    if kind == "ap":
        return arithmetic_progression(M, k, 2 * int(rng.integers(0, 1 << (M - 2))) + 1, rng)
    if kind == "uoh":       # two parts of every size 2^0 .. 2^a inside a homogeneous K, a = log2 k - 2
        a = int(np.floor(np.log2(k))) - 2
        l = random_pivots(M, a + 4, rng)
        return union_of_homogeneous(M, l, [2] * (a + 1), rng, rng)[0]
    s_h = int(np.ceil(np.log2(k))) + 2
    return bernoulli_subset_of_homogeneous(M, s_h, k, rng)[0]


def union_of_homogeneous(M: int, l: Sequence[int], etas: Sequence[int], K_rng: np.random.Generator,
                         rng: np.random.Generator):
    """A union as in Theorem "UoE2": K homogeneous with pivots l (drawn with
    K_rng), and for each i, etas[i] sets J_ij of 2^i elements of K that are
    homogeneous with the first i pivots of l (their bits at the other pivots
    fixed at random). l = 0..M-1 (K = Z_N) gives a union of elementary sets
    (Lemma "UoE1"). Returns (J sorted and deduplicated, the parts)."""
    K = homogeneous_support(M, l, K_rng)
    l = [int(x) for x in l]
    bits = np.stack([(K >> np.uint64(p)) & np.uint64(1) for p in l], axis=1)   # K's pivot bits
    parts = []
    for i, eta in enumerate(etas):
        for _ in range(int(eta)):
            fixed = rng.integers(0, 2, size=len(l) - i)
            sel = np.all(bits[:, i:] == fixed[None, :].astype(np.uint64), axis=1)
            parts.append(np.sort(K[sel]))
    J = np.unique(np.concatenate(parts)).astype(np.uint64)
    return J, parts
