"""Plain FP64 CPU oracle for Shift-and-Sample (SAS), Algorithm "shift-sample".

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this module:
only the tests, the smoke check and the bench's CPU legs may call it. It shares
no code with the CUDA path.

SAS computes (Ff)_J for supports J that are r-part-homogeneous (Definition
"part-H-tree"): the congruence tree T(J) has no splits below level r_max other
than at the levels of r. The steps, in the order of Algorithm "shift-sample":

  0. the truncated tree at level rho = r_max + 1: the classes v of J modulo
     2^rho ("nodes at level rho"), mu(v) members each, mu* = max mu(v);
  1. for a = 0 .. mu* - 1, the Hi-DFT (Algorithm 1, height 0) of the shifted
     signal, sampled at I_r + a;
  2. at every node v, the mu(v) x mu(v) Vandermonde system of eq. "alg1_system"
     in the unknown coefficients of v's members.

Readings taken here (each pinned by a test in tests/test_oracle_sas.py):
  * Pivots: the first R split levels of T(J). Every set is part-homogeneous
    for such an r (no other split lies below r_max), and each level of r is a
    pivot. R is a parameter (the library chooses it; tests pass the same R).
  * Shift: the a-th sample set is I_r + a (mod N), i.e. samples f(i + a). With
    f = F^{-1} c this gives, at node v, (N / 2^R) F(v, I_r) f_(I_r + a)
    = sum_{j in v} c_j z_j^a with z_j = exp(+2 pi i j / N) (Lemma
    "shift-mod-Hi-DFT" with the 1/N restored, eq. "alg1_system").
  * Algorithm 1 needs a homogeneous support of exactly 2^R elements. Occupied
    classes contribute their residue mod 2^rho; an empty class gets a residue
    that keeps the set homogeneous with pivots r (see `virtual_support`); the
    values computed there are 0 and unused.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

from .fp64 import pivots_by_tree, sample_set, transform_levels


def split_levels(J: Sequence[int], M: int) -> List[int]:
    """Every level at which T(J) splits (Definition 8 applied to any set)."""
    return pivots_by_tree(J, M)


def sas_pivots(J: Sequence[int], M: int, R: int) -> List[int]:
    """The first R split levels of T(J)."""
    levels = split_levels(J, M)
    if R > len(levels):
        raise ValueError("fewer split levels than R")
    return levels[:R]


def node_key(j: int, r: Sequence[int]) -> int:
    """Index of j's class at level r_max + 1 in canonical order: bit q of the
    key is bit r_q of j (the class is fixed by these bits when J is
    r-part-homogeneous)."""
    return sum(((int(j) >> p) & 1) << q for q, p in enumerate(r))


def sas_nodes(J: Sequence[int], r: Sequence[int]) -> Dict[int, List[int]]:
    """key -> sorted members of J in that class."""
    nodes: Dict[int, List[int]] = {}
    for j in J:
        nodes.setdefault(node_key(j, r), []).append(int(j))
    return {t: sorted(m) for t, m in nodes.items()}


def virtual_support(J: Sequence[int], M: int, r: Sequence[int]) -> np.ndarray:
    """2^R residues, entry t for the class with key t, forming a set that is
    homogeneous with pivots r. Occupied class: its members' residue mod 2^rho.
    Empty class t: take the longest key prefix of t that some member of J has
    (length q0); copy that member's bits below r_{q0}, then set bit r_q to
    bit q of t for q >= q0 and leave the other bits 0."""
    R = len(r)
    rho = (r[-1] + 1) if R else 0
    nodes = sas_nodes(J, r)
    keys = {t: m[0] for t, m in nodes.items()}
    out = np.zeros(1 << R, dtype=np.uint64)
    for t in range(1 << R):
        if t in keys:
            out[t] = keys[t] % (1 << rho)
            continue
        q0, member = 0, None
        for q in range(R, -1, -1):          # longest prefix first
            mask = (1 << q) - 1
            hits = [j for tt, j in keys.items() if (tt & mask) == (t & mask)]
            if hits:
                q0, member = q, hits[0]
                break
        v = member % (1 << r[q0])
        for q in range(q0, R):
            v |= ((t >> q) & 1) << r[q]
        out[t] = v
    return out


def sas_sample_sets(M: int, r: Sequence[int], mu_star: int) -> np.ndarray:
    """(mu*, 2^R) sample indices: row a is I_r + a mod N in sample order."""
    N = 1 << M
    I = np.asarray(sample_set(M, r), dtype=np.uint64)
    return np.stack([(I + np.uint64(a)) % np.uint64(N) for a in range(mu_star)])


def sas_mu(J: Sequence[int], r: Sequence[int]) -> Dict[int, int]:
    return {t: len(m) for t, m in sas_nodes(J, r).items()}


def _z_powers(M: int, members: Sequence[int], mu: int) -> np.ndarray:
    """A[a, u] = exp(+2 pi i a l_u / N), the exponent reduced mod N exactly."""
    N = 1 << M
    a = np.arange(mu, dtype=object)[:, None]
    l = np.asarray([int(x) for x in members], dtype=object)[None, :]
    p = np.asarray((a * l) % N, dtype=np.float64)
    return np.exp(2j * np.pi * p / N)


def sas_node_values(M: int, J: Sequence[int], r: Sequence[int], F_shift) -> np.ndarray:
    """Step 1: (mu*, 2^R) values; row a is the Hi-DFT (with the N/2^R scale) of
    the samples at I_r + a over the virtual support, in key order."""
    V = virtual_support(J, M, r)
    F_shift = np.asarray(F_shift, dtype=np.complex128)
    return np.stack([transform_levels(M, r, V, F_shift[a]) for a in range(F_shift.shape[0])])


def sas_transform(M: int, J: Sequence[int], r: Sequence[int], F_shift) -> np.ndarray:
    """Steps 1-2: the coefficients c_j for j in J, in the order J is given.
    F_shift[a] holds f at I_r + a (sample order), a = 0 .. mu* - 1."""
    Y = sas_node_values(M, J, r, F_shift)
    coeff = {}
    for t, members in sas_nodes(J, r).items():
        mu = len(members)
        if mu > Y.shape[0]:
            raise ValueError("fewer shifts than the largest class")
        A = _z_powers(M, members, mu)
        x = np.linalg.solve(A, Y[:mu, t])
        for l, v in zip(members, x):
            coeff[l] = v
    return np.asarray([coeff[int(j)] for j in J], dtype=np.complex128)


def sas_samples_direct(M: int, J: Sequence[int], c, idx) -> np.ndarray:
    """f(n) = (1/N) sum_j c_j exp(+2 pi i j n / N) at the indices idx (any
    shape), by the direct sum with exact reduction of j n mod N."""
    N = 1 << M
    J = [int(j) for j in J]
    c = np.asarray(c, dtype=np.complex128)
    flat = np.asarray(idx, dtype=np.uint64).reshape(-1)
    out = np.zeros(flat.size, dtype=np.complex128)
    for j, cj in zip(J, c):
        p = np.asarray([(j * int(n)) % N for n in flat], dtype=np.float64)
        out += cj * np.exp(2j * np.pi * p / N)
    return (out / N).reshape(np.shape(idx))


def sas_cost(R: int, mu: Dict[int, int]) -> float:
    """Operation count of steps 1-2 by Lemma "computation_shift_sample":
    c1 R 2^R mu* + c2 sum_v mu(v)^2 with c1 = 3/2, c2 = 6."""
    mu_star = max(mu.values()) if mu else 0
    return 1.5 * R * (1 << R) * mu_star + 6.0 * sum(m * m for m in mu.values())
