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

from .fp64 import hidft, pivots_by_tree, sample_set, transform_levels


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


def sas_node_values(M: int, J: Sequence[int], r: Sequence[int], F_shift,
                    counter: Dict[str, int] = None) -> np.ndarray:
    """Step 1: (mu*, 2^R) values; row a is the Hi-DFT (with the N/2^R scale) of
    the samples at I_r + a over the virtual support, in key order.

    `counter` (optional): each row then runs the recursive Algorithm 1 (`hidft`)
    and the counter accumulates "transforms" (one per shift) and
    "transform_ops", 3 operations per butterfly (one complex product and two
    complex sums, the accounting of Theorem "computation_Hi-DFT"'s proof, which
    gives c1 n 2^n with c1 = 3/2 for a transform of 2^n values)."""
    V = virtual_support(J, M, r)
    F_shift = np.asarray(F_shift, dtype=np.complex128)
    if counter is None:
        return np.stack([transform_levels(M, r, V, F_shift[a]) for a in range(F_shift.shape[0])])
    scale = float(2.0 ** (M - len(r)))
    rows = []
    for a in range(F_shift.shape[0]):
        local: Dict[str, int] = {}
        rows.append(scale * hidft(F_shift[a], r, V, M, local))
        counter["transforms"] = counter.get("transforms", 0) + 1
        counter["transform_ops"] = counter.get("transform_ops", 0) + 3 * local.get("butterflies", 0)
    return np.stack(rows)


def vandermonde_solve(z, y, counter: Dict[str, int] = None) -> np.ndarray:
    """x with sum_u x_u z_u^a = y_a for a = 0 .. mu - 1 (the class system of eq.
    "alg1_system", A[a, u] = z_u^a), in O(mu^2) operations by the elimination of
    Bjorck and Pereyra (Math. Comp. 24, 1970) for this "primal" system: first
    mu - 1 sweeps y_i <- y_i - z_k y_{i-1} (i from the bottom up to k + 1), then,
    for k from mu - 2 down to 0, y_i <- y_i / (z_i - z_{i-k-1}) for i > k and
    y_i <- y_i - y_{i+1} for k <= i < mu - 1. Exact in exact arithmetic for
    distinct z (the paper cites fast Vandermonde solvers for its c2 mu^2 term).

    `counter` (optional) accumulates "solve_ops": one per complex product,
    quotient, sum or difference, 5 mu (mu - 1) / 2 in all (5 for a 2 x 2
    system, 0 for a class of one)."""
    z = np.asarray(z, dtype=np.complex128)
    x = np.array(y, dtype=np.complex128)
    n = z.size
    ops = 0
    for k in range(n - 1):
        for i in range(n - 1, k, -1):
            x[i] = x[i] - z[k] * x[i - 1]
            ops += 2
    for k in range(n - 2, -1, -1):
        for i in range(k + 1, n):
            x[i] = x[i] / (z[i] - z[i - k - 1])
            ops += 2
        for i in range(k, n - 1):
            x[i] = x[i] - x[i + 1]
            ops += 1
    if counter is not None:
        counter["solve_ops"] = counter.get("solve_ops", 0) + ops
    return x


def sas_transform(M: int, J: Sequence[int], r: Sequence[int], F_shift,
                  counter: Dict[str, int] = None) -> np.ndarray:
    """Steps 1-2: the coefficients c_j for j in J, in the order J is given.
    F_shift[a] holds f at I_r + a (sample order), a = 0 .. mu* - 1.

    Without `counter` each class system is solved by LU with partial pivoting
    (a library solve). With `counter` the run is instrumented: step 1 counts as
    in `sas_node_values`, each class is solved by `vandermonde_solve` (counting
    "solve_ops"), and "solve_mu2" accumulates mu(v)^2 over the classes solved,
    so the count can be set beside Lemma "computation_shift_sample"."""
    Y = sas_node_values(M, J, r, F_shift, counter)
    coeff = {}
    for t, members in sas_nodes(J, r).items():
        mu = len(members)
        if mu > Y.shape[0]:
            raise ValueError("fewer shifts than the largest class")
        if counter is None:
            A = _z_powers(M, members, mu)
            x = np.linalg.solve(A, Y[:mu, t])
        else:
            x = vandermonde_solve(_z_powers(M, members, 2)[1], Y[:mu, t], counter)
            counter["solve_mu2"] = counter.get("solve_mu2", 0) + mu * mu
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
    c1 R 2^R mu* + c2 sum_v mu(v)^2 with c1 = 3/2, c2 = 6. The first term is the
    count an instrumented `sas_transform` makes of its mu* transforms; the
    second bounds the count of its O(mu^2) class solves (`vandermonde_solve`)."""
    mu_star = max(mu.values()) if mu else 0
    return 1.5 * R * (1 << R) * mu_star + 6.0 * sum(m * m for m in mu.values())
