"""The seeded input recipes: the synthetic workloads follow their stated
distributions and structure, are reproducible from their seeds, and produce
supports that the oracle finds homogeneous with the recorded pivots
(Definition 9, Proposition "hom-tree-prop")."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def test_seeds_reproduce():
    a, b = W.workload_single(), W.workload_single()
    assert a.M == 10 and a.s == 5
    assert np.array_equal(a.J, b.J) and np.array_equal(a.coeffs, b.coeffs)
    c = W.workload_single(salt=1)
    assert not np.array_equal(a.J, c.J)


@pytest.mark.parametrize("M,s", [(4, 2), (10, 5), (12, 0), (12, 12), (16, 7)])
def test_homogeneous_support_has_the_drawn_pivots(M, s):
    rng = np.random.default_rng(1000 + 17 * M + s)
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    assert J.size == 1 << s and np.unique(J).size == J.size
    assert int(J.max()) < 1 << M
    assert O.pivots_by_tree(J, M) == [int(p) for p in piv]
    assert O.is_homogeneous(J, M) and O.splits_are_even_and_levelwise(J, M)


def test_pivot_recipes():
    rng = np.random.default_rng(5)
    offsets = set()
    for _ in range(200):
        p = W.contiguous_pivots(30, 20, rng)
        assert np.array_equal(p, np.arange(p[0], p[0] + 20))
        assert 0 <= p[0] <= 10
        offsets.add(int(p[0]))
        q = W.random_pivots(30, 20, rng)
        assert q.size == 20 and np.unique(q).size == 20 and np.all(np.diff(q) > 0)
        assert 0 <= q[0] and q[-1] < 30
    assert offsets == set(range(11))            # every offset 0..M-s is drawn
    with pytest.raises(ValueError):
        W.random_pivots(4, 5, rng)


def test_coefficient_distributions():
    rng = np.random.default_rng(6)
    z = W.complex_gaussian(200000, rng)
    assert abs(np.var(z.real) - 0.5) < 0.01 and abs(np.var(z.imag) - 0.5) < 0.01
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.01
    inst, C = W.workload_shared(M=12, s=6, batch=3000)
    mag = np.abs(C)
    assert C.shape == (3000, 64)
    assert mag.min() >= 1e-3 * (1 - 1e-12) and mag.max() <= 1e3 * (1 + 1e-12)
    lg = np.log10(mag).ravel()                     # uniform on [-3, 3]
    assert abs(lg.mean()) < 0.03 and abs(lg.var() - 3.0) < 0.05
    ph = C / mag                                   # uniform phase
    assert abs(ph.mean()) < 0.01
    assert O.is_homogeneous(inst.J, inst.M)


def test_uneven_recipe():
    insts = W.workload_uneven(count=400)
    Ms = np.array([i.M for i in insts])
    ss = np.array([i.s for i in insts])
    assert Ms.min() >= 12 and Ms.max() <= 24 and ss.min() >= 4 and ss.max() <= 16
    assert np.all(ss <= Ms)
    assert set(Ms.tolist()) == set(range(12, 25)) and set(ss.tolist()) == set(range(4, 17))
    for i in insts:
        assert i.J.size == i.k and int(i.J.max()) < 1 << i.M
        if i.s <= 8:
            assert O.pivots_by_tree(i.J, i.M) == [int(p) for p in i.pivots]
    # the first instances do not depend on how many are drawn
    few = W.workload_uneven(count=3)
    for a, b in zip(few, insts):
        assert a.M == b.M and np.array_equal(a.J, b.J)


def test_serving_recipe():
    tr = W.workload_serving(duration=0.05, pool=16)
    n = tr.arrivals.size
    assert abs(n - 1000) < 130                         # Poisson(rate x duration)
    assert np.all(np.diff(tr.arrivals) > 0)
    assert abs(np.mean(np.diff(tr.arrivals)) - 5e-5) < 0.15 * 5e-5
    fresh = tr.plan_ids >= 16
    assert abs(fresh.mean() - 0.2) < 0.05              # 80 % reuse a resident support
    assert len(tr.plans) == 16 + int(fresh.sum())
    assert np.all(tr.plan_ids[~fresh] < 16)
    assert len(set(tr.plan_ids[fresh].tolist())) == int(fresh.sum())   # every fresh support used once
    for p in tr.plans:
        assert 10 <= p.M <= 26 and 4 <= p.s <= 18 and p.s <= p.M and p.J.size == p.k


def test_sas_supports():
    ap = W.workload_sas("ap", M=16, k=300)
    assert ap.size == 300 and np.unique(ap).size == 300
    # a progression with odd difference: consecutive terms differ by d mod N
    N = 1 << 16
    diffs = {(int(ap[i + 1]) - int(ap[i])) % N for i in range(ap.size - 1)}
    assert len(diffs) == 1 and next(iter(diffs)) % 2 == 1
    sub = W.workload_sas("subset", M=16, k=300)
    assert 200 < sub.size < 400 and np.unique(sub).size == sub.size
    assert len(O.pivots_by_tree(sub, 16)) <= int(np.ceil(np.log2(300))) + 2   # inside a homogeneous set of 2^11
    uoh = W.workload_sas("uoh", M=16, k=300)
    assert np.unique(uoh).size == uoh.size and uoh.size > 0


def test_union_of_homogeneous_parts():
    # Theorem "UoE2": part J_ij has 2^i elements of K, homogeneous with the
    # first i pivots of K
    rng = np.random.default_rng(9)
    l = W.random_pivots(14, 8, rng)
    J, parts = W.union_of_homogeneous(14, l, [2, 1, 3, 0, 1], np.random.default_rng(10), rng)
    K = W.homogeneous_support(14, l, np.random.default_rng(10))    # the same K, redrawn
    assert O.pivots_by_tree(K, 14) == [int(x) for x in l]
    assert len(parts) == 7
    sizes = [p.size for p in parts]
    assert sizes == [1, 1, 2, 4, 4, 4, 16]
    for p in parts:
        i = int(np.log2(p.size))
        assert O.pivots_by_tree(p, 14) == [int(x) for x in l[:i]]
    assert np.array_equal(J, np.unique(np.concatenate(parts)))
    assert np.all(np.isin(J, K))
