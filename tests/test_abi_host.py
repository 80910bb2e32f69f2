"""CPU checks of the C ABI: the library loads, exports every declared symbol,
and its host planner agrees bit-for-bit with the oracle (no GPU needed)."""
import re

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import ROOT, read_golden


def _declared_symbols():
    with open(f"{ROOT}/include/sdft.h") as fh:
        text = fh.read()
    return sorted(set(re.findall(r"\b(sdft_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_2211_15299_gb300 import _native as N
    lib = ctypes.CDLL(N.LIB_PATH)
    declared = _declared_symbols()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(N.SIGNATURES), "binding and header disagree"


def test_status_strings():
    from paper_2211_15299_gb300 import _native as N
    for code in N.STATUS:
        assert N.sdft_status_string(code) != "unknown status"


@pytest.mark.parametrize("line", read_golden("pivot_examples.txt"))
def test_plan_validation_matches_paper_examples(line):
    from paper_2211_15299_gb300 import Plan, SdftError
    name, M, J, expect = [x.strip() for x in line.split("|")]
    M = int(M)
    J = [int(x) for x in J.split()]
    if expect == "NOT_HOMOGENEOUS":
        with pytest.raises(SdftError) as ei:
            Plan(M, J, host_only=True)
        assert ei.value.name in ("SDFT_ERR_NOT_HOMOGENEOUS", "SDFT_ERR_NOT_POW2"), name
    else:
        p = Plan(M, J, host_only=True)
        assert [int(x) for x in p.pivots] == [int(x) for x in expect.split()], name


def test_plan_errors():
    from paper_2211_15299_gb300 import Plan, SdftError
    cases = [
        (4, [0, 16], "SDFT_ERR_RANGE"),
        (4, [1, 2, 3], "SDFT_ERR_NOT_POW2"),
        (4, [3, 3, 5, 7], "SDFT_ERR_DUPLICATE"),
        (63, [0], "SDFT_ERR_RANGE"),
        (10, [1, 2, 4, 8], "SDFT_ERR_NOT_HOMOGENEOUS"),
        (2, [0, 1, 2, 3, 0, 1, 2, 3], "SDFT_ERR_DUPLICATE"),
    ]
    for M, J, want in cases:
        with pytest.raises(SdftError) as ei:
            Plan(M, J, host_only=True)
        assert ei.value.name == want, (M, J)
    with pytest.raises(SdftError):
        Plan(4, [], host_only=True)
    with pytest.raises(SdftError) as ei:              # double-float mode is for complex128 plans
        Plan(4, [0, 1, 2, 3], "c64", host_only=True, fp64_df=True)
    assert ei.value.name == "SDFT_ERR_ARG"
    assert Plan(4, [0, 1, 2, 3], "c128", host_only=True, fp64_df=True).k == 4


def test_homogeneity_decision_matches_oracle_on_near_misses():
    # The planner recognises homogeneous sets from the path of their first
    # element and sends everything else to its sorting check; sets one element
    # away from homogeneous (and the two hand-made ones below, whose first
    # element's path shows exactly s levels) must get the oracle's answer.
    from paper_2211_15299_gb300 import Plan, SdftError
    cases = [(3, [0, 1, 2, 5]), (3, [0, 1, 4, 7]), (4, [0, 1, 2, 11]), (3, [0, 1, 2, 7])]
    rng = W.rng_for(0, 4242)
    for _ in range(300):
        s = int(rng.integers(1, 7))
        M = s + int(rng.integers(0, 6))
        piv = W.random_pivots(M, s, rng)
        J = [int(x) for x in W.homogeneous_support(M, piv, rng)]
        if rng.random() < 0.8:                 # replace one element by another value in Z_N
            i = int(rng.integers(0, len(J)))
            J[i] = int(rng.integers(0, 1 << M))
        if rng.random() < 0.5:
            J = [J[i] for i in rng.permutation(len(J))]
        cases.append((M, J))
    for M, J in cases:
        Ja = np.asarray(J, dtype=np.uint64)
        if len(set(J)) < len(J):
            want = "SDFT_ERR_DUPLICATE"
        elif O.is_homogeneous(Ja, M):
            want = None
        else:
            want = "SDFT_ERR_NOT_HOMOGENEOUS"
        if want is None:
            p = Plan(M, J, host_only=True)
            assert [int(x) for x in p.pivots] == [int(x) for x in O.pivots_by_tree(Ja, M)], (M, J)
        else:
            with pytest.raises(SdftError) as ei:
                Plan(M, J, host_only=True)
            assert ei.value.name == want, (M, J)


def test_homogeneity_decision_exhaustive_small():
    # every 4-element subset of Z_16, each in three orders (which element comes
    # first decides the planner's fast path), and 3000 random 8-element subsets
    # of Z_32: the planner's verdict, pivots and canonical order are the oracle's
    from paper_2211_15299_gb300 import Plan, SdftError
    import itertools
    rng = np.random.default_rng(4343)
    cases = [(4, list(c)) for c in itertools.combinations(range(16), 4)]
    cases = [(M, order) for M, J in cases for order in (J, J[::-1], J[1:] + J[:1])]
    cases += [(5, [int(x) for x in rng.choice(32, size=8, replace=False)]) for _ in range(3000)]
    n_hom = 0
    for M, J in cases:
        Ja = np.asarray(J, dtype=np.uint64)
        if O.is_homogeneous(Ja, M):
            n_hom += 1
            p = Plan(M, J, host_only=True)
            piv = O.pivots_by_tree(Ja, M)
            assert [int(x) for x in p.pivots] == [int(x) for x in piv], (M, J)
            assert [int(x) for x in p.support_order] == [int(x) for x in O.canonical_support_by_key(Ja, piv)]
        else:
            with pytest.raises(SdftError) as ei:
                Plan(M, J, host_only=True)
            assert ei.value.name == "SDFT_ERR_NOT_HOMOGENEOUS", (M, J)
    assert n_hom > 1000


def test_host_only_plan_refuses_execution():
    from paper_2211_15299_gb300 import _native as N
    h = N.sdft_plan_create(4, [0, 1, 2, 3], N.SDFT_C64, N.SDFT_PLAN_HOST_ONLY)
    try:
        with pytest.raises(N.SdftError) as ei:
            N.sdft_execute(h, 16, 16, None)
        assert ei.value.name == "SDFT_ERR_NO_DEVICE"
        host = np.zeros(8, dtype=np.complex64)
        with pytest.raises(N.SdftError) as ei:
            N.sdft_execute_strided_host(h, 1, host.ctypes.data, host.ctypes.data, 16, 16, 0, None)
        assert ei.value.name == "SDFT_ERR_NO_DEVICE"
        with pytest.raises(N.SdftError) as ei:       # batched execution needs device plans
            N.sdft_execute_batched([h, h], 16, 16, 16, None)
        assert ei.value.name == "SDFT_ERR_NO_DEVICE"
        h2 = N.sdft_plan_create(4, [0, 1, 2, 3], N.SDFT_C128, N.SDFT_PLAN_HOST_ONLY)
        try:
            with pytest.raises(N.SdftError) as ei:   # one precision per call
                N.sdft_execute_batched([h, h2], 16, 16, 16, None)
            assert ei.value.name in ("SDFT_ERR_NO_DEVICE", "SDFT_ERR_PRECISION")
        finally:
            N.sdft_plan_destroy(h2)
        with pytest.raises(N.SdftError) as ei:       # host buffers neither identical nor disjoint
            N.sdft_execute_strided_host(h, 1, None, host.ctypes.data, 16, 16, 0, None)
        assert ei.value.name == "SDFT_ERR_ARG"
    finally:
        N.sdft_plan_destroy(h)


def test_host_tensors_are_refused_not_computed():
    # no host fallback: every execute entry point of the binding refuses tensors
    # in host memory before anything runs, and host-only objects refuse to run
    import torch
    from paper_2211_15299_gb300 import Plan, Sas, SdftError, execute_batched
    p = Plan(10, [0, 1, 2, 3], host_only=True)
    x = torch.zeros(4, dtype=torch.complex64)
    for call in (lambda: p.execute(x), lambda: p.execute_strided(x), lambda: p.synthesize(x),
                 lambda: p.to_user_order(x)):
        with pytest.raises(ValueError, match="CUDA device"):
            call()
    with pytest.raises(TypeError):
        p.execute_strided(x.numpy())
    with pytest.raises(TypeError, match="CUDA int64"):
        execute_batched([p], x, torch.tensor([0, 4]))
    sas = Sas(10, [0, 1, 2, 5, 7], host_only=True)
    with pytest.raises(ValueError, match="CUDA device"):
        sas.execute(torch.zeros(sas.n_samples, dtype=torch.complex64))
    h = torch.zeros(4, dtype=torch.complex64).pin_memory() if torch.cuda.is_available() else None
    if h is not None:
        with pytest.raises(SdftError):
            p.execute_host(h)


def test_plan_tables_match_oracle():
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(31)
    for trial in range(300):
        M = int(rng.integers(1, 41))
        s = int(rng.integers(0, min(M, 14) + 1))
        piv = W.random_pivots(M, s, rng)
        J = W.homogeneous_support(M, piv, rng)
        p = Plan(M, J, host_only=True)
        assert [int(x) for x in p.pivots] == [int(x) for x in piv]
        assert np.array_equal(p.sample_indices, O.sample_set(M, piv))
        if s <= 11:
            assert np.array_equal(p.support_order, O.canonical_support(J, piv))
        if s <= 9:
            # twiddles: the omega vectors Algorithm 1 uses at each recursion depth
            tw = p.twiddles()
            Jc = p.support_order
            for m in range(1, s + 1):
                a = 1 << (M - 1 - int(piv[m - 1]))
                w = O.F_sub(M, np.array([a], dtype=np.uint64), Jc[: 1 << (m - 1)])[0]
                got = tw[(1 << (m - 1)) - 1:(1 << m) - 1]
                assert np.max(np.abs(got - w)) < 1e-15


def test_plan_at_config_sizes_host_only():
    from paper_2211_15299_gb300 import Plan
    inst, _ = W.workload_large(M=30, s=20, batch=1, coeffs=False)
    p = Plan(inst.M, inst.J, host_only=True)
    assert [int(x) for x in p.pivots] == [int(x) for x in inst.pivots]
    I = p.sample_indices
    assert np.array_equal(I, O.sample_set_closed_form(inst.M, inst.pivots)) if inst.s <= 12 else True
    # the pivot-bit key of every canonical element spells its position
    Jc = p.support_order
    t = np.arange(Jc.size, dtype=np.uint64)
    key = np.zeros_like(Jc)
    for q, r in enumerate(inst.pivots):
        key |= ((Jc >> np.uint64(r)) & np.uint64(1)) << np.uint64(q)
    assert np.array_equal(key, t)
    assert np.array_equal(np.sort(Jc), np.sort(inst.J))
