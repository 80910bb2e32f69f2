"""CPU checks of the Shift-and-Sample planner (host-only plans) against the
oracle: pivots, classes, sample sets, output order, the choice of R."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _sas(M, J, R=0):
    from paper_2211_15299_gb300 import Sas
    return Sas(M, J, "c64", R=R, host_only=True)


def _sets(rng, n):
    out = [(10, [0, 512, 1, 6, 7]), (10, [0, 256, 1, 6, 7])]
    for _ in range(n):
        M = int(rng.integers(4, 13))
        k = int(rng.integers(1, min(200, 1 << M) + 1))
        out.append((M, sorted(int(x) for x in rng.choice(1 << M, size=k, replace=False))))
    return out


@pytest.mark.parametrize("seed", range(4))
def test_planner_matches_oracle(seed):
    rng = np.random.default_rng(40 + seed)
    for M, J in _sets(rng, 25):
        levels = O.split_levels(J, M)
        for R in sorted({1, len(levels) // 2, len(levels)} & set(range(1, len(levels) + 1))):
            r = O.sas_pivots(J, M, R)
            mu = O.sas_mu(J, r)
            if max(mu.values()) > 64:              # beyond the decoder's class size
                from paper_2211_15299_gb300 import SdftError
                with pytest.raises(SdftError) as ei:
                    _sas(M, J, R)
                assert ei.value.name == "SDFT_ERR_UNSUPPORTED"
                continue
            p = _sas(M, J, R)
            assert list(p.pivots) == r
            assert p.mu_star == max(mu.values()) and p.occupied == len(mu)
            assert np.array_equal(p.sample_indices, O.sas_sample_sets(M, r, p.mu_star))
            want = sorted(J, key=lambda j: (O.node_key(j, r), j))
            assert [int(x) for x in p.support_order] == want
            assert p.max_cond >= 1.0 - 1e-12
            if p.mu_star == 1:
                assert abs(p.max_cond - 1.0) < 1e-12


def test_automatic_R_minimises_the_lemma_cost():
    # the cheapest R (Lemma "computation_shift_sample") among those whose
    # class systems are well conditioned (1-norm condition <= 32 for complex64)
    rng = np.random.default_rng(9)
    for M, J in _sets(rng, 30):
        levels = O.split_levels(J, M)
        if not levels:
            continue
        p = _sas(M, J, 0)
        lk = int(np.ceil(np.log2(len(J)))) if len(J) > 1 else 0
        cands = [c for c in range(max(0, lk - 4), min(len(levels), lk + 2, 24) + 1)
                 if max(O.sas_mu(J, levels[:c]).values()) <= 64]
        cond = {c: (_sas(M, J, c).max_cond if c else 1.0) for c in cands}
        ok = [c for c in cands if cond[c] <= 32.0]
        if ok:
            cost = {c: O.sas_cost(c, O.sas_mu(J, levels[:c])) for c in ok}
            best = min(cost.values())
            assert p.R == min(c for c in ok if cost[c] == best), (M, len(J))
        else:
            assert p.R == min(cands, key=lambda c: (cond[c], c))


def test_homogeneous_set_gives_one_shift():
    rng = np.random.default_rng(4)
    M, s = 16, 9
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    p = _sas(M, J, s)
    assert p.mu_star == 1 and p.occupied == 1 << s and list(p.pivots) == [int(x) for x in piv]


def test_sas_errors():
    from paper_2211_15299_gb300 import SdftError
    with pytest.raises(SdftError) as ei:
        _sas(4, [1, 2, 2])
    assert ei.value.name == "SDFT_ERR_DUPLICATE"
    with pytest.raises(SdftError) as ei:
        _sas(4, [1, 16])
    assert ei.value.name == "SDFT_ERR_RANGE"
    with pytest.raises(SdftError) as ei:
        _sas(6, [0, 1, 2, 3], R=5)               # only 2 split levels
    assert ei.value.name == "SDFT_ERR_ARG"


def test_random_subset_at_the_theorems_pivot_count():
    # Theorem "hom_rand_subset": with n = floor(log2 k - log2 log2 k) pivots of the
    # homogeneous set K, the planner takes K's first n pivots and the classes
    # stay below Lemma "bound_mu_r_star"'s bound. The class systems there are
    # ill-conditioned (exact arithmetic is assumed by the theorem), so numeric
    # parity runs on the planner's own R (tests/test_gpu_sas.py).
    log2k = 10
    rng = W.rng_for(0, 4321)
    J, piv = W.bernoulli_subset_of_homogeneous(18, log2k + 3, 1 << log2k, rng)
    n = int(np.floor(log2k - np.log2(log2k)))
    for prec in ("c64", "c128"):
        from paper_2211_15299_gb300 import Sas
        p = Sas(18, [int(j) for j in J], prec, R=n, host_only=True)
        assert [int(x) for x in p.pivots] == [int(x) for x in piv[:n]]
        r = O.sas_pivots([int(j) for j in J], 18, n)
        assert p.mu_star == max(O.sas_mu([int(j) for j in J], r).values())
        assert p.mu_star < (4 + 3 * np.log(2)) * log2k
        auto = Sas(18, [int(j) for j in J], prec, host_only=True)
        assert auto.max_cond <= (32.0 if prec == "c64" else 100.0)


@pytest.mark.parametrize("kind,k,prec", [("ap", 3000, "c64"), ("ap", 1000, "c64"), ("subset", 3000, "c64"),
                                         ("uoh", 2000, "c64"), ("subset", 3000, "c128"), ("ap", 3000, "c128"),
                                         ("subset", 600, "c64")])
def test_execution_path_follows_the_tile_shapes(kind, k, prec):
    """sdft_sas_path: one launch and no workspace under complete isolation with
    one to four virtual instances per tile (R in [TB - 2, TB], k <= 2^TB); two
    launches with only the k gathered values per instance in the workspace for
    mu* > 1 on those shapes (k <= 8192); the whole mu* x 2^R stage-1 output
    otherwise and always under SDFT_SAS_TWO_STAGE."""
    from paper_2211_15299_gb300 import Sas
    J = [int(j) for j in W.workload_sas(kind, k=k)]
    p = Sas(20, J, prec, host_only=True)
    two = Sas(20, J, prec, host_only=True, two_stage=True)
    tb = 12 if prec == "c64" else 11
    tile = tb - 2 <= p.R <= tb
    whole = p.mu_star << p.R
    if tile and p.mu_star == 1 and p.k <= (1 << tb):
        want = (1, 0)
    elif tile and 1 < p.mu_star <= 64 and p.k <= 8192:
        want = (2, p.k)
    else:
        want = (2, whole)
    assert (p.launches, p.work_values) == want, (p.R, p.mu_star, p.k)
    assert (two.launches, two.work_values) == (2, whole)
