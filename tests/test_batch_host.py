"""CPU checks of the uneven-batch planner (host-only plans; no GPU)."""
import numpy as np
import pytest

import workloads as W


def _plans(instances, prec="c64"):
    from paper_2211_15299_gb300 import Plan
    return [Plan(i.M, i.J, prec, host_only=True) for i in instances]


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_packing_and_item_invariants(prec):
    from paper_2211_15299_gb300 import Batch
    insts = W.workload_uneven(count=400, salt=3)
    plans = _plans(insts, prec)
    b = Batch(plans)
    ks = np.array([p.k for p in plans])
    assert b.total == int(ks.sum())
    # every instance starts at a multiple of its own k, and the ranges tile [0, total)
    assert all(int(o) % int(k) == 0 for o, k in zip(b.offsets, ks))
    spans = sorted((int(o), int(o) + int(k)) for o, k in zip(b.offsets, ks))
    assert spans[0][0] == 0 and spans[-1][1] == b.total
    assert all(a[1] == c[0] for a, c in zip(spans, spans[1:]))
    n_items, n_ctr, grid = b.stats()          # raises if the dependency invariants fail
    multi = sum(1 for p in plans if p.s > (12 if prec == "c64" else 11))
    assert n_ctr >= multi and grid == 304 and n_items > 0


def test_large_instances_three_levels():
    from paper_2211_15299_gb300 import Batch
    rng = W.rng_for(4, 77)
    insts = []
    for s in (22, 21, 20, 14, 13, 5, 4, 0):
        M = s + 4
        piv = W.random_pivots(M, s, rng)
        insts.append(W.Instance(M, piv, W.homogeneous_support(M, piv, rng)))
    b = Batch(_plans(insts))
    n_items, n_ctr, grid = b.stats()
    # s = 21, 22 have three levels (two counters each), s = 20, 14, 13 two levels
    assert n_ctr == 2 + 2 + 1 + 1 + 1


def test_host_only_batch_cannot_execute():
    from paper_2211_15299_gb300 import Batch, SdftError, _native as N
    b = Batch(_plans(W.workload_uneven(count=5, salt=9)))
    with pytest.raises(SdftError) as ei:
        N.sdft_batch_execute(b.handle, 16, 16, None)
    assert ei.value.name == "SDFT_ERR_NO_DEVICE"


@pytest.mark.parametrize("schedule", ["lanes", "round_robin"])
def test_schedule_invariants_full_uneven_workload(schedule):
    # 10,000 instances, far more units than CTAs
    from paper_2211_15299_gb300 import Batch
    insts = W.workload_uneven(count=10000)
    plans = _plans(insts)
    b = Batch(plans)
    b.set_schedule(schedule)
    n_items, n_ctr, grid = b.stats()        # raises if a dependency is closer than 4 x grid
    multi = sum(1 for p in plans if p.s > 12)
    assert n_ctr == multi
    assert n_items >= sum(max(1, p.k >> 12) for p in plans if p.s > 12)


@pytest.mark.parametrize("schedule", ["lanes", "round_robin", "auto"])
@pytest.mark.parametrize("grid", [0, 152, 7])
def test_schedules_keep_invariants(schedule, grid):
    # every queue shape the autotuner may pick satisfies the ordering invariants
    from paper_2211_15299_gb300 import Batch
    insts = W.workload_uneven(count=600, salt=11)
    b = Batch(_plans(insts))
    _, n_ctr0, _ = b.stats()
    b.set_schedule(schedule, grid)
    n_items, n_ctr, g = b.stats()             # raises if a dependency is closer than 4 x grid
    assert n_ctr == n_ctr0
    assert g == (grid if grid else 304)
    multi_items = sum(max(1, p.k >> 12) for p in b.plans if p.s > 12)
    assert n_items >= 2 * multi_items


def test_unknown_schedule_rejected():
    from paper_2211_15299_gb300 import Batch, SdftError, _native as N
    b = Batch(_plans(W.workload_uneven(count=5, salt=9)))
    with pytest.raises(SdftError) as ei:
        N.sdft_batch_set_schedule(b.handle, 7, 0)
    assert ei.value.name == "SDFT_ERR_ARG"


@pytest.mark.parametrize("schedule", ["lanes", "round_robin"])
def test_dependency_distance(schedule):
    # a later level follows its producers by lag x grid list places (default 6,
    # at least 4): every choice keeps the ordering invariants, and a longer lag
    # only adds places (padding) to the list
    from paper_2211_15299_gb300 import Batch, SdftError, _native as N
    b = Batch(_plans(W.workload_uneven(count=600, salt=13)))
    assert N.sdft_batch_get_lag(b.handle) == 6
    b.set_schedule(schedule)
    counts = []
    for lag in (4, 6, 8, 12):
        N.sdft_batch_set_lag(b.handle, lag)
        assert N.sdft_batch_get_lag(b.handle) == lag
        n_items, n_ctr, grid = b.stats()       # raises if a dependency is closer than 4 x grid
        counts.append(n_items)
    assert counts == sorted(counts)
    for bad in (0, 3, 65):
        with pytest.raises(SdftError) as ei:
            N.sdft_batch_set_lag(b.handle, bad)
        assert ei.value.name == "SDFT_ERR_ARG"
    assert N.sdft_batch_get_lag(b.handle) == 12
