"""GPU checks of the tunable tile parameters: three or four butterfly stages per
pass give the same bits for strided plans (both strategies) and uneven batches,
and the autotuners store the choice they keep in the tuning cache, which a
fresh plan or batch of the same key then applies without timing."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import rel_l2

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("M,s,batch", [(10, 5, 37), (14, 8, 33), (16, 11, 9), (20, 12, 13), (22, 13, 5),
                                       (24, 16, 3), (24, 20, 2)])
def test_stages_per_pass_bit_identical(M, s, batch):
    torch = _torch()
    from paper_2211_15299_gb300 import Plan, _native as N
    rng = np.random.default_rng(9100 + s)
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    plan = Plan(M, J, 0)
    x = torch.randn((batch, plan.k), dtype=torch.complex64, device="cuda")
    outs = {}
    strategies = ("levels", "queue") if s > 12 else ("levels",)
    for strat in strategies:
        plan.set_strategy(strat)
        for spp in (4, 3):
            N.sdft_plan_set_stages_per_pass(plan.handle, spp)
            outs[(strat, spp)] = plan.execute_strided(x)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    ref = outs[("levels", 4)]
    for key, y in outs.items():
        assert torch.equal(y, ref), key
    Jc = O.canonical_support_by_key(J, piv)
    want = O.transform_levels(M, piv, Jc, x[:2].cpu().numpy().astype(np.complex128))
    assert rel_l2(ref[:2].cpu().numpy(), want) < 1e-5


def test_batch_queue_variants_bit_identical():
    # three or four stages per pass x tables in registers / staged whole in
    # shared memory: four kernels, one result; also every dependency distance
    torch = _torch()
    from paper_2211_15299_gb300 import Batch, Plan, _native as N
    insts = W.workload_uneven(count=300, salt=11)
    b = Batch([Plan(i.M, i.J, 0) for i in insts])
    x = torch.randn(b.total, dtype=torch.complex64, device="cuda")
    outs = {}
    for spp in (4, 3):
        for staged in (False, True):
            N.sdft_batch_set_stages_per_pass(b.handle, spp)
            N.sdft_batch_set_table_staging(b.handle, staged)
            assert N.sdft_batch_get_stages_per_pass(b.handle) == spp
            assert N.sdft_batch_get_table_staging(b.handle) == staged
            outs[(spp, staged)] = b.execute(x)
    # the dependency distance reorders the items and changes no bits either
    N.sdft_batch_set_stages_per_pass(b.handle, 4)
    N.sdft_batch_set_table_staging(b.handle, False)
    for lag in (4, 8, 12):
        N.sdft_batch_set_lag(b.handle, lag)
        outs[("lag", lag)] = b.execute(x)
    torch.cuda.synchronize()
    assert b.device_status() == 0
    for key, y in outs.items():
        assert torch.equal(y, outs[(4, False)]), key
    # and against the oracle for a few instances
    xs, ys = x.cpu().numpy(), outs[(4, True)].cpu().numpy()
    for i in (0, 1, len(insts) // 2, len(insts) - 1):
        inst = insts[i]
        o, kk = int(b.offsets[i]), 1 << int(inst.s)
        Jc = O.canonical_support_by_key(inst.J, inst.pivots)
        ref = O.transform_levels(inst.M, inst.pivots, Jc, xs[o:o + kk][None].astype(np.complex128))[0]
        assert rel_l2(ys[o:o + kk], ref) < 1e-5, i


def test_autotuners_store_and_apply(tmp_path):
    torch = _torch()
    from paper_2211_15299_gb300 import Batch, Plan, _native as N
    N.sdft_autotune_cache_clear()
    rng = np.random.default_rng(9200)
    M, s, batch = 24, 14, 64
    piv = W.random_pivots(M, s, rng)
    plan = Plan(M, W.homogeneous_support(M, piv, rng), 0)
    x = torch.randn((batch, plan.k), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    chosen, ms_lv, ms_q = N.sdft_plan_autotune(plan.handle, batch, x, y, None, 3)
    spp = N.sdft_plan_get_stages_per_pass(plan.handle)
    assert spp in (3, 4) and ms_lv > 0 and ms_q > 0
    assert N.sdft_autotune_cache_size() == 1
    # a fresh plan of the same key (other pivots) takes the stored choice
    piv2 = W.random_pivots(M, s, rng)
    fresh = Plan(M, W.homogeneous_support(M, piv2, rng), 0)
    assert N.sdft_plan_apply_tuning(fresh.handle, batch + 17)
    assert N.sdft_plan_get_stages_per_pass(fresh.handle) == spp
    ref = fresh.execute_strided(x)
    N.sdft_plan_set_strategy(fresh.handle, N.SDFT_STRATEGY_LEVELS)
    N.sdft_plan_set_stages_per_pass(fresh.handle, 4)
    assert torch.equal(fresh.execute_strided(x), ref)       # the choice changes no bits
    insts = W.workload_uneven(count=120, salt=12)
    b = Batch([Plan(i.M, i.J, 0) for i in insts])
    xb = torch.randn(b.total, dtype=torch.complex64, device="cuda")
    yb = torch.empty_like(xb)
    N.sdft_batch_autotune(b.handle, xb, yb, None, 2)
    assert N.sdft_autotune_cache_size() == 2
    f = tmp_path / "tune.json"
    N.sdft_autotune_cache_save(str(f))
    N.sdft_autotune_cache_clear()
    N.sdft_autotune_cache_load(str(f))
    b2 = Batch([Plan(i.M, i.J, 0) for i in insts])
    assert N.sdft_batch_apply_tuning(b2.handle)
    assert N.sdft_batch_get_stages_per_pass(b2.handle) == N.sdft_batch_get_stages_per_pass(b.handle)
    assert N.sdft_batch_get_table_staging(b2.handle) == N.sdft_batch_get_table_staging(b.handle)
    assert torch.equal(b2.execute(xb), b.execute(xb))
    torch.cuda.synchronize()
    assert b.device_status() == 0 and b2.device_status() == 0
    N.sdft_autotune_cache_clear()
