"""GPU parity of the uneven-batch work-queue kernel against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _instances(rng, sizes, M_extra=(0, 8)):
    out = []
    for s in sizes:
        M = max(s, 1) + int(rng.integers(M_extra[0], M_extra[1] + 1))
        piv = W.random_pivots(M, s, rng)
        out.append(W.Instance(M, piv, W.homogeneous_support(M, piv, rng)))
    return out


def _run_batch(insts, prec, rng, batch=None):
    torch = _torch()
    from paper_2211_15299_gb300 import Batch, Plan
    plans = [Plan(i.M, i.J, prec) for i in insts]
    b = Batch(plans) if batch is None else batch
    Jcs, Cs, Fs = [], [], []
    for i in insts:
        Jc = O.canonical_support_by_key(i.J, i.pivots)
        C = W.complex_gaussian(i.k, rng)
        Jcs.append(Jc)
        Cs.append(C)
        Fs.append(O.synthesize_levels(i.M, i.pivots, Jc, C))
    np_dt = np.complex64 if prec == 0 else np.complex128
    flat = b.pack(Fs).astype(np_dt)
    x = torch.from_numpy(flat).cuda()
    y = b.execute(x)
    torch.cuda.synchronize()
    st = b.device_status()
    got = b.unpack(y.cpu().numpy().astype(np.complex128))
    f_in = b.unpack(flat.astype(np.complex128))
    return b, plans, st, got, f_in, Jcs, Cs


@pytest.mark.parametrize("prec", [0, 1])
def test_uneven_batch_all_paths(prec):
    rng = np.random.default_rng(900 + prec)
    tb = 12 if prec == 0 else 11
    # small (s <= 4), whole-instance tiles with partial groups, one- and two-level large
    sizes = [0, 1, 2, 3, 4, 4, 5, 5, 5, 6, 7, 8, 8, 9, 10, 11, tb, tb, tb + 1, tb + 2, tb + 4]
    sizes += list(rng.integers(0, tb + 3, size=40))
    insts = _instances(rng, [int(s) for s in rng.permutation(sizes)])
    b, plans, st, got, f_in, Jcs, Cs = _run_batch(insts, prec, rng)
    assert st == 0
    for i, inst in enumerate(insts):
        ref = O.transform_levels(inst.M, inst.pivots, Jcs[i], f_in[i])
        assert rel_l2(got[i], ref) < TOL[prec], (i, inst.s)


def test_uneven_workload_reduced():
    """The uneven workload's recipe at 400 instances (M in 12..24, s in 4..16)."""
    rng = np.random.default_rng(4040)
    insts = W.workload_uneven(count=400, salt=11)
    b, plans, st, got, f_in, Jcs, Cs = _run_batch(insts, 0, rng)
    assert st == 0
    n_items, n_ctr, grid = b.stats()
    assert n_ctr > 0
    worst = max(rel_l2(got[i], Cs[i]) for i in range(len(insts)))
    assert worst < 1e-5
    for i in range(0, len(insts), 37):
        ref = O.transform_levels(insts[i].M, insts[i].pivots, Jcs[i], f_in[i])
        assert rel_l2(got[i], ref) < 1e-5


def test_three_level_instances_in_batch():
    rng = np.random.default_rng(4141)
    insts = _instances(rng, [21, 13, 20, 6, 0, 21])
    b, plans, st, got, f_in, Jcs, Cs = _run_batch(insts, 0, rng)
    assert st == 0
    for i, inst in enumerate(insts):
        assert rel_l2(got[i], Cs[i]) < 1e-5, inst.s


def test_batch_equals_strided():
    torch = _torch()
    from paper_2211_15299_gb300 import Batch, Plan
    rng = np.random.default_rng(4242)
    inst, _ = W.workload_shared(M=22, s=14, batch=1, coeffs=False, salt=5)
    plan = Plan(inst.M, inst.J, 0)
    B = 12
    x = torch.randn((B, inst.k), dtype=torch.complex64, device="cuda")
    ref = plan.execute_strided(x)
    b = Batch([plan] * B)
    xb = torch.empty(b.total, dtype=torch.complex64, device="cuda")
    for i in range(B):
        xb[b.offsets[i]:b.offsets[i] + inst.k] = x[i]
    yb = b.execute(xb)
    torch.cuda.synchronize()
    for i in range(B):
        got = yb[b.offsets[i]:b.offsets[i] + inst.k]
        assert float(torch.linalg.vector_norm(got - ref[i]) / torch.linalg.vector_norm(ref[i])) < 1e-6


def test_batch_graph_capture_replay():
    torch = _torch()
    from paper_2211_15299_gb300 import Batch, Plan
    rng = np.random.default_rng(4343)
    insts = _instances(rng, [14, 9, 3, 12, 16])
    plans = [Plan(i.M, i.J, 0) for i in insts]
    b = Batch(plans)
    x = torch.randn(b.total, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    ref = b.execute(x).clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.execute(x, y, stream=s.cuda_stream)
    for _ in range(3):
        y.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(y, ref)
    assert b.device_status() == 0


def test_dependency_wait_times_out_and_recovers():
    """A dependency target that is never reached ends the launch with
    SDFT_ERR_TIMEOUT in the status word; the context stays usable."""
    torch = _torch()
    from paper_2211_15299_gb300 import Batch, Plan
    rng = np.random.default_rng(4444)
    insts = _instances(rng, [14, 13])
    plans = [Plan(i.M, i.J, 0) for i in insts]
    b = Batch(plans)
    x = torch.randn(b.total, dtype=torch.complex64, device="cuda")
    b.set_wait(timeout_ns=20_000_000, need_bias=1)
    b.execute(x)
    torch.cuda.synchronize()
    assert b.device_status(clear=True) == 9          # SDFT_ERR_TIMEOUT
    b.set_wait(0, 0)
    y = b.execute(x)
    torch.cuda.synchronize()
    assert b.device_status() == 0
    for i, p in enumerate(plans):
        ref = p.execute_strided(x[b.offsets[i]:b.offsets[i] + p.k].clone())
        got = y[b.offsets[i]:b.offsets[i] + p.k]
        assert float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref)) < 1e-6


@pytest.mark.parametrize("s", [14, 20, 21])
def test_strided_queue_strategy_matches_oracle(s):
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(4500 + s)
    inst = _instances(rng, [s])[0]
    plan = Plan(inst.M, inst.J, 0)
    Jc = O.canonical_support_by_key(inst.J, inst.pivots)
    B = 3
    C = W.complex_gaussian((B, inst.k), rng)
    F = O.synthesize_levels(inst.M, inst.pivots, Jc, C).astype(np.complex64)
    x = torch.from_numpy(F).cuda()
    ref = plan.execute_strided(x).clone()
    plan.set_strategy("queue")
    y = plan.execute_strided(x)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    got = y.cpu().numpy().astype(np.complex128)
    assert rel_l2(got, C) < 1e-5
    assert float(torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref)) < 1e-6


def test_autotune_chooses_a_strategy():
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(4600)
    inst = _instances(rng, [16])[0]
    plan = Plan(inst.M, inst.J, 0)
    x = torch.randn((8, inst.k), dtype=torch.complex64, device="cuda")
    name, ms_levels, ms_queue = plan.autotune(x.clone(), reps=2)
    assert name in ("levels", "queue") and ms_levels > 0 and ms_queue > 0
    y = plan.execute_strided(x)
    plan.set_strategy("levels")
    ref = plan.execute_strided(x)
    torch.cuda.synchronize()
    assert float(torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref)) < 1e-6


def test_queue_shapes_bit_identical_and_autotune():
    """Every item order and grid the autotuner may choose gives the same bits;
    the autotuned batch still matches the oracle."""
    torch = _torch()
    rng = np.random.default_rng(5151)
    insts = W.workload_uneven(count=300, salt=13)
    b, plans, st, got, f_in, Jcs, Cs = _run_batch(insts, 0, rng)
    assert st == 0
    x = torch.from_numpy(b.pack(f_in).astype(np.complex64)).cuda()
    ref = b.execute(x).clone()
    full = b.stats()[2]
    for schedule, grid in (("lanes", 0), ("round_robin", 0), ("lanes", full // 2), ("round_robin", 37)):
        b.set_schedule(schedule, grid)
        y = b.execute(x)
        torch.cuda.synchronize()
        assert b.device_status() == 0
        assert b.stats()[2] == (grid if grid else full)
        assert torch.equal(y.view(torch.float32), ref.view(torch.float32)), (schedule, grid)
    name, grid, ms = b.autotune(x, reps=2)
    assert name in ("lanes", "round_robin") and grid in (full, full // 2) and ms > 0
    y = b.execute(x)
    torch.cuda.synchronize()
    assert torch.equal(y.view(torch.float32), ref.view(torch.float32))
    out = b.unpack(y.cpu().numpy().astype(np.complex128))
    worst = max(rel_l2(out[i], Cs[i]) for i in range(len(insts)))
    assert worst < 1e-5


@pytest.mark.parametrize("prec", [0, 1])
def test_execute_batched_at_caller_offsets(prec):
    """sdft_execute_batched: instances packed in the caller's order (not the
    batch's by decreasing k); each equals its strided transform bit for bit; in
    place; graph capture of a warmed-up call."""
    torch = _torch()
    from paper_2211_15299_gb300 import Plan, execute_batched
    rng = np.random.default_rng(7300 + prec)
    tb = 12 if prec == 0 else 11
    sizes = [int(s) for s in rng.permutation([0, 3, 5, 7, 9, 10, tb, tb, tb + 1, tb + 3, 4, 6])]
    insts = _instances(rng, sizes)
    plans = [Plan(i.M, i.J, prec) for i in insts]
    dt = torch.complex64 if prec == 0 else torch.complex128
    # packing in the given order (offsets[i+1] - offsets[i] = k_i, no 16-byte
    # alignment of the instances needed), then the list reversed, in place
    packed = np.concatenate([[0], np.cumsum([p.k for p in plans])]).astype(np.int64)
    xs = torch.randn(int(packed[-1]), dtype=dt, device="cuda")
    d_off = torch.from_numpy(packed).cuda()
    y = execute_batched(plans, xs, d_off)
    torch.cuda.synchronize()
    assert plans[0].device_status() == 0
    for i, p in enumerate(plans):
        a, b = int(packed[i]), int(packed[i + 1])
        ref = p.execute_strided(xs[a:b].clone())
        assert torch.equal(y[a:b], ref), i
    rplans = plans[::-1]
    rpacked = np.concatenate([[0], np.cumsum([p.k for p in rplans])]).astype(np.int64)
    xr = torch.randn(int(rpacked[-1]), dtype=dt, device="cuda")
    yr = xr.clone()
    execute_batched(rplans, yr, torch.from_numpy(rpacked).cuda(), yr)       # in place
    torch.cuda.synchronize()
    for i, p in enumerate(rplans):
        a, b = int(rpacked[i]), int(rpacked[i + 1])
        assert torch.equal(yr[a:b], p.execute_strided(xr[a:b].clone())), i
    # graph capture of a warmed-up call, replayed on new samples
    s = torch.cuda.Stream()
    out = torch.empty_like(xs)
    with torch.cuda.stream(s):
        execute_batched(plans, xs, d_off, out, stream=s.cuda_stream)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        execute_batched(plans, xs, d_off, out, stream=s.cuda_stream)
    xs.copy_(torch.randn_like(xs))
    g.replay()
    torch.cuda.synchronize()
    for i, p in enumerate(plans):
        a, b = int(packed[i]), int(packed[i + 1])
        assert torch.equal(out[a:b], p.execute_strided(xs[a:b].clone())), i
    assert plans[0].device_status() == 0


def test_execute_batched_reports_offsets_that_do_not_fit():
    torch = _torch()
    from paper_2211_15299_gb300 import Plan, execute_batched
    rng = np.random.default_rng(7400)
    plans = [Plan(i.M, i.J, 0) for i in _instances(rng, [6, 12, 8])]
    ks = [p.k for p in plans]
    bad = np.array([0, ks[0], ks[0] + ks[1] - 2, sum(ks)], dtype=np.int64)   # instance 1 two values short
    x = torch.randn(sum(ks), dtype=torch.complex64, device="cuda")
    execute_batched(plans, x, torch.from_numpy(bad).cuda())
    torch.cuda.synchronize()
    assert plans[0].device_status(clear=True) == 0x104
    assert plans[0].device_status() == 0


def test_execute_batched_cache_released_with_its_plans():
    """Destroying a plan of a cached execute_batched list frees that list's batch
    and staging buffers (2 x 2^24 complex64 values here, 256 MiB); a new list of
    new plans then runs correctly."""
    torch = _torch()
    from paper_2211_15299_gb300 import Plan, execute_batched
    rng = np.random.default_rng(7500)
    insts = _instances(rng, [12] * 4)
    plans = [Plan(insts[0].M, insts[0].J, 0)] * 4096     # one plan, repeated
    ks = plans[0].k
    off = torch.arange(0, ks * 4097, ks, dtype=torch.int64, device="cuda")
    x = torch.randn(ks * 4096, dtype=torch.complex64, device="cuda")
    y = execute_batched(plans, x, off)
    torch.cuda.synchronize()
    assert torch.equal(y[:ks], plans[0].execute_strided(x[:ks].clone()))
    del y
    torch.cuda.empty_cache()
    free0, _ = torch.cuda.mem_get_info()
    plans[0].close()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 - free0 >= 2 * ks * 4096 * 8            # the two staging halves
    fresh = [Plan(i.M, i.J, 0) for i in insts[:3]]
    packed = torch.tensor([0, ks, 2 * ks, 3 * ks], dtype=torch.int64, device="cuda")
    z = execute_batched(fresh, x[:3 * ks], packed)
    torch.cuda.synchronize()
    for i, p in enumerate(fresh):
        assert torch.equal(z[i * ks:(i + 1) * ks], p.execute_strided(x[i * ks:(i + 1) * ks].clone())), i
    assert fresh[0].device_status() == 0


def test_execute_batched_pinned_list_survives_eviction():
    """A pinned execute_batched list (the one a CUDA graph was captured on) is
    never freed by building other lists; unpinned, it is evicted by age like any
    other. The graph is replayed only while its list is pinned."""
    torch = _torch()
    from paper_2211_15299_gb300 import Plan, execute_batched, _native as N
    rng = np.random.default_rng(7600)
    pool = [Plan(i.M, i.J, 0) for i in _instances(rng, [5, 6, 7, 8, 9, 10, 11, 12, 13, 4, 3])]
    base = [pool[0], pool[7], pool[8]]                   # the list the graph is captured on
    ks = [p.k for p in base]
    packed = np.concatenate([[0], np.cumsum(ks)]).astype(np.int64)
    d_off = torch.from_numpy(packed).cuda()
    xs = torch.randn(int(packed[-1]), dtype=torch.complex64, device="cuda")
    out = torch.empty_like(xs)
    N.sdft_execute_batched_pin([p.handle for p in base], True)
    assert N.sdft_execute_batched_cache_info([p.handle for p in base])[:2] == (True, True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        execute_batched(base, xs, d_off, out, stream=s.cuda_stream)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        execute_batched(base, xs, d_off, out, stream=s.cuda_stream)
    # nine other lists: more than the eight unpinned lists kept
    others = [[pool[i], pool[(i + 1) % len(pool)]] for i in range(1, 10)]
    for lst in others:
        k2 = [p.k for p in lst]
        off2 = torch.tensor([0, k2[0], k2[0] + k2[1]], dtype=torch.int64, device="cuda")
        execute_batched(lst, torch.randn(sum(k2), dtype=torch.complex64, device="cuda"), off2)
    torch.cuda.synchronize()
    assert N.sdft_execute_batched_cache_info([p.handle for p in base])[:2] == (True, True)
    assert N.sdft_execute_batched_cache_info([p.handle for p in others[0]])[0] is False   # oldest unpinned: freed
    assert N.sdft_execute_batched_cache_info([p.handle for p in others[-1]])[0] is True
    xs.copy_(torch.randn_like(xs))
    g.replay()                                           # its list is still pinned and cached
    torch.cuda.synchronize()
    for i, p in enumerate(base):
        a, b = int(packed[i]), int(packed[i + 1])
        assert torch.equal(out[a:b], p.execute_strided(xs[a:b].clone())), i
    del g                                                # no replay after this point
    N.sdft_execute_batched_pin([p.handle for p in base], False)
    assert N.sdft_execute_batched_cache_info([p.handle for p in base])[:2] == (True, False)
    k2 = [pool[10].k, pool[9].k]
    off2 = torch.tensor([0, k2[0], k2[0] + k2[1]], dtype=torch.int64, device="cuda")
    execute_batched([pool[10], pool[9]], torch.randn(sum(k2), dtype=torch.complex64, device="cuda"), off2)
    torch.cuda.synchronize()
    assert N.sdft_execute_batched_cache_info([p.handle for p in base])[0] is False    # now the oldest: freed
    assert pool[0].device_status() == 0
