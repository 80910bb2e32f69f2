"""GPU tests of the serving engine: continuous batching under a memory budget."""
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


def _requests(rng, sizes):
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    reqs = []
    for s in sizes:
        M = max(s, 1) + int(rng.integers(0, 8))
        piv = W.random_pivots(M, s, rng)
        J = W.homogeneous_support(M, piv, rng)
        plan = Plan(M, J, 0)
        Jc = O.canonical_support_by_key(J, piv)
        c = W.complex_gaussian(1 << s, rng)
        f = O.synthesize_levels(M, piv, Jc, c).astype(np.complex64)
        h_in = torch.from_numpy(f).pin_memory()
        reqs.append((plan, h_in, c, M, piv, Jc))
    return reqs


def _serve(srv, reqs):
    torch = _torch()
    outs = []
    for i, (plan, h_in, *_rest) in enumerate(reqs):
        h_out = torch.empty_like(h_in).pin_memory()
        outs.append(h_out)
        srv.submit(plan, h_in, h_out, i)
    srv.drain(timeout_ms=60_000)
    got = {}
    while len(got) < len(reqs):
        tags, lat, st = srv.poll()
        for t, l, s_ in zip(tags, lat, st):
            got[int(t)] = (float(l), int(s_))
        if not len(tags):
            break
    return outs, got


def test_each_result_same_alone_and_in_the_mix():
    from paper_2211_15299_gb300 import Server
    rng = np.random.default_rng(5150)
    sizes = [int(s) for s in rng.permutation([0, 2, 4, 5, 7, 9, 11, 12, 12, 13, 14, 16, 3, 8, 10, 15] * 3)]
    reqs = _requests(rng, sizes)
    srv = Server("c64", budget_bytes=64 << 20, n_slots=2, max_batch=8)
    alone = []
    for i, r in enumerate(reqs):                       # one request at a time
        out, got = _serve(srv, [r])
        assert got[0][1] == 0
        alone.append(out[0].clone())
    mixed, got = _serve(srv, reqs)                      # all at once
    st = srv.stats()
    assert st["micro_batches"] > len(reqs) and st["max_inflight"] > 1
    assert srv.device_status() == 0
    for i, r in enumerate(reqs):
        plan, h_in, c, M, piv, Jc = r
        assert got[i][1] == 0 and got[i][0] > 0
        x = mixed[i].numpy().astype(np.complex128)
        assert np.array_equal(mixed[i].numpy(), alone[i].numpy()), i
        ref = O.transform_levels(M, piv, Jc, h_in.numpy().astype(np.complex128))
        assert rel_l2(x, ref) < 1e-5, (i, plan.s)
    srv.close()


def test_admission_respects_the_budget():
    torch = _torch()
    from paper_2211_15299_gb300 import Server
    rng = np.random.default_rng(5151)
    reqs = _requests(rng, [16] * 6)                     # 512 KiB each
    srv = Server("c64", budget_bytes=1 << 20, n_slots=4, max_batch=4)   # room for two
    outs, got = _serve(srv, reqs)
    st = srv.stats()
    assert st["completed"] == 6 and st["arena_peak_bytes"] <= 1 << 20
    assert st["max_inflight"] <= 2
    for i, r in enumerate(reqs):
        assert rel_l2(outs[i].numpy().astype(np.complex128), r[2]) < 1e-5
    # a request that can never fit is completed with SDFT_ERR_BUDGET
    big = _requests(rng, [18])
    outs, got = _serve(srv, big)
    assert got[0][1] == 7
    srv.close()


def test_deferred_plans_through_the_server():
    """Plans built with their device tables kept on the host (no device
    allocation at creation) give the same results through a server as plans
    uploaded at creation, and cannot run outside a server."""
    torch = _torch()
    from paper_2211_15299_gb300 import Batch, Plan, SdftError, Server
    rng = np.random.default_rng(5152)
    reqs = _requests(rng, [3, 6, 12, 13, 15, 17])
    srv = Server("c64", budget_bytes=64 << 20, n_slots=2, max_batch=4)
    ref, _ = _serve(srv, reqs)
    deferred = []
    for plan, h_in, c, M, piv, Jc in reqs:
        J = np.asarray(plan.support_order)
        deferred.append((Plan(M, J, 0, defer=True), h_in, c, M, piv, Jc))
    got, status = _serve(srv, deferred)
    assert all(status[i][1] == 0 for i in range(len(reqs)))
    for i in range(len(reqs)):
        assert np.array_equal(got[i].numpy(), ref[i].numpy()), i
    x = torch.zeros(deferred[0][0].k, dtype=torch.complex64, device="cuda")
    with pytest.raises(SdftError):
        deferred[0][0].execute(x)
    with pytest.raises(SdftError):
        Batch([deferred[0][0]])
    srv.close()


def test_requests_that_bring_their_support():
    """Supports planned by the engine's planner threads give the same bits as
    caller-built plans of the same support; an invalid support completes with
    its validation status."""
    torch = _torch()
    from paper_2211_15299_gb300 import Server
    rng = np.random.default_rng(5153)
    reqs = _requests(rng, [0, 4, 7, 12, 13, 16, 17])
    srv = Server("c64", budget_bytes=64 << 20, n_slots=2, max_batch=4, n_planners=3)
    ref, _ = _serve(srv, reqs)
    outs = []
    for i, (plan, h_in, c, M, piv, Jc) in enumerate(reqs):
        h_out = torch.empty_like(h_in).pin_memory()
        outs.append(h_out)
        # the caller's support in its own (shuffled) order
        J = np.asarray(plan.support_order)[rng.permutation(plan.k)]
        srv.submit_support(M, J, h_in, h_out, 100 + i)
    bad_in = torch.zeros(4, dtype=torch.complex64).pin_memory()
    bad_out = torch.empty_like(bad_in).pin_memory()
    srv.submit_support(6, np.array([0, 1, 2, 4], dtype=np.uint64), bad_in, bad_out, 999)   # 3 pivots, k = 4
    srv.drain(timeout_ms=60_000)
    got = {}
    for _ in range(100):
        tags, lat, st = srv.poll()
        for t, l, s_ in zip(tags, lat, st):
            got[int(t)] = (float(l), int(s_))
        if len(got) == len(reqs) + 1:
            break
    assert got[999][1] == 5                                # SDFT_ERR_NOT_HOMOGENEOUS
    for i in range(len(reqs)):
        assert got[100 + i][1] == 0 and got[100 + i][0] > 0
        assert np.array_equal(outs[i].numpy(), ref[i].numpy()), i
    st = srv.stats()
    assert st["planned"] == len(reqs) and st["failed"] == 1
    srv.close()


def test_host_side_fault_injection():
    """The engine's host-side injector (no device fault): dropped requests never
    complete and the client finds them by their absence, failed ones complete
    at once with SDFT_ERR_CUDA, delayed ones run late; every other result is the
    same as when nothing is injected."""
    import time
    from paper_2211_15299_gb300 import Server, _native as N
    rng = np.random.default_rng(5170)
    reqs = _requests(rng, [int(s) for s in rng.permutation([4, 6, 8, 10, 12, 13, 14, 9, 7, 5, 11, 12])])
    srv = Server("c64", budget_bytes=64 << 20, n_slots=2, max_batch=4)
    ref, got = _serve(srv, reqs)
    assert all(got[i][1] == 0 for i in range(len(reqs)))
    # drop every third request
    N.sdft_server_inject(srv.handle, N.SDFT_INJECT_DROP, 3)
    before = srv.stats()["injected"]
    outs, got = _serve(srv, reqs)
    dropped = {i for i in range(len(reqs)) if i not in got}
    assert len(dropped) == len(reqs) // 3 and srv.stats()["injected"] - before == len(dropped)
    for i in got:
        assert got[i][1] == 0 and np.array_equal(outs[i].numpy(), ref[i].numpy()), i
    # fail every fourth
    N.sdft_server_inject(srv.handle, N.SDFT_INJECT_FAIL, 4)
    outs, got = _serve(srv, reqs)
    assert len(got) == len(reqs)
    failed = {i for i, (_, st) in got.items() if st != 0}
    assert len(failed) == len(reqs) // 4
    assert all(got[i][1] == N.STATUS_CODE["SDFT_ERR_CUDA"] for i in failed)
    for i in set(got) - failed:
        assert np.array_equal(outs[i].numpy(), ref[i].numpy()), i
    # delay every second by 20 ms: all complete, the delayed ones late
    N.sdft_server_inject(srv.handle, N.SDFT_INJECT_DELAY, 2, 20_000)
    t0 = time.perf_counter()
    outs, got = _serve(srv, reqs)
    assert len(got) == len(reqs) and all(st == 0 for _, st in got.values())
    assert time.perf_counter() - t0 >= 0.02 * (len(reqs) // 2)
    assert max(l for l, _ in got.values()) >= 0.02
    for i in got:
        assert np.array_equal(outs[i].numpy(), ref[i].numpy()), i
    N.sdft_server_inject(srv.handle, N.SDFT_INJECT_OFF)
    outs, got = _serve(srv, reqs)
    assert len(got) == len(reqs) and all(np.array_equal(outs[i].numpy(), ref[i].numpy()) for i in got)
    assert srv.device_status() == 0
    from paper_2211_15299_gb300 import SdftError
    with pytest.raises(SdftError):
        N.sdft_server_inject(srv.handle, N.SDFT_INJECT_DROP, 0)
    srv.close()
