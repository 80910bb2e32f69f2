"""GPU parity of Shift-and-Sample against the FP64 oracle (oracle/sas.py)."""
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


# Flat tolerances, the bounds the transform itself is held to. They hold because
# the planner keeps every class system's 1-norm condition at or below 32
# (complex64) or 100 (complex128): stage 1 carries the transform's rounding
# (about 2e-7 relative for complex64, 2e-15 for complex128) and each class solve
# multiplies a relative error by at most its condition.
_COND_CAP = {"c64": 32.0, "c128": 100.0}


def _tol(prec, cond):
    assert cond <= _COND_CAP[prec], f"class condition {cond} above the planner's cap"
    return 1e-5 if prec == "c64" else 1e-12


def _case(M, J, prec, R, batch, rng):
    """Plan, draw `batch` coefficient vectors, synthesise the shifted samples by
    the direct sum, run on the GPU; returns (plan, got, c in output order,
    the FP64 oracle on the same rounded samples)."""
    torch = _torch()
    from paper_2211_15299_gb300 import Sas
    J = [int(j) for j in J]
    p = Sas(M, J, prec, R=R)
    order = [int(j) for j in p.support_order]
    r = [int(x) for x in p.pivots]
    assert r == O.sas_pivots(J, M, p.R)
    idx = p.sample_indices
    C = W.complex_gaussian((batch, len(J)), rng)
    F = np.stack([O.sas_samples_direct(M, order, C[b], idx) for b in range(batch)])
    np_dt = np.complex64 if prec == "c64" else np.complex128
    x = torch.from_numpy(F.reshape(batch, -1).astype(np_dt)).cuda()
    y = p.execute(x)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    f_in = x.cpu().numpy().astype(np.complex128).reshape(batch, p.mu_star, -1)
    ref = np.stack([O.sas_transform(M, order, r, f_in[b]) for b in range(batch)])
    return p, got, C, ref


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_paper_example(prec):
    rng = np.random.default_rng(61)
    p, got, C, ref = _case(10, [0, 512, 1, 6, 7], prec, 2, 3, rng)
    assert p.mu_star == 2 and p.n_samples == 8
    assert rel_l2(got, ref) < _tol(prec, p.max_cond)
    assert rel_l2(got, C) < _tol(prec, p.max_cond)


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("seed", range(4))
def test_arbitrary_sets(prec, seed):
    rng = np.random.default_rng(700 + seed)
    M = int(rng.integers(8, 17))
    k = int(rng.integers(5, min(600, 1 << M)))
    J = sorted(int(x) for x in rng.choice(1 << M, size=k, replace=False))
    p, got, C, ref = _case(M, J, prec, 0, 2, rng)
    assert rel_l2(got, ref) < _tol(prec, p.max_cond), (p.R, p.mu_star, p.max_cond)
    assert rel_l2(got, C) < _tol(prec, p.max_cond)


@pytest.mark.parametrize("kind", ["ap", "subset", "uoh"])
def test_workloads_reduced(kind):
    # the bench's supports (N = 2^20, k = 3000) on a few instances
    rng = np.random.default_rng(62)
    J = W.workload_sas(kind)
    p, got, C, ref = _case(20, J, "c64", 0, 2, rng)
    assert rel_l2(got, C) < _tol("c64", p.max_cond) and rel_l2(got, ref) < _tol("c64", p.max_cond)


def test_batch_rows_are_independent():
    torch = _torch()
    from paper_2211_15299_gb300 import Sas
    J = W.workload_sas("subset", M=16, k=500, salt=3)
    p = Sas(16, J, "c64")
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    x = torch.randn((37, p.n_samples), dtype=torch.complex64, device="cuda", generator=g)
    y = p.execute(x)
    for b in (0, 17, 36):
        assert torch.equal(p.execute(x[b:b + 1].clone())[0], y[b])
    # in place: the samples buffer as workspace
    x2 = x.clone()
    y2 = p.execute(x2, work=x2)
    torch.cuda.synchronize()
    assert torch.equal(y2, y)


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_random_subset_of_a_homogeneous_set(prec):
    # Theorem "hom_rand_subset"'s family (the pivot count of the theorem itself is
    # checked on the host in tests/test_sas_host.py: its class systems are far
    # too ill-conditioned for floating point); the planner's R on the GPU
    log2k = 10
    rng = W.rng_for(0, 4321)
    J, piv = W.bernoulli_subset_of_homogeneous(18, log2k + 3, 1 << log2k, rng)
    p, got, C, ref = _case(18, [int(j) for j in J], prec, 0, 2, np.random.default_rng(8))
    assert [int(x) for x in p.pivots] == [int(x) for x in piv[:p.R]]
    assert rel_l2(got, ref) < _tol(prec, p.max_cond), p.max_cond
    assert rel_l2(got, C) < _tol(prec, p.max_cond)


@pytest.mark.parametrize("kind,k,prec,batch", [("ap", 3000, "c64", 700), ("ap", 3000, "c64", 5),
                                               ("ap", 2000, "c128", 333), ("subset", 3000, "c64", 5)])
def test_one_launch_and_two_launch_paths_agree_bitwise(kind, k, prec, batch):
    """Under complete isolation (mu* = 1) with one virtual instance per tile
    (R = 12 complex64, 11 complex128) both stages share one launch; the two-launch
    path (SDFT_SAS_TWO_STAGE) gives the same bits, and both match the oracle
    (the subset case, mu* = 3, runs two launches either way)."""
    torch = _torch()
    from paper_2211_15299_gb300 import Sas
    J = [int(j) for j in W.workload_sas(kind, k=k)]
    one = Sas(20, J, prec)
    two = Sas(20, J, prec, two_stage=True)
    assert (one.R, one.mu_star) == (two.R, two.mu_star)
    if kind == "ap":
        assert one.mu_star == 1 and one.R == (12 if prec == "c64" else 11)
    dt = torch.complex64 if prec == "c64" else torch.complex128
    g = torch.Generator(device="cuda")
    g.manual_seed(77)
    x = torch.randn((batch, one.n_samples), dtype=dt, device="cuda", generator=g)
    x_keep = x.clone()
    y1 = one.execute(x)
    y2 = two.execute(x)
    torch.cuda.synchronize()
    assert torch.equal(x, x_keep)               # the samples are left alone
    assert torch.equal(y1, y2)
    # a few rows against the oracle on the same rounded samples
    order = [int(j) for j in one.support_order]
    r = [int(v) for v in one.pivots]
    f_in = x.cpu().numpy().astype(np.complex128).reshape(batch, one.mu_star, -1)
    got = y1.cpu().numpy().astype(np.complex128)
    for b in (0, batch - 1):
        ref = O.sas_transform(20, order, r, f_in[b])
        assert rel_l2(got[b], ref) < _tol(prec, one.max_cond)


@pytest.mark.parametrize("kind,k,prec,batch", [("subset", 3000, "c64", 700), ("subset", 3000, "c64", 1),
                                               ("subset", 4000, "c64", 33), ("uoh", 3000, "c64", 301),
                                               ("uoh", 2000, "c64", 51), ("subset", 3000, "c128", 45),
                                               ("subset", 2000, "c128", 19), ("subset", 1000, "c128", 37),
                                               ("subset", 1000, "c64", 99),
                                               ("ap", 2000, "c64", 301), ("ap", 1000, "c64", 7)])
def test_tile_paths_agree_bitwise_with_the_two_launch_path(kind, k, prec, batch):
    """Where one to four virtual instances fill a tile (TB - 2 <= R <= TB):
    with mu* = 1 (k <= 2^TB) both stages share one launch; with mu* > 1
    (k <= 8192) stage 1 writes only the values the class solves read, k per
    instance in output order, for the decoder launch. Each gives the same bits
    as the two-launch path over the whole stage-1 output, as a second call, as
    the in-place call (samples buffer as workspace, which takes the
    whole-output path), and matches the oracle on a few rows. The batches leave
    the last tile part-filled where a tile holds several rows."""
    torch = _torch()
    from paper_2211_15299_gb300 import Sas
    J = [int(j) for j in W.workload_sas(kind, k=k)]
    one = Sas(20, J, prec)
    two = Sas(20, J, prec, two_stage=True)
    tb = 12 if prec == "c64" else 11
    assert tb - 2 <= one.R <= tb
    if one.mu_star == 1:
        assert (one.launches, one.work_values) == (1, 0)
    else:
        assert (one.launches, one.work_values, one.gathered) == (2, one.k, True)
    assert (two.launches, two.work_values) == (2, one.mu_star << one.R)
    dt = torch.complex64 if prec == "c64" else torch.complex128
    g = torch.Generator(device="cuda")
    g.manual_seed(78)
    x = torch.randn((batch, one.n_samples), dtype=dt, device="cuda", generator=g)
    x_keep = x.clone()
    y1 = one.execute(x)
    y1b = one.execute(x)                       # a second call on the same workspace sizes
    y2 = two.execute(x)
    torch.cuda.synchronize()
    assert torch.equal(x, x_keep)
    assert torch.equal(y1, y2) and torch.equal(y1b, y1)
    x3 = x.clone()
    y3 = one.execute(x3, work=x3)               # in place
    torch.cuda.synchronize()
    assert torch.equal(y3, y1)
    order = [int(j) for j in one.support_order]
    r = [int(v) for v in one.pivots]
    f_in = x.cpu().numpy().astype(np.complex128).reshape(batch, one.mu_star, -1)
    got = y1.cpu().numpy().astype(np.complex128)
    for b in sorted({0, batch // 2, batch - 1}):
        ref = O.sas_transform(20, order, r, f_in[b])
        assert rel_l2(got[b], ref) < _tol(prec, one.max_cond)
