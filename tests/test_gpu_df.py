"""GPU: complex128 plans in double-float arithmetic (SDFT_PLAN_FP64_DF) against
the FP64 oracle (1e-12) and against the FP64-pipe path."""
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


def _instance(rng, M, s):
    piv = np.sort(rng.choice(np.arange(M), size=s, replace=False))
    return piv, W.homogeneous_support(M, piv, rng)


@pytest.mark.parametrize("M,s,batch", [(16, 5, 3), (16, 8, 70), (16, 11, 9), (20, 12, 5), (22, 16, 3),
                                       (24, 20, 1), (26, 21, 1)])
def test_df_against_oracle_and_fp64(M, s, batch):
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(9100 + 10 * s + M)
    piv, J = _instance(rng, M, s)
    df = Plan(M, J, "c128", fp64_df=True)
    f64 = Plan(M, J, "c128")
    assert df.device_bytes == 2 * f64.device_bytes - 256     # a second table of the same size
    Jc = O.canonical_support_by_key(J, piv)
    C = W.complex_gaussian((batch, df.k), rng)
    F = O.synthesize_levels(M, piv, Jc, C)
    x = torch.from_numpy(F).cuda()
    y = df.execute_strided(x)
    y64 = f64.execute_strided(x)
    torch.cuda.synchronize()
    assert df.device_status() == 0
    got = y.cpu().numpy()
    for b in range(batch):
        assert rel_l2(got[b], C[b]) < 1e-12
    assert float(torch.linalg.vector_norm(y - y64) / torch.linalg.vector_norm(y64)) < 1e-12
    # synthesis in double-float returns the samples
    f_back = df.synthesize(y)
    torch.cuda.synchronize()
    assert float(torch.linalg.vector_norm(f_back - x) / torch.linalg.vector_norm(x)) < 1e-12


def test_df_largest_N():
    # N = 2^62: the last stage's twiddles carry N/k = 2^49 (FP32 range), samples ~ 2^-56
    torch = _torch()
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(9200)
    M, s = 62, 13
    piv, J = _instance(rng, M, s)
    p = Plan(M, J, "c128", fp64_df=True)
    Jc = O.canonical_support_by_key(J, piv)
    C = W.complex_gaussian((2, p.k), rng)
    F = O.synthesize_levels(M, piv, Jc, C)
    y = p.execute_strided(torch.from_numpy(F).cuda())
    torch.cuda.synchronize()
    assert p.device_status() == 0
    assert rel_l2(y.cpu().numpy(), C) < 1e-12
