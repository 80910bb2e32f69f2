"""CPU checks of the bench's host-side helpers and of its reference arm (the
oracle timed on the host cores), none of which needs a GPU."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_committed_traffic_matches_kernel_source():
    # the committed DRAM figure is used only while the kernel source it was
    # captured on is unchanged; an unknown workload has none
    import hashlib
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        entry = json.load(fh)["20/12/4096"]
    with open(os.path.join(ROOT, "paper_2211_15299_gb300", "csrc", "kernels.cuh"), "rb") as fh:
        current = hashlib.sha256(fh.read()).hexdigest()[:16]
    v = bench._committed_traffic(20, 12, 4096)
    if entry["kernels_cuh_sha"] == current:
        assert v == entry["dram_bytes_per_launch"] and v > 0
    else:
        assert v is None
    assert bench._committed_traffic(20, 12, 4095) is None


def test_clock_summary_reasons():
    s = bench.ClockSampler(0)
    s.lines = ["1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "2010, 2070, 1210.5, 0x4, Not Active, Not Active, Not Active, Active",
               "2032, 2070, 1250.0, 0x4, Not Active, Not Active, Not Active, Active",
               "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbled"]
    out = s.summary()
    assert out["sm_mhz"] == 2010.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 3


def test_cpu_oracle_rows_against_numpy_oracle():
    # the C Algorithm 1 leg reports ~0 relative L2 for rows that are the
    # numpy oracle's own output, and O(1) for rows that are not
    rng = np.random.default_rng(71)
    M, s = 14, 6
    piv = W.random_pivots(M, s, rng)
    J = W.homogeneous_support(M, piv, rng)
    Jc = O.canonical_support_by_key(J, piv)
    F = W.complex_gaussian((7, 1 << s), rng)
    ref = O.transform_levels(M, piv, Jc, F)
    dt, used, err = bench._cpu_oracle_rows(M, piv, J, F, ref, threads=2)
    assert dt >= 0 and used >= 1
    assert err < 1e-13
    _, _, bad = bench._cpu_oracle_rows(M, piv, J, F, ref[:, ::-1], threads=2)
    assert bad > 0.1


def test_reference_arm_line():
    # `bench.py --impl reference` runs the oracle alone, without CUDA, and prints
    # one JSON line in the bench's format
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--batch", "16"],
                       capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 2 and d["warmup"] == 3          # warm-up raised to the minimum of 3
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["batch"] == 16
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}



def test_cpu_baseline_leg():
    # the bench's cpu_baseline object on a small shared-support batch, with the
    # oracle's own output standing in for the GPU rows
    import torch
    inst, _ = W.workload_shared(M=12, s=6, batch=1, coeffs=False)
    rng = np.random.default_rng(72)
    F = W.complex_gaussian((32, inst.k), rng)
    Jc = O.canonical_support_by_key(inst.J, inst.pivots)
    C = O.transform_levels(inst.M, inst.pivots, Jc, F)
    x32 = torch.from_numpy(F.astype(np.complex64))
    y32 = torch.from_numpy(C.astype(np.complex64))
    d = bench.cpu_baseline(inst, x32, y32, 4)
    assert d["kind"] == "oracle" and d["unit"] == bench.UNIT and d["cores"] >= 1
    assert d["passes"] >= 3 and d["value"] == pytest.approx(32 * inst.k / d["seconds"])
    assert d["rel_l2_gpu_fp32_vs_oracle"] < 1e-6
    assert d["dense_solve"]["rel_l2_gpu_fp32_vs_oracle"] < 1e-6
    assert d["alg1_numpy"]["rel_l2_gpu_fp32_vs_oracle"] < 1e-6


@pytest.mark.parametrize("per_set", [1, 58 << 20, 92 << 20, 225 << 20, 268 << 20, 1 << 30, 3 << 30])
def test_rotating_sets_keep_inputs_out_of_l2(per_set):
    # the steady-state timing rotates over enough buffer sets that at least
    # 1 GiB (several L2 capacities) passes between two uses of one set; a set
    # of 1 GiB or more is used alone
    n = bench.steady_sets(per_set)
    assert 1 <= n <= 32
    if per_set >= 1 << 30:
        assert n == 1
    else:
        assert (n - 1) * per_set >= 1 << 30 or n == 32
