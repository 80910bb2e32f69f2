"""CPU checks of the autotuners' cache (no GPU): the JSON file round trip, the
keys (precision, log2 k, batch bucket; batches by instance count and total),
applying a stored choice to host-only plans and batches, and rejection of
malformed files and of choices a plan cannot take."""
import json

import numpy as np
import pytest

import workloads as W


def _plan(M, s, prec="c64", seed=0):
    from paper_2211_15299_gb300 import Plan
    rng = np.random.default_rng(seed)
    piv = W.random_pivots(M, s, rng)
    return Plan(M, W.homogeneous_support(M, piv, rng), prec, host_only=True)


@pytest.fixture(autouse=True)
def _empty_cache():
    from paper_2211_15299_gb300 import _native as N
    N.sdft_autotune_cache_clear()
    yield
    N.sdft_autotune_cache_clear()


def test_cache_file_round_trip(tmp_path):
    from paper_2211_15299_gb300 import _native as N
    src = {"plan/c64/s12/b12": {"strategy": 1, "schedule": 0, "grid": 0, "stages_per_pass": 3, "ms": 0.05},
           "plan/c128/s20/b6": {"strategy": 2, "schedule": 0, "grid": 0, "stages_per_pass": 4, "ms": 1.5},
           "batch/c64/n13/t26": {"strategy": 0, "schedule": 2, "grid": 152, "stages_per_pass": 4, "lag": 8,
                                 "ms": 0.46}}
    f = tmp_path / "tune.json"
    f.write_text(json.dumps(src))
    N.sdft_autotune_cache_load(str(f))
    assert N.sdft_autotune_cache_size() == 3
    out = tmp_path / "out.json"
    N.sdft_autotune_cache_save(str(out))
    back = json.loads(out.read_text())
    assert back.keys() == src.keys()
    for k in src:
        for field, v in src[k].items():
            assert back[k][field] == pytest.approx(v, rel=1e-6), (k, field)
    # loading merges: a second file adds to (and overrides) the first
    f2 = tmp_path / "more.json"
    f2.write_text(json.dumps({"plan/c64/s12/b12": {"strategy": 1, "stages_per_pass": 4}}))
    N.sdft_autotune_cache_load(str(f2))
    assert N.sdft_autotune_cache_size() == 3
    N.sdft_autotune_cache_save(str(out))
    assert json.loads(out.read_text())["plan/c64/s12/b12"]["stages_per_pass"] == 4


@pytest.mark.parametrize("text", ["", "[]", "{", '{"a": 1}', '{"a": {"strategy": "x"}}',
                                  '{"a": {"unknown": 1}}', '{"a": {}} trailing'])
def test_malformed_files_are_rejected_and_leave_the_cache(tmp_path, text):
    from paper_2211_15299_gb300 import SdftError, _native as N
    good = tmp_path / "good.json"
    good.write_text(json.dumps({"plan/c64/s5/b0": {"strategy": 1, "stages_per_pass": 4}}))
    N.sdft_autotune_cache_load(str(good))
    bad = tmp_path / "bad.json"
    bad.write_text(text)
    with pytest.raises(SdftError) as ei:
        N.sdft_autotune_cache_load(str(bad))
    assert ei.value.name == "SDFT_ERR_ARG"
    assert N.sdft_autotune_cache_size() == 1
    with pytest.raises(SdftError):
        N.sdft_autotune_cache_load(str(tmp_path / "missing.json"))


def test_plan_choice_applied_by_key(tmp_path):
    # key: precision, log2 k and floor(log2 batch); pivot positions do not matter
    from paper_2211_15299_gb300 import _native as N
    f = tmp_path / "tune.json"
    f.write_text(json.dumps({"plan/c64/s12/b12": {"strategy": 1, "stages_per_pass": 3}}))
    N.sdft_autotune_cache_load(str(f))
    for seed in range(3):
        p = _plan(20, 12, seed=seed)
        assert N.sdft_plan_get_stages_per_pass(p.handle) == 4
        assert not N.sdft_plan_apply_tuning(p.handle, 2048)        # bucket 11: none
        assert N.sdft_plan_get_stages_per_pass(p.handle) == 4
        assert N.sdft_plan_apply_tuning(p.handle, 4096)            # 4096 .. 8191
        assert N.sdft_plan_get_stages_per_pass(p.handle) == 3
        q = _plan(20, 12, seed=seed)
        assert N.sdft_plan_apply_tuning(q.handle, 8191)
        assert not N.sdft_plan_apply_tuning(_plan(20, 11, seed=seed).handle, 4096)   # other k
        assert not N.sdft_plan_apply_tuning(_plan(20, 12, "c128", seed).handle, 4096)  # other precision


def test_stages_per_pass_limits():
    from paper_2211_15299_gb300 import SdftError, _native as N
    p64, p128 = _plan(16, 10), _plan(16, 10, "c128")
    for v in (3, 4):
        N.sdft_plan_set_stages_per_pass(p64.handle, v)
        assert N.sdft_plan_get_stages_per_pass(p64.handle) == v
    N.sdft_plan_set_stages_per_pass(p128.handle, 4)
    for h, bad in ((p64.handle, 2), (p64.handle, 5), (p128.handle, 3)):
        with pytest.raises(SdftError) as ei:
            N.sdft_plan_set_stages_per_pass(h, bad)
        assert ei.value.name == "SDFT_ERR_ARG"


def test_cached_choice_a_plan_cannot_take_is_rejected(tmp_path):
    from paper_2211_15299_gb300 import SdftError, _native as N
    f = tmp_path / "tune.json"
    f.write_text(json.dumps({"plan/c128/s10/b0": {"strategy": 1, "stages_per_pass": 3}}))
    N.sdft_autotune_cache_load(str(f))
    p = _plan(16, 10, "c128")
    with pytest.raises(SdftError):
        N.sdft_plan_apply_tuning(p.handle, 1)
    assert N.sdft_plan_get_stages_per_pass(p.handle) == 4


def test_batch_choice_applied_and_item_list_rebuilt(tmp_path):
    # a host-only batch: its item list is built for inspection; applying a
    # cached choice sets the schedule, grid and stages per pass
    from paper_2211_15299_gb300 import Batch, _native as N
    insts = W.workload_uneven(count=200, salt=5)
    from paper_2211_15299_gb300 import Plan
    plans = [Plan(i.M, i.J, "c64", host_only=True) for i in insts]
    b = Batch(plans)
    n_bits = int(np.floor(np.log2(len(plans))))
    t_bits = int(np.floor(np.log2(b.total)))
    key = f"batch/c64/n{n_bits}/t{t_bits}"
    f = tmp_path / "tune.json"
    f.write_text(json.dumps({key: {"schedule": 1, "grid": 100, "stages_per_pass": 3, "table_staging": 1,
                                   "lag": 5}}))
    assert not N.sdft_batch_apply_tuning(b.handle)
    N.sdft_autotune_cache_load(str(f))
    assert N.sdft_batch_apply_tuning(b.handle)
    assert N.sdft_batch_get_stages_per_pass(b.handle) == 3
    assert N.sdft_batch_get_table_staging(b.handle)
    assert N.sdft_batch_get_lag(b.handle) == 5
    items, counters, grid = b.stats()
    assert grid == 100 and items > 0


def test_cached_dependency_distance_below_the_minimum_is_rejected(tmp_path):
    # a lag under 4 would let a persistent launch wait on a counter that is
    # never published in time: the cache entry is refused, the batch unchanged
    from paper_2211_15299_gb300 import Batch, Plan, SdftError, _native as N
    insts = W.workload_uneven(count=200, salt=5)
    b = Batch([Plan(i.M, i.J, "c64", host_only=True) for i in insts])
    key = f"batch/c64/n{int(np.floor(np.log2(len(insts))))}/t{int(np.floor(np.log2(b.total)))}"
    f = tmp_path / "tune.json"
    f.write_text(json.dumps({key: {"schedule": 1, "grid": 100, "stages_per_pass": 4, "lag": 3}}))
    N.sdft_autotune_cache_load(str(f))
    with pytest.raises(SdftError) as ei:
        N.sdft_batch_apply_tuning(b.handle)
    assert ei.value.name == "SDFT_ERR_ARG"
    assert N.sdft_batch_get_lag(b.handle) == 6
