"""ctypes binding of libsdft.so: the C ABI of include/sdft.h, same names.

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels. Device buffers are passed as raw pointers; any object with a
`data_ptr()` method (a torch tensor) or an int address is accepted. Streams
are passed as cudaStream_t values (int) or objects with a `cuda_stream`
attribute (torch.cuda.Stream). There is no fallback: if the library is not
built, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsdft.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)

c_u32, c_u64, c_int, c_vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
P_u32 = ctypes.POINTER(ctypes.c_uint32)
P_u64 = ctypes.POINTER(ctypes.c_uint64)
P_f64 = ctypes.POINTER(ctypes.c_double)

SDFT_C64, SDFT_C128 = 0, 1
SDFT_STRATEGY_LEVELS, SDFT_STRATEGY_QUEUE = 1, 2
SDFT_SCHEDULE_AUTO, SDFT_SCHEDULE_LANES, SDFT_SCHEDULE_ROUND_ROBIN = 0, 1, 2
SDFT_PLAN_HOST_ONLY = 0x1
SDFT_PLAN_FP64_DF = 0x8
SDFT_PLAN_USER_ORDER = 0x10
SDFT_SAS_TWO_STAGE = 0x4
SDFT_PLAN_DEFER_DEVICE = 0x2

STATUS = {
    0: "SDFT_OK", 1: "SDFT_ERR_ARG", 2: "SDFT_ERR_NOT_POW2", 3: "SDFT_ERR_RANGE",
    4: "SDFT_ERR_DUPLICATE", 5: "SDFT_ERR_NOT_HOMOGENEOUS", 6: "SDFT_ERR_NOMEM",
    7: "SDFT_ERR_BUDGET", 8: "SDFT_ERR_CUDA", 9: "SDFT_ERR_TIMEOUT", 10: "SDFT_ERR_UNSUPPORTED",
    11: "SDFT_ERR_NO_DEVICE", 12: "SDFT_ERR_PRECISION",
}
STATUS_CODE = {v: k for k, v in STATUS.items()}

class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "submitted", "completed", "failed", "micro_batches", "coeffs", "inflight", "max_inflight",
        "arena_bytes", "arena_peak_bytes", "planned", "injected")]


# Every symbol declared in include/sdft.h: name -> (restype, argtypes)
SIGNATURES = {
    "sdft_plan_create": (c_int, [c_u32, P_u64, c_u64, c_int, c_u32, ctypes.POINTER(c_vp)]),
    "sdft_plan_info": (c_int, [c_vp, P_u32, P_u32, ctypes.POINTER(c_int)]),
    "sdft_plan_pivots": (c_int, [c_vp, P_u32]),
    "sdft_plan_sample_indices": (c_int, [c_vp, P_u64]),
    "sdft_plan_support_order": (c_int, [c_vp, P_u64]),
    "sdft_plan_twiddles": (c_int, [c_vp, P_f64]),
    "sdft_plan_device_bytes": (c_int, [c_vp, P_u64]),
    "sdft_execute": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "sdft_execute_strided": (c_int, [c_vp, c_u64, c_vp, c_vp, c_vp]),
    "sdft_execute_strided_host": (c_int, [c_vp, c_u64, c_vp, c_vp, c_vp, c_vp, c_u64, c_vp]),
    "sdft_execute_batched": (c_int, [c_vp, c_u64, c_vp, c_vp, c_vp, c_vp]),
    "sdft_execute_batched_pin": (c_int, [c_vp, c_u64, c_int]),
    "sdft_debug_bounds_violations": (c_int, [ctypes.POINTER(c_int), P_u64, c_int]),
    "sdft_plan_set_stages_per_pass": (c_int, [c_vp, c_u32]),
    "sdft_plan_get_stages_per_pass": (c_int, [c_vp, P_u32]),
    "sdft_plan_apply_tuning": (c_int, [c_vp, c_u64, ctypes.POINTER(c_int)]),
    "sdft_batch_set_stages_per_pass": (c_int, [c_vp, c_u32]),
    "sdft_batch_get_stages_per_pass": (c_int, [c_vp, P_u32]),
    "sdft_batch_apply_tuning": (c_int, [c_vp, ctypes.POINTER(c_int)]),
    "sdft_batch_set_table_staging": (c_int, [c_vp, c_int]),
    "sdft_server_inject": (c_int, [c_vp, c_u32, c_u64, c_u64]),
    "sdft_batch_get_table_staging": (c_int, [c_vp, ctypes.POINTER(c_int)]),
    "sdft_batch_set_lag": (c_int, [c_vp, c_u32]),
    "sdft_batch_get_lag": (c_int, [c_vp, P_u32]),
    "sdft_autotune_cache_save": (c_int, [ctypes.c_char_p]),
    "sdft_autotune_cache_load": (c_int, [ctypes.c_char_p]),
    "sdft_autotune_cache_clear": (c_int, []),
    "sdft_autotune_cache_size": (c_int, [P_u64]),
    "sdft_execute_batched_cache_info": (c_int, [c_vp, c_u64, ctypes.POINTER(c_int), ctypes.POINTER(c_int), P_u64]),
    "sdft_plan_to_user_order": (c_int, [c_vp, c_u64, c_vp, c_vp, c_vp]),
    "sdft_synthesize_strided_host": (c_int, [c_vp, c_u64, c_vp, c_vp, c_vp, c_vp, c_u64, c_vp]),
    "sdft_synthesize": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "sdft_synthesize_strided": (c_int, [c_vp, c_u64, c_vp, c_vp, c_vp]),
    "sdft_plan_set_strategy": (c_int, [c_vp, c_int]),
    "sdft_plan_autotune": (c_int, [c_vp, c_u64, c_vp, c_vp, c_vp, c_int, ctypes.POINTER(c_int),
                                   ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "sdft_plan_device_status": (c_int, [c_vp, c_int]),
    "sdft_plan_destroy": (c_int, [c_vp]),
    "sdft_batch_create": (c_int, [ctypes.POINTER(c_vp), c_u64, ctypes.POINTER(c_vp)]),
    "sdft_batch_info": (c_int, [c_vp, P_u64, P_u64]),
    "sdft_batch_execute": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "sdft_batch_execute_noalloc": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "sdft_batch_device_status": (c_int, [c_vp, c_int]),
    "sdft_batch_set_wait": (c_int, [c_vp, c_u64, c_u32]),
    "sdft_batch_set_schedule": (c_int, [c_vp, c_int, c_u32]),
    "sdft_batch_autotune": (c_int, [c_vp, c_vp, c_vp, c_vp, c_int, ctypes.POINTER(c_int), P_u32,
                                    ctypes.POINTER(ctypes.c_float)]),
    "sdft_batch_stats": (c_int, [c_vp, P_u64, P_u64, ctypes.POINTER(c_int)]),
    "sdft_batch_destroy": (c_int, [c_vp]),
    "sdft_sas_create": (c_int, [c_u32, P_u64, c_u64, c_int, c_u32, c_u32, ctypes.POINTER(c_vp)]),
    "sdft_sas_info": (c_int, [c_vp, P_u32, P_u32, P_u64, P_u32, P_f64]),
    "sdft_sas_pivots": (c_int, [c_vp, P_u32]),
    "sdft_sas_sample_indices": (c_int, [c_vp, P_u64]),
    "sdft_sas_support_order": (c_int, [c_vp, P_u64]),
    "sdft_sas_workspace_bytes": (c_int, [c_vp, c_u64, P_u64]),
    "sdft_sas_path": (c_int, [c_vp, P_u32, P_u64]),
    "sdft_sas_execute": (c_int, [c_vp, c_u64, c_vp, c_vp, c_vp, c_vp]),
    "sdft_sas_destroy": (c_int, [c_vp]),
    "sdft_server_create": (c_int, [c_int, c_u64, c_u32, c_u32, c_u32, ctypes.POINTER(c_vp)]),
    "sdft_server_submit": (c_int, [c_vp, c_vp, c_vp, c_vp, c_u64]),
    "sdft_server_submit_support": (c_int, [c_vp, c_u32, P_u64, c_u64, c_vp, c_vp, c_u64]),
    "sdft_server_poll": (c_int, [c_vp, P_u64, P_f64, ctypes.POINTER(ctypes.c_int32), c_u64, P_u64]),
    "sdft_server_drain": (c_int, [c_vp, c_u64]),
    "sdft_server_get_stats": (c_int, [c_vp, ctypes.POINTER(ServerStats)]),
    "sdft_server_device_status": (c_int, [c_vp, c_int]),
    "sdft_server_destroy": (c_int, [c_vp]),
    "sdft_status_string": (ctypes.c_char_p, [c_int]),
    "sdft_last_cuda_error": (c_int, []),
    "sdft_version": (c_int, []),
}

for _name, (_res, _args) in SIGNATURES.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class SdftError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        self.name = STATUS.get(self.status, f"status {status}")
        msg = f"{where}: {self.name} ({_lib.sdft_status_string(self.status).decode()})"
        if self.status == 8:
            msg += f" [cuda error {_lib.sdft_last_cuda_error()}]"
        super().__init__(msg)


def _check(status: int, where: str) -> None:
    if status != 0:
        raise SdftError(status, where)


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    raise TypeError(f"cannot take a device pointer from {type(x)!r}")


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    raise TypeError(f"cannot take a cudaStream_t from {type(s)!r}")


# ---------------------------------------------------------------------------
# Functions with the C names
# ---------------------------------------------------------------------------

def sdft_plan_create(log2N: int, J: Sequence[int], prec: int = SDFT_C64, flags: int = 0) -> int:
    arr = np.ascontiguousarray(np.asarray(J, dtype=np.uint64))
    out = c_vp()
    _check(_lib.sdft_plan_create(int(log2N), arr.ctypes.data_as(P_u64), int(arr.size), int(prec),
                                 int(flags), ctypes.byref(out)), "sdft_plan_create")
    return int(out.value)


def sdft_plan_info(plan: int):
    m, s, p = c_u32(), c_u32(), c_int()
    _check(_lib.sdft_plan_info(plan, ctypes.byref(m), ctypes.byref(s), ctypes.byref(p)), "sdft_plan_info")
    return int(m.value), int(s.value), int(p.value)


def sdft_plan_pivots(plan: int) -> np.ndarray:
    s = sdft_plan_info(plan)[1]
    out = np.zeros(max(s, 1), dtype=np.uint32)
    _check(_lib.sdft_plan_pivots(plan, out.ctypes.data_as(P_u32)), "sdft_plan_pivots")
    return out[:s]


def sdft_plan_sample_indices(plan: int) -> np.ndarray:
    k = 1 << sdft_plan_info(plan)[1]
    out = np.zeros(k, dtype=np.uint64)
    _check(_lib.sdft_plan_sample_indices(plan, out.ctypes.data_as(P_u64)), "sdft_plan_sample_indices")
    return out


def sdft_plan_support_order(plan: int) -> np.ndarray:
    k = 1 << sdft_plan_info(plan)[1]
    out = np.zeros(k, dtype=np.uint64)
    _check(_lib.sdft_plan_support_order(plan, out.ctypes.data_as(P_u64)), "sdft_plan_support_order")
    return out


def sdft_plan_twiddles(plan: int) -> np.ndarray:
    """FP64 twiddles, stage-major, complex array of k-1 entries."""
    k = 1 << sdft_plan_info(plan)[1]
    out = np.zeros(2 * max(k - 1, 1), dtype=np.float64)
    _check(_lib.sdft_plan_twiddles(plan, out.ctypes.data_as(P_f64)), "sdft_plan_twiddles")
    return out[: 2 * (k - 1)].view(np.complex128)


def sdft_plan_device_bytes(plan: int) -> int:
    b = c_u64()
    _check(_lib.sdft_plan_device_bytes(plan, ctypes.byref(b)), "sdft_plan_device_bytes")
    return int(b.value)


def sdft_execute(plan: int, d_samples, d_coeffs, stream=None) -> None:
    _check(_lib.sdft_execute(plan, _ptr(d_samples), _ptr(d_coeffs), _stream(stream)), "sdft_execute")


def sdft_execute_strided(plan: int, batch: int, d_samples, d_coeffs, stream=None) -> None:
    _check(_lib.sdft_execute_strided(plan, int(batch), _ptr(d_samples), _ptr(d_coeffs), _stream(stream)),
           "sdft_execute_strided")


def sdft_execute_strided_host(plan: int, batch: int, h_samples, h_coeffs, d_samples, d_coeffs, chunk: int = 0,
                              stream=None) -> None:
    _check(_lib.sdft_execute_strided_host(plan, int(batch), _ptr(h_samples), _ptr(h_coeffs), _ptr(d_samples),
                                          _ptr(d_coeffs), int(chunk), _stream(stream)), "sdft_execute_strided_host")


def sdft_plan_to_user_order(plan: int, batch: int, d_canonical, d_user, stream=None) -> None:
    _check(_lib.sdft_plan_to_user_order(plan, int(batch), _ptr(d_canonical), _ptr(d_user), _stream(stream)),
           "sdft_plan_to_user_order")


def sdft_execute_batched(plans, d_samples, d_offsets, d_coeffs, stream=None) -> None:
    """plans: sequence of plan handles; d_offsets: device array of n + 1 uint64 offsets."""
    arr = (c_vp * len(plans))(*[int(p) for p in plans])
    _check(_lib.sdft_execute_batched(arr, len(plans), _ptr(d_samples), _ptr(d_offsets), _ptr(d_coeffs),
                                     _stream(stream)), "sdft_execute_batched")


def sdft_plan_set_stages_per_pass(plan: int, stages_per_pass: int) -> None:
    _check(_lib.sdft_plan_set_stages_per_pass(plan, int(stages_per_pass)), "sdft_plan_set_stages_per_pass")


def sdft_plan_get_stages_per_pass(plan: int) -> int:
    v = c_u32(0)
    _check(_lib.sdft_plan_get_stages_per_pass(plan, ctypes.byref(v)), "sdft_plan_get_stages_per_pass")
    return int(v.value)


def sdft_plan_apply_tuning(plan: int, batch: int) -> bool:
    found = c_int(0)
    _check(_lib.sdft_plan_apply_tuning(plan, int(batch), ctypes.byref(found)), "sdft_plan_apply_tuning")
    return bool(found.value)


def sdft_batch_set_stages_per_pass(batch: int, stages_per_pass: int) -> None:
    _check(_lib.sdft_batch_set_stages_per_pass(batch, int(stages_per_pass)), "sdft_batch_set_stages_per_pass")


def sdft_batch_get_stages_per_pass(batch: int) -> int:
    v = c_u32(0)
    _check(_lib.sdft_batch_get_stages_per_pass(batch, ctypes.byref(v)), "sdft_batch_get_stages_per_pass")
    return int(v.value)


SDFT_INJECT_OFF, SDFT_INJECT_DROP, SDFT_INJECT_FAIL, SDFT_INJECT_DELAY = 0, 1, 2, 3


def sdft_server_inject(srv: int, mode: int, every: int = 0, delay_us: int = 0) -> None:
    _check(_lib.sdft_server_inject(srv, int(mode), int(every), int(delay_us)), "sdft_server_inject")


def sdft_batch_set_table_staging(batch: int, staged: bool) -> None:
    _check(_lib.sdft_batch_set_table_staging(batch, 1 if staged else 0), "sdft_batch_set_table_staging")


def sdft_batch_get_table_staging(batch: int) -> bool:
    v = c_int(0)
    _check(_lib.sdft_batch_get_table_staging(batch, ctypes.byref(v)), "sdft_batch_get_table_staging")
    return bool(v.value)


def sdft_batch_set_lag(batch: int, lag: int) -> None:
    _check(_lib.sdft_batch_set_lag(batch, int(lag)), "sdft_batch_set_lag")


def sdft_batch_get_lag(batch: int) -> int:
    v = c_u32(0)
    _check(_lib.sdft_batch_get_lag(batch, ctypes.byref(v)), "sdft_batch_get_lag")
    return int(v.value)


def sdft_batch_apply_tuning(batch: int) -> bool:
    found = c_int(0)
    _check(_lib.sdft_batch_apply_tuning(batch, ctypes.byref(found)), "sdft_batch_apply_tuning")
    return bool(found.value)


def sdft_autotune_cache_save(path: str) -> None:
    _check(_lib.sdft_autotune_cache_save(os.fsencode(path)), "sdft_autotune_cache_save")


def sdft_autotune_cache_load(path: str) -> None:
    _check(_lib.sdft_autotune_cache_load(os.fsencode(path)), "sdft_autotune_cache_load")


def sdft_autotune_cache_clear() -> None:
    _check(_lib.sdft_autotune_cache_clear(), "sdft_autotune_cache_clear")


def sdft_autotune_cache_size() -> int:
    v = c_u64(0)
    _check(_lib.sdft_autotune_cache_size(ctypes.byref(v)), "sdft_autotune_cache_size")
    return int(v.value)


def sdft_debug_bounds_violations(clear: bool = False):
    """(enabled, count): range-check violations of the debug build on the current device."""
    en, cnt = c_int(0), c_u64(0)
    _check(_lib.sdft_debug_bounds_violations(ctypes.byref(en), ctypes.byref(cnt), 1 if clear else 0),
           "sdft_debug_bounds_violations")
    return bool(en.value), int(cnt.value)


def sdft_execute_batched_pin(plans, pin: bool) -> None:
    """Pin (build if needed) or unpin the cached sdft_execute_batched list of plans."""
    arr = (c_vp * len(plans))(*[int(p) for p in plans])
    _check(_lib.sdft_execute_batched_pin(arr, len(plans), 1 if pin else 0), "sdft_execute_batched_pin")


def sdft_execute_batched_cache_info(plans=()):
    """(cached, pinned, number of cached lists) for the list of plans."""
    arr = (c_vp * len(plans))(*[int(p) for p in plans]) if len(plans) else None
    cached, pinned, n = c_int(0), c_int(0), c_u64(0)
    _check(_lib.sdft_execute_batched_cache_info(arr, len(plans), ctypes.byref(cached), ctypes.byref(pinned),
                                                ctypes.byref(n)), "sdft_execute_batched_cache_info")
    return bool(cached.value), bool(pinned.value), int(n.value)


def sdft_synthesize_strided_host(plan: int, batch: int, h_coeffs, h_samples, d_coeffs, d_samples, chunk: int = 0,
                                 stream=None) -> None:
    _check(_lib.sdft_synthesize_strided_host(plan, int(batch), _ptr(h_coeffs), _ptr(h_samples), _ptr(d_coeffs),
                                             _ptr(d_samples), int(chunk), _stream(stream)),
           "sdft_synthesize_strided_host")


def sdft_plan_set_strategy(plan: int, strategy: int) -> None:
    _check(_lib.sdft_plan_set_strategy(plan, int(strategy)), "sdft_plan_set_strategy")


def sdft_synthesize(plan: int, d_coeffs, d_samples, stream=None) -> None:
    _check(_lib.sdft_synthesize(plan, _ptr(d_coeffs), _ptr(d_samples), _stream(stream)), "sdft_synthesize")


def sdft_synthesize_strided(plan: int, batch: int, d_coeffs, d_samples, stream=None) -> None:
    _check(_lib.sdft_synthesize_strided(plan, int(batch), _ptr(d_coeffs), _ptr(d_samples), _stream(stream)),
           "sdft_synthesize_strided")


def sdft_plan_autotune(plan: int, batch: int, d_samples, d_coeffs, stream=None, reps: int = 5):
    """Returns (chosen strategy, ms per call with per-level launches, ms with the work queue)."""
    ch, a, b = c_int(), ctypes.c_float(), ctypes.c_float()
    _check(_lib.sdft_plan_autotune(plan, int(batch), _ptr(d_samples), _ptr(d_coeffs), _stream(stream), int(reps),
                                   ctypes.byref(ch), ctypes.byref(a), ctypes.byref(b)), "sdft_plan_autotune")
    return int(ch.value), float(a.value), float(b.value)


def sdft_plan_device_status(plan: int, clear: bool = False) -> int:
    """Returns the status code (0 = ok) held in the plan's device status word."""
    return int(_lib.sdft_plan_device_status(plan, int(bool(clear))))


def sdft_plan_destroy(plan: int) -> None:
    _check(_lib.sdft_plan_destroy(plan), "sdft_plan_destroy")


def sdft_batch_create(plans: Sequence[int]) -> int:
    arr = (c_vp * len(plans))(*[int(p) for p in plans])
    out = c_vp()
    _check(_lib.sdft_batch_create(arr, len(plans), ctypes.byref(out)), "sdft_batch_create")
    return int(out.value)


def sdft_batch_info(batch: int, n: int):
    total = c_u64()
    offs = np.zeros(n + 1, dtype=np.uint64)
    _check(_lib.sdft_batch_info(batch, ctypes.byref(total), offs.ctypes.data_as(P_u64)), "sdft_batch_info")
    return int(total.value), offs


def sdft_batch_execute(batch: int, d_samples, d_coeffs, stream=None) -> None:
    _check(_lib.sdft_batch_execute(batch, _ptr(d_samples), _ptr(d_coeffs), _stream(stream)), "sdft_batch_execute")


def sdft_batch_execute_noalloc(batch: int, d_samples, d_coeffs, stream=None) -> None:
    _check(_lib.sdft_batch_execute_noalloc(batch, _ptr(d_samples), _ptr(d_coeffs), _stream(stream)),
           "sdft_batch_execute_noalloc")


def sdft_batch_device_status(batch: int, clear: bool = False) -> int:
    return int(_lib.sdft_batch_device_status(batch, int(bool(clear))))


def sdft_batch_set_wait(batch: int, timeout_ns: int = 0, need_bias: int = 0) -> None:
    _check(_lib.sdft_batch_set_wait(batch, int(timeout_ns), int(need_bias)), "sdft_batch_set_wait")


def sdft_batch_set_schedule(batch: int, schedule: int = SDFT_SCHEDULE_AUTO, grid: int = 0) -> None:
    _check(_lib.sdft_batch_set_schedule(batch, int(schedule), int(grid)), "sdft_batch_set_schedule")


def sdft_batch_autotune(batch: int, d_samples, d_coeffs, stream=None, reps: int = 3):
    """Returns (chosen schedule, chosen grid, ms per run of the chosen shape)."""
    ch, g, ms = c_int(), c_u32(), ctypes.c_float()
    _check(_lib.sdft_batch_autotune(batch, _ptr(d_samples), _ptr(d_coeffs), _stream(stream), int(reps),
                                    ctypes.byref(ch), ctypes.byref(g), ctypes.byref(ms)), "sdft_batch_autotune")
    return int(ch.value), int(g.value), float(ms.value)


def sdft_batch_stats(batch: int):
    ni, nc, g = c_u64(), c_u64(), c_int()
    _check(_lib.sdft_batch_stats(batch, ctypes.byref(ni), ctypes.byref(nc), ctypes.byref(g)), "sdft_batch_stats")
    return int(ni.value), int(nc.value), int(g.value)


def sdft_batch_destroy(batch: int) -> None:
    _check(_lib.sdft_batch_destroy(batch), "sdft_batch_destroy")


def sdft_sas_create(log2N: int, J, prec: int = SDFT_C64, R: int = 0, flags: int = 0) -> int:
    arr = np.ascontiguousarray(np.asarray(J, dtype=np.uint64))
    out = c_vp()
    _check(_lib.sdft_sas_create(int(log2N), arr.ctypes.data_as(P_u64), int(arr.size), int(prec), int(R), int(flags),
                                ctypes.byref(out)), "sdft_sas_create")
    return int(out.value)


def sdft_sas_info(sas: int):
    """Returns (R, mu*, samples per instance, occupied classes, largest class condition number)."""
    R, mu, ns, occ, cond = c_u32(), c_u32(), c_u64(), c_u32(), ctypes.c_double()
    _check(_lib.sdft_sas_info(sas, ctypes.byref(R), ctypes.byref(mu), ctypes.byref(ns), ctypes.byref(occ),
                              ctypes.byref(cond)), "sdft_sas_info")
    return int(R.value), int(mu.value), int(ns.value), int(occ.value), float(cond.value)


def sdft_sas_pivots(sas: int, R: int) -> np.ndarray:
    out = np.zeros(max(R, 1), dtype=np.uint32)
    _check(_lib.sdft_sas_pivots(sas, out.ctypes.data_as(P_u32)), "sdft_sas_pivots")
    return out[:R]


def sdft_sas_sample_indices(sas: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    _check(_lib.sdft_sas_sample_indices(sas, out.ctypes.data_as(P_u64)), "sdft_sas_sample_indices")
    return out


def sdft_sas_support_order(sas: int, k: int) -> np.ndarray:
    out = np.zeros(k, dtype=np.uint64)
    _check(_lib.sdft_sas_support_order(sas, out.ctypes.data_as(P_u64)), "sdft_sas_support_order")
    return out


def sdft_sas_workspace_bytes(sas: int, batch: int) -> int:
    out = c_u64()
    _check(_lib.sdft_sas_workspace_bytes(sas, int(batch), ctypes.byref(out)), "sdft_sas_workspace_bytes")
    return int(out.value)


def sdft_sas_path(sas: int):
    """Returns (launches per call, values per instance stage 1 leaves in the workspace)."""
    l, v = c_u32(), c_u64()
    _check(_lib.sdft_sas_path(sas, ctypes.byref(l), ctypes.byref(v)), "sdft_sas_path")
    return int(l.value), int(v.value)


def sdft_sas_execute(sas: int, batch: int, d_samples, d_work, d_coeffs, stream=None) -> None:
    _check(_lib.sdft_sas_execute(sas, int(batch), _ptr(d_samples), _ptr(d_work), _ptr(d_coeffs), _stream(stream)),
           "sdft_sas_execute")


def sdft_sas_destroy(sas: int) -> None:
    _check(_lib.sdft_sas_destroy(sas), "sdft_sas_destroy")


def sdft_server_create(prec: int, budget_bytes: int, n_slots: int = 2, max_batch: int = 64,
                       n_planners: int = 4) -> int:
    out = c_vp()
    _check(_lib.sdft_server_create(int(prec), int(budget_bytes), int(n_slots), int(max_batch), int(n_planners),
                                   ctypes.byref(out)), "sdft_server_create")
    return int(out.value)


def sdft_server_submit(server: int, plan: int, h_samples, h_coeffs, tag: int) -> None:
    _check(_lib.sdft_server_submit(server, plan, _ptr(h_samples), _ptr(h_coeffs), int(tag)), "sdft_server_submit")


def sdft_server_submit_support(server: int, log2N: int, J, h_samples, h_coeffs, tag: int) -> None:
    Ja = np.ascontiguousarray(np.asarray(J, dtype=np.uint64))
    _check(_lib.sdft_server_submit_support(server, int(log2N), Ja.ctypes.data_as(P_u64), int(Ja.size),
                                           _ptr(h_samples), _ptr(h_coeffs), int(tag)), "sdft_server_submit_support")


def sdft_server_poll(server: int, cap: int = 4096):
    tags = np.zeros(cap, dtype=np.uint64)
    lat = np.zeros(cap, dtype=np.float64)
    st = np.zeros(cap, dtype=np.int32)
    n = c_u64()
    _check(_lib.sdft_server_poll(server, tags.ctypes.data_as(P_u64), lat.ctypes.data_as(P_f64),
                                 st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cap, ctypes.byref(n)),
           "sdft_server_poll")
    k = int(n.value)
    return tags[:k], lat[:k], st[:k]


def sdft_server_drain(server: int, timeout_ms: int = 0) -> None:
    _check(_lib.sdft_server_drain(server, int(timeout_ms)), "sdft_server_drain")


def sdft_server_get_stats(server: int) -> dict:
    st = ServerStats()
    _check(_lib.sdft_server_get_stats(server, ctypes.byref(st)), "sdft_server_get_stats")
    return {n: int(getattr(st, n)) for n, _ in ServerStats._fields_}


def sdft_server_device_status(server: int, clear: bool = False) -> int:
    return int(_lib.sdft_server_device_status(server, int(bool(clear))))


def sdft_server_destroy(server: int) -> None:
    _check(_lib.sdft_server_destroy(server), "sdft_server_destroy")


def sdft_status_string(status: int) -> str:
    return _lib.sdft_status_string(int(status)).decode()


def sdft_last_cuda_error() -> int:
    return int(_lib.sdft_last_cuda_error())


def sdft_version() -> int:
    return int(_lib.sdft_version())
