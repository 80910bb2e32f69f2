"""Object wrappers over the C ABI: `Plan` (one support) and `Batch` (many).

Torch is used for device buffers and streams only; every transform step runs
in libsdft.so. Output tensors are allocated here when the caller passes none.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from . import _native as N

_PREC = {"c64": N.SDFT_C64, "complex64": N.SDFT_C64, "c128": N.SDFT_C128, "complex128": N.SDFT_C128}


def _torch():
    import torch
    return torch


def _dtype(prec: int):
    torch = _torch()
    return torch.complex64 if prec == N.SDFT_C64 else torch.complex128


def _current_stream(stream):
    if stream is not None:
        return stream
    torch = _torch()
    return torch.cuda.current_stream().cuda_stream


def _numel(t, what: str) -> int:
    if not isinstance(t, _torch().Tensor):
        raise TypeError(f"{what} must be a torch tensor")
    return t.numel()


def _check_tensor(t, dtype, numel: int, what: str):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{what} must live on a CUDA device")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{what} must hold {numel} values, got {t.numel()}")


class Plan:
    """A validated homogeneous support with its sample set and device twiddles."""

    def __init__(self, log2N: int, J: Sequence[int], prec="c64", host_only: bool = False, defer: bool = False,
                 fp64_df: bool = False, user_order: bool = False):
        """host_only: host tables only (introspection). defer: device tables kept in host
        memory until a Server uploads them with a request (no device allocation).
        fp64_df (complex128): butterflies in double-float arithmetic on the FP32 pipes."""
        code = _PREC[prec] if isinstance(prec, str) else int(prec)
        flags = (N.SDFT_PLAN_HOST_ONLY if host_only else 0) | (N.SDFT_PLAN_DEFER_DEVICE if defer else 0)
        flags |= N.SDFT_PLAN_FP64_DF if fp64_df else 0
        flags |= N.SDFT_PLAN_USER_ORDER if user_order else 0
        self.handle = N.sdft_plan_create(log2N, J, code, flags)
        self.log2N, self.s, self.prec = N.sdft_plan_info(self.handle)
        self.k = 1 << self.s
        self._cache = {}

    # -- introspection ---------------------------------------------------
    @property
    def pivots(self) -> np.ndarray:
        if "pivots" not in self._cache:
            self._cache["pivots"] = N.sdft_plan_pivots(self.handle)
        return self._cache["pivots"]

    @property
    def sample_indices(self) -> np.ndarray:
        if "I" not in self._cache:
            self._cache["I"] = N.sdft_plan_sample_indices(self.handle)
        return self._cache["I"]

    @property
    def support_order(self) -> np.ndarray:
        if "Jc" not in self._cache:
            self._cache["Jc"] = N.sdft_plan_support_order(self.handle)
        return self._cache["Jc"]

    def twiddles(self) -> np.ndarray:
        return N.sdft_plan_twiddles(self.handle)

    @property
    def device_bytes(self) -> int:
        return N.sdft_plan_device_bytes(self.handle)

    @property
    def dtype(self):
        return _dtype(self.prec)

    # -- execution ---------------------------------------------------------
    def execute(self, samples, coeffs=None, stream=None):
        """One instance: samples[t] = f(I[t]) -> coeffs[t] = (F f)(Jc[t])."""
        return self.execute_strided(samples, coeffs, stream, batch=1)

    def execute_strided(self, samples, coeffs=None, stream=None, batch: Optional[int] = None):
        """`batch` packed instances (samples shaped [batch, k] or flat)."""
        if batch is None:
            batch = _numel(samples, "samples") // self.k
        _check_tensor(samples, self.dtype, batch * self.k, "samples")
        if coeffs is None:
            coeffs = _torch().empty_like(samples)
        _check_tensor(coeffs, self.dtype, batch * self.k, "coeffs")
        N.sdft_execute_strided(self.handle, batch, samples, coeffs, _current_stream(stream))
        return coeffs

    def execute_host(self, h_samples, h_coeffs=None, d_samples=None, d_coeffs=None, chunk: int = 0,
                     stream=None, batch: Optional[int] = None):
        """execute_strided on host tensors (pinned for overlap): copy-in, transform
        and copy-out in overlapped chunks of `chunk` instances (0: about 16 MiB).
        Device staging buffers are allocated here when not given. The result is in
        `h_coeffs` once `stream` (the current stream by default) reaches this point."""
        return self._host(N.sdft_execute_strided_host, h_samples, h_coeffs, d_samples, d_coeffs, chunk, stream,
                          batch)

    def synthesize_host(self, h_coeffs, h_samples=None, d_coeffs=None, d_samples=None, chunk: int = 0,
                        stream=None, batch: Optional[int] = None):
        """synthesize on host tensors, copies overlapped in chunks (see execute_host)."""
        return self._host(N.sdft_synthesize_strided_host, h_coeffs, h_samples, d_coeffs, d_samples, chunk, stream,
                          batch)

    def _host(self, fn, h_in, h_out, d_in, d_out, chunk, stream, batch):
        torch = _torch()
        if batch is None:
            batch = _numel(h_in, "host input") // self.k
        for t, what in ((h_in, "host input"), (h_out, "host output")):
            if t is None:
                continue
            if not isinstance(t, torch.Tensor) or t.is_cuda:
                raise ValueError(f"{what} must be a host tensor")
            if t.dtype != self.dtype or not t.is_contiguous() or t.numel() != batch * self.k:
                raise ValueError(f"{what} must be a contiguous {self.dtype} tensor of {batch * self.k} values")
        if h_out is None:
            h_out = torch.empty_like(h_in, pin_memory=True)
        dev = torch.device("cuda", torch.cuda.current_device())
        if d_in is None:
            d_in = torch.empty(batch * self.k, dtype=self.dtype, device=dev)
        if d_out is None:
            d_out = torch.empty(batch * self.k, dtype=self.dtype, device=dev)
        _check_tensor(d_in, self.dtype, batch * self.k, "device input")
        _check_tensor(d_out, self.dtype, batch * self.k, "device output")
        fn(self.handle, batch, h_in, h_out, d_in, d_out, chunk, _current_stream(stream))
        return h_out

    def to_user_order(self, coeffs, out=None, stream=None, batch: Optional[int] = None):
        """Coefficients from canonical order into the order of J as given to the
        plan (plans created with user_order=True)."""
        if batch is None:
            batch = _numel(coeffs, "coeffs") // self.k
        _check_tensor(coeffs, self.dtype, batch * self.k, "coeffs")
        if out is None:
            out = _torch().empty_like(coeffs)
        _check_tensor(out, self.dtype, batch * self.k, "out")
        N.sdft_plan_to_user_order(self.handle, batch, coeffs, out, _current_stream(stream))
        return out

    def synthesize(self, coeffs, samples=None, stream=None, batch: Optional[int] = None):
        """Samples from coefficients (the inverse of execute_strided)."""
        if batch is None:
            batch = _numel(coeffs, "coeffs") // self.k
        _check_tensor(coeffs, self.dtype, batch * self.k, "coeffs")
        if samples is None:
            samples = _torch().empty_like(coeffs)
        _check_tensor(samples, self.dtype, batch * self.k, "samples")
        N.sdft_synthesize_strided(self.handle, batch, coeffs, samples, _current_stream(stream))
        return samples

    def set_strategy(self, strategy: str):
        """'levels' (one launch per butterfly level) or 'queue' (one work-queue launch)."""
        N.sdft_plan_set_strategy(self.handle, {"levels": N.SDFT_STRATEGY_LEVELS, "queue": N.SDFT_STRATEGY_QUEUE}[strategy])

    def autotune(self, samples, coeffs=None, stream=None, reps: int = 5):
        """Time both strategies on these buffers, keep the faster; returns
        (strategy name, ms levels, ms queue)."""
        batch = _numel(samples, "samples") // self.k
        _check_tensor(samples, self.dtype, batch * self.k, "samples")
        if coeffs is None:
            coeffs = _torch().empty_like(samples)
        ch, a, b = N.sdft_plan_autotune(self.handle, batch, samples, coeffs, _current_stream(stream), reps)
        return ("levels" if ch == N.SDFT_STRATEGY_LEVELS else "queue"), a, b

    def device_status(self, clear: bool = False) -> int:
        return N.sdft_plan_device_status(self.handle, clear)

    def close(self):
        if getattr(self, "handle", None):
            N.sdft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def execute_batched(plans: Sequence["Plan"], samples, offsets, coeffs=None, stream=None):
    """Instances at the caller's offsets (sdft_execute_batched): plans[i] transforms
    samples[offsets[i]:offsets[i+1]] into the same range of coeffs. `offsets` is a
    device int64 tensor of len(plans) + 1 entries."""
    torch = _torch()
    dt = plans[0].dtype
    if not isinstance(offsets, torch.Tensor) or not offsets.is_cuda or offsets.dtype != torch.int64:
        raise TypeError("offsets must be a CUDA int64 tensor")
    if offsets.numel() != len(plans) + 1 or not offsets.is_contiguous():
        raise ValueError("offsets must hold len(plans) + 1 values")
    _check_tensor(samples, dt, samples.numel(), "samples")
    if coeffs is None:
        coeffs = torch.empty_like(samples)
    _check_tensor(coeffs, dt, samples.numel(), "coeffs")
    N.sdft_execute_batched([p.handle for p in plans], samples, offsets, coeffs, _current_stream(stream))
    return coeffs


class Batch:
    """Many instances with their own plans, run by one persistent kernel."""

    def __init__(self, plans: Sequence[Plan]):
        if not plans:
            raise ValueError("empty batch")
        self.plans = list(plans)            # keep the plans alive
        self.prec = self.plans[0].prec
        self.handle = N.sdft_batch_create([p.handle for p in self.plans])
        self.total, offs = N.sdft_batch_info(self.handle, len(self.plans))
        self.offsets = offs[:-1].astype(np.int64)   # element offset of each instance (caller's order)

    def stats(self):
        """(work items, dependency counters, grid); raises if the item list breaks its invariants."""
        return N.sdft_batch_stats(self.handle)

    def set_wait(self, timeout_ns: int = 0, need_bias: int = 0):
        N.sdft_batch_set_wait(self.handle, timeout_ns, need_bias)

    _SCHEDULES = {"auto": N.SDFT_SCHEDULE_AUTO, "lanes": N.SDFT_SCHEDULE_LANES,
                  "round_robin": N.SDFT_SCHEDULE_ROUND_ROBIN}

    def set_schedule(self, schedule: str = "auto", grid: int = 0):
        """Item order ("auto", "lanes", "round_robin") on `grid` CTAs (0: all co-resident)."""
        N.sdft_batch_set_schedule(self.handle, self._SCHEDULES[schedule], grid)

    def autotune(self, samples, coeffs=None, stream=None, reps: int = 3):
        """Time the queue shapes on these buffers, keep the fastest; returns
        (schedule name, grid, ms per run)."""
        _check_tensor(samples, self.dtype, self.total, "samples")
        if coeffs is None:
            coeffs = _torch().empty_like(samples)
        _check_tensor(coeffs, self.dtype, self.total, "coeffs")
        ch, g, ms = N.sdft_batch_autotune(self.handle, samples, coeffs, _current_stream(stream), reps)
        name = {v: k for k, v in self._SCHEDULES.items()}[ch]
        return name, g, ms

    def pack(self, per_instance):
        """Host-side helper: place per-instance numpy arrays at their offsets."""
        out = np.zeros(self.total, dtype=np.complex128)
        for p, off, x in zip(self.plans, self.offsets, per_instance):
            out[off:off + p.k] = x
        return out

    def unpack(self, flat):
        return [flat[off:off + p.k] for p, off in zip(self.plans, self.offsets)]

    @property
    def dtype(self):
        return _dtype(self.prec)

    def execute(self, samples, coeffs=None, stream=None):
        _check_tensor(samples, self.dtype, self.total, "samples")
        if coeffs is None:
            coeffs = _torch().empty_like(samples)
        _check_tensor(coeffs, self.dtype, self.total, "coeffs")
        N.sdft_batch_execute(self.handle, samples, coeffs, _current_stream(stream))
        return coeffs

    def device_status(self, clear: bool = False) -> int:
        return N.sdft_batch_device_status(self.handle, clear)

    def close(self):
        if getattr(self, "handle", None):
            N.sdft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sas:
    """Shift-and-Sample for an arbitrary support (sdft_sas_*): mu* transforms of
    a homogeneous virtual support over shifted sample sets, then one small
    Vandermonde solve per class."""

    def __init__(self, log2N: int, J: Sequence[int], prec="c64", R: int = 0, host_only: bool = False,
                 two_stage: bool = False):
        """two_stage: always run the class solves as their own launch (otherwise
        both stages share one launch where one virtual instance fills a tile)."""
        self.prec = _PREC[prec] if isinstance(prec, str) else int(prec)
        J = np.asarray(J, dtype=np.uint64)
        self.log2N, self.k = int(log2N), int(J.size)
        flags = (N.SDFT_PLAN_HOST_ONLY if host_only else 0) | (N.SDFT_SAS_TWO_STAGE if two_stage else 0)
        self.handle = N.sdft_sas_create(log2N, J, self.prec, R, flags)
        self.R, self.mu_star, self.n_samples, self.occupied, self.max_cond = N.sdft_sas_info(self.handle)
        # launches per execute and the values per instance that stage 1 leaves
        # in the workspace, with the three buffers apart (sdft_sas_path)
        self.launches, self.work_values = N.sdft_sas_path(self.handle)
        # stage 1 writes only the values the class solves read
        self.gathered = self.mu_star > 1 and self.work_values == self.k

    @property
    def pivots(self) -> np.ndarray:
        return N.sdft_sas_pivots(self.handle, self.R)

    @property
    def sample_indices(self) -> np.ndarray:
        """(mu*, 2^R): row a is the sample set shifted by a."""
        return N.sdft_sas_sample_indices(self.handle, self.n_samples).reshape(self.mu_star, 1 << self.R)

    @property
    def support_order(self) -> np.ndarray:
        return N.sdft_sas_support_order(self.handle, self.k)

    @property
    def dtype(self):
        return _dtype(self.prec)

    def execute(self, samples, coeffs=None, work=None, stream=None):
        """samples: (batch, mu* x 2^R) or (mu* x 2^R,) device tensor; returns (batch, k)."""
        torch = _torch()
        _numel(samples, "samples")
        x = samples.reshape(-1, self.n_samples)
        batch = x.shape[0]
        _check_tensor(x, self.dtype, batch * self.n_samples, "samples")
        if coeffs is None:
            coeffs = torch.empty((batch, self.k), dtype=x.dtype, device=x.device)
        _check_tensor(coeffs, self.dtype, batch * self.k, "coeffs")
        if work is None:
            work = torch.empty_like(x)
        _check_tensor(work, self.dtype, batch * self.n_samples, "work")
        N.sdft_sas_execute(self.handle, batch, x, work, coeffs, _current_stream(stream))
        return coeffs

    def close(self):
        if getattr(self, "handle", None):
            N.sdft_sas_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching serving engine (sdft_server_*).

    Requests carry a Plan (or a support, planned by the engine's own planner
    threads) and pinned host tensors; the engine copies samples in, runs
    micro-batches as persistent work-queue launches on a few streams, copies
    coefficients out and reports per-request latency."""

    def __init__(self, prec="c64", budget_bytes: int = 1 << 30, n_slots: int = 2, max_batch: int = 64,
                 n_planners: int = 4):
        self.prec = _PREC[prec] if isinstance(prec, str) else int(prec)
        self.handle = N.sdft_server_create(self.prec, budget_bytes, n_slots, max_batch, n_planners)
        self._live = {}      # tag -> (plan, h_in, h_out) kept alive until completion

    def submit(self, plan: Plan, h_in, h_out, tag: int):
        self._live[int(tag)] = (plan, h_in, h_out)
        N.sdft_server_submit(self.handle, plan.handle, h_in, h_out, tag)

    def submit_support(self, log2N: int, J, h_in, h_out, tag: int):
        """A request with its own support: planned inside the engine; h_in holds
        the samples at the support's sample set (sample order), h_out receives
        the coefficients in canonical order."""
        self._live[int(tag)] = (None, h_in, h_out)
        N.sdft_server_submit_support(self.handle, log2N, J, h_in, h_out, tag)

    def poll(self, cap: int = 4096):
        tags, lat, st = N.sdft_server_poll(self.handle, cap)
        for t in tags:
            self._live.pop(int(t), None)
        return tags, lat, st

    def drain(self, timeout_ms: int = 0):
        N.sdft_server_drain(self.handle, timeout_ms)

    def stats(self) -> dict:
        return N.sdft_server_get_stats(self.handle)

    def device_status(self, clear: bool = False) -> int:
        return N.sdft_server_device_status(self.handle, clear)

    def close(self):
        if getattr(self, "handle", None):
            N.sdft_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
