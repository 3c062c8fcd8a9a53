"""Python face of the SVD-compressed M2L library (thin marshalling layer).

Every step of the translation runs in libkifmm_m2l.so; this module turns
torch tensors and NumPy arrays into pointers and sizes.  PyTorch is used
for device memory and streams only.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import PREC, Params, call, lib


KERNELS = {"laplace": 0, "yukawa": 1}


def _params(p: int, eps: float, d: float, precision: str, kernel="laplace", kappa: float = 0.0,
            box_halfwidth: float = 0.0) -> Params:
    if precision not in PREC:
        raise ValueError(f"precision must be one of {sorted(PREC)}")
    kid = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    return Params(kid, int(p), float(eps), float(d), PREC[precision], float(kappa), float(box_halfwidth))


def surface_count(p: int) -> int:
    """Equivalent / check points per surface: 6(p-1)^2 + 2."""
    return 6 * (p - 1) ** 2 + 2


def factors_host(p: int, eps: float, d: float = 0.1, kernel="laplace", kappa: float = 0.0,
                 box_halfwidth: float = 0.0):
    """Run the library's FP64 precompute on the host.

    Returns (sigma [n], U [n, r], C [316, r, r]) as float64 arrays (for the
    Yukawa kernel: of h K at box half-width h, see ``M2LPlan``).
    """
    prm = _params(p, eps, d, "fp32", kernel, kappa, box_halfwidth)
    n, r = ctypes.c_int(0), ctypes.c_int(0)
    call("kifmm_m2l_factors_host", ctypes.byref(prm), ctypes.byref(n), ctypes.byref(r), None, None, None)
    sigma = np.empty(n.value)
    U = np.empty((n.value, r.value))
    C = np.empty((_lib.N_OFFSETS, r.value, r.value))
    call("kifmm_m2l_factors_host", ctypes.byref(prm), ctypes.byref(n), ctypes.byref(r),
         sigma.ctypes.data, U.ctypes.data, C.ctypes.data)
    return sigma, U, C


def stage2_host(p: int, eps: float, c2: float, d: float = 0.1):
    """The library's host stage-2 factoring (Sec. 3.2): (ranks [316] int32,
    truncated cores Uhat_o Vhat_o [316, r, r] float64)."""
    prm = _params(p, eps, d, "fp32")
    n, r = ctypes.c_int(0), ctypes.c_int(0)
    call("kifmm_m2l_factors_host", ctypes.byref(prm), ctypes.byref(n), ctypes.byref(r), None, None, None)
    k = np.zeros(_lib.N_OFFSETS, np.int32)
    core = np.empty((_lib.N_OFFSETS, r.value, r.value))
    call("kifmm_m2l_stage2_host", ctypes.byref(prm), float(c2), k.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
         core.ctypes.data)
    return k, core


def pairs_host(level: int, box_ijk):
    """Interaction-list pairs built by the library on the host.

    Returns (targets, sources, offset_index) int32 arrays sorted by offset
    then target.
    """
    box = np.ascontiguousarray(box_ijk, dtype=np.int32).reshape(-1, 3)
    cnt = ctypes.c_int64(0)
    call("kifmm_m2l_pairs_host", int(level), box.shape[0], box.ctypes.data, ctypes.byref(cnt), None, None, None)
    tg = np.empty(cnt.value, np.int32)
    sr = np.empty(cnt.value, np.int32)
    of = np.empty(cnt.value, np.int32)
    call("kifmm_m2l_pairs_host", int(level), box.shape[0], box.ctypes.data, ctypes.byref(cnt),
         tg.ctypes.data, sr.ctypes.data, of.ctypes.data)
    return tg, sr, of


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_tensor(x, name, shape):
    import torch

    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {tuple(shape)}")


class M2LPlan:
    """A precomputed compressed M2L operator plus registered octree levels.

    ``precision``: "fp32" (CUDA cores), "bf16", "split3", "split6" or
    "f16x3" (tcgen05 tensor cores; split6 and f16x3 keep FP32-level
    accuracy).  ``kernel``: "laplace", or "yukawa" with ``kappa`` and the
    half-width ``box_halfwidth`` of the one level the plan serves (the
    kernel is not homogeneous: one plan per level, Sec. 3.1).
    """

    def __init__(self, p: int, eps: float, d: float = 0.1, precision: str = "split6", kernel="laplace",
                 kappa: float = 0.0, box_halfwidth: float = 0.0):
        self.p, self.eps, self.d, self.precision = int(p), float(eps), float(d), precision
        self._h = ctypes.c_void_p(None)
        prm = _params(p, eps, d, precision, kernel, kappa, box_halfwidth)
        call("kifmm_m2l_precompute", ctypes.byref(prm), ctypes.byref(self._h))
        r, rp, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        call("kifmm_m2l_plan_rank", self._h, ctypes.byref(r), ctypes.byref(rp), ctypes.byref(n))
        self.r, self.r_pad, self.n = r.value, rp.value, n.value
        self._levels = {}

    # -- lifetime -------------------------------------------------------
    def close(self) -> None:
        if self._h:
            lib().kifmm_m2l_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- levels ---------------------------------------------------------
    def set_level(self, level: int, box_ijk, root_halfwidth: float, instance: int = 0) -> int:
        """Register the boxes of one level; returns the number of M2L pairs."""
        box = np.ascontiguousarray(box_ijk, dtype=np.int32).reshape(-1, 3)
        call("kifmm_m2l_set_level", self._h, int(instance), int(level), float(root_halfwidth), box.shape[0],
             box.ctypes.data)
        cnt = ctypes.c_int64(0)
        call("kifmm_m2l_level_pairs", self._h, int(instance), int(level), ctypes.byref(cnt))
        self._levels[(instance, level)] = box.shape[0]
        return cnt.value

    def n_boxes(self, level: int, instance: int = 0) -> int:
        return self._levels[(instance, level)]

    # -- translation ----------------------------------------------------
    def _run(self, fname, x, level, instance, out, beta, stream):
        import torch

        if (instance, level) not in self._levels:
            cnt = ctypes.c_int64(0)  # the library reports the unregistered level
            call("kifmm_m2l_level_pairs", self._h, int(instance), int(level), ctypes.byref(cnt))
        nb = self._levels[(instance, level)]
        squeeze = x.dim() == 2
        nrhs = 1 if squeeze else x.shape[1]
        shape = (nb, self.n) if squeeze else (nb, nrhs, self.n)
        _check_tensor(x, "input", shape)
        if out is None:
            out = torch.empty(shape, device=x.device, dtype=torch.float32)
            beta = 0.0
        _check_tensor(out, "out", shape)
        call(fname, self._h, int(instance), int(level), int(nrhs), ctypes.c_void_p(x.data_ptr()),
             ctypes.c_void_p(out.data_ptr()), float(beta), _stream_handle(stream))
        return out

    def apply(self, q_up, level: int, instance: int = 0, out=None, beta: float = 0.0, stream=None):
        """Compressed M2L: out = beta*out + U~ s_l sum K~ R~^T q_up."""
        return self._run("kifmm_m2l_apply", q_up, level, instance, out, beta, stream)

    def apply_adjoint(self, pbar, level: int, instance: int = 0, out=None, beta: float = 0.0, stream=None):
        """Transpose of ``apply``: out = beta*out + R~ s_l sum K~^T U~^T pbar."""
        return self._run("kifmm_m2l_apply_adjoint", pbar, level, instance, out, beta, stream)

    def apply_levels(self, x_all, level_lo: int, level_hi: int, instance: int = 0, out=None, beta: float = 0.0,
                     stream=None, adjoint: bool = False):
        """Levels level_lo..level_hi in one batch; x_all / out hold the
        levels' [n_boxes, nrhs, n] (or [n_boxes, n]) arrays back to back."""
        import torch

        for l in range(level_lo, level_hi + 1):
            if (instance, l) not in self._levels:
                cnt = ctypes.c_int64(0)
                call("kifmm_m2l_level_pairs", self._h, int(instance), int(l), ctypes.byref(cnt))
        nb = sum(self._levels[(instance, l)] for l in range(level_lo, level_hi + 1))
        squeeze = x_all.dim() == 2
        nrhs = 1 if squeeze else x_all.shape[1]
        shape = (nb, self.n) if squeeze else (nb, nrhs, self.n)
        _check_tensor(x_all, "input", shape)
        if out is None:
            out = torch.empty(shape, device=x_all.device, dtype=torch.float32)
            beta = 0.0
        _check_tensor(out, "out", shape)
        fname = "kifmm_m2l_apply_levels_adjoint" if adjoint else "kifmm_m2l_apply_levels"
        call(fname, self._h, int(instance), int(level_lo), int(level_hi), int(nrhs),
             ctypes.c_void_p(x_all.data_ptr()), ctypes.c_void_p(out.data_ptr()), float(beta),
             _stream_handle(stream))
        return out

    def apply_levels_host(self, x_all, level_lo: int, level_hi: int, out, instance: int = 0, beta: float = 0.0,
                          stream=None):
        """apply_levels on HOST float32 tensors (pin them for overlapped
        copies): the library copies the rows in and the results out in
        chunks that overlap the compression and the expansion, all ordered
        on `stream`."""
        import torch

        nb = sum(self._levels[(instance, l)] for l in range(level_lo, level_hi + 1))
        nrhs = 1 if x_all.dim() == 2 else x_all.shape[1]
        shape = (nb, self.n) if x_all.dim() == 2 else (nb, nrhs, self.n)
        for t, name in ((x_all, "input"), (out, "out")):
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float32:
                raise TypeError(f"{name} must be a host float32 tensor")
            if not t.is_contiguous() or tuple(t.shape) != tuple(shape):
                raise ValueError(f"{name} must be contiguous with shape {tuple(shape)}")
        call("kifmm_m2l_apply_levels_host", self._h, int(instance), int(level_lo), int(level_hi), int(nrhs),
             ctypes.c_void_p(x_all.data_ptr()), ctypes.c_void_p(out.data_ptr()), float(beta), _stream_handle(stream))
        return out

    def apply_dense(self, q_up, level: int, instance: int = 0, out=None, beta: float = 0.0, stream=None):
        """Uncompressed FP32 M2L (the baseline)."""
        return self._run("kifmm_m2l_apply_dense", q_up, level, instance, out, beta, stream)

    def apply_dense_tc(self, q_up, level: int, instance: int = 0, out=None, beta: float = 0.0, stream=None):
        """Uncompressed M2L on the tensor cores in f16x3 arithmetic (the baseline at equal accuracy)."""
        return self._run("kifmm_m2l_apply_dense_tc", q_up, level, instance, out, beta, stream)

    def profile(self, enable: bool = True) -> None:
        """Turn per-stage CUDA-event tracing on or off."""
        call("kifmm_m2l_profile_enable", self._h, 1 if enable else 0)

    def profile_read(self):
        """Stage times since the last read: ({'compress','core','expand': ms}, launches)."""
        ms = (ctypes.c_double * 3)()
        n = ctypes.c_int64(0)
        call("kifmm_m2l_profile_read", self._h, ms, ctypes.byref(n))
        return {"compress": ms[0], "core": ms[1], "expand": ms[2]}, n.value

    def autotune(self, x_all, level_lo: int, level_hi: int, instance: int = 0, reps: int = 5, out=None,
                 stream=None) -> dict:
        """Pick the core launch's work assignment on this workload (see
        kifmm_m2l_autotune); ``out`` receives the M2L of ``x_all``."""
        import torch

        for l in range(level_lo, level_hi + 1):
            if (instance, l) not in self._levels:
                cnt = ctypes.c_int64(0)
                call("kifmm_m2l_level_pairs", self._h, int(instance), int(l), ctypes.byref(cnt))
        nb = sum(self._levels[(instance, l)] for l in range(level_lo, level_hi + 1))
        nrhs = 1 if x_all.dim() == 2 else x_all.shape[1]
        shape = (nb, self.n) if x_all.dim() == 2 else (nb, nrhs, self.n)
        _check_tensor(x_all, "input", shape)
        if out is None:
            out = torch.empty(shape, device=x_all.device, dtype=torch.float32)
        _check_tensor(out, "out", shape)
        res = _lib.TuneResult()
        call("kifmm_m2l_autotune", self._h, int(instance), int(level_lo), int(level_hi), int(nrhs),
             ctypes.c_void_p(x_all.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(reps), ctypes.byref(res),
             _stream_handle(stream))
        return {"n_chunk": res.n_chunk, "contiguous": res.contiguous, "variant": res.variant,
                "core_ms": res.core_ms, "from_cache": bool(res.from_cache)}

    def set_stage2(self, c2: float) -> None:
        """Per-offset low-rank cores (Sec. 3.2) with eps2 = c2 * eps / r;
        c2 <= 0 switches them off (see kifmm_m2l_set_stage2)."""
        call("kifmm_m2l_set_stage2", self._h, float(c2))

    def stage2_ranks(self):
        """The 316 per-offset ranks k_o of stage 2 (numpy int32)."""
        import numpy as np

        k = np.zeros(316, np.int32)
        call("kifmm_m2l_stage2_ranks", self._h, k.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return k

    def sync(self, stream=None) -> None:
        """Synchronise the stream and raise on device-side failures."""
        call("kifmm_m2l_sync", self._h, _stream_handle(stream))

    def set_wait_limit(self, ns: int = 0) -> None:
        """Bound of the core kernels' device waits in ns from the next apply on (0: the default 2 s)."""
        call("kifmm_m2l_set_wait_limit", self._h, int(ns))


def apply_batch(items, use_graph: bool = False, stream=None):
    """Compressed M2L of many instances in one batch.

    ``items``: sequence of dicts with keys plan (M2LPlan), level_lo, level_hi,
    x (CUDA float32 [boxes, nrhs, n] or [boxes, n], levels back to back),
    out (same shape), and optional instance (0) and beta (0.0).
    """
    arr = (_lib.BatchItem * len(items))()
    for i, it in enumerate(items):
        plan, x, out = it["plan"], it["x"], it["out"]
        inst, lo, hi = it.get("instance", 0), it["level_lo"], it["level_hi"]
        nb = sum(plan._levels[(inst, l)] for l in range(lo, hi + 1))
        nrhs = 1 if x.dim() == 2 else x.shape[1]
        shape = (nb, plan.n) if x.dim() == 2 else (nb, nrhs, plan.n)
        _check_tensor(x, "x", shape)
        _check_tensor(out, "out", shape)
        arr[i] = _lib.BatchItem(plan._h.value, inst, lo, hi, nrhs, x.data_ptr(), out.data_ptr(),
                                float(it.get("beta", 0.0)))
    call("kifmm_m2l_apply_batch", len(items), arr, 1 if use_graph else 0, _stream_handle(stream))
