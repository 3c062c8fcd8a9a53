"""Potential of a point cloud on itself through the compressed KIFMM.

Binding of the ``kifmm_fmm_*`` entry points (include/kifmm_m2l.h): the
complete algorithm of Sec. 4 for point sources, p_i = sum_{j != i}
G(x_i, x_j) q_j (Eq. (1)), with the near field summed directly and the
far field through S~, M~, the compressed M2L, L~ and T~ (Sec. 3.3).  Every
step runs in the library's kernels; this module only marshals arguments.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import call, lib
from .m2l import M2LPlan, _params, _stream_handle

NEAR, FAR, ALL = 1, 2, 3


def pass_ops_host(p: int, eps: float, d: float = 0.1, rcond: float = 1e-9):
    """The library's FP64 pass operators (kept, Ws [r, n], Mt [8, r, r])."""
    from .m2l import factors_host

    _, U, _ = factors_host(p, eps, d)
    n, r = U.shape
    prm = _params(p, eps, d, "fp32")
    kept = ctypes.c_int(0)
    Ws = np.empty((r, n))
    Mt = np.empty((8, r, r))
    call("kifmm_m2l_pass_ops_host", ctypes.byref(prm), float(rcond), ctypes.byref(kept), Ws.ctypes.data,
         Mt.ctypes.data)
    return kept.value, Ws, Mt


class PointFMM:
    """The octree of one point cloud bound to an ``M2LPlan`` (tensor-core
    precision).  ``points``: float64 [N, 3]; ``depth``: leaf level; the root
    cube is (centre, r0) when given, else the padded bounding cube.
    ``normals`` (float64 [N, 3]) makes the sources dipoles: the double-layer
    potential sum_j dG(x_i, x_j)/dn(x_j) q_j (Sec. 4, Eq. (26))."""

    def __init__(self, plan: M2LPlan, points, depth: int, centre=None, r0: float | None = None, normals=None):
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        self.plan = plan
        self.n_points = pts.shape[0]
        self._h = ctypes.c_void_p(None)
        c = None
        if r0 is not None and r0 > 0:
            c = np.ascontiguousarray(centre, dtype=np.float64).reshape(3)
        call("kifmm_fmm_create", plan._h, self.n_points, pts.ctypes.data,
             int(depth), None if c is None else c.ctypes.data, float(r0 or 0.0), ctypes.byref(self._h))
        self.double_layer = False
        if normals is not None:
            self.set_normals(normals)

    def set_normals(self, normals) -> None:
        """Dipole sources with these normals (float64 [N, 3]); None: point charges."""
        if normals is None:
            call("kifmm_fmm_set_normals", self._h, None)
            self.double_layer = False
            return
        nrm = np.ascontiguousarray(normals, dtype=np.float64).reshape(-1, 3)
        if nrm.shape[0] != self.n_points:
            raise ValueError(f"normals has {nrm.shape[0]} rows, expected {self.n_points}")
        call("kifmm_fmm_set_normals", self._h, nrm.ctypes.data)
        self.double_layer = True

    def close(self) -> None:
        if self._h:
            lib().kifmm_fmm_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        depth = ctypes.c_int(0)
        vals = [ctypes.c_int64(0) for _ in range(4)]
        call("kifmm_fmm_info", self._h, ctypes.byref(depth), *[ctypes.byref(v) for v in vals])
        return {"depth": depth.value, "leaves": vals[0].value, "boxes": vals[1].value,
                "m2l_pairs": vals[2].value, "near_pairs": vals[3].value}

    def evaluate(self, q, parts: int = ALL, out=None, stream=None):
        """Potential at every point from the densities q (CUDA float32 [N])."""
        import torch

        if not isinstance(q, torch.Tensor) or not q.is_cuda or q.dtype != torch.float32:
            raise TypeError("q must be a CUDA float32 tensor")
        q = q.contiguous()
        if q.numel() != self.n_points:
            raise ValueError(f"q has {q.numel()} entries, expected {self.n_points}")
        if out is None:
            out = torch.empty_like(q)
        call("kifmm_fmm_evaluate", self._h, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(out.data_ptr()),
             int(parts), _stream_handle(stream))
        return out


def _autograd():
    import torch

    class FMMPotential(torch.autograd.Function):
        """p = A q with A the evaluated potential operator.  A is symmetric
        (T = S^T and L = M^T on the swapped surfaces of Sec. 2.1, K_o^T =
        K_{-o}, and G symmetric), so the gradient is A applied to the
        incoming gradient."""

        @staticmethod
        def forward(ctx, q, fmm, parts):
            ctx.fmm, ctx.parts = fmm, parts
            return fmm.evaluate(q.detach(), parts)

        @staticmethod
        def backward(ctx, g):
            if ctx.fmm.double_layer:
                raise NotImplementedError("the double-layer evaluation is not symmetric: its adjoint is not built")
            return ctx.fmm.evaluate(g.contiguous(), ctx.parts), None, None

    return FMMPotential


_FMMPotential = None


def fmm_potential(fmm: PointFMM, q, parts: int = ALL):
    """Differentiable ``fmm.evaluate(q)`` with respect to q."""
    global _FMMPotential
    if _FMMPotential is None:
        _FMMPotential = _autograd()
    return _FMMPotential.apply(q, fmm, parts)
