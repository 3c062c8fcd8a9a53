"""GB300-native SVD-compressed KIFMM M2L translation (arXiv 1211.2517).

The translation p^{t,d} = U~ s_l sum_{s in I^t} K~_{t-s} R~^T q^{s,u} runs
in hand-written sm_103a kernels behind the C ABI of include/kifmm_m2l.h
(libkifmm_m2l.so, built in-tree by ``paper_1211_2517_gb300.build``).
``PointFMM`` evaluates the potential of a point cloud with the complete
algorithm and the compressed upward / downward passes (Sec. 3.3), for point
charges or dipoles (the double layer of Sec. 4).  ``M2LPlan(...,
kernel="yukawa", kappa=, box_halfwidth=)`` holds the operators of one level
of the non-homogeneous Yukawa kernel (Sec. 3.1's per-level precompute).
"""
from ._lib import EXPORTED, KifmmError, lib  # noqa: F401
from .m2l import M2LPlan, apply_batch, factors_host, pairs_host, stage2_host, surface_count  # noqa: F401
from .fmm import PointFMM, fmm_potential, pass_ops_host  # noqa: F401

__all__ = ["M2LPlan", "apply_batch", "factors_host", "pairs_host", "stage2_host", "surface_count", "KifmmError", "lib",
           "EXPORTED", "PointFMM", "fmm_potential", "pass_ops_host"]
