"""FP64 CPU oracle of the SVD-compressed KIFMM M2L translation (arXiv 1211.2517).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (``paper_1211_2517_gb300``) never imports,
links or executes anything here, and this package never imports the product.
The two share only the seeded input generators of ``synth``.

The oracle is plain NumPy in float64: slow, unblocked, written to be read
against the paper.  Each function cites the section / equation it follows.

Modules:
  geometry  -- surfaces (Sec. 2.1), the 316 offsets (Sec. 3.1), interaction
               lists (Sec. 2.1), the Laplace kernel and its double-layer
               normal derivative (Sec. 4), the Yukawa kernel.
  m2l       -- dense M2L (Eq. (4)), the fat/thin SVDs and the truncated
               compressed M2L (Eqs. (8), (10), (11), (13), (14)),
               level scaling by homogeneity (Sec. 3.1) or per-level factors
               for a non-homogeneous kernel, the adjoint, the stage-2
               per-offset low-rank factors (Eq. (17)).
  upward    -- S2M / M2M (Eqs. (2), (3)) to make realistic M2L inputs,
               and direct summation (Eq. (1)) for brute-force checks.
  fmm       -- the complete evaluation for point sources: near field (S2T),
               far field through S2M, M2M, M2L, L2L, L2T (Eqs. (2) ..
               (7)), uncompressed and with Sec. 3.3's compressed
               operators S~, M~, L~, T~; direct summation; dipole sources
               (the double layer of Sec. 4).

Every function here is pinned by a ``-m "not gpu"`` test against a closed
form, an invariant, a bound or brute force; none is "parity unpinned".
"""
from . import fmm, geometry, m2l, upward  # noqa: F401
