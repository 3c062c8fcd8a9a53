"""Geometry of the KIFMM translation: surfaces, offsets, interaction lists.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import itertools

import numpy as np

FOUR_PI = 4.0 * np.pi


def laplace_kernel(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """G(x, y) = 1 / (4 pi |x - y|), the single-layer Laplace kernel (Sec. 4).

    ``x`` [m,3], ``y`` [n,3] -> [m,n] float64.
    """
    diff = x[:, None, :] - y[None, :, :]
    with np.errstate(divide="ignore"):
        return 1.0 / (FOUR_PI * np.sqrt(np.einsum("mnk,mnk->mn", diff, diff)))


def yukawa_kernel(x: np.ndarray, y: np.ndarray, kappa: float) -> np.ndarray:
    """G(x, y) = exp(-kappa |x - y|) / (4 pi |x - y|), the screened Coulomb
    (Yukawa, modified Helmholtz) kernel: radial, so translation invariant
    with K^T = K for swapped surfaces, but not homogeneous (Sec. 3.1's
    O(L) case).  ``kappa = 0`` is ``laplace_kernel``.

    ``x`` [m,3], ``y`` [n,3] -> [m,n] float64.
    """
    diff = x[:, None, :] - y[None, :, :]
    r = np.sqrt(np.einsum("mnk,mnk->mn", diff, diff))
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.exp(-kappa * r) / (FOUR_PI * r)


def laplace_double_layer_kernel(x: np.ndarray, y: np.ndarray, n: np.ndarray) -> np.ndarray:
    """dG(x, y)/dn(y) = n(y) . (x - y) / (4 pi |x - y|^3): the double-layer
    kernel that replaces G in S2T and in the first step of S2M for a double
    layer integral (Sec. 4, Eq. (26)).  Gradient of G = 1/(4 pi |x - y|)
    with respect to y, projected on the normal n(y) at the source.

    ``x`` [m,3], ``y`` [k,3], ``n`` [k,3] -> [m,k] float64.
    """
    diff = x[:, None, :] - y[None, :, :]
    r2 = np.einsum("mnk,mnk->mn", diff, diff)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.einsum("mnk,nk->mn", diff, n) / (FOUR_PI * r2 * np.sqrt(r2))


def surface_grid(p: int) -> np.ndarray:
    """Integer grid points (i,j,k) in {0..p-1}^3 on the cube boundary.

    Sec. 2.1 places equivalent / check points on cube surfaces, p points per
    cube edge (Sec. 1).  Ordering: lexicographic in (i, j, k).  The count is
    p^3 - (p-2)^3 = 6(p-1)^2 + 2.
    """
    pts = [(i, j, k) for i in range(p) for j in range(p) for k in range(p)
           if min(i, j, k) == 0 or max(i, j, k) == p - 1]
    return np.array(pts, dtype=np.int64)


def unit_surface(p: int) -> np.ndarray:
    """Surface points of the cube [-1,1]^3: 2*ijk/(p-1) - 1, float64 [n,3].
    Sec. 2.1 (equivalent and check surfaces)."""
    return 2.0 * surface_grid(p) / (p - 1) - 1.0


def surface_points(p: int, centre, halfwidth: float) -> np.ndarray:
    """Points on the boundary of the cube with the given centre and half-width.
    Sec. 2.1 (equivalent and check surfaces)."""
    return np.asarray(centre, dtype=np.float64)[None, :] + halfwidth * unit_surface(p)


def m2l_offsets() -> np.ndarray:
    """The 316 relative positions o = t - s of M2L pairs (Sec. 3.1).

    A source s is in the interaction field of a target t when their parents
    are adjacent (or equal) and s, t are not adjacent (Sec. 2.1), so o lies
    in {-3..3}^3 with max|o_i| >= 2; 7^3 - 3^3 = 316.  Lexicographic order.
    """
    offs = [o for o in itertools.product(range(-3, 4), repeat=3) if max(abs(c) for c in o) >= 2]
    return np.array(offs, dtype=np.int64)


def offset_index_table() -> dict:
    """Map tuple(o) -> index into ``m2l_offsets()``. Sec. 3.1 (the 316 offsets)."""
    return {tuple(o): k for k, o in enumerate(m2l_offsets())}


def _linear_keys(ijk: np.ndarray) -> np.ndarray:
    """Injective integer key of box coordinates in [-8, 2**20)^3. Sec. 2.1 (integer box coordinates)."""
    ijk = ijk.astype(np.int64) + 8
    return (ijk[..., 0] << 42) | (ijk[..., 1] << 21) | ijk[..., 2]


def interaction_lists(box_ijk: np.ndarray):
    """Interaction field I^t = F^t minus F^parent(t) for each box (Sec. 2.1).

    ``box_ijk`` [B,3] integer coordinates of the non-empty boxes of one level.
    Near field of a box: boxes of the same level sharing at least one vertex
    (|s - t|_inf <= 1).  Far field: the rest.  A box s is in I^t when s is in
    t's far field but not in the far field of t's parent, i.e. parent(s) is
    in the near field of parent(t).  Candidates are built as the children of
    the parent's near-field boxes (27 x 8 of them, for all targets at once);
    empty boxes are skipped.

    Returns (targets, sources, offset_idx) int64 arrays, one entry per pair,
    sorted by target then offset index.
    """
    box_ijk = np.asarray(box_ijk, dtype=np.int64)
    nb = box_ijk.shape[0]
    keys = _linear_keys(box_ijk)
    order = np.argsort(keys)
    skeys = keys[order]
    otab = offset_index_table()
    par = box_ijk >> 1
    tg, sr, ok = [], [], []
    for dp in itertools.product((-1, 0, 1), repeat=3):
        for ch in itertools.product((0, 1), repeat=3):
            s_ijk = 2 * (par + np.array(dp)) + np.array(ch)          # [B, 3]
            o = box_ijk - s_ijk
            far = np.abs(o).max(axis=1) >= 2                          # not in t's near field
            pos = np.searchsorted(skeys, _linear_keys(s_ijk))
            pos = np.minimum(pos, nb - 1)
            hit = far & (skeys[pos] == _linear_keys(s_ijk))
            t_idx = np.nonzero(hit)[0]
            tg.append(t_idx)
            sr.append(order[pos[hit]])
            ok.append(np.array([otab[tuple(v)] for v in o[hit]], dtype=np.int64))
    tg, sr, ok = (np.concatenate(a) if a else np.zeros(0, np.int64) for a in (tg, sr, ok))
    srt = np.lexsort((ok, tg))
    return tg[srt], sr[srt], ok[srt]


def interaction_lists_bruteforce(box_ijk: np.ndarray):
    """O(B^2) statement of the same set: all pairs with |o|_inf >= 2 and
    |parent(t) - parent(s)|_inf <= 1.  For tiny inputs only. Sec. 2.1 (interaction field)."""
    box_ijk = np.asarray(box_ijk, dtype=np.int64)
    otab = offset_index_table()
    tg, sr, ok = [], [], []
    for t, bt in enumerate(box_ijk):
        for s, bs in enumerate(box_ijk):
            if np.max(np.abs(bt - bs)) >= 2 and np.max(np.abs((bt >> 1) - (bs >> 1))) <= 1:
                tg.append(t)
                sr.append(s)
                ok.append(otab[tuple(bt - bs)])
    tg, sr, ok = (np.array(a, dtype=np.int64) for a in (tg, sr, ok))
    order = np.lexsort((ok, tg))
    return tg[order], sr[order], ok[order]
