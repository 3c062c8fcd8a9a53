"""Upward pass (S2M, M2M) and direct summation, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The M2L translation consumes upward equivalent densities q^{s,u}.  To feed
it realistic values, this module runs the KIFMM upward pass of Sec. 2.2
(Eqs. (2), (3)) on a point cloud.  Sec. 2.1 puts the upward
equivalent surface at half-width (1+d) h and the upward check surface at
(3-2d) h.  The paper calls S and M "translating matrices" without giving
their form; the reading used here is the KIFMM one: check potentials are
matched on the upward check surface, and the equivalent densities solve
K_{check<-equiv} q = p^{check} with a truncated-SVD pseudo-inverse
(relative cutoff 1e-12).
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo

PINV_RCOND = 1e-12


def check_to_equivalent(p: int, d: float, h: float, rcond: float = PINV_RCOND) -> np.ndarray:
    """Truncated-SVD pseudo-inverse of K(x^u, y^u) for a box of half-width h
    (singular values below rcond * sigma_max dropped). Sec. 2.2 (S and M) on the surfaces of Sec. 2.1."""
    x = geo.surface_points(p, np.zeros(3), (3.0 - 2.0 * d) * h)
    y = geo.surface_points(p, np.zeros(3), (1.0 + d) * h)
    return np.linalg.pinv(geo.laplace_kernel(x, y), rcond=rcond)


def s2m(tree, points: np.ndarray, p: int, d: float, q_points: np.ndarray) -> np.ndarray:
    """Leaf upward equivalent densities q^{B,u} = S q (Eq. (2)).

    Check potentials on the leaf's upward check surface from the points
    inside the leaf, then the check-to-equivalent solve.  [B_leaf, n].
    """
    L = tree.depth
    h = tree.halfwidth(L)
    centres = tree.box_centres(L)
    pinv = check_to_equivalent(p, d, h)
    ux = geo.unit_surface(p) * (3.0 - 2.0 * d) * h
    nb = centres.shape[0]
    out = np.zeros((nb, ux.shape[0]))
    order = np.argsort(tree.leaf_of_point, kind="stable")
    bounds = np.searchsorted(tree.leaf_of_point[order], np.arange(nb + 1))
    for b in range(nb):
        idx = order[bounds[b]:bounds[b + 1]]
        if idx.size == 0:
            continue
        xc = centres[b][None, :] + ux
        pc = geo.laplace_kernel(xc, points[idx]) @ q_points[idx]
        out[b] = pinv @ pc
    return out


def m2m(tree, p: int, d: float, q_child: np.ndarray, level: int) -> np.ndarray:
    """Parent densities at ``level`` from children at level+1 (Eq. (3)).

    Check potentials on the parent's upward check surface produced by the
    children's upward equivalent densities, then the check-to-equivalent
    solve at the parent's size.
    """
    hp = tree.halfwidth(level)
    hc = tree.halfwidth(level + 1)
    pinv = check_to_equivalent(p, d, hp)
    par_ijk = tree.levels[level].astype(np.int64)
    ch_ijk = tree.levels[level + 1].astype(np.int64)
    par_index = {tuple(b): i for i, b in enumerate(par_ijk)}
    pc = np.zeros((par_ijk.shape[0], q_child.shape[1]))
    ux = geo.unit_surface(p)
    for c, cijk in enumerate(ch_ijk):
        pi = par_index[tuple(cijk >> 1)]
        # relative position of the child's centre to the parent's centre
        rel = ((2 * cijk + 1) * hc) - ((2 * par_ijk[pi] + 1) * hp)
        x = ux * (3.0 - 2.0 * d) * hp
        y = rel[None, :] + ux * (1.0 + d) * hc
        pc[pi] += geo.laplace_kernel(x, y) @ q_child[c]
    return pc @ pinv.T


def upward_pass(tree, points: np.ndarray, p: int, d: float, q_points: np.ndarray) -> dict:
    """Upward equivalent densities for every level 2..depth, {level: [B_l, n]}. Eqs. (2), (3) (Sec. 2.2)."""
    out = {tree.depth: s2m(tree, points, p, d, q_points)}
    for level in range(tree.depth - 1, 1, -1):
        out[level] = m2m(tree, p, d, out[level + 1], level)
    return out


def direct_far_field(tree, points: np.ndarray, level: int, p: int, d: float, q_points: np.ndarray,
                     targets) -> np.ndarray:
    """Brute force: potential at each target box's downward check points from
    every point in the boxes of its interaction list (Eq. (1) restricted
    to I^t).  [len(targets), n]."""
    box_ijk = tree.levels[level].astype(np.int64)
    tg, sr, _ = geo.interaction_lists(box_ijk)
    h = tree.halfwidth(level)
    centres = tree.box_centres(level)
    pts = np.asarray(points, dtype=np.float64)
    # ancestor of each point at this level
    anc = tree.levels[tree.depth][tree.leaf_of_point].astype(np.int64) >> (tree.depth - level)
    index = {tuple(b): i for i, b in enumerate(box_ijk)}
    box_of_point = np.array([index[tuple(a)] for a in anc])
    out = np.zeros((len(targets), geo.unit_surface(p).shape[0]))
    for row, t in enumerate(targets):
        srcs = sr[tg == t]
        mask = np.isin(box_of_point, srcs)
        x = geo.surface_points(p, centres[t], (1.0 + d) * h)
        out[row] = geo.laplace_kernel(x, pts[mask]) @ q_points[mask]
    return out
