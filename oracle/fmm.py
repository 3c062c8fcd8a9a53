"""Complete SVD-KIFMM potential evaluation for point sources, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The potential at every point of a cloud from every other point (Eq. (1))
is split as in Sec. 2.2 and the complete algorithm of Sec. 4: the near field
by direct summation (S2T) and the far field by S2M, M2M, M2L, L2L, L2T
(Eqs. (2) .. (6), composed as Eq. (7)).  Sec. 3.3 compresses the
upward and downward passes with the M2L bases: S~ = R~^T S, M~ = R~^T M R~,
L~ = U~^T L U~, T~ = T U~, and the M2L then maps q~ to p~ with the cores
K~_o alone.  Both forms are here: ``fmm_uncompressed`` forms every operator
from the surfaces at the box's own size, ``fmm_compressed`` follows Sec. 3.3.

Readings (the paper names the translating matrices without giving their form;
these are the KIFMM ones it cites):
* S, M: the upward check potentials (surface x^u, half-width (3-2d)h) are
  matched by equivalent densities on y^u ((1+d)h) through the truncated
  pseudo-inverse of K(x^u, y^u) (``upward.check_to_equivalent``).
* The pseudo-inverses drop singular values below ``FMM_RCOND`` = 1e-9 of
  the largest.  The paper states no cutoff; this one keeps the FP64 error
  of the whole evaluation at its 1e-12 value (p = 6) or lower (p = 8: 6.6e-8
  against 8.4e-8 on 3000 points in the unit cube) while bounding |S~| and
  |T~| entries by 3e6 at p = 8 (5e7 with 1e-12), which keeps an FP32
  evaluation of them within 3.2e-7 of FP64.
* L: the parent's downward check potentials (x^d, (1+d)h) give its downward
  equivalent densities on y^d ((3-2d)h) through the pseudo-inverse of
  K(x^d, y^d); these densities produce the child's downward check
  potentials.
* T: a leaf's downward equivalent densities, found the same way, produce the
  potentials at the leaf's points.
* The near field of a leaf is every leaf sharing at least one vertex with it,
  itself included (Sec. 2.1); a point does not act on itself.
* Double layer (Sec. 4, Eq. (26)): with normals n(y_j) given, the
  sources are dipoles of density q_j, and G is replaced by dG/dn(y) in S2T
  and in the leaf check potentials (the first step of S2M); the equivalent
  densities and every later step stay single layer.
* All leaves lie at the tree's depth.  Levels 0 and 1 have empty interaction
  lists, so M2L runs on levels 2..depth and L2L starts from level 2.
* Octant of a child: c = 4 (i & 1) + 2 (j & 1) + (k & 1) from its integer
  box coordinates; its centre lies at (2 (ijk & 1) - 1) h_child from the
  parent's.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import geometry as geo
from . import m2l as m2l_mod
from .upward import check_to_equivalent

FMM_RCOND = 1e-9


# ---------------------------------------------------------------------------
# translating matrices (Sec. 2.2)
# ---------------------------------------------------------------------------
def downward_check_to_equivalent(p: int, d: float, h: float, rcond: float = FMM_RCOND) -> np.ndarray:
    """Truncated-SVD pseudo-inverse of K(x^d, y^d) for a box of half-width h.
    Sec. 2.2 (L and T of the downward pass) on the surfaces of Sec. 2.1."""
    x = geo.surface_points(p, np.zeros(3), (1.0 + d) * h)
    y = geo.surface_points(p, np.zeros(3), (3.0 - 2.0 * d) * h)
    return np.linalg.pinv(geo.laplace_kernel(x, y), rcond=rcond)


def child_signs() -> np.ndarray:
    """[8, 3] signs (2 b - 1) of the octant c = 4 b_x + 2 b_y + b_z. Sec. 2.1 (children of an octree box)."""
    return np.array([[2 * ((c >> 2) & 1) - 1, 2 * ((c >> 1) & 1) - 1, 2 * (c & 1) - 1]
                     for c in range(8)], dtype=np.float64)


def octant(ijk: np.ndarray) -> np.ndarray:
    """Octant index of boxes within their parents, from integer coordinates. Sec. 2.1 (children of an octree box)."""
    ijk = np.asarray(ijk, dtype=np.int64)
    return 4 * (ijk[:, 0] & 1) + 2 * (ijk[:, 1] & 1) + (ijk[:, 2] & 1)


def m2m_matrix(p: int, d: float, hp: float, c: int, rcond: float = FMM_RCOND) -> np.ndarray:
    """M for the child in octant c of a parent of half-width hp (Eq. (3)):
    child upward equivalent densities -> parent upward equivalent densities."""
    hc = 0.5 * hp
    x = geo.surface_points(p, np.zeros(3), (3.0 - 2.0 * d) * hp)
    y = geo.surface_points(p, child_signs()[c] * hc, (1.0 + d) * hc)
    return check_to_equivalent(p, d, hp, rcond) @ geo.laplace_kernel(x, y)


def l2l_matrix(p: int, d: float, hp: float, c: int, rcond: float = FMM_RCOND) -> np.ndarray:
    """L for the child in octant c of a parent of half-width hp (Eq. (5)):
    parent downward check potentials -> child downward check potentials."""
    hc = 0.5 * hp
    x = geo.surface_points(p, child_signs()[c] * hc, (1.0 + d) * hc)
    y = geo.surface_points(p, np.zeros(3), (3.0 - 2.0 * d) * hp)
    return geo.laplace_kernel(x, y) @ downward_check_to_equivalent(p, d, hp, rcond)


# ---------------------------------------------------------------------------
# compressed pass operators (Sec. 3.3)
# ---------------------------------------------------------------------------
@dataclass
class PassOperators:
    """Sec. 3.3's operators at unit (parent) half-width.

    Ws [r, n]     R~^T E_u(1): S~ of a leaf of half-width h is h Ws K(x^u, points)
    Mt [8, r, r]  R~^T M_c R~
    Lt [8, r, r]  U~^T L_c U~
    Wt [n, r]     E_d(1) U~: T~ of a leaf of half-width h is h K(points, y^d) Wt
    E_u(h) = h E_u(1) and E_d(h) = h E_d(1) because G is homogeneous of
    degree -1; M_c and L_c do not depend on the size.
    """

    Ws: np.ndarray
    Mt: np.ndarray
    Lt: np.ndarray
    Wt: np.ndarray


def pass_operators(f: m2l_mod.SvdFactors, p: int, d: float, rcond: float = FMM_RCOND) -> PassOperators:
    """S~, M~, L~, T~ of Sec. 3.3 from the M2L bases R~ (f.R) and U~ (f.U)."""
    Ws = f.R.T @ check_to_equivalent(p, d, 1.0, rcond)
    Wt = downward_check_to_equivalent(p, d, 1.0, rcond) @ f.U
    Mt = np.stack([f.R.T @ m2m_matrix(p, d, 1.0, c, rcond) @ f.R for c in range(8)])
    Lt = np.stack([f.U.T @ l2l_matrix(p, d, 1.0, c, rcond) @ f.U for c in range(8)])
    return PassOperators(Ws=Ws, Mt=Mt, Lt=Lt, Wt=Wt)


# ---------------------------------------------------------------------------
# tree helpers
# ---------------------------------------------------------------------------
def leaf_points(tree):
    """(order, bounds): points of leaf b are order[bounds[b]:bounds[b+1]]. Sec. 2.1 (leaves of the octree)."""
    nb = tree.levels[tree.depth].shape[0]
    order = np.argsort(tree.leaf_of_point, kind="stable")
    bounds = np.searchsorted(tree.leaf_of_point[order], np.arange(nb + 1))
    return order, bounds


def parent_rows(tree, level: int) -> np.ndarray:
    """Row of each level-``level`` box's parent in ``tree.levels[level - 1]``. Sec. 2.1 (parent of an octree box)."""
    par = {tuple(b): i for i, b in enumerate(tree.levels[level - 1].astype(np.int64))}
    return np.array([par[tuple(b)] for b in (tree.levels[level].astype(np.int64) >> 1)], dtype=np.int64)


def near_leaves(tree, b: int) -> np.ndarray:
    """Leaves sharing at least one vertex with leaf b, b included (Sec. 2.1)."""
    ijk = tree.levels[tree.depth].astype(np.int64)
    return np.nonzero(np.max(np.abs(ijk - ijk[b][None, :]), axis=1) <= 1)[0]


# ---------------------------------------------------------------------------
# direct summation and near field (Eq. (1))
# ---------------------------------------------------------------------------
def source_kernel(x, pts, src, normals=None) -> np.ndarray:
    """Kernel from the sources pts[src] to the points x: G, or dG/dn(y) with
    the sources' normals for a double layer. Eq. (1)'s kernel; the double layer of Sec. 4, Eq. (26)."""
    if normals is None:
        return geo.laplace_kernel(x, pts[src])
    return geo.laplace_double_layer_kernel(x, pts[src], np.asarray(normals, dtype=np.float64)[src])


def direct_sum(points, q, targets=None, normals=None) -> np.ndarray:
    """p_i = sum_{j != i} G(x_i, x_j) q_j for the listed targets (all by
    default); with ``normals``, dG(x_i, x_j)/dn(x_j) in place of G. Eq. (1)."""
    pts = np.asarray(points, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    idx = np.arange(pts.shape[0]) if targets is None else np.asarray(targets)
    out = np.zeros(idx.size)
    every = np.arange(pts.shape[0])
    for c0 in range(0, idx.size, 256):
        t = idx[c0:c0 + 256]
        k = source_kernel(pts[t], pts, every, normals)
        k[np.arange(t.size), t] = 0.0
        out[c0:c0 + 256] = k @ q
    return out


def near_field(tree, points, q, normals=None) -> np.ndarray:
    """S2T: potential at every point from the points of its leaf's near field.
    Sec. 2.2 (S2T) over the near field of Sec. 2.1."""
    pts = np.asarray(points, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    order, bounds = leaf_points(tree)
    out = np.zeros(pts.shape[0])
    for b in range(bounds.size - 1):
        tgt = order[bounds[b]:bounds[b + 1]]
        if tgt.size == 0:
            continue
        src = np.concatenate([order[bounds[s]:bounds[s + 1]] for s in near_leaves(tree, b)])
        k = source_kernel(pts[tgt], pts, src, normals)
        k[tgt[:, None] == src[None, :]] = 0.0
        out[tgt] = k @ q[src]
    return out


# ---------------------------------------------------------------------------
# uncompressed far field (Eqs. (2) .. (6))
# ---------------------------------------------------------------------------
def _upward(tree, points, p, d, q, rcond, normals=None):
    """Upward equivalent densities of levels 2..depth (S2M, M2M), every
    operator formed at the box's own half-width. Eqs. (2), (3)."""
    pts = np.asarray(points, dtype=np.float64)
    L = tree.depth
    order, bounds = leaf_points(tree)
    h = tree.halfwidth(L)
    centres = tree.box_centres(L)
    E = check_to_equivalent(p, d, h, rcond)
    qu = {L: np.zeros((centres.shape[0], geo.unit_surface(p).shape[0]))}
    for b in range(centres.shape[0]):
        idx = order[bounds[b]:bounds[b + 1]]
        x = geo.surface_points(p, centres[b], (3.0 - 2.0 * d) * h)
        qu[L][b] = E @ (source_kernel(x, pts, idx, normals) @ q[idx])
    for level in range(L - 1, 1, -1):
        hp = tree.halfwidth(level)
        M = [m2m_matrix(p, d, hp, c, rcond) for c in range(8)]
        par = parent_rows(tree, level + 1)
        oc = octant(tree.levels[level + 1])
        qu[level] = np.zeros((tree.levels[level].shape[0], qu[L].shape[1]))
        for c in range(tree.levels[level + 1].shape[0]):
            qu[level][par[c]] += M[oc[c]] @ qu[level + 1][c]
    return qu


def fmm_uncompressed_far(tree, points, p: int, d: float, q, rcond: float = FMM_RCOND, normals=None) -> np.ndarray:
    """Far-field potential at every point: T L K M S q (Eq. (7)) summed
    over the levels, each translating matrix formed at its box size."""
    pts = np.asarray(points, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    L = tree.depth
    qu = _upward(tree, pts, p, d, q, rcond, normals)
    pd = {}
    for level in range(2, L + 1):
        pd[level] = m2l_mod.m2l_dense(tree.levels[level], level, tree.r0, p, d, qu[level],
                                      centre=tree.centre)
        if level > 2:
            hp = tree.halfwidth(level - 1)
            Lm = [l2l_matrix(p, d, hp, c, rcond) for c in range(8)]
            par = parent_rows(tree, level)
            oc = octant(tree.levels[level])
            for e in range(tree.levels[level].shape[0]):
                pd[level][e] += Lm[oc[e]] @ pd[level - 1][par[e]]
    h = tree.halfwidth(L)
    centres = tree.box_centres(L)
    E = downward_check_to_equivalent(p, d, h, rcond)
    order, bounds = leaf_points(tree)
    out = np.zeros(pts.shape[0])
    for b in range(centres.shape[0]):
        idx = order[bounds[b]:bounds[b + 1]]
        y = geo.surface_points(p, centres[b], (3.0 - 2.0 * d) * h)
        out[idx] = geo.laplace_kernel(pts[idx], y) @ (E @ pd[L][b])
    return out


# ---------------------------------------------------------------------------
# compressed far field (Sec. 3.3)
# ---------------------------------------------------------------------------
def leaf_check_potentials(tree, points, p: int, d: float, q, normals=None) -> np.ndarray:
    """K(x^u, points in the leaf) q for every leaf, [B_depth, n]: the part of
    S that depends on the points (double-layer kernel with ``normals``).
    Eq. (2) (its first step); the double layer of Eq. (26)."""
    pts = np.asarray(points, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    L = tree.depth
    order, bounds = leaf_points(tree)
    h = tree.halfwidth(L)
    centres = tree.box_centres(L)
    out = np.zeros((centres.shape[0], geo.unit_surface(p).shape[0]))
    for b in range(centres.shape[0]):
        idx = order[bounds[b]:bounds[b + 1]]
        x = geo.surface_points(p, centres[b], (3.0 - 2.0 * d) * h)
        out[b] = source_kernel(x, pts, idx, normals) @ q[idx]
    return out


def compressed_upward(tree, points, f, ops: PassOperators, p: int, d: float, q, normals=None) -> dict:
    """q~ of levels 2..depth: q~ = S~ q at the leaves, q~_C = sum_c M~_c q~_c. Sec. 3.3 (S~ and M~)."""
    L = tree.depth
    qt = {L: tree.halfwidth(L) * leaf_check_potentials(tree, points, p, d, q, normals) @ ops.Ws.T}
    for level in range(L - 1, 1, -1):
        par = parent_rows(tree, level + 1)
        oc = octant(tree.levels[level + 1])
        qt[level] = np.zeros((tree.levels[level].shape[0], f.r))
        for c in range(tree.levels[level + 1].shape[0]):
            qt[level][par[c]] += ops.Mt[oc[c]] @ qt[level + 1][c]
    return qt


def compressed_m2l(box_ijk, level: int, r0: float, f, qt) -> np.ndarray:
    """p~^t = (r0/2**l)^(-1) sum_{s in I^t} K~_{t-s} q~^s (Eq. (14) between
    the compressed vectors)."""
    tg, sr, ok = geo.interaction_lists(box_ijk)
    pt = np.zeros((np.asarray(box_ijk).shape[0], f.r))
    for k in np.unique(ok):
        sel = ok == k
        pt[tg[sel]] += qt[sr[sel]] @ f.C[k].T
    return m2l_mod.level_scale(level, r0) * pt


def compressed_downward(tree, f, ops: PassOperators, qt: dict) -> dict:
    """p~ of levels 2..depth: M2L of each level plus p~_E += L~_c p~_parent. Sec. 3.3 (the compressed M2L and L~)."""
    L = tree.depth
    pt = {}
    for level in range(2, L + 1):
        pt[level] = compressed_m2l(tree.levels[level], level, tree.r0, f, qt[level])
        if level > 2:
            par = parent_rows(tree, level)
            oc = octant(tree.levels[level])
            for e in range(tree.levels[level].shape[0]):
                pt[level][e] += ops.Lt[oc[e]] @ pt[level - 1][par[e]]
    return pt


def leaf_l2t(tree, points, p: int, d: float, e_leaf) -> np.ndarray:
    """Potential at every point from its leaf's downward equivalent densities
    e_leaf [B_depth, n] placed on y^d. Eq. (6) (Sec. 2.2)."""
    pts = np.asarray(points, dtype=np.float64)
    L = tree.depth
    h = tree.halfwidth(L)
    centres = tree.box_centres(L)
    order, bounds = leaf_points(tree)
    out = np.zeros(pts.shape[0])
    for b in range(centres.shape[0]):
        idx = order[bounds[b]:bounds[b + 1]]
        y = geo.surface_points(p, centres[b], (3.0 - 2.0 * d) * h)
        out[idx] = geo.laplace_kernel(pts[idx], y) @ e_leaf[b]
    return out


def fmm_compressed_far(tree, points, f, ops: PassOperators, p: int, d: float, q, normals=None) -> np.ndarray:
    """Far-field potential with Sec. 3.3's operators: T~ L~ K~ M~ S~ q."""
    qt = compressed_upward(tree, points, f, ops, p, d, q, normals)
    pt = compressed_downward(tree, f, ops, qt)
    L = tree.depth
    e_leaf = tree.halfwidth(L) * pt[L] @ ops.Wt.T
    return leaf_l2t(tree, points, p, d, e_leaf)


def fmm_potential(tree, points, q, p: int, d: float, f=None, ops: PassOperators | None = None,
                  rcond: float = FMM_RCOND, normals=None) -> np.ndarray:
    """Near field plus far field; compressed (Sec. 3.3) when ``f`` is given;
    a double layer with ``normals``."""
    if f is None:
        far = fmm_uncompressed_far(tree, points, p, d, q, rcond, normals)
    else:
        if ops is None:
            ops = pass_operators(f, p, d, rcond)
        far = fmm_compressed_far(tree, points, f, ops, p, d, q, normals)
    return near_field(tree, points, q, normals) + far
