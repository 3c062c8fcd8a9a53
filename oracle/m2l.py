"""Dense and SVD-compressed M2L in float64 (Secs. 2.2, 3.1, 3.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions
-----------
* Offsets o = t - s index the 316 translation matrices (``geometry.m2l_offsets``).
* M2L uses the source's upward equivalent surface y^{s,u} and the target's
  downward check surface x^{t,d}, both at half-width (1+d) h (Sec. 2.1).
* At unit half-width, K_o[i,j] = G(2 o + (1+d)(u_i - u_j)) with u the
  points of the cube [-1,1]^3 boundary.  A level-l box has half-width
  h_l = r0 / 2**l and, G being homogeneous of degree m = -1,
  K_{l,o} = (r0 / 2**l)^(-1) K_o (Sec. 3.1).
* Densities are laid out [boxes, n] (one right-hand side) or
  [boxes, nrhs, n].
* Non-homogeneous kernels (the Yukawa kernel exp(-kappa r) / (4 pi r)) have
  no such scaling: Sec. 3.1 compresses the translation matrices of every
  level separately.  ``svd_factors(..., kappa=, h=)`` forms the 316 matrices
  of boxes of half-width h from their coordinates and compresses them; the
  result carries ``h`` and the M2L of a level with that box size applies it
  with no level scale.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import geometry as geo


# ---------------------------------------------------------------------------
# translation matrices
# ---------------------------------------------------------------------------
def kernel_matrix(x, y, kappa: float = 0.0) -> np.ndarray:
    """G(x_i, y_j): Laplace, or Yukawa with screening ``kappa`` > 0.
    Sec. 4 (Laplace kernel); Sec. 3.1 (non-homogeneous case)."""
    return geo.laplace_kernel(x, y) if kappa == 0.0 else geo.yukawa_kernel(x, y, kappa)


def m2l_matrix_geometric(p: int, d: float, centre_t, centre_s, h: float, kappa: float = 0.0) -> np.ndarray:
    """K_ij = G(x_i, y_j), x on the target's downward check surface and y on
    the source's upward equivalent surface, both at half-width (1+d) h
    (Eq. (4) with the surfaces of Sec. 2.1).  Formed from coordinates."""
    x = geo.surface_points(p, centre_t, (1.0 + d) * h)
    y = geo.surface_points(p, centre_s, (1.0 + d) * h)
    return kernel_matrix(x, y, kappa)


def unit_m2l_matrices(p: int, d: float, kappa: float = 0.0, h: float = 1.0) -> np.ndarray:
    """The 316 translation matrices K_o of boxes of half-width h (unit by
    default) with centres 2 o h apart, [316, n, n]. Eq. (4); Sec. 3.1 (the 316 matrices)."""
    offs = geo.m2l_offsets()
    zero = np.zeros(3)
    return np.stack([m2l_matrix_geometric(p, d, 2.0 * h * o.astype(np.float64), zero, h, kappa)
                     for o in offs])


# ---------------------------------------------------------------------------
# stage-1 compression (Sec. 3.1)
# ---------------------------------------------------------------------------
@dataclass
class SvdFactors:
    """Truncated factors of Eq. (13) at unit half-width.

    U   [n, r]   left basis  (columns of U of the fat SVD, Eq. (10))
    R   [n, r]   right basis (columns of R of the thin SVD, Eq. (11))
    C   [316, r, r]  compressed cores  K~_o = U~^T K_o R~
    sigma        singular values of K_fat (all n)
    lam          singular values of K_thin (all n)
    r            retained rank
    """

    U: np.ndarray
    R: np.ndarray
    C: np.ndarray
    sigma: np.ndarray
    lam: np.ndarray
    r: int
    K: np.ndarray
    h: float | None = None   # box half-width of per-level factors (non-homogeneous kernels)
    kappa: float = 0.0


def truncation_rank(sigma: np.ndarray, eps: float, tie_tol: float = 1e-13) -> int:
    """Number of singular values not less than eps * sigma_0 (Sec. 3.1).

    ``eps <= 0`` keeps every singular value.  The paper does not say how to
    treat a cut through a cluster of equal singular values (the cube's
    symmetry makes many clusters).  Reading: the cut moves past the whole
    cluster, i.e. while sigma[r-1] - sigma[r] <= tie_tol * sigma_0, r grows
    by one.  Exact ties differ by ~1e-15 sigma_0 in FP64 while distinct
    values near any cut with eps >= 1e-12 differ by >= 1e-11 sigma_0.
    """
    if eps <= 0:
        return int(sigma.size)
    r = int(np.sum(sigma >= eps * sigma[0]))
    while 0 < r < sigma.size and sigma[r - 1] - sigma[r] <= tie_tol * sigma[0]:
        r += 1
    return r


def _fix_signs(m: np.ndarray) -> np.ndarray:
    """Make the largest-magnitude entry of each column positive (an arbitrary
    but deterministic choice; singular vectors are defined up to sign).
    Sec. 3.1 (singular vectors; the sign is a reading)."""
    idx = np.argmax(np.abs(m), axis=0)
    s = np.sign(m[idx, np.arange(m.shape[1])])
    s[s == 0] = 1.0
    return m * s[None, :]


def svd_factors(p: int, d: float, eps: float, r: int | None = None, kappa: float = 0.0,
                h: float | None = None) -> SvdFactors:
    """Fat and thin SVDs, truncation, compressed cores (Eqs. (8) .. (13)).

    K_fat = [K_1 ... K_316] = U Sigma [V_1^T ... V_316^T]   (Eq. (10))
    K_thin = [K_1; ...; K_316] = [Q_1; ...; Q_316] Lambda R^T  (Eq. (11))
    U~, R~ keep the columns whose singular value is >= eps * Sigma_00, and
    K~_o = U~^T K_o R~.  ``r`` overrides the rank when given.  With ``h``
    (needed for kappa > 0) the matrices are those of boxes of half-width h.
    """
    if kappa != 0.0 and h is None:
        raise ValueError("a non-homogeneous kernel needs the box half-width h")
    K = unit_m2l_matrices(p, d, kappa, 1.0 if h is None else h)
    n = K.shape[1]
    k_fat = np.concatenate(list(K), axis=1)          # n x 316n
    k_thin = np.concatenate(list(K), axis=0)         # 316n x n
    U, sigma, _ = np.linalg.svd(k_fat, full_matrices=False)
    _, lam, Rt = np.linalg.svd(k_thin, full_matrices=False)
    R = Rt.T
    if r is None:
        r = truncation_rank(sigma, eps)
    r = min(int(r), n)
    Ut = _fix_signs(U[:, :r])
    Rr = _fix_signs(R[:, :r])
    C = np.matmul(np.matmul(Ut.T[None, :, :], K), Rr[None, :, :])   # U~^T K_o R~
    return SvdFactors(U=Ut, R=Rr, C=C, sigma=sigma, lam=lam, r=r, K=K, h=h, kappa=kappa)


def level_scale(level: int, r0: float) -> float:
    """(r0 / 2**l)^m with m = -1 for the Laplace kernel (Sec. 3.1)."""
    return (1 << level) / r0


def factors_scale(f: SvdFactors, level: int, r0: float) -> float:
    """Scale that takes f's cores to boxes of this level: Sec. 3.1's
    homogeneity for unit-size factors, 1 for per-level factors (which must
    have been formed at this level's half-width)."""
    if f.h is None:
        return level_scale(level, r0)
    h = r0 / (1 << level)
    if abs(h - f.h) > 1e-12 * f.h:
        raise ValueError(f"factors formed for half-width {f.h}, level {level} has {h}")
    return 1.0


# ---------------------------------------------------------------------------
# M2L on a level of boxes
# ---------------------------------------------------------------------------
def _as3(q):
    """Layout helper; no passage of the paper."""
    q = np.asarray(q, dtype=np.float64)
    return (q[:, None, :], True) if q.ndim == 2 else (q, False)


def m2l_dense(box_ijk, level: int, r0: float, p: int, d: float, q_up, centre=None,
              targets=None, kappa: float = 0.0) -> np.ndarray:
    """Uncompressed M2L, p^{t,d} = sum_{s in I^t} K(t,s) q^{s,u} (Eq. (4)).

    Every pair's K(t,s)_ij = G(x_i^t, y_j^s) is formed from that pair's own
    surface coordinates at this level (no homogeneity shortcut); pairs are
    only batched by offset to keep NumPy busy.  q_up [B, n] or [B, nrhs, n].
    ``kappa`` > 0: the Yukawa kernel exp(-kappa r) / (4 pi r).
    ``targets`` restricts the work to those target boxes (other rows stay 0).
    """
    q, squeeze = _as3(q_up)
    box_ijk = np.asarray(box_ijk, dtype=np.int64)
    h = r0 / (1 << level)
    if centre is None:
        centre = np.zeros(3)
    centres = (np.asarray(centre) - r0)[None, :] + (2.0 * box_ijk + 1.0) * h
    u = geo.unit_surface(p) * (1.0 + d) * h
    tg, sr, ok = geo.interaction_lists(box_ijk)
    if targets is not None:
        keep = np.isin(tg, np.asarray(targets))
        tg, sr, ok = tg[keep], sr[keep], ok[keep]
    out = np.zeros_like(q)
    for k in np.unique(ok):
        sel = np.nonzero(ok == k)[0]
        for c0 in range(0, sel.size, 64):
            idx = sel[c0:c0 + 64]
            x = centres[tg[idx]][:, None, :] + u[None, :, :]          # [P, n, 3]
            y = centres[sr[idx]][:, None, :] + u[None, :, :]
            diff = x[:, :, None, :] - y[:, None, :, :]                # [P, n, n, 3]
            dist = np.sqrt(np.einsum("pijk,pijk->pij", diff, diff))
            kts = np.exp(-kappa * dist) / (geo.FOUR_PI * dist)
            out[tg[idx]] += np.einsum("pij,prj->pri", kts, q[sr[idx]])
    return out[:, 0, :] if squeeze else out


def m2l_dense_unit(box_ijk, level: int, r0: float, K: np.ndarray, q_up, lists=None) -> np.ndarray:
    """Uncompressed M2L through the unit matrices and level scaling
    (Eq. (4) with Sec. 3.1's homogeneity), grouped by offset.  `lists`
    (target, source, offset arrays of interaction_lists) may restrict the
    pairs, e.g. to a sample of the targets."""
    q, squeeze = _as3(q_up)
    tg, sr, ok = geo.interaction_lists(box_ijk) if lists is None else lists
    out = np.zeros_like(q)
    for k in np.unique(ok):
        sel = ok == k
        out[tg[sel]] += q[sr[sel]] @ K[k].T
    out *= level_scale(level, r0)
    return out[:, 0, :] if squeeze else out


def m2l_svd(box_ijk, level: int, r0: float, f: SvdFactors, q_up, lists=None) -> np.ndarray:
    """Compressed M2L, Eq. (14) restricted to the translation:

        q~^s = R~^T q^{s,u}
        p~^t = (r0/2**l)^(-1) sum_{s in I^t} K~_{t-s} q~^s
        p^{t,d} = U~ p~^t

    (no (r0/2**l)^(-1) for per-level factors of a non-homogeneous kernel).
    """
    q, squeeze = _as3(q_up)
    tg, sr, ok = lists if lists is not None else geo.interaction_lists(box_ijk)
    qt = q @ f.R                                     # [B, nrhs, r]
    pt = np.zeros(q.shape[:2] + (f.r,))
    for k in np.unique(ok):
        sel = ok == k
        pt[tg[sel]] += qt[sr[sel]] @ f.C[k].T          # K~_o q~ for every pair of offset o
    pt *= factors_scale(f, level, r0)
    out = pt @ f.U.T
    return out[:, 0, :] if squeeze else out


def m2l_svd_adjoint(box_ijk, level: int, r0: float, f: SvdFactors, pbar, lists=None) -> np.ndarray:
    """Transpose of ``m2l_svd``: q-bar^s = s_l R~ sum_{t: s in I^t} K~_{t-s}^T U~^T p-bar^t.
    The transpose of Eq. (14) (Sec. 3.1)."""
    pb, squeeze = _as3(pbar)
    tg, sr, ok = lists if lists is not None else geo.interaction_lists(box_ijk)
    pt = pb @ f.U                                    # [B, nrhs, r]
    qt = np.zeros(pb.shape[:2] + (f.r,))
    for k in np.unique(ok):
        sel = ok == k
        qt[sr[sel]] += pt[tg[sel]] @ f.C[k]            # K~_o^T p~bar
    qt *= factors_scale(f, level, r0)
    out = qt @ f.R.T
    return out[:, 0, :] if squeeze else out


def m2l_svd_targets(box_ijk, level: int, r0: float, f: SvdFactors, q_up, targets) -> np.ndarray:
    """``m2l_svd`` evaluated for a few target boxes only, one at a time.

    For sampled checks at sizes where the full oracle is too slow.
    Returns [len(targets), nrhs, n].
    Eq. (14) (Sec. 3.1)."""
    q, _ = _as3(q_up)
    box_ijk = np.asarray(box_ijk, dtype=np.int64)
    index = {tuple(b): i for i, b in enumerate(box_ijk)}
    otab = geo.offset_index_table()
    offs = geo.m2l_offsets()
    out = np.zeros((len(targets), q.shape[1], f.U.shape[0]))
    for row, t in enumerate(targets):
        bt = box_ijk[t]
        acc = np.zeros((q.shape[1], f.r))
        for o in offs:
            bs = bt - o
            s = index.get(tuple(bs))
            if s is None or np.max(np.abs((bt >> 1) - (bs >> 1))) > 1:
                continue
            acc += (q[s] @ f.R) @ f.C[otab[tuple(o)]].T
        out[row] = factors_scale(f, level, r0) * acc @ f.U.T
    return out


# ---------------------------------------------------------------------------
# stage-2 per-offset low rank (Sec. 3.2)
# ---------------------------------------------------------------------------
def stage2_factors(f: SvdFactors, eps2: float):
    """K~_o = U_o S_o Q_o^T, drop singular values < eps2 * ||K_fat||_2, and
    return (Uhat_o [r,k_o], Vhat_o = Shat_o Qhat_o^T [k_o,r]) per offset
    (Eq. (17))."""
    out = []
    thr = eps2 * f.sigma[0]
    for Ck in f.C:
        u, s, vt = np.linalg.svd(Ck)
        k = int(np.sum(s >= thr))
        out.append((u[:, :k], s[:k, None] * vt[:k]))
    return out


def m2l_svd_stage2(box_ijk, level: int, r0: float, f: SvdFactors, s2, q_up, lists=None) -> np.ndarray:
    """Compressed M2L with the second stage of Sec. 3.2 (Eq. (17)): every
    core K~_o is replaced by its truncation Uhat_o Vhat_o (``s2`` from
    ``stage2_factors``), applied as two products:

        t    = Vhat_o q~^s
        p~^t = s_l sum_{s in I^t} Uhat_o t
    """
    q, squeeze = _as3(q_up)
    tg, sr, ok = lists if lists is not None else geo.interaction_lists(box_ijk)
    qt = q @ f.R
    pt = np.zeros(q.shape[:2] + (f.r,))
    for k in np.unique(ok):
        sel = ok == k
        uh, vh = s2[k]
        pt[tg[sel]] += (qt[sr[sel]] @ vh.T) @ uh.T
    pt *= factors_scale(f, level, r0)
    out = pt @ f.U.T
    return out[:, 0, :] if squeeze else out


def m2l_svd_stage2_adjoint(box_ijk, level: int, r0: float, f: SvdFactors, s2, pbar, lists=None) -> np.ndarray:
    """Transpose of ``m2l_svd_stage2``: q-bar~^s = s_l sum_t Vhat_o^T (Uhat_o^T p-bar~^t).
    The transpose of Eq. (17)'s products (Sec. 3.2)."""
    pb, squeeze = _as3(pbar)
    tg, sr, ok = lists if lists is not None else geo.interaction_lists(box_ijk)
    pt = pb @ f.U
    qt = np.zeros(pb.shape[:2] + (f.r,))
    for k in np.unique(ok):
        sel = ok == k
        uh, vh = s2[k]
        qt[sr[sel]] += (pt[tg[sel]] @ uh) @ vh
    qt *= factors_scale(f, level, r0)
    out = qt @ f.R.T
    return out[:, 0, :] if squeeze else out


def eps2_from_c2(c2: float, eps1: float, r: int) -> float:
    """eps2 = C2 eps1 / p~ with p~ the compressed dimension (Eq. (18))."""
    return c2 * eps1 / r


def eps1_from_c1(c1: float, n_levels: int) -> float:
    """eps1 = C1 2^(-L) / L (Eq. (16))."""
    return c1 * 2.0 ** (-n_levels) / n_levels
