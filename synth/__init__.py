"""Seeded synthetic inputs for the SVD-compressed M2L translation.

This module produces the point clouds, point densities and octree box
coordinates that stand in for the paper's BEM meshes (the ellipsoid of
Sec. 5.1, the shaft of Sec. 5.2 and the engine block of Sec. 5.3 are not
available, so element centroids are replaced by synthetic surface points,
as Sec. 4.1 builds the octree on element centroids).

It holds no arithmetic of the method itself: no surfaces, kernels,
translation matrices, interaction lists or SVDs.  Both the FP64 oracle and
the CUDA path consume what it returns, which is the only code they share.

Every generator takes an explicit seed and uses NumPy's PCG64
(``numpy.random.default_rng``), so a workload is reproducible on any host.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "points_uniform_cube",
    "points_sphere",
    "points_torus",
    "points_ellipsoid",
    "densities_uniform",
    "densities_normal",
    "Tree",
    "build_tree",
    "morton_keys",
    "random_box_densities",
    "random_box_densities32",
    "ellipsoid_instance",
    "Workload",
    "workload",
    "WORKLOADS",
]


# ---------------------------------------------------------------------------
# point clouds
# ---------------------------------------------------------------------------
def points_uniform_cube(n: int, seed: int) -> np.ndarray:
    """``n`` points uniform in the unit cube [0,1]^3, float64 [n,3]."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 3))


def points_sphere(n: int, seed: int, radius: float = 1.0) -> np.ndarray:
    """``n`` points uniform on a sphere (normalised Gaussian vectors)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return radius * g


def points_torus(n: int, seed: int, big_r: float = 1.0, small_r: float = 0.3) -> np.ndarray:
    """``n`` points area-uniform on a torus with radii (big_r, small_r).

    Angles are drawn uniformly and a candidate is accepted with probability
    (R + r cos t) / (R + r), the ratio of the local area element to its
    maximum, so accepted points are uniform in surface area.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 1024
        t = rng.random(m) * 2.0 * np.pi
        ph = rng.random(m) * 2.0 * np.pi
        u = rng.random(m)
        keep = u < (big_r + small_r * np.cos(t)) / (big_r + small_r)
        t, ph = t[keep], ph[keep]
        ring = big_r + small_r * np.cos(t)
        pts = np.stack([ring * np.cos(ph), ring * np.sin(ph), small_r * np.sin(t)], axis=1)
        out = np.concatenate([out, pts], axis=0)
    return out[:n]


def points_ellipsoid(n: int, seed: int, axes) -> np.ndarray:
    """Sphere samples scaled per axis onto an ellipsoid (not area-uniform)."""
    p = points_sphere(n, seed)
    return p * np.asarray(axes, dtype=np.float64)[None, :]


# ---------------------------------------------------------------------------
# densities
# ---------------------------------------------------------------------------
def densities_uniform(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """Point densities U[-1,1], float64 [nrhs, n] (squeezed when nrhs == 1)."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(-1.0, 1.0, size=(nrhs, n))
    return q[0] if nrhs == 1 else q


def densities_normal(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """Point densities N(0,1), float64 [nrhs, n] (squeezed when nrhs == 1)."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((nrhs, n))
    return q[0] if nrhs == 1 else q


def random_box_densities32(n_boxes: int, nrhs: int, n_surf: int, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) upward-equivalent densities drawn directly in float32
    (half the memory and time of ``random_box_densities`` for the multi-GB
    inputs of the 64-instance batch), layout [n_boxes, nrhs, n_surf]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_boxes, nrhs, n_surf), dtype=np.float32)


def random_box_densities(n_boxes: int, nrhs: int, n_surf: int, seed: int,
                         dtype=np.float32) -> np.ndarray:
    """i.i.d. N(0,1) upward-equivalent densities, layout [n_boxes, nrhs, n_surf].

    Used where only the cost of the translation matters (its cost does not
    depend on the values).
    """
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_boxes, nrhs, n_surf)).astype(dtype)


# ---------------------------------------------------------------------------
# octree (uniform depth, empty boxes skipped)
# ---------------------------------------------------------------------------
def _spread_bits(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.uint64)
    out = np.zeros_like(v)
    for b in range(21):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def morton_keys(ijk: np.ndarray) -> np.ndarray:
    """Morton (Z-order) key of integer box coordinates [m,3] -> uint64 [m]."""
    ijk = np.asarray(ijk)
    return (_spread_bits(ijk[:, 0]) << np.uint64(2)) | (_spread_bits(ijk[:, 1]) << np.uint64(1)) \
        | _spread_bits(ijk[:, 2])


@dataclass
class Tree:
    """A uniform-depth octree over a point cloud, empty boxes skipped.

    ``levels[l]`` is an int32 array [B_l, 3] of the integer coordinates of
    the non-empty boxes of level ``l`` (0 <= i,j,k < 2**l), sorted by Morton
    key.  Boxes of level ``l`` have half-width ``r0 / 2**l`` and centre
    ``centre - r0 + (2*ijk + 1) * r0 / 2**l``.  ``leaf_of_point[i]`` is the
    row of point ``i``'s box in ``levels[depth]``.
    """

    centre: np.ndarray
    r0: float
    depth: int
    levels: dict = field(default_factory=dict)
    leaf_of_point: np.ndarray | None = None

    def halfwidth(self, level: int) -> float:
        return self.r0 / (1 << level)

    def box_centres(self, level: int) -> np.ndarray:
        h = self.halfwidth(level)
        return (self.centre - self.r0)[None, :] + (2.0 * self.levels[level] + 1.0) * h


def build_tree(points: np.ndarray, depth: int, centre=None, r0=None) -> Tree:
    """Bin ``points`` into a uniform octree of the given depth.

    Root cube: when ``centre``/``r0`` are not given, the centre of the
    bounding box and half-width = max half-extent * (1 + 2**-20).  The box
    index of a point at level l is min(floor((x - (c - r0)) / (2 r0) * 2**l),
    2**l - 1) per coordinate.
    """
    points = np.asarray(points, dtype=np.float64)
    if centre is None or r0 is None:
        lo, hi = points.min(axis=0), points.max(axis=0)
        centre = 0.5 * (lo + hi)
        r0 = float(0.5 * (hi - lo).max() * (1.0 + 2.0 ** -20))
    centre = np.asarray(centre, dtype=np.float64)
    tree = Tree(centre=centre, r0=float(r0), depth=depth)
    rel = (points - (centre - r0)[None, :]) / (2.0 * r0)
    m = 1 << depth
    ijk_leaf = np.clip(np.floor(rel * m).astype(np.int64), 0, m - 1)
    for level in range(depth + 1):
        ijk = ijk_leaf >> (depth - level)
        keys = morton_keys(ijk)
        uniq, first, inv = np.unique(keys, return_index=True, return_inverse=True)
        tree.levels[level] = ijk[first].astype(np.int32)
        if level == depth:
            tree.leaf_of_point = inv.astype(np.int64)
    return tree


# ---------------------------------------------------------------------------
# named workloads (shapes of the paper's BEM problems, synthetic)
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    """One synthetic M2L workload: points, point densities and its tree."""

    name: str
    p: int
    eps: float
    d: float
    depth: int
    points: np.ndarray
    densities: np.ndarray
    tree: Tree
    nrhs: int = 1
    seed: int = 0


def _wl_cube16k(seed=0, n=16384, depth=3):
    pts = points_uniform_cube(n, seed)
    q = densities_uniform(n, seed + 1)
    tree = build_tree(pts, depth, centre=np.array([0.5, 0.5, 0.5]), r0=0.5)
    return Workload("cube16k_p6", 6, 1e-8, 0.1, depth, pts, q, tree, seed=seed)


def _wl_sphere2m(seed=0, n=2_097_152, depth=6):
    pts = points_sphere(n, seed)
    q = densities_normal(n, seed + 1)
    return Workload("sphere2m_p8", 8, 1e-7, 0.1, depth, pts, q, build_tree(pts, depth), seed=seed)


def _wl_torus4m(seed=0, n=4_194_304, depth=6):
    pts = points_torus(n, seed)
    q = densities_uniform(n, seed + 1)
    return Workload("torus4m_p10", 10, 1e-8, 0.1, depth, pts, q, build_tree(pts, depth), seed=seed)


def _wl_sphere1m(seed=0, n=1_048_576, depth=5):
    pts = points_sphere(n, seed)
    q = densities_uniform(n, seed + 1)
    return Workload("sphere1m_p8", 8, 1e-7, 0.1, depth, pts, q, build_tree(pts, depth), seed=seed)


def ellipsoid_instance(i: int):
    """Instance ``i`` of the 64-instance mixed batch.

    N log-uniform in [5e4, 1e6], axes U[0.5, 2], depth uniform in {3..6},
    p uniform in {6, 8, 10}; points use seed 1000 + i.
    """
    rng = np.random.default_rng(1000 + i)
    n = int(np.exp(rng.uniform(np.log(5e4), np.log(1e6))))
    axes = rng.uniform(0.5, 2.0, size=3)
    depth = int(rng.integers(3, 7))
    p = int(rng.choice([6, 8, 10]))
    pts = points_ellipsoid(n, 1000 + i, axes)
    return Workload(f"ellipsoid{i}", p, 1e-7, 0.1, depth, pts, np.zeros(0),
                    build_tree(pts, depth), nrhs=16, seed=1000 + i)


WORKLOADS = {
    "cube16k_p6": _wl_cube16k,
    "sphere2m_p8": _wl_sphere2m,
    "torus4m_p10": _wl_torus4m,
    "sphere1m_p8": _wl_sphere1m,
}


def workload(name: str, **kw) -> Workload:
    """Build a named workload (see ``WORKLOADS``)."""
    return WORKLOADS[name](**kw)
