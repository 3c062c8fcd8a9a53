"""Pins of the FMM oracle (``oracle/fmm.py``): complete potential evaluation
with the compressed passes of Sec. 3.3, checked against closed forms, brute
force, potential theory and the direct sum (Eq. (1)).  CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import fmm, m2l, upward
from oracle import geometry as geo

D = 0.1


@pytest.fixture(scope="module")
def cube_case():
    """1500 points uniform in the unit cube, depth-3 tree (M2L on levels 2
    and 3, so one L2L level), the direct sum at every point."""
    pts = synth.points_uniform_cube(1500, 0)
    q = synth.densities_uniform(1500, 1)
    tree = synth.build_tree(pts, 3, centre=np.array([0.5, 0.5, 0.5]), r0=0.5)
    return tree, pts, q, fmm.direct_sum(pts, q)


def test_direct_sum_closed_form():
    # three charges on a line at 0, 1 and 3: hand-computed 1/(4 pi r) sums
    pts = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [3.0, 0.0, 0.0]])
    q = np.array([1.0, 2.0, -3.0])
    c = 1.0 / (4.0 * np.pi)
    want = c * np.array([2.0 / 1.0 - 3.0 / 3.0, 1.0 / 1.0 - 3.0 / 2.0, 1.0 / 3.0 + 2.0 / 2.0])
    np.testing.assert_allclose(fmm.direct_sum(pts, q), want, rtol=1e-15)
    np.testing.assert_allclose(fmm.direct_sum(pts, q, targets=[2, 0]), want[[2, 0]], rtol=1e-15)


def test_near_field_matches_bruteforce_neighbour_rule():
    # leaf coordinates computed here from the points alone; near = the two
    # points' leaves differ by at most one in every coordinate; i != j
    pts = synth.points_sphere(700, 3)
    q = synth.densities_normal(700, 4)
    depth = 3
    tree = synth.build_tree(pts, depth)
    lo = tree.centre - tree.r0
    ijk = np.clip(np.floor((pts - lo) / (2.0 * tree.r0) * (1 << depth)).astype(np.int64), 0, (1 << depth) - 1)
    want = np.zeros(700)
    for i in range(700):
        for j in range(700):
            if i != j and np.max(np.abs(ijk[i] - ijk[j])) <= 1:
                want[i] += q[j] / (4.0 * np.pi * np.linalg.norm(pts[i] - pts[j]))
    np.testing.assert_allclose(fmm.near_field(tree, pts, q), want, rtol=1e-12, atol=0)


def test_octant_signs_and_parents():
    # octant c = 4 bx + 2 by + bz; the child centre sits at (2b - 1) h_child
    np.testing.assert_array_equal(fmm.child_signs()[5], [1.0, -1.0, 1.0])
    np.testing.assert_array_equal(fmm.octant(np.array([[3, 2, 5], [0, 1, 0]])), [5, 2])
    tree = synth.build_tree(synth.points_torus(2000, 1), 4)
    for level in (2, 3, 4):
        par = fmm.parent_rows(tree, level)
        np.testing.assert_array_equal(tree.levels[level - 1][par], tree.levels[level] >> 1)
        # the child's centre from its parent's, its octant and its half-width
        cc = tree.box_centres(level)
        pc = tree.box_centres(level - 1)[par]
        off = fmm.child_signs()[fmm.octant(tree.levels[level])] * tree.halfwidth(level)
        np.testing.assert_allclose(pc + off, cc, rtol=0, atol=1e-14)


def test_check_to_equivalent_homogeneity():
    # G is homogeneous of degree -1, so E(h) = h E(1) (Sec. 3.1's argument).
    # Entries of a pseudo-inverse with a 1e-9 cutoff carry noise along the
    # directions near the cutoff, so the identity is checked on what E acts
    # on: check potentials of charges inside the box (upward) and of charges
    # outside its far-field boundary (downward), the same charges scaled by h.
    rng = np.random.default_rng(0)
    inside = rng.uniform(-1.0, 1.0, size=(20, 3))
    outside = _shell_points(20, 1, 3.5, 6.0)
    q = rng.standard_normal(20)
    for h in (0.25, 3.0):
        for E, surf, src in ((upward.check_to_equivalent, 3.0 - 2.0 * D, inside),
                             (fmm.downward_check_to_equivalent, 1.0 + D, outside)):
            e1 = E(6, D, 1.0, fmm.FMM_RCOND) @ (geo.laplace_kernel(geo.surface_points(6, np.zeros(3), surf), src) @ q)
            eh = h * E(6, D, 1.0, fmm.FMM_RCOND) @ (
                geo.laplace_kernel(geo.surface_points(6, np.zeros(3), surf * h), h * src) @ q)
            eh_direct = E(6, D, h, fmm.FMM_RCOND) @ (
                geo.laplace_kernel(geo.surface_points(6, np.zeros(3), surf * h), h * src) @ q)
            assert np.linalg.norm(eh - e1) <= 2e-8 * np.linalg.norm(e1)
            assert np.linalg.norm(eh_direct - e1) <= 2e-8 * np.linalg.norm(e1)


def _shell_points(n, seed, lo, hi):
    """n points with lo <= max-norm <= hi around the origin."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        x = rng.uniform(-hi, hi, 3)
        if np.max(np.abs(x)) >= lo:
            out.append(x)
    return np.array(out)


@pytest.mark.parametrize("c", [0, 5, 6])
def test_s2m_m2m_reproduce_far_potential(c):
    # points inside the child in octant c of a unit parent at the origin; the
    # parent's upward equivalent densities must reproduce their potential
    # outside the parent's far-field boundary (potential theory, Sec. 2.2)
    p, hc = 6, 0.5
    centre = np.array([(c >> 2) & 1, (c >> 1) & 1, c & 1], dtype=np.float64) - 0.5
    rng = np.random.default_rng(c)
    src = centre + rng.uniform(-hc, hc, size=(30, 3))
    q = rng.standard_normal(30)
    xu = geo.surface_points(p, centre, (3.0 - 2.0 * D) * hc)
    q_child = upward.check_to_equivalent(p, D, hc, fmm.FMM_RCOND) @ (geo.laplace_kernel(xu, src) @ q)
    q_parent = fmm.m2m_matrix(p, D, 1.0, c) @ q_child
    far = _shell_points(40, 10 + c, 3.0, 5.0)
    got = geo.laplace_kernel(far, geo.surface_points(p, np.zeros(3), 1.0 + D)) @ q_parent
    want = geo.laplace_kernel(far, src) @ q
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-5


@pytest.mark.parametrize("c", [1, 2, 7])
def test_l2l_l2t_reproduce_far_potential(c):
    # sources beyond a unit parent's far-field boundary; the parent's exact
    # downward check potentials, L2L to child c and L2T must give the
    # sources' potential at points inside the child (Sec. 2.2)
    p, hc = 6, 0.5
    src = _shell_points(40, 20 + c, 3.5, 6.0)
    q = np.random.default_rng(c).standard_normal(40)
    xd = geo.surface_points(p, np.zeros(3), 1.0 + D)
    pd_child = fmm.l2l_matrix(p, D, 1.0, c) @ (geo.laplace_kernel(xd, src) @ q)
    centre = np.array([(c >> 2) & 1, (c >> 1) & 1, c & 1], dtype=np.float64) - 0.5
    tgt = centre + np.random.default_rng(50 + c).uniform(-hc, hc, size=(25, 3))
    yd = geo.surface_points(p, centre, (3.0 - 2.0 * D) * hc)
    got = geo.laplace_kernel(tgt, yd) @ (fmm.downward_check_to_equivalent(p, D, hc) @ pd_child)
    want = geo.laplace_kernel(tgt, src) @ q
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-5


def test_uncompressed_fmm_converges_to_direct_sum(cube_case):
    tree, pts, q, exact = cube_case
    near = fmm.near_field(tree, pts, q)
    errs = {}
    for p in (4, 5):
        pot = near + fmm.fmm_uncompressed_far(tree, pts, p, D, q)
        errs[p] = np.linalg.norm(pot - exact) / np.linalg.norm(exact)
    assert errs[4] < 5e-4 and errs[5] < 5e-5 and errs[5] < errs[4] / 5.0, errs


def test_compressed_passes_at_full_rank_equal_uncompressed(cube_case):
    # with every singular value kept, R~ R~^T = I and Sec. 3.3's operators
    # reproduce the operators formed at each box's own size
    tree, pts, q, _ = cube_case
    f = m2l.svd_factors(4, D, 0.0)
    assert f.r == f.U.shape[0]
    far_c = fmm.fmm_compressed_far(tree, pts, f, fmm.pass_operators(f, 4, D), 4, D, q)
    far_u = fmm.fmm_uncompressed_far(tree, pts, 4, D, q)
    assert np.linalg.norm(far_c - far_u) / np.linalg.norm(far_u) < 1e-10


@pytest.mark.parametrize("p,eps,tol", [(6, 1e-7, 5e-6), (8, 1e-7, 3e-7)])
def test_compressed_fmm_matches_direct_sum(cube_case, p, eps, tol):
    tree, pts, q, exact = cube_case
    f = m2l.svd_factors(p, D, eps)
    pot = fmm.fmm_potential(tree, pts, q, p, D, f=f)
    assert np.linalg.norm(pot - exact) / np.linalg.norm(exact) < tol


def test_compressed_fmm_operator_is_symmetric(cube_case):
    # T = S^T and L = M^T (the downward surfaces are the upward ones swapped),
    # K_o^T = K_{-o}, and R~ R~^T = U~ U~^T: <A q, w> = <q, A w>
    tree, pts, q, _ = cube_case
    f = m2l.svd_factors(6, D, 1e-7)
    ops = fmm.pass_operators(f, 6, D)
    w = synth.densities_normal(pts.shape[0], 7)
    aq = fmm.fmm_potential(tree, pts, q, 6, D, f=f, ops=ops)
    aw = fmm.fmm_potential(tree, pts, w, 6, D, f=f, ops=ops)
    assert abs(aq @ w - aw @ q) <= 1e-8 * abs(aq @ w)
    # and the structural identities behind it
    # (two separately computed pseudo-inverses: equal up to their noise)
    np.testing.assert_allclose(fmm.l2l_matrix(6, D, 1.0, 3), fmm.m2m_matrix(6, D, 1.0, 3).T, rtol=0,
                               atol=1e-7 * np.abs(fmm.m2m_matrix(6, D, 1.0, 3)).max())


# ---------------------------------------------------------------------------
# double layer (Sec. 4, Eq. (26)): dG/dn(y) in S2T and in S2M's
# first step
# ---------------------------------------------------------------------------
def _sphere_quadrature(nt, nphi):
    """Points, outward normals and weights of a product rule on the unit
    sphere: Gauss-Legendre in cos(theta), trapezoid in phi (spectrally
    accurate for integrands analytic on the sphere)."""
    t, wt = np.polynomial.legendre.leggauss(nt)
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1.0 - t * t)
    y = np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)), np.outer(t, np.ones(nphi))], -1).reshape(-1, 3)
    w = np.outer(wt, np.full(nphi, 2.0 * np.pi / nphi)).reshape(-1)
    return y, y.copy(), w


def test_double_layer_kernel_gauss_law():
    # the double-layer potential of unit density on a closed surface is -1
    # inside and 0 outside (Gauss); the rule integrates it to rounding
    y, n, w = _sphere_quadrature(32, 64)
    assert abs(w.sum() - 4.0 * np.pi) < 1e-12
    rng = np.random.default_rng(3)
    inside = rng.uniform(-1.0, 1.0, size=(20, 3))
    inside *= 0.5 * rng.uniform(0.0, 1.0, size=(20, 1)) / np.linalg.norm(inside, axis=1, keepdims=True)
    outside = rng.standard_normal((20, 3))
    outside *= rng.uniform(2.5, 6.0, size=(20, 1)) / np.linalg.norm(outside, axis=1, keepdims=True)
    np.testing.assert_allclose(geo.laplace_double_layer_kernel(inside, y, n) @ w, -1.0, rtol=0, atol=1e-11)
    np.testing.assert_allclose(geo.laplace_double_layer_kernel(outside, y, n) @ w, 0.0, rtol=0, atol=1e-11)
    # and it is the normal derivative of G at the source: finite differences
    x, y0, n0 = np.array([[0.3, -0.2, 0.9]]), np.array([[0.1, 0.4, -0.2]]), np.array([[0.6, 0.0, 0.8]])
    hh = 1e-5
    fd = (geo.laplace_kernel(x, y0 + hh * n0) - geo.laplace_kernel(x, y0 - hh * n0)) / (2 * hh)
    np.testing.assert_allclose(geo.laplace_double_layer_kernel(x, y0, n0), fd, rtol=1e-9)


def test_double_layer_direct_sum_closed_form():
    # dipoles at (0,0,0), (1,0,0), (0,2,0) with normals x, (0.6,0.8,0), z and
    # densities 1, 2, 3: p_i = sum_j q_j n_j.(x_i - x_j) / (4 pi |x_i - x_j|^3)
    pts = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    nrm = np.array([[1.0, 0.0, 0.0], [0.6, 0.8, 0.0], [0.0, 0.0, 1.0]])
    q = np.array([1.0, 2.0, 3.0])
    want = np.array([-1.2 / (4.0 * np.pi), 1.0 / (4.0 * np.pi), 1.0 / (10.0 * np.sqrt(5.0) * np.pi)])
    np.testing.assert_allclose(fmm.direct_sum(pts, q, normals=nrm), want, rtol=1e-14, atol=1e-17)


def test_double_layer_near_field_bruteforce():
    pts = synth.points_sphere(600, 5)
    nrm = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    q = synth.densities_normal(600, 6)
    depth = 3
    tree = synth.build_tree(pts, depth)
    lo = tree.centre - tree.r0
    ijk = np.clip(np.floor((pts - lo) / (2.0 * tree.r0) * (1 << depth)).astype(np.int64), 0, (1 << depth) - 1)
    want = np.zeros(600)
    for i in range(600):
        for j in range(600):
            if i != j and np.max(np.abs(ijk[i] - ijk[j])) <= 1:
                dx = pts[i] - pts[j]
                want[i] += q[j] * (nrm[j] @ dx) / (4.0 * np.pi * np.linalg.norm(dx) ** 3)
    np.testing.assert_allclose(fmm.near_field(tree, pts, q, normals=nrm), want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("c", [0, 3])
def test_double_layer_s2m_reproduces_far_potential(c):
    # dipoles inside child c of a unit parent: single-layer equivalent
    # densities solved from their double-layer check potentials
    # (Eq. (26)) reproduce their potential beyond the far-field
    # boundary
    p, hc = 6, 0.5
    centre = np.array([(c >> 2) & 1, (c >> 1) & 1, c & 1], dtype=np.float64) - 0.5
    rng = np.random.default_rng(40 + c)
    src = centre + rng.uniform(-hc, hc, size=(30, 3))
    nrm = rng.standard_normal((30, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    q = rng.standard_normal(30)
    xu = geo.surface_points(p, centre, (3.0 - 2.0 * D) * hc)
    q_child = upward.check_to_equivalent(p, D, hc, fmm.FMM_RCOND) @ (geo.laplace_double_layer_kernel(xu, src, nrm) @ q)
    q_parent = fmm.m2m_matrix(p, D, 1.0, c) @ q_child
    far = _shell_points(40, 60 + c, 3.0, 5.0)
    got = geo.laplace_kernel(far, geo.surface_points(p, np.zeros(3), 1.0 + D)) @ q_parent
    want = geo.laplace_double_layer_kernel(far, src, nrm) @ q
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-4


@pytest.fixture(scope="module")
def dipole_case():
    """1500 points on the unit sphere with their outward normals, depth 3,
    and the direct double-layer sum at every point."""
    pts = synth.points_sphere(1500, 8)
    nrm = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    q = synth.densities_normal(1500, 9)
    tree = synth.build_tree(pts, 3)
    return tree, pts, nrm, q, fmm.direct_sum(pts, q, normals=nrm)


def test_double_layer_fmm_converges_to_direct_sum(dipole_case):
    tree, pts, nrm, q, exact = dipole_case
    near = fmm.near_field(tree, pts, q, normals=nrm)
    errs = {}
    for p in (4, 6):
        pot = near + fmm.fmm_uncompressed_far(tree, pts, p, D, q, normals=nrm)
        errs[p] = np.linalg.norm(pot - exact) / np.linalg.norm(exact)
    f = m2l.svd_factors(8, D, 1e-7)
    pot8 = fmm.fmm_potential(tree, pts, q, 8, D, f=f, normals=nrm)
    errs[8] = np.linalg.norm(pot8 - exact) / np.linalg.norm(exact)
    assert errs[4] < 5e-3 and errs[6] < 1e-4 and errs[8] < 4e-6, errs
    assert errs[6] < errs[4] / 5.0 and errs[8] < errs[6] / 5.0, errs


def test_double_layer_compressed_at_full_rank_equals_uncompressed(dipole_case):
    # every singular value kept: Sec. 3.3's compressed passes applied to the
    # dipoles' check potentials reproduce the uncompressed far field
    tree, pts, nrm, q, _ = dipole_case
    f = m2l.svd_factors(4, D, 0.0)
    far_c = fmm.fmm_compressed_far(tree, pts, f, fmm.pass_operators(f, 4, D), 4, D, q, normals=nrm)
    far_u = fmm.fmm_uncompressed_far(tree, pts, 4, D, q, normals=nrm)
    assert np.linalg.norm(far_c - far_u) / np.linalg.norm(far_u) < 1e-10
