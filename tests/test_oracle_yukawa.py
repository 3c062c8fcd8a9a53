"""Pins of the oracle's non-homogeneous kernel path (Sec. 3.1: the
translation matrices of every level are compressed separately when G is not
homogeneous): the Yukawa kernel G = exp(-kappa r) / (4 pi r) and the
per-level factors ``oracle.m2l.svd_factors(..., kappa=, h=)``.  CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from oracle import geometry as geo
from oracle import m2l

D = 0.1


def test_yukawa_kernel_shell_closed_form():
    # unit-density shell of radius a: integrating over the distance rho gives
    # phi(R) = a / (2 kappa R) (exp(-kappa |R - a|) - exp(-kappa (R + a)))
    # inside and outside; the product rule (Gauss-Legendre in cos(theta),
    # trapezoid in phi) is spectrally accurate away from the shell
    a, kappa = 0.7, 2.5
    t, wt = np.polynomial.legendre.leggauss(40)
    ph = 2.0 * np.pi * np.arange(80) / 80
    st = np.sqrt(1.0 - t * t)
    y = a * np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(t, np.ones(80))], -1).reshape(-1, 3)
    w = a * a * np.outer(wt, np.full(80, 2.0 * np.pi / 80)).reshape(-1)
    rng = np.random.default_rng(2)
    dirs = rng.standard_normal((12, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    R = np.concatenate([rng.uniform(0.05, 0.35, 6), rng.uniform(1.4, 3.0, 6)])
    x = dirs * R[:, None]
    want = a / (2.0 * kappa * R) * (np.exp(-kappa * np.abs(R - a)) - np.exp(-kappa * (R + a)))
    np.testing.assert_allclose(geo.yukawa_kernel(x, y, kappa) @ w, want, rtol=1e-11)
    # kappa = 0 is the Laplace kernel
    np.testing.assert_array_equal(geo.yukawa_kernel(x, y, 0.0), geo.laplace_kernel(x, y))


@pytest.fixture(scope="module")
def level3():
    """The non-empty level-3 boxes of 3000 points on the unit sphere (root:
    bounding cube) with N(0,1) densities."""
    pts = synth.points_sphere(3000, 4)
    tree = synth.build_tree(pts, 3)
    q = np.random.default_rng(5).standard_normal((tree.levels[3].shape[0], 56))
    return tree, q


def test_yukawa_full_rank_equals_dense(level3):
    # every singular value kept: the per-level compressed M2L is the dense
    # M2L of that level, every pair's matrix formed from its coordinates
    tree, q = level3
    kappa, h = 3.0, tree.halfwidth(3)
    f = m2l.svd_factors(4, D, 0.0, kappa=kappa, h=h)
    assert f.r == 56
    got = m2l.m2l_svd(tree.levels[3], 3, tree.r0, f, q)
    want = m2l.m2l_dense(tree.levels[3], 3, tree.r0, 4, D, q, centre=tree.centre, kappa=kappa)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12


def test_yukawa_truncation_bound_and_symmetry():
    # ||K_o - U~ K~_o R~^T||_2 <= 2 sigma_{r+1}(K_fat), and K~_o^T = K~_{-o}
    # (G radial, both surfaces the same pattern)
    f = m2l.svd_factors(6, D, 1e-5, kappa=4.0, h=0.125)
    assert f.r < f.U.shape[0]
    bound = 2.0 * f.sigma[f.r]
    for k in range(0, 316, 5):
        assert np.linalg.norm(f.K[k] - f.U @ f.C[k] @ f.R.T, 2) <= bound * (1 + 1e-9), k
    offs = geo.m2l_offsets()
    tab = geo.offset_index_table()
    # R~ spans U~'s space (K_thin is a row-block permutation of K_fat^T)
    np.testing.assert_allclose(np.linalg.svd(f.U.T @ f.R, compute_uv=False), 1.0, atol=1e-8)
    Cu = f.U.T[None] @ f.K @ f.U[None]  # U~^T K_o U~
    for k in (0, 40, 200):
        np.testing.assert_allclose(Cu[k].T, Cu[tab[tuple(-offs[k])]], rtol=0, atol=1e-10 * np.abs(Cu).max())


def test_kappa_zero_per_level_reproduces_homogeneous(level3):
    # the per-level path at kappa = 0 is Sec. 3.1's homogeneity shortcut
    tree, q = level3
    f_unit = m2l.svd_factors(4, D, 1e-4)
    f_lvl = m2l.svd_factors(4, D, 1e-4, kappa=0.0, h=tree.halfwidth(3))
    a = m2l.m2l_svd(tree.levels[3], 3, tree.r0, f_unit, q)
    b = m2l.m2l_svd(tree.levels[3], 3, tree.r0, f_lvl, q)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-12


def test_yukawa_needs_per_level_factors(level3):
    # with kappa > 0 the factors of one box size are wrong at another: the
    # level-3 result from level-2 factors (Laplace-style scaling) is far off,
    # and the oracle refuses factors of a different half-width
    tree, q = level3
    kappa = 3.0
    f3 = m2l.svd_factors(4, D, 0.0, kappa=kappa, h=tree.halfwidth(3))
    f2 = m2l.svd_factors(4, D, 0.0, kappa=kappa, h=tree.halfwidth(2))
    want = m2l.m2l_svd(tree.levels[3], 3, tree.r0, f3, q)
    wrong = 2.0 * m2l.m2l_svd(tree.levels[3], 2, tree.r0, f2, q)  # K_2 scaled as if homogeneous
    assert np.linalg.norm(wrong - want) / np.linalg.norm(want) > 0.1
    with pytest.raises(ValueError):
        m2l.m2l_svd(tree.levels[3], 3, tree.r0, f2, q)


def test_yukawa_adjoint_dot_product(level3):
    tree, q = level3
    f = m2l.svd_factors(4, D, 1e-6, kappa=2.0, h=tree.halfwidth(3))
    y = np.random.default_rng(8).standard_normal(q.shape)
    ax = m2l.m2l_svd(tree.levels[3], 3, tree.r0, f, q)
    aty = m2l.m2l_svd_adjoint(tree.levels[3], 3, tree.r0, f, y)
    assert abs(np.sum(ax * y) - np.sum(q * aty)) <= 1e-13 * np.linalg.norm(ax) * np.linalg.norm(y)
