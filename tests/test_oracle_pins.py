"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/paper_counts.txt), closed forms, brute force on
tiny inputs, error bounds of the truncated SVD, invariants (homogeneity,
symmetry, linearity, translation invariance) and special cases that reduce
to the textbook dense product.  A plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a wrong level scale)
fails at least one of them.
"""
import os

import numpy as np
import pytest

import synth
from oracle import geometry as geo
from oracle import m2l, upward

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        vals[tuple(parts[:-1])] = int(parts[-1])
    return vals


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
def test_offset_count_matches_paper():
    offs = geo.m2l_offsets()
    assert offs.shape == (_golden()[("offsets",)], 3)
    assert len({tuple(o) for o in offs}) == 316
    assert np.all(np.abs(offs).max(axis=1) >= 2) and np.all(np.abs(offs) <= 3)
    # the set is closed under negation (needed by the adjoint's reversed offset)
    s = {tuple(o) for o in offs}
    assert all(tuple(-o) in s for o in offs)


def test_surface_point_count_matches_paper_and_closed_form():
    g = _golden()
    assert geo.surface_grid(8).shape[0] == g[("surface_points", "8")]
    for p in range(2, 13):
        pts = geo.surface_grid(p)
        assert pts.shape[0] == 6 * (p - 1) ** 2 + 2
        # every point is on the boundary, no duplicates
        assert len({tuple(x) for x in pts}) == pts.shape[0]
        assert np.all((pts.min(axis=1) == 0) | (pts.max(axis=1) == p - 1))


def test_surface_points_lie_on_cube_boundary():
    c = np.array([0.3, -1.0, 2.0])
    pts = geo.surface_points(6, c, 0.7)
    dist = np.abs(pts - c).max(axis=1)
    assert np.allclose(dist, 0.7, rtol=0, atol=1e-15)


def test_laplace_kernel_values():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 2.0]])
    y = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    g = geo.laplace_kernel(x, y)
    assert g[0, 0] == pytest.approx(1.0 / (4 * np.pi))
    assert g[1, 1] == pytest.approx(1.0 / (4 * np.pi * 3.0))
    assert g[1, 0] == pytest.approx(1.0 / (4 * np.pi * np.sqrt(8.0)))
    assert g[0, 1] == np.inf  # coincident points: the kernel is singular


def test_interaction_lists_match_bruteforce_on_random_sets():
    rng = np.random.default_rng(3)
    for level, nbox in ((2, 40), (3, 120), (4, 200)):
        m = 1 << level
        allb = np.array([(i, j, k) for i in range(m) for j in range(m) for k in range(m)])
        box = allb[rng.choice(allb.shape[0], size=min(nbox, allb.shape[0]), replace=False)]
        a = geo.interaction_lists(box)
        b = geo.interaction_lists_bruteforce(box)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        tg, sr, ok = a
        offs = geo.m2l_offsets()
        assert np.array_equal(box[tg] - box[sr], offs[ok])


def test_full_grid_pair_counts_closed_form():
    # Full grid of m = 2**l boxes per side: per dimension the candidates
    # (children of the parent's neighbours) sum to 6m-8 and the near field to
    # 3m-2, so the number of M2L pairs is (6m-8)^3 - (3m-2)^3, and an
    # interior target has 6^3 - 3^3 = 189 sources.
    for level in (2, 3):
        m = 1 << level
        box = np.array([(i, j, k) for i in range(m) for j in range(m) for k in range(m)])
        tg, _, _ = geo.interaction_lists(box)
        assert tg.size == (6 * m - 8) ** 3 - (3 * m - 2) ** 3
        assert np.bincount(tg).max() == 189 if m >= 8 else True
    assert (6 * 4 - 8) ** 3 - (3 * 4 - 2) ** 3 == 3096


def test_interaction_relation_is_symmetric():
    rng = np.random.default_rng(4)
    m = 8
    allb = np.array([(i, j, k) for i in range(m) for j in range(m) for k in range(m)])
    box = allb[rng.choice(allb.shape[0], size=150, replace=False)]
    tg, sr, ok = geo.interaction_lists(box)
    fwd = set(zip(tg.tolist(), sr.tolist()))
    assert fwd == set(zip(sr.tolist(), tg.tolist()))


# ---------------------------------------------------------------------------
# translation matrices
# ---------------------------------------------------------------------------
def test_m2l_matrix_transpose_is_reversed_offset():
    # G is radial and both surfaces use the same point pattern, so
    # K_o^T = K_{-o}: the paper's "symmetric" remark (Sec. 3.1) read correctly.
    K = m2l.unit_m2l_matrices(4, 0.1)
    offs = geo.m2l_offsets()
    tab = geo.offset_index_table()
    for k, o in enumerate(offs):
        np.testing.assert_allclose(K[k].T, K[tab[tuple(-o)]], rtol=1e-14, atol=0)
    # and K_o itself is not symmetric
    assert np.abs(K[0] - K[0].T).max() > 1e-3 * np.abs(K[0]).max()


def test_homogeneity_level_scaling():
    # Sec. 3.1: G homogeneous of degree m = -1 => K_l = (r0/2^l)^-1 K_0.
    p, d, r0 = 4, 0.1, 0.75
    K = m2l.unit_m2l_matrices(p, d)
    offs = geo.m2l_offsets()
    for level in (2, 5):
        h = r0 / (1 << level)
        for k in (0, 57, 200, 315):
            geom = m2l.m2l_matrix_geometric(p, d, 2 * h * offs[k] + 0.3, np.array([0.3, 0.3, 0.3]), h)
            np.testing.assert_allclose(geom, m2l.level_scale(level, r0) * K[k], rtol=2e-14)


# ---------------------------------------------------------------------------
# SVD compression (Sec. 3.1)
# ---------------------------------------------------------------------------
def test_truncation_rank_rule():
    s = np.array([1.0, 0.5, 0.5, 0.1])
    assert m2l.truncation_rank(s, 0.5) == 3       # not less than eps*sigma0 keeps ties
    assert m2l.truncation_rank(s, 0.49) == 3
    assert m2l.truncation_rank(s, 0.51) == 1
    s2 = np.array([1.0, 0.6, 0.5, 0.5 - 1e-15, 0.1])
    assert m2l.truncation_rank(s2, 0.5) == 4       # cluster kept whole
    assert m2l.truncation_rank(s2, 0.0) == 5


@pytest.mark.parametrize("p,eps", [(4, 1e-4), (6, 1e-7)])
def test_svd_truncation_error_bound(oracle_factors, p, eps):
    # ||K_o - U~ C_o R~^T||_2 <= ||(I-U~U~^T) K_o|| + ||K_o (I-R~R~^T)||
    #                          <= sigma_r(K_fat) + lambda_r(K_thin)
    f = oracle_factors(p, 0.1, eps)
    n = f.U.shape[0]
    assert f.r < n
    bound = f.sigma[f.r] + f.lam[f.r]
    for k in range(0, 316, 7):
        err = np.linalg.norm(f.K[k] - f.U @ f.C[k] @ f.R.T, 2)
        assert err <= bound * (1 + 1e-6) + 1e-13 * f.sigma[0]
    # and the bound is not vacuous: some offset is near it
    worst = max(np.linalg.norm(f.K[k] - f.U @ f.C[k] @ f.R.T, 2) for k in range(316))
    assert worst > 0.1 * f.sigma[f.r]
    # orthonormal bases, and the fat and thin SVDs span the same space
    assert np.abs(f.U.T @ f.U - np.eye(f.r)).max() < 1e-13
    assert np.abs(f.R.T @ f.R - np.eye(f.r)).max() < 1e-13
    assert np.linalg.norm(f.U @ f.U.T - f.R @ f.R.T, 2) < 1e-6
    # sigma_0 = ||K_fat||_2 = Lambda_00 (Sec. 3.1)
    assert f.sigma[0] == pytest.approx(f.lam[0], rel=1e-13)


def test_svd_ranks_for_cutoffs(oracle_factors):
    f = oracle_factors(6, 0.1, 1e-8)
    assert f.r == 152  # no truncation at 1e-8 for p = 6, d = 0.1
    assert [m2l.truncation_rank(f.sigma, e) for e in (1e-6, 1e-7)] == [127, 146]


def test_compressed_core_transpose_is_reversed_offset(oracle_factors):
    # Through the operators: (U~ C_o R~^T)^T = U~ C_{-o} R~^T up to the
    # subspace sensitivity of the two SVDs.
    f = oracle_factors(4, 0.1, 1e-4)
    assert f.r < f.U.shape[0]
    offs = geo.m2l_offsets()
    tab = geo.offset_index_table()
    for k in (0, 100, 315):
        a = (f.U @ f.C[k] @ f.R.T).T
        b = f.U @ f.C[tab[tuple(-offs[k])]] @ f.R.T
        assert np.abs(a - b).max() < 1e-6 * f.sigma[0]


# ---------------------------------------------------------------------------
# M2L on boxes
# ---------------------------------------------------------------------------
def _small_case(seed=0, n=4000, depth=3, p=4):
    pts = synth.points_uniform_cube(n, seed)
    tree = synth.build_tree(pts, depth, centre=np.array([0.5, 0.5, 0.5]), r0=0.5)
    q = synth.densities_uniform(n, seed + 1)
    return pts, tree, q, p


def test_dense_m2l_matches_direct_sum():
    # M2L(S2M(q)) at the downward check points equals the direct potential of
    # the interaction-list points (Eq. (1)) within the KIFMM
    # discretisation error; p = 6, d = 0.1 measured ~1e-5.
    pts, tree, q, _ = _small_case(n=3000, p=6)
    p, d = 6, 0.1
    qup = upward.upward_pass(tree, pts, p, d, q)
    for level in (2, 3):
        box = tree.levels[level]
        tg = [0, box.shape[0] // 2, box.shape[0] - 1]
        pd = m2l.m2l_dense(box, level, tree.r0, p, d, qup[level], centre=tree.centre, targets=tg)
        direct = upward.direct_far_field(tree, pts, level, p, d, q, tg)
        err = np.linalg.norm(pd[tg] - direct) / np.linalg.norm(direct)
        assert err < 1e-4, err
    # with a wrong level (wrong surface size) the agreement is lost
    box = tree.levels[3]
    bad = m2l.m2l_dense(box, 3, tree.r0 * 1.5, p, d, qup[3], centre=tree.centre, targets=[0])
    direct = upward.direct_far_field(tree, pts, 3, p, d, q, [0])
    assert np.linalg.norm(bad[[0]] - direct) / np.linalg.norm(direct) > 1e-2


def test_dense_unit_equals_geometric():
    pts, tree, q, p = _small_case()
    K = m2l.unit_m2l_matrices(p, 0.1)
    rng = np.random.default_rng(1)
    for level in (2, 3):
        box = tree.levels[level]
        qq = rng.standard_normal((box.shape[0], K.shape[1]))
        a = m2l.m2l_dense(box, level, tree.r0, p, 0.1, qq, centre=tree.centre)
        b = m2l.m2l_dense_unit(box, level, tree.r0, K, qq)
        np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-12 * np.abs(a).max())


def test_svd_full_rank_reduces_to_dense():
    # eps -> 0 keeps r = n and the compressed product is the dense one.
    pts, tree, q, p = _small_case()
    f = m2l.svd_factors(p, 0.1, 0.0)
    assert f.r == f.U.shape[0]
    rng = np.random.default_rng(2)
    for level in (2, 3):
        box = tree.levels[level]
        qq = rng.standard_normal((box.shape[0], f.r))
        a = m2l.m2l_dense(box, level, tree.r0, p, 0.1, qq, centre=tree.centre)
        b = m2l.m2l_svd(box, level, tree.r0, f, qq)
        assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-13


def test_svd_m2l_output_error_bound():
    # per target: ||p_svd - p_dense|| <= s_l * (sigma_r + lambda_r) * sum_s ||q_s||
    pts, tree, q, p = _small_case()
    f = m2l.svd_factors(p, 0.1, 1e-4)
    rng = np.random.default_rng(3)
    level = 3
    box = tree.levels[level]
    qq = rng.standard_normal((box.shape[0], f.U.shape[0]))
    a = m2l.m2l_dense(box, level, tree.r0, p, 0.1, qq, centre=tree.centre)
    b = m2l.m2l_svd(box, level, tree.r0, f, qq)
    tg, sr, _ = geo.interaction_lists(box)
    qn = np.linalg.norm(qq, axis=1)
    bound = m2l.level_scale(level, tree.r0) * (f.sigma[f.r] + f.lam[f.r]) * np.bincount(tg, weights=qn[sr])
    err = np.linalg.norm(a - b, axis=1)
    assert np.all(err <= bound * (1 + 1e-9))
    assert err.max() > 1e-3 * bound.max()


def test_svd_m2l_targets_matches_full():
    pts, tree, q, p = _small_case()
    f = m2l.svd_factors(p, 0.1, 1e-6)
    rng = np.random.default_rng(4)
    box = tree.levels[3]
    qq = rng.standard_normal((box.shape[0], 2, f.U.shape[0]))
    full = m2l.m2l_svd(box, 3, tree.r0, f, qq)
    tg = [0, 7, box.shape[0] - 1]
    one = m2l.m2l_svd_targets(box, 3, tree.r0, f, qq, tg)
    np.testing.assert_allclose(one, full[tg], rtol=1e-12, atol=1e-12 * np.abs(full).max())


def test_adjoint_dot_product_and_linearity():
    pts, tree, q, p = _small_case()
    f = m2l.svd_factors(p, 0.1, 1e-4)
    assert f.r < f.U.shape[0]
    rng = np.random.default_rng(5)
    box = tree.levels[3]
    n = f.U.shape[0]
    x = rng.standard_normal((box.shape[0], n))
    y = rng.standard_normal((box.shape[0], n))
    ax = m2l.m2l_svd(box, 3, tree.r0, f, x)
    aty = m2l.m2l_svd_adjoint(box, 3, tree.r0, f, y)
    lhs, rhs = np.sum(ax * y), np.sum(x * aty)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(ax) * np.linalg.norm(y)
    # linearity
    a2 = m2l.m2l_svd(box, 3, tree.r0, f, 2.0 * x - 3.0 * y)
    np.testing.assert_allclose(a2, 2.0 * ax - 3.0 * m2l.m2l_svd(box, 3, tree.r0, f, y),
                               rtol=1e-11, atol=1e-11 * np.abs(a2).max())
    # the whole compressed M2L is (nearly) symmetric because K_o^T = K_{-o}
    assert np.linalg.norm(aty - m2l.m2l_svd(box, 3, tree.r0, f, y)) <= 1e-6 * np.linalg.norm(aty)


def test_translation_invariance_of_root_cube():
    # moving the root cube moves every surface with it: p^d is unchanged
    pts, tree, q, p = _small_case()
    box = tree.levels[3]
    rng = np.random.default_rng(6)
    qq = rng.standard_normal((box.shape[0], 56))
    a = m2l.m2l_dense(box, 3, tree.r0, p, 0.1, qq, centre=np.array([0.5, 0.5, 0.5]))
    b = m2l.m2l_dense(box, 3, tree.r0, p, 0.1, qq, centre=np.array([10.5, -3.5, 0.25]))
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12 * np.abs(a).max())


# ---------------------------------------------------------------------------
# stage 2 (Sec. 3.2)
# ---------------------------------------------------------------------------
def test_stage2_error_bounds(oracle_factors):
    f = oracle_factors(4, 0.1, 1e-6)
    eps1 = 1e-6
    eps2 = m2l.eps2_from_c2(10.0, eps1, f.r)
    assert eps2 == pytest.approx(10.0 * eps1 / f.r)
    fac = m2l.stage2_factors(f, eps2)
    thr = eps2 * f.sigma[0]
    diffs = []
    for (uh, vh), Ck in zip(fac, f.C):
        d2 = np.linalg.norm(uh @ vh - Ck, 2)
        assert d2 <= thr * (1 + 1e-9) + 1e-14 * f.sigma[0]     # per-offset bound
        assert np.abs(uh @ vh - Ck).max() <= thr * (1 + 1e-9) + 1e-14 * f.sigma[0]  # max-norm bound
        diffs.append(uh @ vh - Ck)
    fat = np.concatenate(diffs, axis=1)
    assert np.linalg.norm(fat, 2) <= eps2 * np.sqrt(316 * f.r ** 2) * f.sigma[0]
    ranks = [uh.shape[1] for uh, _ in fac]
    assert max(ranks) <= f.r and min(ranks) < f.r  # stage 2 does reduce ranks


def test_eps1_formula():
    assert m2l.eps1_from_c1(0.1, 6) == pytest.approx(0.1 * 2.0 ** -6 / 6)


def _stage2_case():
    pts, tree, q, p = _small_case(n=4000, p=4)
    box = tree.levels[3]
    rng = np.random.default_rng(11)
    qq = rng.standard_normal((box.shape[0], 2, 6 * (p - 1) ** 2 + 2))
    return tree, box, qq, p


def test_stage2_m2l_reduces_to_stage1_without_truncation(oracle_factors):
    # eps2 below every singular value of every core: Uhat_o Vhat_o = K~_o and
    # the two-product form equals the single-stage compressed M2L
    tree, box, qq, p = _stage2_case()
    f = oracle_factors(p, 0.1, 1e-6)
    fac = m2l.stage2_factors(f, 1e-300)
    a = m2l.m2l_svd_stage2(box, 3, tree.r0, f, fac, qq)
    b = m2l.m2l_svd(box, 3, tree.r0, f, qq)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_stage2_m2l_error_bound(oracle_factors):
    # per target t: |p_s2 - p_1| <= s_l |U~|_2 sum_s sigma_{k_o+1}(K~_o) |q~_s|
    # with |U~|_2 = 1 and sigma_{k_o+1} < eps2 sigma_0 (Eq. (17) truncation)
    tree, box, qq, p = _stage2_case()
    f = oracle_factors(p, 0.1, 1e-6)
    eps2 = 3e-4
    fac = m2l.stage2_factors(f, eps2)
    assert min(uh.shape[1] for uh, _ in fac) < f.r
    a = m2l.m2l_svd_stage2(box, 3, tree.r0, f, fac, qq)
    b = m2l.m2l_svd(box, 3, tree.r0, f, qq)
    tg, sr, ok = geo.interaction_lists(box)
    qt = qq @ f.R
    sl = m2l.level_scale(3, tree.r0)
    bound = np.zeros(box.shape[0])
    for t, s in zip(tg, sr):
        bound[t] += sl * eps2 * f.sigma[0] * np.linalg.norm(qt[s])
    err = np.linalg.norm(a - b, axis=2).max(axis=1) if a.ndim == 3 else np.linalg.norm(a - b, axis=1)
    assert np.all(err <= bound * (1 + 1e-9) + 1e-13 * np.abs(b).max())
    assert err.max() > 0  # the truncation is visible


def test_stage2_adjoint_is_the_transpose(oracle_factors):
    tree, box, qq, p = _stage2_case()
    f = oracle_factors(p, 0.1, 1e-6)
    fac = m2l.stage2_factors(f, m2l.eps2_from_c2(10.0, 1e-6, f.r))
    rng = np.random.default_rng(12)
    y = rng.standard_normal(qq.shape)
    ax = m2l.m2l_svd_stage2(box, 3, tree.r0, f, fac, qq)
    aty = m2l.m2l_svd_stage2_adjoint(box, 3, tree.r0, f, fac, y)
    lhs, rhs = float(np.sum(ax * y)), float(np.sum(qq * aty))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(ax) * np.linalg.norm(y)
