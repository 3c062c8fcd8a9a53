"""GPU parity of the point-source evaluation (kifmm_fmm_*: near field plus
the far field through S~, M~, M2L, L~, T~ of Sec. 3.3) against the FP64
oracle (``oracle.fmm``), called through the C ABI.

Tolerances (relative L2 over the compared points):
  against the oracle's compressed FMM, same operators:
    near field     1e-6   FP32 sums over coordinates relative to the leaf
                          centre (~1e-7 per term)
    far field      2e-6 of the far field's own norm: S~ and T~ carry
                   entries up to ~3e6 (p = 8) from the check-to-equivalent
                   pseudo-inverse; an FP32 evaluation of them was simulated
                   at 3e-7 of the total potential
    total          1e-6   (split6 and f16x3; split3 3e-5, bf16 1e-2 as for the
                          M2L)
  against the direct sum (Eq. (1)): the method's own error (p = 8,
  eps = 1e-7: ~1e-7 in FP64) plus the above, 1e-6.
"""
import os
import tempfile

import numpy as np
import pytest

import synth
from oracle import fmm as ofmm
from oracle import m2l as om

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

D = 0.1
TOL = {"split6": 1e-6, "f16x3": 1e-6, "split3": 3e-5, "bf16": 1e-2}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    os.environ.setdefault("KIFMM_M2L_CACHE", tempfile.mkdtemp(prefix="kifmm_cache_"))
    from paper_1211_2517_gb300 import build

    build.build()
    import paper_1211_2517_gb300 as pkg

    return pkg


def oracle_parts(tree, pts, q, p, eps):
    f = om.svd_factors(p, D, eps)
    ops = ofmm.pass_operators(f, p, D)
    return ofmm.near_field(tree, pts, q), ofmm.fmm_compressed_far(tree, pts, f, ops, p, D, q)


@pytest.fixture(scope="module")
def cube_case():
    """16384 points uniform in the unit cube, depth 3, p = 6."""
    wl = synth.workload("cube16k_p6")
    near, far = oracle_parts(wl.tree, wl.points, wl.densities, 6, 1e-7)
    return wl, near, far


@pytest.fixture(scope="module")
def sphere_case():
    """65536 points on the unit sphere (bounding-cube root, empty boxes,
    ragged leaves), depth 5, p = 8, N(0,1) densities."""
    pts = synth.points_sphere(65_536, 11)
    q = synth.densities_normal(65_536, 12)
    tree = synth.build_tree(pts, 5)
    near, far = oracle_parts(tree, pts, q, 8, 1e-7)
    return pts, q, tree, near, far


def run(g, plan, pts, q, depth, centre=None, r0=None, parts=3):
    tree = g.PointFMM(plan, pts, depth, centre=centre, r0=r0)
    out = tree.evaluate(torch.tensor(q, dtype=torch.float32, device="cuda"), parts)
    torch.cuda.synchronize()
    return tree, out.cpu().numpy().astype(np.float64)


def test_cube_matches_oracle_by_part(g, cube_case):
    wl, near, far = cube_case
    plan = g.M2LPlan(6, 1e-7, D, "split6")
    c, r0 = wl.tree.centre, wl.tree.r0
    tree, got = run(g, plan, wl.points, wl.densities, 3, c, r0)
    info = tree.info()
    assert info["leaves"] == wl.tree.levels[3].shape[0] and info["depth"] == 3
    assert info["boxes"] == sum(wl.tree.levels[l].shape[0] for l in (2, 3))
    _, got_near = run(g, plan, wl.points, wl.densities, 3, c, r0, parts=1)
    _, got_far = run(g, plan, wl.points, wl.densities, 3, c, r0, parts=2)
    e_all, e_near, e_far = rel(got, near + far), rel(got_near, near), rel(got_far, far)
    print(f"cube16k p=6: total {e_all:.3e} near {e_near:.3e} far {e_far:.3e}")
    assert e_near < 1e-6 and e_far < 1e-6 and e_all < 1e-6


def test_sphere_ragged_matches_oracle(g, sphere_case):
    pts, q, otree, near, far = sphere_case
    plan = g.M2LPlan(8, 1e-7, D, "split6")
    tree, got = run(g, plan, pts, q, 5)
    _, got_far = run(g, plan, pts, q, 5, parts=2)
    info = tree.info()
    want_pairs = sum(len(ofmm.geo.interaction_lists(otree.levels[l])[0]) for l in range(2, 6))
    assert info["m2l_pairs"] == want_pairs
    e_all, e_far = rel(got, near + far), rel(got_far, far)
    print(f"sphere65k p=8: total {e_all:.3e} far {e_far:.3e} ({info})")
    assert e_far < 1e-6 and e_all < 1e-6


def test_sphere_f16x3_matches_oracle(g, sphere_case):
    """The f16x3 core (per-box scaled FP16 pieces of every level's q~) on the
    ragged sphere tree: far field and total against the oracle."""
    pts, q, _, near, far = sphere_case
    plan = g.M2LPlan(8, 1e-7, D, "f16x3")
    _, got = run(g, plan, pts, q, 5)
    _, got_far = run(g, plan, pts, q, 5, parts=2)
    e_all, e_far = rel(got, near + far), rel(got_far, far)
    print(f"sphere65k p=8 f16x3: total {e_all:.3e} far {e_far:.3e}")
    assert e_far < 1e-6 and e_all < TOL["f16x3"]


def test_sphere_matches_direct_sum(g, sphere_case):
    pts, q, _, _, _ = sphere_case
    plan = g.M2LPlan(8, 1e-7, D, "split6")
    _, got = run(g, plan, pts, q, 5)
    targets = np.random.default_rng(5).choice(pts.shape[0], 400, replace=False)
    exact = ofmm.direct_sum(pts, q, targets)
    e = rel(got[targets], exact)
    print(f"sphere65k p=8 against the direct sum at 400 points: {e:.3e}")
    assert e < 1e-6


@pytest.mark.parametrize("precision", ["f16x3", "split3", "bf16"])
def test_core_precisions(g, cube_case, precision):
    wl, near, far = cube_case
    plan = g.M2LPlan(6, 1e-7, D, precision)
    _, got = run(g, plan, wl.points, wl.densities, 3, wl.tree.centre, wl.tree.r0)
    e = rel(got, near + far)
    print(f"cube16k p=6 {precision}: total {e:.3e}")
    assert e < TOL[precision]


def test_symmetry_and_gradient(g, sphere_case):
    pts, q, _, _, _ = sphere_case
    plan = g.M2LPlan(8, 1e-7, D, "split6")
    tree = g.PointFMM(plan, pts, 5)
    qt = torch.tensor(q, dtype=torch.float32, device="cuda", requires_grad=True)
    w = torch.tensor(synth.densities_uniform(pts.shape[0], 13), dtype=torch.float32, device="cuda")
    pot = g.fmm_potential(tree, qt)
    (pot * w).sum().backward()
    aw = tree.evaluate(w)
    torch.cuda.synchronize()
    # the core's scatter adds in arrival order: equal up to FP32 rounding
    assert rel(qt.grad.cpu().numpy(), aw.cpu().numpy().astype(np.float64)) < 1e-6
    lhs = float(torch.dot(pot.detach().double(), w.double()))
    rhs = float(torch.dot(qt.detach().double(), aw.double()))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_edge_cases(g):
    plan = g.M2LPlan(6, 1e-7, D, "split6")
    # one point: nothing acts on it
    _, got = run(g, plan, np.array([[0.3, 0.2, 0.1]]), np.array([2.0]), 2)
    assert got[0] == 0.0
    # two points in one leaf: the closed form
    pts = np.array([[0.1, 0.1, 0.1], [0.15, 0.1, 0.1]])
    _, got = run(g, plan, pts, np.array([1.0, -2.0]), 3, np.array([0.5, 0.5, 0.5]), 0.5)
    np.testing.assert_allclose(got, [-2.0 / (4 * np.pi * 0.05), 1.0 / (4 * np.pi * 0.05)], rtol=2e-6)
    # depth 2 (M2L on level 2 only, no L2L), points on the faces of the root cube
    pts = synth.points_uniform_cube(3000, 21)
    pts[:40, 0] = 1.0
    pts[40:80, 2] = 0.0
    q = synth.densities_uniform(3000, 22)
    tree = synth.build_tree(pts, 2, centre=np.array([0.5, 0.5, 0.5]), r0=0.5)
    near, far = oracle_parts(tree, pts, q, 6, 1e-7)
    _, got = run(g, plan, pts, q, 2, np.array([0.5, 0.5, 0.5]), 0.5)
    assert rel(got, near + far) < 1e-6


@pytest.fixture(scope="module")
def sphere_dl_case(sphere_case):
    """The 65,536-point sphere with its outward normals as dipole sources
    (the double layer of Sec. 4, Eq. (26)): the oracle's near field
    and compressed far field at p = 8."""
    pts, q, tree, _, _ = sphere_case
    nrm = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    f = om.svd_factors(8, D, 1e-7)
    ops = ofmm.pass_operators(f, 8, D)
    near = ofmm.near_field(tree, pts, q, normals=nrm)
    far = ofmm.fmm_compressed_far(tree, pts, f, ops, 8, D, q, normals=nrm)
    return pts, q, nrm, near, far


@pytest.mark.parametrize("precision", ["split6", "f16x3"])
def test_double_layer_matches_oracle(g, sphere_case, sphere_dl_case, precision):
    """Near field (n . d by the compensated dot product on two-word normals)
    and far field (per-point S~ rows of the dipoles and T~ rows of the
    targets, formed in FP64 and applied in FP32) within 1e-6 of the oracle,
    each of its own norm, and the total within 1e-6.  Against the direct
    double-layer sum the bound is the oracle's own distance to it (the
    method's FP64 error at p = 8 on these points) plus 1e-6."""
    pts, q, nrm, near, far = sphere_dl_case
    plan = g.M2LPlan(8, 1e-7, D, precision)
    tree = g.PointFMM(plan, pts, 5, normals=nrm)
    qd = torch.tensor(q, dtype=torch.float32, device="cuda")
    got = {k: tree.evaluate(qd, k).cpu().numpy().astype(np.float64) for k in (1, 2, 3)}
    e_near, e_far, e_all = rel(got[1], near), rel(got[2], far), rel(got[3], near + far)
    targets = np.random.default_rng(6).choice(pts.shape[0], 400, replace=False)
    direct = ofmm.direct_sum(pts, q, targets, normals=nrm)
    e_direct = rel(got[3][targets], direct)
    e_method = rel((near + far)[targets], direct)
    print(f"sphere65k double layer {precision}: near {e_near:.3e} far {e_far:.3e} total {e_all:.3e} "
          f"direct {e_direct:.3e} (oracle vs direct {e_method:.3e})")
    assert e_near < 1e-6 and e_far < 1e-6 and e_all < 1e-6 and e_direct < e_method + 1e-6
    # back to point charges on the same tree
    tree.set_normals(None)
    single = tree.evaluate(qd).cpu().numpy().astype(np.float64)
    _, _, _, sl_near, sl_far = sphere_case
    assert rel(single, sl_near + sl_far) < 1e-6
    # the double-layer operator is not symmetric: no gradient through it
    tree.set_normals(nrm)
    qt = qd.clone().requires_grad_(True)
    with pytest.raises(NotImplementedError):
        g.fmm_potential(tree, qt).sum().backward()


def test_double_layer_edge_cases(g):
    plan = g.M2LPlan(6, 1e-7, D, "split6")
    # two dipoles in one leaf: q_j n_j . (x_i - x_j) / (4 pi |x_i - x_j|^3)
    pts = np.array([[0.1, 0.1, 0.1], [0.15, 0.1, 0.1]])
    nrm = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    tree = g.PointFMM(plan, pts, 3, centre=np.array([0.5, 0.5, 0.5]), r0=0.5, normals=nrm)
    got = tree.evaluate(torch.tensor([1.0, -2.0], dtype=torch.float32, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(got, [2.0 / (0.01 * np.pi), 1.0 / (0.01 * np.pi)], rtol=2e-6)
    # random normals in the unit cube, depth 2 (no L2L), against the oracle
    pts = synth.points_uniform_cube(3000, 31)
    nrm = np.random.default_rng(32).standard_normal((3000, 3))
    q = synth.densities_uniform(3000, 33)
    otree = synth.build_tree(pts, 2, centre=np.array([0.5, 0.5, 0.5]), r0=0.5)
    f = om.svd_factors(6, D, 1e-7)
    want = ofmm.fmm_potential(otree, pts, q, 6, D, f=f, normals=nrm)
    tree = g.PointFMM(plan, pts, 2, centre=np.array([0.5, 0.5, 0.5]), r0=0.5, normals=nrm)
    got = tree.evaluate(torch.tensor(q, dtype=torch.float32, device="cuda")).cpu().numpy()
    err = rel(got, want)
    print(f"random dipoles in the cube, depth 2, p = 6: rel L2 {err:.3e}")
    assert err < 1e-6
    from paper_1211_2517_gb300 import KifmmError

    bad = nrm.copy()
    bad[5, 2] = np.inf
    with pytest.raises(KifmmError, match="INVALID_ARG"):
        tree.set_normals(bad)
    with pytest.raises(ValueError):
        tree.set_normals(nrm[:10])


def test_argument_errors(g):
    from paper_1211_2517_gb300 import KifmmError

    plan = g.M2LPlan(6, 1e-7, D, "split6")
    pts = synth.points_uniform_cube(100, 1)
    with pytest.raises(KifmmError, match="INVALID_ARG"):
        g.PointFMM(plan, pts, 1)
    bad = pts.copy()
    bad[7, 1] = np.nan
    with pytest.raises(KifmmError, match="INVALID_ARG"):
        g.PointFMM(plan, bad, 3)
    tree = g.PointFMM(plan, pts, 3)
    q = torch.zeros(100, dtype=torch.float32, device="cuda")
    with pytest.raises(KifmmError, match="INVALID_ARG"):
        tree.evaluate(q, parts=0)
    with pytest.raises(KifmmError, match="UNSUPPORTED"):
        g.PointFMM(g.M2LPlan(6, 1e-7, D, "fp32"), pts, 3)


def test_full_size_sphere2m_sampled(g):
    """The 2,097,152-point sphere at depth 6 (the M2L benchmark's tree): the
    GPU evaluation against the direct sum at sampled points, and its M2L pair
    count against the workload's."""
    wl = synth.workload("sphere2m_p8")
    plan = g.M2LPlan(8, 1e-7, D, "split6")
    tree, got = run(g, plan, wl.points, wl.densities, 6)
    assert tree.info()["m2l_pairs"] == 1_158_296
    targets = np.random.default_rng(9).choice(wl.points.shape[0], 48, replace=False)
    exact = np.concatenate([ofmm.direct_sum(wl.points, wl.densities, [t]) for t in targets])
    e = rel(got[targets], exact)
    print(f"sphere2m p=8 against the direct sum at 48 points: {e:.3e}")
    assert e < 1e-6
