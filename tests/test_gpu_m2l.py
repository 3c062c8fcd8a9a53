"""GPU parity of the compressed M2L (and its adjoint and dense baseline)
against the FP64 oracle, called through the C ABI.

Tolerances (relative L2 over all outputs of a level):
  fp32, split6 : 1e-6  (the gate; an FP32 pipeline lands at ~5e-7 because
                 V^T compression, core sums and U expansion each round)
  split3       : 3e-5  (2-piece BF16 split keeps ~16 significand bits)
  bf16         : 1e-2  (8 significand bits)
The oracle runs at the same eps, so both sides truncate at the same rank
and only rounding differs.
"""
import os
import tempfile

import numpy as np
import pytest

import synth
from oracle import geometry as geo
from oracle import m2l as om
from oracle import upward

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "split6": 1e-6, "split3": 3e-5, "bf16": 1e-2, "f16x3": 1e-6}


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


@pytest.fixture(scope="module")
def cube():
    """Uniform cube, 16384 points, depth 3, p = 6, eps = 1e-8, S2M/M2M inputs."""
    wl = synth.workload("cube16k_p6")
    qup = upward.upward_pass(wl.tree, wl.points, wl.p, wl.d, wl.densities)
    return wl, {l: qup[l].astype(np.float32) for l in (2, 3)}


@pytest.fixture(scope="module")
def sphere_small():
    """Sphere, 60000 points, depth 4, p = 8, eps = 1e-7 (random densities, 3 rhs)."""
    pts = synth.points_sphere(60_000, 7)
    tree = synth.build_tree(pts, 4)
    qs = {l: synth.random_box_densities(tree.levels[l].shape[0], 3, 296, 100 + l) for l in (2, 3, 4)}
    return tree, qs


def make_plan(g, p, eps, precision, tree, levels):
    plan = g.M2LPlan(p, eps, 0.1, precision)
    for l in levels:
        plan.set_level(l, tree.levels[l], tree.r0)
    return plan


@pytest.mark.parametrize("precision", ["fp32", "split6", "split3", "bf16", "f16x3"])
def test_compressed_parity_cube(g, oracle_factors, cube, precision):
    wl, qup = cube
    f = oracle_factors(wl.p, wl.d, wl.eps)
    plan = make_plan(g, wl.p, wl.eps, precision, wl.tree, (2, 3))
    assert plan.r == f.r
    for l in (2, 3):
        box = wl.tree.levels[l]
        ref = om.m2l_svd(box, l, wl.tree.r0, f, qup[l].astype(np.float64))
        out = plan.apply(torch.from_numpy(qup[l]).cuda(), l)
        plan.sync()
        err = rel(out.cpu().numpy(), ref)
        print(f"cube p=6 level {l} {precision}: rel L2 {err:.3e}")
        assert err <= TOL[precision], err


@pytest.mark.parametrize("precision", ["fp32", "split6", "split3", "f16x3"])
def test_compressed_parity_multi_rhs(g, oracle_factors, sphere_small, precision):
    tree, qs = sphere_small
    f = oracle_factors(8, 0.1, 1e-7)
    plan = make_plan(g, 8, 1e-7, precision, tree, (2, 3, 4))
    for l in (2, 3, 4):
        ref = om.m2l_svd(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64))
        out = plan.apply(torch.from_numpy(qs[l]).cuda(), l)
        plan.sync()
        err = rel(out.cpu().numpy(), ref)
        print(f"sphere p=8 level {l} nrhs=3 {precision}: rel L2 {err:.3e}")
        assert err <= TOL[precision], err


def test_dense_parity(g, cube):
    wl, qup = cube
    K = om.unit_m2l_matrices(wl.p, wl.d)
    plan = make_plan(g, wl.p, wl.eps, "fp32", wl.tree, (2, 3))
    for l in (2, 3):
        ref = om.m2l_dense_unit(wl.tree.levels[l], l, wl.tree.r0, K, qup[l].astype(np.float64))
        out = plan.apply_dense(torch.from_numpy(qup[l]).cuda(), l)
        plan.sync()
        err = rel(out.cpu().numpy(), ref)
        print(f"dense p=6 level {l}: rel L2 {err:.3e}")
        assert err <= 1e-6, err


def test_dense_tensor_core_parity(g, cube, sphere_small):
    """The uncompressed M2L on the tensor cores (f16x3 pieces of q^u and K_o,
    K = N = n_pad: p = 6 -> 160, p = 8 -> 304 in two N parts) against the
    oracle's FP64 dense M2L: cube levels 2-3 and sphere levels 2-4 with 3
    rhs, both beta rules."""
    wl, qup = cube
    K6 = om.unit_m2l_matrices(wl.p, wl.d)
    plan = make_plan(g, wl.p, wl.eps, "f16x3", wl.tree, (2, 3))
    for l in (2, 3):
        ref = om.m2l_dense_unit(wl.tree.levels[l], l, wl.tree.r0, K6, qup[l].astype(np.float64))
        out = plan.apply_dense_tc(torch.from_numpy(qup[l]).cuda(), l)
        plan.sync()
        err = rel(out.cpu().numpy(), ref)
        print(f"dense tensor-core p=6 level {l}: rel L2 {err:.3e}")
        assert err <= 1e-6, err
    plan.close()
    tree, qs = sphere_small
    K8 = om.unit_m2l_matrices(8, 0.1)
    plan = make_plan(g, 8, 1e-7, "f16x3", tree, (2, 3, 4))
    for l in (2, 3, 4):
        ref = om.m2l_dense_unit(tree.levels[l], l, tree.r0, K8, qs[l].astype(np.float64))
        x = torch.from_numpy(qs[l]).cuda()
        out = plan.apply_dense_tc(x, l)
        plan.sync()
        err = rel(out.cpu().numpy(), ref)
        prev = torch.randn_like(out)
        acc = prev.clone()
        plan.apply_dense_tc(x, l, out=acc, beta=1.0)
        plan.sync()
        err_b = rel((acc - prev).cpu().numpy(), ref)
        print(f"dense tensor-core p=8 level {l} (3 rhs): rel L2 {err:.3e}, accumulate {err_b:.3e}")
        assert err <= 1e-6 and err_b <= 1e-6, (err, err_b)
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split6", "f16x3"])
def test_adjoint_parity_and_dot_product(g, oracle_factors, sphere_small, precision):
    tree, qs = sphere_small
    f = oracle_factors(8, 0.1, 1e-7)
    plan = make_plan(g, 8, 1e-7, precision, tree, (3, 4))
    rng = np.random.default_rng(9)
    for l in (3, 4):
        y = rng.standard_normal(qs[l].shape).astype(np.float32)
        ref = om.m2l_svd_adjoint(tree.levels[l], l, tree.r0, f, y.astype(np.float64))
        x = torch.from_numpy(qs[l]).cuda()
        yt = torch.from_numpy(y).cuda()
        aty = plan.apply_adjoint(yt, l)
        ax = plan.apply(x, l)
        plan.sync()
        err = rel(aty.cpu().numpy(), ref)
        print(f"adjoint level {l} {precision}: rel L2 {err:.3e}")
        assert err <= TOL[precision], err
        lhs = float((ax.double() * yt.double()).sum())
        rhs = float((x.double() * aty.double()).sum())
        assert abs(lhs - rhs) <= 1e-5 * ax.double().norm().item() * yt.double().norm().item()


def test_beta_accumulates(g, cube):
    wl, qup = cube
    plan = make_plan(g, wl.p, wl.eps, "split6", wl.tree, (3,))
    x = torch.from_numpy(qup[3]).cuda()
    base = plan.apply(x, 3)
    prev = torch.randn_like(base)
    out = prev.clone()
    plan.apply(x, 3, out=out, beta=0.5)
    plan.sync()
    torch.testing.assert_close(out, 0.5 * prev + base, rtol=1e-5, atol=1e-5 * base.abs().max().item())
    dense = plan.apply_dense(x, 3)
    out2 = prev.clone()
    plan.apply_dense(x, 3, out=out2, beta=1.0)
    plan.sync()
    torch.testing.assert_close(out2, prev + dense, rtol=1e-5, atol=1e-5 * dense.abs().max().item())


def test_edge_cases(g):
    from paper_1211_2517_gb300._lib import KifmmError

    plan = g.M2LPlan(4, 1e-4, 0.1, "split6")
    n = plan.n
    # empty level
    plan.set_level(2, np.zeros((0, 3), np.int32), 1.0)
    out = plan.apply(torch.zeros((0, n), device="cuda"), 2)
    assert out.shape == (0, n)
    # a single box has no interaction partners: output zero
    plan.set_level(3, np.array([[3, 4, 5]]), 1.0)
    out = plan.apply(torch.randn(1, n, device="cuda"), 3)
    plan.sync()
    assert torch.count_nonzero(out).item() == 0
    # apply before set_level
    with pytest.raises(KifmmError):
        plan.apply(torch.zeros((4, n), device="cuda"), 5)
    # wrong shape is caught before the call
    with pytest.raises(ValueError):
        plan.apply(torch.zeros((2, n), device="cuda"), 3)


def test_autograd_central_differences(g, oracle_factors):
    """Loss 0.5 ||A q - phi||^2 w.r.t. the densities q (sphere, p = 8)."""
    from paper_1211_2517_gb300.autograd import m2l

    pts = synth.points_sphere(80_000, 21)
    tree = synth.build_tree(pts, 4)
    l = 4
    plan = make_plan(g, 8, 1e-7, "split6", tree, (l,))
    nb = tree.levels[l].shape[0]
    rng = np.random.default_rng(22)
    q = torch.from_numpy(rng.standard_normal((nb, 296)).astype(np.float32)).cuda().requires_grad_(True)
    phi = torch.from_numpy(rng.standard_normal((nb, 296)).astype(np.float32)).cuda()

    def loss(x):
        return 0.5 * ((m2l(x, plan, l).double() - phi.double()) ** 2).sum()

    L = loss(q)
    L.backward()
    grad = q.grad.double()
    # against the oracle's transpose product A^T (A q - phi)
    f = oracle_factors(8, 0.1, 1e-7)
    box = tree.levels[l]
    qn = q.detach().cpu().numpy().astype(np.float64)
    resid = om.m2l_svd(box, l, tree.r0, f, qn) - phi.cpu().numpy()
    gref = om.m2l_svd_adjoint(box, l, tree.r0, f, resid)
    assert rel(grad.cpu().numpy(), gref) < 1e-5
    # Central differences, h = 1e-3, along seeded directions v = g/rms(g) + z/2
    # (z ~ N(0,1)): O(1) entries survive FP32 rounding of q + h v, and the
    # gradient component keeps <grad L, v> well above the rounding noise of
    # the FP32 forward (the loss is quadratic: only rounding separates them).
    h = 1e-3
    gdir = grad.float() / grad.float().pow(2).mean().sqrt()
    for j in range(8):
        z = torch.from_numpy(rng.standard_normal((nb, 296)).astype(np.float32)).cuda()
        v = gdir + 0.5 * z
        with torch.no_grad():
            lp = float(loss(q + h * v))
            lm = float(loss(q - h * v))
        fd = (lp - lm) / (2 * h)
        an = float((grad * v.double()).sum())
        assert abs(fd - an) <= 1e-3 * abs(an), (fd, an)


@pytest.fixture(scope="module")
def sphere1m_upward():
    """The 1,048,576-point sphere at depth 5 with its upward-equivalent
    densities from the oracle's S2M/M2M of the U[-1,1] point densities."""
    wl = synth.workload("sphere1m_p8")
    qup = upward.upward_pass(wl.tree, wl.points, wl.p, wl.d, wl.densities)
    return wl, {l: qup[l].astype(np.float32) for l in range(2, 6)}


@pytest.mark.parametrize("precision", ["fp32", "split6"])
def test_full_size_adjoint_autograd_sphere1m(g, oracle_factors, sphere1m_upward, precision):
    """Loss 0.5 ||phi - phi_t||^2, phi = M2L(q^u) over levels 2..5 of the
    1,048,576-point sphere at depth 5 (p = 8, eps = 1e-7, phi_t ~ N(0,1),
    q^u from S2M/M2M of the point densities), differentiated through the
    levels-batch autograd Function: the gradient against the oracle's
    transpose product (C_k^T on the reversed offsets), then central
    differences with h = 1e-3 along 8 seeded directions."""
    from paper_1211_2517_gb300.autograd import m2l_levels

    wl, qup = sphere1m_upward
    tree = wl.tree
    levels = range(2, 6)
    plan = make_plan(g, 8, 1e-7, precision, tree, levels)
    nbs = [tree.levels[l].shape[0] for l in levels]
    rng = np.random.default_rng(55)
    q0 = np.concatenate([qup[l] for l in levels])
    phi_t = rng.standard_normal(q0.shape).astype(np.float32)
    q = torch.from_numpy(q0).cuda().requires_grad_(True)
    phit = torch.from_numpy(phi_t).cuda()

    def loss(x):
        return 0.5 * ((m2l_levels(x, plan, 2, 5).double() - phit.double()) ** 2).sum()

    L = loss(q)
    L.backward()
    grad = q.grad.double()
    f = oracle_factors(8, 0.1, 1e-7)
    gn = grad.cpu().numpy()
    row = 0
    for nb, l in zip(nbs, levels):
        box = tree.levels[l]
        sl = slice(row, row + nb)
        resid = om.m2l_svd(box, l, tree.r0, f, q0[sl].astype(np.float64)) - phi_t[sl]
        gref = om.m2l_svd_adjoint(box, l, tree.r0, f, resid)
        err = rel(gn[sl], gref)
        print(f"sphere1m {precision} level {l}: gradient rel L2 {err:.3e}")
        assert err <= 1e-5, err
        row += nb
    # Directions with O(1) entries (the gradient's direction, scaled to unit
    # RMS, plus seeded N(0,1)/2): a unit-norm direction would move each of
    # the 1.9M FP32 entries by ~1e-9, below their resolution.
    h = 1e-3
    gdir = grad.float() / grad.float().pow(2).mean().sqrt()
    for j in range(8):
        z = torch.from_numpy(rng.standard_normal(q0.shape).astype(np.float32)).cuda()
        v = gdir + 0.5 * z
        with torch.no_grad():
            lp = float(loss(q + h * v))
            lm = float(loss(q - h * v))
        fd = (lp - lm) / (2 * h)
        an = float((grad * v.double()).sum())
        print(f"sphere1m {precision} direction {j}: fd {fd:.9e} analytic {an:.9e}")
        assert abs(fd - an) <= 1e-3 * abs(an), (fd, an)
    plan.close()


def test_full_size_sphere_sampled(g, oracle_factors):
    """The 2M-point sphere at depth 6, p = 8, eps = 1e-7 (the benchmark
    workload, split6), every level, on sampled targets the oracle computes
    one by one."""
    wl = synth.workload("sphere2m_p8")
    tree = wl.tree
    f = oracle_factors(8, 0.1, 1e-7)
    plan = make_plan(g, 8, 1e-7, "split6", tree, range(2, 7))
    rng = np.random.default_rng(5)
    for l in range(2, 7):
        nb = tree.levels[l].shape[0]
        q = synth.random_box_densities(nb, 1, 296, 300 + l)[:, 0, :]
        out = plan.apply(torch.from_numpy(q).cuda(), l)
        plan.sync()
        tg = np.sort(rng.choice(nb, size=min(24, nb), replace=False))
        ref = om.m2l_svd_targets(tree.levels[l], l, tree.r0, f, q.astype(np.float64), tg)[:, 0, :]
        err = rel(out.cpu().numpy()[tg], ref)
        print(f"sphere2m level {l}: sampled rel L2 {err:.3e}")
        assert err <= 1e-6, err


@pytest.mark.parametrize("precision", ["split6", "fp32", "f16x3"])
def test_levels_batch_parity(g, oracle_factors, sphere_small, precision):
    """kifmm_m2l_apply_levels (levels 2..4 in one batch, 3 rhs) against the
    oracle on every level, forward and adjoint."""
    tree, qs = sphere_small
    f = oracle_factors(8, 0.1, 1e-7)
    plan = make_plan(g, 8, 1e-7, precision, tree, (2, 3, 4))
    x_all = torch.from_numpy(np.concatenate([qs[l] for l in (2, 3, 4)])).cuda()
    for adjoint in (False, True):
        out = plan.apply_levels(x_all, 2, 4, adjoint=adjoint)
        plan.sync()
        o = out.cpu().numpy()
        row = 0
        for l in (2, 3, 4):
            nb = tree.levels[l].shape[0]
            fn = om.m2l_svd_adjoint if adjoint else om.m2l_svd
            ref = fn(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64))
            err = rel(o[row:row + nb], ref)
            print(f"levels batch {precision} adjoint={adjoint} level {l}: rel L2 {err:.3e}")
            assert err <= TOL[precision], err
            row += nb
    # re-registering a level invalidates the merged batch state
    plan.set_level(3, tree.levels[3], tree.r0)
    out2 = plan.apply_levels(x_all, 2, 4)
    plan.sync()
    ref_all = plan.apply_levels(x_all, 2, 4)
    plan.sync()
    assert rel(out2.cpu().numpy(), ref_all.cpu().numpy().astype(np.float64)) < 1e-6


def test_full_size_sphere_f16x3_sampled(g, oracle_factors):
    """The benchmark workload (2M-point sphere, depth 6, p = 8, eps = 1e-7) in
    the FP16 split with per-box scaling, all levels in one batch, forward and
    adjoint, on sampled targets the oracle computes one by one."""
    wl = synth.workload("sphere2m_p8")
    tree = wl.tree
    f = oracle_factors(8, 0.1, 1e-7)
    plan = make_plan(g, 8, 1e-7, "f16x3", tree, range(2, 7))
    qs = {l: synth.random_box_densities(tree.levels[l].shape[0], 1, 296, 900 + l)[:, 0] for l in range(2, 7)}
    x_all = torch.from_numpy(np.concatenate([qs[l] for l in range(2, 7)])).cuda()
    rng = np.random.default_rng(6)
    out = plan.apply_levels(x_all, 2, 6).cpu().numpy()
    plan.sync()
    row = 0
    for l in range(2, 7):
        nb = tree.levels[l].shape[0]
        tg = np.sort(rng.choice(nb, size=min(24, nb), replace=False))
        ref = om.m2l_svd_targets(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64), tg)[:, 0, :]
        err = rel(out[row:row + nb][tg], ref)
        print(f"sphere2m f16x3 level {l}: sampled rel L2 {err:.3e}")
        assert err <= 1e-6, err
        row += nb


def test_f16x3_scaling_extremes(g, oracle_factors, sphere_small):
    """Per-box scaling keeps FP16 accuracy when box densities span 30 orders
    of magnitude (and for all-zero boxes): each level's rows are scaled by
    10^k, k from -15 to 15, some rows zero."""
    tree, qs = sphere_small
    f = oracle_factors(8, 0.1, 1e-7)
    plan = make_plan(g, 8, 1e-7, "f16x3", tree, (3,))
    q = qs[3].astype(np.float64).copy()
    rng = np.random.default_rng(12)
    q *= 10.0 ** rng.integers(-15, 16, size=(q.shape[0], 1, 1))
    q[::17] = 0.0
    out = plan.apply(torch.from_numpy(q.astype(np.float32)).cuda(), 3).cpu().numpy()
    plan.sync()
    ref = om.m2l_svd(tree.levels[3], 3, tree.r0, f, q.astype(np.float32).astype(np.float64))
    # judge each target against the size of its own potential: the scales differ by 1e30
    for t in rng.choice(q.shape[0], 64, replace=False):
        if np.linalg.norm(ref[t]) > 0:
            assert rel(out[t], ref[t]) <= 1e-5, t
    err = rel(out, ref)
    print(f"f16x3 with 1e-15..1e15 box scales: rel L2 {err:.3e}")
    assert err <= 1e-6


@pytest.mark.parametrize("precision", ["f16x3", "split6"])
def test_apply_levels_host_matches_device(g, sphere_small, precision):
    """kifmm_m2l_apply_levels_host (host buffers, chunked copies overlapping
    the compression and expansion) against kifmm_m2l_apply_levels on device
    buffers, levels 2-4 with 3 right-hand sides, beta = 0 and beta = 1 (the
    latter doubles the host array); pinned and pageable host memory."""
    tree, qs = sphere_small
    plan = make_plan(g, 8, 1e-7, precision, tree, (2, 3, 4))
    x = np.concatenate([qs[l] for l in (2, 3, 4)]).astype(np.float32)
    ref = plan.apply_levels(torch.from_numpy(x).cuda(), 2, 4).cpu()
    torch.cuda.synchronize()
    for pin in (True, False):
        hx = torch.from_numpy(x.copy())
        hp = torch.full_like(hx, float("nan"))
        if pin:
            hx, hp = hx.pin_memory(), hp.pin_memory()
        plan.apply_levels_host(hx, 2, 4, out=hp)
        plan.sync()
        err = float((hp - ref).double().norm() / ref.double().norm())
        print(f"host apply {precision} pinned={pin}: rel L2 against the device apply {err:.3e}")
        assert err < 1e-6, err
        plan.apply_levels_host(hx, 2, 4, out=hp, beta=1.0)
        plan.sync()
        err2 = float((hp - 2 * ref).double().norm() / (2 * ref).double().norm())
        assert err2 < 1e-6, err2
    plan.close()


def test_f16x3_unsupported_paths(g, sphere_small):
    """The allocation-free apply refuses f16x3 plans (its rows-mode kernels
    have no per-row FP16 scaling); nothing is written."""
    import ctypes

    tree, qs = sphere_small
    plan = make_plan(g, 8, 1e-7, "f16x3", tree, (3,))
    x = torch.from_numpy(qs[3]).cuda()
    out = torch.full_like(x, 7.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = g.lib().kifmm_m2l_apply_noalloc(plan._h, 0, 3, 3, ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), 0.0, stream)
    torch.cuda.synchronize()
    assert st == -2  # KIFMM_ERR_UNSUPPORTED
    assert bool((out == 7.0).all())
    plan.close()


@pytest.fixture(scope="module")
def torus_mid():
    """Torus R=1, r=0.3, 300000 points, depth 5, p = 10, eps = 1e-8 (r = 271 > 256:
    the core runs two MMAs per K step)."""
    pts = synth.points_torus(300_000, 3)
    tree = synth.build_tree(pts, 5)
    qs = {l: synth.random_box_densities(tree.levels[l].shape[0], 1, 488, 500 + l)[:, 0] for l in range(2, 6)}
    return tree, qs


@pytest.mark.parametrize("precision", ["split6", "fp32", "f16x3"])
def test_p10_parity_levels_batch(g, oracle_factors, torus_mid, precision):
    tree, qs = torus_mid
    f = oracle_factors(10, 0.1, 1e-8)
    plan = make_plan(g, 10, 1e-8, precision, tree, range(2, 6))
    assert (plan.r, plan.r_pad, plan.n) == (f.r, 272, 488)
    x_all = torch.from_numpy(np.concatenate([qs[l] for l in range(2, 6)])).cuda()
    out = plan.apply_levels(x_all, 2, 5).cpu().numpy()
    plan.sync()
    row = 0
    for l in range(2, 6):
        nb = tree.levels[l].shape[0]
        ref = om.m2l_svd(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64))
        err = rel(out[row:row + nb], ref)
        print(f"torus p=10 {precision} level {l}: rel L2 {err:.3e}")
        assert err <= TOL[precision], err
        row += nb


def test_autotune_keeps_parity_and_caches(g, oracle_factors, torus_mid, monkeypatch, tmp_path):
    """kifmm_m2l_autotune on the p = 10 torus (four candidates: N chunk 144 or
    80, round-robin or contiguous items): whatever it keeps, apply_levels still
    matches the oracle; the choice is written to and read back from the JSON
    cache file."""
    import json

    tree, qs = torus_mid
    f = oracle_factors(10, 0.1, 1e-8)
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("KIFMM_M2L_AUTOTUNE_CACHE", str(cache))
    plan = make_plan(g, 10, 1e-8, "split6", tree, range(2, 6))
    x_all = torch.from_numpy(np.concatenate([qs[l] for l in range(2, 6)])).cuda()
    res = plan.autotune(x_all, 2, 5, reps=2)
    print("autotune", res)
    assert not res["from_cache"] and res["core_ms"] > 0
    assert res["n_chunk"] in (144, 80) and res["contiguous"] in (0, 1)
    entries = json.loads(cache.read_text())
    assert len(entries) == 1 and list(entries.values())[0]["n_chunk"] == res["n_chunk"]
    # every candidate is forced in turn through the cache file
    key = list(entries)[0]
    refs = {l: om.m2l_svd(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64)) for l in range(2, 6)}
    for chunk in (144, 80):
        for contig in (0, 1):
            cache.write_text('{\n"%s": {"n_chunk": %d, "contiguous": %d, "variant": 0, "core_ms": 1.0}\n}\n'
                             % (key, chunk, contig))
            got = plan.autotune(x_all, 2, 5, reps=1)
            assert got["from_cache"] and (got["n_chunk"], got["contiguous"]) == (chunk, contig), got
            out = plan.apply_levels(x_all, 2, 5).cpu().numpy()
            plan.sync()
            row = 0
            for l in range(2, 6):
                nb = tree.levels[l].shape[0]
                err = rel(out[row:row + nb], refs[l])
                print(f"autotune chunk {chunk} contiguous {contig} level {l}: rel L2 {err:.3e}")
                assert err <= TOL["split6"], (chunk, contig, l, err)
                row += nb
    plan.close()


def test_f16x3_core_variants_match_oracle(g, oracle_factors, sphere_small, monkeypatch, tmp_path):
    """The core variants an FP16-split plan can run (drained partials of
    three, two or one K-chunks, issued one, two or three chunks per MMA
    step, rows reduced through the transpose, without it or by TMA bulk
    reductions, the classic kernel with N = 192 or 96, round-robin or
    contiguous tiles) against the oracle, forward and adjoint."""
    tree, qs = sphere_small
    f = oracle_factors(8, 0.1, 1e-7)
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("KIFMM_M2L_AUTOTUNE_CACHE", str(cache))
    plan = make_plan(g, 8, 1e-7, "f16x3", tree, (2, 3, 4))
    x_all = torch.from_numpy(np.concatenate([qs[l] for l in (2, 3, 4)])).cuda()
    res = plan.autotune(x_all, 2, 4, reps=2)
    print("autotune f16x3", res)
    assert res["variant"] in (0, 2, 3, 4, 5, 6, 9, 10, 11, 12, 13)
    import json

    key = list(json.loads(cache.read_text()))[0]
    refs = {(l, adj): (om.m2l_svd_adjoint if adj else om.m2l_svd)(tree.levels[l], l, tree.r0, f,
                                                                   qs[l].astype(np.float64))
            for l in (2, 3, 4) for adj in (False, True)}
    for chunk, contig, variant in [(192, 0, 2), (192, 1, 2), (192, 0, 3), (192, 0, 4), (192, 1, 5), (192, 0, 6),
                                   (192, 1, 6), (192, 0, 9), (192, 0, 10), (192, 1, 10), (192, 0, 11), (192, 1, 11),
                                   (192, 0, 12), (192, 1, 12), (192, 1, 13), (192, 0, 0), (96, 1, 0)]:
        cache.write_text('{\n"%s": {"n_chunk": %d, "contiguous": %d, "variant": %d, "core_ms": 1.0}\n}\n'
                         % (key, chunk, contig, variant))
        got = plan.autotune(x_all, 2, 4, reps=1)
        assert got["from_cache"]
        for adj in (False, True):
            out = plan.apply_levels(x_all, 2, 4, adjoint=adj).cpu().numpy()
            plan.sync()
            row = 0
            for l in (2, 3, 4):
                nb = tree.levels[l].shape[0]
                err = rel(out[row:row + nb], refs[(l, adj)])
                print(f"f16x3 chunk {chunk} contiguous {contig} variant {variant} adjoint {adj} level {l}: "
                      f"rel L2 {err:.3e}")
                assert err <= TOL["f16x3"], (chunk, contig, variant, adj, l, err)
                row += nb
    plan.close()


def _force_variant(plan, x_all, lo, hi, cache, key, chunk, contig, variant):
    cache.write_text('{\n"%s": {"n_chunk": %d, "contiguous": %d, "variant": %d, "core_ms": 1.0}\n}\n'
                     % (key, chunk, contig, variant))
    got = plan.autotune(x_all, lo, hi, reps=1)
    assert got["from_cache"] and got["variant"] == variant, got


@pytest.mark.parametrize("precision", ["f16x3", "split3", "bf16"])
def test_resident_core_matches_oracle(g, oracle_factors, sphere_small, torus_mid, monkeypatch, tmp_path, precision):
    """Core variant 13 (K~_o resident in shared memory, only the gathered A
    rows streamed) against the oracle, forward and adjoint: p = 8 (r_pad 192,
    one N part; levels 2-4 with 3 rhs, so tiles end raggedly inside every
    offset group) and p = 10 at eps = 1e-8 (r_pad 272: two N parts of 144
    and 128 columns, a 16-wide last K-chunk)."""
    import json

    cache = tmp_path / "tune.json"
    monkeypatch.setenv("KIFMM_M2L_AUTOTUNE_CACHE", str(cache))
    tree, qs = sphere_small
    f = oracle_factors(8, 0.1, 1e-7)
    plan = make_plan(g, 8, 1e-7, precision, tree, (2, 3, 4))
    x_all = torch.from_numpy(np.concatenate([qs[l] for l in (2, 3, 4)])).cuda()
    c0 = plan.autotune(x_all, 2, 4, reps=1)["n_chunk"]
    key = list(json.loads(cache.read_text()))[0]
    _force_variant(plan, x_all, 2, 4, cache, key, c0, 1, 13)
    for adj in (False, True):
        out = plan.apply_levels(x_all, 2, 4, adjoint=adj).cpu().numpy()
        plan.sync()
        row = 0
        for l in (2, 3, 4):
            nb = tree.levels[l].shape[0]
            ref = (om.m2l_svd_adjoint if adj else om.m2l_svd)(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64))
            err = rel(out[row:row + nb], ref)
            print(f"resident core p=8 {precision} adjoint {adj} level {l}: rel L2 {err:.3e}")
            assert err <= TOL[precision], (adj, l, err)
            row += nb
    plan.close()
    cache.unlink()
    tree, qs = torus_mid
    f = oracle_factors(10, 0.1, 1e-8)
    plan = make_plan(g, 10, 1e-8, precision, tree, range(2, 6))
    assert plan.r_pad == 272
    x_all = torch.from_numpy(np.concatenate([qs[l] for l in range(2, 6)])).cuda()
    c0 = plan.autotune(x_all, 2, 5, reps=1)["n_chunk"]
    key = list(json.loads(cache.read_text()))[0]
    _force_variant(plan, x_all, 2, 5, cache, key, c0, 1, 13)
    for adj in (False, True):
        out = plan.apply_levels(x_all, 2, 5, adjoint=adj).cpu().numpy()
        plan.sync()
        row = 0
        for l in range(2, 6):
            nb = tree.levels[l].shape[0]
            ref = (om.m2l_svd_adjoint if adj else om.m2l_svd)(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64))
            err = rel(out[row:row + nb], ref)
            print(f"resident core p=10 {precision} adjoint {adj} level {l}: rel L2 {err:.3e}")
            assert err <= TOL[precision], (adj, l, err)
            row += nb
    plan.close()


def test_core_variants_match_oracle(g, oracle_factors, sphere_small, monkeypatch, tmp_path):
    """Every core variant the autotuner can pick for a p = 8 split6 plan
    (partials of two or one K-chunks drained into registers; the A-resident kernel, which
    streams K~_o in two column blocks of 96; the classic kernel with N = 192
    or 96 per item; round-robin or contiguous tiles) against the oracle,
    forward and adjoint, levels 2..4 with 3 rhs."""
    tree, qs = sphere_small
    f = oracle_factors(8, 0.1, 1e-7)
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("KIFMM_M2L_AUTOTUNE_CACHE", str(cache))
    plan = make_plan(g, 8, 1e-7, "split6", tree, (2, 3, 4))
    x_all = torch.from_numpy(np.concatenate([qs[l] for l in (2, 3, 4)])).cuda()
    res = plan.autotune(x_all, 2, 4, reps=2)
    print("autotune", res)
    import json

    key = list(json.loads(cache.read_text()))[0]
    refs = {(l, adj): (om.m2l_svd_adjoint if adj else om.m2l_svd)(tree.levels[l], l, tree.r0, f,
                                                                   qs[l].astype(np.float64))
            for l in (2, 3, 4) for adj in (False, True)}
    for chunk, contig, variant in [(192, 0, 2), (192, 1, 2), (192, 0, 3), (192, 0, 4), (192, 1, 4), (192, 0, 5),
                                   (192, 0, 9), (192, 1, 9), (192, 0, 1), (192, 1, 1), (192, 0, 0), (192, 1, 0),
                                   (96, 0, 0)]:
        cache.write_text('{\n"%s": {"n_chunk": %d, "contiguous": %d, "variant": %d, "core_ms": 1.0}\n}\n'
                         % (key, chunk, contig, variant))
        got = plan.autotune(x_all, 2, 4, reps=1)
        assert got["from_cache"] and (got["n_chunk"], got["contiguous"], got["variant"]) == (chunk, contig, variant)
        for adj in (False, True):
            out = plan.apply_levels(x_all, 2, 4, adjoint=adj).cpu().numpy()
            plan.sync()
            row = 0
            for l in (2, 3, 4):
                nb = tree.levels[l].shape[0]
                err = rel(out[row:row + nb], refs[(l, adj)])
                print(f"variant chunk {chunk} contiguous {contig} variant {variant} adjoint {adj} level {l}: "
                      f"rel L2 {err:.3e}")
                assert err <= TOL["split6"], (chunk, contig, variant, adj, l, err)
                row += nb
    plan.close()


@pytest.mark.parametrize("precision", ["split6", "split3", "bf16", "f16x3"])
def test_stage2_parity(g, oracle_factors, sphere_small, precision):
    """Stage 2 (Sec. 3.2) with c2 = 1 on the p = 8 sphere: the library's
    per-offset ranks equal the oracle's, and apply_levels (forward and
    adjoint, levels 2..4, 3 rhs) and apply match the oracle's two-product
    M2L; switching stage 2 off restores the single-stage operator."""
    tree, qs = sphere_small
    f = oracle_factors(8, 0.1, 1e-7)
    fac = om.stage2_factors(f, om.eps2_from_c2(1.0, 1e-7, f.r))
    plan = make_plan(g, 8, 1e-7, precision, tree, (2, 3, 4))
    plan.set_stage2(1.0)
    k = plan.stage2_ranks()
    assert np.array_equal(k, [uh.shape[1] for uh, _ in fac])
    print(f"stage-2 ranks: min {k.min()} mean {k.mean():.1f} max {k.max()} (r = {f.r})")
    x_all = torch.from_numpy(np.concatenate([qs[l] for l in (2, 3, 4)])).cuda()
    for adjoint in (False, True):
        out = plan.apply_levels(x_all, 2, 4, adjoint=adjoint).cpu().numpy()
        plan.sync()
        row = 0
        for l in (2, 3, 4):
            nb = tree.levels[l].shape[0]
            fn = om.m2l_svd_stage2_adjoint if adjoint else om.m2l_svd_stage2
            ref = fn(tree.levels[l], l, tree.r0, f, fac, qs[l].astype(np.float64))
            err = rel(out[row:row + nb], ref)
            print(f"stage2 {precision} adjoint={adjoint} level {l}: rel L2 {err:.3e}")
            assert err <= TOL[precision], err
            row += nb
    ref = om.m2l_svd_stage2(tree.levels[4], 4, tree.r0, f, fac, qs[4].astype(np.float64))
    out = plan.apply(torch.from_numpy(qs[4]).cuda(), 4)
    plan.sync()
    assert rel(out.cpu().numpy(), ref) <= TOL[precision]
    plan.set_stage2(0.0)
    out = plan.apply(torch.from_numpy(qs[4]).cuda(), 4)
    plan.sync()
    ref1 = om.m2l_svd(tree.levels[4], 4, tree.r0, f, qs[4].astype(np.float64))
    assert rel(out.cpu().numpy(), ref1) <= TOL[precision]
    plan.close()


def test_full_size_torus_p10_sampled(g, oracle_factors):
    """The 4,194,304-point torus at depth 6, p = 10, eps = 1e-8, split6, all
    levels in one batch, on sampled targets the oracle computes one by one."""
    wl = synth.workload("torus4m_p10")
    tree = wl.tree
    f = oracle_factors(10, 0.1, 1e-8)
    plan = make_plan(g, 10, 1e-8, "split6", tree, range(2, 7))
    qs = {l: synth.random_box_densities(tree.levels[l].shape[0], 1, 488, 700 + l)[:, 0] for l in range(2, 7)}
    out = plan.apply_levels(torch.from_numpy(np.concatenate([qs[l] for l in range(2, 7)])).cuda(), 2, 6)
    plan.sync()
    out = out.cpu().numpy()
    rng = np.random.default_rng(8)
    row = 0
    for l in range(2, 7):
        nb = tree.levels[l].shape[0]
        tg = np.sort(rng.choice(nb, size=min(12, nb), replace=False))
        ref = om.m2l_svd_targets(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64), tg)[:, 0, :]
        err = rel(out[row:row + nb][tg], ref)
        print(f"torus4m level {l}: sampled rel L2 {err:.3e}")
        assert err <= 1e-6, err
        row += nb


def _ellipsoid_batch(n_inst, seed0=0):
    """Small instances of the mixed batch: ellipsoids of uneven sizes, depth 3-5,
    p in {6, 8, 10}, nrhs in {1, 2, 3}."""
    rng = np.random.default_rng(seed0)
    out = []
    for i in range(n_inst):
        n = int(np.exp(rng.uniform(np.log(5_000), np.log(60_000))))
        axes = rng.uniform(0.5, 2.0, size=3)
        depth = int(rng.integers(3, 6))
        p = (6, 8, 10)[i % 3]
        nrhs = int(rng.integers(1, 4))
        pts = synth.points_ellipsoid(n, 2000 + i, axes)
        out.append((p, depth, nrhs, synth.build_tree(pts, depth)))
    return out


@pytest.mark.parametrize("precision", ["split6", "split3", "f16x3"])
def test_batch_matches_levels_and_graph_replay(g, oracle_factors, precision):
    """kifmm_m2l_apply_batch over instances of uneven sizes and three
    operators (p = 6, 8, 10) against each instance's own batched-levels
    apply, in eager and CUDA-graph mode, and one instance against the oracle.
    In split3 and f16x3 the three operators' cores are one grouped launch
    (ranks 271 > 192 and smaller ones side by side); split6 runs one core
    launch per operator."""
    from paper_1211_2517_gb300 import apply_batch

    inst = _ellipsoid_batch(9, 11)
    plans = {p: g.M2LPlan(p, 1e-7, 0.1, precision) for p in (6, 8, 10)}
    items, refs = [], []
    for i, (p, depth, nrhs, tree) in enumerate(inst):
        plan = plans[p]
        for l in range(2, depth + 1):
            plan.set_level(l, tree.levels[l], tree.r0, instance=i)
        nb = sum(tree.levels[l].shape[0] for l in range(2, depth + 1))
        x = torch.from_numpy(synth.random_box_densities(nb, nrhs, plan.n, 3000 + i)).cuda()
        items.append({"plan": plan, "instance": i, "level_lo": 2, "level_hi": depth, "x": x,
                      "out": torch.zeros_like(x)})
    for it in items:
        refs.append(it["plan"].apply_levels(it["x"], 2, it["level_hi"], instance=it["instance"]))
    torch.cuda.synchronize()
    for use_graph in (False, True, True):  # eager; graph capture (eager result); graph replay
        for it in items:
            it["out"].fill_(float("nan"))
        apply_batch(items, use_graph=use_graph)
        torch.cuda.synchronize()
        for it, ref in zip(items, refs):
            err = float((it["out"] - ref).double().norm() / ref.double().norm())
            assert err < 1e-6, (use_graph, err)
    # accumulate: beta = 1 doubles the result
    for it in items:
        it["beta"] = 1.0
    apply_batch(items)
    torch.cuda.synchronize()
    for it, ref in zip(items, refs):
        err = float((it["out"] - 2 * ref).double().norm() / (2 * ref).double().norm())
        assert err < 1e-6, err
    # one p = 8 instance against the oracle, level by level
    i8 = next(i for i, c in enumerate(inst) if c[0] == 8)
    p, depth, nrhs, tree = inst[i8]
    f = oracle_factors(8, 0.1, 1e-7)
    o = refs[i8].cpu().numpy()
    x = items[i8]["x"].cpu().numpy().astype(np.float64)
    row = 0
    for l in range(2, depth + 1):
        nb = tree.levels[l].shape[0]
        ref = om.m2l_svd(tree.levels[l], l, tree.r0, f, x[row:row + nb])
        assert rel(o[row:row + nb], ref) <= TOL[precision]
        row += nb
    for pl in plans.values():
        pl.close()


def test_batch64_full_config(g, oracle_factors):
    """The 64-instance mixed batch at full size: ellipsoids with N
    log-uniform in [5e4, 1e6], depth 3-6, p in {6, 8, 10}, 16 rhs each
    (6.0M (box, rhs) rows, 8.2 GB of input), all M2L levels, in one grouped
    batch captured into a CUDA graph and replayed; each instance against its
    own batched-levels apply, and one instance per p against the oracle on
    sampled targets of its deepest level."""
    from paper_1211_2517_gb300 import apply_batch

    inst = [synth.ellipsoid_instance(i) for i in range(64)]
    plans = {p: g.M2LPlan(p, 1e-7, 0.1, "f16x3") for p in (6, 8, 10)}
    items = []
    for i, wl in enumerate(inst):
        plan = plans[wl.p]
        for l in range(2, wl.depth + 1):
            plan.set_level(l, wl.tree.levels[l], wl.tree.r0, instance=i)
        nb = sum(wl.tree.levels[l].shape[0] for l in range(2, wl.depth + 1))
        x = torch.from_numpy(synth.random_box_densities32(nb, 16, plan.n, 5000 + i)).cuda()
        items.append({"plan": plan, "instance": i, "level_lo": 2, "level_hi": wl.depth, "x": x,
                      "out": torch.empty_like(x)})
    rows = sum(it["x"].shape[0] * 16 for it in items)
    print(f"batch64: {rows} (box, rhs) rows, {sum(it['x'].numel() for it in items) * 4 / 1e9:.2f} GB input")
    apply_batch(items, use_graph=True)   # eager pass + capture
    torch.cuda.synchronize()
    first = [it["out"].clone() for it in items[:8]]
    for it in items:
        it["out"].fill_(float("nan"))
    apply_batch(items, use_graph=True)   # graph replay
    torch.cuda.synchronize()
    for a, it in zip(first, items[:8]):
        assert rel(it["out"].cpu().numpy(), a.cpu().numpy().astype(np.float64)) <= 1e-6
    # each instance against its own batched-levels apply
    for it in items[::7]:
        ref = it["plan"].apply_levels(it["x"], 2, it["level_hi"], instance=it["instance"])
        torch.cuda.synchronize()
        err = float((it["out"] - ref).double().norm() / ref.double().norm())
        assert err <= 1e-6, (it["instance"], err)
    # one instance per p against the oracle, sampled targets of the deepest level
    rng = np.random.default_rng(64)
    for p in (6, 8, 10):
        i = min((j for j, wl in enumerate(inst) if wl.p == p and wl.depth >= 4),
                key=lambda j: inst[j].tree.levels[inst[j].depth].shape[0])
        wl = inst[i]
        f = oracle_factors(p, 0.1, 1e-7)
        l = wl.depth
        row0 = sum(wl.tree.levels[m].shape[0] for m in range(2, l))
        nb = wl.tree.levels[l].shape[0]
        q = items[i]["x"][row0:row0 + nb].cpu().numpy().astype(np.float64)
        tg = np.sort(rng.choice(nb, size=min(16, nb), replace=False))
        ref = om.m2l_svd_targets(wl.tree.levels[l], l, wl.tree.r0, f, q, tg)
        out = items[i]["out"][row0:row0 + nb].cpu().numpy()[tg]
        err = rel(out, ref)
        print(f"batch64 instance {i} (p={p}, depth {l}, {nb} boxes): sampled rel L2 {err:.3e}")
        assert err <= 1e-6, err
    for plan in plans.values():
        plan.close()


_YUKAWA = {}


@pytest.mark.parametrize("precision", ["split3", "f16x3"])
def test_yukawa_levels_one_batch(g, sphere_small, precision):
    """The per-level Yukawa plans of levels 2-4 (each its own rank r_l and
    cores, Sec. 3.1's O(L) case) applied as one batch, whose cores run as one
    grouped launch, eager and replayed from a CUDA graph; each level against
    the oracle's per-level factors."""
    from paper_1211_2517_gb300 import apply_batch

    tree, qs = sphere_small
    kappa = 3.0
    items, refs, ranks = [], [], []
    for l in (2, 3, 4):
        h = tree.r0 / (1 << l)
        f = _yukawa_factors(kappa, h)
        plan = g.M2LPlan(8, 1e-7, 0.1, precision, "yukawa", kappa, h)
        plan.set_level(l, tree.levels[l], tree.r0)
        ranks.append(plan.r)
        x = torch.from_numpy(qs[l]).cuda()
        items.append({"plan": plan, "level_lo": l, "level_hi": l, "x": x, "out": torch.empty_like(x)})
        refs.append(om.m2l_svd(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64)))
    assert len(set(ranks)) > 1, ranks  # the groups differ in rank
    for use_graph in (False, True, True):
        for it in items:
            it["out"].fill_(float("nan"))
        apply_batch(items, use_graph=use_graph)
        torch.cuda.synchronize()
        for l, it, ref in zip((2, 3, 4), items, refs):
            err = rel(it["out"].cpu().numpy(), ref)
            print(f"yukawa batch level {l} (r = {it['plan'].r}) {precision} graph={use_graph}: {err:.3e}")
            assert err <= TOL[precision], (l, err)
    for it in items:
        it["plan"].close()


def _yukawa_factors(kappa, h):
    if (kappa, h) not in _YUKAWA:
        _YUKAWA[(kappa, h)] = om.svd_factors(8, 0.1, 1e-7, kappa=kappa, h=h)
    return _YUKAWA[(kappa, h)]


@pytest.mark.parametrize("precision", ["fp32", "split6", "f16x3"])
def test_yukawa_per_level_plans(g, sphere_small, precision):
    """The Yukawa kernel exp(-kappa r) / (4 pi r) is not homogeneous, so the
    translation matrices of every level are compressed separately (Sec. 3.1's
    O(L) case): one plan per level, formed at its box half-width.  Forward
    and adjoint against the oracle's per-level factors, the FP32 dense
    baseline against the oracle's dense Yukawa M2L, and the level check."""
    from paper_1211_2517_gb300 import KifmmError

    tree, qs = sphere_small
    kappa = 3.0
    rng = np.random.default_rng(77)
    for l in (2, 3, 4):
        h = tree.r0 / (1 << l)
        f = _yukawa_factors(kappa, h)
        plan = g.M2LPlan(8, 1e-7, 0.1, precision, "yukawa", kappa, h)
        assert plan.r == f.r
        plan.set_level(l, tree.levels[l], tree.r0)
        ref = om.m2l_svd(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64))
        out = plan.apply(torch.from_numpy(qs[l]).cuda(), l)
        y = rng.standard_normal(qs[l].shape).astype(np.float32)
        aty = plan.apply_adjoint(torch.from_numpy(y).cuda(), l)
        plan.sync()
        ref_adj = om.m2l_svd_adjoint(tree.levels[l], l, tree.r0, f, y.astype(np.float64))
        err, err_adj = rel(out.cpu().numpy(), ref), rel(aty.cpu().numpy(), ref_adj)
        print(f"yukawa kappa={kappa} level {l} (kappa h = {kappa * h:.3f}, r = {f.r}) {precision}: "
              f"forward {err:.3e} adjoint {err_adj:.3e}")
        assert err <= TOL[precision] and err_adj <= TOL[precision], (err, err_adj)
        if precision == "fp32" and l == 2:
            dense = plan.apply_dense(torch.from_numpy(qs[l]).cuda(), l)
            plan.sync()
            ref_d = om.m2l_dense(tree.levels[l], l, tree.r0, 8, 0.1, qs[l].astype(np.float64), centre=tree.centre,
                                 kappa=kappa)
            assert rel(dense.cpu().numpy(), ref_d) <= 1e-6
        other = 3 if l != 3 else 4
        with pytest.raises(KifmmError, match="INVALID_ARG"):
            plan.set_level(other, tree.levels[other], tree.r0)
        if l == 2 and precision != "fp32":
            with pytest.raises(KifmmError, match="UNSUPPORTED"):
                g.PointFMM(plan, synth.points_uniform_cube(100, 1), 3)
        plan.close()
