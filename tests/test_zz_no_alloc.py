"""kifmm_m2l_apply_noalloc against kifmm_m2l_apply, through the C ABI.

The allocation-free entry point is for callers that cannot allocate device
memory once their run has started (a memory manager that reserved the
device, a fixed memory budget, a latency-critical loop that cannot take
cudaMalloc's synchronisation).  It must give what kifmm_m2l_apply gives;
it is called twice in a row on each case, since its static scratch keeps
the previous call's contents and the second call must not see them.
"""
import ctypes
import os
import tempfile

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"split6": 1e-6, "fp32": 1e-6, "split3": 1e-6, "bf16": 1e-6}  # against plan.apply (same arithmetic)


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    os.environ.setdefault("KIFMM_M2L_CACHE", tempfile.mkdtemp(prefix="kifmm_cache_"))
    from paper_1211_2517_gb300 import build

    build.build()
    import paper_1211_2517_gb300 as pkg

    return pkg


def _noalloc(g, plan, level, nrhs, x, out, beta):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return g.lib().kifmm_m2l_apply_noalloc(plan._h, 0, level, nrhs, ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), float(beta), stream)


@pytest.mark.parametrize("precision,stage2", [("split6", 0.0), ("fp32", 0.0), ("split3", 0.0), ("bf16", 0.0),
                                             ("split6", 10.0)])
def test_noalloc_matches_apply_on_two_calls(g, precision, stage2):
    pts = synth.points_sphere(200_000, 3)
    tree = synth.build_tree(pts, 5)
    plan = g.M2LPlan(8, 1e-7, 0.1, precision)
    if stage2:
        plan.set_stage2(stage2)
    levels = (3, 5)
    for l in levels:
        plan.set_level(l, tree.levels[l], tree.r0)
    nrhs = 2
    for l in levels:
        nb = tree.levels[l].shape[0]
        x = torch.from_numpy(synth.random_box_densities(nb, nrhs, plan.n, 40 + l)).cuda()
        ref = plan.apply(x, l)
        plan.sync()
        for call in range(2):
            # stale contents in the output must not matter with beta = 0
            out = torch.full_like(ref, float(call + 7))
            assert _noalloc(g, plan, l, nrhs, x, out, 0.0) == 0, g.lib().kifmm_m2l_last_error()
            plan.sync()
            err = float((out - ref).double().norm() / ref.double().norm())
            assert err <= TOL[precision], (precision, l, call, err)
        # accumulate mode
        prev = torch.randn_like(ref)
        out = prev.clone()
        assert _noalloc(g, plan, l, nrhs, x, out, 1.0) == 0
        plan.sync()
        err = float((out - prev - ref).double().norm() / ref.double().norm())
        assert err <= TOL[precision], err
    plan.close()


def test_noalloc_allocates_nothing_on_a_fresh_plan(g):
    """A plan that never ran kifmm_m2l_apply: the allocation-free call, after
    one warm-up call that loads its kernels, leaves the device's free memory
    unchanged, and its result matches kifmm_m2l_apply run afterwards."""
    pts = synth.points_sphere(120_000, 9)
    tree = synth.build_tree(pts, 5)
    warm = g.M2LPlan(8, 1e-7, 0.1, "split6")
    warm.set_level(4, tree.levels[4], tree.r0)
    xw = torch.from_numpy(synth.random_box_densities(tree.levels[4].shape[0], 1, warm.n, 7)).cuda()
    assert _noalloc(g, warm, 4, 1, xw, torch.zeros_like(xw), 0.0) == 0
    warm.sync()
    plan = g.M2LPlan(8, 1e-7, 0.1, "split6")
    plan.set_level(5, tree.levels[5], tree.r0)
    x = torch.from_numpy(synth.random_box_densities(tree.levels[5].shape[0], 1, plan.n, 8)).cuda()
    out = torch.zeros_like(x)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _noalloc(g, plan, 5, 1, x, out, 0.0) == 0, g.lib().kifmm_m2l_last_error()
    plan.sync()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    ref = plan.apply(x, 5)
    plan.sync()
    err = float((out - ref).double().norm() / ref.double().norm())
    assert err <= TOL["split6"], err
    plan.close()
    warm.close()


def test_noalloc_rejects_oversized_requests(g):
    pts = synth.points_sphere(200_000, 4)
    tree = synth.build_tree(pts, 5)
    plan = g.M2LPlan(8, 1e-7, 0.1, "split6")
    plan.set_level(5, tree.levels[5], tree.r0)
    nb = tree.levels[5].shape[0]
    nrhs = 16  # needs ~ nb * 16 * 192 * 10 bytes > 64 MiB
    x = torch.zeros((nb, nrhs, plan.n), device="cuda")
    out = torch.zeros_like(x)
    st = _noalloc(g, plan, 5, nrhs, x, out, 0.0)
    assert st == -1
    assert b"static scratch" in g.lib().kifmm_m2l_last_error()
    plan.close()
