"""Failure detection on the GPU without faulting it: the core kernels' device
waits are bounded, and a plan whose bound is set to a few nanoseconds makes
the first wait that is not already complete give up.  The kernel then stops
every role, waits for its copies and MMAs in flight, frees its tensor memory
and raises the plan's error flag; kifmm_m2l_sync reports KIFMM_ERR_TIMEOUT,
and the same plan, with the default bound restored, computes correct
results again (checked against the FP64 oracle)."""
import ctypes
import json
import os
import tempfile

import numpy as np
import pytest

import synth
from oracle import m2l as om

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

LEVELS = (3, 4)


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    os.environ.setdefault("KIFMM_M2L_CACHE", tempfile.mkdtemp(prefix="kifmm_cache_"))
    from paper_1211_2517_gb300 import build

    build.build()
    import paper_1211_2517_gb300 as pkg

    return pkg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,variant", [("split6", 2), ("f16x3", 11), ("f16x3", 13), ("split3", 13)])
def test_wait_limit_timeout_then_recovery(g, oracle_factors, monkeypatch, tmp_path, precision, variant):
    from paper_1211_2517_gb300 import _lib

    pts = synth.points_sphere(60_000, 7)
    tree = synth.build_tree(pts, 4)
    f = oracle_factors(8, 0.1, 1e-7)
    qs = {l: synth.random_box_densities(tree.levels[l].shape[0], 1, 296, 300 + l)[:, 0] for l in LEVELS}
    plan = g.M2LPlan(8, 1e-7, 0.1, precision)
    for l in LEVELS:
        plan.set_level(l, tree.levels[l], tree.r0)
    x_all = torch.from_numpy(np.concatenate([qs[l] for l in LEVELS])).cuda()
    # the core variant under test, forced through the autotune cache
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("KIFMM_M2L_AUTOTUNE_CACHE", str(cache))
    c0 = plan.autotune(x_all, LEVELS[0], LEVELS[-1], reps=1)["n_chunk"]
    key = list(json.loads(cache.read_text()))[0]
    cache.write_text('{\n"%s": {"n_chunk": %d, "contiguous": 1, "variant": %d, "core_ms": 1.0}\n}\n'
                     % (key, c0, variant))
    assert plan.autotune(x_all, LEVELS[0], LEVELS[-1], reps=1)["variant"] == variant

    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    plan.set_wait_limit(1)
    plan.apply_levels(x_all, LEVELS[0], LEVELS[-1])
    st = _lib.lib().kifmm_m2l_sync(plan._h, stream)
    msg = _lib.lib().kifmm_m2l_last_error().decode()
    print(f"{precision} variant {variant}: sync after a 1 ns bound -> {st} ({msg})")
    assert st == _lib.KIFMM_ERR_TIMEOUT, (st, msg)
    # the flag was cleared by the report, and the context is intact
    assert _lib.lib().kifmm_m2l_sync(plan._h, stream) == _lib.KIFMM_OK

    plan.set_wait_limit(0)
    out = plan.apply_levels(x_all, LEVELS[0], LEVELS[-1]).cpu().numpy()
    plan.sync()
    row = 0
    tol = {"split6": 1e-6, "f16x3": 1e-6, "split3": 3e-5}[precision]
    for l in LEVELS:
        nb = tree.levels[l].shape[0]
        ref = om.m2l_svd(tree.levels[l], l, tree.r0, f, qs[l].astype(np.float64))
        err = rel(out[row:row + nb], ref)
        print(f"{precision} variant {variant} after recovery, level {l}: rel L2 {err:.3e}")
        assert err <= tol, (l, err)
        row += nb
    plan.close()
