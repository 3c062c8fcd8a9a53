"""Host-side logic of the native library, checked on the CPU.

The FP64 precompute and the interaction-list builder of libkifmm_m2l.so run
on the host; here they are compared with the oracle (which shares no code
with them).  Also: the library loads and exports every symbol the header
declares, and bad arguments are rejected with the documented codes.
No GPU work is launched.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import geometry as geo
from oracle import m2l as om

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_1211_2517_gb300 import build

    build.build()
    import paper_1211_2517_gb300 as g

    return g


def test_library_exports_every_header_symbol(native):
    hdr = open(os.path.join(ROOT, "include", "kifmm_m2l.h")).read()
    declared = set(re.findall(r"^(?:int|const char\*)\s+(kifmm_\w+)\(", hdr, flags=re.M))
    assert declared == set(native.EXPORTED)
    L = native.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert b"sm_103a" in L.kifmm_m2l_version()


def test_param_validation(native):
    from paper_1211_2517_gb300._lib import Params

    L = native.lib()
    n, r = ctypes.c_int(), ctypes.c_int()
    bad = [
        (Params(2, 6, 1e-7, 0.1, 0), -2),   # unsupported kernel
        (Params(1, 6, 1e-7, 0.1, 0, 0.0, 0.5), -1),    # Yukawa without kappa
        (Params(1, 6, 1e-7, 0.1, 0, 2.0, 0.0), -1),    # Yukawa without box half-width
        (Params(1, 6, 1e-7, 0.1, 0, 200.0, 1.0), -1),  # kappa h > 64
        (Params(0, 1, 1e-7, 0.1, 0), -1),   # p too small
        (Params(0, 13, 1e-7, 0.1, 0), -1),  # p too large
        (Params(0, 6, 1e-13, 0.1, 0), -1),  # eps below 1e-12
        (Params(0, 6, 1.0, 0.1, 0), -1),    # eps >= 1
        (Params(0, 6, 1e-7, 0.7, 0), -1),   # d > 2/3
        (Params(0, 6, 1e-7, 0.1, 9), -1),   # precision
    ]
    for prm, code in bad:
        st = L.kifmm_m2l_factors_host(ctypes.byref(prm), ctypes.byref(n), ctypes.byref(r), None, None, None)
        assert st == code, (prm.kernel_id, prm.p, prm.eps, prm.d, prm.precision, st)
        assert L.kifmm_m2l_last_error()
    assert L.kifmm_m2l_factors_host(None, None, None, None, None, None) == -1
    assert L.kifmm_m2l_destroy(None) == 0
    assert L.kifmm_fmm_set_normals(None, None) == -1  # no tree
    yuk = Params(1, 6, 1e-7, 0.1, 0, 2.0, 0.25)
    assert L.kifmm_m2l_pass_ops_host(ctypes.byref(yuk), 1e-9, None, None, None) == -2  # Laplace passes only
    cnt = ctypes.c_int64()
    assert L.kifmm_m2l_pairs_host(2, 1, np.array([[4, 0, 0]], np.int32).ctypes.data, ctypes.byref(cnt),
                                  None, None, None) == -1  # coordinate out of range
    assert L.kifmm_m2l_pairs_host(2, 2, np.array([[1, 0, 0], [1, 0, 0]], np.int32).ctypes.data,
                                  ctypes.byref(cnt), None, None, None) == -1  # duplicate


@pytest.mark.parametrize("p,eps", [(4, 1e-4), (6, 1e-7), (8, 1e-7)])
def test_factors_match_oracle_through_products(native, oracle_factors, p, eps):
    sigma, U, C = native.factors_host(p, eps, 0.1)
    f = oracle_factors(p, 0.1, eps)
    # same rank decision (both FP64), same singular values
    assert U.shape[1] == f.r
    np.testing.assert_allclose(sigma, f.sigma, rtol=0, atol=1e-12 * f.sigma[0])
    # orthonormal basis spanning the oracle's (up to the subspace sensitivity
    # eps_mach * sigma_0 / gap at the cut)
    assert np.abs(U.T @ U - np.eye(f.r)).max() < 1e-12
    assert np.linalg.norm(U @ U.T - f.U @ f.U.T, 2) < 1e-6
    # the compressed operators agree: U~ K~_o U~^T (library, R~ = U~) vs U~ K~_o R~^T (oracle)
    kmax = np.abs(f.K).max()
    for k in range(0, 316, 3):
        a = U @ C[k] @ U.T
        b = f.U @ f.C[k] @ f.R.T
        assert np.abs(a - b).max() < 1e-11 * kmax, k
    # symmetry used by the adjoint: K~_o^T = K~_{-o}
    offs = geo.m2l_offsets()
    tab = geo.offset_index_table()
    for k in (0, 17, 158, 315):
        np.testing.assert_allclose(C[k].T, C[tab[tuple(-offs[k])]], rtol=0, atol=1e-12 * np.abs(C).max())


def test_yukawa_factors_match_oracle(native):
    # the library compresses its unit operator h K_h (K_h the Yukawa
    # matrices of boxes of half-width h, Sec. 3.1's per-level case): the
    # oracle's per-level factors with singular values and cores times h
    kappa, h = 3.0, 0.125
    sigma, U, C = native.factors_host(6, 1e-5, 0.1, "yukawa", kappa, h)
    f = om.svd_factors(6, 0.1, 1e-5, kappa=kappa, h=h)
    assert U.shape[1] == f.r
    np.testing.assert_allclose(sigma, h * f.sigma, rtol=0, atol=1e-12 * h * f.sigma[0])
    kmax = np.abs(f.K).max()
    for k in range(0, 316, 7):
        assert np.abs(U @ C[k] @ U.T - h * (f.U @ f.C[k] @ f.R.T)).max() < 1e-11 * h * kmax, k
    # a different kappa h is a different operator
    _, U2, C2 = native.factors_host(6, 1e-5, 0.1, "yukawa", kappa, 2 * h)
    assert U2.shape[1] != U.shape[1] or np.abs(U2 @ C2[0] @ U2.T - U @ C[0] @ U.T).max() > 1e-3 * np.abs(C[0]).max()


def test_factors_full_rank_and_truncation_rule(native):
    sigma, U, _ = native.factors_host(4, 0.0, 0.1)
    assert U.shape == (56, 56)
    r = U.shape[1]
    s2, U2, _ = native.factors_host(4, 1e-3, 0.1)
    assert U2.shape[1] == om.truncation_rank(s2, 1e-3)


def test_pairs_match_oracle_lists(native):
    rng = np.random.default_rng(11)
    for level, nbox in ((2, 40), (3, 300), (5, 2000)):
        m = 1 << level
        flat = rng.choice(m ** 3, size=min(nbox, m ** 3), replace=False)
        box = np.stack([flat // (m * m), (flat // m) % m, flat % m], axis=1)
        tg, sr, of = native.pairs_host(level, box)
        otg, osr, oof = geo.interaction_lists(box)
        a = np.lexsort((tg, of))
        assert np.all(a == np.arange(tg.size))  # sorted by offset, then target
        ref = sorted(zip(oof.tolist(), otg.tolist(), osr.tolist()))
        got = list(zip(of.tolist(), tg.tolist(), sr.tolist()))
        assert got == ref


def test_pairs_on_synthetic_sphere_level(native):
    pts = synth.points_sphere(200_000, 0)
    tree = synth.build_tree(pts, 5)
    box = tree.levels[5]
    tg, sr, of = native.pairs_host(5, box)
    otg, osr, oof = geo.interaction_lists(box)
    assert tg.size == otg.size
    assert np.bincount(tg, minlength=box.shape[0]).max() <= 189
    offs = geo.m2l_offsets()
    assert np.array_equal(box[tg] - box[sr], offs[of])


def test_pairs_edge_cases(native):
    # no boxes, one box, two adjacent boxes: no pairs
    for box in (np.zeros((0, 3), np.int32), np.array([[1, 1, 1]]), np.array([[0, 0, 0], [1, 1, 1]])):
        tg, _, _ = native.pairs_host(2, box)
        assert tg.size == 0
    # two boxes two apart under adjacent parents: one pair each way
    tg, sr, of = native.pairs_host(2, np.array([[0, 0, 0], [2, 0, 0]]))
    assert sorted(zip(tg.tolist(), sr.tolist())) == [(0, 1), (1, 0)]
    # too far apart (parents not adjacent): none
    tg, _, _ = native.pairs_host(3, np.array([[0, 0, 0], [4, 0, 0]]))
    assert tg.size == 0


@pytest.mark.parametrize("p,eps,c2", [(4, 1e-4, 10.0), (6, 1e-7, 1.0)])
def test_stage2_host_matches_oracle(native, oracle_factors, p, eps, c2):
    """The library's FP64 stage-2 factoring (Sec. 3.2) against the oracle's:
    the same per-offset ranks and the same truncated operators, compared
    through U~ (Uhat_o Vhat_o) R~^T since the two precomputes pick different
    bases of the same subspace."""
    k, core = native.stage2_host(p, eps, c2, 0.1)
    sigma, U, _ = native.factors_host(p, eps, 0.1)
    f = oracle_factors(p, 0.1, eps)
    fac = om.stage2_factors(f, om.eps2_from_c2(c2, eps, f.r))
    ranks = np.array([uh.shape[1] for uh, _ in fac])
    assert np.array_equal(k, ranks)
    assert ranks.min() < f.r
    kmax = np.abs(f.K).max()
    for o in range(0, 316, 5):
        uh, vh = fac[o]
        a = U @ core[o] @ U.T
        b = f.U @ (uh @ vh) @ f.R.T
        assert np.abs(a - b).max() < 1e-10 * kmax, o


@pytest.mark.parametrize("p", [4, 6])
def test_pass_ops_host_matches_oracle(native, p):
    """The library's FP64 pass operators of Sec. 3.3 against the oracle's,
    compared through the basis: U~ Ws = P E_u and U~ M~_c U~^T = P M_c P with
    P the projector on the M2L basis (the two precomputes pick different
    bases of the same subspace).  The pseudo-inverse with the 1e-9 cutoff
    carries noise of about 1e-9 relative along the cut directions."""
    from oracle import fmm as ofmm

    eps = 1e-7
    kept, Ws, Mt = native.pass_ops_host(p, eps, 0.1, ofmm.FMM_RCOND)
    _, U, _ = native.factors_host(p, eps, 0.1)
    f = om.svd_factors(p, 0.1, eps)
    ops = ofmm.pass_operators(f, p, 0.1)
    n = U.shape[0]
    assert 0 < kept <= n
    a, b = U @ Ws, f.R @ ops.Ws
    assert np.linalg.norm(a - b) <= 1e-7 * np.linalg.norm(b)
    for c in range(8):
        a = U @ Mt[c] @ U.T
        b = f.R @ ops.Mt[c] @ f.R.T
        assert np.linalg.norm(a - b) <= 1e-7 * np.linalg.norm(b), c
    # L~_c = M~_c^T: the oracle forms L from the downward surfaces itself
    for c in (1, 6):
        a = U @ Mt[c].T @ U.T
        b = f.U @ ops.Lt[c] @ f.U.T
        assert np.linalg.norm(a - b) <= 1e-7 * np.linalg.norm(b), c


def test_every_entry_point_cites_its_passage():
    # each declaration of the C ABI is preceded by a comment that cites the
    # passage of the paper it computes, or says that it has none
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "kifmm_m2l.h")).read()
    names = re.findall(r"^(?:int|const char\*)\s+(kifmm_\w+)\(", hdr, flags=re.M)
    assert len(names) >= 25
    for name in names:
        start = re.search(r"^(?:int|const char\*)\s+" + name + r"\(", hdr, flags=re.M).start()
        end = hdr.rfind("*/", 0, start)
        comment = hdr[hdr.rfind("/*", 0, end):end]
        between = [ln for ln in hdr[end + 2:start].splitlines() if ln.strip()]
        assert all(ln.startswith("#define") for ln in between), name
        assert re.search(r"Sec\.|Eq\.|Step |no passage of the paper", comment), name
