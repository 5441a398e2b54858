"""GPU parity of the Neumann boundary (mirrored ghost node) and of the
per-sweep stopping test ||u^n - u^(n-1)||_inf < tol (Sec. 4.2.2) against the
FP64 oracle, through the C ABI.

FP64 tolerances as in test_gpu_parity: identical level sequences and sweep
counts (the stop may fall inside a cycle, so the sweep count checks the
per-sweep test), solutions within 1e-10 relative.
"""
import math

import numpy as np
import pytest

from paper_2011_06636_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_06636_gb300 import _build, srj
    _build.build()
    srj.load(build_if_missing=False)
    torch.cuda.init()
    return srj


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _solve(S, n, bc, f, u0, tol, tol_kind, selector=None, prec=None, **kw):
    prec = S.SRJ_PREC_F64 if prec is None else prec
    selector = S.SRJ_SEL_HEURISTIC if selector is None else selector
    dt = torch.float64 if prec == S.SRJ_PREC_F64 else torch.float32
    h = S.srj_create(n, bc=bc, precision=prec, tol_kind=tol_kind, selector=selector,
                     trace_capacity=100000, **kw)
    try:
        fd, ud = dev(f, dt), dev(u0, dt)
        st = S.srj_solve(h, fd.data_ptr(), ud.data_ptr(), tol)
        lv, rn = S.srj_get_trace(h)
        return st, ud.cpu().double().numpy(), lv, rn
    finally:
        S.srj_destroy(h)


LAPLACE = [([64, 64], "heuristic"), ([128, 128], "heuristic"), ([128, 128], "increasing"),
           ([45, 70], "heuristic"), ([300, 7], "heuristic")]


@pytest.mark.parametrize("n,rule", LAPLACE)
def test_laplace_neumann_dinf_matches_oracle(S, orc, n, rule):
    # Sec. 4.2.2: A x = 0, homogeneous Neumann on every side, random start,
    # stop when the largest change of a sweep falls below 1e-10
    P = orc.Problem(n, bc=[1, 1])
    f = np.zeros(P.size)
    u0 = inputs.uniform_rhs(n, seed=3).ravel()
    ref = orc.srj_solve(P, f, u0, tol=1e-10, tol_kind="dinf", rule=rule)
    sel = S.SRJ_SEL_HEURISTIC if rule == "heuristic" else S.SRJ_SEL_INCREASING
    st, u, lv, rn = _solve(S, n, [1, 1], f, u0, 1e-10, S.SRJ_TOL_DINF, sel)
    assert ref["status"] == 0 and st["status"] == S.SRJ_OK
    np.testing.assert_array_equal(lv, ref["levels"])
    assert st["sweeps"] == ref["sweeps"]
    assert st["cycles"] == ref["cycles"]
    np.testing.assert_allclose(u, ref["u"], rtol=0, atol=1e-10 * np.abs(ref["u"]).max())
    assert st["rn"] == pytest.approx(ref["rn"], rel=1e-6, abs=1e-12 * ref["r0"])


@pytest.mark.parametrize("n,bc", [([40, 9, 33], [1, 0, 1]), ([257], [0]), ([100, 66], [0, 1]),
                                  ([17, 23, 5], [1, 1, 1])])
def test_neumann_rel_tol_solve_matches_oracle(S, orc, n, bc):
    # Poisson with mixed boundaries, relative L2 tolerance; with every axis
    # Neumann the right-hand side is projected onto the range (trapezoid
    # weighted mean removed) so that A u = f has solutions
    P = orc.Problem(n, bc=bc)
    f = inputs.uniform_rhs(n, seed=7).ravel()
    if all(bc):
        w = np.ones(1)
        for a in reversed(range(len(n))):
            t = np.ones(n[a]); t[0] = t[-1] = 0.5
            w = np.kron(w, t)
        # the left null vector of A is w (A^T w = 0): make w . f = 0
        f = f - (w @ f) / (w @ w) * w
    ref = orc.srj_solve(P, f, tol=1e-8)
    st, u, lv, rn = _solve(S, n, bc, f, np.zeros(P.size), 1e-8, S.SRJ_TOL_REL)
    assert ref["status"] == 0 and st["status"] == S.SRJ_OK
    np.testing.assert_array_equal(lv, ref["levels"])
    assert st["sweeps"] == ref["sweeps"]
    np.testing.assert_allclose(u, ref["u"], rtol=0, atol=1e-10 * np.abs(ref["u"]).max())
    np.testing.assert_allclose(rn, ref["rns"], rtol=1e-10, atol=1e-13 * ref["r0"])


@pytest.mark.parametrize("level,k,tol", [(4, 3, 1e-6), (9, 1, 1e-8), (12, 2, 1e-10)])
def test_dinf_stop_closed_form_on_gpu(S, orc, level, k, tol):
    # one cosine mode, fixed level: the stopping sweep in closed form
    n = 17
    v = np.cos(math.pi * k * np.arange(n) / (n - 1))
    mu = 1 - math.cos(math.pi * k / (n - 1))
    g, s_exp = 1.0, None
    for s, w in enumerate(np.tile(orc.level_omegas(level), 40), start=1):
        if abs(w * mu * g) < tol:
            s_exp = s
            break
        g *= 1 - w * mu
    st, u, lv, rn = _solve(S, [n], [1], np.zeros(n), v, tol, S.SRJ_TOL_DINF, S.SRJ_SEL_FIXED,
                           fixed_level=level, level0=level)
    assert st["status"] == S.SRJ_OK and st["sweeps"] == s_exp


def test_generic_pass_with_several_rows_per_thread(S, orc):
    # 1030 x 700 nodes: 33 x 88 column tiles of 32 x 8, more than 16 per SM,
    # so each thread of the one-sweep pass takes two rows (ragged in both
    # axes); the per-sweep stop folds the block maxima of 33 x 44 CTAs
    n = [1030, 700]
    P = orc.Problem(n, bc=[1, 1])
    f = np.zeros(P.size)
    u0 = inputs.uniform_rhs(n, seed=11).ravel()
    ref = orc.srj_solve(P, f, u0, tol=1e-4, tol_kind="dinf")
    st, u, lv, rn = _solve(S, n, [1, 1], f, u0, 1e-4, S.SRJ_TOL_DINF)
    assert ref["status"] == 0 and st["status"] == S.SRJ_OK
    np.testing.assert_array_equal(lv, ref["levels"])
    assert st["sweeps"] == ref["sweeps"] and st["cycles"] == ref["cycles"]
    np.testing.assert_allclose(u, ref["u"], rtol=0, atol=1e-12 * np.abs(ref["u"]).max())


def test_dinf_dirichlet_f32(S, orc):
    # the per-sweep test in FP32: the stop lands within a sweep or two of the
    # FP64 oracle's and the solution within FP32 accuracy of it
    n = [96, 80]
    P = orc.Problem(n)
    f = inputs.uniform_rhs(n, seed=2).ravel()
    ref = orc.srj_solve(P, f, tol=1e-7, tol_kind="dinf")
    st, u, lv, rn = _solve(S, n, None, f, np.zeros(P.size), 1e-7, S.SRJ_TOL_DINF,
                           prec=S.SRJ_PREC_F32)
    assert st["status"] == S.SRJ_OK
    assert abs(st["sweeps"] - ref["sweeps"]) <= max(2, ref["sweeps"] // 50)
    assert np.abs(u - ref["u"]).max() < 1e-4 * np.abs(ref["u"]).max()


def test_null_space_start_stops_after_one_sweep(S):
    n = [33, 20]
    u0 = np.full(33 * 20, 2.5)
    st, u, lv, rn = _solve(S, n, [1, 1], np.zeros(u0.size), u0, 1e-10, S.SRJ_TOL_DINF)
    assert st["status"] == S.SRJ_OK and st["sweeps"] == 1 and st["cycles"] == 0
    np.testing.assert_array_equal(u, u0)


def test_neumann_residual_norm(S, orc):
    n = [50, 31, 12]
    bc = [1, 0, 1]
    P = orc.Problem(n, bc=bc)
    f = inputs.uniform_rhs(n, seed=4).ravel()
    u = inputs.uniform_rhs(n, seed=5).ravel()
    h = S.srj_create(n, bc=bc)
    try:
        fd, ud = dev(f), dev(u)
        got = S.srj_residual_norm(h, fd.data_ptr(), ud.data_ptr())
    finally:
        S.srj_destroy(h)
    assert got == pytest.approx(orc.residual_norm(P, u, f), rel=1e-12)


def test_unsupported_combinations(S):
    import ctypes as C
    L = S.load()
    kt = dev(np.ones(6 * 6))

    def rc(n, bc, **kw):
        k_ptr = kw.pop("k_ptr", None)
        g = S._grid(n, None, bc)
        stc = S.srj_stencil()
        stc.k = k_ptr
        o = S.srj_opts()
        for key, val in kw.items():
            setattr(o, key, val)
        hnd = C.c_void_p()
        r = L.srj_create(C.byref(g), C.byref(stc), C.byref(o), None, C.byref(hnd))
        if r == S.SRJ_OK:
            L.srj_destroy(hnd)
        return r

    assert rc([4, 4], [1, 1], precision=S.SRJ_PREC_MIXED) == S.SRJ_EUNSUPPORTED
    assert rc([4, 4], [0, 0], precision=S.SRJ_PREC_MIXED,
              tol_kind=S.SRJ_TOL_DINF) == S.SRJ_EUNSUPPORTED
    assert rc([4, 4], [1, 0], k_ptr=kt.data_ptr()) == S.SRJ_EUNSUPPORTED
    assert rc([1, 4], [1, 0]) == S.SRJ_EINVAL
    assert rc([4, 4], [2, 0]) == S.SRJ_EINVAL
    assert rc([4, 4], [1, 1], tol_kind=3) == S.SRJ_EINVAL
    assert rc([4, 4], [0, 1]) == S.SRJ_OK
    # batched handles are Dirichlet only
    grids = (S.srj_grid * 1)(S._grid([8, 8], None, [1, 0]))
    o = S.srj_opts()
    o.precision = S.SRJ_PREC_MIXED
    hnd = C.c_void_p()
    assert L.srj_create_batched(1, grids, None, C.byref(o), None,
                                C.byref(hnd)) == S.SRJ_EUNSUPPORTED
