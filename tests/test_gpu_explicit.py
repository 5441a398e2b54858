"""GPU parity of the explicit symmetric operator (srj_stencil.a_diag /
a_off): Sec. 4.1's random symmetric diagonally dominant tridiagonal systems
and 2D/3D analogues, against the FP64 oracle through the C ABI.  FP64
tolerances as in test_gpu_parity (identical levels and sweeps, 1e-10)."""
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


def _random_sdd(n, seed):
    """Random symmetric operator, diagonally dominant (weakly in the interior)."""
    rng = np.random.default_rng(seed)
    N = int(np.prod(n))
    aoff = [-rng.random(N) for _ in n]
    adiag = np.zeros(N)
    idx = np.arange(N)
    stride = 1
    for a in range(len(n)):
        coord = (idx // stride) % n[a]
        has_p = coord + 1 < n[a]
        aoff[a] = np.where(has_p, aoff[a], 0.0)
        adiag += np.abs(aoff[a])
        adiag[idx[coord > 0]] += np.abs(aoff[a][idx[coord > 0] - stride])
        stride *= n[a]
    adiag *= 1.0 + 0.05 * rng.random(N)
    return adiag, aoff


def _solve(S, n, adiag, aoff, f, tol, tol_kind, prec=None, selector=None):
    prec = S.SRJ_PREC_F64 if prec is None else prec
    sel = S.SRJ_SEL_HEURISTIC if selector is None else selector
    dt = torch.float32 if prec == S.SRJ_PREC_F32 else torch.float64
    ad = dev(adiag)
    ao = [dev(a) for a in aoff]
    h = S.srj_create(n, precision=prec, tol_kind=tol_kind, selector=sel, trace_capacity=100000,
                     a_diag_ptr=ad.data_ptr(), a_off_ptrs=[a.data_ptr() for a in ao])
    try:
        fd = dev(f, dt)
        ud = torch.zeros_like(fd)
        st = S.srj_solve(h, fd.data_ptr(), ud.data_ptr(), tol)
        lv, rn = S.srj_get_trace(h)
        return st, ud.cpu().double().numpy(), lv, rn
    finally:
        S.srj_destroy(h)


@pytest.mark.parametrize("N,seed", [(2, 1), (10, 2), (100, 3), (1000, 4), (1000, 5)])
@pytest.mark.parametrize("rule", ["heuristic", "increasing"])
def test_random_tridiagonal_matches_oracle(S, orc, N, seed, rule):
    # Sec. 4.1: b = 1, u0 = 0, absolute L2 tolerance 1e-7
    d, e = inputs.random_sdd_tridiagonal(N, seed=seed)
    b = np.ones(N)
    P = orc.Problem([N], adiag=d, aoff=[e])
    ref = orc.srj_solve(P, b, tol=1e-7, tol_kind="abs", rule=rule)
    sel = S.SRJ_SEL_HEURISTIC if rule == "heuristic" else S.SRJ_SEL_INCREASING
    st, u, lv, rn = _solve(S, [N], d, [e], b, 1e-7, S.SRJ_TOL_ABS, selector=sel)
    assert ref["status"] == 0 and st["status"] == S.SRJ_OK
    np.testing.assert_array_equal(lv, ref["levels"])
    assert st["sweeps"] == ref["sweeps"]
    np.testing.assert_allclose(u, ref["u"], rtol=0, atol=1e-10 * np.abs(ref["u"]).max())
    # evaluating f - A u loses about eps || |A| |u| || to cancellation, and the
    # two iterates carry independent rounding: the per-cycle norms agree to
    # that scale (64 eps of it), not relative to a tiny late-cycle norm
    absA = orc.Problem([N], adiag=np.abs(d), aoff=[np.abs(e)])
    floor = np.linalg.norm(orc.apply_A(absA, np.abs(ref["u"])))
    np.testing.assert_allclose(rn, ref["rns"], rtol=1e-9, atol=64 * 2.0 ** -52 * floor)


@pytest.mark.parametrize("n", [[70, 45], [33, 20, 17]])
def test_explicit_2d_3d_matches_oracle(S, orc, n):
    adiag, aoff = _random_sdd(n, seed=len(n))
    f = inputs.uniform_rhs(n, seed=8).ravel()
    P = orc.Problem(n, adiag=adiag, aoff=aoff)
    ref = orc.srj_solve(P, f, tol=1e-8)
    st, u, lv, rn = _solve(S, n, adiag, aoff, f, 1e-8, S.SRJ_TOL_REL)
    assert ref["status"] == 0 and st["status"] == S.SRJ_OK
    np.testing.assert_array_equal(lv, ref["levels"])
    np.testing.assert_allclose(u, ref["u"], rtol=0, atol=1e-10 * np.abs(ref["u"]).max())


def test_explicit_mixed_precision_residual(S, orc):
    # FP64 refinement around FP32-pair sweeps on the explicit operator: the
    # FP64 residual of the returned solution meets the tolerance
    n = [300, 200]
    adiag, aoff = _random_sdd(n, seed=11)
    f = inputs.uniform_rhs(n, seed=12).ravel()
    st, u, lv, rn = _solve(S, n, adiag, aoff, f, 1e-8, S.SRJ_TOL_REL, prec=S.SRJ_PREC_MIXED)
    P = orc.Problem(n, adiag=adiag, aoff=aoff)
    assert st["status"] == S.SRJ_OK
    r0 = orc.residual_norm(P, np.zeros(P.size), f)
    assert orc.residual_norm(P, u, f) < 1e-8 * r0 * 1.0000001


def test_explicit_poisson_coefficients_equal_constant_path(S):
    # Poisson written out explicitly gives the constant-coefficient levels
    n = [64, 48]
    c = [(n[0] + 1) ** 2, (n[1] + 1) ** 2]
    N = n[0] * n[1]
    f = inputs.uniform_rhs(n, seed=2).ravel()
    st, u, lv, rn = _solve(S, n, np.full(N, 2.0 * (c[0] + c[1])),
                           [np.full(N, -float(c[0])), np.full(N, -float(c[1]))], f, 1e-8,
                           S.SRJ_TOL_REL)
    h = S.srj_create(n, trace_capacity=100000)
    try:
        fd = dev(f)
        ud = torch.zeros_like(fd)
        st0 = S.srj_solve(h, fd.data_ptr(), ud.data_ptr(), 1e-8)
        lv0, _ = S.srj_get_trace(h)
    finally:
        S.srj_destroy(h)
    np.testing.assert_array_equal(lv, lv0)
    np.testing.assert_allclose(u, ud.cpu().numpy(), rtol=0, atol=1e-10 * np.abs(u).max())


def test_explicit_argument_checks(S):
    import ctypes as C
    L = S.load()
    ad = dev(np.full(16, 4.0))
    ao = dev(np.full(16, -1.0))

    def rc(k=None, off=True, **kw):
        g = S._grid([4, 4], None, kw.pop("bc", None))
        stc = S.srj_stencil()
        stc.k = k
        stc.a_diag = ad.data_ptr()
        stc.a_off[0] = ao.data_ptr()
        stc.a_off[1] = ao.data_ptr() if off else None
        o = S.srj_opts()
        for key, val in kw.items():
            setattr(o, key, val)
        hnd = C.c_void_p()
        r = L.srj_create(C.byref(g), C.byref(stc), C.byref(o), None, C.byref(hnd))
        if r == S.SRJ_OK:
            L.srj_destroy(hnd)
        return r

    assert rc() == S.SRJ_OK
    assert rc(k=ad.data_ptr()) == S.SRJ_EINVAL
    assert rc(off=False) == S.SRJ_EINVAL
    assert rc(bc=[1, 0]) == S.SRJ_EUNSUPPORTED
    assert rc(tol_kind=S.SRJ_TOL_DINF) == S.SRJ_EUNSUPPORTED
