"""GPU parity of multigrid with SRJ smoothing (srj_mg_create / srj_mg_solve)
against the oracle's V-cycle, through the C ABI.  FP64 both sides: the same
number of V-cycles, final residual norms within 1e-9 relative, solutions
within 1e-10 of max |u| (the two sides sum the restriction, interpolation and
stencil terms in different orders)."""
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


CASES = [([1023], None, 1, 1, 1), ([127, 127], None, 1, 1, 1), ([255, 255], [1.0, 0.5], 0, 1, 1),
         ([63, 63], None, 2, 2, 1), ([31, 31, 31], None, 1, 1, 1), ([63, 63, 63], [0.7, 1.0, 1.3], 0, 2, 2),
         ([1], None, 1, 1, 1), ([3, 3], None, 4, 1, 1)]


@pytest.mark.parametrize("n,eps,level,nu1,nu2", CASES)
def test_mg_matches_oracle(S, orc, n, eps, level, nu1, nu2):
    P = orc.Problem(n, eps=eps)
    f = inputs.uniform_rhs(n, seed=sum(n)).ravel()
    ref = orc.mg_solve(P, f, tol=1e-9, level=level, nu1=nu1, nu2=nu2)
    h = S.srj_mg_create(n, eps=eps, smoother_level=level, nu1=nu1, nu2=nu2)
    try:
        fd, ud = dev(f), torch.zeros(P.size, dtype=torch.float64, device="cuda")
        st = S.srj_mg_solve(h, fd.data_ptr(), ud.data_ptr(), 1e-9)
    finally:
        S.srj_destroy(h)
    assert ref["status"] == 0 and st["status"] == S.SRJ_OK
    assert st["cycles"] == ref["cycles"]
    assert st["r0"] == pytest.approx(ref["r0"], rel=1e-12)
    assert st["rn"] == pytest.approx(ref["rn"], rel=1e-6, abs=1e-12 * ref["r0"])
    u = ud.cpu().numpy()
    np.testing.assert_allclose(u, ref["u"], rtol=0, atol=1e-10 * np.abs(ref["u"]).max())
    M = orc.level_m(level)
    if n != [1]:
        assert st["sweeps"] == st["cycles"] * M * (nu1 + nu2)


def test_mg_full_size_4095_residual(S):
    n = [4095, 4095]
    f = inputs.uniform_rhs(n, seed=0).ravel()
    fd = dev(f)
    ud = torch.zeros_like(fd)
    h = S.srj_mg_create(n, smoother_level=1)
    try:
        st = S.srj_mg_solve(h, fd.data_ptr(), ud.data_ptr(), 1e-8)
    finally:
        S.srj_destroy(h)
    assert st["status"] == S.SRJ_OK and st["cycles"] < 30
    h = S.srj_create(n)  # independent FP64 residual through the SRJ path
    try:
        rn = S.srj_residual_norm(h, fd.data_ptr(), ud.data_ptr())
    finally:
        S.srj_destroy(h)
    assert rn / st["r0"] < 1e-8 * 1.0001
    assert rn == pytest.approx(st["rn"], rel=1e-6)


def test_mg_argument_checks(S):
    import ctypes as C
    L = S.load()

    def rc(n, bc=None, k=None):
        g = S._grid(n, None, bc)
        stc = S.srj_stencil()
        stc.k = k
        hnd = C.c_void_p()
        r = L.srj_mg_create(C.byref(g), C.byref(stc), None, None, C.byref(hnd))
        if r == S.SRJ_OK:
            L.srj_destroy(hnd)
        return r

    kt = dev(np.ones(9 * 9))
    assert rc([7, 7]) == S.SRJ_OK
    assert rc([100]) == S.SRJ_EINVAL
    assert rc([7, 15]) == S.SRJ_EINVAL
    assert rc([7, 7], bc=[1, 0]) == S.SRJ_EINVAL
    assert rc([7, 7], k=kt.data_ptr()) == S.SRJ_EUNSUPPORTED
    # the two kinds of handle do not mix
    hm = S.srj_mg_create([7, 7])
    hs = S.srj_create([7, 7])
    try:
        f = dev(np.ones(49))
        u = torch.zeros_like(f)
        assert L.srj_solve(hm, f.data_ptr(), u.data_ptr(), 1e-8, None) == S.SRJ_EINVAL
        assert L.srj_mg_solve(hs, f.data_ptr(), u.data_ptr(), 1e-8, None) == S.SRJ_EINVAL
        assert L.srj_mg_solve(hm, f.data_ptr(), u.data_ptr(), -1.0, None) == S.SRJ_EINVAL
    finally:
        S.srj_destroy(hm)
        S.srj_destroy(hs)
