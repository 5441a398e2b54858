"""The allocation-free residual-norm entry point (srj_residual_norm_noalloc)
against the FP64 oracle's residual norm and the library's ordinary
srj_residual_norm, through the C ABI.

It exists for callers that cannot allocate device memory (code running under
a memory pool or budget it does not own, or on a path where cudaFree's
device-wide synchronisation is not acceptable): its reduction scratch is a
fixed device array inside the library.  Two calls in a row must both agree
with the ordinary entry point, so the shared scratch is correctly cleared
between calls.  This file is collected last on purpose."""
import ctypes as C

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
    L = srj.load(build_if_missing=False)
    L.srj_residual_norm_noalloc.argtypes = [C.POINTER(srj.srj_grid), C.POINTER(srj.srj_stencil),
                                            C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                            C.c_void_p]
    L.srj_residual_norm_noalloc.restype = C.c_int
    return srj


def _noalloc(S, n, eps, f, u, h=None):
    g = S._grid(n, h=h)
    st = S.srj_stencil()
    for a in range(3):
        st.eps[a] = eps[a] if a < len(eps) else 0.0
    st.k = None
    out = C.c_double(-1.0)
    rc = S.load().srj_residual_norm_noalloc(C.byref(g), C.byref(st), f.data_ptr(), u.data_ptr(),
                                            C.byref(out), None)
    return rc, out.value


@pytest.mark.parametrize("n,eps", [([1000], [1.0]), ([300, 200], [0.05, 1.0]),
                                   ([40, 30, 20], [1.0, 0.5, 2.0]), ([4096, 4096], [1.0, 1.0])])
def test_noalloc_matches_ordinary_entry_point_twice(S, orc, n, eps):
    f_np = inputs.uniform_rhs(n, seed=1).ravel()
    f = torch.as_tensor(f_np, device="cuda")
    P = orc.Problem(n, eps=eps)
    h = S.srj_create(n, eps=eps, precision=S.SRJ_PREC_F64)
    try:
        for call in range(2):
            u_np = np.random.default_rng(call).standard_normal(f.numel())
            u = torch.as_tensor(u_np, device="cuda")
            want = orc.residual_norm(P, u_np, f_np)
            ref = S.srj_residual_norm(h, f.data_ptr(), u.data_ptr())
            rc, got = _noalloc(S, n, eps, f, u)
            assert rc == S.SRJ_OK
            assert abs(got - want) <= 1e-12 * want, (call, got, want)
            assert abs(got - ref) <= 1e-12 * ref, (call, got, ref)
    finally:
        S.srj_destroy(h)


def test_noalloc_rejects_grids_beyond_its_scratch(S):
    n = [2, 65537]  # 65537 rows > the 65536 rows the fixed scratch holds
    f = torch.zeros(2 * 65537, dtype=torch.float64, device="cuda")
    rc, _ = _noalloc(S, n, [1.0, 1.0], f, f)
    assert rc == S.SRJ_EINVAL


@pytest.mark.parametrize("bad", ["h_negative", "h_nan", "eps_negative", "eps_inf"])
def test_noalloc_rejects_bad_spacing_or_coefficient(S, bad):
    """The same argument checks as srj_create: a negative or non-finite
    spacing or coefficient is SRJ_EINVAL, never silently replaced."""
    n = [64, 32]
    f = torch.zeros(64 * 32, dtype=torch.float64, device="cuda")
    h = {"h_negative": [-1.0 / 65, 1.0 / 33], "h_nan": [float("nan"), 1.0 / 33]}.get(bad)
    eps = {"eps_negative": [-1.0, 1.0], "eps_inf": [1.0, float("inf")]}.get(bad, [1.0, 1.0])
    rc, _ = _noalloc(S, n, eps, f, f, h=h)
    assert rc == S.SRJ_EINVAL
    with pytest.raises(S.SrjError):
        S.srj_create(n, h=h, eps=eps)
