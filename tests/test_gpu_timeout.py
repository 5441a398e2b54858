"""Failure detection without a GPU fault: the 3D pass waits for every plane it
stages in shared memory a bounded number of polls.  A limit of zero polls
makes the first wait give up at once, deterministically; the solve must then
end with SRJ_ETIMEOUT (after the pass has drained the copies it had in
flight), return cleanly, and the same handle must solve normally once the
default limit is restored.  Nothing here faults, traps or hangs the GPU: the
waits that run out are waits on copies that do complete."""
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
    srj.load(build_if_missing=False)
    return srj


def _solve_raw(S, h, f, u, tol):
    st = S.srj_stats()
    rc = S.load().srj_solve(h, f.data_ptr(), u.data_ptr(), float(tol), C.byref(st))
    return rc, st.as_dict()


# several 32 x 8 column tiles and z chunks, too large for the one-CTA solve
GRID = [40, 24, 70]


@pytest.mark.parametrize("depth", [0, 2])
@pytest.mark.parametrize("prec", ["F64", "MIXED"])
def test_wait_that_runs_out_ends_the_solve_cleanly(S, orc, prec, depth):
    """depth 2: the graph runs the two-sweep pass and the one-sweep tail pass
    side by side; the first pass (the initial residual, a tail pass) gives up."""
    p = getattr(S, "SRJ_PREC_" + prec)
    f_np = inputs.uniform_rhs(GRID, seed=31).ravel()
    f = torch.as_tensor(f_np, device="cuda")
    h = S.srj_create(GRID, precision=p, temporal_depth=depth)
    try:
        for _ in range(2):  # two timed-out solves in a row
            S.srj_set_wait_limit(h, 0)
            u = torch.zeros_like(f)
            rc, st = _solve_raw(S, h, f, u, 1e-8)
            torch.cuda.synchronize()  # the context is intact
            assert rc == S.SRJ_ETIMEOUT, (rc, st)
            assert st["status"] == S.SRJ_ETIMEOUT
            assert st["sweeps"] == 0
            assert torch.isfinite(u).all()
        # the default limit again: a normal solve on the same handle
        S.srj_set_wait_limit(h, -1)
        u = torch.zeros_like(f)
        rc, st = _solve_raw(S, h, f, u, 1e-8)
        ug = u.cpu().numpy()
    finally:
        S.srj_destroy(h)
    assert rc == S.SRJ_OK, (rc, st)
    P = orc.Problem(GRID)
    ref = orc.srj_solve(P, f_np, tol=1e-8)
    assert orc.residual_norm(P, ug, f_np) / ref["r0"] < 1e-8
    if prec == "F64":
        assert st["sweeps"] == ref["sweeps"]
        assert np.max(np.abs(ug - ref["u"])) <= 1e-10 * np.max(np.abs(ref["u"]))


def test_wait_limit_argument_checks(S):
    with pytest.raises(S.SrjError):
        S.srj_set_wait_limit(None, 5)
    h = S.srj_create(GRID)
    try:
        S.srj_set_wait_limit(h, 1 << 30)  # a long limit is accepted as is
        S.srj_set_wait_limit(h, -5)       # any negative value: the default
    finally:
        S.srj_destroy(h)
