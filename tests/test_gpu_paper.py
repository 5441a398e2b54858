"""The paper's iteration-count results reproduced with the GPU solver
(Sec. 4.1 and Sec. 4.2.3), FP64.

Jacobi counts come from the exact spectral closed form that
test_oracle_solver pins against the oracle's plain Jacobi; SRJ counts are the
GPU solver's.  The paper prints approximate numbers read off its figures;
the bands below are the ones the oracle reproduces (15 % for Table 3 at
32^3-64^3) and a wider 30 % where the paper says "approximately"."""
import numpy as np
import pytest

from conftest import read_golden
from test_oracle_solver import _jacobi_sweeps_closed_form

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


def _gpu_srj_sweeps(S, n, rule):
    f = torch.ones(int(np.prod(n)), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = S.srj_create(n, precision=S.SRJ_PREC_F64, selector=rule)
    try:
        st = S.srj_solve(h, f.data_ptr(), u.data_ptr(), 1e-8)
    finally:
        S.srj_destroy(h)
    assert st["status"] == S.SRJ_OK
    return st["sweeps"]


@pytest.mark.parametrize("side", [32, 48, 64, 96, 128, 192, 256])
def test_table3_speedups_on_gpu(S, side):
    """Sec. 4.2.3, Table 3: Jacobi / SRJ+heuristic iterations, 3D Poisson
    f = 1, relative residual 1e-8."""
    table = {int(r[0]): float(r[1]) for r in read_golden("table3_speedup.txt")}
    n = [side] * 3
    srj_sweeps = _gpu_srj_sweeps(S, n, S.SRJ_SEL_HEURISTIC)
    jac = _jacobi_sweeps_closed_form(n, 1e-8)
    ratio = jac / srj_sweeps
    band = 0.15 if side <= 64 else 0.30
    assert abs(ratio / table[side] - 1) <= band, (side, jac, srj_sweeps, ratio)


@pytest.mark.parametrize("side,approx", [(128, 1000), (256, 3000)])
def test_sec423_iteration_counts(S, side, approx):
    """Sec. 4.2.3: SRJ with the heuristic needs approximately 1000 (128^3) and
    3000 (256^3) iterations; the increasing rule needs more."""
    n = [side] * 3
    heur = _gpu_srj_sweeps(S, n, S.SRJ_SEL_HEURISTIC)
    assert abs(heur / approx - 1) <= 0.30, (side, heur)
    inc = _gpu_srj_sweeps(S, n, S.SRJ_SEL_INCREASING)
    assert inc > heur


# ----------------------------------------------- plain Jacobi on the GPU
def _gpu_solve(S, n, f_np, tol, tol_kind=None, **kw):
    f = torch.as_tensor(np.ascontiguousarray(f_np, dtype=np.float64).ravel(), device="cuda")
    u = torch.zeros_like(f)
    if tol_kind is not None:
        kw["tol_kind"] = tol_kind
    h = S.srj_create(n, precision=S.SRJ_PREC_F64, **kw)
    try:
        st = S.srj_solve(h, f.data_ptr(), u.data_ptr(), tol)
    finally:
        S.srj_destroy(h)
    return st, u.cpu().numpy()


@pytest.mark.parametrize("n", [[300], [70, 45], [130, 90], [20, 18, 16], [40, 24, 35]],
                         ids=lambda n: "x".join(map(str, n)))
@pytest.mark.parametrize("check_level", [0, 3])
def test_plain_jacobi_matches_oracle(S, orc, n, check_level):
    """SRJ_SEL_JACOBI (Sec. 2, Eq. jacobi: omega = 1 every sweep) against the
    oracle's plain Jacobi with the residual tested every M(check_level)
    sweeps: the same sweep count and the solution within 1e-10.  The grids
    take the one-CTA solve, the temporally blocked 2D pass and the 3D pass."""
    from paper_2011_06636_gb300 import inputs
    f = inputs.uniform_rhs(n, seed=41).ravel()
    every = S.srj_level_m(check_level)
    st, ug = _gpu_solve(S, n, f, 1e-5, selector=S.SRJ_SEL_JACOBI, fixed_level=check_level)
    ref = orc.jacobi_solve(orc.Problem(n), f, tol=1e-5, check_every=every)
    assert ref["status"] == 0 and st["status"] == S.SRJ_OK
    assert st["sweeps"] == ref["sweeps"]
    assert st["sweeps"] % every == 0
    assert np.max(np.abs(ug - ref["u"])) <= 1e-10 * np.max(np.abs(ref["u"]))


@pytest.mark.parametrize("side", [32, 48, 64])
def test_table3_jacobi_counts_on_gpu(S, side):
    """Table 3's Jacobi iterations run on the GPU (3D Poisson, f = 1, rel
    1e-8, residual tested after every sweep): equal to the exact spectral
    count up to one sweep of rounding at the threshold, and the Jacobi / SRJ
    ratio within 15 % of the paper's."""
    table = {int(r[0]): float(r[1]) for r in read_golden("table3_speedup.txt")}
    n = [side] * 3
    st, _ = _gpu_solve(S, n, np.ones(side ** 3), 1e-8, selector=S.SRJ_SEL_JACOBI)
    assert st["status"] == S.SRJ_OK
    jac = _jacobi_sweeps_closed_form(n, 1e-8)
    assert abs(st["sweeps"] - jac) <= 1, (st["sweeps"], jac)
    srj_sweeps = _gpu_srj_sweeps(S, n, S.SRJ_SEL_HEURISTIC)
    ratio = st["sweeps"] / srj_sweeps
    assert abs(ratio / table[side] - 1) <= 0.15, (side, st["sweeps"], srj_sweeps, ratio)


# Sec. 4.1 in-sample study: 1D Poisson, b = 1, x0 = 0, ||b - A x||_2 < 1e-7
IN_SAMPLE_N = [2, 5, 10, 20, 35, 50, 75, 100, 125, 150, 200, 250, 300, 350, 400]


def test_in_sample_heuristic_vs_increasing_on_gpu(S, orc):
    """Sec. 4.1: over the in-sample sizes N = 2 ... 400 the GPU solver takes the
    oracle's sweep counts with both rules (identical decisions), and the
    heuristic needs at most half the iterations of the increasing rule from
    N = 50 on (the paper's "generally"; below that both need few cycles)."""
    for N in IN_SAMPLE_N:
        counts = {}
        for label, sel, rule in (("heur", S.SRJ_SEL_HEURISTIC, "heuristic"),
                                 ("inc", S.SRJ_SEL_INCREASING, "increasing")):
            st, _ = _gpu_solve(S, [N], np.ones(N), 1e-7, tol_kind=S.SRJ_TOL_ABS, selector=sel)
            ref = orc.srj_solve(orc.Problem([N]), np.ones(N), tol=1e-7, tol_kind="abs", rule=rule)
            assert st["status"] == S.SRJ_OK and ref["status"] == 0
            assert st["sweeps"] == ref["sweeps"], (N, label, st["sweeps"], ref["sweeps"])
            counts[label] = st["sweeps"]
        if N >= 50:
            assert counts["heur"] <= 0.5 * counts["inc"], (N, counts)
