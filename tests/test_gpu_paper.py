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
