"""GPU parity of the Sec. 3 data collection (srj_collect_moves, one trial per
CTA) with the oracle's (oracle_collect_moves), through the C ABI.

The moves come from the same counter-based generator on both sides, so the
walks agree exactly -- levels and actions -- over every step both make.  The
residual norms are FP64 computations in different rounding orders, and a
cycle amplifies a rounding error by at most its partial-product growth
(<= M^2 for the application order, pinned in test_oracle_schemes); the walks
reach levels far above what the small systems need, where that noise reaches
1e-8.  So every norm must agree within 1e-9 relative plus
noise = 1e-14 ||b|| Mmax^2 (Mmax: the largest M the walk has tried so far),
the previous ratio q = r_before / r_prev within 1e-9 q + (noise + q noise) /
r_prev, and the two walks may stop at different steps only where the
stopping residual lies within that noise of the tolerance."""
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


def _gpu(S, n, ntrials, max_steps, seed, tol=1e-8, max_level=24, f=None, trial0=0):
    rec_bytes = 32
    out = torch.zeros(ntrials * 3 * max_steps * rec_bytes // 8, dtype=torch.float64,
                      device="cuda")
    counts = torch.zeros(ntrials, dtype=torch.int32, device="cuda")
    fd = None if f is None else torch.as_tensor(f, device="cuda")
    S.srj_collect_moves(n, None if fd is None else fd.data_ptr(), tol, max_level, seed, trial0,
                        ntrials, max_steps, out.data_ptr(), counts.data_ptr())
    recs = out.cpu().numpy().view(np.dtype(S.MOVE_RECORD_DTYPE)).reshape(ntrials, 3 * max_steps)
    return recs, counts.cpu().numpy()


CASES = [(1, 24, 3, None), (2, 24, 4, None), (5, 24, 5, None), (37, 24, 6, None),
         (100, 24, 7, None), (400, 24, 8, None), (60, 3, 9, None), (90, 24, 10, "random")]


@pytest.mark.parametrize("n,max_level,seed,rhs", CASES,
                         ids=["N%d_top%d_%s" % (c[0], c[1], c[3] or "ones") for c in CASES])
def test_collection_matches_oracle(S, orc, n, max_level, seed, rhs):
    ntrials, max_steps, tol = 6, 3000, 1e-8
    f = inputs.uniform_rhs([n], seed=seed).ravel() if rhs else np.ones(n)
    recs, counts = _gpu(S, n, ntrials, max_steps, seed, tol, max_level,
                        f=f if rhs else None, trial0=5)
    P = orc.Problem([n])
    bnorm = float(np.linalg.norm(f))
    LM = np.array([S.srj_level_m(l) for l in range(25)], dtype=np.float64)
    for i in range(ntrials):
        ref = orc.collect_moves(P, f, tol=tol, max_level=max_level, seed=seed, trial=5 + i,
                                max_steps=max_steps)
        m = min(int(counts[i]), len(ref["action"]))
        g = recs[i, :counts[i]]
        lv, ac = ref["level"], ref["action"]
        np.testing.assert_array_equal(g["level"][:m], lv[:m])
        np.testing.assert_array_equal(g["action"][:m], ac[:m])
        mmax = np.maximum.accumulate(LM[lv + ac])
        noise = 1e-14 * bnorm * mmax ** 2
        for key in ("r_before", "r_after"):
            err = np.abs(g[key][:m] - ref[key][:m])
            assert np.all(err <= 1e-9 * ref[key][:m] + noise[:m]), (key, i, err.max())
        q = ref["prev_ratio"][:m]
        rprev = ref["r_before"][:m] / q
        err = np.abs(g["prev_ratio"][:m] - q)
        assert np.all(err <= 1e-9 * q + (noise[:m] + q * noise[:m]) / rprev), (i, err.max())
        if counts[i] != len(ref["action"]):
            # one walk stopped and the other did not: the taken residual there
            # must lie within the noise of the tolerance
            last = ref["r_after"][m - 1]
            assert abs(last - tol) <= noise[m - 1] + 1e-9 * tol, (i, counts[i], len(lv), last)
        assert ref["taken"].max() <= max_level


def test_collection_argument_checks(S):
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    counts = torch.zeros(2, dtype=torch.int32, device="cuda")
    for bad in (dict(n=0), dict(n=4097), dict(max_level=25), dict(tol=0.0), dict(ntrials=0),
                dict(max_steps=0)):
        kw = dict(n=10, tol=1e-8, max_level=24, ntrials=1, max_steps=1)
        kw.update(bad)
        with pytest.raises(S.SrjError):
            S.srj_collect_moves(kw["n"], None, kw["tol"], kw["max_level"], 0, 0, kw["ntrials"],
                                kw["max_steps"], out.data_ptr(), counts.data_ptr())
