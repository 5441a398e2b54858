"""GPU parity of the learned selector: device inference and training against
the numpy oracle (oracle/mlp_oracle.py), and a solve driven by the selector
against an oracle loop that makes its decisions with the oracle network.

Argmax decisions are compared where the oracle's top-two logit margin is
larger than the FP32 accumulation error bound (64 products of BF16 weights and
FP32 activations per dot product: |error| <= 1e-4 scale here); within the
margin the device pick must be one of the tied levels."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M
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


def _bits(seed, bias_scale=0.3):
    th = inputs.mlp_init(seed).astype(np.float32)
    rng = np.random.default_rng(seed + 1)
    th[M.N_PARAMS - 25:] = rng.standard_normal(25) * bias_scale
    return M.bf16_bits(th)


def test_device_inference_matches_oracle(S):
    bits = _bits(11)
    theta = M.bits_to_f32(bits).astype(np.float64)
    X = np.random.default_rng(2).standard_normal((500, 12)).astype(np.float32)
    pick, logits = S.srj_mlp_forward(bits, X)
    ref = M.forward(theta, X.astype(np.float64))
    assert np.max(np.abs(logits - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))
    srt = np.sort(ref, axis=1)
    margin = srt[:, -1] - srt[:, -2]
    clear = margin > 1e-3
    assert clear.mean() > 0.9
    assert np.array_equal(pick[clear], np.argmax(ref, axis=1)[clear])
    for i in np.where(~clear)[0]:
        assert ref[i, pick[i]] >= srt[i, -1] - 1e-3


def test_device_training_matches_oracle_adam(S):
    rng = np.random.default_rng(4)
    n, B, steps, lr = 256, 32, 5, 1e-3
    X = rng.standard_normal((n, 12)).astype(np.float32)
    y = rng.integers(0, 25, size=n).astype(np.int32)
    order = inputs.minibatch_order(n, 1, 9)[:steps * B]
    th0 = inputs.mlp_init(7)
    theta = torch.as_tensor(th0, device="cuda")
    xd, yd, od = (torch.as_tensor(a, device="cuda") for a in (X, y, order))
    loss = S.srj_mlp_train(xd.data_ptr(), yd.data_ptr(), n, od.data_ptr(), steps, B, lr,
                           theta.data_ptr())
    got = theta.cpu().numpy().astype(np.float64)
    ref = th0.astype(np.float64)
    m = np.zeros_like(ref)
    v = np.zeros_like(ref)
    ref_loss = []
    gabs = np.zeros_like(ref)
    for t in range(steps):
        idx = order[t * B:(t + 1) * B]
        lo, g = M.loss_and_grad(ref, X[idx].astype(np.float64), y[idx])
        ref_loss.append(lo)
        gabs = np.maximum(gabs, np.abs(g))
        ref, m, v = M.adam_step(ref, m, v, g, t + 1, lr)
    assert np.allclose(loss, ref_loss, rtol=1e-5, atol=1e-6)
    # Adam normalises each gradient component; components whose gradient is
    # tiny can flip sign between FP32 and FP64, so only well-conditioned
    # components are compared tightly, the rest within the step bound
    well = gabs > 1e-4
    assert np.max(np.abs(got - ref)[well]) <= 1e-5
    assert np.max(np.abs(got - ref)) <= steps * lr * 1.0001


def _oracle_mlp_solve(orc, P, f, theta, tol, max_cycles=400):
    """The solver loop of Sec. 3 with the level chosen by the oracle network
    among the moves {L-1, L, L+1} (ties to the lower level) and Alg. 1 as
    judge: after a picked cycle that did not shrink the residual, or shrank
    it more slowly per sweep (average convergence rate, Sec. 3) than the
    latest cycle Alg. 1 chose, Alg. 1 takes the next decision."""
    u = np.zeros(P.size)
    r0 = orc.residual_norm(P, u, f)
    rprev, level, hist, levels, by_mlp = r0, 0, [], [], False
    alg1_rate = 0.0
    npts = P.size
    for _ in range(max_cycles):
        u, rn = orc.run_levels(P, f, u, [level])
        rn = rn[0]
        levels.append(level)
        ratio = rn / rprev
        rprev = rn
        rate = -math.log(ratio) / orc.level_m(level)
        hist = [min(5.0, max(-20.0, math.log(ratio)))] + hist
        if rn / r0 < tol:
            return u, levels
        if not by_mlp:
            alg1_rate = rate
        if by_mlp and (ratio >= 1.0 or rate < alg1_rate):
            level = orc.next_level(0, ratio, level)
            by_mlp = False
        else:
            x = M.features([math.exp(v) for v in hist[:8]], npts, len(P.n), level)
            z = M.forward(theta, x[None, :].astype(np.float32).astype(np.float64))[0]
            moves = [c for c in (level - 1, level, level + 1) if 0 <= c <= 24]
            level = max(moves, key=lambda c: (z[c], -c))
            by_mlp = True
    raise AssertionError("oracle loop did not converge")


@pytest.mark.parametrize("n", [[384], [96, 80]])
def test_selector_solve_matches_oracle_loop(S, orc, n):
    """The library's trained weights (committed with the package) drive both
    the GPU solve and the oracle loop; decisions and solutions must agree."""
    from paper_2011_06636_gb300 import selector
    bits = selector.load_weights()
    theta = M.bits_to_f32(bits).astype(np.float64)
    f = inputs.uniform_rhs(n, seed=3).ravel()
    P = orc.Problem(n)
    u_ref, lv_ref = _oracle_mlp_solve(orc, P, f, theta, 1e-8)
    h = S.srj_create(n, selector=S.SRJ_SEL_MLP, precision=S.SRJ_PREC_F64, max_sweeps=200000)
    fd = torch.as_tensor(f, device="cuda")
    ud = torch.zeros_like(fd)
    try:
        S.srj_mlp_set_weights(h, bits)
        st = S.srj_solve(h, fd.data_ptr(), ud.data_ptr(), 1e-8)
        lv, _ = S.srj_get_trace(h)
    finally:
        S.srj_destroy(h)
    assert st["status"] == S.SRJ_OK
    assert list(lv) == lv_ref
    assert np.max(np.abs(ud.cpu().numpy() - u_ref)) <= 1e-10 * np.max(np.abs(u_ref))


def test_selector_requires_weights(S):
    h = S.srj_create([64], selector=S.SRJ_SEL_MLP)
    fd = torch.ones(64, dtype=torch.float64, device="cuda")
    ud = torch.zeros_like(fd)
    try:
        with pytest.raises(S.SrjError):
            S.srj_solve(h, fd.data_ptr(), ud.data_ptr(), 1e-8, raise_on_notconv=True)
    finally:
        S.srj_destroy(h)
