"""Pins of the learned-selector oracle (oracle/mlp_oracle.py) against torch's
independent implementations (nn.Linear, autograd, optim.Adam, bfloat16) and
central finite differences."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2011_06636_gb300 import inputs

torch = pytest.importorskip("torch")


def _torch_net(theta):
    W1, b1, W2, b2, W3, b3 = [torch.tensor(a) for a in M.unpack(theta)]
    net = torch.nn.Sequential(torch.nn.Linear(12, 64), torch.nn.ReLU(), torch.nn.Linear(64, 64),
                              torch.nn.ReLU(), torch.nn.Linear(64, 25)).double()
    with torch.no_grad():
        for lin, W, b in zip([net[0], net[2], net[4]], [W1, W2, W3], [b1, b2, b3]):
            lin.weight.copy_(W)
            lin.bias.copy_(b)
    return net


def _data(n=37, seed=1):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 12)), rng.integers(0, 25, size=n)


def test_param_count_and_init():
    assert M.N_PARAMS == 6617
    th = inputs.mlp_init(0)
    assert th.shape == (6617,) and th.dtype == np.float32
    W1 = M.unpack(th)[0]
    assert np.max(np.abs(W1)) <= math.sqrt(6 / 12)


def test_forward_matches_torch():
    th = inputs.mlp_init(3).astype(np.float64)
    th[6000:] += 0.1  # nonzero biases in the last layer
    X, _ = _data()
    ref = _torch_net(th)(torch.tensor(X)).detach().numpy()
    assert np.max(np.abs(M.forward(th, X) - ref)) < 1e-12


def test_gradient_matches_autograd_and_finite_differences():
    th = inputs.mlp_init(4).astype(np.float64)
    X, y = _data()
    loss, g = M.loss_and_grad(th, X, y)
    net = _torch_net(th)
    tl = torch.nn.functional.cross_entropy(net(torch.tensor(X)), torch.tensor(y))
    tl.backward()
    tg = np.concatenate([p.grad.numpy().ravel() for p in [net[0].weight, net[0].bias, net[2].weight,
                                                          net[2].bias, net[4].weight, net[4].bias]])
    assert abs(loss - tl.item()) < 1e-12
    assert np.max(np.abs(g - tg)) < 1e-12
    rng = np.random.default_rng(9)
    for i in rng.choice(M.N_PARAMS, size=25, replace=False):
        e = np.zeros_like(th)
        e[i] = 1e-6
        fd = (M.loss_and_grad(th + e, X, y)[0] - M.loss_and_grad(th - e, X, y)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_adam_step_matches_torch():
    th = inputs.mlp_init(5).astype(np.float64)
    X, y = _data()
    net = _torch_net(th)
    opt = torch.optim.Adam(net.parameters(), lr=1e-3)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for t in range(1, 4):
        _, g = M.loss_and_grad(th, X, y)
        th, m, v = M.adam_step(th, m, v, g, t, 1e-3)
        opt.zero_grad()
        torch.nn.functional.cross_entropy(net(torch.tensor(X)), torch.tensor(y)).backward()
        opt.step()
    ref = np.concatenate([p.detach().numpy().ravel() for p in net.parameters()])
    assert np.max(np.abs(th - ref)) < 1e-12


def test_bf16_rounding_matches_torch():
    a = np.random.default_rng(6).standard_normal(10000).astype(np.float32) * 10
    a[:4] = [0.0, -0.0, 1.0000001, 3.0e-39]
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(M.bf16_round(a), ref)
    assert np.array_equal(M.bits_to_f32(M.bf16_bits(a)), ref)


def test_features():
    x = M.features([0.5, 0.25], npoints=4096 * 4096, dim=2, level=24)
    assert x[0] == pytest.approx(math.log(0.5)) and x[1] == pytest.approx(math.log(0.25))
    assert np.all(x[2:8] == 0)
    assert x[8] == pytest.approx(math.log10(4096 ** 2) / 10)
    assert x[9] == pytest.approx(2 / 3) and x[10] == 1.0 and x[11] == pytest.approx(1.0)
    assert M.features([1e-30], 10, 1, 0)[0] == -20.0


def _theta_with_logits(z):
    """Parameters whose network returns the logits z for every input: all
    weights zero, the last bias set to z (the hidden layers output zeros)."""
    th = np.zeros(M.N_PARAMS)
    th[-M.N_OUT:] = z
    return th


def test_decide_moves_clamps_and_ties():
    """The selector's move rule: argmax of the logits over {L-1, L, L+1}
    inside [0, 24], ties to the lower level.  Each case fails a plausible
    slip: a global argmax, ties to the higher level, no clamp at either end."""
    x = np.zeros(12)
    # global maximum far away: only the three neighbouring levels count
    z = np.zeros(25)
    z[20] = 9.0
    z[6] = 1.0
    assert M.decide(_theta_with_logits(z), x, 5) == 6
    z = np.zeros(25)
    z[0] = 9.0
    z[4] = 1.0
    assert M.decide(_theta_with_logits(z), x, 5) == 4
    # all equal: the lowest of the three moves
    assert M.decide(_theta_with_logits(np.zeros(25)), x, 5) == 4
    # a tie between two moves above a third: the lower of the two
    z = np.zeros(25)
    z[5] = z[6] = 2.0
    assert M.decide(_theta_with_logits(z), x, 5) == 5
    z = np.zeros(25)
    z[4] = z[6] = 2.0
    assert M.decide(_theta_with_logits(z), x, 5) == 4
    # level 0 cannot decrease; with equal logits it stays
    assert M.decide(_theta_with_logits(np.zeros(25)), x, 0) == 0
    z = np.zeros(25)
    z[1] = 1.0
    assert M.decide(_theta_with_logits(z), x, 0) == 1
    # the top level cannot increase, even when its own logit loses
    z = np.zeros(25)
    z[23] = 1.0
    assert M.decide(_theta_with_logits(z), x, 24) == 23
    assert M.decide(_theta_with_logits(np.zeros(25)), x, 24) == 23
    z = np.zeros(25)
    z[24] = 1.0
    assert M.decide(_theta_with_logits(z), x, 24) == 24
    # a lowered top clamps the move set too
    z = np.zeros(25)
    z[11] = 5.0
    z[10] = 1.0
    assert M.decide(_theta_with_logits(z), x, 10, top=10) == 10
    # every decision is one of the allowed moves, on random logits
    rng = np.random.default_rng(4)
    for _ in range(200):
        z = rng.standard_normal(25)
        L = int(rng.integers(0, 25))
        got = M.decide(_theta_with_logits(z), x, L)
        allowed = [c for c in (L - 1, L, L + 1) if 0 <= c <= 24]
        assert got in allowed
        assert z[got] == max(z[c] for c in allowed)
