"""Plain numpy oracle of the learned scheme selector.

TEST INFRASTRUCTURE ONLY (imported by tests/ and nowhere in the product).

The paper selects the next scheme level with Alg. 1 (Sec. 3), a rule read off
convergence data collected by trying the three moves up / same / down from
solver states (Sec. 3, data-collection procedure).  The learned selector
replaces that rule by a small MLP over the same kind of state; it is not in
the paper.  This module is the slow, obviously correct CPU statement of what
the library's kernels compute:

  features (12): log of the last 8 residual ratios (most recent first, 0 when
                 fewer cycles ran, clipped to [-20, 5]); log10(#points)/10;
                 dim/3; level/24; log(M(level))/log(2362)
  network:       h1 = relu(W1 x + b1)   64 x 12
                 h2 = relu(W2 h1 + b2)  64 x 64
                 z  = W3 h2 + b3        25 x 64   (one logit per level)
  decision:      argmax z over the moves {L-1, L, L+1} from the current
                 level L inside [0, 24] (ties to the lower level)
  weights:       BF16 (round to nearest even) for inference, FP32 masters for
                 training; parameter vector = W1, b1, W2, b2, W3, b3 row-major.
  training:      softmax cross-entropy, mean over the batch, Adam.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_H, N_OUT = 12, 64, 25
SHAPES = [(N_H, N_IN), (N_H,), (N_H, N_H), (N_H,), (N_OUT, N_H), (N_OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)  # 6617
LEVEL_M = [1, 2, 3, 5, 7, 10, 14, 19, 26, 35, 47, 63, 84, 111, 147, 194, 256, 338,
           446, 589, 778, 1027, 1356, 1790, 2362]


def unpack(theta):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def features(ratios_recent_first, npoints, dim, level):
    x = np.zeros(N_IN)
    for i, r in enumerate(list(ratios_recent_first)[:8]):
        x[i] = min(5.0, max(-20.0, math.log(r))) if r > 0 else -20.0
    x[8] = math.log10(npoints) / 10.0
    x[9] = dim / 3.0
    x[10] = level / 24.0
    x[11] = math.log(LEVEL_M[level]) / math.log(2362.0)
    return x


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest even), returned as float32."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def bf16_bits(a):
    return (bf16_round(a).view(np.uint32) >> 16).astype(np.uint16)


def bits_to_f32(bits):
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32)


def forward(theta, X):
    """Logits (n x 25) in FP64 for features X (n x 12)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ W3.T + b3


def predict(theta, X):
    return np.argmax(forward(theta, X), axis=1)


def loss_and_grad(theta, X, y):
    """Mean softmax cross-entropy and its gradient (backpropagation)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    y = np.asarray(y, dtype=np.int64)
    n = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3.T + b3
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    p = e / e.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(p[np.arange(n), y])))
    dz = p.copy()
    dz[np.arange(n), y] -= 1.0
    dz /= n
    gW3 = dz.T @ h2
    gb3 = dz.sum(axis=0)
    dh2 = dz @ W3
    da2 = dh2 * (a2 > 0)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * (a1 > 0)
    gW1 = da1.T @ X
    gb1 = da1.sum(axis=0)
    g = np.concatenate([t.ravel() for t in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g


def adam_step(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba): returns new (theta, m, v); t counts from 1."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def decide(theta, x, level, top=24):
    """The selector's next level from features x at current level `level`."""
    z = forward(theta, np.asarray(x, dtype=np.float64)[None, :])[0]
    moves = [c for c in (level - 1, level, level + 1) if 0 <= c <= top]
    return max(moves, key=lambda c: (z[c], -c))
