"""Normalising-flow importance sampler (oracle, numpy float64).

Not in the paper: the learned proposal that stands in for the Vegas map.  The
flow is a bijection of the open unit cube built from affine coupling layers in
logit space (Dinh, Sohl-Dickstein, Bengio, "Density estimation using Real NVP",
2017), used for importance sampling as in neural importance sampling (Muller et
al., 2019).  Notation of this module:

    a = logit(x);  for layer l = 0..L-1 with conditioning set A_l and
    transformed set B_l:  (s, t) = MLP_l(a masked to A_l),  s = S tanh(raw_s / S),
                          a_j <- a_j exp(s_j) + t_j  (j in B_l);
    z = sigmoid(a)  is uniform under the model, so
    log q(x) = sum_j [-log x_j - log(1 - x_j)] + sum_l sum_{j in B_l} s_lj
               + sum_j [log z_j + log(1 - z_j)].

Sampling runs the layers backwards from z ~ U(0,1)^d.  MLP_l: 16 -> 64 -> 64 ->
16 with ReLU; input j < 8 is a_j on A_l and 0 elsewhere; outputs 0..7 are raw_s,
8..15 are t.  Masks: A_0 = even j, A_1 = odd j, A_2 = j < ceil(d/2),
A_3 = j >= ceil(d/2).  Training minimises L = -sum_i w_i log q(x_i) over
samples of the current flow with fixed normalised weights w_i proportional
to (|f_i| / q_i)^p (p = 1: KL divergence; p = 2: variance of f/q).
"""
from __future__ import annotations

import numpy as np

L_LAYERS = 4
HID = 64
IN = 16
OUT = 16
S_BOUND = 4.0

# parameter layout per layer (float32 master copy; the same order on the device)
SHAPES = [("W1", (IN, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, OUT)), ("b3", (OUT,))]
PER_LAYER = sum(int(np.prod(s)) for _, s in SHAPES)
N_PARAMS = L_LAYERS * PER_LAYER


def masks(d):
    half = (d + 1) // 2
    A = [[j % 2 == 0 for j in range(d)], [j % 2 == 1 for j in range(d)],
         [j < half for j in range(d)], [j >= half for j in range(d)]]
    return [np.array(m, dtype=bool) for m in A]


def unpack(theta):
    out = []
    off = 0
    for _ in range(L_LAYERS):
        layer = {}
        for name, shape in SHAPES:
            n = int(np.prod(shape))
            layer[name] = theta[off:off + n].reshape(shape)
            off += n
        out.append(layer)
    return out


def init_params(rng, scale=0.05):
    """Small random hidden weights and zero output layer: the flow starts as the identity."""
    theta = np.zeros(N_PARAMS)
    layers = unpack(theta)
    for p in layers:
        p["W1"][...] = rng.normal(0, scale, p["W1"].shape)
        p["W2"][...] = rng.normal(0, scale, p["W2"].shape)
    return theta


def _mlp(p, inp):
    h1p = inp @ p["W1"] + p["b1"]
    h1 = np.maximum(h1p, 0)
    h2p = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(h2p, 0)
    out = h2 @ p["W3"] + p["b3"]
    return h1p, h1, h2p, h2, out


def _cond_input(a, A):
    n, d = a.shape
    inp = np.zeros((n, IN))
    inp[:, :d] = np.where(A[None, :], a, 0.0)
    return inp


def _st(out, d):
    raw = out[:, :d]
    s = S_BOUND * np.tanh(raw / S_BOUND)
    t = out[:, 8:8 + d]
    return s, t, raw


def log_q(theta, x):
    """log q(x) for points x (n, d) in (0,1)^d."""
    n, d = x.shape
    layers = unpack(theta)
    M = masks(d)
    a = np.log(x) - np.log1p(-x)
    lq = -np.sum(np.log(x) + np.log1p(-x), axis=1)
    for l in range(L_LAYERS):
        A = M[l]
        B = ~A
        *_, out = _mlp(layers[l], _cond_input(a, A))
        s, t, _ = _st(out, d)
        a = np.where(B[None, :], a * np.exp(s) + t, a)
        lq += np.sum(np.where(B[None, :], s, 0.0), axis=1)
    z = 1.0 / (1.0 + np.exp(-a))
    lq += np.sum(-np.logaddexp(0, -a) - np.logaddexp(0, a), axis=1)     # log z + log(1 - z)
    return lq


def sample(theta, z):
    """x and log q(x) for base points z (n, d) in (0,1)^d (layers run backwards)."""
    n, d = z.shape
    layers = unpack(theta)
    M = masks(d)
    a = np.log(z) - np.log1p(-z)
    lq = np.sum(np.log(z) + np.log1p(-z), axis=1)
    for l in reversed(range(L_LAYERS)):
        A = M[l]
        B = ~A
        *_, out = _mlp(layers[l], _cond_input(a, A))
        s, t, _ = _st(out, d)
        a = np.where(B[None, :], (a - t) * np.exp(-s), a)
        lq += np.sum(np.where(B[None, :], s, 0.0), axis=1)
    x = 1.0 / (1.0 + np.exp(-a))
    lq += np.sum(np.logaddexp(0, -a) + np.logaddexp(0, a), axis=1)      # -log x - log(1 - x)
    return x, lq


def loss_and_grad(theta, x, w):
    """L = -sum_i w_i log q(x_i) and dL/dtheta by reverse-mode differentiation (float64)."""
    n, d = x.shape
    layers = unpack(theta)
    M = masks(d)
    a = np.log(x) - np.log1p(-x)
    lq = -np.sum(np.log(x) + np.log1p(-x), axis=1)
    cache = []
    for l in range(L_LAYERS):
        A = M[l]
        B = ~A
        inp = _cond_input(a, A)
        h1p, h1, h2p, h2, out = _mlp(layers[l], inp)
        s, t, raw = _st(out, d)
        cache.append((a.copy(), inp, h1p, h1, h2p, h2, s, raw))
        a = np.where(B[None, :], a * np.exp(s) + t, a)
        lq += np.sum(np.where(B[None, :], s, 0.0), axis=1)
    sig = 1.0 / (1.0 + np.exp(-a))
    lq += np.sum(-np.logaddexp(0, -a) - np.logaddexp(0, a), axis=1)
    L = -np.sum(w * lq)
    # backward: g = dL/da, c = dL/d lq = -w
    c = -w
    g = c[:, None] * (1.0 - 2.0 * sig)
    grad = np.zeros_like(theta)
    glayers = unpack(grad)
    for l in reversed(range(L_LAYERS)):
        A = M[l]
        B = ~A
        a_in, inp, h1p, h1, h2p, h2, s, raw = cache[l]
        p = layers[l]
        gp = glayers[l]
        es = np.exp(s)
        ds = np.where(B[None, :], g * a_in * es + c[:, None], 0.0)
        dt = np.where(B[None, :], g, 0.0)
        g_in = np.where(B[None, :], g * es, g)
        draw = ds * (1.0 - np.tanh(raw / S_BOUND) ** 2)
        dout = np.zeros((n, OUT))
        dout[:, :d] = draw
        dout[:, 8:8 + d] = dt
        gp["W3"] += h2.T @ dout
        gp["b3"] += dout.sum(0)
        dh2 = (dout @ p["W3"].T) * (h2p > 0)
        gp["W2"] += h1.T @ dh2
        gp["b2"] += dh2.sum(0)
        dh1 = (dh2 @ p["W2"].T) * (h1p > 0)
        gp["W1"] += inp.T @ dh1
        gp["b1"] += dh1.sum(0)
        dinp = dh1 @ p["W1"].T
        g = g_in + np.where(A[None, :], dinp[:, :d], 0.0)
    return L, grad


def adam_step(theta, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015); returns the new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
