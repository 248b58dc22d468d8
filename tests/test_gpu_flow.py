"""GPU tests of the learned proposal: the tensor-core sampler and the training
kernel against the flow oracle, unbiasedness, and the gain over Vegas."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import flow as F

from gpu_common import need_gpu, feynman

pytestmark = pytest.mark.gpu


def _bf16(a):
    """Round to bfloat16 (nearest even), returned as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _sampler_bf16(theta, z):
    """The sampler as the device computes it: BF16 weights, MLP inputs and hidden activations."""
    n, d = z.shape
    layers = F.unpack(theta)
    M = F.masks(d)
    z = z.astype(np.float32).astype(np.float64)
    a = np.log(z) - np.log1p(-z)
    lq = np.sum(np.log(z) + np.log1p(-z), axis=1)
    for l in reversed(range(F.L_LAYERS)):
        p = layers[l]
        inp = _bf16(F._cond_input(a, M[l]))
        h1 = _bf16(np.maximum(inp @ _bf16(p["W1"]) + p["b1"], 0))
        h2 = _bf16(np.maximum(h1 @ _bf16(p["W2"]) + p["b2"], 0))
        out = h2 @ _bf16(p["W3"]) + p["b3"]
        s, t, _ = F._st(out, d)
        B = ~M[l]
        a = np.where(B[None, :], (a - t) * np.exp(-s), a)
        lq += np.sum(np.where(B[None, :], s, 0.0), axis=1)
    x = 1 / (1 + np.exp(-a))
    lq += np.sum(np.logaddexp(0, -a) + np.logaddexp(0, a), axis=1)
    return x, lq


def _loss_grad_bf16(theta, x, w):
    """L and dL/dtheta as the tensor-core training kernel computes them: the oracle's
    reverse mode with BF16 rounding of every MMA operand (layer inputs, weights,
    hidden activations, dout, dH2, dH1) and the ReLU masks taken on the rounded
    activations; sums and the coupling arithmetic unrounded."""
    n, d = x.shape
    layers = F.unpack(theta)
    M = F.masks(d)
    a = np.log(x) - np.log1p(-x)
    lq = -np.sum(np.log(x) + np.log1p(-x), axis=1)

    def mlp(p, inp):
        inb = _bf16(inp)
        h1 = _bf16(np.maximum(inb @ _bf16(p["W1"]) + p["b1"], 0))
        h2 = _bf16(np.maximum(h1 @ _bf16(p["W2"]) + p["b2"], 0))
        return inb, h1, h2, h2 @ _bf16(p["W3"]) + p["b3"]

    cache = []
    for l in range(F.L_LAYERS):
        B = ~M[l]
        inp = F._cond_input(a, M[l])
        inb, h1, h2, out = mlp(layers[l], inp)
        s, t, raw = F._st(out, d)
        cache.append((a.copy(), inb, h1, h2, raw))
        a = np.where(B[None, :], a * np.exp(s) + t, a)
        lq += np.sum(np.where(B[None, :], s, 0.0), axis=1)
    sig = 1 / (1 + np.exp(-a))
    lq += np.sum(-np.logaddexp(0, -a) - np.logaddexp(0, a), axis=1)
    L = -np.sum(w * lq)
    g = -w[:, None] * (1 - 2 * sig)
    grad = np.zeros_like(theta)
    gl = F.unpack(grad)
    for l in reversed(range(F.L_LAYERS)):
        A, B = M[l], ~M[l]
        a_in, inb, h1, h2, raw = cache[l]
        p, gp = layers[l], gl[l]
        th = np.tanh(raw / F.S_BOUND)
        es = np.exp(F.S_BOUND * th)
        ds = np.where(B[None, :], (g * a_in * es - w[:, None]) * (1 - th * th), 0.0)
        dt = np.where(B[None, :], g, 0.0)
        g_in = np.where(B[None, :], g * es, g)
        dout = np.zeros((n, F.OUT))
        dout[:, :d] = ds
        dout[:, 8:8 + d] = dt
        dout = _bf16(dout)
        gp["W3"] += h2.T @ dout
        gp["b3"] += dout.sum(0)
        dh2 = _bf16((dout @ _bf16(p["W3"]).T) * (h2 > 0))
        gp["W2"] += h1.T @ dh2
        gp["b2"] += dh2.sum(0)
        dh1 = _bf16((dh2 @ _bf16(p["W2"]).T) * (h1 > 0))
        gp["W1"] += inb.T @ dh1
        gp["b1"] += dh1.sum(0)
        dinp = dh1 @ _bf16(p["W1"]).T
        g = g_in + np.where(A[None, :], dinp[:, :d], 0.0)
    return L, lq, grad


def _random_theta(seed):
    rng = np.random.default_rng(seed)
    th = F.init_params(rng, 0.15)
    for p in F.unpack(th):
        p["W3"][...] = rng.normal(0, 0.05, p["W3"].shape)
        p["b3"][...] = rng.normal(0, 0.05, p["b3"].shape)
        p["b1"][...] = rng.normal(0, 0.05, p["b1"].shape)
    return th.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("dim", [3, 6])
def test_flow_kernels_match_oracle(dim):
    need_gpu()
    from paper_1511_03614_gb300 import parse_text, Integrator
    expr = "+".join(f"x[{j + 1}]*{j + 1}.5" for j in range(dim)) + "+0.25"
    integ = Integrator(parse_text(f"{dim}; 0; {expr}; |"))
    integ.flow_init(seed=3)
    th = _random_theta(dim)
    integ.set_flow_params(0, th.astype(np.float32))
    assert np.array_equal(integ.flow_params(0), th.astype(np.float32))
    rng = np.random.default_rng(7)
    n = 500
    z = rng.uniform(0.02, 0.98, size=(n, dim))
    w = rng.uniform(size=n)
    w /= w.sum()
    out = integ.flow_check(0, z, w)
    # sampler (tensor cores, BF16) against its emulation
    x_ref, lq_ref = _sampler_bf16(th, z)
    assert np.median(np.abs(out["x"] - x_ref)) < 1e-5 and np.max(np.abs(out["x"] - x_ref)) < 2e-3
    assert np.median(np.abs(out["logq"] - lq_ref)) < 1e-4 and np.max(np.abs(out["logq"] - lq_ref)) < 2e-2
    # integrand at the sampled points
    fx = 0.25 + sum((j + 1.5) * out["x"][:, j] for j in range(dim))
    assert np.max(np.abs(out["f"] - fx) / fx) < 1e-12
    # training pass (tensor cores, BF16 operands, binary32 accumulation) at the sampler's
    # x: against its rounding emulation closely, and against the oracle's binary64
    # reverse mode within what BF16 operands allow
    X = out["x"]
    Le, lqe, ge = _loss_grad_bf16(th, X, w)
    dl = np.abs(out["logq_train"] - lqe)
    assert np.median(dl) < 1e-4 and np.max(dl) < 2e-2, (np.median(dl), np.max(dl))
    assert abs(out["loss"] - Le) <= 1e-3 * max(1.0, abs(Le))
    gmax = np.max(np.abs(ge))
    de = np.abs(out["grad"] - ge) / gmax
    print(f"grad vs emulation: median {np.median(de):.2e}, max {np.max(de):.2e}")
    assert np.max(de) <= 2e-3 and np.median(de) <= 1e-6, (np.median(de), np.max(de))
    L, g = F.loss_and_grad(th, X, w)
    assert abs(out["loss"] - L) <= 1e-2 * max(1.0, abs(L))
    d64 = np.abs(out["grad"] - g) / np.max(np.abs(g))
    print(f"grad vs binary64 oracle: median {np.median(d64):.2e}, max {np.max(d64):.2e}")
    assert np.max(d64) <= 3e-2, np.max(d64)


def test_flow_estimates_are_unbiased_on_the_box():
    need_gpu()
    from paper_1511_03614_gb300 import Integrator
    from paper_1511_03614_gb300.api import run_flow
    prep, _ = feynman("box")
    res = run_flow(Integrator(prep), target=1e-3, points=200_000, keep=2048, train_rounds=4, steps_per_round=10,
                   max_rounds=12)
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        s = res["errors"][n]
        assert abs(res["values"][n] - v) < 4 * s + 1e-5, (n, res["values"][n], v, s)


def test_flow_on_fused_units():
    """One flow per sector for all its eps orders (trained on the norm of the result
    vector): the box's closed form within 4 sigma, and the per-result records."""
    need_gpu()
    from paper_1511_03614_gb300 import Integrator, prepare_feynman
    from paper_1511_03614_gb300.api import run_flow
    prep = prepare_feynman(W.box(), fuse_orders=True)
    integ = Integrator(prep)
    integ.flow_init(seed=3)
    m, v, st = integ.flow_sample(20_000, keep=256)
    assert len(m) == sum(u.n_out for u in prep.units) and np.all(v > 0)
    res = run_flow(integ, target=1e-3, points=200_000, keep=2048, train_rounds=4, steps_per_round=10,
                   max_rounds=12)
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, val in exact.items():
        s = res["errors"][n]
        assert abs(res["values"][n] - val) < 4 * s + 1e-5, (n, res["values"][n], val, s)


def test_flow_beats_vegas_on_a_diagonal_ridge():
    """f = 1/((x1 - x2)^2 + a^2): concentrated along the diagonal, which a separable
    Vegas grid cannot follow.  The trained flow's variance per point is lower."""
    need_gpu()
    from paper_1511_03614_gb300 import parse_text, Integrator
    a = 0.1
    exact = 2 * ((1 / a) * math.atan(1 / a) - 0.5 * math.log((1 + a * a) / (a * a)))
    prep = parse_text(f"2; 0; 1/((x[1]-x[2])*(x[1]-x[2])+{a * a!r}); |")
    integ = Integrator(prep)
    N = 200_000
    rv = integ.integrate(n_iter=12, points=N, seed=1)
    m, v = integ.iterations(0, 12)
    vegas_var = v[-1] * N                       # per-point variance on the adapted grid
    assert abs(rv.values[0] - exact) < 4 * rv.errors[0]
    integ.flow_init(seed=2)
    for r in range(12):
        mf, vf, _ = integ.flow_sample(N, seed=5, iteration=r, keep=4096)
        integ.flow_train(25, lr=3e-3, power=1)
    mf, vf, _ = integ.flow_sample(N, seed=5, iteration=100)
    flow_var = vf[0] * N
    assert abs(mf[0] - exact) < 4 * math.sqrt(vf[0])
    assert flow_var < 0.5 * vegas_var, (flow_var, vegas_var)
