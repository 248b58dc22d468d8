"""Pins of the flow oracle: gradients by finite differences, log q by the
numerical Jacobian determinant, sampling as the inverse of the normalising map,
and normalisation of q."""
import numpy as np

from oracle import flow as F


def _theta(seed=0, out_scale=0.3, hidden=0.3):
    rng = np.random.default_rng(seed)
    th = F.init_params(rng, hidden)
    for p in F.unpack(th):
        p["W3"][...] = rng.normal(0, out_scale, p["W3"].shape)
        p["b3"][...] = rng.normal(0, out_scale, p["b3"].shape)
        p["b1"][...] = rng.normal(0, 0.1, p["b1"].shape)
        p["b2"][...] = rng.normal(0, 0.1, p["b2"].shape)
    return th


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    d = 5
    th = _theta()
    x = rng.uniform(0.02, 0.98, size=(16, d))
    w = rng.uniform(size=16)
    w /= w.sum()
    L, g = F.loss_and_grad(th, x, w)
    idx = rng.choice(F.N_PARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        fd = (F.loss_and_grad(th + e, x, w)[0] - F.loss_and_grad(th - e, x, w)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert abs(L + np.sum(w * F.log_q(th, x))) < 1e-12


def test_log_q_is_the_log_jacobian_determinant():
    rng = np.random.default_rng(2)
    d = 3
    th = _theta(3, 0.05, 0.15)
    z = rng.uniform(0.05, 0.95, size=(5, d))
    x, lq = F.sample(th, z)

    def G(xx):          # normalising map x -> z
        a = np.log(xx) - np.log1p(-xx)
        layers = F.unpack(th)
        M = F.masks(d)
        for l in range(F.L_LAYERS):
            *_, out = F._mlp(layers[l], F._cond_input(a, M[l]))
            s, t, _ = F._st(out, d)
            a = np.where(~M[l][None, :], a * np.exp(s) + t, a)
        return 1 / (1 + np.exp(-a))
    assert np.max(np.abs(G(x) - z)) < 1e-10                     # sampling inverts the normalising map
    h = 1e-6
    for i in range(5):
        J = np.zeros((d, d))
        for k in range(d):
            e = np.zeros(d)
            e[k] = h
            J[:, k] = (G(x[i:i + 1] + e) - G(x[i:i + 1] - e))[0] / (2 * h)
        assert abs(np.log(abs(np.linalg.det(J))) - lq[i]) < 1e-6
    assert np.max(np.abs(F.log_q(th, x) - lq)) < 1e-9


def test_density_is_normalised():
    """int q = 1: the importance-sampling estimate of 1 with points from q is exactly 1,
    and the uniform-sample average of q over the cube is 1 within its error."""
    rng = np.random.default_rng(4)
    th = _theta(5, 0.05, 0.15)
    X = rng.uniform(size=(200000, 2))
    q = np.exp(F.log_q(th, X))
    assert abs(q.mean() - 1) < 4 * q.std() / np.sqrt(len(q))


def test_identity_at_initialisation():
    th = F.init_params(np.random.default_rng(0))
    z = np.random.default_rng(1).uniform(size=(10, 6))
    x, lq = F.sample(th, z)
    assert np.max(np.abs(x - z)) < 1e-12 and np.max(np.abs(lq)) < 1e-9
