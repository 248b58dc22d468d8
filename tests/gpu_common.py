"""Shared helpers of the GPU tests (prepared problems cached per process)."""
import functools

import numpy as np
import pytest

import workloads as W
from oracle import pipeline as P


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_03614_gb300 import build
    build.build()
    return torch


@functools.lru_cache(maxsize=None)
def feynman(name):
    from paper_1511_03614_gb300 import prepare_feynman
    prob = getattr(W, name)()
    return prepare_feynman(prob), P.feynman_problem(prob)


@functools.lru_cache(maxsize=None)
def integrator(name):
    from paper_1511_03614_gb300 import Integrator
    prep, _ = feynman(name)
    return Integrator(prep)


@functools.lru_cache(maxsize=None)
def stress(n):
    from paper_1511_03614_gb300 import prepare_direct, Integrator
    probs = W.stress_suite(n)
    prep = prepare_direct(probs)
    return probs, prep, Integrator(prep)


def sample_points(dim, rng, n_random=96):
    """Random interior points plus boundary points (coordinates at 2^-40, 2^-20, 1 - 2^-20, 1/2)."""
    X = [rng.uniform(0.0, 1.0, size=(n_random, dim))]
    edge = np.array([2.0 ** -40, 2.0 ** -20, 1 - 2.0 ** -20, 0.5])
    B = rng.choice(edge, size=(32, dim))
    X.append(B)
    for j in range(dim):
        Y = np.full((len(edge), dim), 0.5)
        Y[:, j] = edge
        X.append(Y)
    return np.concatenate(X)
