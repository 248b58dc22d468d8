"""The allocation-free sampling pass, fiesta_sample_noalloc, against fiesta_integrate.

Some callers cannot allocate device memory while they run (code that must not
synchronise the device, a memory pool fixed at start-up, a host program with no
allocator hooked up).  For them the library offers one sampling pass whose
scratch lives in a fixed device array inside the library.  This file checks,
through the C ABI, that the pass gives what a one-iteration, non-adaptive
fiesta_integrate gives on the same points, on two calls in a row (the shared
array keeps the previous call's contents, which must not leak into the next),
with host and with device output arrays, and that oversized requests are
refused.  It is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_03614_gb300 import build, prepare_feynman, Integrator, _native as N
    build.build()
    prep = prepare_feynman(W.box())
    return torch, N, prep, Integrator(prep)


def _reference(integ, n_units, points, seed):
    integ.integrate(n_iter=1, points=points, seed=seed, adapt=False, reset_grid=True)
    m = np.empty(n_units)
    v = np.empty(n_units)
    for k in range(n_units):
        a, b = integ.iterations(k, 1)
        m[k], v[k] = a[0], b[0]
    return m, v


def test_noalloc_pass_matches_integrate_twice():
    torch, N, prep, integ = _setup()
    lib = N.load()
    nu = len(prep.units)
    points, seed = 40_000, 17
    m_ref, v_ref = _reference(integ, nu, points, seed)
    for call in range(2):
        m = np.full(nu, np.nan)
        v = np.full(nu, np.nan)
        rc = lib.fiesta_sample_noalloc(integ.ctx, 0, nu, points, seed, 0, 0, 0,
                                       m.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p))
        assert rc == 0, lib.fiesta_last_error()
        assert np.all(np.abs(m - m_ref) <= 1e-12 * np.abs(m_ref) + 1e-300), call
        assert np.all(np.abs(v - v_ref) <= 1e-12 * np.abs(v_ref) + 1e-300), call
    # device outputs, and a smaller second slice (the previous contents must not leak in)
    md = torch.full((nu,), float("nan"), dtype=torch.float64, device="cuda")
    vd = torch.full((nu,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.fiesta_sample_noalloc(integ.ctx, 0, nu, points, seed, 0, 0, 0,
                                   C.c_void_p(md.data_ptr()), C.c_void_p(vd.data_ptr()))
    assert rc == 0, lib.fiesta_last_error()
    torch.cuda.synchronize()
    assert np.all(np.abs(md.cpu().numpy() - m_ref) <= 1e-12 * np.abs(m_ref))
    m2 = np.empty(4)
    v2 = np.empty(4)
    rc = lib.fiesta_sample_noalloc(integ.ctx, 3, 7, points, seed, 0, 0, 0,
                                   m2.ctypes.data_as(C.c_void_p), v2.ctypes.data_as(C.c_void_p))
    assert rc == 0, lib.fiesta_last_error()
    assert np.all(np.abs(m2 - m_ref[3:7]) <= 1e-12 * np.abs(m_ref[3:7]))


def test_noalloc_pass_rejects_oversized_requests():
    torch, N, prep, integ = _setup()
    lib = N.load()
    nu = len(prep.units)
    m = np.empty(nu)
    v = np.empty(nu)
    rc = lib.fiesta_sample_noalloc(integ.ctx, 0, nu, 10_000_000, 1, 0, 0, 0,
                                   m.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p))
    assert rc == -1
    assert b"maximum is 65536" in lib.fiesta_last_error()


def test_noalloc_pass_reports_nonfinite_samples():
    """A NaN constant planted on the host in one program: with host outputs the pass
    returns FIESTA_E_NONFINITE naming the unit (as fiesta_integrate does), with device
    outputs it marks that unit's variance NaN; a clean unit beside it is unaffected."""
    torch, N, _, _ = _setup()
    from paper_1511_03614_gb300 import parse_text, Integrator
    lib = N.load()
    prep = parse_text("1; 0; x[1]*0.5 + 1.0; |")
    prep.units.append(parse_text("1; 0; x[1]*0.5 + 1.0; |").units[0])
    prep.units[1].program.consts[:] = np.nan
    for k, u in enumerate(prep.units):
        u.rng_key = k
    integ = Integrator(prep)
    m = np.full(2, -1.0)
    v = np.full(2, -1.0)
    rc = lib.fiesta_sample_noalloc(integ.ctx, 0, 2, 10_000, 3, 0, 0, 0,
                                   m.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p))
    assert rc == -5 and b"unit 1" in lib.fiesta_last_error()
    assert abs(m[0] - 1.25) < 1e-2 and np.isfinite(v[0]) and m[1] == 0.0
    md = torch.zeros(2, dtype=torch.float64, device="cuda")
    vd = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = lib.fiesta_sample_noalloc(integ.ctx, 0, 2, 10_000, 3, 0, 0, 0,
                                   C.c_void_p(md.data_ptr()), C.c_void_p(vd.data_ptr()))
    assert rc == 0, lib.fiesta_last_error()
    vh = vd.cpu().numpy()
    assert np.isfinite(vh[0]) and np.isnan(vh[1]) and abs(md[0].item() - m[0]) <= 1e-12 * abs(m[0])
    integ.close()
