"""Host-side tests of the product path that need no GPU: the preprocessor
against the oracle (through a test-only bytecode interpreter), the validator,
and the C ABI library's exports."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import pipeline as P
from paper_1511_03614_gb300 import bytecode as B, prepare_feynman, prepare_direct, parse_text
from paper_1511_03614_gb300 import prefactor as PF
from oracle.prefactor import prefactor_series

from bytecode_interp import run

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("name", ["bubble", "box"])
def test_programs_match_oracle_integrands(name):
    prob = getattr(W, name)()
    prep = prepare_feynman(prob)
    orc = P.feynman_problem(prob)
    assert [(u.sector, u.order) for u in prep.units] == [(u.sector, u.order) for u in orc.units]
    rng = np.random.default_rng(1)
    for u, o in zip(prep.units, orc.units):
        X = rng.uniform(0.05, 1.0, size=(64, u.dim))
        a, b = run(u.program, X), o.f_numpy(X)
        assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)) < 1e-12


def test_double_box_programs_sample():
    prob = W.double_box()
    prep = prepare_feynman(prob)
    orc = P.feynman_problem(prob)
    assert len(prep.units) == len(orc.units)
    assert [(u.sector, u.order) for u in prep.units] == [(u.sector, u.order) for u in orc.units]
    rng = np.random.default_rng(2)
    for i in rng.choice(len(prep.units), 25, replace=False):
        u, o = prep.units[i], orc.units[i]
        X = rng.uniform(0.05, 1.0, size=(32, u.dim))
        a, b = run(u.program, X), o.f_numpy(X)
        M = P.magnitude_numpy(o, X)
        assert np.all(np.abs(a - b) <= 1e-13 * M), i


def test_stress_programs_sample():
    probs = W.stress_suite(40)
    prep = prepare_direct(probs)
    rng = np.random.default_rng(3)
    for k, prob in enumerate(probs):
        orc = P.direct_problem(prob)
        assert len(orc.units) == 1
        X = rng.uniform(0.0, 1.0, size=(32, prob.dim))
        a, b = run(prep.units[k].program, X), orc.units[0].f_numpy(X)
        M = P.magnitude_numpy(orc.units[0], X)
        assert np.all(np.abs(a - b) <= 1e-13 * M)


def test_prefactor_matches_oracle():
    for idx, L, k in [((1, 1), 1, 4), ((1, 1, 1, 1), 1, 3), ((1,) * 7, 2, 5), ((2, 1), 1, 3)]:
        q1, a = PF.series(idx, L, k)
        q2, b = prefactor_series(idx, L, k)
        assert q1 == q2
        assert max(abs(x - float(y)) for x, y in zip(a, b)) < 1e-13


def test_text_format():
    prep = parse_text("1;\n0;\nx[1]+0.2;\n|")
    assert run(prep.units[0].program, np.array([[0.25]]))[0] == 0.45
    prep = parse_text("2; 1; l[x[1]+x[2]]; p[f[1],2]*x[2] - 1/(1+x[1]); |")
    X = np.array([[0.3, 0.6]])
    assert abs(run(prep.units[0].program, X)[0] - (np.log(0.9) ** 2 * 0.6 - 1 / 1.3)) < 1e-15
    with pytest.raises(ValueError):
        parse_text("1; 0; x[2]; |")


def test_validator_rejects_bad_programs():
    prep = parse_text("1; 0; x[1]*x[1]+0.5; |")
    prog = prep.units[0].program
    B.validate(prog)
    bad = B.Program(prog.code.copy(), prog.consts, prog.n_slots, prog.out_slot, prog.dim, {})
    bad.code[0] = B.encode("ADD", 0, 3, 3)
    with pytest.raises(ValueError):
        B.validate(bad)


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "fiesta.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fiesta_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1511_03614_gb300 import build, _native
    if not os.path.exists(build.LIB):
        try:
            build.build()
        except Exception as e:          # no nvcc here: nothing to check
            pytest.skip(f"cannot build the library: {e}")
    lib = C.CDLL(build.LIB)
    names = _declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_native.EXPORTS)


def test_structure_layouts_match_the_library():
    """Every ctypes mirror has the size of its C structure as the library was compiled
    (host-only call, no GPU)."""
    from paper_1511_03614_gb300 import build, _native as N
    if not os.path.exists(build.LIB):
        pytest.skip("library not built")
    lib = N.load()
    sizes = (C.c_int64 * 16)()
    n = lib.fiesta_abi_sizes(sizes, 16)
    assert n == len(N.ABI_STRUCTS)
    for i, name in enumerate(N.ABI_STRUCTS):
        assert C.sizeof(getattr(N, name)) == sizes[i], (name, C.sizeof(getattr(N, name)), sizes[i])


def test_load_rejects_invalid_program_without_gpu():
    """The validator runs before any device call, so this works on a CPU-only host."""
    from paper_1511_03614_gb300 import build, _native as N
    if not os.path.exists(build.LIB):
        pytest.skip("library not built")
    lib = N.load()
    code = (C.c_uint32 * 1)(B.encode("ADD", 0, 1, 1))
    cons = (C.c_double * 1)(0.0)
    progs = (N.Program * 1)(N.Program(1, 1, 0, 2, 0, 0, 0, 0, code, cons))
    ctx = C.c_void_p()
    rc = lib.fiesta_load_sectors(C.byref(ctx), progs, 1, None, None)
    assert rc == -1 and b"read before written" in lib.fiesta_last_error()


@pytest.mark.parametrize("name", ["bubble", "box", "double_box"])
def test_fused_programs_match_oracle(name):
    """A fused unit's results are the oracle's per-order integrands of its sector."""
    prob = getattr(W, name)()
    prep = prepare_feynman(prob, fuse_orders=True)
    orc = P.feynman_problem(prob)
    by = {(u.sector, u.order): u for u in orc.units}
    assert sum(u.n_out for u in prep.units) >= len(orc.units)
    rng = np.random.default_rng(5)
    idx = range(len(prep.units)) if len(prep.units) < 20 else rng.choice(len(prep.units), 12, replace=False)
    for i in idx:
        u = prep.units[i]
        X = rng.uniform(0.05, 1.0, size=(24, u.dim))
        Fv = run(u.program, X)
        Fv = Fv[:, None] if Fv.ndim == 1 else Fv
        for k in range(u.n_out):
            o = by.get((u.sector, u.order + k))
            if o is None:
                assert np.all(Fv[:, k] == 0)
                continue
            assert np.all(np.abs(Fv[:, k] - o.f_numpy(X)) <= 1e-13 * P.magnitude_numpy(o, X))


@pytest.mark.parametrize("fuse", [False, True])
def test_complex_programs_match_oracle(fuse):
    """Physical box (s > 0, t < 0): each deformed-contour program returns, per eps
    order, the real and imaginary parts of the oracle's deformed integrand."""
    prob = W.box_physical()
    prep = prepare_feynman(prob, fuse_orders=fuse)
    assert prep.complex and all(u.cplx and u.n_out % 2 == 0 for u in prep.units)
    lams = {l for l in prep.lams if l is not None}
    assert len(lams) == 1
    orc = P.feynman_problem(prob, lam=lams.pop())
    by = {(u.sector, u.order): u for u in orc.units}
    rng = np.random.default_rng(6)
    for u in prep.units:
        X = rng.uniform(0.02, 0.98, size=(24, u.dim))
        Fv = run(u.program, X)
        for k in range(u.n_out // 2):
            o = by[(u.sector, u.order + k)]
            b = o.f_numpy(X)
            a = Fv[:, 2 * k] + 1j * Fv[:, 2 * k + 1]
            assert np.all(np.abs(a - b) <= 1e-12 * np.maximum(P.magnitude_numpy(o, X), np.abs(b))), (u.sector, k)



def test_combine_shards_complex_records():
    """Sharded per-unit records of complex units sum re and im separately."""
    from paper_1511_03614_gb300.shard import combine_shards
    r0 = [dict(order=-1, part=0, value=1.0, sigma=0.3), dict(order=-1, part=1, value=2.0, sigma=0.4)]
    r1 = [dict(order=-1, part=0, value=0.5, sigma=0.4), dict(order=-1, part=1, value=-1.0, sigma=0.3)]
    v, e = combine_shards([r0, r1], (-1,))
    assert v[-1] == complex(1.5, 1.0) and abs(e[-1] - complex(0.5, 0.5)) < 1e-15
    v, e = combine_shards([[dict(order=0, value=1.0, sigma=0.6)], [dict(order=0, value=2.0, sigma=0.8)]], (0,))
    assert v[0] == 3.0 and abs(e[0] - 1.0) < 1e-15


def test_no_cpu_fallback():
    """Without a GPU the product path refuses to run (no silent CPU fallback)."""
    import torch
    from paper_1511_03614_gb300 import Integrator
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="CUDA"):
        Integrator(prepare_feynman(W.bubble()))


@pytest.mark.parametrize("name,group", [("box", 3), ("double_box", 4)])
def test_mixed_sector_programs_match_oracle_sums(name, group):
    """MixSectors: every sector lands in exactly one mixed unit, and each result of a
    mixed program is the sum over its sectors of the oracle's integrands of that order."""
    prob = getattr(W, name)()
    prep = prepare_feynman(prob, mix_sectors=group)
    orc = P.feynman_problem(prob)
    cover = sorted(i for u in prep.units for i in u.sectors)
    assert cover == list(range(len(prep.sectors)))
    by = {(u.sector, u.order): u for u in orc.units}
    rng = np.random.default_rng(8)
    idx = range(len(prep.units)) if len(prep.units) < 12 else rng.choice(len(prep.units), 10, replace=False)
    for i in idx:
        u = prep.units[i]
        X = rng.uniform(0.05, 0.95, size=(16, u.dim))
        Fv = run(u.program, X)
        Fv = Fv[:, None] if Fv.ndim == 1 else Fv
        for k in range(u.n_out):
            ref = np.zeros(len(X))
            mag = np.zeros(len(X))
            for s in u.sectors:
                o = by.get((s, u.order + k))
                if o is not None:
                    ref += o.f_numpy(X)
                    mag += P.magnitude_numpy(o, X)
            assert np.all(np.abs(Fv[:, k] - ref) <= 1e-12 * np.maximum(mag, 1e-300)), (i, k)


def test_corner_differences_vanish_exactly_at_the_boundary():
    """Where t_j is so small that its terms fall below half an ulp, a corner value
    P(t_W) and P(t_W, t_j = 0) are the same number, and the subtraction difference
    G(W) - G(W u {j}) must be exactly 0: the following 1/t_j factors would otherwise
    amplify a rounding difference into garbage (in binary32, into inf).  So every corner
    is evaluated by the same operation sequence; this is checked by evaluating every
    fused double-box program in binary32 at extreme coordinates (down to 1e-30, the
    binary32 range a flow sampler reaches, and 1 - 2^-24, 1) and requiring finite
    values."""
    prep = prepare_feynman(W.double_box(), fuse_orders=True)
    vals = np.array([1e-3, 1e-8, 4.7e-15, 1e-20, 1e-30, 0.5, 1.0 - 2.0 ** -24, 1.0])
    rng = np.random.default_rng(41)
    for k, u in enumerate(prep.units):
        X = rng.choice(vals, size=(400, u.dim)).astype(np.float32).astype(np.float64)
        f = run(u.program, X, np.float32)
        assert np.all(np.isfinite(f)), k


@pytest.mark.parametrize("name,fuse", [("box", False), ("box", True), ("double_box", True)])
def test_separate_term_programs_match_oracle(name, fuse):
    """SeparateTerms units: each program (over the variables outside its term's set T)
    computes the oracle's T term of its sector at every order it carries."""
    prob = getattr(W, name)()
    prep = prepare_feynman(prob, fuse_orders=fuse, separate_terms=True)
    rng = np.random.default_rng(8)
    idx = range(len(prep.units)) if name == "box" else rng.choice(len(prep.units), 12, replace=False)
    orc_units = {}
    from oracle import sectors as OS
    full = P.feynman_problem(prob) if name == "box" else None
    secs = full.sectors if full is not None else None
    if secs is None:
        from oracle.uf import symanzik as osym
        U, F, xs = osym(prob)
        prim = OS.primary_sectors(U, F, xs, prob.indices, len(prob.loop_momenta))
        secs = [s for p in prim for s in OS.decompose(p, "M")]
    for i in idx:
        u = prep.units[i]
        sec = secs[u.sector]
        X = rng.uniform(0.05, 1.0, size=(16, u.dim))
        Fv = run(u.program, X)
        Fv = Fv[:, None] if Fv.ndim == 1 else Fv
        for k in range(u.n_out):
            e = OS.unit_integrand(sec, u.order + k, term=u.term)
            var = tuple(j for j in sec.variables if j not in u.term) or (sec.variables[0],)
            o = P.Unit(u.sector, u.order + k, var, e)
            assert o.dim == u.dim
            assert np.all(np.abs(Fv[:, k] - o.f_numpy(X)) <= 1e-13 * P.magnitude_numpy(o, X)), (i, k)


def test_higher_pole_programs_match_oracle():
    """Sectors with a pole of order 2 (Taylor subtraction of order 1, composed with an
    order-0 one in the 2-dimensional cases): every program against the oracle's
    integrand at 50 digits, within 64 u M."""
    import mpmath as mp
    for prob in W.higher_pole_suite():
        prep = prepare_direct([prob])
        orc = P.direct_problem(prob)
        by = {(u.sector, u.order): u for u in orc.units}
        assert len(prep.units) == len(orc.units)
        rng = np.random.default_rng(13)
        for u in prep.units:
            o = by[(u.sector, u.order)]
            X = np.concatenate([rng.uniform(0.05, 1.0, size=(12, u.dim)), np.exp2(-rng.uniform(1, 20, (8, u.dim)))])
            f = run(u.program, X)
            with mp.workdps(50):
                ref = np.array([float(o.f_mp(x, 50)) for x in X])
            M = P.magnitude_numpy(o, X)
            assert np.all(np.abs(f - ref) <= 64 * 2.0 ** -53 * M), (prob.name, u.order)
