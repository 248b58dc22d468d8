"""The forwarded form the evaluation kernels execute (``fiesta_micro_ops``, a host-only
call of the library): evaluated on the CPU it gives the word program's results bit for
bit, every multiply-add has the fixed operands that make fma(X, Y, Z) equal to its
opcode, and it is never longer than the program."""
import ctypes as C
import os

import numpy as np
import pytest

import workloads as W
from paper_1511_03614_gb300 import build, _native as N, prepare_feynman, prepare_direct
from paper_1511_03614_gb300.bytecode import NAMES, Program, encode

import bytecode_interp as BI

REF_SLOT, REF_X, REF_FIXED = 0xC000, 0xD000, 0xE000
FIX_ZERO, FIX_ONE, FIX_MONE = REF_FIXED, REF_FIXED + 1, REF_FIXED + 2
FIXED = (-0.0, 1.0, -1.0)
# opcode -> the references fixed by its multiply-add form: (position, reference)
ROLES = {"ADD": ((1, FIX_ONE),), "SUB": ((1, FIX_MONE),), "MUL": ((2, FIX_ZERO),),
         "NEG": ((1, FIX_MONE), (2, FIX_ZERO)), "MAC": (), "ADDC": ((1, FIX_ONE),),
         "MULC": ((2, FIX_ZERO),), "MACC": (), "MOV": ((1, FIX_ONE), (2, FIX_ZERO))}


def _lib():
    if not os.path.exists(build.LIB):
        pytest.skip("library not built")
    return N.load()


def micro_ops(lib, prog, dim):
    code = np.ascontiguousarray(prog.code, dtype=np.uint32)
    cons = np.ascontiguousarray(prog.consts, dtype=np.float64)
    if cons.size == 0:
        cons = np.zeros(1)
    outs = np.ascontiguousarray(prog.out_slots, dtype=np.int32)
    p = N.Program(dim, code.size, len(prog.consts), prog.n_slots, prog.out_slot, 0, 0, 0,
                  code.ctypes.data_as(C.POINTER(C.c_uint32)), cons.ctypes.data_as(C.POINTER(C.c_double)),
                  len(prog.out_slots), outs.ctypes.data_as(C.POINTER(C.c_int32)), 0)
    n = lib.fiesta_micro_ops(C.byref(p), None, 0)
    assert n >= 0, lib.fiesta_last_error()
    out = (C.c_uint64 * max(n, 1))()
    assert lib.fiesta_micro_ops(C.byref(p), out, n) == n
    return [int(w) for w in out[:n]]


def run_forwarded(words, prog, X):
    """The forwarded words on the CPU, each opcode computed as the word interpreter
    computes it, its operands fetched by reference."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    s = np.zeros((prog.n_slots, n))
    c = np.asarray(prog.consts, dtype=np.float64)

    def val(r):
        if r < REF_SLOT:
            return np.full(n, c[r])
        if r < REF_X:
            return s[r - REF_SLOT]
        if r < REF_FIXED:
            return X[:, r - REF_X]
        return np.full(n, FIXED[r - REF_FIXED])

    with np.errstate(all="ignore"):
        for w in words:
            op, d = w & 0xFF, (w >> 8) & 0xFF
            x, y, z = (w >> 16) & 0xFFFF, (w >> 32) & 0xFFFF, w >> 48
            name = NAMES[op]
            if name in ("ADD", "ADDC"):
                r = val(x) + val(z)
            elif name == "SUB":
                r = val(z) - val(x)
            elif name in ("MUL", "MULC"):
                r = val(x) * val(y)
            elif name == "NEG":
                r = -val(x)
            elif name in ("MAC", "MACC"):
                r = val(x) * val(y) + val(z)
            elif name == "MOV":
                r = val(x).copy()
            elif name == "DIV":
                r = val(x) / val(y)
            elif name == "POWI":
                e = y - 256 if y >= 128 else y
                r = val(x) ** e
            elif name == "LOG":
                r = np.log(val(x))
            elif name == "INV":
                r = 1.0 / val(x)
            elif name == "ATAN2":
                r = np.arctan2(val(x), val(y))
            else:
                raise AssertionError(f"{name} must not be executed")
            s[d] = r
    if len(prog.out_slots) > 1:
        return np.stack([s[o].copy() for o in prog.out_slots], axis=1)
    return s[prog.out_slot].copy()


def _check(lib, prog, dim, rng):
    words = micro_ops(lib, prog, dim)
    assert len(words) <= len(prog.code)
    for w in words:
        name = NAMES[w & 0xFF]
        assert name not in ("LDX", "LDC")
        refs = ((w >> 16) & 0xFFFF, (w >> 32) & 0xFFFF, w >> 48)
        for pos, ref in ROLES.get(name, ()):
            assert refs[pos] == ref, (name, refs)
    X = rng.uniform(0.01, 0.99, size=(48, dim))
    np.testing.assert_array_equal(run_forwarded(words, prog, X), BI.run(prog, X))
    return len(words), len(prog.code)


def _sample(units, k, rng):
    by_slots = sorted(range(len(units)), key=lambda i: -units[i].program.n_slots)[:4]
    rest = rng.choice(len(units), size=min(k, len(units)), replace=False).tolist()
    return sorted(set(by_slots) | set(rest))


@pytest.mark.parametrize("name,kind", [("box", "fused"), ("double_box", "fused"), ("double_box", "unfused"),
                                       ("box", "mixed"), ("box", "terms"), ("stress", "direct"),
                                       ("higher_poles", "direct")])
def test_forwarded_program_matches_word_program(name, kind):
    lib = _lib()
    rng = np.random.default_rng(71)
    if kind == "direct":
        probs = W.stress_suite(300) if name == "stress" else W.higher_pole_suite()
        prep = prepare_direct(probs, name)
    else:
        prep = prepare_feynman(getattr(W, name)(), fuse_orders=kind != "unfused",
                               mix_sectors=3 if kind == "mixed" else 1, separate_terms=kind == "terms")
    done, before = 0, 0
    for i in _sample(prep.units, 24, rng):
        u = prep.units[i]
        a, b = _check(lib, u.program, u.dim, rng)
        done += a
        before += b
    assert done < before          # every workload loads coordinates, so something was forwarded


def test_forwarded_program_copies():
    """A MOV read after the next instruction stays a copy; results held by LDX, LDC or
    MOV are settled in their slots; a MOV folded into a multiply-add takes its source."""
    lib = _lib()
    rng = np.random.default_rng(72)
    code = [encode("LDX", 0, 0), encode("LDX", 1, 1), encode("MOV", 2, 0), encode("ADD", 3, 2, 1),
            encode("MOV", 4, 3), encode("MAC", 4, 0, 1), encode("MUL", 5, 2, 4), encode("LDC", 6, 0, 0),
            encode("MOV", 7, 5)]
    prog = Program(np.array(code, dtype=np.uint32), np.array([2.5]), 8, 7, 2, {}, (7, 6, 1, 4))
    words = micro_ops(lib, prog, 2)
    names = [NAMES[w & 0xFF] for w in words]
    # MOV 2 <- 0 is read two instructions later: a copy; MOV 4 <- 3 folds into the MAC;
    # the results 7 (MOV), 6 (LDC) and 1 (LDX) are settled by copies at the end
    assert names == ["MOV", "ADD", "MAC", "MUL", "MOV", "MOV", "MOV"], names
    X = rng.uniform(0.1, 0.9, size=(16, 2))
    np.testing.assert_array_equal(run_forwarded(words, prog, X), BI.run(prog, X))
