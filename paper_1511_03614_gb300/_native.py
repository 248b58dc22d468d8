"""ctypes declarations of the C ABI in include/fiesta.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

FIESTA_OK = 0
ERRORS = {-1: "FIESTA_E_INVALID", -2: "FIESTA_E_NOMEM", -3: "FIESTA_E_CUDA",
          -4: "FIESTA_E_TIMEOUT", -5: "FIESTA_E_NONFINITE"}
RNG = {"philox": 0, "sobol": 1}
PROPOSAL = {"vegas": 0, "flow": 1}
METHOD = {"vegas": 0, "rqmc": 1, "cuhre": 2}
PRECISION = {"fp64": 0, "fp32": 1, "auto": 2, "dd": 3}
NBINS = 128
MAX_DIM = 8
FLOW_PARAMS = 4 * (16 * 64 + 64 + 64 * 64 + 64 + 64 * 16 + 16)


class Program(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_instr", C.c_int32), ("n_const", C.c_int32), ("n_slots", C.c_int32),
                ("out_slot", C.c_int32), ("order", C.c_int32), ("sector", C.c_int32), ("rng_key", C.c_uint32),
                ("code", C.POINTER(C.c_uint32)), ("consts", C.POINTER(C.c_double)), ("n_out", C.c_int32),
                ("out_slots", C.POINTER(C.c_int32)), ("cplx", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Alloc(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("rng", C.c_int32), ("precision", C.c_int32), ("n_iter", C.c_int32), ("adapt", C.c_int32),
                ("points_per_iter", C.c_int64), ("seed", C.c_uint64), ("alpha", C.c_double),
                ("skip_first", C.c_int32), ("order_lo", C.c_int32), ("unit_begin", C.c_int64),
                ("unit_end", C.c_int64), ("timeout_ms", C.c_int64), ("threads", C.c_int32),
                ("reset_grid", C.c_int32), ("iter_offset", C.c_int32), ("points_per_thread", C.c_int32),
                ("probe_points", C.c_int64), ("fp32_budget", C.c_double), ("no_graph", C.c_int32),
                ("accumulate", C.c_int32), ("small_x", C.c_double),
                ("unit_points", C.POINTER(C.c_int64)), ("small_x32", C.c_double), ("proposal", C.c_int32),
                ("flow_train_steps", C.c_int32), ("flow_keep", C.c_int64), ("flow_lr", C.c_double),
                ("flow_power", C.c_int32), ("wide_threads", C.c_int32)]


class AccuracyOptions(C.Structure):
    _fields_ = [("method", C.c_int32), ("proposal", C.c_int32), ("precision", C.c_int32), ("allocate", C.c_int32),
                ("target", C.c_double), ("floor", C.c_double), ("points", C.c_int64),
                ("iters_per_call", C.c_int32), ("max_iters", C.c_int32), ("skip", C.c_int32),
                ("max_calls", C.c_int32), ("seed", C.c_uint64), ("max_gpu_s", C.c_double),
                ("small_x", C.c_double), ("small_x32", C.c_double), ("pre", C.POINTER(C.c_double)),
                ("n_pre", C.c_int32), ("pre_q", C.c_int32), ("correlated", C.c_int32), ("out_lo", C.c_int32),
                ("replicates", C.c_int32), ("adapt_iters", C.c_int32), ("adapt_points", C.c_int64),
                ("max_points", C.c_int64), ("train_rounds", C.c_int32), ("steps_per_round", C.c_int32),
                ("lr", C.c_double), ("power", C.c_int32), ("reserved", C.c_int32), ("keep", C.c_int64),
                ("rel_tol", C.c_double), ("shrink", C.c_double), ("max_passes", C.c_int32),
                ("reserved2", C.c_int32), ("max_regions", C.c_int64)]


class AccuracyState(C.Structure):
    _fields_ = [("sw", C.POINTER(C.c_double)), ("swi", C.POINTER(C.c_double)), ("n_used", C.POINTER(C.c_double)),
                ("iterations", C.c_int32), ("converged", C.c_int32), ("gpu_ms", C.c_double), ("points", C.c_int64),
                ("ratio", C.c_double), ("points_per_replicate", C.c_int64), ("rel_tol", C.c_double),
                ("order_sw", C.POINTER(C.c_double)), ("order_swi", C.POINTER(C.c_double))]


class UnitResult(C.Structure):
    _fields_ = [("value", C.c_double), ("sigma", C.c_double), ("chi2_dof", C.c_double), ("n_points", C.c_int64),
                ("order", C.c_int32), ("sector", C.c_int32), ("n_nonfinite", C.c_int64), ("precision", C.c_int32),
                ("unit", C.c_int32), ("part", C.c_int32), ("pad", C.c_int32), ("fp32_error", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("gpu_ms", C.c_double), ("eval_ms", C.c_double), ("points", C.c_int64),
                ("points_per_s", C.c_double), ("kernels_launched", C.c_int32), ("eval_launches", C.c_int32),
                ("units_fp32", C.c_int64), ("unit_points", C.c_int64), ("threads", C.c_int32 * 2),
                ("points_per_thread", C.c_int32 * 2), ("points_ext", C.c_int64),
                ("wide_threads", C.c_int32 * 2), ("wide_points_per_thread", C.c_int32 * 2),
                ("eval_groups", C.c_int32), ("pad", C.c_int32)]


class CuhreOptions(C.Structure):
    _fields_ = [("rel_tol", C.c_double), ("abs_tol", C.c_double), ("max_passes", C.c_int32),
                ("order_lo", C.c_int32), ("max_regions", C.c_int64), ("unit_begin", C.c_int64),
                ("unit_end", C.c_int64), ("timeout_ms", C.c_int64), ("threads", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class CuhreResult(C.Structure):
    _fields_ = [("value", C.c_double), ("error", C.c_double), ("n_regions", C.c_int64), ("n_points", C.c_int64),
                ("order", C.c_int32), ("sector", C.c_int32), ("unit", C.c_int32), ("part", C.c_int32),
                ("converged", C.c_int32), ("passes", C.c_int32)]


EXPORTS = {
    "fiesta_load_sectors": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Program), C.c_int64, C.POINTER(Alloc),
                                      C.c_void_p]),
    "fiesta_integrate": (C.c_int, [C.c_void_p, C.POINTER(Options), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.c_int32, C.POINTER(UnitResult), C.POINTER(Stats)]),
    "fiesta_integrate_to_accuracy": (C.c_int, [C.c_void_p, C.POINTER(AccuracyOptions), C.POINTER(AccuracyState),
                                               C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                               C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                               C.POINTER(C.c_double)]),
    "fiesta_assemble": (C.c_int, [C.POINTER(AccuracyOptions), C.c_int64, C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int32,
                                  C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "fiesta_allocate_points": (C.c_int, [C.POINTER(AccuracyOptions), C.c_int64, C.POINTER(C.c_double), C.c_int64,
                                         C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "fiesta_eval_batch": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p]),
    "fiesta_iterations": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    "fiesta_precision_probe": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_uint64,
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "fiesta_get_grid": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    "fiesta_set_grid": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    "fiesta_refine": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.POINTER(C.c_double),
                                C.POINTER(C.c_double)]),
    "fiesta_probe_peaks": (C.c_int, [C.POINTER(C.c_double), C.c_int32]),
    "fiesta_sample_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_uint64, C.c_int32,
                                        C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "fiesta_flow_init": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double]),
    "fiesta_flow_params": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_float), C.c_int32]),
    "fiesta_flow_sample": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_uint64, C.c_int32, C.c_int32,
                                     C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(Stats)]),
    "fiesta_flow_train": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_double, C.c_int32,
                                    C.POINTER(C.c_double), C.POINTER(Stats)]),
    "fiesta_flow_check": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_float)]),
    "fiesta_cuhre": (C.c_int, [C.c_void_p, C.POINTER(CuhreOptions), C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.c_int32, C.POINTER(CuhreResult), C.POINTER(Stats)]),
    "fiesta_cuhre_regions": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "fiesta_free": (None, [C.c_void_p]),
    "fiesta_last_error": (C.c_char_p, []),
    "fiesta_version": (C.c_int, []),
    "fiesta_abi_sizes": (C.c_int, [C.POINTER(C.c_int64), C.c_int32]),
    "fiesta_micro_ops": (C.c_int64, [C.c_void_p, C.POINTER(C.c_uint64), C.c_int64]),
}

# the ctypes mirrors in the order fiesta_abi_sizes reports the C structures
ABI_STRUCTS = ("Program", "Alloc", "Options", "UnitResult", "Stats", "AccuracyOptions", "AccuracyState",
               "CuhreOptions", "CuhreResult")

_lib = None


class FiestaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path=None):
    """Load the compiled library; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() "
                           "(or python -m paper_1511_03614_gb300.build) on a machine with nvcc")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code):
    if code != FIESTA_OK:
        msg = _lib.fiesta_last_error().decode(errors="replace") if _lib else ""
        raise FiestaError(code, msg)
