"""Python binding of the C ABI: argument marshalling only.

Every step of the integration runs in the CUDA library; PyTorch provides the
device, the stream and (through allocator callbacks) the device memory.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math

import numpy as np

from . import _native as N
from .preprocess import assemble


@dataclasses.dataclass
class Result:
    values: dict              # eps order -> sum over units of that order
    errors: dict              # eps order -> mean-square combined error
    per_unit: list            # dicts: value, sigma, chi2_dof, n_points, order, sector, n_nonfinite
    stats: dict
    assembled: dict = None    # eps order -> value with the prefactor series multiplied in
    assembled_errors: dict = None


def _n_orders(u):
    return u.n_out // 2 if u.cplx else u.n_out


def _record_key(u, o):
    """(eps order, part) of result o of unit u; part 1 is an imaginary part."""
    return (u.order + o // 2, o & 1) if u.cplx else (u.order + o, 0)


def _sum_parts(records):
    """Sums over units per eps order of (order, part, value, sigma) records: complex
    values, and errors complex(sigma_re, sigma_im) each combined in the mean-square norm."""
    v, e = {}, {}
    for K, part, val, sig in records:
        v.setdefault(K, [0.0, 0.0])[part] += val
        e.setdefault(K, [0.0, 0.0])[part] += sig * sig
    return ({K: complex(*x) for K, x in v.items()},
            {K: complex(math.sqrt(x[0]), math.sqrt(x[1])) for K, x in e.items()})


def _assembled(prep, recs, val, sig):
    """Per-order sums of (unit, result) records with values ``val`` and standard errors
    ``sig`` (mean-square combination, Sec. 4.3), then the prefactor series: complex
    values for a problem with complex units.  Returns (assembled, errors, per-order sums)."""
    values, errors = _sum_parts([_record_key(prep.units[unit], o) + (val[k], sig[k])
                                 for k, (unit, o) in enumerate(recs)])
    if not prep.complex:
        values = {K: z.real for K, z in values.items()}
        errors = {K: z.real for K, z in errors.items()}
    R, E = assemble(prep, values, errors)
    return R, E, values


class Integrator:
    """Holds the device copy of a Prepared set of units (one fiesta_ctx)."""

    def __init__(self, prep, device=None, stream=None, torch_alloc=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the integrator has no CPU path")
        self.lib = N.load()
        self.prep = prep
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._torch = torch
        self._bufs = {}
        n = len(prep.units)
        progs = (N.Program * n)()
        keep = []
        for i, u in enumerate(prep.units):
            code = np.ascontiguousarray(u.program.code, dtype=np.uint32)
            cons = np.ascontiguousarray(u.program.consts, dtype=np.float64)
            if cons.size == 0:
                cons = np.zeros(1)
            outs = np.ascontiguousarray(u.program.out_slots, dtype=np.int32)
            keep += [code, cons, outs]
            progs[i] = N.Program(u.dim, code.size, len(u.program.consts), u.program.n_slots, u.program.out_slot,
                                 u.order, u.sector, u.rng_key & 0xFFFFFFFF,
                                 code.ctypes.data_as(C.POINTER(C.c_uint32)),
                                 cons.ctypes.data_as(C.POINTER(C.c_double)), int(u.n_out),
                                 outs.ctypes.data_as(C.POINTER(C.c_int32)), int(bool(u.cplx)))
        self._keep = keep
        alloc = None
        if torch_alloc:
            dev = self.device

            def _alloc(nbytes, user):
                t = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
                self._bufs[t.data_ptr()] = t
                return t.data_ptr()

            def _free(ptr, user):
                self._bufs.pop(ptr, None)
            self._alloc_cb = N.ALLOC_FN(_alloc)
            self._free_cb = N.FREE_FN(_free)
            alloc = N.Alloc(self._alloc_cb, self._free_cb, None)
        ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            N.check(self.lib.fiesta_load_sectors(C.byref(ctx), progs, n, C.byref(alloc) if alloc else None,
                                                 C.c_void_p(self.stream.cuda_stream)))
        self.ctx = ctx

    # ------------------------------------------------------------------ integrate
    def integrate(self, n_iter=10, points=100_000, seed=1, rng="philox", precision="fp64", adapt=True,
                  alpha=1.5, skip_first=False, units=None, timeout_ms=0, threads=0, reset_grid=True,
                  iter_offset=0, assemble_result=True, raise_nonfinite=True, points_per_thread=0,
                  probe_points=0, fp32_budget=0.0, graph=True, small_x=0.0, unit_points=None, small_x32=0.0,
                  accumulate="auto"):
        lo = min(u.order for u in self.prep.units)
        hi = max(u.order + _n_orders(u) - 1 for u in self.prep.units)
        nord = hi - lo + 1
        b, e = (0, len(self.prep.units)) if units is None else units
        opt = N.Options(N.RNG[rng], N.PRECISION[precision], int(n_iter), int(adapt), int(points),
                        int(seed) & 0xFFFFFFFFFFFFFFFF, float(alpha), int(bool(skip_first)), lo, int(b), int(e),
                        int(timeout_ms), int(threads), int(bool(reset_grid)), int(iter_offset),
                        int(points_per_thread), int(probe_points), float(fp32_budget), int(not graph),
                        {"auto": 0, "registers": 1, "shared": 2}[accumulate],
                        float(small_x), None, float(small_x32))
        if unit_points is not None:
            upts = np.ascontiguousarray(unit_points, dtype=np.int64)
            if upts.shape != (e - b,):
                raise ValueError("unit_points needs one entry per unit of the slice")
            opt.unit_points = upts.ctypes.data_as(C.POINTER(C.c_int64))
        val = (C.c_double * nord)()
        err = (C.c_double * nord)()
        per = (N.UnitResult * sum(u.n_out for u in self.prep.units[b:e]))()
        st = N.Stats()
        with self._torch.cuda.device(self.device):
            rc = self.lib.fiesta_integrate(self.ctx, C.byref(opt), val, err, nord, per, C.byref(st))
        if rc != N.FIESTA_OK and not (rc == -5 and not raise_nonfinite):
            N.check(rc)
        pu = [dict(value=r.value, sigma=r.sigma, chi2_dof=r.chi2_dof, n_points=r.n_points, order=r.order,
                   sector=r.sector, n_nonfinite=r.n_nonfinite, precision=("fp64", "fp32")[r.precision],
                   unit=r.unit, fp32_error=r.fp32_error, part=r.part) for r in per]
        if self.prep.complex:
            values, errors = _sum_parts([(d["order"], d["part"], d["value"], d["sigma"]) for d in pu])
        else:
            values = {lo + k: val[k] for k in range(nord)}
            errors = {lo + k: err[k] for k in range(nord)}
        stats = dict(gpu_ms=st.gpu_ms, eval_ms=st.eval_ms, points=st.points, points_per_s=st.points_per_s,
                     kernels_launched=st.kernels_launched, eval_launches=st.eval_launches,
                     units_fp32=st.units_fp32, unit_points=st.unit_points, threads=tuple(st.threads),
                     points_per_thread=tuple(st.points_per_thread), points_ext=st.points_ext)
        res = Result(values, errors, pu, stats)
        if assemble_result and units is None:
            res.assembled, res.assembled_errors = assemble(self.prep, values, errors)
        return res

    # ------------------------------------------------------------------ cubature
    def cuhre(self, rel_tol=1e-6, abs_tol=1e-12, max_passes=40, max_regions=1 << 22, units=None, timeout_ms=0,
              threads=0, assemble_result=True):
        """Deterministic adaptive cubature (Genz-Malik rule, region splitting in passes)
        of every unit: per-order values and errors (summed linearly: the region errors
        are bounds), per-result records (value, error, regions, points, converged) and,
        for the whole problem, the assembled series (linear error bound)."""
        lo = min(u.order for u in self.prep.units)
        hi = max(u.order + _n_orders(u) - 1 for u in self.prep.units)
        nord = hi - lo + 1
        b, e = (0, len(self.prep.units)) if units is None else units
        opt = N.CuhreOptions(float(rel_tol), float(abs_tol), int(max_passes), lo, int(max_regions), int(b), int(e),
                             int(timeout_ms), int(threads))
        val = (C.c_double * nord)()
        err = (C.c_double * nord)()
        per = (N.CuhreResult * sum(u.n_out for u in self.prep.units[b:e]))()
        st = N.Stats()
        with self._torch.cuda.device(self.device):
            N.check(self.lib.fiesta_cuhre(self.ctx, C.byref(opt), val, err, nord, per, C.byref(st)))
        pu = [dict(value=r.value, error=r.error, n_regions=r.n_regions, n_points=r.n_points, order=r.order,
                   sector=r.sector, unit=r.unit, part=r.part, converged=bool(r.converged), passes=r.passes)
              for r in per]
        if self.prep.complex:
            values, errors = {}, {}
            for d in pu:
                values.setdefault(d["order"], [0.0, 0.0])[d["part"]] += d["value"]
                errors.setdefault(d["order"], [0.0, 0.0])[d["part"]] += d["error"]
            values = {K: complex(*x) for K, x in values.items()}
            errors = {K: complex(*x) for K, x in errors.items()}
        else:
            values = {lo + k: val[k] for k in range(nord)}
            errors = {lo + k: err[k] for k in range(nord)}
        stats = dict(gpu_ms=st.gpu_ms, eval_ms=st.eval_ms, points=st.points, points_per_s=st.points_per_s,
                     kernels_launched=st.kernels_launched, eval_launches=st.eval_launches,
                     unit_points=st.unit_points)
        res = Result(values, errors, pu, stats)
        if assemble_result and units is None:
            res.assembled, res.assembled_errors = assemble(self.prep, values, errors, correlated=True)
        return res

    def cuhre_regions(self, unit, cap=1 << 20):
        """The regions of ``unit`` evaluated in the last pass of the last cuhre call:
        (center (n, m), half (n, m), value (n, n_out), error (n, n_out), axis (n,)), m = max(dim, 2)."""
        u = self.prep.units[unit]
        m = max(u.dim, 2)
        n = C.c_int64()
        with self._torch.cuda.device(self.device):
            N.check(self.lib.fiesta_cuhre_regions(self.ctx, int(unit), 0, None, None, None, None, None, C.byref(n)))
        k = min(n.value, cap)
        cen, half = np.zeros((k, m)), np.zeros((k, m))
        val, err = np.zeros((k, u.n_out)), np.zeros((k, u.n_out))
        ax = np.zeros(k, dtype=np.int32)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        with self._torch.cuda.device(self.device):
            N.check(self.lib.fiesta_cuhre_regions(self.ctx, int(unit), k, dp(cen), dp(half), dp(val), dp(err),
                                                  ax.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n)))
        return cen, half, val, err, ax

    # ------------------------------------------------------------------ per point
    def eval_batch(self, unit, x, precision="fp64"):
        """f at points x (n, dim): a torch CUDA tensor (result on the device) or a host array.
        A fused unit returns (n, n_out); a complex unit returns complex values, (n,) for
        one order or (n, n_out / 2) for several."""
        torch = self._torch
        u = self.prep.units[unit]
        nout = u.n_out
        shape = (x.shape[0],) if nout == 1 else (x.shape[0], nout)
        if isinstance(x, torch.Tensor) and x.is_cuda:
            x = x.to(torch.float64).contiguous()
            f = torch.empty(shape, dtype=torch.float64, device=x.device)
            with torch.cuda.device(self.device):
                N.check(self.lib.fiesta_eval_batch(self.ctx, int(unit), N.PRECISION[precision],
                                                   C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(f.data_ptr())))
            if u.cplx:
                f = torch.view_as_complex(f.view(x.shape[0], nout // 2, 2))
                return f[:, 0] if nout == 2 else f
            return f
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        f = np.empty(shape)
        with torch.cuda.device(self.device):
            N.check(self.lib.fiesta_eval_batch(self.ctx, int(unit), N.PRECISION[precision],
                                               x.ctypes.data_as(C.c_void_p), x.shape[0], f.ctypes.data_as(C.c_void_p)))
        if u.cplx:
            f = f[:, 0::2] + 1j * f[:, 1::2]
            return f[:, 0] if nout == 2 else f
        return f

    def precision_probe(self, n_points=16384, seed=1, units=None):
        """Per unit (err_mean, err_max) of binary32 against binary64 at the same points."""
        b, e = (0, len(self.prep.units)) if units is None else units
        m = np.empty(e - b)
        x = np.empty(e - b)
        N.check(self.lib.fiesta_precision_probe(self.ctx, b, e, int(n_points), int(seed),
                                                m.ctypes.data_as(C.POINTER(C.c_double)),
                                                x.ctypes.data_as(C.POINTER(C.c_double))))
        return m, x

    # ------------------------------------------------------------------ learned proposal
    def flow_init(self, seed=1, scale=0.05):
        """Per-unit flows: random hidden weights, zero output layer (identity map)."""
        N.check(self.lib.fiesta_flow_init(self.ctx, int(seed), float(scale)))

    def flow_params(self, unit):
        p = np.empty(N.FLOW_PARAMS, dtype=np.float32)
        N.check(self.lib.fiesta_flow_params(self.ctx, int(unit), p.ctypes.data_as(C.POINTER(C.c_float)), 0))
        return p

    def set_flow_params(self, unit, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        N.check(self.lib.fiesta_flow_params(self.ctx, int(unit), p.ctypes.data_as(C.POINTER(C.c_float)), 1))

    def flow_sample(self, points, seed=1, iteration=0, precision="fp32", keep=0, units=None):
        """One pass of flow importance sampling: mean of f/q and its variance, one entry
        per result of the units (n_out per unit, in unit order)."""
        b, e = (0, len(self.prep.units)) if units is None else units
        nrec = sum(u.n_out for u in self.prep.units[b:e])
        m = np.empty(nrec)
        v = np.empty(nrec)
        st = N.Stats()
        N.check(self.lib.fiesta_flow_sample(self.ctx, b, e, int(points), int(seed), int(iteration),
                                            N.PRECISION[precision], int(keep),
                                            m.ctypes.data_as(C.POINTER(C.c_double)),
                                            v.ctypes.data_as(C.POINTER(C.c_double)), C.byref(st)))
        return m, v, dict(gpu_ms=st.gpu_ms, points=st.points, kernels_launched=st.kernels_launched)

    def flow_train(self, steps, lr=1e-3, power=1, units=None):
        b, e = (0, len(self.prep.units)) if units is None else units
        loss = np.empty(e - b)
        st = N.Stats()
        N.check(self.lib.fiesta_flow_train(self.ctx, b, e, int(steps), float(lr), int(power),
                                           loss.ctypes.data_as(C.POINTER(C.c_double)), C.byref(st)))
        return loss, dict(gpu_ms=st.gpu_ms, kernels_launched=st.kernels_launched)

    def flow_check(self, unit, z, w, precision="fp64"):
        """Sampler outputs at given base points z and the training pass (log q, loss,
        gradient) at the sampled x with weights w; for parity checks."""
        z = np.ascontiguousarray(z, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        n, d = z.shape
        x = np.empty((n, d))
        lq = np.empty(n)
        f = np.empty(n)
        lqt = np.empty(n)
        loss = np.empty(1)
        g = np.empty(N.FLOW_PARAMS, dtype=np.float32)
        dp = C.POINTER(C.c_double)
        N.check(self.lib.fiesta_flow_check(self.ctx, int(unit), n, N.PRECISION[precision], z.ctypes.data_as(dp),
                                           x.ctypes.data_as(dp), lq.ctypes.data_as(dp), f.ctypes.data_as(dp),
                                           w.ctypes.data_as(dp), lqt.ctypes.data_as(dp), loss.ctypes.data_as(dp),
                                           g.ctypes.data_as(C.POINTER(C.c_float))))
        return dict(x=x, logq=lq, f=f, logq_train=lqt, loss=loss[0], grad=g)

    def iterations(self, unit, n_iter, out=0):
        m = (C.c_double * n_iter)()
        v = (C.c_double * n_iter)()
        N.check(self.lib.fiesta_iterations(self.ctx, int(unit), int(out), int(n_iter), m, v))
        return np.array(m[:]), np.array(v[:])

    def get_grid(self, unit):
        d = self.prep.units[unit].dim
        g = np.empty(d * (N.NBINS + 1))
        N.check(self.lib.fiesta_get_grid(self.ctx, int(unit), g.ctypes.data_as(C.POINTER(C.c_double))))
        return g.reshape(d, N.NBINS + 1)

    def set_grid(self, unit, grid):
        g = np.ascontiguousarray(grid, dtype=np.float64).ravel()
        N.check(self.lib.fiesta_set_grid(self.ctx, int(unit), g.ctypes.data_as(C.POINTER(C.c_double))))

    def refine(self, grids, hists, alpha=1.5):
        """Device refinement of grids (n, dim, NB+1) from histograms (n, dim, NB); returns new grids."""
        g = np.ascontiguousarray(grids, dtype=np.float64).copy()
        h = np.ascontiguousarray(hists, dtype=np.float64)
        n, dim = g.shape[0], g.shape[1]
        N.check(self.lib.fiesta_refine(self.ctx, dim, n, float(alpha), g.ctypes.data_as(C.POINTER(C.c_double)),
                                       h.ctypes.data_as(C.POINTER(C.c_double))))
        return g

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.fiesta_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


CHECKPOINT_MAGIC = b"FIESTACK"
CHECKPOINT_VERSION = 1


def save_checkpoint(path, integ, state):
    """Write the Vegas state (every unit's grid, the running weighted sums, the
    iteration count and the stream seed) to ``path``: magic, version, a JSON
    header and the float64 payload, protected by a CRC-32.  The paper's pool
    keeps per-integral partial results for restarts (``-continue``, Sec. 4.5)."""
    import json
    import struct
    import zlib
    grids = [integ.get_grid(k) for k in range(len(integ.prep.units))]
    header = json.dumps({"n_units": len(grids), "n_rec": len(state["sw"]), "dims": [g.shape[0] for g in grids],
                         "it": state["it"],
                         "seed": state["seed"], "precision": state["precision"], "rng": state["rng"],
                         "points": state["points"], "gpu_ms": state["gpu_ms"],
                         "points_done": state["points_done"]}).encode()
    payload = np.concatenate([g.ravel() for g in grids] + [state["sw"], state["swi"]]).astype("<f8").tobytes()
    body = struct.pack("<I", len(header)) + header + payload
    with open(path + ".tmp", "wb") as f:
        f.write(CHECKPOINT_MAGIC + struct.pack("<II", CHECKPOINT_VERSION, zlib.crc32(body)) + body)
    import os
    os.replace(path + ".tmp", path)


def load_checkpoint(path, integ=None):
    """Read a checkpoint written by save_checkpoint; verify it and, given an
    Integrator, restore its grids.  Raises ValueError on a damaged file."""
    import json
    import struct
    import zlib
    raw = open(path, "rb").read()
    if len(raw) < 16 or raw[:8] != CHECKPOINT_MAGIC:
        raise ValueError("not a checkpoint file")
    version, crc = struct.unpack("<II", raw[8:16])
    if version != CHECKPOINT_VERSION:
        raise ValueError(f"unsupported checkpoint version {version}")
    body = raw[16:]
    if zlib.crc32(body) != crc:
        raise ValueError("checkpoint checksum mismatch (file damaged or truncated)")
    (hl,) = struct.unpack("<I", body[:4])
    h = json.loads(body[4:4 + hl].decode())
    data = np.frombuffer(body[4 + hl:], dtype="<f8")
    n = h["n_units"]
    nr = h.get("n_rec", n)
    need = sum(d * (N.NBINS + 1) for d in h["dims"]) + 2 * nr
    if data.size != need:
        raise ValueError("checkpoint payload has the wrong size")
    grids = []
    off = 0
    for d in h["dims"]:
        grids.append(data[off:off + d * (N.NBINS + 1)].reshape(d, N.NBINS + 1))
        off += d * (N.NBINS + 1)
    sw = data[off:off + nr].copy()
    swi = data[off + nr:off + 2 * nr].copy()
    if integ is not None:
        if len(integ.prep.units) != n or any(u.dim != d for u, d in zip(integ.prep.units, h["dims"])):
            raise ValueError("checkpoint does not match these units")
        for k, g in enumerate(grids):
            integ.set_grid(k, g)
    state = dict(h, sw=sw, swi=swi, grids=grids)
    return state


def allocate_points(prep, sig, n_used, values, target, floor, points, lo_frac=0.01, hi_mult=64):
    """Points per unit for the next iterations: Neyman allocation for the assembled
    series.  Unit u's per-point standard deviation of its eps-order-K integral is
    s_uK = sigma_uK sqrt(points used so far); its share of the error of result order n
    is sum_K |c_(n-K)| s_uK / sqrt(N_u) (c the prefactor series); with
    B_u = max_n (sum_K |c_(n-K)| s_uK / tau_n)^2 and a cost per point w_u (program
    length + map), N_u proportional to sqrt(B_u / w_u) minimises the cost at a given
    error.  The total cost equals that of ``points`` per unit; each N_u is clamped to
    [lo_frac * points, hi_mult * points]."""
    q, coeffs = prep.prefactor
    R = assemble(prep, values, {K: 0.0 for K in values})[0]
    big = max(abs(v) for v in R.values())
    tau = {n: target * max(abs(R[n]), floor * big) for n in R}
    s = {}
    k = 0
    for ui, u in enumerate(prep.units):
        for o in range(u.n_out):
            K, part = _record_key(u, o)
            s.setdefault(ui, {}).setdefault(K, 0.0)
            s[ui][K] += (sig[k] ** 2) * n_used[ui]
            k += 1
    cost = np.array([len(u.program.code) + 4 * u.dim + 8 for u in prep.units], dtype=float)
    B = np.zeros(len(prep.units))
    for ui in range(len(prep.units)):
        for n, t in tau.items():
            acc = 0.0
            for K, s2 in s[ui].items():
                i = n - K + q
                if 0 <= i < len(coeffs):
                    acc += abs(float(coeffs[i])) * math.sqrt(s2)
            B[ui] = max(B[ui], (acc / t) ** 2)
    wgt = np.sqrt(np.maximum(B, 0.0) / cost)
    if not np.any(wgt > 0):
        return np.full(len(prep.units), int(points), dtype=np.int64)
    N = wgt * (points * cost.sum()) / float(np.sum(wgt * cost))
    N = np.clip(N, max(2, lo_frac * points), hi_mult * points)
    return np.maximum(N.astype(np.int64), 2)


def run_to_accuracy(integ, target=1e-4, points=1_000_000, iters_per_call=2, max_iters=200, seed=1,
                    precision="fp64", rng="philox", floor=1e-2, skip_first=1, checkpoint=None, resume=None,
                    stop_after=None, allocate=False, small_x=0.0, small_x32=0.0, max_gpu_s=None):
    """Vegas until every eps order of the assembled result has sigma <= target * max(|R|, floor * max|R|).

    Iterations are combined per unit with inverse-variance weights across calls
    (the first ``skip_first`` iterations, spent adapting the grid, are left out),
    units are summed per order with mean-square errors (Sec. 4.3 of the paper)
    and the prefactor series is multiplied in.  ``checkpoint`` writes the state
    after every call; ``resume`` continues from such a file with the same point
    streams (iteration numbers continue); ``stop_after`` ends after that many
    iterations (to emulate an interrupted job).  Returns a dict with the GPU
    seconds (the library's device time over all calls), the points, the
    iterations and the final values and errors.  ``allocate`` spends the points of
    every call after the first where the variance is (``allocate_points``) instead of
    evenly; the total points per iteration stay nu * points.  ``small_x`` /
    ``small_x32`` promote points near the boundary of binary64 / binary32 units one
    precision level (see fiesta_options).  ``max_gpu_s`` stops once that much device
    time is spent; ``ratio`` in the result is max over orders of error / target.
    """
    prep = integ.prep
    recs = [(k, o) for k, u in enumerate(prep.units) for o in range(u.n_out)]
    unit_pts = None
    n_used = np.zeros(len(prep.units))
    nu = len(recs)
    sw = np.zeros(nu)
    swi = np.zeros(nu)
    gpu_ms = 0.0
    points_done = 0
    it = 0
    res = None
    if resume is not None:
        st = load_checkpoint(resume, integ)
        sw, swi, it = st["sw"], st["swi"], st["it"]
        gpu_ms, points_done, seed = st["gpu_ms"], st["points_done"], st["seed"]
    while it < max_iters:
        r = integ.integrate(n_iter=iters_per_call, points=points, seed=seed, rng=rng, precision=precision,
                            adapt=2, reset_grid=(it == 0), iter_offset=it, assemble_result=False,
                            unit_points=unit_pts, small_x=small_x, small_x32=small_x32)
        gpu_ms += r.stats["gpu_ms"]
        points_done += r.stats["unit_points"]
        used_now = np.full(len(prep.units), float(points)) if unit_pts is None else unit_pts.astype(float)
        n_used += used_now * sum(1 for j in range(iters_per_call) if it + j >= skip_first)
        for k, (unit, o) in enumerate(recs):
            m, v = integ.iterations(unit, iters_per_call, o)
            for j in range(iters_per_call):
                if it + j < skip_first:
                    continue
                w = 1.0 / v[j] if v[j] > 0 else 1e300
                sw[k] += w
                swi[k] += w * m[j]
        it += iters_per_call
        if checkpoint is not None:
            save_checkpoint(checkpoint, integ, dict(it=it, seed=seed, precision=precision, rng=rng, points=points,
                                                    gpu_ms=gpu_ms, points_done=points_done, sw=sw, swi=swi))
        if it <= skip_first:
            continue
        val = swi / sw
        sig = np.sqrt(1.0 / sw)
        R, E, values = _assembled(prep, recs, val, sig)
        big = max(abs(v) for v in R.values())
        ratio = _worst_ratio(R, E, target, floor)
        ok = ratio <= 1.0
        res = dict(gpu_s=gpu_ms * 1e-3, points=points_done, iterations=it, values=R, errors=E, converged=ok,
                   unit_values=val.copy(), unit_sigmas=sig.copy(), ratio=ratio)
        if ok or (stop_after is not None and it >= stop_after) or (max_gpu_s and gpu_ms * 1e-3 >= max_gpu_s):
            break
        if allocate and np.all(n_used > 0):
            unit_pts = allocate_points(prep, sig, n_used, values, target, floor, points)
    return res


def _worst_ratio(R, E, target, floor):
    """max over eps orders n of |error_n| / (target * max(|R_n|, floor * max_k |R_k|))."""
    big = max(abs(v) for v in R.values())
    return max(abs(E[n]) / (target * max(abs(R[n]), floor * big)) for n in R)


def run_cuhre_to_accuracy(integ, target=1e-4, floor=1e-2, rel_tol=None, shrink=0.1, max_rounds=6, max_passes=60,
                          max_regions=1 << 22):
    """Adaptive cubature until every eps order of the assembled result has an error
    bound <= target * max(|R|, floor * max|R|) (the rule of run_to_accuracy with the
    cubature's linear error bound in place of sigma).  The per-unit relative
    tolerance starts at ``rel_tol`` (default: target) and shrinks by ``shrink``
    while the assembled bound misses the target (sector contributions can cancel);
    GPU seconds add up over all attempts."""
    tol = target if rel_tol is None else rel_tol
    gpu_ms, pts, res = 0.0, 0, None
    for k in range(max_rounds):
        r = integ.cuhre(rel_tol=tol, max_passes=max_passes, max_regions=max_regions)
        gpu_ms += r.stats["gpu_ms"]
        pts += r.stats["points"]
        R, E = r.assembled, r.assembled_errors
        big = max(abs(v) for v in R.values())
        ok = all(abs(E[n]) <= target * max(abs(R[n]), floor * big) for n in R)
        res = dict(gpu_s=gpu_ms * 1e-3, points=pts, rounds=k + 1, rel_tol=tol, values=R, errors=E, converged=ok,
                   regions=sum(d["n_regions"] for d in r.per_unit))
        if ok:
            break
        tol *= shrink
    return res


def run_to_accuracy_rqmc(integ, target=1e-4, points=1 << 18, replicates=8, adapt_iters=6, adapt_points=None,
                         max_rounds=12, seed=1, precision="fp64", floor=1e-2, max_points=1 << 24):
    """Randomised quasi-Monte Carlo on Vegas grids.  The grids are first adapted with
    ``adapt_iters`` Philox iterations; then each round integrates every unit with
    ``replicates`` independent digital shifts of a Sobol sequence of N points on the
    frozen grids (one iteration each, no adaptation).  The replicate means are
    independent unbiased estimates, so a unit's estimate is their average and its
    error their standard deviation over sqrt(replicates) (no variance formula for
    correlated points is needed).  N doubles every round (Sobol points come in powers
    of two) until every eps order meets the target (the rule of run_to_accuracy);
    rounds are combined with inverse-variance weights; the sequence stops growing at
    ``max_points`` per replicate.  Binary64 is the intended precision: binary32
    rounding near the boundary adds point-wise noise that the replicate spread does
    not average like the quadrature error.  Returns what run_to_accuracy returns, with
    ``rounds`` and ``points_per_replicate``."""
    prep = integ.prep
    recs = [(k, o) for k, u in enumerate(prep.units) for o in range(u.n_out)]
    gpu_ms, pts = 0.0, 0
    r = integ.integrate(n_iter=adapt_iters, points=adapt_points or points, seed=seed, rng="philox",
                        precision=precision, adapt=2, reset_grid=True, assemble_result=False)
    gpu_ms += r.stats["gpu_ms"]
    pts += r.stats["unit_points"]
    sw = np.zeros(len(recs))
    swi = np.zeros(len(recs))
    n = int(points)
    res = None
    for rnd in range(max_rounds):
        r = integ.integrate(n_iter=replicates, points=n, seed=seed + 1 + rnd, rng="sobol", precision=precision,
                            adapt=False, reset_grid=False, iter_offset=1000 + rnd * replicates,
                            assemble_result=False)
        gpu_ms += r.stats["gpu_ms"]
        pts += r.stats["unit_points"]
        for k, (unit, o) in enumerate(recs):
            m, _ = integ.iterations(unit, replicates, o)
            mu = float(np.mean(m))
            var = float(np.var(m, ddof=1)) / replicates if replicates > 1 else 0.0
            w = 1.0 / var if var > 0 else 1e300
            sw[k] += w
            swi[k] += w * mu
        val = swi / sw
        sig = np.sqrt(1.0 / sw)
        R, E, values = _assembled(prep, recs, val, sig)
        ratio = _worst_ratio(R, E, target, floor)
        ok = ratio <= 1.0
        res = dict(gpu_s=gpu_ms * 1e-3, points=pts, rounds=rnd + 1, points_per_replicate=n, values=R, errors=E,
                   converged=ok, unit_values=val.copy(), unit_sigmas=sig.copy(), ratio=ratio)
        if ok or 2 * n > max_points:
            break
        n *= 2
    return res


def run_flow(integ, target=1e-4, points=1_000_000, keep=4096, train_rounds=8, steps_per_round=20, lr=2e-3,
             power=1, max_rounds=200, seed=1, precision="fp32", floor=1e-2, skip_rounds=None, max_gpu_s=None):
    """Learned proposal: per unit, alternate flow sampling (an unbiased estimate each
    round) and training on the round's kept points; stop when every eps order meets
    the target (same rule as run_to_accuracy).  Rounds while training are combined
    too, with inverse-variance weights, except the first ``skip_rounds`` (default:
    half of the training rounds).  GPU seconds include the training."""
    prep = integ.prep
    recs = [(k, o) for k, u in enumerate(prep.units) for o in range(u.n_out)]
    integ.flow_init(seed=seed)
    skip = train_rounds // 2 if skip_rounds is None else skip_rounds
    sw = np.zeros(len(recs))
    swi = np.zeros(len(recs))
    gpu_ms = 0.0
    pts = 0
    res = None
    for r in range(max_rounds):
        m, v, st = integ.flow_sample(points, seed=seed, iteration=r, precision=precision,
                                     keep=keep if r < train_rounds else 0)
        gpu_ms += st["gpu_ms"]
        pts += st["points"]
        if r >= skip:
            w = np.where(v > 0, 1.0 / np.maximum(v, 1e-300), 1e300)
            sw += w
            swi += w * m
        if r < train_rounds:
            _, tst = integ.flow_train(steps_per_round, lr=lr, power=power)
            gpu_ms += tst["gpu_ms"]
        if r < skip:
            continue
        val = swi / sw
        sig = np.sqrt(1.0 / sw)
        R, E, values = _assembled(prep, recs, val, sig)
        ratio = _worst_ratio(R, E, target, floor)
        ok = ratio <= 1.0
        res = dict(gpu_s=gpu_ms * 1e-3, points=pts, rounds=r + 1, values=R, errors=E, converged=ok,
                   unit_values=val.copy(), unit_sigmas=sig.copy(), ratio=ratio)
        if (ok and r >= train_rounds) or (max_gpu_s and gpu_ms * 1e-3 >= max_gpu_s):
            break
    return res
