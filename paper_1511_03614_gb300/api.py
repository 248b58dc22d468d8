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


def assemble_records(prep, orders, parts, vals, sigs, linear=False, prefactor=True):
    """fiesta_assemble on per-result records: the per-order sums (errors in the
    mean-square norm, or added when ``linear``) and, with ``prefactor``, the eps series
    of ``prep``; complex values for problems with complex units.  Returns (values,
    errors) dicts keyed by eps order.  Marshalling only: the sums run in the library."""
    lib = N.load()
    if prefactor:
        out_orders = tuple(prep.out_orders)
        opts, keep = accuracy_options(prep, points=2)
    else:
        out_orders = tuple(range(min(orders), max(orders) + 1))
        opts, keep = accuracy_options(prep, points=2)
        one = np.ones(1)
        keep = (keep, one)
        opts.pre, opts.n_pre, opts.pre_q, opts.correlated = one.ctypes.data_as(C.POINTER(C.c_double)), 1, 0, 0
        opts.out_lo = out_orders[0]
    n = len(out_orders)
    o = np.ascontiguousarray(orders, dtype=np.int32)
    p = np.ascontiguousarray(parts, dtype=np.int32)
    v = np.ascontiguousarray(vals, dtype=np.float64)
    s = np.ascontiguousarray(sigs, dtype=np.float64)
    val, err, vim, eim = (np.zeros(n) for _ in range(4))
    dp = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
    ip = lambda x: x.ctypes.data_as(C.POINTER(C.c_int32))
    N.check(lib.fiesta_assemble(C.byref(opts), len(v), ip(o), ip(p), dp(v), dp(s), int(bool(linear)), n, dp(val),
                                dp(err), dp(vim), dp(eim), None))
    if prep.complex:
        return ({m: complex(val[i], vim[i]) for i, m in enumerate(out_orders)},
                {m: complex(err[i], eim[i]) for i, m in enumerate(out_orders)})
    return ({m: float(val[i]) for i, m in enumerate(out_orders)}, {m: float(err[i]) for i, m in enumerate(out_orders)})


# Binary32 and AUTO units evaluate points with a coordinate below 2^-20 in binary64: below
# it a coordinate's terms fall under half a binary32 ulp of the corner polynomials and the
# pole-subtraction differences f(t) - f(t|t_j = 0) would vanish instead of reaching their
# finite limit.
SMALL_X32_DEFAULT = 2.0 ** -20


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
                  probe_points=0, fp32_budget=0.0, graph=True, small_x=0.0, unit_points=None, small_x32=None,
                  accumulate="auto", proposal="vegas", flow_train_steps=0, flow_keep=0, flow_lr=0.0, flow_power=0,
                  wide_threads=0):
        lo = min(u.order for u in self.prep.units)
        hi = max(u.order + _n_orders(u) - 1 for u in self.prep.units)
        nord = hi - lo + 1
        b, e = (0, len(self.prep.units)) if units is None else units
        if small_x32 is None:
            small_x32 = SMALL_X32_DEFAULT if precision in ("fp32", "auto") else 0.0
        opt = N.Options(N.RNG[rng], N.PRECISION[precision], int(n_iter), int(adapt), int(points),
                        int(seed) & 0xFFFFFFFFFFFFFFFF, float(alpha), int(bool(skip_first)), lo, int(b), int(e),
                        int(timeout_ms), int(threads), int(bool(reset_grid)), int(iter_offset),
                        int(points_per_thread), int(probe_points), float(fp32_budget), int(not graph),
                        {"auto": 0, "registers": 1, "shared": 2}[accumulate],
                        float(small_x), None, float(small_x32), N.PROPOSAL[proposal], int(flow_train_steps),
                        int(flow_keep), float(flow_lr), int(flow_power), int(wide_threads))
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
        recs = ([d["order"] for d in pu], [d["part"] for d in pu], [d["value"] for d in pu], [d["sigma"] for d in pu])
        if self.prep.complex:
            values, errors = assemble_records(self.prep, *recs, prefactor=False)
        else:
            values = {lo + k: val[k] for k in range(nord)}
            errors = {lo + k: err[k] for k in range(nord)}
        stats = dict(gpu_ms=st.gpu_ms, eval_ms=st.eval_ms, points=st.points, points_per_s=st.points_per_s,
                     kernels_launched=st.kernels_launched, eval_launches=st.eval_launches,
                     units_fp32=st.units_fp32, unit_points=st.unit_points, threads=tuple(st.threads),
                     points_per_thread=tuple(st.points_per_thread), points_ext=st.points_ext,
                     wide_threads=tuple(st.wide_threads), wide_points_per_thread=tuple(st.wide_points_per_thread),
                     eval_groups=st.eval_groups)
        res = Result(values, errors, pu, stats)
        if assemble_result and units is None:
            res.assembled, res.assembled_errors = assemble_records(self.prep, *recs)
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
        recs = ([d["order"] for d in pu], [d["part"] for d in pu], [d["value"] for d in pu], [d["error"] for d in pu])
        if self.prep.complex:
            values, errors = assemble_records(self.prep, *recs, linear=True, prefactor=False)
        else:
            values = {lo + k: val[k] for k in range(nord)}
            errors = {lo + k: err[k] for k in range(nord)}
        stats = dict(gpu_ms=st.gpu_ms, eval_ms=st.eval_ms, points=st.points, points_per_s=st.points_per_s,
                     kernels_launched=st.kernels_launched, eval_launches=st.eval_launches,
                     unit_points=st.unit_points)
        res = Result(values, errors, pu, stats)
        if assemble_result and units is None:
            res.assembled, res.assembled_errors = assemble_records(self.prep, *recs, linear=True)
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


def _records(prep):
    """(unit, result) of every record, in the library's order (n_out per unit)."""
    return [(k, o) for k, u in enumerate(prep.units) for o in range(u.n_out)]


def accuracy_options(prep, method="vegas", proposal="vegas", target=1e-4, floor=1e-2, points=1_000_000,
                     precision="fp64", allocate=False, iters_per_call=2, max_iters=200, skip=1, max_calls=0, seed=1,
                     max_gpu_s=0.0, small_x=0.0, small_x32=None, replicates=8, adapt_iters=6, adapt_points=0,
                     max_points=1 << 22, train_rounds=8, steps_per_round=20, lr=2e-3, power=1, keep=4096,
                     rel_tol=0.0, shrink=0.1, max_passes=60, max_regions=1 << 22):
    """fiesta_accuracy_options for a Prepared problem (its prefactor series, its assembled
    orders, correlated errors for fused units) -- marshalling only."""
    q, coeffs = prep.prefactor
    pre = np.ascontiguousarray([float(c) for c in coeffs], dtype=np.float64)
    if small_x32 is None:
        small_x32 = SMALL_X32_DEFAULT if precision in ("fp32", "auto") else 0.0
    o = N.AccuracyOptions()
    o.method, o.proposal, o.precision = N.METHOD[method], N.PROPOSAL[proposal], N.PRECISION[precision]
    o.allocate, o.target, o.floor, o.points = int(bool(allocate)), float(target), float(floor), int(points)
    o.iters_per_call, o.max_iters, o.skip, o.max_calls = int(iters_per_call), int(max_iters), int(skip), int(max_calls)
    o.seed, o.max_gpu_s = int(seed) & 0xFFFFFFFFFFFFFFFF, float(max_gpu_s or 0.0)
    o.small_x, o.small_x32 = float(small_x), float(small_x32)
    o.pre, o.n_pre, o.pre_q = pre.ctypes.data_as(C.POINTER(C.c_double)), len(pre), int(q)
    o.correlated = int(any(_n_orders(u) > 1 for u in prep.units))
    o.out_lo = int(min(prep.out_orders))
    o.replicates, o.adapt_iters, o.adapt_points, o.max_points = (int(replicates), int(adapt_iters),
                                                                 int(adapt_points or 0), int(max_points))
    o.train_rounds, o.steps_per_round, o.lr, o.power, o.keep = (int(train_rounds), int(steps_per_round), float(lr),
                                                                 int(power), int(keep))
    o.rel_tol, o.shrink, o.max_passes, o.max_regions = float(rel_tol), float(shrink), int(max_passes), int(max_regions)
    return o, pre


def new_accuracy_state(prep):
    """Zeroed running sums for fiesta_integrate_to_accuracy (numpy arrays + the struct)."""
    nrec = sum(u.n_out for u in prep.units)
    n_orders = len(prep.out_orders)
    arrays = dict(sw=np.zeros(nrec), swi=np.zeros(nrec), n_used=np.zeros(len(prep.units)),
                  order_sw=np.zeros(2 * n_orders), order_swi=np.zeros(2 * n_orders))
    st = N.AccuracyState()
    for k, v in arrays.items():
        setattr(st, k, v.ctypes.data_as(C.POINTER(C.c_double)))
    return st, arrays


def integrate_to_accuracy(integ, state=None, **kw):
    """One call of fiesta_integrate_to_accuracy on ``integ``'s units; ``state`` (from
    new_accuracy_state, or None for a fresh start) continues across calls.  Returns the
    result dict (assembled values and errors per order, complex where the problem has
    complex units; per-record values and sigmas; device seconds, points, iterations,
    converged, ratio) and the state."""
    prep = integ.prep
    opts, keep_alive = accuracy_options(prep, **kw)
    st, arrays = state if state is not None else new_accuracy_state(prep)
    orders = tuple(prep.out_orders)
    n = len(orders)
    nrec = sum(u.n_out for u in prep.units)
    val, err, vim, eim = (np.zeros(n) for _ in range(4))
    uv, us = np.zeros(nrec), np.zeros(nrec)
    dp = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
    with integ._torch.cuda.device(integ.device):
        N.check(integ.lib.fiesta_integrate_to_accuracy(integ.ctx, C.byref(opts), C.byref(st), n, dp(val), dp(err),
                                                       dp(vim), dp(eim), dp(uv), dp(us)))
    if prep.complex:
        values = {m: complex(val[i], vim[i]) for i, m in enumerate(orders)}
        errors = {m: complex(err[i], eim[i]) for i, m in enumerate(orders)}
    else:
        values = {m: float(val[i]) for i, m in enumerate(orders)}
        errors = {m: float(err[i]) for i, m in enumerate(orders)}
    res = dict(gpu_s=st.gpu_ms * 1e-3, points=st.points, iterations=st.iterations, values=values, errors=errors,
               converged=bool(st.converged), ratio=st.ratio, unit_values=uv, unit_sigmas=us,
               points_per_replicate=st.points_per_replicate, rel_tol=st.rel_tol)
    return res, (st, arrays)


def run_to_accuracy(integ, target=1e-4, points=1_000_000, iters_per_call=2, max_iters=200, seed=1,
                    precision="fp64", floor=1e-2, skip_first=1, checkpoint=None, resume=None,
                    stop_after=None, allocate=False, small_x=0.0, small_x32=None, max_gpu_s=None):
    """Vegas until every eps order of the assembled result has sigma <= target * max(|R|,
    floor * max|R|): fiesta_integrate_to_accuracy with FIESTA_METHOD_VEGAS (iterations
    combined per result across calls, the first ``skip_first`` left out; ``allocate``:
    Neyman allocation of the points across units).  ``checkpoint`` writes the state
    after every call, ``resume`` continues from such a file with the same point streams,
    ``stop_after`` ends after that many iterations (an interrupted job): then the library
    is called one fiesta_integrate call at a time and the file is written in between."""
    kw = dict(method="vegas", target=target, floor=floor, points=points, precision=precision, allocate=allocate,
              iters_per_call=iters_per_call, max_iters=max_iters, skip=skip_first, seed=seed,
              max_gpu_s=max_gpu_s or 0.0, small_x=small_x, small_x32=small_x32)
    state = new_accuracy_state(integ.prep)
    if resume is not None:
        ck = load_checkpoint(resume, integ)
        st, arrays = state
        arrays["sw"][:], arrays["swi"][:] = ck["sw"], ck["swi"]
        st.iterations, st.gpu_ms, st.points = ck["it"], ck["gpu_ms"], ck["points_done"]
        kw["seed"] = ck["seed"]
    step = checkpoint is not None or stop_after is not None
    while True:
        res, state = integrate_to_accuracy(integ, state, max_calls=1 if step else 0, **kw)
        st, arrays = state
        if checkpoint is not None:
            save_checkpoint(checkpoint, integ, dict(it=st.iterations, seed=kw["seed"], precision=precision,
                                                    rng="philox", points=points, gpu_ms=st.gpu_ms,
                                                    points_done=st.points, sw=arrays["sw"], swi=arrays["swi"]))
        if (not step or res["converged"] or st.iterations >= max_iters or
                (stop_after is not None and st.iterations >= stop_after) or
                (max_gpu_s and st.gpu_ms * 1e-3 >= max_gpu_s)):
            return res


def run_cuhre_to_accuracy(integ, target=1e-4, floor=1e-2, rel_tol=None, shrink=0.1, max_rounds=6, max_passes=60,
                          max_regions=1 << 22):
    """Adaptive cubature until every eps order meets the target with its error bound
    (FIESTA_METHOD_CUHRE: the per-unit tolerance starts at ``rel_tol``, default the
    target, and shrinks by ``shrink`` after every attempt that misses)."""
    res, _ = integrate_to_accuracy(integ, method="cuhre", target=target, floor=floor, rel_tol=rel_tol or 0.0,
                                   shrink=shrink, max_iters=max_rounds, max_passes=max_passes,
                                   max_regions=max_regions, points=2)
    res["rounds"] = res["iterations"]
    return res


def run_to_accuracy_rqmc(integ, target=1e-4, points=1 << 18, replicates=8, adapt_iters=6, adapt_points=None,
                         max_rounds=12, seed=1, precision="fp64", floor=1e-2, max_points=1 << 24, max_gpu_s=None):
    """Randomised quasi-Monte Carlo on adapted Vegas grids (FIESTA_METHOD_RQMC):
    ``adapt_iters`` Philox iterations adapt the grids, then every round integrates each
    unit with ``replicates`` independent digital shifts of a Sobol sequence of N points
    (N = points, doubling per round up to ``max_points``); a result's round estimate is
    the replicate mean, its error their spread over sqrt(replicates); rounds are
    combined with inverse-variance weights.  Binary64 is the intended precision."""
    res, _ = integrate_to_accuracy(integ, method="rqmc", target=target, floor=floor, points=points,
                                   replicates=replicates, adapt_iters=adapt_iters, adapt_points=adapt_points or 0,
                                   max_iters=max_rounds, seed=seed, precision=precision, max_points=max_points,
                                   max_gpu_s=max_gpu_s or 0.0)
    res["rounds"] = res["iterations"]
    return res


def run_flow(integ, target=1e-4, points=1_000_000, keep=4096, train_rounds=8, steps_per_round=20, lr=2e-3,
             power=1, max_rounds=200, seed=1, precision="fp32", floor=1e-2, skip_rounds=None, max_gpu_s=None):
    """Learned proposal (FIESTA_METHOD_VEGAS with FIESTA_PROPOSAL_FLOW): per unit,
    alternate flow sampling (an unbiased estimate each round) and training on the round's
    kept points for the first ``train_rounds`` rounds; rounds from ``skip_rounds``
    (default: half of the training rounds) on are combined with inverse-variance
    weights; device time includes the training."""
    skip = train_rounds // 2 if skip_rounds is None else skip_rounds
    res, _ = integrate_to_accuracy(integ, method="vegas", proposal="flow", target=target, floor=floor, points=points,
                                   keep=keep, train_rounds=train_rounds, steps_per_round=steps_per_round, lr=lr,
                                   power=power, max_iters=max_rounds, seed=seed, precision=precision, skip=skip,
                                   max_gpu_s=max_gpu_s or 0.0)
    res["rounds"] = res["iterations"]
    return res


def allocate_points(prep, sig, n_used, values, target, floor, points):
    """fiesta_allocate_points: Neyman allocation of ``points`` per unit for the assembled
    series (per-result errors ``sig`` in the library's record order, points used so far
    per unit ``n_used``, assembled values ``values`` by eps order setting the targets).
    Marshalling only."""
    lib = N.load()
    opts, keep = accuracy_options(prep, target=target, floor=floor, points=points)
    recs = _records(prep)
    units = np.array([k for k, _ in recs], dtype=np.int64)
    orders = np.array([_record_key(prep.units[k], o)[0] for k, o in recs], dtype=np.int32)
    cost = np.array([len(u.program.code) + 4 * u.dim + 8 for u in prep.units], dtype=np.float64)
    out = tuple(prep.out_orders)
    re = np.array([complex(values.get(m, 0.0)).real for m in out])
    im = np.array([complex(values.get(m, 0.0)).imag for m in out])
    sig = np.ascontiguousarray(sig, dtype=np.float64)
    n_used = np.ascontiguousarray(n_used, dtype=np.float64)
    res = np.zeros(len(prep.units), dtype=np.int64)
    dp = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
    N.check(lib.fiesta_allocate_points(C.byref(opts), len(prep.units), dp(cost), len(recs),
                                       units.ctypes.data_as(C.POINTER(C.c_int64)),
                                       orders.ctypes.data_as(C.POINTER(C.c_int32)), dp(sig), dp(n_used), len(out),
                                       dp(re), dp(im), res.ctypes.data_as(C.POINTER(C.c_int64))))
    return res
