// cuhre.cuh -- deterministic adaptive cubature over the units' programs, the
// Cuhre alternative to Vegas among the integrators of Sec. 4.4; included at the
// end of fiesta.cu (same translation unit).
//
// Rule: Genz and Malik's degree-7 fully symmetric rule for an n-cube with the
// embedded degree-5 rule (J. Comput. Appl. Math. 6 (1980) 295):
//   I7 = V (w1 f(c) + w2 S2 + w3 S3 + w4 S4 + w5 S5),  I5 = V (v1 f(c) + v2 S2 + v3 S3 + v4 S4),
// S2/S3 the sums over c +- lam2/lam3 h_j e_j, S4 over c +- lam4 h_j e_j +- lam4 h_k e_k
// (j < k), S5 over the 2^n points c + lam5 (+-h_1, ..., +-h_n); region error |I7 - I5|;
// split axis: the largest fourth difference
//   |f(c + lam2 e_j) + f(c - lam2 e_j) - 2 f(c) - (lam2/lam3)^2 (f(c + lam3 e_j) + f(c - lam3 e_j) - 2 f(c))|
// summed over the unit's results.
//
// The subdivision runs in passes over every live region of every unit of the
// slice.  The live list is kept sorted by unit (children replace their parent in
// place order), so each unit owns one contiguous run of regions and every
// per-unit step is a fixed-order block reduction.  Per pass:
//   k_cuhre_eval    one block per batch of a unit's regions (about CU_ITEM_PTS rule
//                   points): one thread per (region, rule point) runs the program
//                   (micro-op form, as in k_eval) into a shared-memory buffer, then one warp per region
//                   forms I7, I5, |I7 - I5| per result and the split axis;
//   k_cuhre_decide  one block per unit: sums over its live regions, tolerances,
//                   convergence; regions within their volume's share of the
//                   tolerance are frozen (their sums added to the unit's frozen
//                   totals), the others flagged for splitting;
//   k_cuhre_split   one block per unit: block scan of the flags, children written
//                   to the next live list.
// The host reads the per-unit split counts once per pass to size the next list and
// uploads two prefix tables of nu + 1 entries (regions and blocks per unit).

namespace {

constexpr int CU_STRIDE = FIESTA_MAX_DIM;          // doubles per region centre / half-width
constexpr int CU_ITEM_PTS = 512;                   // rule points per block (a batch of whole regions)

struct CuRule {
    double w[5];     // degree-7 weights, volume-1 region
    double v[4];     // degree-5 weights
};

struct CuConsts {
    double lam2, lam3, lam4, lam5, ratio;
    CuRule rule[CU_STRIDE + 1];      // by n = 2..8
};

__host__ __device__ inline int cu_n(int dim) { return dim < 2 ? 2 : dim; }
__host__ __device__ inline int cu_points(int n) { return 1 + 4 * n + 2 * n * (n - 1) + (1 << n); }

CuConsts cu_consts() {
    CuConsts K{};
    K.lam2 = std::sqrt(9.0 / 70.0);
    K.lam3 = std::sqrt(9.0 / 10.0);
    K.lam4 = std::sqrt(9.0 / 10.0);
    K.lam5 = std::sqrt(9.0 / 19.0);
    const double q = K.lam2 / K.lam3;
    K.ratio = q * q;
    for (int n = 2; n <= CU_STRIDE; ++n) {
        const double d = n;
        CuRule &R = K.rule[n];
        R.w[0] = (12824.0 - 9120.0 * d + 400.0 * d * d) / 19683.0;
        R.w[1] = 980.0 / 6561.0;
        R.w[2] = (1820.0 - 400.0 * d) / 19683.0;
        R.w[3] = 200.0 / 19683.0;
        R.w[4] = 6859.0 / 19683.0 / std::ldexp(1.0, n);
        R.v[0] = (729.0 - 950.0 * d + 50.0 * d * d) / 729.0;
        R.v[1] = 245.0 / 486.0;
        R.v[2] = (265.0 - 100.0 * d) / 1458.0;
        R.v[3] = 25.0 / 729.0;
    }
    return K;
}

// Coordinate j (on [-1, 1]) of rule point p of an n-cube.  Order: the centre;
// +lam2 e_0, -lam2 e_0, +lam2 e_1, ...; the same for lam3; for each pair j < k in
// lexicographic order the four sign pairs (++, +-, -+, --) of lam4; the 2^n lam5
// points with coordinate 0 the most significant sign bit (bit set: minus).
__device__ __forceinline__ double cu_gen(int p, int j, int n, const CuConsts &K) {
    if (p == 0) return 0.0;
    int t = p - 1;
    if (t < 2 * n) return (t >> 1) == j ? ((t & 1) ? -K.lam2 : K.lam2) : 0.0;
    t -= 2 * n;
    if (t < 2 * n) return (t >> 1) == j ? ((t & 1) ? -K.lam3 : K.lam3) : 0.0;
    t -= 2 * n;
    const int n4 = 2 * n * (n - 1);
    if (t < n4) {
        int m = t >> 2, a = 0;
        while (m >= n - 1 - a) {
            m -= n - 1 - a;
            ++a;
        }
        const int b = a + 1 + m;
        if (j == a) return (t & 2) ? -K.lam4 : K.lam4;
        if (j == b) return (t & 1) ? -K.lam4 : K.lam4;
        return 0.0;
    }
    t -= n4;
    return ((t >> (n - 1 - j)) & 1) ? -K.lam5 : K.lam5;
}

// the program in its micro-op form (uops.cuh): shared memory viewed as binary64 holds the
// constants (then -0, 1, -1) below the per-thread region of coordinates and slot file
struct CuSmem {
    size_t uops, cons, logtab, x, slots, f, total;
};

__host__ __device__ inline CuSmem cu_smem(int max_instr, int max_const, int max_slots, int threads) {
    CuSmem L;
    size_t off = 0;
    L.uops = off; off = align16(off + sizeof(uint64_t) * (max_instr + 1));
    L.cons = off; off = align16(off + sizeof(double) * (max_const + 3));
    L.logtab = off; off = align16(off + sizeof(double) * LOGTAB_DOUBLES);
    L.x = off; off = align16(off + sizeof(double) * MAXD * threads);
    L.slots = off; off = align16(off + sizeof(double) * max_slots * threads);
    L.f = off; off = align16(off + sizeof(double) * CU_ITEM_PTS * MAXO);
    L.total = off;
    return L;
}

// Regions per block for rule points P: whole regions, about CU_ITEM_PTS points.
__host__ __device__ inline int cu_batch(int P) { return P >= CU_ITEM_PTS ? 1 : CU_ITEM_PTS / P; }

__global__ void k_cuhre_init(int64_t nu, double *rc, double *rh, int32_t *runit) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nu * CU_STRIDE) return;
    rc[i] = 0.5;
    rh[i] = 0.5;
    if (i % CU_STRIDE == 0) runit[i / CU_STRIDE] = static_cast<int32_t>(i / CU_STRIDE);
}

// Block = item: a batch of consecutive regions of one unit (item_off: first item of
// each unit position, reg_off: its first live region).
__global__ void __launch_bounds__(256) k_cuhre_eval(const DevUnit *__restrict__ units, int64_t unit_begin,
                                                    const uint64_t *__restrict__ pre,
                                                    const double *__restrict__ cons64,
                                                    const double *__restrict__ logtab,
                                                    const int64_t *__restrict__ item_off,
                                                    const int64_t *__restrict__ reg_off, int64_t n_pos,
                                                    const double *__restrict__ rc, const double *__restrict__ rh,
                                                    double *__restrict__ rval, double *__restrict__ rerr,
                                                    int32_t *__restrict__ raxis, CuConsts K, int max_instr,
                                                    int max_const, int max_slots) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t item = blockIdx.x;
    int64_t lo = 0, hi = n_pos;                       // item_off[lo] <= item < item_off[lo + 1]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (item_off[mid] <= item) lo = mid;
        else hi = mid;
    }
    const int64_t up = lo;
    const DevUnit u = units[unit_begin + up];
    const int nt = blockDim.x, tid = threadIdx.x;
    const CuSmem L = cu_smem(max_instr, max_const, max_slots, nt);
    uint64_t *s_uops = reinterpret_cast<uint64_t *>(smem + L.uops);
    double *s_cons = reinterpret_cast<double *>(smem + L.cons);
    double *s_logtab = reinterpret_cast<double *>(smem + L.logtab);
    double *s_x = reinterpret_cast<double *>(smem + L.x);
    double *s_slots = reinterpret_cast<double *>(smem + L.slots);
    double *s_f = reinterpret_cast<double *>(smem + L.f);
    const int cons_base = static_cast<int>(L.cons / sizeof(double)), k_zero = cons_base + max_const;
    const int pt = static_cast<int>(L.x / sizeof(double)), slot_base = static_cast<int>(L.slots / sizeof(double));
    for (int i = tid; i < LOGTAB_DOUBLES; i += nt) s_logtab[i] = logtab[i];
    for (int i = tid; i < u.n_uop; i += nt) s_uops[i] = uop_from_pre(pre[u.uop_off + i], cons_base, k_zero, pt, slot_base, nt);
    for (int i = tid; i < u.n_const; i += nt) s_cons[i] = cons64[u.const_off + i];
    if (tid == 0) {
        s_uops[u.n_uop] = 0ull;                          // fetched after the last word, never executed
        s_cons[max_const] = -0.0;
        s_cons[max_const + 1] = 1.0;
        s_cons[max_const + 2] = -1.0;
    }
    __syncthreads();
    const int n = cu_n(u.dim), P = cu_points(n), no = u.n_out;
    const int64_t r0 = reg_off[up] + (item - item_off[up]) * cu_batch(P);
    const int nr = static_cast<int>(min(static_cast<int64_t>(cu_batch(P)), reg_off[up + 1] - r0));
    const int npts = nr * P;
    for (int q = tid; q < npts; q += nt) {
        const int64_t r = r0 + q / P;
        const int p = q % P;
        const double *c = rc + r * CU_STRIDE;
        const double *h = rh + r * CU_STRIDE;
        for (int j = 0; j < u.dim; ++j) s_x[j * nt + tid] = __dadd_rn(c[j], __dmul_rn(cu_gen(p, j, n, K), h[j]));
        interpret_uop<double>(s_uops, u.n_uop, reinterpret_cast<double *>(smem), pt, tid, s_logtab);
        for (int o = 0; o < no; ++o) s_f[q * no + o] = s_slots[tid + u.outs[o] * nt];
    }
    __syncthreads();
    const int lane = tid & 31, nw = nt >> 5;
    const CuRule &W = K.rule[n];
    const int e1 = 2 * n, e2 = 4 * n, e3 = 4 * n + 2 * n * (n - 1);
    for (int rr = tid >> 5; rr < nr; rr += nw) {
        const int64_t r = r0 + rr;
        const double *f = s_f + rr * P * no;
        const double *h = rh + r * CU_STRIDE;
        double a7[MAXO], a5[MAXO];
#pragma unroll
        for (int o = 0; o < MAXO; ++o) a7[o] = a5[o] = 0.0;
        for (int p = lane; p < P; p += 32) {
            double w7, w5;
            if (p == 0) { w7 = W.w[0]; w5 = W.v[0]; }
            else if (p <= e1) { w7 = W.w[1]; w5 = W.v[1]; }
            else if (p <= e2) { w7 = W.w[2]; w5 = W.v[2]; }
            else if (p <= e3) { w7 = W.w[3]; w5 = W.v[3]; }
            else { w7 = W.w[4]; w5 = 0.0; }
#pragma unroll
            for (int o = 0; o < MAXO; ++o)
                if (o < no) {
                    const double y = f[p * no + o];
                    a7[o] = fma(w7, y, a7[o]);
                    a5[o] = fma(w5, y, a5[o]);
                }
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1)
#pragma unroll
            for (int o = 0; o < MAXO; ++o)
                if (o < no) {
                    a7[o] += __shfl_xor_sync(0xffffffffu, a7[o], s);
                    a5[o] += __shfl_xor_sync(0xffffffffu, a5[o], s);
                }
        // fourth differences: lane j < n for coordinate j
        double D = -1.0, hj = 0.0;
        int jj = lane;
        if (lane < n) {
            D = 0.0;
            hj = h[lane];
            for (int o = 0; o < no; ++o) {
                const double f0 = f[o];
                const double y2p = f[(1 + 2 * lane) * no + o];
                const double y2m = f[(2 + 2 * lane) * no + o];
                const double y3p = f[(1 + e1 + 2 * lane) * no + o];
                const double y3m = f[(2 + e1 + 2 * lane) * no + o];
                const double t2 = __dsub_rn(__dadd_rn(y2p, y2m), __dmul_rn(2.0, f0));
                const double t3 = __dsub_rn(__dadd_rn(y3p, y3m), __dmul_rn(2.0, f0));
                D = __dadd_rn(D, fabs(__dsub_rn(t2, __dmul_rn(K.ratio, t3))));
            }
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            const double D2 = __shfl_xor_sync(0xffffffffu, D, s);
            const double h2 = __shfl_xor_sync(0xffffffffu, hj, s);
            const int j2 = __shfl_xor_sync(0xffffffffu, jj, s);
            if (D2 > D || (D2 == D && (h2 > hj || (h2 == hj && j2 < jj)))) {
                D = D2;
                hj = h2;
                jj = j2;
            }
        }
        if (lane == 0) {
            double V = 1.0;
            for (int j = 0; j < n; ++j) V *= 2.0 * h[j];
            for (int o = 0; o < no; ++o) {
                const double i7 = V * a7[o], i5 = V * a5[o];
                rval[r * MAXO + o] = i7;
                rerr[r * MAXO + o] = fabs(i7 - i5);
            }
            raxis[r] = jj;
        }
    }
}

// Fixed-order sum over the block of (a[0..MAXO), b[0..MAXO), c); the totals land
// in red[0..2*MAXO] and are visible to every thread after the call.
__device__ __forceinline__ void cu_block_sum(double (&a)[MAXO], double (&b)[MAXO], double &c, double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
#pragma unroll
        for (int o = 0; o < MAXO; ++o) {
            a[o] += __shfl_xor_sync(0xffffffffu, a[o], s);
            b[o] += __shfl_xor_sync(0xffffffffu, b[o], s);
        }
        c += __shfl_xor_sync(0xffffffffu, c, s);
    }
    constexpr int W = 2 * MAXO + 1;
    if (lane == 0) {
#pragma unroll
        for (int o = 0; o < MAXO; ++o) {
            red[W + wid * W + o] = a[o];
            red[W + wid * W + MAXO + o] = b[o];
        }
        red[W + wid * W + 2 * MAXO] = c;
    }
    __syncthreads();
    if (threadIdx.x < W) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[W + w * W + threadIdx.x];
        red[threadIdx.x] = s;
    }
    __syncthreads();
}

struct CuDecideArgs {
    const DevUnit *units;
    int64_t unit_begin;
    const int64_t *reg_off;       // [nu + 1]
    const double *rh, *rval, *rerr;
    uint8_t *rflag;
    const double *frz_v, *frz_e;  // committed frozen totals [nu * MAXO]
    double *tot_v, *tot_e;        // out: frozen + live [nu * MAXO]
    double *fp_v, *fp_e;          // out: sums of the regions frozen in this pass
    int64_t *nsplit;              // out
    int32_t *conv;                // out
    int32_t *bad;                 // out: non-finite total seen
    double rel_tol, abs_tol;
    int final_pass;
};

__global__ void __launch_bounds__(256) k_cuhre_decide(CuDecideArgs A) {
    __shared__ double red[(2 * MAXO + 1) * 9];
    __shared__ double s_tau[MAXO];
    const int64_t up = blockIdx.x;
    const int64_t a = A.reg_off[up], b = A.reg_off[up + 1];
    if (a == b) return;
    const DevUnit u = A.units[A.unit_begin + up];
    const int no = u.n_out, n = cu_n(u.dim);
    double lv[MAXO], le[MAXO], cnt = 0.0;
#pragma unroll
    for (int o = 0; o < MAXO; ++o) lv[o] = le[o] = 0.0;
    for (int64_t r = a + threadIdx.x; r < b; r += blockDim.x)
#pragma unroll
        for (int o = 0; o < MAXO; ++o)
            if (o < no) {
                lv[o] += A.rval[r * MAXO + o];
                le[o] += A.rerr[r * MAXO + o];
            }
    cu_block_sum(lv, le, cnt, red);
    if (threadIdx.x == 0) {
        double tv[MAXO], te[MAXO];
        bool conv = true, finite = true;
        for (int o = 0; o < no; ++o) {
            tv[o] = A.frz_v[up * MAXO + o] + red[o];
            te[o] = A.frz_e[up * MAXO + o] + red[MAXO + o];
            finite = finite && isfinite(tv[o]) && isfinite(te[o]);
        }
        for (int o = 0; o < no; ++o) {
            const double s = u.cplx ? hypot(tv[o & ~1], tv[o | 1]) : fabs(tv[o]);
            const double tau = fmax(A.abs_tol, A.rel_tol * s);
            s_tau[o] = tau;
            conv = conv && te[o] <= tau;
            A.tot_v[up * MAXO + o] = tv[o];
            A.tot_e[up * MAXO + o] = te[o];
        }
        if (!finite) *A.bad = 1;
        A.conv[up] = conv ? 1 : 0;
        if (conv)
            for (int o = 0; o < no; ++o) s_tau[o] = INFINITY;
    }
    __syncthreads();
    if (A.final_pass) return;
    double fv[MAXO], fe[MAXO], ns = 0.0;
#pragma unroll
    for (int o = 0; o < MAXO; ++o) fv[o] = fe[o] = 0.0;
    for (int64_t r = a + threadIdx.x; r < b; r += blockDim.x) {
        const double *h = A.rh + r * CU_STRIDE;
        double V = 1.0;
        for (int j = 0; j < n; ++j) V *= 2.0 * h[j];
        bool split = false;
        for (int o = 0; o < no; ++o) split = split || A.rerr[r * MAXO + o] > s_tau[o] * V;
        A.rflag[r] = split ? 1 : 0;
        if (split) {
            ns += 1.0;
        } else {
#pragma unroll
            for (int o = 0; o < MAXO; ++o)
                if (o < no) {
                    fv[o] += A.rval[r * MAXO + o];
                    fe[o] += A.rerr[r * MAXO + o];
                }
        }
    }
    cu_block_sum(fv, fe, ns, red);
    if (threadIdx.x == 0) {
        for (int o = 0; o < MAXO; ++o) {
            A.fp_v[up * MAXO + o] = o < no ? red[o] : 0.0;
            A.fp_e[up * MAXO + o] = o < no ? red[MAXO + o] : 0.0;
        }
        A.nsplit[up] = static_cast<int64_t>(red[2 * MAXO]);
    }
}

struct CuSplitArgs {
    const int64_t *reg_off, *new_off;   // [nu + 1]
    const uint8_t *rflag;
    const int32_t *raxis;
    const double *rc, *rh;
    double *nc, *nh;
    int32_t *nunit;
    double *frz_v, *frz_e;
    const double *fp_v, *fp_e;
};

__global__ void __launch_bounds__(256) k_cuhre_split(CuSplitArgs A) {
    __shared__ int s_w[8];
    const int up = blockIdx.x;
    const int64_t a = A.reg_off[up], b = A.reg_off[up + 1];
    if (a == b) return;
    if (threadIdx.x < MAXO) {
        A.frz_v[up * MAXO + threadIdx.x] += A.fp_v[up * MAXO + threadIdx.x];
        A.frz_e[up * MAXO + threadIdx.x] += A.fp_e[up * MAXO + threadIdx.x];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t base = A.new_off[up];
    int64_t running = 0;
    for (int64_t t0 = a; t0 < b; t0 += blockDim.x) {
        const int64_t r = t0 + threadIdx.x;
        const bool f = r < b && A.rflag[r];
        const unsigned ballot = __ballot_sync(0xffffffffu, f);
        if (lane == 0) s_w[wid] = __popc(ballot);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) before += s_w[w];
            total += s_w[w];
        }
        if (f) {
            const int64_t k = base + 2 * (running + before + __popc(ballot & ((1u << lane) - 1u)));
            const int ax = A.raxis[r];
            for (int j = 0; j < CU_STRIDE; ++j) {
                const double c = A.rc[r * CU_STRIDE + j], h = A.rh[r * CU_STRIDE + j];
                A.nc[k * CU_STRIDE + j] = c;
                A.nc[(k + 1) * CU_STRIDE + j] = c;
                A.nh[k * CU_STRIDE + j] = h;
                A.nh[(k + 1) * CU_STRIDE + j] = h;
            }
            const double hh = A.rh[r * CU_STRIDE + ax] * 0.5;
            const double c = A.rc[r * CU_STRIDE + ax];
            A.nh[k * CU_STRIDE + ax] = hh;
            A.nh[(k + 1) * CU_STRIDE + ax] = hh;
            A.nc[k * CU_STRIDE + ax] = c - hh;
            A.nc[(k + 1) * CU_STRIDE + ax] = c + hh;
            A.nunit[k] = up;
            A.nunit[k + 1] = up;
        }
        running += total;
        __syncthreads();
    }
}

}  // namespace

struct CuhreState {
    // live lists (double-buffered): centres, half-widths, unit positions
    double *rc[2] = {nullptr, nullptr}, *rh[2] = {nullptr, nullptr};
    int32_t *runit[2] = {nullptr, nullptr};
    int64_t list_cap[2] = {0, 0};
    int cur = 0;
    // per live region of the current pass
    double *rval = nullptr, *rerr = nullptr;
    int32_t *raxis = nullptr;
    uint8_t *rflag = nullptr;
    int64_t reg_cap = 0;
    // per unit of the slice
    int64_t *reg_off = nullptr, *new_off = nullptr, *item_off = nullptr, *nsplit = nullptr;
    double *frz_v = nullptr, *frz_e = nullptr, *tot_v = nullptr, *tot_e = nullptr, *fp_v = nullptr, *fp_e = nullptr;
    int32_t *conv = nullptr, *bad = nullptr;
    int64_t unit_cap = 0;
    // the last call: slice and the live list of its last pass
    int64_t last_begin = 0, last_n = 0;
    std::vector<int64_t> last_off;
    bool have_last = false;
};

void cuhre_state_delete(CuhreState *s) { delete s; }   // device arrays belong to the context

namespace {

int cu_grow_list(fiesta_ctx *c, CuhreState &S, int which, int64_t need) {
    if (need <= S.list_cap[which] && S.rc[which]) return FIESTA_OK;
    const int64_t n = std::max<int64_t>({need, S.list_cap[which] * 2, 64});
    c->dfree(S.rc[which]);
    c->dfree(S.rh[which]);
    c->dfree(S.runit[which]);
    S.rc[which] = static_cast<double *>(c->dmalloc(sizeof(double) * CU_STRIDE * n));
    S.rh[which] = static_cast<double *>(c->dmalloc(sizeof(double) * CU_STRIDE * n));
    S.runit[which] = static_cast<int32_t *>(c->dmalloc(sizeof(int32_t) * n));
    if (!S.rc[which] || !S.rh[which] || !S.runit[which]) {
        S.list_cap[which] = 0;
        return fail(FIESTA_E_NOMEM, "fiesta_cuhre: device allocation failed");
    }
    S.list_cap[which] = n;
    return FIESTA_OK;
}

int cu_grow_regions(fiesta_ctx *c, CuhreState &S, int64_t need) {
    if (need <= S.reg_cap && S.rval) return FIESTA_OK;
    const int64_t n = std::max<int64_t>({need, S.reg_cap * 2, 64});
    c->dfree(S.rval);
    c->dfree(S.rerr);
    c->dfree(S.raxis);
    c->dfree(S.rflag);
    S.rval = static_cast<double *>(c->dmalloc(sizeof(double) * MAXO * n));
    S.rerr = static_cast<double *>(c->dmalloc(sizeof(double) * MAXO * n));
    S.raxis = static_cast<int32_t *>(c->dmalloc(sizeof(int32_t) * n));
    S.rflag = static_cast<uint8_t *>(c->dmalloc(n));
    if (!S.rval || !S.rerr || !S.raxis || !S.rflag) {
        S.reg_cap = 0;
        return fail(FIESTA_E_NOMEM, "fiesta_cuhre: device allocation failed");
    }
    S.reg_cap = n;
    return FIESTA_OK;
}

int cu_grow_units(fiesta_ctx *c, CuhreState &S, int64_t nu) {
    if (nu <= S.unit_cap && S.reg_off) return FIESTA_OK;
    void **ptrs[] = {(void **)&S.reg_off, (void **)&S.new_off, (void **)&S.item_off,
                     (void **)&S.nsplit, (void **)&S.frz_v, (void **)&S.frz_e, (void **)&S.tot_v,
                     (void **)&S.tot_e, (void **)&S.fp_v, (void **)&S.fp_e, (void **)&S.conv, (void **)&S.bad};
    for (void **p : ptrs) {
        c->dfree(*p);
        *p = nullptr;
    }
    const int64_t n = nu + 1;
    S.reg_off = static_cast<int64_t *>(c->dmalloc(sizeof(int64_t) * n));
    S.new_off = static_cast<int64_t *>(c->dmalloc(sizeof(int64_t) * n));
    S.item_off = static_cast<int64_t *>(c->dmalloc(sizeof(int64_t) * n));
    S.nsplit = static_cast<int64_t *>(c->dmalloc(sizeof(int64_t) * n));
    S.frz_v = static_cast<double *>(c->dmalloc(sizeof(double) * MAXO * n));
    S.frz_e = static_cast<double *>(c->dmalloc(sizeof(double) * MAXO * n));
    S.tot_v = static_cast<double *>(c->dmalloc(sizeof(double) * MAXO * n));
    S.tot_e = static_cast<double *>(c->dmalloc(sizeof(double) * MAXO * n));
    S.fp_v = static_cast<double *>(c->dmalloc(sizeof(double) * MAXO * n));
    S.fp_e = static_cast<double *>(c->dmalloc(sizeof(double) * MAXO * n));
    S.conv = static_cast<int32_t *>(c->dmalloc(sizeof(int32_t) * n));
    S.bad = static_cast<int32_t *>(c->dmalloc(sizeof(int32_t) * 4));
    for (void **p : ptrs)
        if (!*p) {
            S.unit_cap = 0;
            return fail(FIESTA_E_NOMEM, "fiesta_cuhre: device allocation failed");
        }
    S.unit_cap = nu;
    return FIESTA_OK;
}

}  // namespace

extern "C" {

int fiesta_cuhre(fiesta_ctx *c, const fiesta_cuhre_options *opt, double *value, double *error, int32_t n_orders,
                 fiesta_cuhre_result *per, fiesta_stats *stats) {
    if (!c || !opt || n_orders < 0 || (n_orders > 0 && (!value || !error)))
        return fail(FIESTA_E_INVALID, "fiesta_cuhre: bad arguments");
    const int64_t total = static_cast<int64_t>(c->units.size());
    const int64_t b = opt->unit_begin, e = opt->unit_end <= 0 ? total : opt->unit_end;
    if (b < 0 || e > total || b >= e) return fail(FIESTA_E_INVALID, "fiesta_cuhre: bad unit range");
    if (!(opt->rel_tol >= 0.0) || !(opt->abs_tol >= 0.0) || (opt->rel_tol == 0.0 && opt->abs_tol == 0.0))
        return fail(FIESTA_E_INVALID, "fiesta_cuhre: tolerances must be >= 0 and not both 0");
    const int threads = opt->threads ? opt->threads : 128;
    if (threads < 32 || threads > 256 || threads % 32) return fail(FIESTA_E_INVALID, "fiesta_cuhre: threads must be 32..256, a multiple of 32");
    if (opt->max_passes < 0 || opt->max_regions < 0) return fail(FIESTA_E_INVALID, "fiesta_cuhre: negative limit");
    const int max_passes = opt->max_passes ? opt->max_passes : 40;
    const int64_t max_regions = opt->max_regions ? opt->max_regions : (int64_t(1) << 22);
    const int64_t nu = e - b;
    if (nu > max_regions) return fail(FIESTA_E_INVALID, "fiesta_cuhre: max_regions is below the number of units");
    if (!c->cuhre) c->cuhre = new CuhreState();
    CuhreState &S = *c->cuhre;
    S.have_last = false;
    cudaStream_t st = c->stream;
    const SliceInfo si = slice_info(c, b, e);
    const CuConsts K = cu_consts();
    const CuSmem L = cu_smem(si.max_instr, si.max_const, si.max_slots, threads);
    if (cudaFuncSetAttribute(k_cuhre_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total) != cudaSuccess)
        return fail(FIESTA_E_NOMEM, "fiesta_cuhre: shared memory for these programs exceeds the device limit");
    int rc = cu_grow_units(c, S, nu);
    if (!rc) rc = cu_grow_list(c, S, 0, nu);
    if (!rc) rc = cu_grow_list(c, S, 1, nu);
    if (rc) return rc;
    S.cur = 0;
    std::vector<int> P(nu), NO(nu);
    for (int64_t k = 0; k < nu; ++k) {
        P[k] = cu_points(cu_n(c->units[b + k].dim));
        NO[k] = c->units[b + k].n_out;
    }
    std::vector<int64_t> nreg(nu, 1), off(nu + 1), nfrozen(nu, 0), npts(nu, 0), nsp(nu);
    std::vector<int32_t> passes_u(nu, 0), conv(nu, 0), hconv(nu);
    std::vector<double> htv(nu * MAXO, 0.0), hte(nu * MAXO, 0.0), tv(nu * MAXO), te(nu * MAXO);
    int bad = 0;
    struct Events {                      // destroyed on every return path
        cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Events() {
            for (cudaEvent_t e : ev)
                if (e) cudaEventDestroy(e);
        }
    } events;
    for (cudaEvent_t &e : events.ev) CUDA_TRY(cudaEventCreate(&e));
    cudaEvent_t e0 = events.ev[0], e1 = events.ev[1], p0 = events.ev[2], p1 = events.ev[3];
    CUDA_TRY(cudaEventRecord(e0, st));
    k_cuhre_init<<<(unsigned)((nu * CU_STRIDE + 255) / 256), 256, 0, st>>>(nu, S.rc[0], S.rh[0], S.runit[0]);
    CUDA_TRY(cudaMemsetAsync(S.frz_v, 0, sizeof(double) * MAXO * nu, st));
    CUDA_TRY(cudaMemsetAsync(S.frz_e, 0, sizeof(double) * MAXO * nu, st));
    CUDA_TRY(cudaMemsetAsync(S.bad, 0, sizeof(int32_t), st));
    int launches = 1;
    int eval_launches = 0;
    double eval_ms = 0.0;
    int64_t frozen_total = 0;
    bool timed_out = false;
    const auto t_start = std::chrono::steady_clock::now();
    std::vector<int64_t> item_off(nu + 1);
    for (int pass = 0;; ++pass) {
        off[0] = 0;
        for (int64_t k = 0; k < nu; ++k) off[k + 1] = off[k] + nreg[k];
        const int64_t live = off[nu];
        if (live == 0) break;
        rc = cu_grow_regions(c, S, live);
        if (rc) break;
        CUDA_TRY(cudaMemcpyAsync(S.reg_off, off.data(), sizeof(int64_t) * (nu + 1), cudaMemcpyHostToDevice, st));
        // blocks: per unit, batches of whole regions (cu_batch regions each)
        item_off[0] = 0;
        for (int64_t k = 0; k < nu; ++k) {
            const int bt = cu_batch(P[k]);
            item_off[k + 1] = item_off[k] + (nreg[k] + bt - 1) / bt;
        }
        CUDA_TRY(cudaMemcpyAsync(S.item_off, item_off.data(), sizeof(int64_t) * (nu + 1), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaEventRecord(p0, st));
        k_cuhre_eval<<<(unsigned)item_off[nu], threads, L.total, st>>>(
            c->d_units, b, c->d_pre, c->d_cons64, c->d_logtab, S.item_off, S.reg_off, nu, S.rc[S.cur],
            S.rh[S.cur], S.rval, S.rerr, S.raxis, K, si.max_instr, si.max_const, si.max_slots);
        launches += 1;
        eval_launches += 1;
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaEventRecord(p1, st));
        const bool final_pass = pass + 1 >= max_passes;
        CuDecideArgs A{};
        A.units = c->d_units;
        A.unit_begin = b;
        A.reg_off = S.reg_off;
        A.rh = S.rh[S.cur];
        A.rval = S.rval;
        A.rerr = S.rerr;
        A.rflag = S.rflag;
        A.frz_v = S.frz_v;
        A.frz_e = S.frz_e;
        A.tot_v = S.tot_v;
        A.tot_e = S.tot_e;
        A.fp_v = S.fp_v;
        A.fp_e = S.fp_e;
        A.nsplit = S.nsplit;
        A.conv = S.conv;
        A.bad = S.bad;
        A.rel_tol = opt->rel_tol;
        A.abs_tol = opt->abs_tol;
        A.final_pass = final_pass ? 1 : 0;
        CUDA_TRY(cudaMemsetAsync(S.nsplit, 0, sizeof(int64_t) * nu, st));
        k_cuhre_decide<<<(unsigned)nu, 256, 0, st>>>(A);
        launches += 1;
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(nsp.data(), S.nsplit, sizeof(int64_t) * nu, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(hconv.data(), S.conv, sizeof(int32_t) * nu, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(tv.data(), S.tot_v, sizeof(double) * MAXO * nu, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(te.data(), S.tot_e, sizeof(double) * MAXO * nu, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(&bad, S.bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        float pms = 0.f;
        cudaEventElapsedTime(&pms, p0, p1);
        eval_ms += pms;
        int64_t new_live = 0, frozen_now = 0;
        for (int64_t u = 0; u < nu; ++u) {
            if (nreg[u] == 0) continue;
            passes_u[u] += 1;
            npts[u] += nreg[u] * P[u];
            conv[u] = hconv[u];
            for (int o = 0; o < NO[u]; ++o) {
                htv[u * MAXO + o] = tv[u * MAXO + o];
                hte[u * MAXO + o] = te[u * MAXO + o];
            }
            new_live += 2 * nsp[u];
            frozen_now += nreg[u] - nsp[u];
        }
        S.last_begin = b;
        S.last_n = nu;
        S.last_off = off;
        S.have_last = true;
        if (bad || final_pass || new_live == 0) break;
        if (frozen_total + frozen_now + new_live > max_regions) break;
        if (opt->timeout_ms > 0) {
            const double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
            if (el > (double)opt->timeout_ms) {
                timed_out = true;
                break;
            }
        }
        // next live list
        const int nxt = 1 - S.cur;
        rc = cu_grow_list(c, S, nxt, new_live);
        if (rc) break;
        std::vector<int64_t> noff(nu + 1, 0);
        for (int64_t u = 0; u < nu; ++u) noff[u + 1] = noff[u] + 2 * (nreg[u] ? nsp[u] : 0);
        CUDA_TRY(cudaMemcpyAsync(S.new_off, noff.data(), sizeof(int64_t) * (nu + 1), cudaMemcpyHostToDevice, st));
        CuSplitArgs B{};
        B.reg_off = S.reg_off;
        B.new_off = S.new_off;
        B.rflag = S.rflag;
        B.raxis = S.raxis;
        B.rc = S.rc[S.cur];
        B.rh = S.rh[S.cur];
        B.nc = S.rc[nxt];
        B.nh = S.rh[nxt];
        B.nunit = S.runit[nxt];
        B.frz_v = S.frz_v;
        B.frz_e = S.frz_e;
        B.fp_v = S.fp_v;
        B.fp_e = S.fp_e;
        k_cuhre_split<<<(unsigned)nu, 256, 0, st>>>(B);
        launches += 1;
        CUDA_TRY(cudaGetLastError());
        S.cur = nxt;
        for (int64_t u = 0; u < nu; ++u) {
            if (nreg[u] == 0) continue;
            nfrozen[u] += nreg[u] - nsp[u];
            nreg[u] = 2 * nsp[u];
        }
        frozen_total += frozen_now;
        S.have_last = false;
    }
    CUDA_TRY(cudaEventRecord(e1, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rc) return rc;
    // results
    const int lo = opt->order_lo;
    for (int k = 0; k < n_orders; ++k) value[k] = error[k] = 0.0;
    int64_t rec = 0, pts_all = 0, unit_pts = 0;
    for (int64_t u = 0; u < nu; ++u) {
        const DevUnit &du = c->units[b + u];
        pts_all += npts[u];
        unit_pts += npts[u] * (du.cplx ? NO[u] / 2 : NO[u]);
        for (int o = 0; o < NO[u]; ++o) {
            const int order = du.order + (du.cplx ? o / 2 : o);
            const int part = du.cplx ? (o & 1) : 0;
            if (part == 0 && order - lo >= 0 && order - lo < n_orders) {
                value[order - lo] += htv[u * MAXO + o];
                error[order - lo] += hte[u * MAXO + o];
            }
            if (per) {
                fiesta_cuhre_result &R = per[rec];
                R.value = htv[u * MAXO + o];
                R.error = hte[u * MAXO + o];
                R.n_regions = nfrozen[u] + nreg[u];
                R.n_points = npts[u];
                R.order = order;
                R.sector = du.pad;
                R.unit = (int32_t)(b + u);
                R.part = part;
                R.converged = conv[u];
                R.passes = passes_u[u];
            }
            ++rec;
        }
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->gpu_ms = ms;
        stats->eval_ms = eval_ms;
        stats->points = pts_all;
        stats->points_per_s = ms > 0 ? pts_all / (ms * 1e-3) : 0.0;
        stats->kernels_launched = launches;
        stats->eval_launches = eval_launches;
        stats->unit_points = unit_pts;
        stats->threads[0] = threads;
        stats->points_per_thread[0] = CU_ITEM_PTS / threads;
    }
    if (bad) return fail(FIESTA_E_NONFINITE, "fiesta_cuhre: a unit's estimate is not finite");
    if (timed_out) return fail(FIESTA_E_TIMEOUT, "fiesta_cuhre: time budget exceeded");
    return FIESTA_OK;
}

int fiesta_cuhre_regions(fiesta_ctx *c, int64_t unit, int64_t cap, double *center, double *half, double *value,
                         double *error, int32_t *axis, int64_t *n) {
    if (!c || !n || cap < 0 || (cap > 0 && (!center || !half || !value || !error || !axis)))
        return fail(FIESTA_E_INVALID, "fiesta_cuhre_regions: bad arguments");
    if (!c->cuhre || !c->cuhre->have_last) return fail(FIESTA_E_INVALID, "fiesta_cuhre_regions: no finished fiesta_cuhre call");
    CuhreState &S = *c->cuhre;
    if (unit < S.last_begin || unit >= S.last_begin + S.last_n)
        return fail(FIESTA_E_INVALID, "fiesta_cuhre_regions: unit not in the last call");
    const int64_t up = unit - S.last_begin;
    const int64_t a = S.last_off[up], cnt = S.last_off[up + 1] - a;
    *n = cnt;
    const int64_t m = std::min(cnt, cap);
    if (m == 0) return FIESTA_OK;
    const DevUnit &u = c->units[unit];
    const int nn = cu_n(u.dim), no = u.n_out;
    std::vector<double> cc(m * CU_STRIDE), hh(m * CU_STRIDE), vv(m * MAXO), ee(m * MAXO);
    cudaStream_t st = c->stream;
    CUDA_TRY(cudaMemcpyAsync(cc.data(), S.rc[S.cur] + a * CU_STRIDE, sizeof(double) * m * CU_STRIDE, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hh.data(), S.rh[S.cur] + a * CU_STRIDE, sizeof(double) * m * CU_STRIDE, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(vv.data(), S.rval + a * MAXO, sizeof(double) * m * MAXO, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(ee.data(), S.rerr + a * MAXO, sizeof(double) * m * MAXO, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(axis, S.raxis + a, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < m; ++i) {
        for (int j = 0; j < nn; ++j) {
            center[i * nn + j] = cc[i * CU_STRIDE + j];
            half[i * nn + j] = hh[i * CU_STRIDE + j];
        }
        for (int o = 0; o < no; ++o) {
            value[i * no + o] = vv[i * MAXO + o];
            error[i * no + o] = ee[i * MAXO + o];
        }
    }
    return FIESTA_OK;
}

}  // extern "C"
