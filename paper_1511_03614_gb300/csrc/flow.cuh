// flow.cuh -- learned importance sampler (a normalising flow) standing in for
// the Vegas map; included at the end of fiesta.cu (same translation unit).
//
// The flow is a bijection of the open unit cube: a = logit(x); four affine
// coupling layers a_B <- a_B exp(s) + t with (s, t) = MLP(a_A), s = 4 tanh(raw/4),
// MLP 16 -> 64 -> 64 -> 16 with ReLU; z = sigmoid(a) is uniform under the
// model.  Conditioning sets: A_0 even j, A_1 odd j, A_2 j < ceil(d/2),
// A_3 j >= ceil(d/2).  Sampling runs the layers backwards from z ~ U(0,1)^d and
// the estimator of a unit's integral is f(x) / q(x).
//
// k_flow_sample: one warp carries 32 points through the flow together, as two
//   16-row tiles of mma.sync.m16n8k16 (BF16 inputs, FP32 accumulation).  Lane
//   (g, t) = (lane / 4, lane % 4) owns coordinates 2t, 2t+1 of points g, g+8 (and
//   16+g, 24+g): exactly the entries of the A fragment of the first layer and of
//   the C fragment of the last, so s and t arrive in the lane that applies them,
//   and each layer's C fragments are the next layer's A fragments.  Then every
//   lane evaluates its own point with the bytecode interpreter.
// k_flow_train_tc: the gradient of L = -sum_i w_i log q(x_i) on the tensor cores:
//   one warp per 16 training points, forward pass, then per layer the MLP's
//   reverse mode as MMAs (BF16 operands, binary32 accumulation), the weight
//   gradients with the points as the MMA's K dimension (movmatrix transposes),
//   summed per block in shared memory.
// k_flow_adam: Adam update of the binary32 master weights; k_flow_pack: the
//   BF16 transposed copies the sampler reads.

namespace {

constexpr int FL_L = 4, FL_HID = 64, FL_IN = 16, FL_OUT = 16;
constexpr int FL_W1 = 0, FL_B1 = FL_W1 + FL_IN * FL_HID, FL_W2 = FL_B1 + FL_HID, FL_B2 = FL_W2 + FL_HID * FL_HID,
              FL_W3 = FL_B2 + FL_HID, FL_B3 = FL_W3 + FL_HID * FL_OUT, FL_PER_LAYER = FL_B3 + FL_OUT;
constexpr int FL_PARAMS = FL_L * FL_PER_LAYER;                       // 25152 floats per unit
// packed inference layout per layer: bf16 W1t[64][S1], W2t[64][S2], W3t[16][S2] (transposed,
// rows padded to S1 = 24 / S2 = 72 halves so that the eight row groups g of a B-fragment
// load, rows g*S words apart, land in distinct shared-memory banks); then f32 b1, b2, b3
constexpr int FLP_S1 = FL_IN + 8, FLP_S2 = FL_HID + 8;
constexpr int FLP_W1 = 0, FLP_W2 = FLP_W1 + FL_HID * FLP_S1, FLP_W3 = FLP_W2 + FL_HID * FLP_S2,
              FLP_HALVES = FLP_W3 + FL_OUT * FLP_S2;                 // 7296 bf16 per layer
constexpr int FLP_BIAS = FL_HID + FL_HID + FL_OUT;                   // 144 floats per layer
constexpr size_t FLP_LAYER_BYTES = FLP_HALVES * 2 + FLP_BIAS * 4;    // 15168
constexpr size_t FLP_UNIT_BYTES = FLP_LAYER_BYTES * FL_L;            // 60672
constexpr float FL_S = 4.0f;
constexpr int FL_THREADS = 128;                  // sampler block; FL_THREADS_MAX when only one block fits an SM
constexpr int FL_THREADS_MAX = 256;

__device__ __forceinline__ bool fl_in_A(int l, int j, int d) {
    const int half = (d + 1) >> 1;
    switch (l) {
    case 0: return (j & 1) == 0;
    case 1: return (j & 1) == 1;
    case 2: return j < half;
    default: return j >= half;
    }
}

__device__ __forceinline__ float softplusf(float y) { return y > 20.f ? y : log1pf(__expf(y)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// MLP of one layer for one 16-point tile.  in0/in1: this lane's two input
// coordinates (2t, 2t+1) of rows g and g+8 (already masked); out: raw_s and t of
// this lane's coordinates for rows g (o[0..1] s, o[2..3] t) and g+8 (o[4..7]).
// H1, H2: the two hidden activations after the ReLU, rounded to BF16, as the A
// fragments of the next MMA (k-tile kt: [0] row g, columns 16kt + 2t, +1; [1] row
// g + 8; [2], [3] the same rows at columns 16kt + 8 + 2t, +1); the training kernel
// keeps them for the reverse pass.
__device__ __forceinline__ void fl_mlp_tile_keep(const unsigned char *__restrict__ lay, float in_g0, float in_g1,
                                                 float in_h0, float in_h1, uint32_t (&A)[4][4], uint32_t (&A2)[4][4],
                                                 float (&o)[8]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 *W1t = reinterpret_cast<const __nv_bfloat16 *>(lay) + FLP_W1;
    const __nv_bfloat16 *W2t = reinterpret_cast<const __nv_bfloat16 *>(lay) + FLP_W2;
    const __nv_bfloat16 *W3t = reinterpret_cast<const __nv_bfloat16 *>(lay) + FLP_W3;
    const float *bias = reinterpret_cast<const float *>(lay + FLP_HALVES * 2);
    const float *b1 = bias, *b2 = bias + FL_HID, *b3 = bias + 2 * FL_HID;
    // layer 1: K = 16 (inputs 8..15 are zero), N = 64
    const uint32_t a0 = pack_bf16(in_g0, in_g1), a1 = pack_bf16(in_h0, in_h1);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t bb0 = *reinterpret_cast<const uint32_t *>(W1t + (nt * 8 + g) * FLP_S1 + 2 * t);
        mma_bf16(c, a0, a1, 0u, 0u, bb0, 0u);
        const float bx = b1[nt * 8 + 2 * t], by = b1[nt * 8 + 2 * t + 1];
        const uint32_t r0 = pack_bf16(fmaxf(c[0] + bx, 0.f), fmaxf(c[1] + by, 0.f));
        const uint32_t r1 = pack_bf16(fmaxf(c[2] + bx, 0.f), fmaxf(c[3] + by, 0.f));
        A[nt >> 1][(nt & 1) * 2 + 0] = r0;
        A[nt >> 1][(nt & 1) * 2 + 1] = r1;
    }
    // layer 2: K = 64, N = 64
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const __nv_bfloat16 *col = W2t + (nt * 8 + g) * FLP_S2 + kt * 16 + 2 * t;
            mma_bf16(c, A[kt][0], A[kt][1], A[kt][2], A[kt][3], *reinterpret_cast<const uint32_t *>(col),
                     *reinterpret_cast<const uint32_t *>(col + 8));
        }
        const float bx = b2[nt * 8 + 2 * t], by = b2[nt * 8 + 2 * t + 1];
        A2[nt >> 1][(nt & 1) * 2 + 0] = pack_bf16(fmaxf(c[0] + bx, 0.f), fmaxf(c[1] + by, 0.f));
        A2[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16(fmaxf(c[2] + bx, 0.f), fmaxf(c[3] + by, 0.f));
    }
    // layer 3: K = 64, N = 16 (n-tile 0: raw_s, n-tile 1: t)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const __nv_bfloat16 *col = W3t + (nt * 8 + g) * FLP_S2 + kt * 16 + 2 * t;
            mma_bf16(c, A2[kt][0], A2[kt][1], A2[kt][2], A2[kt][3], *reinterpret_cast<const uint32_t *>(col),
                     *reinterpret_cast<const uint32_t *>(col + 8));
        }
        const float bx = b3[nt * 8 + 2 * t], by = b3[nt * 8 + 2 * t + 1];
        o[nt * 2 + 0] = c[0] + bx;
        o[nt * 2 + 1] = c[1] + by;
        o[4 + nt * 2 + 0] = c[2] + bx;
        o[4 + nt * 2 + 1] = c[3] + by;
    }
}

__device__ __forceinline__ void fl_mlp_tile(const unsigned char *__restrict__ lay, float in_g0, float in_g1,
                                            float in_h0, float in_h1, float (&o)[8]) {
    uint32_t A[4][4], A2[4][4];
    fl_mlp_tile_keep(lay, in_g0, in_g1, in_h0, in_h1, A, A2, o);
}

struct FlowSampleParams {
    const DevUnit *units;
    const uint64_t *pre;               // forwarded programs (uops.cuh)
    const double *cons64;
    const float *cons32;
    const double *logtab;
    const unsigned char *packed;       // [unit][FLP_UNIT_BYTES]
    double *part_sv, *part_sv2;
    unsigned long long *part_bad;
    int64_t unit_begin, blocks_per_unit, points;
    uint32_t seed, iteration;
    int max_instr, max_const, max_slots;
    int64_t keep;                      // training points kept per unit
    float *tr_x;                       // [unit][keep][8]
    float *tr_lq, *tr_f;               // [unit][keep]
    const double *z_in;                // nullable: base points [points][dim] (check mode, one unit)
    double *x_out, *lq_out, *f_out;    // nullable: per point outputs (check mode; result 0)
    double *a_out;                     // logit coordinates of x_out (check mode)
    int out_stride;                    // records per block (largest n_out of the slice)
};

template <typename T>
__global__ void __launch_bounds__(FL_THREADS_MAX) k_flow_sample(FlowSampleParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t unit = p.unit_begin + blockIdx.x / p.blocks_per_unit;
    const int64_t blk = blockIdx.x % p.blocks_per_unit;
    const DevUnit u = p.units[unit];
    const int d = u.dim;
    // the program runs in its micro-op form (uops.cuh): shared memory viewed as T holds
    // the constants (then -0, 1, -1) below pt, and from pt on this block's coordinates
    // and slot file, [index][thread]
    size_t off = 0;
    unsigned char *s_flow = smem; off = align16(off + FLP_UNIT_BYTES);
    uint64_t *s_uops = reinterpret_cast<uint64_t *>(smem + off); off = align16(off + 8 * (p.max_instr + 1));
    T *s_cons = reinterpret_cast<T *>(smem + off); off = align16(off + sizeof(T) * (p.max_const + 3));
    double *s_tab = reinterpret_cast<double *>(smem + off); off = align16(off + 8 * LOGTAB_DOUBLES);
    T *s_x = reinterpret_cast<T *>(smem + off); off = align16(off + sizeof(T) * MAXD * nt);
    T *s_slots = reinterpret_cast<T *>(smem + off); off = align16(off + sizeof(T) * p.max_slots * nt);
    float *s_lq = reinterpret_cast<float *>(smem + off); off = align16(off + 4 * nt);
    // x and logit(x) in binary32, rows of nt + 4: the four lanes t of a row group g that
    // write one coordinate land in distinct banks
    const int xs = nt + 4;
    float *s_xf = reinterpret_cast<float *>(smem + off); off = align16(off + 4 * MAXD * xs);
    float *s_af = reinterpret_cast<float *>(smem + off); off = align16(off + 4 * MAXD * xs);
    double *s_acc = reinterpret_cast<double *>(smem + off); off = align16(off + 8 * 2 * MAXO * nt);
    double *s_red = reinterpret_cast<double *>(smem + off);
    T *E = reinterpret_cast<T *>(smem);
    const int cons_base = static_cast<int>((reinterpret_cast<unsigned char *>(s_cons) - smem) / sizeof(T));
    const int k_zero = cons_base + p.max_const;
    const int pt = static_cast<int>((reinterpret_cast<unsigned char *>(s_x) - smem) / sizeof(T));
    const int slot_base = static_cast<int>((reinterpret_cast<unsigned char *>(s_slots) - smem) / sizeof(T));
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.packed + unit * FLP_UNIT_BYTES);
        uint4 *dst = reinterpret_cast<uint4 *>(s_flow);
        for (int i = tid; i < (int)(FLP_UNIT_BYTES / 16); i += nt) dst[i] = src[i];
    }
    for (int i = tid; i < u.n_uop; i += nt)
        s_uops[i] = uop_from_pre(p.pre[u.uop_off + i], cons_base, k_zero, pt, slot_base, nt);
    if (tid == 0) {
        s_uops[u.n_uop] = 0ull;                          // fetched after the last word, never executed
        s_cons[p.max_const] = T(-0.0);
        s_cons[p.max_const + 1] = T(1);
        s_cons[p.max_const + 2] = T(-1);
    }
    for (int i = tid; i < u.n_const; i += nt)
        s_cons[i] = sizeof(T) == 8 ? static_cast<T>(p.cons64[u.const_off + i]) : static_cast<T>(p.cons32[u.const_off + i]);
    for (int i = tid; i < LOGTAB_DOUBLES; i += nt) s_tab[i] = p.logtab[i];
    __syncthreads();

    const int64_t per_block = (p.points + p.blocks_per_unit - 1) / p.blocks_per_unit;
    const int64_t first = blk * per_block, last = min(p.points, first + per_block);
    const int no = u.n_out;
    for (int k = 0; k < 2 * MAXO; ++k) s_acc[k * nt + tid] = 0.0;     // this thread's sums per result
    unsigned long long bad = 0;
    for (int64_t base = first; base < last; base += nt) {
        // this warp's 32 points: base + warp*32 + (0..31)
        const int64_t wbase = base + warp * 32;
        // lane owns coords 2t, 2t+1 of rows r = g, g+8, 16+g, 24+g
        float a[4][2], lq[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int row = (r & 1) * 8 + (r >> 1) * 16 + g;
            const int64_t pi = wbase + row;
            lq[r] = 0.f;
            float zz[2] = {0.5f, 0.5f};
            if (p.z_in) {
                for (int h = 0; h < 2; ++h)
                    if (2 * t + h < d && pi < last) zz[h] = static_cast<float>(p.z_in[pi * d + 2 * t + h]);
            } else if (2 * t < d) {
                uint32_t c0 = static_cast<uint32_t>(pi), c1 = static_cast<uint32_t>(pi >> 32), c2 = p.iteration,
                         c3 = 0x40000000u + t;
                philox4x32_10(c0, c1, c2, c3, p.seed, u.rng_key);
                // uniforms (2k+1) 2^-24 with k of 23 bits: 2k+1 < 2^24 is exact in
                // binary32, so z is never 0 or 1
                zz[0] = static_cast<float>(2u * (c1 >> 9) + 1u) * 0x1p-24f;
                zz[1] = static_cast<float>(2u * (c3 >> 9) + 1u) * 0x1p-24f;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float zv = zz[h];
                const float av = logf(zv) - log1pf(-zv);
                a[r][h] = av;
                if (2 * t + h < d) lq[r] += -softplusf(-av) - softplusf(av);     // log z + log(1 - z)
            }
        }
        for (int l = FL_L - 1; l >= 0; --l) {
            const unsigned char *lay = s_flow + l * FLP_LAYER_BYTES;
            const bool inA0 = fl_in_A(l, 2 * t, d) && 2 * t < d, inA1 = fl_in_A(l, 2 * t + 1, d) && 2 * t + 1 < d;
            const bool inB0 = !fl_in_A(l, 2 * t, d) && 2 * t < d, inB1 = !fl_in_A(l, 2 * t + 1, d) && 2 * t + 1 < d;
#pragma unroll
            for (int m = 0; m < 2; ++m) {              // two 16-point tiles
                float o[8];
                fl_mlp_tile(lay, inA0 ? a[2 * m][0] : 0.f, inA1 ? a[2 * m][1] : 0.f, inA0 ? a[2 * m + 1][0] : 0.f,
                            inA1 ? a[2 * m + 1][1] : 0.f, o);
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    const int r = 2 * m + rr;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const bool inB = h ? inB1 : inB0;
                        if (!inB) continue;
                        const float s = FL_S * tanhf(o[rr * 4 + h] / FL_S);
                        const float tt = o[rr * 4 + 2 + h];
                        a[r][h] = (a[r][h] - tt) * __expf(-s);
                        lq[r] += s;
                    }
                }
            }
        }
        // x = sigmoid(a); log q gets -log x - log(1 - x); the quad sums its lanes' parts
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int row = (r & 1) * 8 + (r >> 1) * 16 + g;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (2 * t + h >= d) continue;
                const float av = a[r][h];
                lq[r] += softplusf(-av) + softplusf(av);
                const float xv = 1.f / (1.f + __expf(-av));
                s_xf[(2 * t + h) * xs + warp * 32 + row] = xv;
                s_af[(2 * t + h) * xs + warp * 32 + row] = av;
            }
            float v = lq[r];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            if (t == 0) s_lq[warp * 32 + row] = v;
        }
        __syncwarp();
        // every lane evaluates its own point
        const int64_t pi = wbase + lane;
        const float lqv = s_lq[tid];
        for (int j = 0; j < d; ++j) s_x[j * nt + tid] = static_cast<T>(s_xf[j * xs + tid]);
        interpret_uop<T>(s_uops, u.n_uop, E, pt, tid, s_tab);
        // a coordinate below the binary32 range (x = sigmoid(a) underflows; measure
        // < 1e-38 per coordinate) makes the point contribute zero
        bool in_range = true;
        for (int j = 0; j < d; ++j) in_range = in_range && s_xf[j * xs + tid] >= 1.17549435e-38f;
        if (pi < last) {
            const double iq = exp(-static_cast<double>(lqv));
            bool finite = true;
            double f2 = 0.0;              // |f|^2 summed over the results: the training target
            for (int k = 0; k < no; ++k) {
                const double fk = static_cast<double>(s_slots[tid + u.outs[k] * nt]);
                finite = finite && isfinite(in_range ? fk * iq : 0.0);
                f2 = fma(fk, fk, f2);
            }
            if (!finite) ++bad;
            for (int k = 0; k < no; ++k) {
                const double v = (finite && in_range) ? static_cast<double>(s_slots[tid + u.outs[k] * nt]) * iq : 0.0;
                s_acc[(2 * k) * nt + tid] += v;
                s_acc[(2 * k + 1) * nt + tid] = fma(v, v, s_acc[(2 * k + 1) * nt + tid]);
            }
            const double f0 = static_cast<double>(s_slots[tid + u.outs[0] * nt]);
            if (pi < p.keep) {
                // training points are kept as logit coordinates a (x may round to 1 in binary32);
                // the target of a unit with several results is the norm of its result vector
                float *dst = p.tr_x + (unit * p.keep + pi) * MAXD;
                for (int j = 0; j < MAXD; ++j) dst[j] = j < d ? s_af[j * xs + tid] : 0.f;
                p.tr_lq[unit * p.keep + pi] = lqv;
                p.tr_f[unit * p.keep + pi] = static_cast<float>(no == 1 ? f0 : sqrt(f2));
            }
            if (p.x_out) {
                for (int j = 0; j < d; ++j) {
                    p.x_out[pi * d + j] = s_xf[j * xs + tid];
                    p.a_out[pi * d + j] = s_af[j * xs + tid];
                }
                p.lq_out[pi] = lqv;
                p.f_out[pi] = f0;
            }
        }
        __syncwarp();
    }
    // block sums in a fixed order -> one record per (unit, block, result)
    double sv[MAXO], sv2[MAXO];
#pragma unroll
    for (int k = 0; k < MAXO; ++k) {
        sv[k] = s_acc[(2 * k) * nt + tid];
        sv2[k] = s_acc[(2 * k + 1) * nt + tid];
    }
    block_sum_vec<MAXO>(sv, sv2, bad, no, reinterpret_cast<unsigned char *>(s_red));
    if (tid == 0) {
        const int64_t item = (unit - p.unit_begin) * p.blocks_per_unit + blk;
#pragma unroll
        for (int k = 0; k < MAXO; ++k)
            if (k < no) {
                p.part_sv[item * p.out_stride + k] = sv[k];
                p.part_sv2[item * p.out_stride + k] = sv2[k];
            }
        p.part_bad[item] = bad;
    }
}

// per-unit normaliser of the training weights: sum_i (|f_i| / q_i)^power
__global__ void k_flow_wsum(const float *tr_lq, const float *tr_f, int64_t keep, int power, int64_t unit_begin,
                            double *wsum) {
    __shared__ double s[128];
    const int64_t unit = unit_begin + blockIdx.x;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < keep; i += blockDim.x) {
        const double r = fabs(static_cast<double>(tr_f[unit * keep + i])) * exp(-static_cast<double>(tr_lq[unit * keep + i]));
        const double w = power == 2 ? r * r : r;
        if (isfinite(w)) acc += w;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) wsum[blockIdx.x] = s[0];
}

struct FlowTrainParams {
    const DevUnit *units;
    const float *params;              // [unit][FL_PARAMS] binary32 master weights
    float *grad;                      // [unit][FL_PARAMS]
    const float *tr_x, *tr_lq, *tr_f; // training points
    const double *wsum;               // [slice position]
    const double *w_in;               // nullable: explicit weights [keep] (check mode, one unit)
    double *loss;                     // [slice position]
    double *lq_out;                   // nullable: log q per point (check mode)
    int64_t unit_begin, keep, blocks_per_unit;
    int64_t buf_unit0;                // training-buffer row of the slice's first unit (rows hold logit coordinates)
    int power;
};

__global__ void k_flow_adam(float *params, const float *grad, float *m, float *v, int64_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// one layer's binary32 master weights -> the packed inference layout (BF16 transposed
// weights + binary32 biases), by the threads of a block
__device__ __forceinline__ void fl_pack_layer(const float *__restrict__ PL, unsigned char *dst) {
    __nv_bfloat16 *h = reinterpret_cast<__nv_bfloat16 *>(dst);
    float *b = reinterpret_cast<float *>(dst + FLP_HALVES * 2);
    for (int e = threadIdx.x; e < FL_HID * FLP_S1; e += blockDim.x) {    // W1t[n][k] = W1[k][n]
        const int n = e / FLP_S1, k = e % FLP_S1;
        h[FLP_W1 + e] = __float2bfloat16_rn(k < FL_IN ? PL[FL_W1 + k * FL_HID + n] : 0.f);
    }
    for (int e = threadIdx.x; e < FL_HID * FLP_S2; e += blockDim.x) {
        const int n = e / FLP_S2, k = e % FLP_S2;
        h[FLP_W2 + e] = __float2bfloat16_rn(k < FL_HID ? PL[FL_W2 + k * FL_HID + n] : 0.f);
    }
    for (int e = threadIdx.x; e < FL_OUT * FLP_S2; e += blockDim.x) {    // W3t[n][k] = W3[k][n]
        const int n = e / FLP_S2, k = e % FLP_S2;
        h[FLP_W3 + e] = __float2bfloat16_rn(k < FL_HID ? PL[FL_W3 + k * FL_OUT + n] : 0.f);
    }
    for (int e = threadIdx.x; e < FLP_BIAS; e += blockDim.x)
        b[e] = e < FL_HID ? PL[FL_B1 + e] : (e < 2 * FL_HID ? PL[FL_B2 + e - FL_HID] : PL[FL_B3 + e - 2 * FL_HID]);
}

// binary32 master -> packed BF16 transposed weights + binary32 biases
__global__ void k_flow_pack(const float *params, unsigned char *packed, int64_t unit_begin) {
    const int64_t unit = unit_begin + blockIdx.x;
    const float *P = params + unit * FL_PARAMS;
    unsigned char *dst = packed + unit * FLP_UNIT_BYTES;
    for (int l = 0; l < FL_L; ++l) fl_pack_layer(P + l * FL_PER_LAYER, dst + l * FLP_LAYER_BYTES);
}

// ---------------------------------------------------------------------------
// Training on the tensor cores.
//
// k_flow_train_tc computes the loss L = -sum_i w_i log q(x_i) and its gradient by
// reverse mode, with every dense product of the MLP on mma.sync.m16n8k16 (BF16
// operands, binary32 accumulation) and the coupling arithmetic in binary32.  One warp takes 16
// training points at a time, in the fragment layout of k_flow_sample: lane
// (g, t) owns coordinates 2t, 2t+1 of points g and g + 8.  Per 16-point tile:
//   forward, layer by layer, keeping each layer's input;
//   reverse, layer by layer: recompute the layer's MLP (hidden activations kept as
//     BF16 A fragments), then
//       dH2 = (dout W3^T) masked by H2 > 0,   dH1 = (dH2 W2^T) masked by H1 > 0,
//       d(input) = dH1 W1^T                                    (MMA, K = 16 / 64)
//       dW3 = H2^T dout,  dW2 = H1^T dH2,  dW1 = In^T dH1      (MMA, K = the 16 points)
//     with the point-major fragments turned into the K = points operands by
//     movmatrix (8x8 transposes in registers); the bias gradients are the same
//     products with an all-ones operand (db1 rides in dW1's spare input row 8).
// The weight gradients of the block accumulate in shared memory (binary32) and are
// added to the unit's gradient once per block.  Rounding: the MMA operands (layer
// inputs, weights, hidden activations, dout, dH2, dH1) are BF16; the ReLU masks
// are taken on the BF16 activations.
// ---------------------------------------------------------------------------

// reverse-pass weight copies per layer (BF16, untransposed, rows padded like the
// inference copy): W1n[8][S2] (input rows 0..7; inputs 8..15 are always zero),
// W2n[64][S2], W3n[64][S1]
constexpr int FLB_W1 = 0, FLB_W2 = FLB_W1 + MAXD * FLP_S2, FLB_W3 = FLB_W2 + FL_HID * FLP_S2,
              FLB_HALVES = FLB_W3 + FL_HID * FLP_S1;                 // 6720 bf16 per layer
// the block's gradient accumulators per layer (binary32), rows padded so that the
// eight row groups of an MMA result fragment fall in distinct bank pairs:
// GW1[8][S2] (input rows 0..7), GW2[64][S2], GW3[64][S1], then gb1[64], gb2[64], gb3[16]
constexpr int FLG_W1 = 0, FLG_W2 = FLG_W1 + MAXD * FLP_S2, FLG_W3 = FLG_W2 + FL_HID * FLP_S2,
              FLG_B1 = FLG_W3 + FL_HID * FLP_S1, FLG_B2 = FLG_B1 + FL_HID, FLG_B3 = FLG_B2 + FL_HID,
              FLG_LAYER = FLG_B3 + FL_OUT;                           // 6864 floats per layer
constexpr int FLT_THREADS = 256;
constexpr size_t FLT_SMEM = FLP_UNIT_BYTES + FL_L * FLB_HALVES * 2 + FL_L * FLG_LAYER * sizeof(float);   // 224 256 B
static_assert(FLP_S1 % 32 == 24 && FLP_S2 % 32 == 8, "padded strides keep the gradient atomics conflict-free");
static_assert(MAXD == 8, "the training tile maps coordinates 2t, 2t+1 of four lanes onto eight dimensions");

// transpose of an 8x8 BF16 matrix held as one pair per lane (row lane/4, columns 2(lane%4), +1)
__device__ __forceinline__ uint32_t mov_t(uint32_t x) {
    uint32_t y;
    asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;\n" : "=r"(y) : "r"(x));
    return y;
}

// the two halves of a BF16 pair masked by the ReLU of another pair (kept where that value is > 0)
__device__ __forceinline__ uint32_t relu_mask_pack(float lo, float hi, uint32_t act) {
    return pack_bf16((act & 0x7fffu) ? lo : 0.f, (act & 0x7fff0000u) ? hi : 0.f);
}

__device__ __forceinline__ void sadd(float *a, float v) {
    if (v != 0.f) atomicAdd(a, v);
}

// adds (lo, hi) to a[0], a[1]; row groups g >= 4 take the two in the other order, so
// that with row strides of 8 or 24 words (mod 32) every shared-memory atomic of the
// warp lands in its own bank
__device__ __forceinline__ void sadd_pair(float *a, float lo, float hi, bool swap) {
    atomicAdd(swap ? a + 1 : a, swap ? hi : lo);
    atomicAdd(swap ? a : a + 1, swap ? lo : hi);
}

__global__ void __launch_bounds__(FLT_THREADS, 1) k_flow_train_tc(FlowTrainParams p) {
    extern __shared__ __align__(16) unsigned char tsm[];
    unsigned char *s_fwd = tsm;
    __nv_bfloat16 *s_bwd = reinterpret_cast<__nv_bfloat16 *>(tsm + FLP_UNIT_BYTES);
    float *s_g = reinterpret_cast<float *>(tsm + FLP_UNIT_BYTES + FL_L * FLB_HALVES * 2);   // [layer][FLG_LAYER]
    __shared__ double s_loss[FLT_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t pos = blockIdx.x / p.blocks_per_unit, unit = p.unit_begin + pos;
    const int64_t blk = blockIdx.x % p.blocks_per_unit;
    const int d = p.units[unit].dim;
    const float *P = p.params + unit * FL_PARAMS;
    for (int l = 0; l < FL_L; ++l) {
        const float *PL = P + l * FL_PER_LAYER;
        fl_pack_layer(PL, s_fwd + l * FLP_LAYER_BYTES);
        __nv_bfloat16 *B = s_bwd + l * FLB_HALVES;
        for (int e = tid; e < MAXD * FLP_S2; e += blockDim.x) {
            const int j = e / FLP_S2, k = e % FLP_S2;
            B[FLB_W1 + e] = __float2bfloat16_rn(k < FL_HID ? PL[FL_W1 + j * FL_HID + k] : 0.f);
        }
        for (int e = tid; e < FL_HID * FLP_S2; e += blockDim.x) {
            const int j = e / FLP_S2, k = e % FLP_S2;
            B[FLB_W2 + e] = __float2bfloat16_rn(k < FL_HID ? PL[FL_W2 + j * FL_HID + k] : 0.f);
        }
        for (int e = tid; e < FL_HID * FLP_S1; e += blockDim.x) {
            const int j = e / FLP_S1, k = e % FLP_S1;
            B[FLB_W3 + e] = __float2bfloat16_rn(k < FL_OUT ? PL[FL_W3 + j * FL_OUT + k] : 0.f);
        }
    }
    for (int i = tid; i < FL_L * FLG_LAYER; i += blockDim.x) s_g[i] = 0.f;
    __syncthreads();

    const uint32_t ONE2 = pack_bf16(1.f, 1.f);
    const bool swap = g >= 4;
    const int64_t per_block = (p.keep + p.blocks_per_unit - 1) / p.blocks_per_unit;
    const int64_t first = blk * per_block, last = min(p.keep, first + per_block);
    const int64_t ntiles = last > first ? (last - first + 15) / 16 : 0;
    double loss = 0.0;
    for (int64_t tile = warp; tile < ntiles; tile += nw) {
        const int64_t rbase = first + tile * 16;
        float a[2][2], al[FL_L][2][2], w[2], lq[2];
        bool valid[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int64_t i = rbase + g + 8 * r;
            valid[r] = i < last;
            a[r][0] = a[r][1] = 0.f;
            w[r] = 0.f;
            if (valid[r]) {
                const int64_t row = (p.buf_unit0 + pos) * p.keep + i;
                a[r][0] = p.tr_x[row * MAXD + 2 * t];
                a[r][1] = p.tr_x[row * MAXD + 2 * t + 1];
                if (p.w_in) {
                    w[r] = static_cast<float>(p.w_in[i]);
                } else {
                    const double rr = fabs(static_cast<double>(p.tr_f[row])) * exp(-static_cast<double>(p.tr_lq[row]));
                    const double ww = (p.power == 2 ? rr * rr : rr) / p.wsum[pos];
                    w[r] = isfinite(ww) ? static_cast<float>(ww) : 0.f;
                }
            }
            // a point with a non-finite coordinate is skipped (all four lanes of its row agree)
            int fin = isfinite(a[r][0]) && isfinite(a[r][1]);
            fin &= __shfl_xor_sync(0xffffffffu, fin, 1);
            fin &= __shfl_xor_sync(0xffffffffu, fin, 2);
            if (!fin) {
                a[r][0] = a[r][1] = 0.f;
                w[r] = 0.f;
            }
            lq[r] = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (2 * t + h < d) lq[r] += softplusf(-a[r][h]) + softplusf(a[r][h]);   // -log x - log(1 - x)
        }
        // normalising pass
#pragma unroll
        for (int l = 0; l < FL_L; ++l) {
            const bool inA0 = 2 * t < d && fl_in_A(l, 2 * t, d), inA1 = 2 * t + 1 < d && fl_in_A(l, 2 * t + 1, d);
            const bool inB0 = 2 * t < d && !fl_in_A(l, 2 * t, d), inB1 = 2 * t + 1 < d && !fl_in_A(l, 2 * t + 1, d);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                al[l][r][0] = a[r][0];
                al[l][r][1] = a[r][1];
            }
            float o[8];
            fl_mlp_tile(s_fwd + l * FLP_LAYER_BYTES, inA0 ? a[0][0] : 0.f, inA1 ? a[0][1] : 0.f, inA0 ? a[1][0] : 0.f,
                        inA1 ? a[1][1] : 0.f, o);
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (h ? inB1 : inB0) {
                        const float s = FL_S * tanhf(o[r * 4 + h] / FL_S);
                        a[r][h] = a[r][h] * __expf(s) + o[r * 4 + 2 + h];
                        lq[r] += s;
                    }
        }
        float gs[2][2];                      // dL/da of this lane's coordinates
#pragma unroll
        for (int r = 0; r < 2; ++r) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                gs[r][h] = 0.f;
                if (2 * t + h < d) {
                    lq[r] += -softplusf(-a[r][h]) - softplusf(a[r][h]);          // log z + log(1 - z)
                    const float sg = 1.f / (1.f + __expf(-a[r][h]));
                    gs[r][h] = -w[r] * (1.f - 2.f * sg);
                }
            }
            float v = lq[r];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            if (t == 0 && valid[r]) {
                loss += -static_cast<double>(w[r]) * v;
                if (p.lq_out) p.lq_out[rbase + g + 8 * r] = v;
            }
        }
        // reverse pass
#pragma unroll
        for (int l = FL_L - 1; l >= 0; --l) {
            const unsigned char *lay = s_fwd + l * FLP_LAYER_BYTES;
            const __nv_bfloat16 *W1n = s_bwd + l * FLB_HALVES + FLB_W1, *W2n = s_bwd + l * FLB_HALVES + FLB_W2,
                                *W3n = s_bwd + l * FLB_HALVES + FLB_W3;
            float *GL = s_g + l * FLG_LAYER;
            const bool inA0 = 2 * t < d && fl_in_A(l, 2 * t, d), inA1 = 2 * t + 1 < d && fl_in_A(l, 2 * t + 1, d);
            const bool inB0 = 2 * t < d && !fl_in_A(l, 2 * t, d), inB1 = 2 * t + 1 < d && !fl_in_A(l, 2 * t + 1, d);
            const float i00 = inA0 ? al[l][0][0] : 0.f, i01 = inA1 ? al[l][0][1] : 0.f;
            const float i10 = inA0 ? al[l][1][0] : 0.f, i11 = inA1 ? al[l][1][1] : 0.f;
            uint32_t H1[4][4], H2[4][4];
            float o[8];
            fl_mlp_tile_keep(lay, i00, i01, i10, i11, H1, H2, o);
            // dL/d(raw s) and dL/dt of this lane's coordinates (zero off B)
            float ds[2][2], dt[2][2];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    ds[r][h] = 0.f;
                    dt[r][h] = 0.f;
                    if (h ? inB1 : inB0) {
                        const float th = tanhf(o[r * 4 + h] / FL_S);
                        const float es = __expf(FL_S * th);
                        ds[r][h] = (gs[r][h] * al[l][r][h] * es - w[r]) * (1.f - th * th);
                        dt[r][h] = gs[r][h];
                        gs[r][h] *= es;
                    }
                }
            // dout as the A fragment of K = 16 outputs (raw s columns 0..7, t columns 8..15)
            const uint32_t dA0 = pack_bf16(ds[0][0], ds[0][1]), dA1 = pack_bf16(ds[1][0], ds[1][1]);
            const uint32_t dA2 = pack_bf16(dt[0][0], dt[0][1]), dA3 = pack_bf16(dt[1][0], dt[1][1]);
            // dout as B fragments with K = the 16 points: [output n-tile][points 0..7 / 8..15]
            const uint32_t Bd[2][2] = {{mov_t(dA0), mov_t(dA1)}, {mov_t(dA2), mov_t(dA3)}};
            // dW3 = H2^T dout (rows: hidden units), db3 = 1^T dout
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                const uint32_t a0 = mov_t(H2[mt][0]), a1 = mov_t(H2[mt][2]), a2 = mov_t(H2[mt][1]), a3 = mov_t(H2[mt][3]);
#pragma unroll
                for (int no = 0; no < 2; ++no) {
                    float c[4] = {0.f, 0.f, 0.f, 0.f};
                    mma_bf16(c, a0, a1, a2, a3, Bd[no][0], Bd[no][1]);
                    float *G = GL + FLG_W3 + (16 * mt + g) * FLP_S1 + 8 * no + 2 * t;
                    sadd_pair(G, c[0], c[1], swap);
                    sadd_pair(G + 8 * FLP_S1, c[2], c[3], swap);
                }
            }
#pragma unroll
            for (int no = 0; no < 2; ++no) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_bf16(c, ONE2, ONE2, ONE2, ONE2, Bd[no][0], Bd[no][1]);
                if (g == 0) {
                    sadd(GL + FLG_B3 + 8 * no + 2 * t, c[0]);
                    sadd(GL + FLG_B3 + 8 * no + 2 * t + 1, c[1]);
                }
            }
            // dH2 = dout W3^T, masked by H2 > 0, as A fragments
            uint32_t G2[4][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                const __nv_bfloat16 *col = W3n + (nt * 8 + g) * FLP_S1 + 2 * t;
                mma_bf16(c, dA0, dA1, dA2, dA3, *reinterpret_cast<const uint32_t *>(col),
                         *reinterpret_cast<const uint32_t *>(col + 8));
                G2[nt >> 1][(nt & 1) * 2 + 0] = relu_mask_pack(c[0], c[1], H2[nt >> 1][(nt & 1) * 2 + 0]);
                G2[nt >> 1][(nt & 1) * 2 + 1] = relu_mask_pack(c[2], c[3], H2[nt >> 1][(nt & 1) * 2 + 1]);
            }
            // dH1 = dH2 W2^T, masked by H1 > 0
            uint32_t G1[4][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kt = 0; kt < 4; ++kt) {
                    const __nv_bfloat16 *col = W2n + (nt * 8 + g) * FLP_S2 + kt * 16 + 2 * t;
                    mma_bf16(c, G2[kt][0], G2[kt][1], G2[kt][2], G2[kt][3], *reinterpret_cast<const uint32_t *>(col),
                             *reinterpret_cast<const uint32_t *>(col + 8));
                }
                G1[nt >> 1][(nt & 1) * 2 + 0] = relu_mask_pack(c[0], c[1], H1[nt >> 1][(nt & 1) * 2 + 0]);
                G1[nt >> 1][(nt & 1) * 2 + 1] = relu_mask_pack(c[2], c[3], H1[nt >> 1][(nt & 1) * 2 + 1]);
            }
            // dW2 = H1^T dH2, db2 = 1^T dH2
            uint32_t H1T[4][4];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                H1T[mt][0] = mov_t(H1[mt][0]);
                H1T[mt][1] = mov_t(H1[mt][2]);
                H1T[mt][2] = mov_t(H1[mt][1]);
                H1T[mt][3] = mov_t(H1[mt][3]);
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint32_t b0 = mov_t(G2[nt >> 1][(nt & 1) * 2 + 0]), b1 = mov_t(G2[nt >> 1][(nt & 1) * 2 + 1]);
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                    float c[4] = {0.f, 0.f, 0.f, 0.f};
                    mma_bf16(c, H1T[mt][0], H1T[mt][1], H1T[mt][2], H1T[mt][3], b0, b1);
                    float *G = GL + FLG_W2 + (16 * mt + g) * FLP_S2 + 8 * nt + 2 * t;
                    sadd_pair(G, c[0], c[1], swap);
                    sadd_pair(G + 8 * FLP_S2, c[2], c[3], swap);
                }
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_bf16(c, ONE2, ONE2, ONE2, ONE2, b0, b1);
                if (g == 0) {
                    sadd(GL + FLG_B2 + 8 * nt + 2 * t, c[0]);
                    sadd(GL + FLG_B2 + 8 * nt + 2 * t + 1, c[1]);
                }
            }
            // d(input) = dH1 W1^T (N = the 8 coordinates): reaches the conditioning coordinates
            {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kt = 0; kt < 4; ++kt) {
                    const __nv_bfloat16 *col = W1n + g * FLP_S2 + kt * 16 + 2 * t;
                    mma_bf16(c, G1[kt][0], G1[kt][1], G1[kt][2], G1[kt][3], *reinterpret_cast<const uint32_t *>(col),
                             *reinterpret_cast<const uint32_t *>(col + 8));
                }
                if (inA0) {
                    gs[0][0] += c[0];
                    gs[1][0] += c[2];
                }
                if (inA1) {
                    gs[0][1] += c[1];
                    gs[1][1] += c[3];
                }
            }
            // dW1 = In^T dH1 with In's input column 8 set to one: row 8 of the product is db1
            {
                const uint32_t a0 = mov_t(pack_bf16(i00, i01)), a2 = mov_t(pack_bf16(i10, i11));
                const uint32_t a1 = g == 0 ? ONE2 : 0u;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const uint32_t b0 = mov_t(G1[nt >> 1][(nt & 1) * 2 + 0]), b1 = mov_t(G1[nt >> 1][(nt & 1) * 2 + 1]);
                    float c[4] = {0.f, 0.f, 0.f, 0.f};
                    mma_bf16(c, a0, a1, a2, a1, b0, b1);
                    if (g < d) sadd_pair(GL + FLG_W1 + g * FLP_S2 + 8 * nt + 2 * t, c[0], c[1], swap);
                    if (g == 0) {
                        sadd(GL + FLG_B1 + 8 * nt + 2 * t, c[2]);
                        sadd(GL + FLG_B1 + 8 * nt + 2 * t + 1, c[3]);
                    }
                }
            }
        }
    }
    // the block's gradient into the unit's (one atomic per nonzero entry), and its loss
    __syncthreads();
    float *G = p.grad + unit * FL_PARAMS;
    for (int i = tid; i < FL_PARAMS; i += blockDim.x) {
        const int l = i / FL_PER_LAYER, e = i % FL_PER_LAYER;
        const float *GL = s_g + l * FLG_LAYER;
        float v = 0.f;
        if (e < FL_B1) {
            const int k = (e - FL_W1) / FL_HID, n = (e - FL_W1) % FL_HID;
            v = k < MAXD ? GL[FLG_W1 + k * FLP_S2 + n] : 0.f;         // inputs 8..15 are always zero
        } else if (e < FL_W2) {
            v = GL[FLG_B1 + e - FL_B1];
        } else if (e < FL_B2) {
            v = GL[FLG_W2 + (e - FL_W2) / FL_HID * FLP_S2 + (e - FL_W2) % FL_HID];
        } else if (e < FL_W3) {
            v = GL[FLG_B2 + e - FL_B2];
        } else if (e < FL_B3) {
            v = GL[FLG_W3 + (e - FL_W3) / FL_OUT * FLP_S1 + (e - FL_W3) % FL_OUT];
        } else {
            v = GL[FLG_B3 + e - FL_B3];
        }
        sadd(G + i, v);
    }
    loss += __shfl_xor_sync(0xffffffffu, loss, 16);
    loss += __shfl_xor_sync(0xffffffffu, loss, 8);
    loss += __shfl_xor_sync(0xffffffffu, loss, 4);
    loss += __shfl_xor_sync(0xffffffffu, loss, 2);
    loss += __shfl_xor_sync(0xffffffffu, loss, 1);
    if (lane == 0) s_loss[warp] = loss;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int k = 0; k < nw; ++k) s += s_loss[k];
        atomicAdd(p.loss + pos, s);
    }
}

__global__ void k_flow_init(float *params, int64_t n_units, uint32_t seed, float scale) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_units * FL_PARAMS) return;
    const int e = static_cast<int>(i % FL_PARAMS) % FL_PER_LAYER;
    float v = 0.f;
    if ((e >= FL_W1 && e < FL_B1) || (e >= FL_W2 && e < FL_B2)) {
        uint32_t c0 = static_cast<uint32_t>(i), c1 = static_cast<uint32_t>(i >> 32), c2 = 0x70000000u, c3 = 0;
        philox4x32_10(c0, c1, c2, c3, seed, 0x5eedu);
        // Box-Muller normal from two 24-bit uniforms
        const float u1 = (static_cast<float>(c0 >> 8) + 0.5f) * 0x1p-24f, u2 = (static_cast<float>(c1 >> 8) + 0.5f) * 0x1p-24f;
        v = scale * sqrtf(-2.f * logf(u1)) * cosf(6.2831853f * u2);
    }
    params[i] = v;
}

}  // namespace

struct FlowState {
    int64_t n = 0, keep_cap = 0;
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    unsigned char *packed = nullptr;
    float *tr_x = nullptr, *tr_lq = nullptr, *tr_f = nullptr;
    int64_t keep = 0;
    int64_t step = 0;
};

void flow_state_delete(FlowState *f) { delete f; }   // its device arrays belong to the context

namespace {
int flow_alloc(fiesta_ctx *c, int64_t keep) {
    FlowState *F = c->flow;
    const int64_t n = (int64_t)c->units.size();
    if (!F) {
        F = new FlowState();
        c->flow = F;
        F->n = n;
        F->params = static_cast<float *>(c->dmalloc(sizeof(float) * n * FL_PARAMS));
        F->grad = static_cast<float *>(c->dmalloc(sizeof(float) * n * FL_PARAMS));
        F->m = static_cast<float *>(c->dmalloc(sizeof(float) * n * FL_PARAMS));
        F->v = static_cast<float *>(c->dmalloc(sizeof(float) * n * FL_PARAMS));
        F->packed = static_cast<unsigned char *>(c->dmalloc(FLP_UNIT_BYTES * n));
        if (!F->params || !F->grad || !F->m || !F->v || !F->packed) return fail(FIESTA_E_NOMEM, "flow: allocation failed");
    }
    if (keep > F->keep_cap) {
        c->dfree(F->tr_x);
        c->dfree(F->tr_lq);
        c->dfree(F->tr_f);
        F->tr_x = static_cast<float *>(c->dmalloc(sizeof(float) * n * keep * MAXD));
        F->tr_lq = static_cast<float *>(c->dmalloc(sizeof(float) * n * keep));
        F->tr_f = static_cast<float *>(c->dmalloc(sizeof(float) * n * keep));
        if (!F->tr_x || !F->tr_lq || !F->tr_f) {
            F->keep_cap = 0;
            return fail(FIESTA_E_NOMEM, "flow: training buffer allocation failed");
        }
        F->keep_cap = keep;
    }
    return FIESTA_OK;
}

size_t flow_sample_smem(int fp32, const SliceInfo &si, int nt) {
    const size_t T = fp32 ? 4 : 8;
    return align16(FLP_UNIT_BYTES) + align16(8 * (si.max_instr + 1)) + align16(T * (si.max_const + 3)) +
           align16(8 * LOGTAB_DOUBLES) + align16(T * MAXD * nt) + align16(T * si.max_slots * nt) +
           align16(4 * nt) + 2 * align16(4 * MAXD * (nt + 4)) + align16(8 * 2 * MAXO * nt) +
           (2 * MAXO * 8 + 8) * 32 + 64;
}

int flow_launch_sample(fiesta_ctx *c, FlowSampleParams &p, int64_t nu, int fp32, const SliceInfo &si) {
    int dev_max = 0, sm_max = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    CUDA_TRY(cudaDeviceGetAttribute(&sm_max, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device));
    // 128-thread blocks (two per SM by registers); when the flow, the program and the
    // slot files leave room for only one such block, 256 threads share one staged flow
    int nt = FL_THREADS;
    size_t sm = flow_sample_smem(fp32, si, nt);
    if (2 * (sm + 1024) > (size_t)sm_max && flow_sample_smem(fp32, si, FL_THREADS_MAX) <= (size_t)dev_max) {
        nt = FL_THREADS_MAX;
        sm = flow_sample_smem(fp32, si, nt);
    }
    if ((int)sm > dev_max) return fail(FIESTA_E_NOMEM, "flow sampler: program too large for shared memory");
    const unsigned blocks = (unsigned)(nu * p.blocks_per_unit);
    if (fp32) {
        CUDA_TRY(cudaFuncSetAttribute(k_flow_sample<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_flow_sample<float><<<blocks, nt, sm, c->stream>>>(p);
    } else {
        CUDA_TRY(cudaFuncSetAttribute(k_flow_sample<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_flow_sample<double><<<blocks, nt, sm, c->stream>>>(p);
    }
    CUDA_TRY(cudaGetLastError());
    return FIESTA_OK;
}

int flow_launch_train(fiesta_ctx *c, FlowTrainParams &tp, int64_t nu) {
    CUDA_TRY(cudaFuncSetAttribute(k_flow_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FLT_SMEM));
    k_flow_train_tc<<<(unsigned)(nu * tp.blocks_per_unit), FLT_THREADS, FLT_SMEM, c->stream>>>(tp);
    CUDA_TRY(cudaGetLastError());
    return FIESTA_OK;
}
}  // namespace

extern "C" {

int fiesta_flow_init(fiesta_ctx *c, uint64_t seed, double init_scale) {
    if (!c || !(init_scale >= 0.0)) return fail(FIESTA_E_INVALID, "fiesta_flow_init: bad arguments");
    int r = flow_alloc(c, 0);
    if (r) return r;
    FlowState *F = c->flow;
    const int64_t n = F->n, total = n * FL_PARAMS;
    k_flow_init<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(F->params, n, (uint32_t)seed, (float)init_scale);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemsetAsync(F->m, 0, sizeof(float) * total, c->stream));
    CUDA_TRY(cudaMemsetAsync(F->v, 0, sizeof(float) * total, c->stream));
    k_flow_pack<<<(unsigned)n, 256, 0, c->stream>>>(F->params, F->packed, 0);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    F->step = 0;
    return FIESTA_OK;
}

int fiesta_flow_params(fiesta_ctx *c, int64_t unit, float *params, int32_t set) {
    if (!c || !c->flow || !params || unit < 0 || unit >= (int64_t)c->units.size())
        return fail(FIESTA_E_INVALID, "fiesta_flow_params: bad arguments (call fiesta_flow_init first)");
    FlowState *F = c->flow;
    if (set) {
        CUDA_TRY(cudaMemcpyAsync(F->params + unit * FL_PARAMS, params, sizeof(float) * FL_PARAMS, cudaMemcpyHostToDevice,
                                 c->stream));
        k_flow_pack<<<1, 256, 0, c->stream>>>(F->params, F->packed, unit);
        CUDA_TRY(cudaGetLastError());
    } else {
        CUDA_TRY(cudaMemcpyAsync(params, F->params + unit * FL_PARAMS, sizeof(float) * FL_PARAMS, cudaMemcpyDeviceToHost,
                                 c->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FIESTA_OK;
}

int fiesta_flow_sample(fiesta_ctx *c, int64_t unit_begin, int64_t unit_end, int64_t points, uint64_t seed,
                       int32_t iteration, int32_t precision, int64_t keep, double *mean, double *var,
                       fiesta_stats *stats) {
    if (!c || !c->flow || !mean || !var) return fail(FIESTA_E_INVALID, "fiesta_flow_sample: bad arguments (init first)");
    const int64_t total = (int64_t)c->units.size();
    if (unit_begin < 0 || unit_end > total || unit_begin >= unit_end || points < 2 || keep < 0 || keep > points)
        return fail(FIESTA_E_INVALID, "fiesta_flow_sample: bad unit range, point count or keep");
    if (precision != FIESTA_FP64 && precision != FIESTA_FP32)
        return fail(FIESTA_E_INVALID, "fiesta_flow_sample: precision must be FP64 or FP32");
    int r = flow_alloc(c, keep);
    if (r) return r;
    FlowState *F = c->flow;
    const int64_t nu = unit_end - unit_begin;
    // blocks of about 8192 points each: enough blocks that units of very different
    // program length balance over the SMs (the flow and program are staged per block)
    const int64_t bpu = std::max<int64_t>(1, (points + 8191) / 8192);
    const SliceInfo si = slice_info(c, unit_begin, unit_end);
    const int ostride = si.max_out;
    r = ensure_buffers(c, nu * bpu, nu, 1, ostride);
    if (r) return r;
    FlowSampleParams p{};
    p.units = c->d_units;
    p.pre = c->d_pre;
    p.cons64 = c->d_cons64;
    p.cons32 = c->d_cons32;
    p.logtab = c->d_logtab;
    p.packed = F->packed;
    p.part_sv = c->d_part_sv;
    p.part_sv2 = c->d_part_sv2;
    p.part_bad = c->d_part_bad;
    p.unit_begin = unit_begin;
    p.blocks_per_unit = bpu;
    p.points = points;
    p.seed = (uint32_t)seed;
    p.iteration = (uint32_t)iteration;
    p.max_instr = si.max_instr;
    p.max_const = si.max_const;
    p.max_slots = si.max_slots;
    p.keep = keep;
    p.tr_x = F->tr_x;
    p.tr_lq = F->tr_lq;
    p.tr_f = F->tr_f;
    p.out_stride = ostride;
    if (keep > 0) F->keep = keep;
    EventPair evp;
    if (int r0 = evp.create()) return r0;
    cudaEvent_t e0 = evp.a, e1 = evp.b;
    CUDA_TRY(cudaEventRecord(e0, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->d_unit_bad, 0, sizeof(unsigned long long) * nu, c->stream));
    r = flow_launch_sample(c, p, nu, precision == FIESTA_FP32, si);
    if (r) return r;
    const unsigned rbo = (unsigned)((nu * ostride * 32 + 255) / 256);
    k_reduce<<<rbo, 256, 0, c->stream>>>(c->d_part_sv, c->d_part_sv2, c->d_part_bad, nu, bpu, points, 1, 0,
                                          c->d_iter_mean, c->d_iter_var, c->d_unit_bad, c->d_units, nullptr,
                                          unit_begin, ostride);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventRecord(e1, c->stream));
    std::vector<unsigned long long> bad(nu);
    std::vector<double> hm(nu * ostride), hv(nu * ostride);
    CUDA_TRY(cudaMemcpyAsync(hm.data(), c->d_iter_mean, sizeof(double) * nu * ostride, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(hv.data(), c->d_iter_var, sizeof(double) * nu * ostride, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(bad.data(), c->d_unit_bad, sizeof(unsigned long long) * nu, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    int64_t rec = 0;                       // one record per result, in unit order
    for (int64_t k = 0; k < nu; ++k)
        for (int o = 0; o < c->units[unit_begin + k].n_out; ++o, ++rec) {
            mean[rec] = hm[k * ostride + o];
            var[rec] = hv[k * ostride + o];
        }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->gpu_ms = ms;
        stats->eval_ms = ms;
        stats->points = points * nu;
        stats->points_per_s = ms > 0 ? points * nu / (ms * 1e-3) : 0.0;
        stats->kernels_launched = 2;
        stats->eval_launches = 1;
    }
    for (int64_t k = 0; k < nu; ++k)
        if (bad[k]) return fail(FIESTA_E_NONFINITE, "unit " + std::to_string(unit_begin + k) + " produced non-finite samples");
    return FIESTA_OK;
}

int fiesta_flow_train(fiesta_ctx *c, int64_t unit_begin, int64_t unit_end, int32_t steps, double lr, int32_t power,
                      double *loss, fiesta_stats *stats) {
    if (!c || !c->flow || steps < 1 || !(lr > 0) || (power != 1 && power != 2))
        return fail(FIESTA_E_INVALID, "fiesta_flow_train: bad arguments");
    FlowState *F = c->flow;
    const int64_t total = (int64_t)c->units.size();
    if (unit_begin < 0 || unit_end > total || unit_begin >= unit_end || F->keep < 32)
        return fail(FIESTA_E_INVALID, "fiesta_flow_train: bad unit range or no training points kept");
    const int64_t nu = unit_end - unit_begin;
    double *d_wsum = static_cast<double *>(c->dmalloc(sizeof(double) * nu));
    double *d_loss = static_cast<double *>(c->dmalloc(sizeof(double) * nu));
    if (!d_wsum || !d_loss) {
        c->dfree(d_wsum);
        c->dfree(d_loss);
        return fail(FIESTA_E_NOMEM, "fiesta_flow_train: allocation failed");
    }
    EventPair evp;
    if (int r0 = evp.create()) {
        c->dfree(d_wsum);
        c->dfree(d_loss);
        return r0;
    }
    cudaEvent_t e0 = evp.a, e1 = evp.b;
    cudaEventRecord(e0, c->stream);
    int rc = FIESTA_OK;
    k_flow_wsum<<<(unsigned)nu, 128, 0, c->stream>>>(F->tr_lq, F->tr_f, F->keep, power, unit_begin, d_wsum);
    FlowTrainParams tp{};
    tp.units = c->d_units;
    tp.params = F->params;
    tp.grad = F->grad;
    tp.tr_x = F->tr_x;
    tp.tr_lq = F->tr_lq;
    tp.tr_f = F->tr_f;
    tp.wsum = d_wsum;
    tp.loss = d_loss;
    tp.unit_begin = unit_begin;
    tp.keep = F->keep;
    // about two blocks per SM over the slice (one resident at a time: 219 KB of shared
    // memory), at least 256 training points per block
    tp.blocks_per_unit = std::max<int64_t>(1, std::min<int64_t>((F->keep + 255) / 256, (2 * c->n_sm + nu - 1) / nu));
    tp.buf_unit0 = unit_begin;
    tp.power = power;
    const int64_t np = nu * FL_PARAMS;
    int launches = 1;
    for (int st = 0; st < steps && rc == FIESTA_OK; ++st) {
        cudaMemsetAsync(F->grad + unit_begin * FL_PARAMS, 0, sizeof(float) * np, c->stream);
        cudaMemsetAsync(d_loss, 0, sizeof(double) * nu, c->stream);
        rc = flow_launch_train(c, tp, nu);
        if (rc) break;
        ++F->step;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)F->step), c2 = 1.f - powf(b2, (float)F->step);
        k_flow_adam<<<(unsigned)((np + 255) / 256), 256, 0, c->stream>>>(F->params + unit_begin * FL_PARAMS,
                                                                         F->grad + unit_begin * FL_PARAMS,
                                                                         F->m + unit_begin * FL_PARAMS,
                                                                         F->v + unit_begin * FL_PARAMS, np, (float)lr,
                                                                         b1, b2, 1e-8f, c1, c2);
        launches += 2;
    }
    if (rc == FIESTA_OK) {
        k_flow_pack<<<(unsigned)nu, 256, 0, c->stream>>>(F->params, F->packed, unit_begin);
        ++launches;
        cudaEventRecord(e1, c->stream);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, d_loss, sizeof(double) * nu, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = fail(FIESTA_E_CUDA, std::string("fiesta_flow_train: ") + cudaGetErrorString(e));
    }
    float ms = 0.f;
    if (rc == FIESTA_OK) cudaEventElapsedTime(&ms, e0, e1);
    if (stats && rc == FIESTA_OK) {
        std::memset(stats, 0, sizeof(*stats));
        stats->gpu_ms = ms;
        stats->kernels_launched = launches;
    }
    c->dfree(d_wsum);
    c->dfree(d_loss);
    return rc;
}

int fiesta_flow_check(fiesta_ctx *c, int64_t unit, int64_t n, int32_t precision, const double *z, double *x,
                      double *logq, double *f, const double *w, double *logq_train, double *loss, float *grad) {
    if (!c || !c->flow || unit < 0 || unit >= (int64_t)c->units.size() || n < 1 || !z || !x || !logq || !f || !w ||
        !logq_train || !loss || !grad)
        return fail(FIESTA_E_INVALID, "fiesta_flow_check: bad arguments");
    FlowState *F = c->flow;
    const int d = c->units[unit].dim;
    const int64_t npad = (n + 127) / 128 * 128;
    double *dz = static_cast<double *>(c->dmalloc(sizeof(double) * npad * d));
    double *dx = static_cast<double *>(c->dmalloc(sizeof(double) * npad * d));
    double *dl = static_cast<double *>(c->dmalloc(sizeof(double) * npad));
    double *df = static_cast<double *>(c->dmalloc(sizeof(double) * npad));
    double *dw = static_cast<double *>(c->dmalloc(sizeof(double) * npad));
    double *dlt = static_cast<double *>(c->dmalloc(sizeof(double) * npad));
    double *dloss = static_cast<double *>(c->dmalloc(sizeof(double)));
    double *da = static_cast<double *>(c->dmalloc(sizeof(double) * npad * d));
    float *dtx = static_cast<float *>(c->dmalloc(sizeof(float) * npad * MAXD));
    int rc = FIESTA_OK;
    if (!dz || !dx || !dl || !df || !dw || !dlt || !dloss || !dtx || !da)
        rc = fail(FIESTA_E_NOMEM, "fiesta_flow_check: allocation");
    std::vector<float> hx(npad * MAXD, 0.f);
    std::vector<double> hw(npad, 0.0);
    cudaStream_t s = c->stream;
    if (rc == FIESTA_OK) {
        if (cudaMemcpyAsync(dz, z, sizeof(double) * n * d, cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = fail(FIESTA_E_CUDA, "fiesta_flow_check: copy");
    }
    int r = rc ? rc : ensure_buffers(c, 1, 1, 1, c->units[unit].n_out);
    if (rc == FIESTA_OK && r) rc = r;
    if (rc == FIESTA_OK) {
        const SliceInfo si = slice_info(c, unit, unit + 1);
        FlowSampleParams p{};
        p.out_stride = c->units[unit].n_out;
        p.units = c->d_units;
        p.pre = c->d_pre;
        p.cons64 = c->d_cons64;
        p.cons32 = c->d_cons32;
        p.logtab = c->d_logtab;
        p.packed = F->packed;
        p.part_sv = c->d_part_sv;
        p.part_sv2 = c->d_part_sv2;
        p.part_bad = c->d_part_bad;
        p.unit_begin = unit;
        p.blocks_per_unit = 1;
        p.points = n;
        p.max_instr = si.max_instr;
        p.max_const = si.max_const;
        p.max_slots = si.max_slots;
        p.z_in = dz;
        p.x_out = dx;
        p.lq_out = dl;
        p.f_out = df;
        p.a_out = da;
        rc = flow_launch_sample(c, p, 1, precision == FIESTA_FP32, si);
    }
    // the training pass on the caller's x (given by the sampler's own outputs below) and weights
    if (rc == FIESTA_OK) {
        for (int64_t i = 0; i < n; ++i) hw[i] = w[i];
        cudaMemcpyAsync(dw, hw.data(), sizeof(double) * npad, cudaMemcpyHostToDevice, s);
        std::vector<double> hxs(n * d);
        if (cudaMemcpyAsync(hxs.data(), da, sizeof(double) * n * d, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = fail(FIESTA_E_CUDA, "fiesta_flow_check: copy back");
        for (int64_t i = 0; i < n && rc == FIESTA_OK; ++i)
            for (int j = 0; j < d; ++j) hx[i * MAXD + j] = static_cast<float>(hxs[i * d + j]);
    }
    if (rc == FIESTA_OK) {
        cudaMemcpyAsync(dtx, hx.data(), sizeof(float) * npad * MAXD, cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(F->grad + unit * FL_PARAMS, 0, sizeof(float) * FL_PARAMS, s);
        cudaMemsetAsync(dloss, 0, sizeof(double), s);
        FlowTrainParams tp{};
        tp.units = c->d_units;
        tp.params = F->params;
        tp.grad = F->grad;
        tp.tr_x = dtx;
        tp.w_in = dw;
        tp.loss = dloss;
        tp.lq_out = dlt;
        tp.unit_begin = unit;
        tp.keep = n;
        tp.blocks_per_unit = 1;
        tp.buf_unit0 = 0;
        tp.power = 1;
        rc = flow_launch_train(c, tp, 1);
    }
    if (rc == FIESTA_OK) {
        cudaError_t e = cudaMemcpyAsync(x, dx, sizeof(double) * n * d, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(logq, dl, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(f, df, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(logq_train, dlt, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(grad, F->grad + unit * FL_PARAMS, sizeof(float) * FL_PARAMS, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(FIESTA_E_CUDA, std::string("fiesta_flow_check: ") + cudaGetErrorString(e));
    } else {
        cudaStreamSynchronize(s);
    }
    for (void *ptr : {(void *)dz, (void *)dx, (void *)dl, (void *)df, (void *)dw, (void *)dlt, (void *)dloss, (void *)dtx,
                      (void *)da})
        c->dfree(ptr);
    return rc;
}

}  // extern "C"
