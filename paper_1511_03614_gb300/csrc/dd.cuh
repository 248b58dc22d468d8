// dd.cuh -- double-double arithmetic and the bytecode interpreter over it; included
// by fiesta.cu after the binary64 interpreter.
//
// A value is hi + lo with hi = round(hi + lo) (about 106 significant bits).  It
// is the extended precision used for points near the boundary of the cube,
// where the subtraction terms of a sector integrand cancel and binary64 loses
// digits: the counterpart of the paper's MPFR mixed mode (Sec. 4.6, MPFR /
// Native / Mixed), with double-double in place of MPFR.
//
// Building blocks (all published): Knuth's TwoSum and Dekker's FastTwoSum for
// exact sums, the exact product a*b = p + fma(a, b, -p); addition with both
// error terms (the "accurate" sum); division by three steps of long division;
// exp by reduction to r = a - k ln2, scaling by 2^-10, the Taylor series of
// expm1 to degree 9 and ten doublings expm1(2s) = expm1(s) (expm1(s) + 2);
// log by one Newton step y = y0 + a exp(-y0) - 1 from the binary64 logarithm
// y0, which doubles the number of correct digits (near a = 1 in a form whose
// error is relative to log a).

struct ddv {
    double hi, lo;
};

__device__ __forceinline__ ddv dd_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ddv dd_fast_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}

__device__ __forceinline__ ddv dd_add(ddv a, ddv b) {
    ddv s = dd_two_sum(a.hi, b.hi);
    const ddv t = dd_two_sum(a.lo, b.lo);
    s.lo = __dadd_rn(s.lo, t.hi);
    s = dd_fast_two_sum(s.hi, s.lo);
    s.lo = __dadd_rn(s.lo, t.lo);
    return dd_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ddv dd_add_d(ddv a, double b) {
    ddv s = dd_two_sum(a.hi, b);
    s.lo = __dadd_rn(s.lo, a.lo);
    return dd_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ddv dd_neg(ddv a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ ddv dd_sub(ddv a, ddv b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ ddv dd_mul(ddv a, ddv b) {
    const double p = __dmul_rn(a.hi, b.hi);
    double e = fma(a.hi, b.hi, -p);
    e = fma(a.hi, b.lo, e);
    e = fma(a.lo, b.hi, e);
    return dd_fast_two_sum(p, e);
}

__device__ __forceinline__ ddv dd_mul_d(ddv a, double b) {
    const double p = __dmul_rn(a.hi, b);
    double e = fma(a.hi, b, -p);
    e = fma(a.lo, b, e);
    return dd_fast_two_sum(p, e);
}

__device__ __noinline__ ddv dd_div(ddv a, ddv b) {
    const double q1 = a.hi / b.hi;
    ddv r = dd_sub(a, dd_mul_d(b, q1));
    const double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul_d(b, q2));
    const double q3 = r.hi / b.hi;
    return dd_add_d(dd_fast_two_sum(q1, q2), q3);
}

// a / b for a binary64 b
__device__ __forceinline__ ddv dd_div_d(ddv a, double b) {
    const double q1 = a.hi / b;
    const double p = __dmul_rn(q1, b);
    const double pe = fma(q1, b, -p);
    ddv r = dd_two_sum(a.hi, -p);
    r.lo = __dadd_rn(__dsub_rn(r.lo, pe), a.lo);
    const double q2 = __dadd_rn(r.hi, r.lo) / b;
    return dd_fast_two_sum(q1, q2);
}

__device__ __forceinline__ ddv dd_ldexp(ddv a, int k) { return {ldexp(a.hi, k), ldexp(a.lo, k)}; }

constexpr double DD_LN2_HI = 0x1.62e42fefa39efp-1;     // ln 2 = hi + lo to 106 bits
constexpr double DD_LN2_LO = 0x1.abc9e3b39803fp-56;

// exp(a) = 2^k (1 + e): returns e = expm1(a - k ln2) and k (|a - k ln2| <= ln2 / 2)
__device__ __noinline__ ddv dd_expm1_reduced(ddv a, int &k) {
    const double kd = rint(a.hi / DD_LN2_HI);
    k = static_cast<int>(kd);
    ddv r = dd_sub(a, dd_mul_d(ddv{DD_LN2_HI, DD_LN2_LO}, kd));
    r = dd_ldexp(r, -10);                                  // |r| <= ln2 / 2^11
    ddv t = dd_add_d(dd_div_d(r, 9.0), 1.0);               // 1 + r/9
    for (int m = 8; m >= 2; --m) t = dd_add_d(dd_mul(dd_div_d(r, (double)m), t), 1.0);
    ddv e = dd_mul(r, t);                                  // expm1(r 2^-10)
    for (int i = 0; i < 10; ++i) e = dd_mul(e, dd_add_d(e, 2.0));
    return e;
}

__device__ ddv dd_exp(ddv a) {
    if (!(a.hi == a.hi)) return {a.hi, 0.0};
    if (a.hi > 709.78) return {INFINITY, 0.0};
    if (a.hi < -745.2) return {0.0, 0.0};
    int k = 0;
    const ddv e = dd_expm1_reduced(a, k);
    return dd_ldexp(dd_add_d(e, 1.0), k);
}

// log by one Newton step on exp from y0 = log(hi): y = y0 + (a exp(-y0) - 1).  Near
// a = 1 the correction is formed as t + m + t m with t = a - 1 (exact) and
// m = expm1(-y0), so that its error stays relative to log(a) and not to 1.
__device__ __noinline__ ddv dd_log(ddv a) {
    if (!(a.hi > 0.0) || isinf(a.hi)) return {log(a.hi), 0.0};
    if (a.hi > 0.5 && a.hi < 1.5) {
        const ddv t = dd_add_d(a, -1.0);
        const double y0 = log1p(t.hi);
        int k = 0;
        ddv m = dd_expm1_reduced(ddv{-y0, 0.0}, k);
        if (k != 0) m = dd_add_d(dd_ldexp(dd_add_d(m, 1.0), k), -1.0);
        const ddv d = dd_add(dd_add(t, m), dd_mul(t, m));
        return dd_add_d(d, y0);
    }
    double shift = 0.0;                                    // keep exp(-y0) in range
    if (a.hi < 0x1p-960) {
        a = dd_ldexp(a, 960);
        shift = -960.0;
    } else if (a.hi > 0x1p+960) {
        a = dd_ldexp(a, -960);
        shift = 960.0;
    }
    const double y0 = log(a.hi);
    const ddv r = dd_add_d(dd_mul(a, dd_exp(ddv{-y0, 0.0})), -1.0);
    ddv y = dd_add_d(r, y0);
    if (shift != 0.0) y = dd_add(y, dd_mul_d(ddv{DD_LN2_HI, DD_LN2_LO}, shift));
    return y;
}

__device__ __forceinline__ ddv dd_powi(ddv a, int n) {
    unsigned m = n < 0 ? static_cast<unsigned>(-n) : static_cast<unsigned>(n);
    ddv r{1.0, 0.0}, b = a;
    while (m) {
        if (m & 1u) r = dd_mul(r, b);
        m >>= 1;
        if (m) b = dd_mul(b, b);
    }
    return n < 0 ? dd_div(ddv{1.0, 0.0}, r) : r;
}

// The bytecode interpreter in double-double: the high parts live in the caller's
// shared-memory slot file (so the results sit where the binary64 interpreter puts
// them, rounded to binary64), the low parts in a per-thread array.  Opcode 16
// (ATAN2, complex units) has no double-double form; callers reject such programs.
constexpr int DD_MAX_SLOTS = 256;

__device__ __noinline__ void interpret_dd(const uint32_t *__restrict__ code, int n, const double *__restrict__ cons,
                                          double *__restrict__ S, const double *__restrict__ X, int stride) {
    double lo[DD_MAX_SLOTS];
    for (int pc = 0; pc < n; ++pc) {
        const uint32_t w = code[pc];
        const int op = w & 0xffu;
        const int d = (w >> 8) & 0xffu;
        const int a = (w >> 16) & 0xffu;
        const int b = w >> 24;
        auto slot = [&](int i) { return ddv{S[i * stride], lo[i]}; };
        ddv r;
        switch (op) {
        case 1: r = ddv{X[a * stride], 0.0}; break;
        case 2: r = ddv{cons[a | (b << 8)], 0.0}; break;
        case 3: r = dd_add(slot(a), slot(b)); break;
        case 4: r = dd_sub(slot(a), slot(b)); break;
        case 5: r = dd_mul(slot(a), slot(b)); break;
        case 6: r = dd_div(slot(a), slot(b)); break;
        case 7: r = dd_neg(slot(a)); break;
        case 8: r = dd_add(dd_mul(slot(a), slot(b)), slot(d)); break;
        case 9: r = dd_add_d(slot(a), cons[b]); break;
        case 10: r = dd_mul_d(slot(a), cons[b]); break;
        case 11: r = dd_add(dd_mul_d(slot(a), cons[b]), slot(d)); break;
        case 12: r = dd_powi(slot(a), static_cast<int>(static_cast<int8_t>(b))); break;
        case 13: r = dd_log(slot(a)); break;
        case 14: r = dd_div(ddv{1.0, 0.0}, slot(a)); break;
        case 15: r = slot(a); break;
        default: r = ddv{NAN, 0.0}; break;
        }
        S[d * stride] = r.hi;
        lo[d] = r.lo;
    }
}
