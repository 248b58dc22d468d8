// Micro-op form of a program for the evaluation kernels (included by fiesta.cu).
//
// Every opcode except the special functions is one fused multiply-add of three operands:
//   ADD a*1 + b   SUB b*(-1) + a   MUL a*b + z   NEG a*(-1) + z   MAC a*b + d
//   ADDC a*1 + c  MULC a*c + z     MACC a*c + d
// with z = -0.0 (x + (-0) = x for every x, signed zeros included), so each result is
// bit-identical to the operation it replaces.  The copies LDX (coordinate to slot) and
// LDC (constant to slot) execute nothing: the loader forwards their source to the
// readers of the slot (forward_program), so an operand may name a coordinate or a
// constant directly.  A MOV whose slot the next instruction overwrites (the emitter's
// copy of a multiply-add's accumulator) is forwarded into that instruction, so MOV then
// MAC becomes one multiply-add into the fresh slot.
//
// Host form ("forwarded program", one 64-bit word per executed instruction):
//   bits 0-7 opcode, 8-15 destination slot, 16-31 / 32-47 / 48-63 operand references
//   X, Y, Z: the multiply-add's operands in order, or for DIV, POWI, LOG, INV, ATAN2 the
//   first and second operand (POWI: Y is the exponent byte).  A reference below
//   REF_SLOT is a constant index; REF_SLOT + s slot s; REF_X + j coordinate j;
//   REF_FIXED + k the fixed constants -0, 1, -1.
// Device form (staged per block): four 16-bit element indices (X, Y, Z, D) into the
// block's shared memory viewed as an array of T; an index at or above `pt` (the start of
// the per-thread region: coordinates and slot file, laid out [index][thread]) is offset
// by the thread index.  A special function has X = UOP_SPECIAL | opcode, Y the second
// operand's index (POWI: the exponent byte), Z the first operand's, D the destination.

constexpr uint32_t REF_SLOT = 0xC000u, REF_X = 0xD000u, REF_FIXED = 0xE000u;
constexpr uint32_t FIX_ZERO = REF_FIXED, FIX_ONE = REF_FIXED + 1u, FIX_MONE = REF_FIXED + 2u;
constexpr int32_t MAX_FORWARD_CONST = static_cast<int32_t>(REF_SLOT);
constexpr uint32_t UOP_SPECIAL = 0xFF00u;     // element indices stay below it (at most 58 112)

inline bool is_special_op(int op) { return op == 6 || op == 12 || op == 13 || op == 14 || op == 16; }

inline uint64_t pre_uop(int op, int d, uint32_t x, uint32_t y, uint32_t z) {
    return static_cast<uint64_t>(op) | (static_cast<uint64_t>(d) << 8) | (static_cast<uint64_t>(x) << 16) |
           (static_cast<uint64_t>(y) << 32) | (static_cast<uint64_t>(z) << 48);
}

// The forwarded program of a validated program (appended to out).  alias[s] is where
// the value of slot s lives: its own slot, a coordinate or a constant (these never
// change, so an alias to them stays valid until s is written again).  A MOV is
// forwarded only into the instruction right after it when that one writes the same slot
// (the emitter's copy of a multiply-add's accumulator), so no alias ever names another
// slot; any other MOV is executed as a copy.  At the end every result is settled in its
// slot.  The form is never longer than the program.  Returns the number of words, or -1
// when the program has more constants than a reference can name.
inline int64_t forward_program(const fiesta_program &p, std::vector<uint64_t> &out) {
    if (p.n_const > MAX_FORWARD_CONST) return -1;
    const size_t start = out.size();
    std::vector<uint32_t> alias(p.n_slots);
    for (int s = 0; s < p.n_slots; ++s) alias[s] = REF_SLOT + s;
    auto dest = [](uint32_t w) { return static_cast<int>((w >> 8) & 0xffu); };
    for (int64_t i = 0; i < p.n_instr; ++i) {
        const uint32_t w = p.code[i];
        const int op = w & 0xffu, d = dest(w), a = (w >> 16) & 0xffu, b = w >> 24;
        if (op == 1) {                                    // LDX
            alias[d] = REF_X + a;
            continue;
        }
        if (op == 2) {                                    // LDC
            alias[d] = static_cast<uint32_t>(a | (b << 8));
            continue;
        }
        if (op == 15) {                                   // MOV
            const uint32_t src = alias[a];
            if (i + 1 < p.n_instr && dest(p.code[i + 1]) == d && (p.code[i + 1] & 0xffu) != 15u) {
                alias[d] = src;                           // read once, by the next instruction
            } else {
                out.push_back(pre_uop(15, d, src, FIX_ONE, FIX_ZERO));
                alias[d] = REF_SLOT + d;
            }
            continue;
        }
        const uint32_t ra = alias[a];
        const uint32_t rb = (op == 3 || op == 4 || op == 5 || op == 6 || op == 8 || op == 16) ? alias[b] : 0u;
        const uint32_t rd = (op == 8 || op == 11) ? alias[d] : 0u;
        uint64_t u;
        switch (op) {
        case 3: u = pre_uop(op, d, ra, FIX_ONE, rb); break;
        case 4: u = pre_uop(op, d, rb, FIX_MONE, ra); break;
        case 5: u = pre_uop(op, d, ra, rb, FIX_ZERO); break;
        case 7: u = pre_uop(op, d, ra, FIX_MONE, FIX_ZERO); break;
        case 8: u = pre_uop(op, d, ra, rb, rd); break;
        case 9: u = pre_uop(op, d, ra, FIX_ONE, static_cast<uint32_t>(b)); break;
        case 10: u = pre_uop(op, d, ra, static_cast<uint32_t>(b), FIX_ZERO); break;
        case 11: u = pre_uop(op, d, ra, static_cast<uint32_t>(b), rd); break;
        case 12: u = pre_uop(op, d, ra, static_cast<uint32_t>(b), 0u); break;
        default: u = pre_uop(op, d, ra, rb, 0u); break;  // DIV, LOG, INV, ATAN2
        }
        out.push_back(u);
        alias[d] = REF_SLOT + d;
    }
    auto settle = [&](int o) {
        if (alias[o] != REF_SLOT + static_cast<uint32_t>(o)) {
            out.push_back(pre_uop(15, o, alias[o], FIX_ONE, FIX_ZERO));
            alias[o] = REF_SLOT + o;
        }
    };
    if (p.n_out > 1)
        for (int k = 0; k < p.n_out; ++k) settle(p.out_slots[k]);
    else
        settle(p.out_slot);
    return static_cast<int64_t>(out.size() - start);
}

// Device form of one forwarded word for a block whose shared memory holds the constants
// at cons_base (then -0, 1, -1 at k_zero), the coordinates at pt and the slot file at
// slot_base, each per-thread row nt elements long.
__device__ __forceinline__ uint64_t uop_from_pre(uint64_t pre, int cons_base, int k_zero, int pt, int slot_base,
                                                 int nt) {
    const uint32_t op = static_cast<uint32_t>(pre) & 0xffu, d = static_cast<uint32_t>(pre >> 8) & 0xffu;
    const uint32_t x = static_cast<uint32_t>(pre >> 16) & 0xffffu, y = static_cast<uint32_t>(pre >> 32) & 0xffffu,
                   z = static_cast<uint32_t>(pre >> 48);
    auto ref = [&](uint32_t r) -> uint64_t {
        if (r < REF_SLOT) return static_cast<uint64_t>(cons_base + static_cast<int>(r));
        if (r < REF_X) return static_cast<uint64_t>(slot_base + static_cast<int>(r - REF_SLOT) * nt);
        if (r < REF_FIXED) return static_cast<uint64_t>(pt + static_cast<int>(r - REF_X) * nt);
        return static_cast<uint64_t>(k_zero + static_cast<int>(r - REF_FIXED));
    };
    const uint64_t D = static_cast<uint64_t>(slot_base + static_cast<int>(d) * nt);
    if (op == 6u || op == 12u || op == 13u || op == 14u || op == 16u)
        return (UOP_SPECIAL | op) | ((op == 12u ? y : ref(y)) << 16) | (ref(x) << 32) | (D << 48);
    return ref(x) | (ref(y) << 16) | (ref(z) << 32) | (D << 48);
}

// A special function: a and b are element indices of the operands (b: the exponent of
// POWI), d the destination's.
template <typename T>
__device__ __noinline__ void exec_special(uint32_t op, uint32_t a, uint32_t b, uint32_t d, T *E, uint32_t pt, int tid,
                                          const double *__restrict__ logtab) {
    const T va = E[a + (a >= pt ? tid : 0)];
    T r;
    switch (op) {
    case 6: r = va / E[b + (b >= pt ? tid : 0)]; break;
    case 12: r = dev_powi<T>(va, static_cast<int>(static_cast<int8_t>(b & 0xffu))); break;
    case 13: r = interp_log<T>(va, logtab); break;
    case 14: r = dev_recip<T>(va); break;
    case 16: r = dev_atan2<T>(va, E[b + (b >= pt ? tid : 0)]); break;
    default: r = T(0); break;
    }
    E[d + tid] = r;
}

// E: shared memory as T; uops: n + 1 words (the last one is fetched, never executed).
template <typename T>
__device__ __forceinline__ void interpret_uop(const uint64_t *__restrict__ uops, int n, T *E, int pt, int tid,
                                              const double *__restrict__ logtab) {
    const uint32_t upt = static_cast<uint32_t>(pt);
    uint64_t w = uops[0];
    for (int pc = 0; pc < n; ++pc) {
        const uint64_t wn = uops[pc + 1];
        const uint32_t xi = static_cast<uint32_t>(w) & 0xffffu;
        const uint32_t yi = static_cast<uint32_t>(w >> 16) & 0xffffu;
        const uint32_t zi = static_cast<uint32_t>(w >> 32) & 0xffffu;
        const uint32_t di = static_cast<uint32_t>(w >> 48);
        if (xi < UOP_SPECIAL) {
            const uint32_t xa = xi + (xi >= upt ? tid : 0);
            const uint32_t ya = yi + (yi >= upt ? tid : 0);
            const uint32_t za = zi + (zi >= upt ? tid : 0);
            E[di + tid] = dev_fma<T>(E[xa], E[ya], E[za]);
        } else {
            exec_special<T>(xi & 0xffu, zi, yi, di, E, upt, tid, logtab);
        }
        w = wn;
    }
}
