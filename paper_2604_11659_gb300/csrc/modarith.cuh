// Device-side 64-bit modular arithmetic for moduli q < 2^62 on the INT32 pipes.
//
//  * Shoup multiplication by a constant w with precomputed w' = floor(w 2^64 / q):
//    x*w - floor(x*w'/2^64)*q lies in [0, 2q) for any x < 2^64.
//  * Montgomery reduction (R = 2^64) of a 128-bit T < q*2^64:
//    REDC(T) = T R^{-1} mod q, using q' = -q^{-1} mod 2^64.
//    Products with one operand stored as w*R mod q reduce straight to x*w mod q.
#pragma once
#include <cstdint>

typedef unsigned long long u64;

struct U128 {
    u64 lo, hi;
};

__device__ __forceinline__ U128 mul_wide(u64 a, u64 b)
{
    U128 r;
    r.lo = a * b;
    r.hi = __umul64hi(a, b);
    return r;
}

__device__ __forceinline__ void add_wide(U128 &acc, U128 x)
{
    u64 lo = acc.lo + x.lo;
    acc.hi += x.hi + (lo < x.lo ? 1ull : 0ull);
    acc.lo = lo;
}

// acc += a * b (128-bit), one carry chain
__device__ __forceinline__ void mac_wide(U128 &acc, u64 a, u64 b)
{
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\tmadc.hi.u64 %1, %2, %3, %1;"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(a), "l"(b));
}

// x in [0, 2q) -> [0, q)
__device__ __forceinline__ u64 csub(u64 x, u64 q) { return x >= q ? x - q : x; }

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) { return csub(a + b, q); }

__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

__device__ __forceinline__ u64 neg_mod(u64 a, u64 q) { return a ? q - a : 0; }

// Shoup: x * w mod q, result in [0, q)
__device__ __forceinline__ u64 mul_shoup(u64 x, u64 w, u64 wp, u64 q)
{
    u64 h = __umul64hi(x, wp);
    u64 r = x * w - h * q;
    return csub(r, q);
}

// Shoup without the final correction: result in [0, 2q)
__device__ __forceinline__ u64 mul_shoup_lazy(u64 x, u64 w, u64 wp, u64 q)
{
    u64 h = __umul64hi(x, wp);
    return x * w - h * q;
}

// Montgomery reduction of T = (hi, lo) < q * 2^64: returns T * 2^-64 mod q in [0, q)
__device__ __forceinline__ u64 redc(U128 t, u64 q, u64 qneg_inv)
{
    // (t + m q) / 2^64 with m = t.lo * (-q^{-1}): the low word cancels, its
    // carry is taken from the same add chain
    const u64 m = t.lo * qneg_inv;
    u64 r;
    asm("{\n\t.reg .u64 lo_;\n\tmad.lo.cc.u64 lo_, %1, %2, %3;\n\tmadc.hi.u64 %0, %1, %2, %4;\n\t}"
        : "=l"(r)
        : "l"(m), "l"(q), "l"(t.lo), "l"(t.hi));
    return csub(r, q);
}

// Per-modulus constants (device copy of the host table).
struct ModConst {
    u64 q;
    u64 qneg_inv;   // -q^{-1} mod 2^64
    u64 r_mod;      // 2^64 mod q      (undoes one REDC factor via Shoup)
    u64 r_mod_p;    // Shoup companion of r_mod
    u64 r2_mod;     // 2^128 mod q     (converts into Montgomery form via REDC)
    u64 n_inv;      // n^{-1} mod q (Shoup pair)
    u64 n_inv_p;
    u64 pad;
};

// a * b mod q for two variable operands (REDC then undo the 2^-64 factor)
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const ModConst &m)
{
    u64 t = redc(mul_wide(a, b), m.q, m.qneg_inv);
    return mul_shoup(t, m.r_mod, m.r_mod_p, m.q);
}

// x -> x * 2^64 mod q (Montgomery form), x < q
__device__ __forceinline__ u64 to_mont(u64 x, const ModConst &m)
{
    return redc(mul_wide(x, m.r2_mod), m.q, m.qneg_inv);
}

// bit reversal of the low `bits` bits
__device__ __forceinline__ unsigned brev_bits(unsigned x, int bits)
{
    return __brev(x) >> (32 - bits);
}
