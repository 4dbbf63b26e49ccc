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

// Shoup multiplication with a truncated quotient: of the four 32x32-bit
// partial products of x * w', the lowest (x0 w'0) is dropped, so the quotient
// estimate is floor(x w' / 2^64) or one less and the result
// x*w - Q'*q mod 2^64 lies in [0, 3q) for any x < 2^64.  Five wide and four
// low 32-bit multiplies in all; nq = 2^64 - q.
__device__ __forceinline__ u64 mul_shoup3(u64 x, u64 w, u64 wp, u64 nq)
{
    u64 r;
    asm("{\n\t"
        ".reg .u32 x0, x1, a0, a1, w0, w1, n0, n1, t0, t1, p0, p1, s1, q0, q1, r0, r1;\n\t"
        ".reg .u64 t, p, s, qq, acc;\n\t"
        "mov.b64 {x0, x1}, %1;\n\t"
        "mov.b64 {a0, a1}, %3;\n\t"
        "mul.wide.u32 t, x1, a0;\n\t"
        "mul.wide.u32 p, x0, a1;\n\t"
        "mov.b64 {t0, t1}, t;\n\t"
        "mov.b64 {p0, p1}, p;\n\t"
        "add.cc.u32 t0, t0, p0;\n\t"
        "addc.cc.u32 t1, t1, p1;\n\t"
        "addc.u32 s1, 0, 0;\n\t"
        "mov.b64 s, {t1, s1};\n\t"
        "mad.wide.u32 qq, x1, a1, s;\n\t"
        "mov.b64 {q0, q1}, qq;\n\t"
        "mov.b64 {w0, w1}, %2;\n\t"
        "mov.b64 {n0, n1}, %4;\n\t"
        "mul.wide.u32 acc, x0, w0;\n\t"
        "mad.wide.u32 acc, q0, n0, acc;\n\t"
        "mov.b64 {r0, r1}, acc;\n\t"
        "mad.lo.u32 r1, x0, w1, r1;\n\t"
        "mad.lo.u32 r1, x1, w0, r1;\n\t"
        "mad.lo.u32 r1, q0, n1, r1;\n\t"
        "mad.lo.u32 r1, q1, n0, r1;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "}"
        : "=l"(r)
        : "l"(x), "l"(w), "l"(wp), "l"(nq));
    return r;
}

// mul_shoup3 with every 32x32 -> 64-bit product taken as its low and high
// halves (mul.lo / mul.hi, carries through the add chain) instead of one
// wide product: the same partial products and the same sums, so the same
// result bit for bit, in fourteen single-word multiplies.  On GB300 a
// product with a 64-bit result occupies the multiply pipe about 2.8 times as
// long as one with a 32-bit result (measured), so this form trades five wide
// products for ten halves.
__device__ __forceinline__ u64 mul_shoup3s(u64 x, u64 w, u64 wp, u64 nq)
{
    u64 r;
    asm("{\n\t"
        ".reg .u32 x0, x1, a0, a1, w0, w1, n0, n1, t0, t1, p0, p1, s1, q0, q1, r0, r1;\n\t"
        "mov.b64 {x0, x1}, %1;\n\t"
        "mov.b64 {a0, a1}, %3;\n\t"
        "mul.lo.u32 t0, x1, a0;\n\t"
        "mul.hi.u32 t1, x1, a0;\n\t"
        "mul.lo.u32 p0, x0, a1;\n\t"
        "mul.hi.u32 p1, x0, a1;\n\t"
        "add.cc.u32 t0, t0, p0;\n\t"
        "addc.cc.u32 t1, t1, p1;\n\t"
        "addc.u32 s1, 0, 0;\n\t"
        "mad.lo.cc.u32 q0, x1, a1, t1;\n\t"
        "madc.hi.u32 q1, x1, a1, s1;\n\t"
        "mov.b64 {w0, w1}, %2;\n\t"
        "mov.b64 {n0, n1}, %4;\n\t"
        "mul.lo.u32 r0, x0, w0;\n\t"
        "mul.hi.u32 r1, x0, w0;\n\t"
        "mad.lo.cc.u32 r0, q0, n0, r0;\n\t"
        "madc.hi.u32 r1, q0, n0, r1;\n\t"
        "mad.lo.u32 r1, x0, w1, r1;\n\t"
        "mad.lo.u32 r1, x1, w0, r1;\n\t"
        "mad.lo.u32 r1, q0, n1, r1;\n\t"
        "mad.lo.u32 r1, q1, n0, r1;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "}"
        : "=l"(r)
        : "l"(x), "l"(w), "l"(wp), "l"(nq));
    return r;
}

// Shoup product whose quotient keeps only the high halves of the two middle
// partial products of x * w': Q' = x1 a1 + hi(x1 a0) + hi(x0 a1).  The
// dropped parts (the two low halves times 2^32, and x0 a0) are each below
// 2^64, so Q' is at most two below floor(x w' / 2^64) and, as
// x*w - floor(x w' / 2^64)*q lies in [0, 2q), the result x*w - Q'*q lies in [0, 4q) for
// any x < 2^64 (q < 2^62).  Twelve single-word multiplies (seven low halves,
// five high halves): two fewer than mul_shoup3s and one carry chain shorter.
__device__ __forceinline__ u64 mul_shoup4s(u64 x, u64 w, u64 wp, u64 nq)
{
    u64 r;
    asm("{\n\t"
        ".reg .u32 x0, x1, a0, a1, w0, w1, n0, n1, h0, h1, q0, q1, r0, r1;\n\t"
        "mov.b64 {x0, x1}, %1;\n\t"
        "mov.b64 {a0, a1}, %3;\n\t"
        "mul.hi.u32 h0, x1, a0;\n\t"
        "mul.hi.u32 h1, x0, a1;\n\t"
        "add.cc.u32 h0, h0, h1;\n\t"
        "addc.u32 h1, 0, 0;\n\t"
        "mad.lo.cc.u32 q0, x1, a1, h0;\n\t"
        "madc.hi.u32 q1, x1, a1, h1;\n\t"
        "mov.b64 {w0, w1}, %2;\n\t"
        "mov.b64 {n0, n1}, %4;\n\t"
        "mul.lo.u32 r0, x0, w0;\n\t"
        "mul.hi.u32 r1, x0, w0;\n\t"
        "mad.lo.cc.u32 r0, q0, n0, r0;\n\t"
        "madc.hi.u32 r1, q0, n0, r1;\n\t"
        "mad.lo.u32 r1, x0, w1, r1;\n\t"
        "mad.lo.u32 r1, x1, w0, r1;\n\t"
        "mad.lo.u32 r1, q0, n1, r1;\n\t"
        "mad.lo.u32 r1, q1, n0, r1;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "}"
        : "=l"(r)
        : "l"(x), "l"(w), "l"(wp), "l"(nq));
    return r;
}

// Butterfly arithmetic of the transform kernels: AR = 0 mul_shoup3 (wide
// partial products), 1 mul_shoup3s (split halves), both with results in
// [0, 3q); AR = 2 mul_shoup4s, results in [0, 4q).
template <int AR> __device__ __forceinline__ u64 mul_shoup_ar(u64 x, u64 w, u64 wp, u64 nq)
{
    if constexpr (AR == 2) return mul_shoup4s(x, w, wp, nq);
    else if constexpr (AR == 1) return mul_shoup3s(x, w, wp, nq);
    else return mul_shoup3(x, w, wp, nq);
}
// multiple of q that bounds mul_shoup_ar<AR>'s result
template <int AR> constexpr u64 shoup_bound() { return AR == 2 ? 4 : 3; }

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

// Carry-free sums of products of operands below 2^60 (base conversions and
// the key-switching inner product).  Each operand is split into 30-bit
// halves x = x1 2^30 + x0, each half product is below 2^60, and the four
// partial-product classes are summed in separate 64-bit words:
//   T = s00 + (s01 + s10) 2^30 + s11 2^60,
// exact for up to 16 terms per word.  A constant stored "split" holds
// x0 in its low 32-bit word and x1 in its high word.
struct Acc30 {
    u64 s00, s01, s10, s11;
};

__device__ __forceinline__ void acc30_zero(Acc30 &a) { a.s00 = a.s01 = a.s10 = a.s11 = 0; }

// a += x * c for x = (x0, x1) and a split constant c
__device__ __forceinline__ void acc30_mac(Acc30 &a, uint32_t x0, uint32_t x1, u64 c)
{
    const uint32_t c0 = (uint32_t)c, c1 = (uint32_t)(c >> 32);
    asm("mad.wide.u32 %0, %4, %6, %0;\n\t"
        "mad.wide.u32 %1, %4, %7, %1;\n\t"
        "mad.wide.u32 %2, %5, %6, %2;\n\t"
        "mad.wide.u32 %3, %5, %7, %3;"
        : "+l"(a.s00), "+l"(a.s01), "+l"(a.s10), "+l"(a.s11)
        : "r"(x0), "r"(x1), "r"(c0), "r"(c1));
}

// a += x * c for a small x < 2^30 (x1 = 0)
__device__ __forceinline__ void acc30_mac_small(Acc30 &a, uint32_t x, u64 c)
{
    const uint32_t c0 = (uint32_t)c, c1 = (uint32_t)(c >> 32);
    asm("mad.wide.u32 %0, %2, %3, %0;\n\t"
        "mad.wide.u32 %1, %2, %4, %1;"
        : "+l"(a.s00), "+l"(a.s01)
        : "r"(x), "r"(c0), "r"(c1));
}

__device__ __forceinline__ void split30(u64 x, uint32_t &x0, uint32_t &x1)
{
    x0 = (uint32_t)x & 0x3fffffffu;
    x1 = (uint32_t)(x >> 30);
}

// The 128-bit value T of an accumulator.
__device__ __forceinline__ U128 acc30_value(const Acc30 &a)
{
    // mid = s01 + s10 as a 65-bit value (carry in mc)
    const u64 mid = a.s01 + a.s10;
    const u64 mc = mid < a.s01 ? 1ull : 0ull;
    U128 t;
    asm("add.cc.u64 %0, %2, %3;\n\t"
        "addc.u64 %1, %4, %5;"
        : "=l"(t.lo), "=l"(t.hi)
        : "l"(a.s00), "l"(mid << 30), "l"(mid >> 34), "l"(a.s11 >> 4));
    asm("add.cc.u64 %0, %0, %2;\n\t"
        "addc.u64 %1, %1, %3;"
        : "+l"(t.lo), "+l"(t.hi)
        : "l"(a.s11 << 60), "l"(mc << 30));
    return t;
}

// The same exact sums with three partial products per term instead of four
// (Karatsuba on the halves): x c = x0 c0 + ((x0 + x1)(c0 + c1) - x0 c0 -
// x1 c1) 2^30 + x1 c1 2^60.  s00 and s11 sum x0 c0 and x1 c1 (each term below
// 2^60: exact for up to 16 terms); the middle products (x0 + x1)(c0 + c1) are
// below 2^62 and are summed into the 128-bit word (mh, m).  The 128-bit value
// T is the same integer as with Acc30, so the reduced result is the same.
struct Acc30K {
    u64 s00, s11, m, mh;
};

__device__ __forceinline__ void acc30k_zero(Acc30K &a) { a.s00 = a.s11 = a.m = a.mh = 0; }

// a += x * c for x = (x0, x1) and a split constant c
__device__ __forceinline__ void acc30k_mac(Acc30K &a, uint32_t x0, uint32_t x1, u64 c)
{
    const uint32_t c0 = (uint32_t)c, c1 = (uint32_t)(c >> 32);
    const uint32_t xs = x0 + x1, cs = c0 + c1;
    asm("{\n\t.reg .u64 t;\n\t"
        "mad.wide.u32 %0, %4, %6, %0;\n\t"
        "mad.wide.u32 %1, %5, %7, %1;\n\t"
        "mul.wide.u32 t, %8, %9;\n\t"
        "add.cc.u64 %2, %2, t;\n\t"
        "addc.u64 %3, %3, 0;\n\t}"
        : "+l"(a.s00), "+l"(a.s11), "+l"(a.m), "+l"(a.mh)
        : "r"(x0), "r"(x1), "r"(c0), "r"(c1), "r"(xs), "r"(cs));
}

// a += x * c for a small x < 2^30 (x1 = 0: the middle product is x (c0 + c1))
__device__ __forceinline__ void acc30k_mac_small(Acc30K &a, uint32_t x, u64 c)
{
    const uint32_t c0 = (uint32_t)c, c1 = (uint32_t)(c >> 32), cs = c0 + c1;
    asm("{\n\t.reg .u64 t;\n\t"
        "mad.wide.u32 %0, %3, %4, %0;\n\t"
        "mul.wide.u32 t, %3, %5;\n\t"
        "add.cc.u64 %1, %1, t;\n\t"
        "addc.u64 %2, %2, 0;\n\t}"
        : "+l"(a.s00), "+l"(a.m), "+l"(a.mh)
        : "r"(x), "r"(c0), "r"(cs));
}

// The 128-bit value T of an accumulator.
__device__ __forceinline__ U128 acc30k_value(const Acc30K &a)
{
    // mid = (mh, m) - s00 - s11 = sum of x0 c1 + x1 c0 (below 2^65)
    u64 ml, mhh;
    asm("sub.cc.u64 %0, %2, %4;\n\t"
        "subc.u64 %1, %3, 0;\n\t"
        "sub.cc.u64 %0, %0, %5;\n\t"
        "subc.u64 %1, %1, 0;"
        : "=l"(ml), "=l"(mhh)
        : "l"(a.m), "l"(a.mh), "l"(a.s00), "l"(a.s11));
    U128 t;
    asm("add.cc.u64 %0, %2, %3;\n\t"
        "addc.u64 %1, %4, %5;"
        : "=l"(t.lo), "=l"(t.hi)
        : "l"(a.s00), "l"(ml << 30), "l"((ml >> 34) | (mhh << 30)), "l"(a.s11 >> 4));
    asm("add.cc.u64 %0, %0, %2;\n\t"
        "addc.u64 %1, %1, 0;"
        : "+l"(t.lo), "+l"(t.hi)
        : "l"(a.s11 << 60));
    return t;
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
    u64 one_p;      // floor(2^64 / q): Shoup companion of 1 (reduces any x < 2^64)
};

// any x < 2^64 -> [0, q) (Shoup multiplication by 1)
__device__ __forceinline__ u64 reduce_any(u64 x, u64 q, u64 one_p) { return csub(x - __umul64hi(x, one_p) * q, q); }

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

// Evaluation-domain automorphism X -> X^g: output slot k reads input slot
// perm_index(k, g) (slot k holds the value at psi^(2 brv(k) + 1)).
__device__ __forceinline__ int perm_index(int k, unsigned g, int log_n)
{
    const unsigned e = 2u * brev_bits((unsigned)k, log_n) + 1u;
    const unsigned e2 = (e * g) & ((2u << log_n) - 1u);
    return (int)brev_bits((e2 - 1u) >> 1, log_n);
}
