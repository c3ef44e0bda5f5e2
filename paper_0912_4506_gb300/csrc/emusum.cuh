// The running sum of Eq. 1 in exact binary64 arithmetic on the integer pipes.
//
// The six-neighbour sum s = ((((x0 + x1) + x2) + x3) + x4) + x5 rounds after every
// addition (round to nearest, ties to even).  For positive normal operands this
// header carries the partial sums unpacked - a 53-bit integer significand R in
// [2^52, 2^53] and a biased exponent E, value R * 2^(E - 1075) - so that each
// addition costs one alignment, one integer sum and one rounding, with no
// packing or unpacking of the running sum in between.
//
// Method (from the definition of binary64 and of rounding to nearest even):
// an operand with biased exponent e <= E and significand m in [2^52, 2^53) is
// aligned on a grid nine bits finer than the running sum's last place,
//     T = R * 2^9 + m * 2^(9 - d),   d = E - e in [0, 9],
// which holds the exact sum because no bit of m falls below that grid.  T lies
// in [2^61, 2^63); with c = 1 when T >= 2^62 the correctly rounded sum is
//     R' = RNE(T / 2^(9 + c)),  E' = E + c,
// and RNE(q) for an integer shifted right by k is (T + 2^(k-1) - 1 + lsb) >> k
// with lsb the last kept bit (a tie goes up exactly when the kept part is odd).
// R' may reach 2^53 (a rounding carry); the next alignment and the final
// packing treat that value correctly, so it is never renormalised.  The first
// addition uses the same formula with both operands aligned to the larger
// exponent (|e0 - e1| <= 9).
//
// The fast path covers exponent gaps 0..9 with the running sum not smaller in
// exponent than the operand; every addition records whether its gap was inside
// that window, and a caller whose warp has any lane outside it recomputes that
// warp's sums on the FP64 unit (same bits).  In a sweep of smooth positive data
// the window holds for nearly every update.  Operands must be positive normal
// numbers whose sums stay finite (the sweeps check the range once per call).
//
// Everything here is plain integer arithmetic, usable on the host too, so that
// the routine can be checked against the host's IEEE-754 addition.
#pragma once

#include <stdint.h>
#include <string.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace jac {
namespace emusum {

struct Unp {      // a positive normal double, unpacked
    uint64_t m;   // significand with the hidden bit, [2^52, 2^53)
    uint32_t e;   // biased exponent
};

struct Acc {      // a running sum
    uint64_t r;   // significand, [2^52, 2^53]
    uint32_t e;   // biased exponent
    uint32_t bad; // nonzero: an addition left the fast path's window
};

__host__ __device__ __forceinline__ uint64_t bits_of(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}

__host__ __device__ __forceinline__ double double_of(uint64_t b) {
    double x;
    memcpy(&x, &b, 8);
    return x;
}

__host__ __device__ __forceinline__ Unp unpack(double x) {
    const uint64_t b = bits_of(x);
    Unp u;
    u.e = (uint32_t)(b >> 52);
    // the significand: the exponent field replaced by the hidden bit
    u.m = b - ((uint64_t)(u.e - 1u) << 52);
    return u;
}

// T in [2^61, 2^63): round to 53 bits at position 9 + c, c = (T >= 2^62).
__host__ __device__ __forceinline__ void round_into(Acc& a, uint64_t T, uint32_t E) {
    const uint32_t c = (uint32_t)(T >> 62);
    const uint32_t k = 9u + c;
    const uint64_t lsb = (T >> k) & 1u;
    const uint64_t inc = (255u + (c << 8)) + lsb;  // 2^(k-1) - 1 + lsb
    a.r = (T + inc) >> k;
    a.e = E + c;
}

// x0 + x1 (the first addition of the sum).
__host__ __device__ __forceinline__ Acc first(const Unp& x0, const Unp& x1) {
    Acc a;
    const uint32_t E = x0.e > x1.e ? x0.e : x1.e;
    const uint32_t d0 = E - x0.e, d1 = E - x1.e;
    // the gap is the larger of d0, d1 (the other is 0)
    a.bad = (d0 | d1) > 9u;
    const uint32_t sh0 = 9u - (d0 > 9u ? 9u : d0), sh1 = 9u - (d1 > 9u ? 9u : d1);
    const uint64_t T = (x0.m << sh0) + (x1.m << sh1);
    round_into(a, T, E);
    return a;
}

// a + x, exact when 0 <= a.e - x.e <= 9 (else a.bad is set and the value is
// meaningless).
__host__ __device__ __forceinline__ void add(Acc& a, const Unp& x) {
    const uint32_t d = a.e - x.e;  // wraps when x.e > a.e: then d > 9
    a.bad |= d > 9u;
    const uint32_t sh = 9u - (d > 9u ? 9u : d);
    const uint64_t T = (a.r << 9) + (x.m << sh);
    round_into(a, T, a.e);
}

// The double a holds (valid when !a.bad).
__host__ __device__ __forceinline__ double pack(const Acc& a) {
    // (E - 1) * 2^52 + R: a carry of R into 2^53 moves into the exponent field
    return double_of(((uint64_t)(a.e - 1u) << 52) + a.r);
}

// ---------------------------------------------------------------------------
// The same arithmetic in 32-bit words, written for the GPU's two integer pipes.
// The GB300 integer ALU pipe (shifts, logic, compares, 3-input adds) is the one
// that binds a sweep doing this work, while the FMA pipe also executes 32-bit
// integer multiply-adds.  Shifts by a known power of two are therefore written
// as multiplications (x << s = lo(x * 2^s), x >> s = hi(x * 2^(32-s))) and most
// additions as multiply-adds by a runtime 1; the multipliers come from a kernel
// argument, so the compiler keeps them as multiplications.  Results equal the
// 64-bit form above bit for bit (checked on the host and on the GPU).
struct Words {    // a running sum in 32-bit words
    uint32_t rl, rh;  // significand R = rh:rl, [2^52, 2^53]
    uint32_t e;       // biased exponent
    uint32_t bad;     // nonzero: an addition left the window
};

struct UnpW {     // an operand in 32-bit words
    uint32_t ml, mh;  // significand with the hidden bit
    uint32_t e;
};

struct Mul {      // runtime multipliers and constants (all derived from a runtime 1)
    uint32_t one, m1, k4, k9, k512, k4096, p20, m20, k10, k255, k256, k2p23, m2p22;
};

__host__ __device__ __forceinline__ Mul make_mul(uint32_t one) {
    Mul k;
    k.one = one;
    k.m1 = 0u - one;
    k.k4 = one << 2;
    k.k9 = 9u * one;
    k.k512 = one << 9;
    k.k4096 = one << 12;
    k.p20 = one << 20;
    k.m20 = 0u - (one << 20);
    k.k10 = 429496730u * one;  // ceil(2^32 / 10): hi(d * k10) = 0 exactly when d <= 9
    k.k255 = 255u * one;
    k.k256 = one << 8;
    k.k2p23 = one << 23;
    k.m2p22 = 0u - (one << 22);
    return k;
}

// 32-bit multiply-adds (FMA pipe on the GPU).
__host__ __device__ __forceinline__ uint32_t mlo(uint32_t a, uint32_t b, uint32_t c) {
#ifdef __CUDA_ARCH__
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
#else
    return a * b + c;
#endif
}
__host__ __device__ __forceinline__ uint32_t mhi(uint32_t a, uint32_t b, uint32_t c) {
#ifdef __CUDA_ARCH__
    uint32_t r;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
#else
    return (uint32_t)(((uint64_t)a * b) >> 32) + c;
#endif
}
// (a * b) as a 64-bit pair
__host__ __device__ __forceinline__ void mwide(uint32_t a, uint32_t b, uint32_t& lo,
                                              uint32_t& hi) {
#ifdef __CUDA_ARCH__
    asm("mul.lo.u32 %0, %2, %3;\n\tmul.hi.u32 %1, %2, %3;"
        : "=r"(lo), "=r"(hi)
        : "r"(a), "r"(b));
#else
    const uint64_t p = (uint64_t)a * b;
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
#endif
}
// T = (rh:rl) * k + (ah:al) with a carry between the words, k < 2^32 and no
// overflow of 64 bits (multiply-adds with carry, FMA pipe)
__host__ __device__ __forceinline__ void mad64(uint32_t rl, uint32_t rh, uint32_t k, uint32_t al,
                                              uint32_t ah, uint32_t& tl, uint32_t& th) {
#ifdef __CUDA_ARCH__
    uint32_t x;
    asm("mad.hi.u32 %2, %3, %5, %7;\n\t"
        "mad.lo.cc.u32 %0, %3, %5, %6;\n\t"
        "madc.lo.u32 %1, %4, %5, %2;"
        : "=r"(tl), "=r"(th), "=&r"(x)
        : "r"(rl), "r"(rh), "r"(k), "r"(al), "r"(ah));
#else
    const uint64_t r = ((uint64_t)rh << 32) | rl, a = ((uint64_t)ah << 32) | al;
    const uint64_t t = r * k + a;
    tl = (uint32_t)t;
    th = (uint32_t)(t >> 32);
#endif
}
// (th:tl) + s, s < 2^32 (3-operand add with carry, ALU pipe)
__host__ __device__ __forceinline__ void add64s(uint32_t tl, uint32_t th, uint32_t s,
                                               uint32_t& ul, uint32_t& uh) {
#ifdef __CUDA_ARCH__
    asm("add.cc.u32 %0, %2, %4;\n\taddc.u32 %1, %3, 0;"
        : "=r"(ul), "=r"(uh)
        : "r"(tl), "r"(th), "r"(s));
#else
    const uint64_t u = ((((uint64_t)th) << 32) | tl) + s;
    ul = (uint32_t)u;
    uh = (uint32_t)(u >> 32);
#endif
}

// x >> n for n in [0, 2^32): 0 once n >= 32 (the PTX shift clamps; ALU pipe)
__host__ __device__ __forceinline__ uint32_t shr_clamp(uint32_t x, uint32_t n) {
#ifdef __CUDA_ARCH__
    uint32_t r;
    asm("shr.u32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(n));
    return r;
#else
    return n < 32u ? x >> n : 0u;
#endif
}

__host__ __device__ __forceinline__ uint32_t lo_word(double x) {
    return (uint32_t)bits_of(x);
}
__host__ __device__ __forceinline__ uint32_t hi_word(double x) {
    return (uint32_t)(bits_of(x) >> 32);
}

__host__ __device__ __forceinline__ UnpW unpack_w(double x, const Mul& k) {
    UnpW u;
    const uint32_t bh = hi_word(x);
    u.ml = lo_word(x);
    // shift and mask on the ALU pipe: the pipes stay balanced this way
    u.e = bh >> 20;
    u.mh = (bh & 0x000FFFFFu) | 0x00100000u;  // the hidden bit replaces the exponent
    (void)k;
    return u;
}

// 64-bit funnel shifts of hi:lo by n in [0, 32] (ALU pipe): the high word of
// (hi:lo) << n, and the low word of (hi:lo) >> n.
__host__ __device__ __forceinline__ uint32_t fshl(uint32_t lo, uint32_t hi, uint32_t n) {
#ifdef __CUDA_ARCH__
    uint32_t r;
    asm("shf.l.clamp.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(lo), "r"(hi), "r"(n));
    return r;
#else
    n = n < 32u ? n : 32u;
    return (uint32_t)(((((uint64_t)hi) << 32 | lo) << n) >> 32);
#endif
}
__host__ __device__ __forceinline__ uint32_t fshr(uint32_t lo, uint32_t hi, uint32_t n) {
#ifdef __CUDA_ARCH__
    uint32_t r;
    asm("shf.r.clamp.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(lo), "r"(hi), "r"(n));
    return r;
#else
    n = n < 32u ? n : 32u;
    return (uint32_t)((((uint64_t)hi) << 32 | lo) >> n);
#endif
}
// x << n for n in [0, 2^32): 0 once n >= 32 (ALU pipe)
__host__ __device__ __forceinline__ uint32_t shl_clamp(uint32_t x, uint32_t n) {
#ifdef __CUDA_ARCH__
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(n));
    return r;
#else
    return n < 32u ? x << n : 0u;
#endif
}
// (ah:al) + (bh:bl) (add with carry, ALU pipe)
__host__ __device__ __forceinline__ void add64w(uint32_t al, uint32_t ah, uint32_t bl,
                                               uint32_t bh, uint32_t& tl, uint32_t& th) {
#ifdef __CUDA_ARCH__
    asm("add.cc.u32 %0, %2, %4;\n\taddc.u32 %1, %3, %5;"
        : "=r"(tl), "=r"(th)
        : "r"(al), "r"(ah), "r"(bl), "r"(bh));
#else
    const uint64_t t = ((((uint64_t)ah) << 32) | al) + ((((uint64_t)bh) << 32) | bl);
    tl = (uint32_t)t;
    th = (uint32_t)(t >> 32);
#endif
}

// (ah:al) * k + (bh:bl) with the carry between the words (multiply-adds with
// carry on the FMA pipe), the high word of al * k ignored: callers pass k = 1,
// or k = 2^9 with the high word's share added separately.
__host__ __device__ __forceinline__ void madd64(uint32_t al, uint32_t ah, uint32_t k,
                                               uint32_t bl, uint32_t bh, uint32_t one,
                                               uint32_t& tl, uint32_t& th) {
#ifdef __CUDA_ARCH__
    asm("mad.lo.cc.u32 %0, %2, %4, %5;\n\tmadc.lo.u32 %1, %3, %7, %6;"
        : "=r"(tl), "=r"(th)
        : "r"(al), "r"(ah), "r"(k), "r"(bl), "r"(bh), "r"(one));
#else
    const uint64_t lo = (uint64_t)(uint32_t)(al * k) + bl;
    tl = (uint32_t)lo;
    th = ah * one + bh + (uint32_t)(lo >> 32);
#endif
}

// Form F of the word arithmetic (bit 0: 64-bit additions as 3-operand ALU adds
// with carry instead of multiply-adds with carry; bit 1: the window test as an
// ALU compare instead of a multiply-high).  All forms give the same bits.
// T = (ah:al * 2^S9) + (bh:bl) with S9 = 9 or 0 applied to the low word only
// (the caller passes the high word of the shifted value in ah).
template <int F, bool S9>
__host__ __device__ __forceinline__ void sum64(uint32_t al, uint32_t ah, uint32_t bl, uint32_t bh,
                                              const Mul& km, uint32_t& tl, uint32_t& th) {
    if constexpr ((F & 1) != 0) {
        const uint32_t pl = S9 ? mlo(al, km.k512, 0u) : al;
        add64w(pl, ah, bl, bh, tl, th);
    } else {
        madd64(al, ah, S9 ? km.k512 : km.one, bl, bh, km.one, tl, th);
    }
}

template <int F>
__host__ __device__ __forceinline__ uint32_t window(uint32_t d, uint32_t bad, const Mul& k) {
    if constexpr ((F & 2) != 0) return bad | (d > 9u ? 1u : 0u);
    return mhi(d, k.k10, bad);
}

// T = (th:tl) in [2^61, 2^63): round into a, exponent E + c.  The shifts run on
// the ALU pipe, the additions and the exponent bookkeeping on the FMA pipe.
template <int F = 0>
__host__ __device__ __forceinline__ void round_w(Words& a, uint32_t tl, uint32_t th, uint32_t E,
                                                const Mul& k) {
    const uint32_t c = th >> 30;                               // T >> 62
    const uint32_t kk = mlo(c, k.one, k.k9);                   // 9 + c
    const uint32_t lsb = (tl >> kk) & 1u;                      // bit k of T
    const uint32_t inc = mlo(lsb, k.one, mlo(c, k.k256, k.k255));  // 2^(k-1) - 1 + lsb
    uint32_t ul, uh;
    sum64<F, false>(tl, th, inc, 0u, k, ul, uh);               // U = T + inc
    a.rl = fshr(ul, uh, kk);                                   // U >> k
    a.rh = uh >> kk;
    a.e = mlo(c, k.one, E);
}

template <int F = 0>
__host__ __device__ __forceinline__ Words first_w(const UnpW& x0, const UnpW& x1, const Mul& k) {
    Words a;
    const uint32_t E = x0.e > x1.e ? x0.e : x1.e;
    const uint32_t d0 = mlo(x0.e, k.m1, E), d1 = mlo(x1.e, k.m1, E);
    a.bad = window<F>(d1, window<F>(d0, 0u, k), k);
    // shifts 9 - d (huge when d >= 10: the sum is then discarded)
    const uint32_t s0 = mlo(d0, k.m1, k.k9), s1 = mlo(d1, k.m1, k.k9);
    uint32_t tl, th;
    sum64<F, false>(shl_clamp(x0.ml, s0), fshl(x0.ml, x0.mh, s0), shl_clamp(x1.ml, s1),
                    fshl(x1.ml, x1.mh, s1), k, tl, th);  // T = m0 * 2^s0 + m1 * 2^s1
    round_w<F>(a, tl, th, E, k);
    return a;
}

template <int F = 0>
__host__ __device__ __forceinline__ void add_w(Words& a, const UnpW& x, const Mul& k) {
    const uint32_t d = mlo(x.e, k.m1, a.e);  // wraps when x.e > a.e
    a.bad = window<F>(d, a.bad, k);
    const uint32_t sh = mlo(d, k.m1, k.k9);  // 9 - d
    uint32_t tl, th;
    // T = R * 2^9 + m * 2^(9 - d): the low word of R * 2^9 is a multiply-add
    sum64<F, true>(a.rl, fshl(a.rl, a.rh, 9u), shl_clamp(x.ml, sh), fshl(x.ml, x.mh, sh), k, tl,
                   th);
    round_w<F>(a, tl, th, a.e, k);
}

__host__ __device__ __forceinline__ double pack_w(const Words& a, const Mul& k) {
    // (E - 1) * 2^52 + R
    const uint32_t hi = mlo(a.e, k.p20, mlo(a.rh, k.one, k.m20));
    return double_of(((uint64_t)hi << 32) | a.rl);
}

}  // namespace emusum
}  // namespace jac
