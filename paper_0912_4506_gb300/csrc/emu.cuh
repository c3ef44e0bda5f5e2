// Exact IEEE-754 binary64 addition (round to nearest, ties to even) on the
// integer pipes, for positive normal operands.
//
// GB300 executes FP64 at 2 operations per clock per SM; the plain FP64 sweep
// (6 operations per lattice-site update) is therefore bound by the FP64 pipe
// while the integer pipes and most issue slots idle.  Doing some of the five
// additions of Eq. 1 with integer instructions lets both pipes work.  The result
// is the correctly rounded sum, identical bit for bit to the FP64 unit's, so
// the sweep stays bit-exact whichever additions are emulated.
//
// Method (written from the definition of binary64 and of rounding to nearest
// even): take the operand X with the larger exponent and the other, Y; shift
// Y's 53-bit significand right by the exponent difference, keeping the bits
// shifted out as a 32-bit fraction; add; renormalise by one bit on a carry
// (folding the lost bit into a sticky bit); round to 53 bits by comparing the
// fraction with one half (ties to the even significand); the exponent follows
// from the carry, and a rounding carry to 2^53 moves into the exponent field
// by itself.  Exponent differences above 31 (the smaller operand then
// only affects the sticky bit, and such lanes are rare) go to the FP64 unit.
// Operands must be positive normal numbers whose sum stays finite; the caller
// guarantees that (see range_check_kernel).
#pragma once

#include <stdint.h>

namespace jac {

__device__ __forceinline__ uint32_t shl32(uint32_t x, uint32_t n) {  // n in [0, 32]
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(n));
    return r;
}

// The FP64-unit addition for the rare pairs the integer path leaves out.  It is
// an out-of-line call so that warps with no such lane jump over it: an inlined
// addition would be issued predicated-off and still hold the FP64 pipe, whose
// time is exactly what the integer path is meant to save.
static __device__ __noinline__ double add_fp64_unit(double a, double b) { return __dadd_rn(a, b); }

// Integer additions on the FMA pipe: a*one + b with `one` a runtime 1 (a kernel
// argument, so the compiler cannot fold it into an ALU add).  The sweep is bound
// by the integer ALU pipe while the FMA pipe idles, so these move work across.
__device__ __forceinline__ uint32_t add_f(uint32_t a, uint32_t b, uint32_t one) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(one), "r"(b));
    return r;
}
__device__ __forceinline__ unsigned long long add64_f(unsigned long long a, unsigned long long b,
                                                      uint32_t one) {
    uint32_t lo, hi;
    asm("mad.lo.cc.u32 %0, %2, %4, %3;\n\tmadc.lo.u32 %1, %5, %4, %6;"
        : "=r"(lo), "=r"(hi)
        : "r"((uint32_t)a), "r"((uint32_t)b), "r"(one), "r"((uint32_t)(a >> 32)),
          "r"((uint32_t)(b >> 32)));
    return ((unsigned long long)hi << 32) | lo;
}

// As add_pos_exact below, with its additions issued to the FMA pipe (a*one + b,
// a*m1 + b with m1 = -one, a*p20 + b with p20 = one << 20, all runtime values).
__device__ __forceinline__ uint32_t mad_u(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

__device__ __forceinline__ double add_pos_exact_f(double a, double b, uint32_t one) {
    const uint32_t m1 = 0u - one, p20 = one << 20, m20 = 0u - p20;  // hoisted out of the loops
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    const bool swap = (uint32_t)(A >> 32) < (uint32_t)(B >> 32);
    const unsigned long long X = swap ? B : A;
    const unsigned long long Y = swap ? A : B;
    const uint32_t ex = (uint32_t)(X >> 52), ey = (uint32_t)(Y >> 52);
    const uint32_t d = mad_u(ey, m1, ex);  // ex - ey
    const uint32_t dd = d > 31u ? 31u : d;
    // significands with the hidden bit: the high word minus (exponent - 1) * 2^20,
    // as multiply-adds (FMA pipe) instead of mask-and-or (integer ALU, the binding
    // pipe of this sweep)
    const unsigned long long mx =
        ((unsigned long long)mad_u(ex, m20, mad_u(one, p20, (uint32_t)(X >> 32))) << 32) |
        (uint32_t)X;
    const unsigned long long my =
        ((unsigned long long)mad_u(ey, m20, mad_u(one, p20, (uint32_t)(Y >> 32))) << 32) |
        (uint32_t)Y;
    const uint32_t F = shl32((uint32_t)my, mad_u(dd, m1, 32u));  // 32 - dd
    const unsigned long long S = add64_f(mx, my >> dd, one);
    const uint32_t c = (uint32_t)(S >> 53);
    const unsigned long long Sn = S >> c;
    const uint32_t Fc = c ? (((uint32_t)S << 31) | (F >> 1) | (F & 1u)) : F;
    const uint32_t up = (uint32_t)(add64_f((unsigned long long)Fc,
                                           mad_u((uint32_t)Sn & 1u, one, 0x7FFFFFFFu), one) >>
                                   32);
    const unsigned long long M = add64_f(Sn, (unsigned long long)up, one);
    // biased exponent (ex + c - 1) placed at bit 52 and added to M (no carry into
    // the low word: the shifted exponent has none)
    const uint32_t e1 = mad_u(ex, one, mad_u(c, one, 0xFFFFFFFFu));
    const uint32_t rhi = mad_u(e1, p20, (uint32_t)(M >> 32));
    double r = __longlong_as_double((long long)(((unsigned long long)rhi << 32) | (uint32_t)M));
    if (__any_sync(__activemask(), d > 31u)) {
        if (d > 31u) r = add_fp64_unit(a, b);
    }
    return r;
}

__device__ __forceinline__ double add_pos_exact(double a, double b) {
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    // order by the high words: when the exponents differ they decide, when they
    // are equal either order works (no alignment shift)
    const bool swap = (uint32_t)(A >> 32) < (uint32_t)(B >> 32);
    const unsigned long long X = swap ? B : A;
    const unsigned long long Y = swap ? A : B;
    const uint32_t ex = (uint32_t)(X >> 52);
    const uint32_t d = ex - (uint32_t)(Y >> 52);
    const uint32_t dd = d > 31u ? 31u : d;  // keeps the integer path defined
    const unsigned long long kMant = 0x000FFFFFFFFFFFFFull, kHidden = 0x0010000000000000ull;
    const unsigned long long mx = (X & kMant) | kHidden;  // 53-bit significands
    const unsigned long long my = (Y & kMant) | kHidden;
    // exact sum = S + F / 2^32: S integer, F the 32-bit fraction of my / 2^dd
    // (dd <= 31, so the bits shifted out fit in the low word)
    const uint32_t F = shl32((uint32_t)my, 32u - dd);
    const unsigned long long S = mx + (my >> dd);           // in [2^52, 2^54)
    const uint32_t c = (uint32_t)(S >> 53);                 // carry: renormalise by 1
    const unsigned long long Sn = S >> c;
    // fraction after the renormalisation, with everything below bit 0 folded
    // into bit 0 (a sticky bit): it still compares with 2^31 exactly
    const uint32_t Fc = c ? (((uint32_t)S << 31) | (F >> 1) | (F & 1u)) : F;
    // round to nearest, ties to even: up when Fc > 2^31, or Fc == 2^31 and Sn odd
    const uint32_t up =
        (uint32_t)(((unsigned long long)Fc + 0x7FFFFFFFull + (Sn & 1ull)) >> 32);
    const unsigned long long M = Sn + up;  // may reach 2^53: the exponent absorbs it
    double r = __longlong_as_double((long long)((((unsigned long long)(ex + c - 1u)) << 52) + M));
    if (__any_sync(__activemask(), d > 31u)) {
        if (d > 31u) r = add_fp64_unit(a, b);
    }
    return r;
}

}  // namespace jac
