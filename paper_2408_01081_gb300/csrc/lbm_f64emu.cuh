// Exact binary64 addition on the integer pipes.
//
// GB300 executes FP64 arithmetic at 2 operations per clock per SM, while its
// integer/logic pipes are nearly idle in the FP64 step kernel.  The step needs
// 35 additions and 12 fused multiply-adds per node; moving part of the additions
// to the integer pipes lets both kinds of pipe work at once.
//
// emu_add() returns the IEEE 754 binary64 sum of two numbers rounded to nearest,
// ties to even (the rounding of the hardware add), computed from the bit patterns:
// align the smaller significand with guard bits and a sticky bit, add or
// subtract, normalise with a leading-zero count, round, repack.  Zero and
// subnormal inputs are handled exactly.  Where the result would be subnormal,
// infinite or NaN (or an input is infinite or NaN) the flag `ok` is cleared and
// the caller recomputes with the hardware instruction, so whenever `ok` stays
// set the result is bit-identical to the hardware sum.
//
// emu_add_faithful_bits() is a cheaper variant rounded faithfully (within 1/2 + 2^-9 units
// in the last place), for callers that need FP64 accuracy but not the hardware's bits;
// its rounding is biased (half up on a truncated sum), which long runs accumulate.
//
// emu_half_add(u, t) returns round(u/2 + t), the value of fma(0.5, u, t): u/2 is
// exact for normal u with exponent field >= 2 (its exponent field minus one) and
// for zero; other u clear `ok`.
//
// The header also compiles as plain C++ (host), where its results are checked
// against the host's hardware addition.
#pragma once

#ifdef __CUDACC__
#define EMU_HD __host__ __device__ __forceinline__
#else
#define EMU_HD inline
#endif

namespace lbmemu {

typedef unsigned long long u64;

EMU_HD int clz64(u64 x)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

// significand of a magnitude x with its hidden bit (none for zero / subnormal) at bits
// 62..10, from 32-bit halves: min(hi, 0x00100000) is the hidden bit exactly when the
// exponent field is nonzero and otherwise lies within the fraction bits
EMU_HD u64 sig_bits(u64 x)
{
    const unsigned hi = (unsigned)(x >> 32), lo = (unsigned)x;
    const unsigned hid = hi < 0x00100000u ? hi : 0x00100000u;
    return ((((u64)((hi & 0x000FFFFFu) | hid)) << 32) | lo) << 10;
}

EMU_HD u64 emu_add_bits(u64 ua, u64 ub, bool& ok)
{
    const u64 SIGN = 0x8000000000000000ull;
    const u64 xa = ua & ~SIGN, xb = ub & ~SIGN;
    const bool sw = xb > xa;                        // order by magnitude: |h| >= |l|
    const u64 h = sw ? ub : ua, l = sw ? ua : ub;
    const u64 xh = h & ~SIGN, xl = l & ~SIGN;
    const int eh = (int)(xh >> 52), el = (int)(xl >> 52);
    const bool finite_in = eh < 2047;
    // significands at bits 62..10, guard bits below (zero / subnormal: no hidden bit, and
    // the exponent acts as 1)
    const u64 mh = sig_bits(xh), ml = sig_bits(xl);
    const int e = eh > 1 ? eh : 1;
    int d = e - (el > 1 ? el : 1);
    d = d < 63 ? d : 63;
    u64 al = ml >> d;
    al |= (u64)((al << d) != ml);                   // sticky bit of what was shifted out
    const u64 neg = (u64)0 - (u64)(((h ^ l) & SIGN) != 0);   // all ones for a subtraction
    u64 s = mh + (al ^ neg) - neg;                  // mh + al or mh - al
    const bool zero = (s == 0);
    const int lz = clz64(s | 1ull);                 // leading one to bit 63
    s <<= lz;
    const int er = e + 1 - lz;                      // exponent field of the result
    u64 m = s >> 11;                                // 53-bit significand
    // round to nearest, ties to even: up when the 11 bits below exceed half, or equal half
    // with m odd
    m += (u64)(((unsigned)s & 0x7FFu) + ((unsigned)m & 1u) > 0x400u);
    const u64 r = ((u64)(er - 1) << 52) + m;        // a carry out of m bumps the exponent
    ok = ok && finite_in && (zero || (er >= 1 && (r >> 52) < 2047ull));
    // an exact zero is +0, except -0 + -0
    return zero ? (ua & ub & SIGN) : (r | (h & SIGN));
}

// The same sum rounded faithfully instead of correctly: the aligned smaller significand
// keeps its ten guard bits and is truncated below them (no sticky bit), and the
// normalised sum is rounded half up.  The smaller operand loses bits only when the
// exponents differ by more than ten, and then the sum cancels at most two leading
// bits, so the truncation moves the result by less than 2^-9 units in the last place:
// |result - exact sum| <= (1/2 + 2^-9) ulp.  Not bit-identical to the hardware sum (it
// differs in the last bit near ties); about 17 % fewer integer instructions than
// emu_add_bits.  The error is biased: the truncation lowers the magnitude of sums and
// raises that of differences, and ties round up.  `ok` is cleared for infinite or NaN inputs and for subnormal or
// overflowing results, as there.
EMU_HD u64 emu_add_faithful_bits(u64 ua, u64 ub, bool& ok)
{
    const u64 SIGN = 0x8000000000000000ull, FRAC = 0x000FFFFFFFFFFFFFull, HID = 0x0010000000000000ull;
    const u64 xa = ua & ~SIGN, xb = ub & ~SIGN;
    const bool sw = xb > xa;                        // order by magnitude: |h| >= |l|
    const u64 h = sw ? ub : ua, l = sw ? ua : ub;
    const u64 xh = h & ~SIGN, xl = l & ~SIGN;
    const int eh = (int)(xh >> 52), el = (int)(xl >> 52);
    const u64 mh = ((xh & FRAC) | (eh ? HID : 0ull)) << 10;
    const u64 ml = ((xl & FRAC) | (el ? HID : 0ull)) << 10;
    const int e = eh > 1 ? eh : 1;
    int d = e - (el > 1 ? el : 1);
    d = d > 63 ? 63 : d;
    const u64 al = ml >> d;                         // truncated below the guard bits
    const bool sub = ((h ^ l) & SIGN) != 0;
    u64 s = sub ? mh - al : mh + al;
    const int lz = clz64(s | 1ull);
    s <<= lz;
    const int er = e + 1 - lz;                      // exponent field of the result
    const u64 m = (s >> 11) + ((s >> 10) & 1ull);   // 53-bit significand, rounded half up
    const u64 r = ((u64)(er - 1) << 52) + m;        // a carry out of m bumps the exponent
    ok = ok && eh < 2047 && (s == 0 || (er >= 1 && (r >> 52) < 2047ull));
    return s == 0 ? 0ull : (r | (h & SIGN));
}

EMU_HD u64 emu_half_bits(u64 u, bool& ok)
{
    const u64 SIGN = 0x8000000000000000ull;
    const u64 x = u & ~SIGN;
    const u64 eu = x >> 52;
    ok = ok && ((eu >= 2 && eu < 2047) || x == 0);
    return (x == 0) ? u : u - (1ull << 52);
}

#ifdef __CUDACC__
// Bit pattern of a double through inline asm: with a plain reinterpretation the
// compiler recognises masking / flipping the sign bit as fabs / negation and
// emits them as FP64 instructions, which is what this path is meant to avoid.
__device__ __forceinline__ u64 bits_of(double x)
{
    u64 u;
    asm("mov.b64 %0, %1;" : "=l"(u) : "d"(x));
    return u;
}

__device__ __forceinline__ double double_of(u64 u)
{
    double x;
    asm("mov.b64 %0, %1;" : "=d"(x) : "l"(u));
    return x;
}

__device__ __forceinline__ double emu_add(double a, double b, bool& ok)
{
    return double_of(emu_add_bits(bits_of(a), bits_of(b), ok));
}

__device__ __forceinline__ double emu_sub(double a, double b, bool& ok)
{
    return double_of(emu_add_bits(bits_of(a), bits_of(b) ^ 0x8000000000000000ull, ok));
}

__device__ __forceinline__ double emu_half_add(double u, double t, bool& ok)
{
    return double_of(emu_add_bits(emu_half_bits(bits_of(u), ok), bits_of(t), ok));
}

// faithfully rounded counterparts (emu_add_faithful_bits)
__device__ __forceinline__ double emu_add_f(double a, double b, bool& ok)
{
    return double_of(emu_add_faithful_bits(bits_of(a), bits_of(b), ok));
}

__device__ __forceinline__ double emu_sub_f(double a, double b, bool& ok)
{
    return double_of(emu_add_faithful_bits(bits_of(a), bits_of(b) ^ 0x8000000000000000ull, ok));
}

__device__ __forceinline__ double emu_half_add_f(double u, double t, bool& ok)
{
    return double_of(emu_add_faithful_bits(emu_half_bits(bits_of(u), ok), bits_of(t), ok));
}
#endif

}  // namespace lbmemu
