// Block floating point for the moment-space deviations (storage LBM_MS_BFP).
//
// The three non-equilibrium moments (dx, dy, dd) of one component of one node,
// already multiplied by the lattice's power-of-two scale s, share one exponent:
//     value = m * 2^(e - 7),   m a signed 15-bit integer in [-16383, 16383], e in 0..7.
// Each of the three 16-bit words holds its mantissa in bits 15..1 and one bit of
// e in bit 0 (bit 0 of e in the dx word, bit 1 in the dy word, bit 2 in the dd
// word), so the three words of a component are always decoded together.
//
// The exponent is the smallest one whose mantissa range holds the largest of the
// three values: for a largest value in [2^q, 2^(q+1)) it is e = q - 6 (at least
// 0), which puts that value's mantissa in [2^13, 2^14).  Its rounding error is
// then at most 2^-14 of the value (FP16: 2^-11), the other two values share the
// same absolute step.  With s chosen so that the largest deviation of the
// initial state sits in [2^10, 2^11), e = 7 leaves a factor of at least 8 of
// headroom; a block whose largest value needs e > 7 is clamped at e = 7 (its
// mantissas saturate at +-16383) and `sat` is set.  Values below 2^-7 of the
// largest step (|value| < 128 at e = 0) keep an absolute step of 2^-7.
//
// The functions compile for host and device: the host build is checked against
// these rules bit for bit (tests/native/bfp_check.cpp).
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define MSC_HD __host__ __device__ __forceinline__
#else
#define MSC_HD inline
#include <cmath>
#endif

namespace lbmc {

constexpr int kBfpMant = 16383;   // largest mantissa magnitude
constexpr int kBfpTop = 7;        // largest exponent

// exact 2^k for -126 <= k <= 127
MSC_HD float pow2f(int k)
{
    union { uint32_t u; float f; } v;
    v.u = (uint32_t)(k + 127) << 23;
    return v.f;
}

// exponent of a block whose largest magnitude is amax (>= 0, finite); kBfpTop + 1 or more
// means the block does not fit
MSC_HD int bfp_exponent(float amax)
{
    union { float f; uint32_t u; } v;
    v.f = amax;
    const int q = (int)((v.u >> 23) & 0xFFu) - 127;   // floor(log2 amax); -127 for zero / subnormal
    const int e = q - 6;
    return e < 0 ? 0 : e;
}

MSC_HD int bfp_round(float x)
{
#ifdef __CUDA_ARCH__
    return __float2int_rn(x);          // round to nearest, ties to even
#else
    return (int)std::nearbyint(x);     // the default rounding mode: nearest, ties to even
#endif
}

MSC_HD uint16_t bfp_word(int m, int ebit)
{
    return (uint16_t)((((uint32_t)m << 1) & 0xFFFEu) | (uint32_t)(ebit & 1));
}

// X, Y, Z: the scaled deviations of one component; sat is set when the block saturates
MSC_HD void bfp_encode(float X, float Y, float Z, uint16_t& wx, uint16_t& wy, uint16_t& wz, bool& sat)
{
    const float ax = X < 0.f ? -X : X, ay = Y < 0.f ? -Y : Y, az = Z < 0.f ? -Z : Z;
    float amax = ax > ay ? ax : ay;
    amax = amax > az ? amax : az;
    int e = bfp_exponent(amax);
    if (e > kBfpTop || !(X == X && Y == Y && Z == Z)) {   // too large, or NaN: clamp and flag
        e = kBfpTop;
        sat = true;
    }
    const float f = pow2f(kBfpTop - e);
    int mx = bfp_round(X * f), my = bfp_round(Y * f), mz = bfp_round(Z * f);
    // only the largest value can round up to 2^14 at the top of its binade: one step of clamping
    mx = mx > kBfpMant ? kBfpMant : (mx < -kBfpMant ? -kBfpMant : mx);
    my = my > kBfpMant ? kBfpMant : (my < -kBfpMant ? -kBfpMant : my);
    mz = mz > kBfpMant ? kBfpMant : (mz < -kBfpMant ? -kBfpMant : mz);
    wx = bfp_word(mx, e);
    wy = bfp_word(my, e >> 1);
    wz = bfp_word(mz, e >> 2);
}

// the unscaled deviations: value * inv_s (inv_s = 1/s, a power of two)
MSC_HD void bfp_decode(uint16_t wx, uint16_t wy, uint16_t wz, float inv_s, float& X, float& Y, float& Z)
{
    const int e = (int)(wx & 1u) | ((int)(wy & 1u) << 1) | ((int)(wz & 1u) << 2);
    const float f = pow2f(e - kBfpTop) * inv_s;
    X = (float)((int)(int16_t)wx >> 1) * f;
    Y = (float)((int)(int16_t)wy >> 1) * f;
    Z = (float)((int)(int16_t)wz >> 1) * f;
}

}  // namespace lbmc
