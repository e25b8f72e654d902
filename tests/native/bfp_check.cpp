// Checks the block-floating-point codec of the moment-space deviations (storage
// LBM_MS_BFP) on the host against its stated rules: rounding error at most half a
// step (a step for the largest value when it rounds up to the top of its binade),
// the smallest exponent that holds the block, saturation exactly beyond 2^14,
// exact scaling by powers of two, and the word layout (mantissa in bits 15..1,
// exponent bits 0, 1, 2 in the dx, dy, dd words).
// Usage: bfp_check <cases> <seed>; prints a summary line; exits non-zero on failure.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "../../paper_2408_01081_gb300/csrc/lbm_mscodec.cuh"

static uint64_t state;
static uint64_t next()   // splitmix64
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double uni() { return (next() >> 11) * (1.0 / 9007199254740992.0); }

static long fails = 0;
static void check(bool ok, const char* what, double x, double y, double z)
{
    if (!ok && fails++ < 10) std::printf("FAIL %s: %.9g %.9g %.9g\n", what, x, y, z);
}

int main(int argc, char** argv)
{
    const long n = argc > 1 ? std::atol(argv[1]) : 100000;
    state = argc > 2 ? std::strtoull(argv[2], nullptr, 10) : 1;
    long sats = 0;
    for (long i = 0; i < n; ++i) {
        float v[3];
        const double top = std::ldexp(1.0, (int)(uni() * 24.0) - 8);   // block scales 2^-8 .. 2^15
        for (int c = 0; c < 3; ++c) {
            const double mag = top * std::pow(2.0, -12.0 * uni());          // members down to 2^-12 of it
            v[c] = (float)((next() & 1) ? -mag : mag);
        }
        if ((next() & 15) == 0) v[next() % 3] = 0.f;
        uint16_t w[3];
        bool sat = false;
        lbmc::bfp_encode(v[0], v[1], v[2], w[0], w[1], w[2], sat);
        // layout: exponent bits, mantissas
        const int e = (w[0] & 1) | ((w[1] & 1) << 1) | ((w[2] & 1) << 2);
        double amax = 0.0;
        for (int c = 0; c < 3; ++c) amax = std::fmax(amax, std::fabs((double)v[c]));
        const bool fits = amax < 16384.0;
        check(sat == !fits, "saturation flag", v[0], v[1], v[2]);
        sats += sat;
        float d[3];
        lbmc::bfp_decode(w[0], w[1], w[2], 1.0f, d[0], d[1], d[2]);
        const double step = std::ldexp(1.0, e - 7);
        for (int c = 0; c < 3; ++c) {
            const int m = (int)(int16_t)w[c] >> 1;                          // independent decode
            check(m >= -16383 && m <= 16383, "mantissa range", v[0], v[1], v[2]);
            check((double)d[c] == m * step, "decode", v[0], v[1], v[2]);
            if (fits) {
                const double err = std::fabs((double)d[c] - (double)v[c]);
                const bool largest = std::fabs((double)v[c]) == amax;
                check(err <= (largest ? 1.0 : 0.5) * step, "rounding error", v[0], v[1], v[2]);
                if (largest && e > 0) check(err <= std::ldexp(amax, -13), "relative error of the largest", v[0], v[1], v[2]);
            }
        }
        if (fits) {
            // the exponent is the smallest that holds the block: one less would overflow the mantissa
            check(e == 0 || amax * std::ldexp(1.0, 7 - (e - 1)) >= 16383.5, "minimal exponent", v[0], v[1], v[2]);
            check(amax * std::ldexp(1.0, 7 - e) < 16384.0, "block fits", v[0], v[1], v[2]);
        }
        // decoding with inv_s = 2^-k scales exactly
        const int k = (int)(next() % 40);
        float q[3];
        lbmc::bfp_decode(w[0], w[1], w[2], std::ldexp(1.0f, -k), q[0], q[1], q[2]);
        for (int c = 0; c < 3; ++c) check((double)q[c] == std::ldexp((double)d[c], -k), "scaled decode", v[0], v[1], v[2]);
    }
    // zero block, a block at the saturation boundary, NaN
    {
        uint16_t w[3];
        bool sat = false;
        lbmc::bfp_encode(0.f, -0.f, 0.f, w[0], w[1], w[2], sat);
        check(w[0] == 0 && w[1] == 0 && w[2] == 0 && !sat, "zero block", 0, 0, 0);
        lbmc::bfp_encode(16383.0f, -1.0f, 0.5f, w[0], w[1], w[2], sat);
        float d[3];
        lbmc::bfp_decode(w[0], w[1], w[2], 1.0f, d[0], d[1], d[2]);
        check(!sat && d[0] == 16383.0f && d[1] == -1.0f && d[2] == 0.f, "boundary block", 16383, -1, 0.5);
        lbmc::bfp_encode(16384.0f, 0.f, 0.f, w[0], w[1], w[2], sat);
        check(sat, "saturation at 2^14", 16384, 0, 0);
        sat = false;
        lbmc::bfp_encode(std::nanf(""), 1.f, 1.f, w[0], w[1], w[2], sat);
        check(sat, "NaN flagged", 0, 1, 1);
    }
    std::printf("%ld cases, %ld saturated, %ld failures\n", n, sats, fails);
    return fails ? 1 : 0;
}
