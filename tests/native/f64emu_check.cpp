// Checks the integer-pipe binary64 addition of the step kernel against the
// host's hardware addition (IEEE 754, round to nearest even) bit for bit.
// Usage: f64emu_check <cases per family> <seed>; prints one line per family and
// exits non-zero on the first mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../paper_2408_01081_gb300/csrc/lbm_f64emu.cuh"

using lbmemu::u64;

static u64 bits(double x) { u64 u; std::memcpy(&u, &x, 8); return u; }
static double dbl(u64 u) { double x; std::memcpy(&x, &u, 8); return x; }

static u64 state;
static u64 next()   // splitmix64
{
    u64 z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static bool normal_or_zero(double x) { return x == 0.0 || std::fpclassify(x) == FP_NORMAL; }

static long fails = 0, fast = 0, total = 0;

static void check_add(u64 a, u64 b)
{
    bool ok = true;
    const u64 r = lbmemu::emu_add_bits(a, b, ok);
    const double ref = dbl(a) + dbl(b);
    ++total;
    if (ok) {
        ++fast;
        if (r != bits(ref)) {
            if (fails++ < 10)
                std::printf("MISMATCH add %016llx + %016llx: emu %016llx hw %016llx\n", a, b, r, bits(ref));
        }
    } else if (std::isfinite(dbl(a)) && std::isfinite(dbl(b)) && normal_or_zero(ref) && std::isfinite(ref)) {
        if (fails++ < 10) std::printf("UNEXPECTED FALLBACK add %016llx + %016llx\n", a, b);
    }
}

static void check_half(u64 u, u64 t)
{
    bool ok = true;
    const u64 h = lbmemu::emu_half_bits(u, ok);
    const u64 r = lbmemu::emu_add_bits(h, t, ok);
    const double ref = std::fma(0.5, dbl(u), dbl(t));
    ++total;
    if (ok) {
        ++fast;
        if (r != bits(ref)) {
            if (fails++ < 10)
                std::printf("MISMATCH half %016llx, %016llx: emu %016llx hw %016llx\n", u, t, r, bits(ref));
        }
    }
}

// faithful variant: within (1/2 + 2^-9) ulp of the exact sum a + b = s + err (TwoSum), and on
// the integer path whenever the exact variant is
static long ffails = 0, ftotal = 0;

static void check_faithful(u64 a, u64 b)
{
    bool ok_exact = true, ok = true;
    lbmemu::emu_add_bits(a, b, ok_exact);
    const u64 r = lbmemu::emu_add_faithful_bits(a, b, ok);
    ++ftotal;
    if (ok_exact && !ok) {
        if (ffails++ < 10) std::printf("FAITHFUL FALLBACK %016llx + %016llx\n", a, b);
        return;
    }
    if (!ok) return;
    const double x = dbl(a), y = dbl(b), s = x + y;
    const double bb = s - x, err = (x - (s - bb)) + (y - bb);       // a + b = s + err exactly
    const double res = dbl(r);
    const double ulp = s != 0.0 ? std::ldexp(1.0, std::ilogb(s) - 52) : std::ldexp(1.0, -1074);
    const double dev = std::fabs((res - s) - err);                  // res - s is exact (Sterbenz)
    if (!(dev <= (0.5 + 1.0 / 512) * ulp) || (s == 0.0 && res != 0.0)) {
        if (ffails++ < 10)
            std::printf("FAITHFUL OFF %016llx + %016llx: emu %016llx hw %016llx (%.3g ulp)\n", a, b, r, bits(s),
                        dev / ulp);
    }
}

static u64 with_exp(u64 x, int e) { return (x & 0x800FFFFFFFFFFFFFull) | ((u64)e << 52); }

int main(int argc, char** argv)
{
    const long n = argc > 1 ? std::atol(argv[1]) : 1000000;
    state = argc > 2 ? std::strtoull(argv[2], 0, 10) : 1;
    // 1. arbitrary bit patterns (NaN, infinity, subnormal, zero included)
    for (long i = 0; i < n; ++i) check_add(next(), next());
    std::printf("random bits: %ld cases, %ld on the fast path, %ld failures\n", total, fast, fails);
    // 2. normal numbers with nearby exponents (every alignment distance 0..70)
    for (long i = 0; i < n; ++i) {
        const int e = 100 + (int)(next() % 1800);
        const int d = (int)(next() % 71);
        check_add(with_exp(next(), e), with_exp(next(), e - d > 0 ? e - d : 1));
    }
    std::printf("nearby exponents: %ld cases, %ld failures\n", total, fails);
    // 3. cancellation: b close to -a (last bits perturbed), and exact negation
    for (long i = 0; i < n; ++i) {
        const u64 a = with_exp(next(), 1 + (int)(next() % 2046));
        const u64 b = (a ^ 0x8000000000000000ull) + (next() % 4096) - 2048;
        check_add(a, b);
        check_add(a, a ^ 0x8000000000000000ull);
    }
    std::printf("cancellation: %ld cases, %ld failures\n", total, fails);
    // 4. ties and carries: significands with few random low bits
    for (long i = 0; i < n; ++i) {
        const int e = 1 + (int)(next() % 2045);
        const u64 a = with_exp(next() & 0x800FFFFFFFFFFC00ull, e);
        const u64 b = with_exp(next(), e - (int)(next() % 12) > 0 ? e - (int)(next() % 12) : 1);
        check_add(a, b);
    }
    std::printf("ties/carries: %ld cases, %ld failures\n", total, fails);
    // 5. special values: zeros, subnormals, extremes, infinities, NaN
    const u64 sp[] = {0ull, 0x8000000000000000ull, 1ull, 0x8000000000000001ull, 0x000FFFFFFFFFFFFFull,
                      0x0010000000000000ull, 0x8010000000000000ull, 0x0020000000000000ull, 0x7FEFFFFFFFFFFFFFull,
                      0xFFEFFFFFFFFFFFFFull, 0x7FF0000000000000ull, 0xFFF0000000000000ull, 0x7FF8000000000000ull,
                      0x3FF0000000000000ull, 0xBFF0000000000000ull, 0x3CA0000000000000ull, 0x7FE0000000000000ull};
    const int ns = sizeof(sp) / sizeof(sp[0]);
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) { check_add(sp[i], sp[j]); check_half(sp[i], sp[j]); }
    for (long i = 0; i < n / 10; ++i)
        for (int j = 0; j < ns; ++j) { check_add(sp[j], next()); check_add(next(), sp[j]); }
    std::printf("special values: %ld cases, %ld failures\n", total, fails);
    // 6. round(u/2 + t) against fma(0.5, u, t)
    for (long i = 0; i < n; ++i) {
        const int e = 1 + (int)(next() % 2046);
        check_half(with_exp(next(), e), with_exp(next(), e - (int)(next() % 60) > 0 ? e - (int)(next() % 60) : 1));
        check_half(next(), next());
    }
    std::printf("half add: %ld cases, %ld on the fast path, %ld failures\n", total, fast, fails);
    // 7. the faithful variant on the same families (ranges that keep a + b normal)
    for (long i = 0; i < n; ++i) {
        const int e = 100 + (int)(next() % 1800);
        const int d = (int)(next() % 71);
        check_faithful(with_exp(next(), e), with_exp(next(), e - d));
        const u64 a = with_exp(next(), 100 + (int)(next() % 1800));
        check_faithful(a, (a ^ 0x8000000000000000ull) + (next() % 4096) - 2048);
        check_faithful(a, a ^ 0x8000000000000000ull);
        check_faithful(with_exp(next() & 0x800FFFFFFFFFFC00ull, e), with_exp(next(), e - (int)(next() % 12)));
        check_faithful(next(), next());
    }
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) check_faithful(sp[i], sp[j]);
    std::printf("faithful add: %ld cases, %ld failures\n", ftotal, ffails);
    return (fails || ffails) ? 1 : 0;
}
