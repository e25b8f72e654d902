// Host check of the fixed-point FP64 node update (lbm_f64fx.cuh): every output of
// fx_node() against the same update evaluated in quad precision (__float128: 113-bit
// significands, exact for these sums and products up to a relative 2^-113), within the
// stated bound of half an ulp of the output plus 10 rho (13 rho with the body-load terms h;
// rho where every input converts exactly); the fallback range exactly
// where the header says; and the FP64 operation sequence's own error for comparison.
//
// usage: f64fx_check <cases> <seed>; the last line reads "<n> cases, <m> failures".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../paper_2408_01081_gb300/csrc/lbm_f64fx.cuh"

typedef unsigned long long u64;
typedef __float128 q128;

static u64 state;
static u64 next()
{
    u64 z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double uni() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
static double gauss()
{
    const double u = uni() + 1e-300, v = uni();
    return std::sqrt(-2.0 * std::log(u)) * std::cos(6.283185307179586 * v);
}
static u64 bits(double x)
{
    u64 u;
    std::memcpy(&u, &x, 8);
    return u;
}
static double dbl(u64 u)
{
    double x;
    std::memcpy(&x, &u, 8);
    return x;
}
static q128 qabs(q128 x) { return x < 0 ? -x : x; }
static double ulp(double x)
{
    x = std::fabs(x);
    if (x == 0.0) return 0.0;
    return std::nextafter(x, INFINITY) - x;
}

int main(int argc, char** argv)
{
    const long n = argc > 1 ? std::atol(argv[1]) : 100000;
    state = argc > 2 ? std::strtoull(argv[2], nullptr, 10) : 1;
    long fails = 0, taken = 0, fallback = 0, worse_than_fp64 = 0;
    double worst = 0.0;   // largest error in units of the bound
    for (long c = 0; c < n; ++c) {
        // material: 2 sqrt(cK^2 + cmu^2) < cl, a = cK / cl, b = cmu / cl (b = 0 now and then)
        const double cK = 0.05 + uni(), cmu = (c % 17 == 0) ? 0.0 : uni();
        const double cl = 2.0 * std::sqrt(cK * cK + cmu * cmu) / (0.05 + 0.949 * uni());
        const double a = cK / cl, b = cmu / cl;
        if (!lbmfx::mul_ok(a) || !lbmfx::mul_ok(b)) continue;
        const lbmfx::Mul A = lbmfx::make_mul(bits(a)), B = lbmfx::make_mul(bits(b));
        // inputs: a scale, then one of several patterns
        const int kind = (int)(c % 10);
        // kinds 5-8: near the largest and smallest exponents the fixed-point path takes, and past them
        const int s = (kind == 5) ? 1015 - (int)(next() % 8) : (kind == 6) ? -960 + (int)(next() % 8)
                    : (kind == 7) ? 1016 + (int)(next() % 8) : (kind == 8) ? -970 + (int)(next() % 8)
                                                                             : (int)(next() % 200) - 100;
        double f[4][5];
        for (int d = 0; d < 4; ++d)
            for (int k = 0; k < 5; ++k) {
                double v = gauss();
                if (kind == 1) v = std::ldexp(v, -(int)(next() % 70));              // wide spread
                if (kind == 2 && next() % 3 == 0) v = 0.0;                          // zeros
                if (kind == 3 && next() % 4 == 0) v = std::ldexp(gauss(), -1074 - s + 20);   // tiny / subnormal
                if (kind == 9) v = (next() & 1 ? 1.0 : -1.0) * (0.0625 + 0.9375 * uni());   // within 2^-4 of 1
                f[d][k] = std::ldexp(v, s);
            }
        if (kind == 4) {                                                           // exact cancellations
            for (int k = 0; k < 5; ++k) {
                f[3][k] = -f[1][k];
                if (k % 2) f[2][k] = -f[0][k];
            }
        }
        // body-load terms h = dt/2 b on every other node (zero on kind 9, whose inputs all convert
        // exactly): sometimes the largest input of the node
        const bool forced = (c & 1) && kind != 9;
        double hv[2] = {0.0, 0.0};
        if (forced)
            for (int q = 0; q < 2; ++q) hv[q] = std::ldexp(gauss() * ((next() % 4 == 0) ? 4.0 : 0.5), s);
        u64 in[4][5], out[4][5], Uo[5];
        const u64 hb[2] = {bits(hv[0]), bits(hv[1])};
        unsigned mx = 0;
        for (int d = 0; d < 4; ++d)
            for (int k = 0; k < 5; ++k) {
                in[d][k] = bits(f[d][k]);
                const unsigned h = (unsigned)(in[d][k] >> 32) & 0x7FFFFFFFu;
                mx = mx > h ? mx : h;
            }
        for (int q = 0; q < 2 && forced; ++q) {
            const unsigned h = (unsigned)(hb[q] >> 32) & 0x7FFFFFFFu;
            mx = mx > h ? mx : h;
        }
        const int E = (int)(mx >> 20);
        const bool ok = forced ? lbmfx::fx_node_h(in, hb, A, B, out, Uo) : lbmfx::fx_node(in, A, B, out, Uo);
        const bool expect = E >= 59 && E <= 2042;
        if (ok != expect) {
            ++fails;
            std::printf("fallback mismatch: E = %d, ok = %d\n", E, (int)ok);
            continue;
        }
        if (!ok) {
            ++fallback;
            continue;
        }
        ++taken;
        // exact (quad) evaluation of the same update
        q128 Q[4][5], U[5], rx[5], ry[5];
        for (int d = 0; d < 4; ++d)
            for (int k = 0; k < 5; ++k) Q[d][k] = (q128)f[d][k];
        for (int k = 0; k < 5; ++k) {
            rx[k] = Q[1][k] + Q[3][k];
            ry[k] = Q[0][k] + Q[2][k];
            U[k] = rx[k] + ry[k];
        }
        // the body load enters U and both pair sums of the two velocity components
        for (int q = 0; q < 2; ++q) {
            U[q] += (q128)hv[q];
            rx[q] += (q128)hv[q];
            ry[q] += (q128)hv[q];
        }
        const q128 qa = a, qb = b;
        q128 t[2][5];
        t[0][0] = qa * U[2] + qb * U[3] - Q[0][0];
        t[0][1] = qb * U[4] - Q[0][1];
        t[0][2] = qa * U[0] - Q[0][2];
        t[0][3] = qb * U[0] - Q[0][3];
        t[0][4] = qb * U[1] - Q[0][4];
        t[1][0] = qb * U[4] - Q[1][0];
        t[1][1] = qa * U[2] - qb * U[3] - Q[1][1];
        t[1][2] = qa * U[1] - Q[1][2];
        t[1][3] = -qb * U[1] - Q[1][3];
        t[1][4] = qb * U[0] - Q[1][4];
        q128 o[4][5];
        for (int k = 0; k < 5; ++k) {
            o[0][k] = U[k] / 2 + t[0][k];
            o[1][k] = U[k] / 2 + t[1][k];
            o[2][k] = rx[k] - o[0][k];
            o[3][k] = ry[k] - o[1][k];
        }
        // the FP64 operation sequence of the other kernels (fused multiply-adds, two roundings of U)
        double g[4][5], Ud[5], rxd[5], ryd[5];
        for (int k = 0; k < 5; ++k) {
            rxd[k] = f[1][k] + f[3][k] + (k < 2 ? hv[k] : 0.0);
            ryd[k] = f[0][k] + f[2][k] + (k < 2 ? hv[k] : 0.0);
            Ud[k] = f[1][k] + f[3][k] + ryd[k];
        }
        double td[2][5];
        td[0][0] = std::fma(a, Ud[2], std::fma(b, Ud[3], -f[0][0]));
        td[0][1] = std::fma(b, Ud[4], -f[0][1]);
        td[0][2] = std::fma(a, Ud[0], -f[0][2]);
        td[0][3] = std::fma(b, Ud[0], -f[0][3]);
        td[0][4] = std::fma(b, Ud[1], -f[0][4]);
        td[1][0] = std::fma(b, Ud[4], -f[1][0]);
        td[1][1] = std::fma(a, Ud[2], std::fma(-b, Ud[3], -f[1][1]));
        td[1][2] = std::fma(a, Ud[1], -f[1][2]);
        td[1][3] = std::fma(-b, Ud[1], -f[1][3]);
        td[1][4] = std::fma(b, Ud[0], -f[1][4]);
        for (int k = 0; k < 5; ++k) {
            g[0][k] = std::fma(0.5, Ud[k], td[0][k]);
            g[1][k] = std::fma(0.5, Ud[k], td[1][k]);
            g[2][k] = rxd[k] - g[0][k];
            g[3][k] = ryd[k] - g[1][k];
        }
        const double rho = std::ldexp(1.0, E - 1080);
        double efx = 0.0, efp = 0.0;   // largest absolute errors of the node's 20 outputs
        for (int d = 0; d < 4; ++d)
            for (int k = 0; k < 5; ++k) {
                const double got = dbl(out[d][k]);
                const double err = (double)qabs((q128)got - o[d][k]);
                // inputs within 2^5 of the node's largest convert exactly (kind 9): only the products
                // round, half a unit each, so each output is within half an ulp plus rho
                const double bound = 0.5 * ulp(got) + (kind == 9 ? 1.0 : forced ? 13.0 : 10.0) * rho;
                if (!(err <= bound)) {
                    if (fails < 20)
                        std::printf("case %ld (kind %d, E %d) out[%d][%d] = %.17g, exact %.17g, err %.3g > bound %.3g\n",
                                    c, kind, E, d, k, got, (double)o[d][k], err, bound);
                    ++fails;
                }
                if (bound > 0 && err / bound > worst) worst = err / bound;
                efx = err > efx ? err : efx;
                const double e2 = (double)qabs((q128)g[d][k] - o[d][k]);
                efp = e2 > efp ? e2 : efp;
            }
        for (int k = 0; k < 5; ++k) {
            const double got = dbl(Uo[k]);
            const double err = (double)qabs((q128)got - U[k]);
            if (!(err <= 0.5 * ulp(got) + (forced ? 5.0 : 4.0) * rho)) {
                if (fails < 20) std::printf("case %ld U[%d] = %.17g exact %.17g\n", c, k, got, (double)U[k]);
                ++fails;
            }
        }
        if (efx > efp) ++worse_than_fp64;
    }
    std::printf("fixed point taken %ld, fallback %ld, largest error / bound %.3f, nodes whose largest "
                "error exceeds the FP64 sequence's %ld\n", taken, fallback, worst, worse_than_fp64);
    std::printf("%ld cases, %ld failures\n", taken + fallback, fails);
    return fails ? 1 : 0;
}
