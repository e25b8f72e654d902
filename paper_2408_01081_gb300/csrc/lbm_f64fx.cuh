// FP64 node update (omega = 2, no body load) in exact 64-bit fixed-point arithmetic on
// the integer pipes, with one correctly rounded conversion to binary64 per output.
//
// The state stays binary64.  Per node, E is the largest exponent field of the 20 pulled
// populations (Eq. streaming), so every input is below 2^(Eu+1), Eu = E - 1023.  Each
// input becomes an integer X = floor(f / rho) with rho = 2^(Eu-57): exact for inputs
// within 2^5 of the node's largest, otherwise below rho (that is 2^-57 of the node's
// magnitude, against 2^-53 for one FP64 rounding there).  Then, exactly in integers:
//   pair sums and U (Eq. cond_eq):   ry = X(1,0) + X(-1,0),  rx = X(0,1) + X(0,-1),  U = rx + ry
//   the seven products a U0, a U1, a U2, b U0, b U1, b U3, b U4 of Phi_x / c and Phi_y / c
//     (Eq. feq; a = cK / c, b = cmu / c), each rounded to the nearest multiple of rho
//   T(1,0) = Phi_x(U) / c - X(1,0),  T(0,1) = Phi_y(U) / c - X(0,1)
//   2 f*(1,0) = U + 2 T(1,0),  2 f*(-1,0) = 2 rx - 2 f*(1,0)     (Eq. collision, omega = 2)
//   2 f*(0,1) = U + 2 T(0,1),  2 f*(0,-1) = 2 ry - 2 f*(0,1)
// and each doubled output is converted to binary64 by one round-to-nearest-even
// conversion and scaled by rho / 2 (an exact change of the exponent field).  With
// a, b < 1/2 (the CFL-like bound 2 sqrt(cK^2 + cmu^2) < c) every intermediate stays
// below 2^63 rho.  Error of every output against exact arithmetic on the same inputs:
// at most half an ulp of the output plus 10 rho (floors of the inputs: 4 rho in U;
// products: half a unit each plus their share of U's error); the FP64 operation
// sequence of the other kernels rounds U twice at up to 2^(Eu-50) each.
//
// The update is not applied (fx_node() returns false) when a node's E is at most 58 (every
// input below about 2^-964, or all zero: outputs could leave the normal range after
// scaling) or at least 2043 (inputs near overflow, infinite or NaN); callers then use the
// FP64 path.  Zero and subnormal inputs in a node with E >= 59 become 0 or -1 (their
// floor).  The header also compiles as plain C++ (host), where the results are checked
// against quad-precision arithmetic.
#pragma once

#ifdef __CUDACC__
#define FX_HD __host__ __device__ __forceinline__
#else
#define FX_HD inline
#endif

namespace lbmfx {

typedef unsigned long long u64;
typedef long long i64;

// multiplier c in [0, 1/2): c = M 2^-k with M = significand << 11 (top bit set), so that
// round(c U) = (mulhi(U, M) + 2^(k-65)) >> (k - 64) with k in [65, 127]
struct Mul {
    u64 m;      // 0 for c = 0
    int k;
    i64 half;   // 2^(k-65) (0 for c = 0)
};

FX_HD u64 bits_of_host(double x)
{
    union { double d; u64 u; } v;
    v.d = x;
    return v.u;
}

// host-side set-up (also usable on the device); c must be 0 or in [2^-60, 1/2)
FX_HD Mul make_mul(u64 cbits)
{
    Mul r;
    const u64 x = cbits & 0x7FFFFFFFFFFFFFFFull;
    if (x == 0) {
        r.m = 0;
        r.k = 65;
        r.half = 0;
        return r;
    }
    const int ec = (int)(x >> 52);
    r.m = ((x & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
    r.k = 1086 - ec;                                  // c = m 2^(ec - 1086)
    r.half = (i64)1 << (r.k - 65);
    return r;
}

// true when make_mul() may be used for c (the fixed-point step's precondition)
FX_HD bool mul_ok(double c)
{
    return c == 0.0 || (c >= 8.673617379884035e-19 /* 2^-60 */ && c < 0.5);
}

FX_HD u64 umulhi(u64 a, u64 b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (u64)(((unsigned __int128)a * b) >> 64);
#endif
}

// round(c U) for |U| < 2^62, to nearest, ties up
FX_HD i64 mul(i64 u, const Mul& c)
{
    // high half of the signed x unsigned product: the unsigned one minus m where u < 0
    const i64 hi = (i64)(umulhi((u64)u, c.m) - (u < 0 ? c.m : 0ull));
    return (hi + c.half) >> (c.k - 64);
}

FX_HD unsigned exp_field(u64 v) { return (unsigned)(v >> 52) & 0x7FFu; }

// X = floor(f / rho) for rho = 2^(E - 1080): the significand placed at bits 57..5
// (E = e), shifted right by E - e, signed
FX_HD i64 to_fixed(u64 v, int E)
{
    const unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
    const unsigned ha = hi & 0x7FFFFFFFu;
    // min(ha, 2^20) is the hidden bit for a normal number and lies within the fraction
    // bits otherwise (zero, subnormal)
    const unsigned hid = ha < 0x00100000u ? ha : 0x00100000u;
    const u64 sig = ((u64)((ha & 0x000FFFFFu) | hid) << 32) | lo;
    int r = E - (int)(ha >> 20);
    r = r < 63 ? r : 63;
    const i64 s = (i64)((int)hi >> 31);               // all ones for a negative input
    const i64 m = ((i64)(sig << 5) ^ s) - s;
    return m >> r;                                    // floor
}

// binary64 of y 2^s, s = add >> 20 (add = (E - 1081) << 20 for the doubled outputs): the
// conversion of y rounds to nearest even, then the exponent field moves by s exactly
// (y = 0 stays +0); the caller keeps the result's exponent field within 1..2046
FX_HD u64 from_fixed(i64 y, int add)
{
#ifdef __CUDA_ARCH__
    const u64 d = (u64)__double_as_longlong(__ll2double_rn(y));
#else
    const u64 d = bits_of_host((double)y);            // round to nearest even (default mode)
#endif
    const unsigned hi = (unsigned)(d >> 32);
    const unsigned hi2 = hi + (hi != 0u ? (unsigned)add : 0u);
    return ((u64)hi2 << 32) | (u64)(unsigned)d;
}

// E of a node: the largest exponent field among its 20 inputs
FX_HD int node_exp(const u64 (&in)[4][5])
{
    unsigned mx = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const unsigned h = (unsigned)(in[d][k] >> 32) & 0x7FFFFFFFu;
            mx = mx > h ? mx : h;
        }
    return (int)(mx >> 20);
}

// the same over the 20 inputs and the two body-load terms h
FX_HD int node_exp_h(const u64 (&in)[4][5], const u64 (&h)[2])
{
    const int e0 = node_exp(in);
    const int e1 = (int)((h[0] >> 52) & 0x7FFu), e2 = (int)((h[1] >> 52) & 0x7FFu);
    const int e12 = e1 > e2 ? e1 : e2;
    return e0 > e12 ? e0 : e12;
}

// nodes the fixed-point update takes (see above)
FX_HD bool exp_ok(int E) { return E >= 59 && E <= 2042; }

// The node update on bit patterns for a node with exp_ok(E): in[d][k] the pulled f*_(d)
// component k (d: (1,0), (0,1), (-1,0), (0,-1)), out the post-collision populations in the
// same order, Uout the moments U (rounded once each; only for the displacement helper).
// With HASH, h = [dt/2 b_x, dt/2 b_y] (binary64, E taken over them too) enters U's two
// velocity components (Eq. cond_eq with a body load); at omega = 2 the collision has no
// other body-load term, and f*_(1,0) + f*_(-1,0) = U - f_(1,0) - f_(-1,0) = rx + h, so the
// pair sums used for the opposite directions carry h too.  Every intermediate then stays
// below 46 * 2^(E - 1023) (U below 10, the doubled outputs below 46 times that), inside the
// 2^63 rho range, and each output is within half an ulp plus 13 rho of the exact update of
// its inputs (five floors in U, three in a pair sum with h).
template <bool HASH>
FX_HD void fx_update_h(const u64 (&in)[4][5], const u64 (&h)[2], int E, const Mul& A, const Mul& B,
                       u64 (&out)[4][5], u64 (&Uout)[5])
{
    i64 X[4][5];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k) X[d][k] = to_fixed(in[d][k], E);
    i64 rx[5], ry[5], U[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        rx[k] = X[1][k] + X[3][k];
        ry[k] = X[0][k] + X[2][k];
        U[k] = rx[k] + ry[k];
    }
    if (HASH) {
        const i64 h0 = to_fixed(h[0], E), h1 = to_fixed(h[1], E);
        U[0] += h0;
        U[1] += h1;
        rx[0] += h0;
        rx[1] += h1;
        ry[0] += h0;
        ry[1] += h1;
    }
    // Phi_x = [cK js + cmu jd, cmu jxy, cK vx, cmu vx, cmu vy],
    // Phi_y = [cmu jxy, cK js - cmu jd, cK vy, -cmu vy, cmu vx]  (U = [vx, vy, js, jd, jxy])
    const i64 aU0 = mul(U[0], A), aU1 = mul(U[1], A), aU2 = mul(U[2], A);
    const i64 bU0 = mul(U[0], B), bU1 = mul(U[1], B), bU3 = mul(U[3], B), bU4 = mul(U[4], B);
    i64 T[2][5];
    T[0][0] = aU2 + bU3 - X[0][0];
    T[0][1] = bU4 - X[0][1];
    T[0][2] = aU0 - X[0][2];
    T[0][3] = bU0 - X[0][3];
    T[0][4] = bU1 - X[0][4];
    T[1][0] = bU4 - X[1][0];
    T[1][1] = aU2 - bU3 - X[1][1];
    T[1][2] = aU1 - X[1][2];
    T[1][3] = -bU1 - X[1][3];
    T[1][4] = bU0 - X[1][4];
    const int add2 = (E - 1081) * (1 << 20);          // doubled outputs: rho / 2 = 2^(E - 1081)
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const i64 y0 = U[k] + T[0][k] + T[0][k];      // 2 f*(1,0)
        const i64 y1 = U[k] + T[1][k] + T[1][k];      // 2 f*(0,1)
        out[0][k] = from_fixed(y0, add2);
        out[1][k] = from_fixed(y1, add2);
        out[2][k] = from_fixed(rx[k] + rx[k] - y0, add2);   // 2 f*(-1,0)
        out[3][k] = from_fixed(ry[k] + ry[k] - y1, add2);   // 2 f*(0,-1)
        Uout[k] = from_fixed(U[k], add2 + (1 << 20));       // U itself: scale rho
    }
}

FX_HD void fx_update(const u64 (&in)[4][5], int E, const Mul& A, const Mul& B, u64 (&out)[4][5], u64 (&Uout)[5])
{
    const u64 h[2] = {0ull, 0ull};
    fx_update_h<false>(in, h, E, A, B, out, Uout);
}

// fx_update() where exp_ok(node_exp(in)); false (nothing written) otherwise
FX_HD bool fx_node(const u64 (&in)[4][5], const Mul& A, const Mul& B, u64 (&out)[4][5], u64 (&Uout)[5])
{
    const int E = node_exp(in);
    if (!exp_ok(E)) return false;
    fx_update(in, E, A, B, out, Uout);
    return true;
}

// the same with the body-load terms h (fx_update_h)
FX_HD bool fx_node_h(const u64 (&in)[4][5], const u64 (&h)[2], const Mul& A, const Mul& B, u64 (&out)[4][5],
                     u64 (&Uout)[5])
{
    const int E = node_exp_h(in, h);
    if (!exp_ok(E)) return false;
    fx_update_h<true>(in, h, E, A, B, out, Uout);
    return true;
}

}  // namespace lbmfx
