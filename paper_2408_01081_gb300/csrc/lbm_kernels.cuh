// Device code of the GB300 D2Q4^5 elastodynamics library (arXiv 2408.01081).
//
// State kept between steps: the post-collision populations f*(x, t) of every
// node, in structure-of-arrays planes [d*5 + k][y][pitch] of the storage type
// (d = velocity (1,0),(0,1),(-1,0),(0,-1); k = component of U = [vx, vy, js,
// jd, jxy]).  One fused kernel per time step pulls f(x, t+dt) = f*(x - c_ij dt, t)
// (Eq. streaming) or, for a missing link on a Dirichlet edge, the reflected
// D f*_{-i,-j}(x, t) + S_ij(x_b, t+dt/2) (Eq. bc_ansatz), forms U^num
// (Eq. cond_eq), collides with omega = 2 (Eqs. feq, collision) and writes
// f*(x, t+dt) back to the node's own, aligned position.
//
// With omega = 2 the collision of Eq. collision reads, per component k,
//     f*_ij = 1/2 U + i px + j py - f_ij,   px = Phi_x(U)/c, py = Phi_y(U)/c,
// and since the four outputs of one axis sum to U - (the other axis' pair),
//     f*_{-1,0} = (U - f_{1,0} - f_{-1,0}) - f*_{1,0},
//     f*_{0,-1} = (U - f_{0,1} - f_{0,-1}) - f*_{0,1}.
// That is 47 FP64 operations per node without forcing (35 additions, 12 fused
// multiply-adds), the FP64 ALU bound on GB300; the SPLIT variants compute part of
// the additions on the integer pipes (collide_split), exactly or faithfully rounded,
// or (split level 12, collide_fixed) the whole node update in exact 64-bit fixed point
// with one binary64 rounding per output (lbm_f64fx.cuh), which leaves only the output
// conversions on the FP64 pipe.
#pragma once

#include "lbm_f64emu.cuh"
#include "lbm_f64fx.cuh"
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbmk {

// ---------------------------------------------------------------------------
// storage formats
// ---------------------------------------------------------------------------
enum Kind { K_F64 = 0, K_F32 = 1, K_BF16 = 2, K_F16 = 3 };

template <int K> struct Fmt;
template <> struct Fmt<K_F64> {
    using E = double;  // element in memory
    using M = double;  // arithmetic type
    static __device__ __forceinline__ M ld(E e) { return e; }
    static __device__ __forceinline__ E st(M m) { return m; }
};
template <> struct Fmt<K_F32> {
    using E = float;
    using M = float;
    static __device__ __forceinline__ M ld(E e) { return e; }
    static __device__ __forceinline__ E st(M m) { return m; }
};
template <> struct Fmt<K_BF16> {
    using E = unsigned short;
    using M = float;
    static __device__ __forceinline__ M ld(E e) { return __bfloat162float(__ushort_as_bfloat16(e)); }
    static __device__ __forceinline__ E st(M m) { return __bfloat16_as_ushort(__float2bfloat16_rn(m)); }
};
template <> struct Fmt<K_F16> {
    using E = unsigned short;
    using M = float;
    static __device__ __forceinline__ M ld(E e) { return __half2float(__ushort_as_half(e)); }
    static __device__ __forceinline__ E st(M m) { return __half_as_ushort(__float2half_rn(m)); }
};

template <int BYTES> struct Raw;
template <> struct Raw<2> { using T = unsigned short; };
template <> struct Raw<4> { using T = unsigned int; };
template <> struct Raw<8> { using T = uint2; };
template <> struct Raw<16> { using T = uint4; };

// V consecutive elements from a (V * sizeof(E))-aligned address, one vector access.
// COHERENT loads bypass L1 (ld.global.cg): needed when the same launch wrote the
// data from other blocks (the persistent batch kernel); otherwise the read-only path.
template <int K, int V, bool COHERENT = false>
__device__ __forceinline__ void vload(const typename Fmt<K>::E* p, typename Fmt<K>::M (&out)[V])
{
    using E = typename Fmt<K>::E;
    using R = typename Raw<sizeof(E) * V>::T;
    union { R r; E e[V]; } u;
    u.r = COHERENT ? __ldcg(reinterpret_cast<const R*>(p)) : __ldg(reinterpret_cast<const R*>(p));
#pragma unroll
    for (int i = 0; i < V; ++i) out[i] = Fmt<K>::ld(u.e[i]);
}

template <int K, int V>
__device__ __forceinline__ void vstore(typename Fmt<K>::E* p, const typename Fmt<K>::M (&in)[V])
{
    using E = typename Fmt<K>::E;
    using R = typename Raw<sizeof(E) * V>::T;
    union { R r; E e[V]; } u;
#pragma unroll
    for (int i = 0; i < V; ++i) u.e[i] = Fmt<K>::st(in[i]);
    *reinterpret_cast<R*>(p) = u.r;
}

template <int K, bool COHERENT = false>
__device__ __forceinline__ typename Fmt<K>::M sload(const typename Fmt<K>::E* p)
{
    return Fmt<K>::ld(COHERENT ? __ldcg(p) : __ldg(p));
}

// ---------------------------------------------------------------------------
// arguments
// ---------------------------------------------------------------------------
struct StepArgs {
    const void* src;       // f*(t) planes
    void* dst;             // f*(t+dt) planes
    double* w;             // u*(t+dt) helper [2][ny][pitch], updated in place, or nullptr
    int nx, ny, pitch;
    long long plane;       // elements per plane = ny * pitch
    double a, b;           // cK / c, cmu / c
    double dt;
    // body load at t+dt: b_c(x_k, y_l) = sum_r X[r][k] Y[r][l] T[c][r]
    int R;
    const double* X;
    const double* Y;
    const double* T;       // row of the time t+dt: [2][R]
    const float* Xf;       // FP32 copies of the tables (reduced-precision formats)
    const float* Yf;
    const float* Tf;
    // Dirichlet data d/dt u_D at t + dt/2 on the wall midpoints, [2][nwall] or nullptr
    const double* g;
    int nwall;
    double omega;          // relaxation rate when the kernel is built for omega != 2
    double neq_scale;      // moment-space storage: scale of the stored deviations
    // FP32 copies for the FP32-arithmetic formats, converted once on the host (a conversion
    // from FP64 runs on the FP64 pipe, two per clock per SM)
    float af, bf;          // a, b
    float scale_f, inv_scale_f;   // neq_scale and its reciprocal (exact: a power of two)
    int* sat = nullptr;    // moment space, block floating point: set when a block saturated
};

// ---------------------------------------------------------------------------
// node arithmetic
// ---------------------------------------------------------------------------

// Collision with omega = 2 for one node.  f[d][k] pulled pre-collision values,
// U already holds sum_d f_d + dt/2 B; rx = U - f0 - f2, ry = U - f1 - f3 per component.
// Phi terms with the population subtracted: t[0][k] = Phi_x(U)_k / c - f_(1,0),k and
// t[1][k] = Phi_y(U)_k / c - f_(0,1),k, so that f*_(1,0) = U/2 + t[0], f*_(0,1) = U/2 + t[1];
// Phi_x = [cK js + cmu jd, cmu jxy, cK vx, cmu vx, cmu vy], Phi_y = [cmu jxy, cK js - cmu jd, cK vy, -cmu vy, cmu vx]
template <typename M>
__device__ __forceinline__ void collide_terms(const M (&f)[4][5], const M (&U)[5], M a, M b, M (&t)[2][5])
{
    t[0][0] = fma(a, U[2], fma(b, U[3], -f[0][0]));
    t[0][1] = fma(b, U[4], -f[0][1]);
    t[0][2] = fma(a, U[0], -f[0][2]);
    t[0][3] = fma(b, U[0], -f[0][3]);
    t[0][4] = fma(b, U[1], -f[0][4]);
    t[1][0] = fma(b, U[4], -f[1][0]);
    t[1][1] = fma(a, U[2], fma(-b, U[3], -f[1][1]));
    t[1][2] = fma(a, U[1], -f[1][2]);
    t[1][3] = fma(-b, U[1], -f[1][3]);
    t[1][4] = fma(b, U[0], -f[1][4]);
}

// omega = 2 collision (Eqs. feq, collision) in the 47-operation form:
// f*_(1,0) = U/2 + Phi_x/c - f_(1,0), f*_(0,1) = U/2 + Phi_y/c - f_(0,1), and the
// opposite directions from the pair sums, f*_(-1,0) = (f_(0,1) + f_(0,-1)) - f*_(1,0)
// (the pair sums of rx / ry are the other axis' populations), likewise (0,-1).
template <typename M>
__device__ __forceinline__ void collide(const M (&f)[4][5], const M (&U)[5], const M (&rx)[5],
                                        const M (&ry)[5], M a, M b, M (&o)[4][5])
{
    const M h = M(0.5);
    M t[2][5];
    collide_terms<M>(f, U, a, b, t);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        o[0][k] = fma(h, U[k], t[0][k]);
        o[1][k] = fma(h, U[k], t[1][k]);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        o[2][k] = rx[k] - o[0][k];   // (-1,0)
        o[3][k] = ry[k] - o[1][k];   // (0,-1)
    }
}

// the default split: the 10 pair sums and the 5 sums U on the integer pipes
constexpr unsigned long long kSplitDefaultMask = 0x001FFFC00ull;
// mask bit 63: the integer-pipe additions are rounded faithfully (emu_add_faithful_bits)
// instead of correctly
constexpr unsigned long long kSplitFaithful = 1ull << 63;
// mask bit 62: the whole node in exact fixed-point arithmetic on the integer pipes, one
// rounding per output (lbm_f64fx.cuh); not bit-identical to the FP64-pipe sequence
constexpr unsigned long long kSplitFixed = 1ull << 62;
// the fastest faithful split measured (opt-in, level 9): the 15 sums and the (-1,0)
// subtraction of component 0; its rounding is biased (half up, no sticky bit), which a
// long run shows as energy drift
constexpr unsigned long long kSplitFastMask = 0x001FFFC01ull | kSplitFaithful;

template <bool EMU, bool FAITHFUL>
__device__ __forceinline__ double split_add(double x, double y, bool& ok)
{
    if constexpr (EMU && FAITHFUL) return lbmemu::emu_add_f(x, y, ok);
    else if constexpr (EMU) return lbmemu::emu_add(x, y, ok);
    else return x + y;
}

template <bool EMU, bool FAITHFUL>
__device__ __forceinline__ double split_sub(double x, double y, bool& ok)
{
    if constexpr (EMU && FAITHFUL) return lbmemu::emu_sub_f(x, y, ok);
    else if constexpr (EMU) return lbmemu::emu_sub(x, y, ok);
    else return x - y;
}

template <bool EMU, bool FAITHFUL>
__device__ __forceinline__ double split_half_add(double u, double t, bool& ok)
{
    if constexpr (EMU && FAITHFUL) return lbmemu::emu_half_add_f(u, t, ok);
    else if constexpr (EMU) return lbmemu::emu_half_add(u, t, ok);
    else return fma(0.5, u, t);
}

// component k of the split update (the addition indices are compile-time constants)
template <unsigned long long M, int k>
__device__ __forceinline__ void split_sums(const double (&f)[4][5], double (&rx)[5], double (&ry)[5],
                                           double (&U)[5], bool& ok)
{
    constexpr bool FA = (M & kSplitFaithful) != 0;
    rx[k] = split_add<((M >> (10 + k)) & 1) != 0, FA>(f[1][k], f[3][k], ok);
    ry[k] = split_add<((M >> (15 + k)) & 1) != 0, FA>(f[0][k], f[2][k], ok);
    U[k] = split_add<((M >> (20 + k)) & 1) != 0, FA>(rx[k], ry[k], ok);
}

template <unsigned long long M, int k>
__device__ __forceinline__ void split_outputs(const double (&U)[5], const double (&rx)[5], const double (&ry)[5],
                                              const double (&t)[2][5], double (&o)[4][5], bool& ok)
{
    constexpr bool FA = (M & kSplitFaithful) != 0;
    o[0][k] = split_half_add<((M >> (25 + k)) & 1) != 0, FA>(U[k], t[0][k], ok);
    o[1][k] = split_half_add<((M >> (30 + k)) & 1) != 0, FA>(U[k], t[1][k], ok);
    o[2][k] = split_sub<((M >> k) & 1) != 0, FA>(rx[k], o[0][k], ok);
    o[3][k] = split_sub<((M >> (5 + k)) & 1) != 0, FA>(ry[k], o[1][k], ok);
}

// The same FP64 node update (pair sums, U, collision; no body load) with the
// additions selected by the bits of M computed exactly on the integer pipes
// (lbm_f64emu.cuh) and the rest, with the 12 fused multiply-adds, on the FP64
// pipe.  Bits: f*_(-1,0) (0-4), f*_(0,-1) (5-9), y-pair sums (10-14), x-pair sums
// (15-19), U (20-24), U/2 + t for (1,0) (25-29) and (0,1) (30-34), component k at
// offset k; bit 63 (kSplitFaithful) rounds the integer-pipe additions faithfully.
// Without it every result is bit-identical to collide<double>; with it each such
// addition is within (1/2 + 2^-9) ulp of the exact sum.  A lane whose operands leave
// the integer path (a subnormal, infinite or NaN result) recomputes on the FP64 pipe.
template <unsigned long long M>
__device__ __forceinline__ void collide_split(const double (&f)[4][5], double a, double b, double (&U)[5],
                                              double (&o)[4][5]);

// The node update in exact fixed-point arithmetic (lbmfx::fx_node): a = cK / c, b = cmu / c
// in [0, 1/2) (the CFL-like bound) and not below 2^-60 unless zero (checked by the host).
// A node outside the fixed-point range (its largest input below about 2^-964 or above
// 2^1019, or not finite) runs the exact split collision instead; the choice depends on
// the node's own inputs only.
__device__ __forceinline__ void collide_fixed(const double (&f)[4][5], double a, double b, double (&U)[5],
                                              double (&o)[4][5])
{
    const lbmfx::Mul A = lbmfx::make_mul(lbmemu::bits_of(a)), B = lbmfx::make_mul(lbmemu::bits_of(b));
    lbmfx::u64 in[4][5], out[4][5], Uo[5];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k) in[d][k] = lbmemu::bits_of(f[d][k]);
    const int E = lbmfx::node_exp(in);
    const bool ok = lbmfx::exp_ok(E);
    if (__all_sync(0xffffffffu, ok)) {
        lbmfx::fx_update(in, E, A, B, out, Uo);
    } else {
        // warp-uniform branch: every lane runs the split collision (it synchronises the warp
        // itself); the lanes inside the fixed-point range then overwrite its results
        double U2[5], o2[4][5];
        collide_split<kSplitDefaultMask>(f, a, b, U2, o2);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            Uo[k] = lbmemu::bits_of(U2[k]);
#pragma unroll
            for (int d = 0; d < 4; ++d) out[d][k] = lbmemu::bits_of(o2[d][k]);
        }
        if (ok) lbmfx::fx_update(in, E, A, B, out, Uo);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        U[k] = lbmemu::double_of(Uo[k]);
#pragma unroll
        for (int d = 0; d < 4; ++d) o[d][k] = lbmemu::double_of(out[d][k]);
    }
}

// The fixed-point node update with a body load (b_x, b_y at the node, hdt = dt/2): U of the two
// velocity components gains h = hdt b (Eq. cond_eq).  Nodes outside the fixed-point range run
// the FP64 sequence of step_kernel's body-load path (the body load folded into the pair sums
// by fused multiply-adds, then the 47-operation collision).
__device__ __forceinline__ void collide_fixed_forced(const double (&f)[4][5], double bx, double by, double hdt,
                                                     double a, double b, double (&U)[5], double (&o)[4][5])
{
    const lbmfx::Mul A = lbmfx::make_mul(lbmemu::bits_of(a)), B = lbmfx::make_mul(lbmemu::bits_of(b));
    lbmfx::u64 in[4][5], out[4][5], Uo[5];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k) in[d][k] = lbmemu::bits_of(f[d][k]);
    const lbmfx::u64 h[2] = {lbmemu::bits_of(hdt * bx), lbmemu::bits_of(hdt * by)};
    const int E = lbmfx::node_exp_h(in, h);
    const bool ok = lbmfx::exp_ok(E);
    if (__all_sync(0xffffffffu, ok)) {
        lbmfx::fx_update_h<true>(in, h, E, A, B, out, Uo);
    } else {
        double rx[5], ry[5], U2[5], o2[4][5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            rx[k] = f[1][k] + f[3][k];
            ry[k] = f[0][k] + f[2][k];
        }
        rx[0] = fma(hdt, bx, rx[0]);
        rx[1] = fma(hdt, by, rx[1]);
        ry[0] = fma(hdt, bx, ry[0]);
        ry[1] = fma(hdt, by, ry[1]);
        U2[0] = rx[0] + (f[0][0] + f[2][0]);
        U2[1] = rx[1] + (f[0][1] + f[2][1]);
#pragma unroll
        for (int k = 2; k < 5; ++k) U2[k] = rx[k] + ry[k];
        collide<double>(f, U2, rx, ry, a, b, o2);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            Uo[k] = lbmemu::bits_of(U2[k]);
#pragma unroll
            for (int d = 0; d < 4; ++d) out[d][k] = lbmemu::bits_of(o2[d][k]);
        }
        if (ok) lbmfx::fx_update_h<true>(in, h, E, A, B, out, Uo);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        U[k] = lbmemu::double_of(Uo[k]);
#pragma unroll
        for (int d = 0; d < 4; ++d) o[d][k] = lbmemu::double_of(out[d][k]);
    }
}

template <unsigned long long M>
__device__ __forceinline__ void collide_split(const double (&f)[4][5], double a, double b, double (&U)[5],
                                              double (&o)[4][5])
{
    if constexpr ((M & kSplitFixed) != 0) {
        collide_fixed(f, a, b, U, o);
        return;
    }
    bool ok = true;
    double rx[5], ry[5];
    split_sums<M, 0>(f, rx, ry, U, ok);
    split_sums<M, 1>(f, rx, ry, U, ok);
    split_sums<M, 2>(f, rx, ry, U, ok);
    split_sums<M, 3>(f, rx, ry, U, ok);
    split_sums<M, 4>(f, rx, ry, U, ok);
    double t[2][5];
    collide_terms<double>(f, U, a, b, t);
    split_outputs<M, 0>(U, rx, ry, t, o, ok);
    split_outputs<M, 1>(U, rx, ry, t, o, ok);
    split_outputs<M, 2>(U, rx, ry, t, o, ok);
    split_outputs<M, 3>(U, rx, ry, t, o, ok);
    split_outputs<M, 4>(U, rx, ry, t, o, ok);
    if (__any_sync(0xffffffffu, !ok)) {
        if (!ok) {
            // the copies through volatile asm keep the compiler from computing this
            // FP64 path speculatively on every lane
            double g[4][5], ga, gb;
#pragma unroll
            for (int d = 0; d < 4; ++d)
#pragma unroll
                for (int k = 0; k < 5; ++k) asm volatile("mov.b64 %0, %1;" : "=d"(g[d][k]) : "d"(f[d][k]));
            asm volatile("mov.b64 %0, %1;" : "=d"(ga) : "d"(a));
            asm volatile("mov.b64 %0, %1;" : "=d"(gb) : "d"(b));
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                rx[k] = g[1][k] + g[3][k];
                ry[k] = g[0][k] + g[2][k];
                U[k] = rx[k] + ry[k];
            }
            collide<double>(g, U, rx, ry, ga, gb, o);
        }
    }
}

// S_ij of Eq. bc_s for wall data (gx, gy) and velocity (i, j); the j rows carry
// the 1/c of the equilibrium difference (a = cK/c, b = cmu/c).
__device__ __forceinline__ void wall_source(int i, int j, double gx, double gy, double a, double b,
                                            double (&S)[5])
{
    S[0] = 0.5 * gx;
    S[1] = 0.5 * gy;
    S[2] = a * (i * gx + j * gy);
    S[3] = b * (i * gx - j * gy);
    S[4] = b * (j * gx + i * gy);
}

// ---------------------------------------------------------------------------
// fused pull-collide step: one thread = V consecutive nodes of one row
// grid: (ceil(ceil(nx/V) / blockDim.x), ny)
// ---------------------------------------------------------------------------
#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 1
#endif
#ifndef LBM_SPLIT_MIN_BLOCKS
#define LBM_SPLIT_MIN_BLOCKS 3      // 80 registers: more warps to overlap the two pipes
#endif

template <int K, int V, bool DIRICHLET, bool FORCING, bool TRACK, bool OMEGA = false, unsigned long long SPLIT = 0>
__global__ void __launch_bounds__(256, SPLIT > 0 ? LBM_SPLIT_MIN_BLOCKS : LBM_STEP_MIN_BLOCKS)
step_kernel(StepArgs A)
{
    using E = typename Fmt<K>::E;
    using M = typename Fmt<K>::M;
    const int y = blockIdx.y;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    const int nchunk = (A.nx + V - 1) / V;
    const bool active = cx < nchunk;
    const int x0 = (active ? cx : nchunk - 1) * V;   // inactive lanes mirror a valid chunk
    const int nx = A.nx, ny = A.ny;
    const long long plane = A.plane;
    const E* __restrict__ src = static_cast<const E*>(A.src);
    E* __restrict__ dst = static_cast<E*>(A.dst);
    const int lane = threadIdx.x & 31;

    // rows the +y and -y planes are pulled from; on a Dirichlet edge row the
    // missing link reflects the node's own opposite plane instead
    const bool bot = DIRICHLET && (y == 0);
    const bool top = DIRICHLET && (y == ny - 1);
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;

    M P0[5][V], P1[5][V], P2[5][V], P3[5][V];   // pulled f_d (edge links patched below)
    M own0[5][V], own2[5][V];                    // f*_{(1,0)}, f*_{(-1,0)} of the own chunk
    const long long row = (long long)y * A.pitch + x0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        vload<K, V>(src + (0 * 5 + k) * plane + row, own0[k]);
        vload<K, V>(src + (2 * 5 + k) * plane + row, own2[k]);
        if (bot) vload<K, V>(src + (3 * 5 + k) * plane + row, P1[k]);
        else     vload<K, V>(src + (1 * 5 + k) * plane + (long long)ym * A.pitch + x0, P1[k]);
        if (top) vload<K, V>(src + (1 * 5 + k) * plane + row, P3[k]);
        else     vload<K, V>(src + (3 * 5 + k) * plane + (long long)yp * A.pitch + x0, P3[k]);
    }
    // x-planes: shift by one node through the neighbouring lanes
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;        // source of P0[0]
    const bool left_in_lane = (lane > 0) && (x0 > 0);
    const bool right_in_lane = (lane < 31) && (x0 + V < nx) && (cx + 1 < nchunk);
    const int xr = (x0 + V >= nx) ? 0 : x0 + V;        // source of P2[V-1] (periodic)
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        M l = __shfl_up_sync(0xffffffffu, own0[k][V - 1], 1);
        M r = __shfl_down_sync(0xffffffffu, own2[k][0], 1);
        if (!left_in_lane) l = sload<K>(src + (0 * 5 + k) * plane + (long long)y * A.pitch + xl);
        if (!right_in_lane) r = sload<K>(src + (2 * 5 + k) * plane + (long long)y * A.pitch + xr);
        P0[k][0] = l;
#pragma unroll
        for (int e = 1; e < V; ++e) P0[k][e] = own0[k][e - 1];
#pragma unroll
        for (int e = 0; e < V - 1; ++e) P2[k][e] = own2[k][e + 1];
        P2[k][V - 1] = r;
    }
    // ragged row end: the node nx-1 may sit inside the chunk; its (-1,0) source wraps to x = 0
    if (!DIRICHLET && x0 + V > nx && x0 <= nx - 1) {
        const int e = nx - 1 - x0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const M r0 = sload<K>(src + (2 * 5 + k) * plane + (long long)y * A.pitch + 0);
#pragma unroll
            for (int q = 0; q < V; ++q)
                if (q == e) P2[k][q] = r0;
        }
    }

    M a, b;
    if constexpr (sizeof(M) == 4) {
        a = A.af;
        b = A.bf;
    } else {
        a = A.a;
        b = A.b;
    }
    M out[4][5][V];
    double wv[2][V];
    double bxs[V], bys[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int x = x0 + e;
        bxs[e] = 0.0;
        bys[e] = 0.0;
        M f[4][5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            f[0][k] = P0[k][e];
            f[1][k] = P1[k][e];
            f[2][k] = P2[k][e];
            f[3][k] = P3[k][e];
        }
        if (DIRICHLET) {
            // missing incoming links: f_ij = D f*_{-i,-j}(x) + S_ij(x_b, t + dt/2), in FP64
            const bool le = (x == 0), ri = (x == nx - 1);
            if (le || ri || bot || top) {
                const double Dk[5] = {-1.0, -1.0, 1.0, 1.0, 1.0};
                double S[5];
                if (le) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g) { gx = A.g[y]; gy = A.g[A.nwall + y]; }
                    wall_source(1, 0, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[0][k] = M(Dk[k] * (double)own2[k][e] + S[k]);
                }
                if (ri) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g) { gx = A.g[ny + y]; gy = A.g[A.nwall + ny + y]; }
                    wall_source(-1, 0, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[2][k] = M(Dk[k] * (double)own0[k][e] + S[k]);
                }
                if (bot) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g && x < nx) { gx = A.g[2 * ny + x]; gy = A.g[A.nwall + 2 * ny + x]; }
                    wall_source(0, 1, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[1][k] = M(Dk[k] * (double)P1[k][e] + S[k]);
                }
                if (top) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g && x < nx) { gx = A.g[2 * ny + nx + x]; gy = A.g[A.nwall + 2 * ny + nx + x]; }
                    wall_source(0, -1, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[3][k] = M(Dk[k] * (double)P3[k][e] + S[k]);
                }
            }
        }
        M U[5], rx[5], ry[5];
        M o[4][5];
        if constexpr (SPLIT > 0 && sizeof(M) == 8 && !FORCING && !OMEGA) {
            collide_split<SPLIT>(f, a, b, U, o);
        } else if constexpr ((SPLIT & kSplitFixed) != 0 && sizeof(M) == 8 && FORCING && !OMEGA) {
            // body load in FP64 as below, then the fixed-point node update with it
            double bx = 0.0, by = 0.0;
            if (x < nx) {
                for (int r = 0; r < A.R; ++r) {
                    const double xy = A.X[(long long)r * nx + x] * A.Y[(long long)r * ny + y];
                    bx = fma(xy, A.T[r], bx);
                    by = fma(xy, A.T[A.R + r], by);
                }
            }
            collide_fixed_forced(f, bx, by, 0.5 * A.dt, a, b, U, o);
        } else {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const M sx = f[0][k] + f[2][k];
                const M sy = f[1][k] + f[3][k];
                rx[k] = sy;
                ry[k] = sx;
            }
            if (FORCING) {
                // body load in the arithmetic type (FP32 tables for the reduced formats)
                M bx = M(0), by = M(0);
                if (x < nx) {
                    if constexpr (sizeof(M) == 8) {
                        for (int r = 0; r < A.R; ++r) {
                            const M xy = A.X[(long long)r * nx + x] * A.Y[(long long)r * ny + y];
                            bx = fma(xy, A.T[r], bx);
                            by = fma(xy, A.T[A.R + r], by);
                        }
                    } else {
                        for (int r = 0; r < A.R; ++r) {
                            const M xy = A.Xf[(long long)r * nx + x] * A.Yf[(long long)r * ny + y];
                            bx = fma(xy, A.Tf[r], bx);
                            by = fma(xy, A.Tf[A.R + r], by);
                        }
                    }
                }
                bxs[e] = (double)bx;
                bys[e] = (double)by;
                rx[0] = fma(M(0.5 * A.dt), bx, rx[0]);
                rx[1] = fma(M(0.5 * A.dt), by, rx[1]);
                ry[0] = fma(M(0.5 * A.dt), bx, ry[0]);
                ry[1] = fma(M(0.5 * A.dt), by, ry[1]);
                U[0] = rx[0] + (f[0][0] + f[2][0]);
                U[1] = rx[1] + (f[0][1] + f[2][1]);
#pragma unroll
                for (int k = 2; k < 5; ++k) U[k] = rx[k] + ry[k];
            } else {
#pragma unroll
                for (int k = 0; k < 5; ++k) U[k] = rx[k] + ry[k];
            }
            collide<M>(f, U, rx, ry, a, b, o);
        }
        if (OMEGA) {
            // omega f^eq + (1 - omega) f + dt (2 - omega) W B  =  (omega/2) o + (1 - omega/2) f + forcing,
            // with o the omega = 2 result and W = 1/8
            const M h = M(0.5 * A.omega);
            const M fw = M(A.dt * (2.0 - A.omega) * 0.125);
#pragma unroll
            for (int d = 0; d < 4; ++d)
#pragma unroll
                for (int k = 0; k < 5; ++k) o[d][k] = fma(h, o[d][k] - f[d][k], f[d][k]);
            if (FORCING) {
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    o[d][0] = fma(fw, M(bxs[e]), o[d][0]);
                    o[d][1] = fma(fw, M(bys[e]), o[d][1]);
                }
            }
        }
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int k = 0; k < 5; ++k) out[d][k][e] = o[d][k];
        if (TRACK) {
            wv[0][e] = (double)U[0];
            wv[1][e] = (double)U[1];
        }
    }
    if (!active) return;
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k) vstore<K, V>(dst + (d * 5 + k) * plane + row, out[d][k]);
    if (TRACK) {
        // u*(t+2dt) = u*(t+dt) + dt v(t+dt)  (steps 1(b) and 2(c) of the summary, Sec. 3.6)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            double* wp = A.w + (long long)c * plane + row;
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (x0 + e < nx) wp[e] = fma(A.dt, wv[c][e], wp[e]);
        }
    }
}

}  // namespace lbmk

namespace lbmk {

// ---------------------------------------------------------------------------
// FP64 per-node helpers for initialisation, output and reductions
// ---------------------------------------------------------------------------
struct NodeArgs {
    const void* S;         // f* planes at the current time (storage type)
    void* Sout;            // f* planes to write (init / set_populations)
    double* w;             // u*(t+dt) [2][ny][pitch] or nullptr
    int nx, ny, pitch;     // ny: the rows these kernels visit (a slab's own rows, not its halo rows)
    int yo = 0;            // storage row of visited row 0 (1 for a slab with a halo row below, else 0)
    long long plane;
    double a, b;           // cK/c, cmu/c
    double cK, cmu;        // wave speeds (stress output)
    double dt, c;
    int R;                 // body load tables at the current time (R = 0: none)
    const double* X;
    const double* Y;
    const double* T;       // [2][R]
    double k[4][25];       // symmetrizer blocks k_ij = g_ij^{-1}
    double omega;          // relaxation rate (2 for the paper's scheme; never 1)
    double neq_scale;      // moment-space storage: scale of the stored deviations
    float* measure;        // moment-space storage: if set, store_node records max |deviation| instead
    int* sat = nullptr;    // moment space, block floating point: set when a stored block saturated
};

// moment-space storage (lbm_ms.cuh)
template <int K> __device__ void ms_load_node(const NodeArgs& A, int x, int y, double (&S)[4][5]);
template <int K> __device__ void ms_store_node(const NodeArgs& A, int x, int y, const double (&S)[4][5]);

__device__ __forceinline__ void body_load(const NodeArgs& A, int x, int y, double& bx, double& by)
{
    bx = 0.0;
    by = 0.0;
    for (int r = 0; r < A.R; ++r) {
        const double xy = A.X[(long long)r * A.nx + x] * A.Y[(long long)r * A.ny + y];
        bx = fma(xy, A.T[r], bx);
        by = fma(xy, A.T[A.R + r], by);
    }
}

template <int K>
__device__ __forceinline__ void load_node(const NodeArgs& A, int x, int y, double (&S)[4][5])
{
    if constexpr (K >= 4) {
        ms_load_node<K>(A, x, y, S);
    } else {
    using E = typename Fmt<K>::E;
    const E* p = static_cast<const E*>(A.S);
    const long long off = (long long)(y + A.yo) * A.pitch + x;
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k) S[d][k] = (double)Fmt<K>::ld(p[(d * 5 + k) * A.plane + off]);
    }
}

template <int K>
__device__ __forceinline__ void store_node(const NodeArgs& A, int x, int y, const double (&S)[4][5])
{
    if constexpr (K >= 4) {
        ms_store_node<K>(A, x, y, S);
    } else {
    using E = typename Fmt<K>::E;
    using M = typename Fmt<K>::M;
    E* p = static_cast<E*>(A.Sout);
    const long long off = (long long)(y + A.yo) * A.pitch + x;
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k) p[(d * 5 + k) * A.plane + off] = Fmt<K>::st((M)S[d][k]);
    }
}

// 2 g_ij U - f_ij for all four velocities, with U = sum_d f_d + shift (per component).
// As collision (shift = +dt/2 B) it maps f to f*; as its inverse (shift = -dt/2 B) f* to f.
__device__ __forceinline__ void reflect_node(const double (&f)[4][5], const double (&shift)[5],
                                             double a, double b, double (&o)[4][5], double (&U)[5])
{
    double rx[5], ry[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        rx[k] = (f[1][k] + f[3][k]) + shift[k];
        ry[k] = (f[0][k] + f[2][k]) + shift[k];
        U[k] = rx[k] + (f[0][k] + f[2][k]);
    }
    collide<double>(f, U, rx, ry, a, b, o);
}

// Collision with relaxation rate omega (Eq. collision): f* = (omega/2)(2 g U - f) + (1 - omega/2) f
// + dt (2 - omega) W B with W = 1/8 and U = sum f + dt/2 B.
__device__ __forceinline__ void collide_node(const double (&f)[4][5], double bx, double by, double dt, double omega,
                                             double a, double b, double (&o)[4][5], double (&U)[5])
{
    const double shift[5] = {0.5 * dt * bx, 0.5 * dt * by, 0.0, 0.0, 0.0};
    reflect_node(f, shift, a, b, o, U);
    if (omega != 2.0) {
        const double h = 0.5 * omega, fw = dt * (2.0 - omega) * 0.125;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
#pragma unroll
            for (int k = 0; k < 5; ++k) o[d][k] = fma(h, o[d][k] - f[d][k], f[d][k]);
            o[d][0] = fma(fw, bx, o[d][0]);
            o[d][1] = fma(fw, by, o[d][1]);
        }
    }
}

// Inverse of collide_node: U = sum f* - dt/2 B for every omega; then
// f = (f* - (omega/2) (2 g U) - dt (2 - omega) W B) / (1 - omega), which for omega = 2 is 2 g U - f*.
__device__ __forceinline__ void uncollide_node(const double (&S)[4][5], double bx, double by, double dt,
                                               double omega, double a, double b, double (&f)[4][5], double (&U)[5])
{
    const double shift[5] = {-0.5 * dt * bx, -0.5 * dt * by, 0.0, 0.0, 0.0};
    reflect_node(S, shift, a, b, f, U);       // f = 2 g U - f*
    if (omega != 2.0) {
        const double h = 0.5 * omega, fw = dt * (2.0 - omega) * 0.125, inv = 1.0 / (1.0 - omega);
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const double two_gU = f[d][k] + S[d][k];
                double v = S[d][k] - h * two_gU;
                if (k == 0) v -= fw * bx;
                if (k == 1) v -= fw * by;
                f[d][k] = v * inv;
            }
    }
}

// scaled fluxes phi_x(v) = Phi_x(v)/c, phi_y(v) = Phi_y(v)/c (Eq. system)
__device__ __forceinline__ void phix(const double (&v)[5], double a, double b, double (&o)[5])
{
    o[0] = a * v[2] + b * v[3];
    o[1] = b * v[4];
    o[2] = a * v[0];
    o[3] = b * v[0];
    o[4] = b * v[1];
}
__device__ __forceinline__ void phiy(const double (&v)[5], double a, double b, double (&o)[5])
{
    o[0] = b * v[4];
    o[1] = a * v[2] - b * v[3];
    o[2] = a * v[1];
    o[3] = -b * v[1];
    o[4] = b * v[0];
}

// Eq. ic_second written with the scaled fluxes (Phi/c), then the first collision.
// Inputs are dense [5][ny][nx] (U0, dU0dx, dU0dy), [2][ny][nx] (B0, u0; may be null).
// HASB: B0 is given (without it every body-load term is zero and skipped).
template <int K, bool HASB>
__global__ void init_kernel(NodeArgs A, const double* __restrict__ U0, const double* __restrict__ Ux,
                            const double* __restrict__ Uy, const double* __restrict__ B0,
                            const double* __restrict__ u0)
{
    const long long n = (long long)A.nx * A.ny;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(id % A.nx), y = (int)(id / A.nx);
        double u[5], ux[5], uy[5], bv[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            u[k] = U0[k * n + id];
            ux[k] = Ux[k * n + id];
            uy[k] = Uy[k * n + id];
        }
        if (HASB) {
            bv[0] = B0[id];
            bv[1] = B0[n + id];
        }
        const double a = A.a, b = A.b, c = A.c;
        // Phi/c is linear, so px(px u_x) + px(py u_y) = px(px u_x + py u_y), likewise py
        double pxu[5], pyu[5], pxb[5], pyb[5], pxx[5], pyy[5], sxy[5], pxs[5], pys[5];
        phix(u, a, b, pxu);
        phiy(u, a, b, pyu);
        if (HASB) {
            phix(bv, a, b, pxb);
            phiy(bv, a, b, pyb);
        }
        phix(ux, a, b, pxx);
        phiy(uy, a, b, pyy);
#pragma unroll
        for (int k = 0; k < 5; ++k) sxy[k] = pxx[k] + pyy[k];
        phix(sxy, a, b, pxs);
        phiy(sxy, a, b, pys);
        // per velocity (i, j), with the zero and unit factors of i, j written out:
        //   f = 1/4 (u + 2 (i px u + j py u)) - dt/8 [ b + 2 (i px b + j py b)
        //       + c (i u_x + (2 i^2 - 1) px u_x - 2 (i px + j py) px u_x)
        //       + c (j u_y + (2 j^2 - 1) py u_y - 2 (i px + j py) py u_y) ]
        // so for (+-1, 0): 1/4 u +- 1/2 px u - dt/8 [ b +- 2 px b + c (px u_x - py u_y)
        //                  +- c (u_x - 2 px (px u_x + py u_y)) ], and (0, +-1) with x, y exchanged
        double f[4][5];
        const double h = 0.125 * A.dt;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const double qu = 0.25 * u[k];
            const double sx = c * (pxx[k] - pyy[k]);                     // the y rows carry -sx
            const double ex = 0.5 * pxu[k], ey = 0.5 * pyu[k];
            const double dxp = c * fma(-2.0, pxs[k], ux[k]);
            const double dyp = c * fma(-2.0, pys[k], uy[k]);
            double gxp = sx + dxp, gxm = sx - dxp, gyp = dyp - sx, gym = -sx - dyp;
            if (HASB) {
                gxp += bv[k] + 2.0 * pxb[k];
                gxm += bv[k] - 2.0 * pxb[k];
                gyp += bv[k] + 2.0 * pyb[k];
                gym += bv[k] - 2.0 * pyb[k];
            }
            f[0][k] = fma(-h, gxp, qu + ex);
            f[2][k] = fma(-h, gxm, qu - ex);
            f[1][k] = fma(-h, gyp, qu + ey);
            f[3][k] = fma(-h, gym, qu - ey);
        }
        double S[4][5], U[5];
        collide_node(f, bv[0], bv[1], A.dt, A.omega, a, b, S, U);
        store_node<K>(A, x, y, S);
        if (A.w) {
            // u*(dt) = u*(0) + dt v(0) with u*(0) = u0 - dt/2 v(0)  (Eq. trapezoidal)
            const long long off = (long long)(y + A.yo) * A.pitch + x;
            const double u0x = u0 ? u0[id] : 0.0, u0y = u0 ? u0[n + id] : 0.0;
            A.w[off] = u0x + 0.5 * A.dt * U[0];
            A.w[A.plane + off] = u0y + 0.5 * A.dt * U[1];
        }
    }
}

// pre-collision f(t) (and U^num(t)) of one node from the stored f*(t)
template <int K>
__device__ __forceinline__ void node_state(const NodeArgs& A, int x, int y, double (&f)[4][5], double (&U)[5])
{
    double S[4][5];
    load_node<K>(A, x, y, S);
    double bx = 0.0, by = 0.0;
    if (A.R > 0) body_load(A, x, y, bx, by);
    uncollide_node(S, bx, by, A.dt, A.omega, A.a, A.b, f, U);
}

// ten output fields (Sec. 3.5) of one node
template <int K>
__device__ __forceinline__ void node_outputs(const NodeArgs& A, int x, int y, double (&o)[10])
{
    double f[4][5], U[5];
    node_state<K>(A, x, y, f, U);
#pragma unroll
    for (int k = 0; k < 5; ++k) o[k] = U[k];
    if (A.w) {
        // u(t) = u*(t) + dt/2 v(t) and the stored helper is u*(t) + dt v(t)
        const long long off = (long long)(y + A.yo) * A.pitch + x;
        o[5] = A.w[off] - 0.5 * A.dt * U[0];
        o[6] = A.w[A.plane + off] - 0.5 * A.dt * U[1];
    } else {
        o[5] = 0.0;
        o[6] = 0.0;
    }
    o[7] = -(A.cK * U[2] + A.cmu * U[3]);   // Eq. sigma_num
    o[8] = -(A.cK * U[2] - A.cmu * U[3]);
    o[9] = -(A.cmu * U[4]);
}

template <int K>
__global__ void moments_kernel(NodeArgs A, double* __restrict__ out)
{
    const long long n = (long long)A.nx * A.ny;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(id % A.nx), y = (int)(id / A.nx);
        double o[10];
        node_outputs<K>(A, x, y, o);
#pragma unroll
        for (int q = 0; q < 10; ++q) out[q * n + id] = o[q];
    }
}

template <int K>
__global__ void get_populations_kernel(NodeArgs A, double* __restrict__ fout, double* __restrict__ ustar)
{
    const long long n = (long long)A.nx * A.ny;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(id % A.nx), y = (int)(id / A.nx);
        double f[4][5], U[5];
        node_state<K>(A, x, y, f, U);
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int k = 0; k < 5; ++k) fout[(d * 5 + k) * n + id] = f[d][k];
        if (ustar) {
            const long long off = (long long)(y + A.yo) * A.pitch + x;
            ustar[id] = A.w ? A.w[off] - A.dt * U[0] : 0.0;
            ustar[n + id] = A.w ? A.w[A.plane + off] - A.dt * U[1] : 0.0;
        }
    }
}

template <int K>
__global__ void set_populations_kernel(NodeArgs A, const double* __restrict__ fin, const double* __restrict__ ustar)
{
    const long long n = (long long)A.nx * A.ny;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(id % A.nx), y = (int)(id / A.nx);
        double f[4][5];
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int k = 0; k < 5; ++k) f[d][k] = fin[(d * 5 + k) * n + id];
        double bx = 0.0, by = 0.0;
        if (A.R > 0) body_load(A, x, y, bx, by);
        double S[4][5], U[5];
        collide_node(f, bx, by, A.dt, A.omega, A.a, A.b, S, U);
        store_node<K>(A, x, y, S);
        if (A.w) {
            const long long off = (long long)(y + A.yo) * A.pitch + x;
            A.w[off] = (ustar ? ustar[id] : 0.0) + A.dt * U[0];
            A.w[A.plane + off] = (ustar ? ustar[n + id] : 0.0) + A.dt * U[1];
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 reductions: per-thread accumulation, warp shuffles, one partial per block
// in a scratch array, then a single-block pass in fixed order (deterministic)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// block reduction of NV values; is_max[q] selects max instead of sum; result valid in thread 0
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], const bool (&is_max)[NV])
{
    __shared__ double red[32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = is_max[q] ? warp_max(v[q]) : warp_sum(v[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[wid][q] = v[q];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double t = (lane < nw) ? red[lane][q] : 0.0;
            v[q] = is_max[q] ? warp_max(t) : warp_sum(t);
        }
    }
}

template <int K>
__device__ __forceinline__ double node_energy(const NodeArgs& A, int x, int y)
{
    double f[4][5], U[5];
    node_state<K>(A, x, y, f, U);
    double e = 0.0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
#pragma unroll
        for (int p = 0; p < 5; ++p) {
            double kf = 0.0;
#pragma unroll
            for (int q = 0; q < 5; ++q) kf = fma(A.k[d][p * 5 + q], f[d][q], kf);
            e = fma(f[d][p], kf, e);
        }
    }
    return e;
}

// ||f||_P^2: partial sums per block into partial[blockIdx.x]
template <int K>
__global__ void __launch_bounds__(256) energy_kernel(NodeArgs A, double* __restrict__ partial)
{
    const long long n = (long long)A.nx * A.ny;
    double v[1] = {0.0};
    const bool is_max[1] = {false};
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(id % A.nx), y = (int)(id / A.nx);
        v[0] += node_energy<K>(A, x, y);
    }
    block_reduce<1>(v, is_max);
    if (threadIdx.x == 0) partial[blockIdx.x] = v[0];
}

// error sums against exact [10][ny][nx]: partial[blockIdx.x][30] = (sum e^2, sum ex^2, max|e|) x 10
template <int K>
__global__ void __launch_bounds__(256) error_kernel(NodeArgs A, const double* __restrict__ exact,
                                                    double* __restrict__ partial)
{
    const long long n = (long long)A.nx * A.ny;
    double v[30];
    bool is_max[30];
#pragma unroll
    for (int q = 0; q < 30; ++q) {
        v[q] = 0.0;
        is_max[q] = (q >= 20);
    }
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(id % A.nx), y = (int)(id / A.nx);
        double o[10];
        node_outputs<K>(A, x, y, o);
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            const double ex = exact[q * n + id];
            const double e = o[q] - ex;
            v[q] = fma(e, e, v[q]);
            v[10 + q] = fma(ex, ex, v[10 + q]);
            v[20 + q] = fmax(v[20 + q], fabs(e));
        }
    }
    block_reduce<30>(v, is_max);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 30; ++q) partial[(long long)blockIdx.x * 30 + q] = v[q];
}

// fold nblk partial rows of width NV into out[NV] (one block, fixed order)
template <int NV>
__global__ void __launch_bounds__(256) finish_kernel(const double* __restrict__ partial, int nblk,
                                                     int nmax_from, double* __restrict__ out)
{
    double v[NV];
    bool is_max[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        v[q] = 0.0;
        is_max[q] = (q >= nmax_from);
    }
    for (int i = threadIdx.x; i < nblk; i += blockDim.x)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const double t = partial[(long long)i * NV + q];
            v[q] = is_max[q] ? fmax(v[q], t) : v[q] + t;
        }
    block_reduce<NV>(v, is_max);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) out[q] = v[q];
}

template <int K>
__global__ void finite_kernel(NodeArgs A, int* flag)
{
    const long long n = (long long)A.nx * A.ny;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        double S[4][5];
        load_node<K>(A, (int)(id % A.nx), (int)(id / A.nx), S);
        bool bad = false;
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int k = 0; k < 5; ++k) bad |= !isfinite(S[d][k]);
        if (bad) atomicOr(flag, 1);
    }
}

}  // namespace lbmk
