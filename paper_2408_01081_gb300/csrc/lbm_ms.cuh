// Moment-space storage of the post-collision state ("deviations from the local
// equilibrium"): per node and component k,
//     m0 = sum_ij f*_ij                       FP32
//     dx = (f*_10 - f*_-10) - Phi_x(m0)/c     16-bit, times a power-of-two scale s
//     dy = (f*_01 - f*_0-1) - Phi_y(m0)/c     16-bit, times s
//     dd = (f*_10 + f*_-10) - (f*_01 + f*_0-1)  16-bit, times s
// Phi_x(m0)/c and Phi_y(m0)/c are the equilibrium values of the first two
// moments (Eq. cond_eq) and the equilibrium value of dd is 0, so dx, dy, dd are
// the non-equilibrium moments, small compared with the populations on smooth
// solutions.  The populations follow exactly from the four moments:
//     f*_{+-1,0} = 1/4 (m0 +- 2 (Phi_x/c + dx) + dd)
//     f*_{0,+-1} = 1/4 (m0 +- 2 (Phi_y/c + dy) - dd)
// Layout of one buffer: 5 FP32 planes of m0, then 15 16-bit planes (dx[5], dy[5],
// dd[5]), each [ny][pitch]: 50 bytes per node.
//
// Three codecs for the 16-bit words (MsCodec): BF16 and FP16 store each scaled
// deviation on its own; block floating point (lbm_mscodec.cuh) stores the three
// deviations of one component with a shared exponent, so the three words of a
// component are always decoded together.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_mscodec.cuh"

namespace lbmk {

enum { K_MSBF16 = 4, K_MSF16 = 5, K_MSBFP = 6, K_RAW16 = 15 };

// raw 16-bit words (no conversion): the moment-space kernels load and store the words
// through this format and convert them with MsCodec
template <> struct Fmt<K_RAW16> {
    using E = unsigned short;
    using M = unsigned short;
    static __device__ __forceinline__ M ld(E e) { return e; }
    static __device__ __forceinline__ E st(M m) { return m; }
};

// one component's three scaled deviations <-> its three words
template <int H>
struct MsFloatCodec {
    static constexpr bool kJoint = false;         // each word decodes on its own
    static constexpr int kH = H;
    static __device__ __forceinline__ void decode(unsigned short wx, unsigned short wy, unsigned short wz, float inv_s,
                                                  float& x, float& y, float& z)
    {
        x = Fmt<H>::ld(wx) * inv_s;
        y = Fmt<H>::ld(wy) * inv_s;
        z = Fmt<H>::ld(wz) * inv_s;
    }
    // X, Y, Z already multiplied by the scale
    static __device__ __forceinline__ void encode(float X, float Y, float Z, unsigned short& wx, unsigned short& wy,
                                                  unsigned short& wz, bool&)
    {
        wx = Fmt<H>::st(X);
        wy = Fmt<H>::st(Y);
        wz = Fmt<H>::st(Z);
    }
};

struct MsBfpCodec {
    static constexpr bool kJoint = true;          // the three words of a component decode together
    static constexpr int kH = K_F16;              // (unused: element type only)
    static __device__ __forceinline__ void decode(unsigned short wx, unsigned short wy, unsigned short wz, float inv_s,
                                                  float& x, float& y, float& z)
    {
        lbmc::bfp_decode(wx, wy, wz, inv_s, x, y, z);
    }
    static __device__ __forceinline__ void encode(float X, float Y, float Z, unsigned short& wx, unsigned short& wy,
                                                  unsigned short& wz, bool& sat)
    {
        lbmc::bfp_encode(X, Y, Z, wx, wy, wz, sat);
    }
};

template <int K> struct Ms;                       // codec of the deviations
template <> struct Ms<K_MSBF16> { using C = MsFloatCodec<K_BF16>; };
template <> struct Ms<K_MSF16> { using C = MsFloatCodec<K_F16>; };
template <> struct Ms<K_MSBFP> { using C = MsBfpCodec; };

template <int K>
__device__ __forceinline__ const float* ms_m0(const void* S) { return static_cast<const float*>(S); }
template <int K>
__device__ __forceinline__ const unsigned short* ms_dev(const void* S, long long plane)
{
    return reinterpret_cast<const unsigned short*>(static_cast<const float*>(S) + 5 * plane);
}

// populations of one direction from the four moments (M = float arithmetic)
__device__ __forceinline__ void ms_dir(int d, const float (&m0)[5], const float (&dxy)[5], const float (&dd)[5],
                                       float a, float b, float (&f)[5])
{
    float p[5];
    if (d == 0 || d == 2) {          // Phi_x(m0)/c
        p[0] = fmaf(a, m0[2], b * m0[3]);
        p[1] = b * m0[4];
        p[2] = a * m0[0];
        p[3] = b * m0[0];
        p[4] = b * m0[1];
    } else {                         // Phi_y(m0)/c
        p[0] = b * m0[4];
        p[1] = fmaf(a, m0[2], -b * m0[3]);
        p[2] = a * m0[1];
        p[3] = -b * m0[1];
        p[4] = b * m0[0];
    }
    const float sg = (d == 0 || d == 1) ? 1.f : -1.f;     // + for (1,0), (0,1)
    const float sd = (d == 0 || d == 2) ? 1.f : -1.f;     // dd enters + on x, - on y
#pragma unroll
    for (int k = 0; k < 5; ++k) f[k] = 0.25f * (m0[k] + sg * 2.f * (p[k] + dxy[k]) + sd * dd[k]);
}

// load the moments of V consecutive nodes (row offset `off`) and rebuild direction d;
// `dxy_base` selects dx (0) or dy (5) planes
template <int K, int V, bool C>
__device__ __forceinline__ void ms_load_dir(const void* S, long long plane, long long off, int d, float a, float b,
                                            float inv_s, float (&out)[5][V])
{
    using Codec = typename Ms<K>::C;
    const float* m0p = ms_m0<K>(S);
    const unsigned short* dv = ms_dev<K>(S, plane);
    const int dxy_base = (d == 0 || d == 2) ? 0 : 5;
    float m0[5][V], g[5][V], dd[5][V];
    if constexpr (!Codec::kJoint) {
        // float words decode on their own: read only the planes this direction needs
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            vload<K_F32, V, C>(m0p + k * plane + off, m0[k]);
            vload<Codec::kH, V, C>(dv + (dxy_base + k) * plane + off, g[k]);
            vload<Codec::kH, V, C>(dv + (10 + k) * plane + off, dd[k]);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                g[k][e] *= inv_s;
                dd[k][e] *= inv_s;
            }
        }
    } else {
        unsigned short wx[5][V], wy[5][V], wz[5][V];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            vload<K_F32, V, C>(m0p + k * plane + off, m0[k]);
            vload<K_RAW16, V, C>(dv + k * plane + off, wx[k]);
            vload<K_RAW16, V, C>(dv + (5 + k) * plane + off, wy[k]);
            vload<K_RAW16, V, C>(dv + (10 + k) * plane + off, wz[k]);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                float x, y, z;
                Codec::decode(wx[k][e], wy[k][e], wz[k][e], inv_s, x, y, z);
                g[k][e] = (d == 0 || d == 2) ? x : y;
                dd[k][e] = z;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
        float mm[5], gg[5], ee[5], f[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            mm[k] = m0[k][e];
            gg[k] = g[k][e];
            ee[k] = dd[k][e];
        }
        ms_dir(d, mm, gg, ee, a, b, f);
#pragma unroll
        for (int k = 0; k < 5; ++k) out[k][e] = f[k];
    }
}

// both x-directions of V nodes from one set of loads
template <int K, int V, bool C>
__device__ __forceinline__ void ms_load_x(const void* S, long long plane, long long off, float a, float b, float inv_s,
                                          float (&f0)[5][V], float (&f2)[5][V])
{
    using Codec = typename Ms<K>::C;
    const float* m0p = ms_m0<K>(S);
    const unsigned short* dv = ms_dev<K>(S, plane);
    float m0[5][V], g[5][V], dd[5][V];
    if constexpr (!Codec::kJoint) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            vload<K_F32, V, C>(m0p + k * plane + off, m0[k]);
            vload<Codec::kH, V, C>(dv + k * plane + off, g[k]);
            vload<Codec::kH, V, C>(dv + (10 + k) * plane + off, dd[k]);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                g[k][e] *= inv_s;
                dd[k][e] *= inv_s;
            }
        }
    } else {
        unsigned short wx[5][V], wy[5][V], wz[5][V];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            vload<K_F32, V, C>(m0p + k * plane + off, m0[k]);
            vload<K_RAW16, V, C>(dv + k * plane + off, wx[k]);
            vload<K_RAW16, V, C>(dv + (5 + k) * plane + off, wy[k]);
            vload<K_RAW16, V, C>(dv + (10 + k) * plane + off, wz[k]);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                float x, y, z;
                Codec::decode(wx[k][e], wy[k][e], wz[k][e], inv_s, x, y, z);
                g[k][e] = x;
                dd[k][e] = z;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
        float mm[5], gg[5], ee[5], fa[5], fb[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            mm[k] = m0[k][e];
            gg[k] = g[k][e];
            ee[k] = dd[k][e];
        }
        ms_dir(0, mm, gg, ee, a, b, fa);
        ms_dir(2, mm, gg, ee, a, b, fb);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            f0[k][e] = fa[k];
            f2[k][e] = fb[k];
        }
    }
}

// moments of one node's four populations; returns m0 and the scaled deviations
__device__ __forceinline__ void ms_moments(const float (&o)[4][5], float a, float b, float (&m0)[5], float (&dx)[5],
                                           float (&dy)[5], float (&dd)[5])
{
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float sx = o[0][k] + o[2][k], sy = o[1][k] + o[3][k];
        m0[k] = sx + sy;
        dx[k] = o[0][k] - o[2][k];
        dy[k] = o[1][k] - o[3][k];
        dd[k] = sx - sy;
    }
    dx[0] -= fmaf(a, m0[2], b * m0[3]);
    dx[1] -= b * m0[4];
    dx[2] -= a * m0[0];
    dx[3] -= b * m0[0];
    dx[4] -= b * m0[1];
    dy[0] -= b * m0[4];
    dy[1] -= fmaf(a, m0[2], -b * m0[3]);
    dy[2] -= a * m0[1];
    dy[3] += b * m0[1];
    dy[4] -= b * m0[0];
}

// ---------------------------------------------------------------------------
// fused pull-collide step on the moment-space state (same structure as step_kernel)
// ---------------------------------------------------------------------------
template <int K, int V, bool DIRICHLET, bool FORCING, bool TRACK, bool OMEGA>
__global__ void __launch_bounds__(256, 2) ms_step_kernel(StepArgs A)
{
    using Codec = typename Ms<K>::C;
    const int y = blockIdx.y;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    const int nchunk = (A.nx + V - 1) / V;
    const bool active = cx < nchunk;
    const int x0 = (active ? cx : nchunk - 1) * V;
    const int nx = A.nx, ny = A.ny;
    const long long plane = A.plane;
    const int lane = threadIdx.x & 31;
    const float fa = A.af, fb = A.bf;
    // the scale is a power of two, its FP32 reciprocal exact; both converted on the host
    const float sc = A.scale_f, inv_s = A.inv_scale_f;
    const bool bot = DIRICHLET && (y == 0);
    const bool top = DIRICHLET && (y == ny - 1);
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;
    const long long row = (long long)y * A.pitch + x0;

    float P0[5][V], P1[5][V], P2[5][V], P3[5][V], own0[5][V], own2[5][V];
    ms_load_x<K, V, false>(A.src, plane, row, fa, fb, inv_s, own0, own2);
    if (bot) ms_load_dir<K, V, false>(A.src, plane, row, 3, fa, fb, inv_s, P1);
    else ms_load_dir<K, V, false>(A.src, plane, (long long)ym * A.pitch + x0, 1, fa, fb, inv_s, P1);
    if (top) ms_load_dir<K, V, false>(A.src, plane, row, 1, fa, fb, inv_s, P3);
    else ms_load_dir<K, V, false>(A.src, plane, (long long)yp * A.pitch + x0, 3, fa, fb, inv_s, P3);

    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;
    const bool left_in_lane = (lane > 0) && (x0 > 0);
    const bool right_in_lane = (lane < 31) && (x0 + V < nx) && (cx + 1 < nchunk);
    const int xr = (x0 + V >= nx) ? 0 : x0 + V;
    float hl[5][1], hr[5][1];
    if (!left_in_lane) ms_load_dir<K, 1, false>(A.src, plane, (long long)y * A.pitch + xl, 0, fa, fb, inv_s, hl);
    if (!right_in_lane) ms_load_dir<K, 1, false>(A.src, plane, (long long)y * A.pitch + xr, 2, fa, fb, inv_s, hr);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        float l = __shfl_up_sync(0xffffffffu, own0[k][V - 1], 1);
        float r = __shfl_down_sync(0xffffffffu, own2[k][0], 1);
        if (!left_in_lane) l = hl[k][0];
        if (!right_in_lane) r = hr[k][0];
        P0[k][0] = l;
#pragma unroll
        for (int e = 1; e < V; ++e) P0[k][e] = own0[k][e - 1];
#pragma unroll
        for (int e = 0; e < V - 1; ++e) P2[k][e] = own2[k][e + 1];
        P2[k][V - 1] = r;
    }
    if (!DIRICHLET && x0 + V > nx && x0 <= nx - 1) {
        float r0[5][1];
        ms_load_dir<K, 1, false>(A.src, plane, (long long)y * A.pitch + 0, 2, fa, fb, inv_s, r0);
        const int e = nx - 1 - x0;
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int q = 0; q < V; ++q)
                if (q == e) P2[k][q] = r0[k][0];
    }

    float m0o[5][V];
    unsigned short wxo[5][V], wyo[5][V], wzo[5][V];
    bool sat = false;
    double wv[2][V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int x = x0 + e;
        float f[4][5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            f[0][k] = P0[k][e];
            f[1][k] = P1[k][e];
            f[2][k] = P2[k][e];
            f[3][k] = P3[k][e];
        }
        if (DIRICHLET) {
            const bool le = (x == 0), ri = (x == nx - 1);
            if (le || ri || bot || top) {
                const double Dk[5] = {-1.0, -1.0, 1.0, 1.0, 1.0};
                double S[5];
                if (le) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g) { gx = A.g[y]; gy = A.g[A.nwall + y]; }
                    wall_source(1, 0, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[0][k] = float(Dk[k] * (double)own2[k][e] + S[k]);
                }
                if (ri) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g) { gx = A.g[ny + y]; gy = A.g[A.nwall + ny + y]; }
                    wall_source(-1, 0, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[2][k] = float(Dk[k] * (double)own0[k][e] + S[k]);
                }
                if (bot) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g && x < nx) { gx = A.g[2 * ny + x]; gy = A.g[A.nwall + 2 * ny + x]; }
                    wall_source(0, 1, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[1][k] = float(Dk[k] * (double)P1[k][e] + S[k]);
                }
                if (top) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g && x < nx) { gx = A.g[2 * ny + nx + x]; gy = A.g[A.nwall + 2 * ny + nx + x]; }
                    wall_source(0, -1, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[3][k] = float(Dk[k] * (double)P3[k][e] + S[k]);
                }
            }
        }
        float U[5], rx[5], ry[5];
        float bx = 0.f, by = 0.f;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            rx[k] = f[1][k] + f[3][k];
            ry[k] = f[0][k] + f[2][k];
        }
        if (FORCING && x < nx) {
            for (int r = 0; r < A.R; ++r) {
                const float xy = A.Xf[(long long)r * nx + x] * A.Yf[(long long)r * ny + y];
                bx = fmaf(xy, A.Tf[r], bx);
                by = fmaf(xy, A.Tf[A.R + r], by);
            }
            const float hb = float(0.5 * A.dt);
            rx[0] = fmaf(hb, float(bx), rx[0]);
            rx[1] = fmaf(hb, float(by), rx[1]);
            U[0] = rx[0] + ry[0];
            U[1] = rx[1] + ry[1];
            ry[0] = fmaf(hb, float(bx), ry[0]);
            ry[1] = fmaf(hb, float(by), ry[1]);
#pragma unroll
            for (int k = 2; k < 5; ++k) U[k] = rx[k] + ry[k];
        } else {
#pragma unroll
            for (int k = 0; k < 5; ++k) U[k] = rx[k] + ry[k];
        }
        float o[4][5];
        collide<float>(f, U, rx, ry, fa, fb, o);
        if (OMEGA) {
            const float h = float(0.5 * A.omega);
            const float fw = float(A.dt * (2.0 - A.omega) * 0.125);
#pragma unroll
            for (int d = 0; d < 4; ++d)
#pragma unroll
                for (int k = 0; k < 5; ++k) o[d][k] = fmaf(h, o[d][k] - f[d][k], f[d][k]);
            if (FORCING) {
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    o[d][0] = fmaf(fw, float(bx), o[d][0]);
                    o[d][1] = fmaf(fw, float(by), o[d][1]);
                }
            }
        }
        float m0[5], dx[5], dy[5], dd[5];
        ms_moments(o, fa, fb, m0, dx, dy, dd);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            m0o[k][e] = m0[k];
            Codec::encode(dx[k] * sc, dy[k] * sc, dd[k] * sc, wxo[k][e], wyo[k][e], wzo[k][e], sat);
        }
        if (TRACK) {
            wv[0][e] = (double)U[0];
            wv[1][e] = (double)U[1];
        }
    }
    if (!active) return;
    if (sat && A.sat) atomicOr(A.sat, 1);
    float* m0p = static_cast<float*>(A.dst);
    unsigned short* dv = reinterpret_cast<unsigned short*>(m0p + 5 * plane);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        vstore<K_F32, V>(m0p + k * plane + row, m0o[k]);
        vstore<K_RAW16, V>(dv + k * plane + row, wxo[k]);
        vstore<K_RAW16, V>(dv + (5 + k) * plane + row, wyo[k]);
        vstore<K_RAW16, V>(dv + (10 + k) * plane + row, wzo[k]);
    }
    if (TRACK) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            double* wp = A.w + (long long)c * plane + row;
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (x0 + e < nx) wp[e] = fma(A.dt, wv[c][e], wp[e]);
        }
    }
}

// ---------------------------------------------------------------------------
// node access for the initialisation, outputs and reductions (FP64 interface)
// ---------------------------------------------------------------------------
template <int K>
__device__ void ms_load_node(const NodeArgs& A, int x, int y, double (&S)[4][5])
{
    using Codec = typename Ms<K>::C;
    const float* m0p = static_cast<const float*>(A.S);
    const unsigned short* dv = reinterpret_cast<const unsigned short*>(m0p + 5 * A.plane);
    const long long off = (long long)(y + A.yo) * A.pitch + x;
    const float inv_s = 1.0f / (float)A.neq_scale;     // exact: the scale is a power of two
    float m0[5], gx[5], gy[5], dd[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        m0[k] = m0p[k * A.plane + off];
        Codec::decode(dv[k * A.plane + off], dv[(5 + k) * A.plane + off], dv[(10 + k) * A.plane + off], inv_s, gx[k],
                      gy[k], dd[k]);
    }
    for (int d = 0; d < 4; ++d) {
        float f[5];
        ms_dir(d, m0, (d == 0 || d == 2) ? gx : gy, dd, (float)A.a, (float)A.b, f);
#pragma unroll
        for (int k = 0; k < 5; ++k) S[d][k] = f[k];
    }
}

template <int K>
__device__ void ms_store_node(const NodeArgs& A, int x, int y, const double (&S)[4][5])
{
    using Codec = typename Ms<K>::C;
    float o[4][5];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k) o[d][k] = (float)S[d][k];
    float m0[5], dx[5], dy[5], dd[5];
    ms_moments(o, (float)A.a, (float)A.b, m0, dx, dy, dd);
    if (A.measure) {
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 5; ++k) mx = fmaxf(mx, fmaxf(fabsf(dx[k]), fmaxf(fabsf(dy[k]), fabsf(dd[k]))));
        atomicMax(reinterpret_cast<unsigned int*>(A.measure), __float_as_uint(mx));
        return;
    }
    float* m0p = static_cast<float*>(A.Sout);
    unsigned short* dv = reinterpret_cast<unsigned short*>(m0p + 5 * A.plane);
    const long long off = (long long)(y + A.yo) * A.pitch + x;
    const float sc = (float)A.neq_scale;
    bool sat = false;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        m0p[k * A.plane + off] = m0[k];
        unsigned short wx, wy, wz;
        Codec::encode(dx[k] * sc, dy[k] * sc, dd[k] * sc, wx, wy, wz, sat);
        dv[k * A.plane + off] = wx;
        dv[(5 + k) * A.plane + off] = wy;
        dv[(10 + k) * A.plane + off] = wz;
    }
    if (sat && A.sat) atomicOr(A.sat, 1);
}

}  // namespace lbmk
