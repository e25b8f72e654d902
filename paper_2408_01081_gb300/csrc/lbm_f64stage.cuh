// FP64 step (omega = 2, no body load; the node update of split level 1, the IEEE operation
// sequence, or 12, the fixed-point update) with each node's inputs staged in shared memory
// by per-thread asynchronous copies (cp.async), one row ahead.
//
// The register step kernel loads the 20 inputs of a node and then waits for them:
// with 80 registers and three 256-thread blocks per SM, about a sixth of its warp
// cycles go to that wait (long scoreboard) while the integer pipe, which shares the
// bound of the split collision with the FP64 pipe, idles.  Here a block of 128 threads
// owns 128 consecutive columns and walks down `rows` rows (the library passes 2 at level 1
// and 4 at level 12), thread t computing column t of each row.  The copies of the next row are issued as soon as
// the current row has been read out of shared memory, so they are in flight during its
// whole collision and occupy no registers.  Each thread copies exactly the 20 values its
// own node pulls (f*_(1,0) from x - 1, f*_(-1,0) from x + 1, f*_(0,1) from y - 1,
// f*_(0,-1) from y + 1, with the periodic wrap or the Dirichlet edge reflection in the
// source address), so no value crosses threads and no barrier or wait loop is needed: a
// thread's copies of a row complete by cp.async.wait_group.  The node arithmetic is
// collide_split of the same level as in step_kernel (lbm_kernels.cuh) on the same inputs,
// so results are bit-identical to it.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_tma.cuh"

namespace lbmk {

#ifndef LBM_SA_THREADS
#define LBM_SA_THREADS 128
#endif
constexpr int SA_THREADS = LBM_SA_THREADS;            // columns per block, one per thread
constexpr int SA_SLOTS = 20;                          // inputs per node
#ifndef LBM_SA_MIN_BLOCKS
#define LBM_SA_MIN_BLOCKS 6                           // 6 x 128 threads at <= 85 registers
#endif
#ifndef LBM_SA_FX_MIN_BLOCKS
#define LBM_SA_FX_MIN_BLOCKS 4                        // fixed-point node update: <= 128 registers
#endif

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ double lds_f64(uint32_t a)
{
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}

// grid: (ceil(nx / SA_THREADS), ceil(ny / rows)), block SA_THREADS; block (cb, r) computes
// the rows r * rows ... of column block cb, one after the other
template <bool DIRICHLET, bool TRACK, unsigned long long SPLIT>
__global__ void __launch_bounds__(SA_THREADS, (SPLIT & kSplitFixed) ? LBM_SA_FX_MIN_BLOCKS : LBM_SA_MIN_BLOCKS)
    step_f64_staged_kernel(StepArgs A, int rows)
{
    __shared__ __align__(16) double slot[SA_SLOTS][SA_THREADS];
    const int t = threadIdx.x;
    const int nx = A.nx, ny = A.ny;
    const int xg = blockIdx.x * SA_THREADS + t;
    const bool active = xg < nx;
    const int x = active ? xg : nx - 1;                // lanes past nx mirror column nx - 1
    const int y0 = blockIdx.y * rows;
    const int y1 = min(ny, y0 + rows);
    const long long plane = A.plane, pitch = A.pitch;
    const double* __restrict__ src = static_cast<const double*>(A.src);
    double* __restrict__ dst = static_cast<double*>(A.dst);
    const int xl = (x == 0) ? nx - 1 : x - 1, xr = (x == nx - 1) ? 0 : x + 1;
    const bool le = DIRICHLET && x == 0, ri = DIRICHLET && x == nx - 1;
    const uint32_t s0 = lbmt::smem_u32(&slot[0][t]);
    constexpr uint32_t SL = SA_THREADS * 8;            // bytes from one slot to the next

    // source of slot d * 5 + k: the population of direction d, component k that node (x, y)
    // pulls; on a Dirichlet edge the missing link's slot gets the node's own opposite population
    auto sources = [&](int y, const double* (&p)[4]) {
        const int ym = (y == 0) ? ny - 1 : y - 1, yp = (y == ny - 1) ? 0 : y + 1;
        const bool bot = DIRICHLET && y == 0, top = DIRICHLET && y == ny - 1;
        const long long r = (long long)y * pitch;
        p[0] = src + (le ? 10 * plane + r + x : r + xl);
        p[1] = src + (bot ? 15 * plane + r + x : 5 * plane + (long long)ym * pitch + x);
        p[2] = src + (ri ? r + x : 10 * plane + r + xr);
        p[3] = src + (top ? 5 * plane + r + x : 15 * plane + (long long)yp * pitch + x);
    };
    auto issue = [&](int y, uint32_t sb) {
        const double* p[4];
        sources(y, p);
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int d = 0; d < 4; ++d) cp_async8(sb + (d * 5 + k) * SL, p[d] + k * plane);
    };

    // one commit group per row
    if (y0 < y1) issue(y0, s0);
    cp_async_commit();
    for (int y = y0; y < y1; ++y) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        double f[4][5];
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int k = 0; k < 5; ++k) f[d][k] = lds_f64(s0 + (d * 5 + k) * SL);
        // the slots have been read: the copies of row y + 1 may overwrite them
        __syncwarp();
        if (y + 1 < y1) issue(y + 1, s0);
        cp_async_commit();
        if (DIRICHLET) {
            // missing incoming links: f_ij = D f*_{-i,-j}(x) + S_ij(x_b, t + dt/2), as in step_kernel
            const bool bot = y == 0, top = y == ny - 1;
            if (le || ri || bot || top) {
                const double Dk[5] = {-1.0, -1.0, 1.0, 1.0, 1.0};
                double S[5];
                if (le) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g) { gx = A.g[y]; gy = A.g[A.nwall + y]; }
                    wall_source(1, 0, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[0][k] = Dk[k] * f[0][k] + S[k];
                }
                if (ri) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g) { gx = A.g[ny + y]; gy = A.g[A.nwall + ny + y]; }
                    wall_source(-1, 0, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[2][k] = Dk[k] * f[2][k] + S[k];
                }
                if (bot) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g) { gx = A.g[2 * ny + x]; gy = A.g[A.nwall + 2 * ny + x]; }
                    wall_source(0, 1, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[1][k] = Dk[k] * f[1][k] + S[k];
                }
                if (top) {
                    double gx = 0.0, gy = 0.0;
                    if (A.g) { gx = A.g[2 * ny + nx + x]; gy = A.g[A.nwall + 2 * ny + nx + x]; }
                    wall_source(0, -1, gx, gy, A.a, A.b, S);
#pragma unroll
                    for (int k = 0; k < 5; ++k) f[3][k] = Dk[k] * f[3][k] + S[k];
                }
            }
        }
        double U[5], o[4][5];
        collide_split<SPLIT>(f, A.a, A.b, U, o);
        if (active) {
            const long long off = (long long)y * pitch + x;
#pragma unroll
            for (int d = 0; d < 4; ++d)
#pragma unroll
                for (int k = 0; k < 5; ++k) dst[(d * 5 + k) * plane + off] = o[d][k];
            if (TRACK) {
                // u*(t+2dt) = u*(t+dt) + dt v(t+dt)  (steps 1(b) and 2(c) of the summary, Sec. 3.6)
                A.w[off] = fma(A.dt, U[0], A.w[off]);
                A.w[plane + off] = fma(A.dt, U[1], A.w[plane + off]);
            }
        }
    }
    // no copy is left in flight: the group committed after the last row is empty
}

}  // namespace lbmk
