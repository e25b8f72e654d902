// Batched stepping of many independent lattices of uneven size and material
// (periodic or homogeneous Dirichlet, b = 0) from one flat tile work-list.
//
// Each lattice has its own planes inside two arenas (A, B).  A tile is
// rows_per_tile x (threads_per_row * V) nodes of one lattice; a CTA of 256
// threads processes one tile at a time, thread (r, c) owning V consecutive
// nodes of row r.  Tiles of all lattices are numbered consecutively, so one
// launch covers the whole batch.  The per-node arithmetic is the single-lattice
// step's (pull, Dirichlet reflection, omega = 2 collision): results are
// bit-identical to stepping each lattice alone.
//
// FP64 batches can also run on staged rows, one block per tile of 128 columns
// (batch mode 3, lbm_batch_f64.cu).
//
// Persistent mode runs `steps` steps in one launch with a grid barrier between
// steps.  The barrier waits with a time limit: on expiry it sets an error flag
// and every block returns, so a launch that cannot make progress ends instead
// of hanging.
#pragma once

#include "lbm_kernels.cuh"

namespace lbmk {

#ifndef LBM_BATCH_F64_FIXED
#define LBM_BATCH_F64_FIXED 1     // FP64 batches: 1 = fixed-point node update, 0 = split level 1
#endif

struct LatDesc {
    long long off;        // element offset of plane 0 of this lattice in each arena
    long long plane;      // elements per plane = ny * pitch
    int nx, ny, pitch, bc;
    double a, b;          // cK / c, cmu / c
    int tpr;              // threads per row of a tile (power of two, 1..256)
    int rpt;              // rows per tile = 256 / tpr
    int tiles_x, tiles_y;
    int first_tile;       // index of this lattice's first tile in the global list
    int pad_;
};

struct BatchArgs {
    const LatDesc* lat;
    const int* tile_lat;          // lattice of each tile
    int ntiles;
    void* arenaA;
    void* arenaB;
    int steps;                    // steps done by this launch
    int parity;                   // 0: the first step reads A and writes B
    unsigned int* bar_count;      // grid barrier state (persistent mode)
    unsigned int* bar_gen;
    int* err;                     // set to 1 when a barrier wait ran out
    unsigned long long timeout_ns;
    unsigned int extra_arrivals;  // arrivals the barrier waits for beyond the grid (test hook; 0 normally)
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sense-reversing grid barrier with a time limit.  Returns false (after setting
// *err) if the other blocks did not arrive in time or another block gave up.
__device__ __forceinline__ bool grid_barrier(const BatchArgs& A)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = A.bar_gen;
        volatile int* err = A.err;
        const unsigned int g = *gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(A.bar_count, 1u) + 1u;
        if (arrived == gridDim.x + A.extra_arrivals) {
            atomicExch(A.bar_count, 0u);
            __threadfence();
            atomicAdd(A.bar_gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g && *err == 0) {
                if (global_ns() - t0 > A.timeout_ns) {
                    atomicExch(A.err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = (*err == 0);
    }
    __syncthreads();
    return ok != 0;
}

// one tile of one lattice, one step (C: coherent loads, for data written earlier in the same launch)
template <int K, int V, bool C>
__device__ __forceinline__ void batch_tile(const LatDesc& L, int local_tile, const typename Fmt<K>::E* __restrict__ srcA,
                                           typename Fmt<K>::E* __restrict__ dstA)
{
    using M = typename Fmt<K>::M;
    using E = typename Fmt<K>::E;
    const int tpr = L.tpr;
    const int r = threadIdx.x / tpr, cc = threadIdx.x % tpr;
    const int ty = local_tile / L.tiles_x, tx = local_tile % L.tiles_x;
    const int nx = L.nx, ny = L.ny;
    const int nchunk = (nx + V - 1) / V;
    const int yr = ty * L.rpt + r;
    const int cx_raw = tx * tpr + cc;
    const bool active = (yr < ny) && (cx_raw < nchunk);
    const int y = yr < ny ? yr : ny - 1;
    const int cx = cx_raw < nchunk ? cx_raw : nchunk - 1;
    const int x0 = cx * V;
    const long long plane = L.plane;
    const E* src = srcA + L.off;
    E* dst = dstA + L.off;
    const int lane = threadIdx.x & 31;
    const bool dir = (L.bc == 1);
    const bool bot = dir && (y == 0);
    const bool top = dir && (y == ny - 1);
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;

    M P0[5][V], P1[5][V], P2[5][V], P3[5][V];
    M own0[5][V], own2[5][V];
    const long long row = (long long)y * L.pitch + x0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        vload<K, V, C>(src + (0 * 5 + k) * plane + row, own0[k]);
        vload<K, V, C>(src + (2 * 5 + k) * plane + row, own2[k]);
        if (bot) vload<K, V, C>(src + (3 * 5 + k) * plane + row, P1[k]);
        else     vload<K, V, C>(src + (1 * 5 + k) * plane + (long long)ym * L.pitch + x0, P1[k]);
        if (top) vload<K, V, C>(src + (1 * 5 + k) * plane + row, P3[k]);
        else     vload<K, V, C>(src + (3 * 5 + k) * plane + (long long)yp * L.pitch + x0, P3[k]);
    }
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;
    const bool left_in_lane = (lane > 0) && (cc > 0) && (x0 > 0);
    const bool right_in_lane = (lane < 31) && (cc < tpr - 1) && (cx + 1 < nchunk) && (x0 + V < nx);
    const int xr = (x0 + V >= nx) ? 0 : x0 + V;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        M l = __shfl_up_sync(0xffffffffu, own0[k][V - 1], 1);
        M rr = __shfl_down_sync(0xffffffffu, own2[k][0], 1);
        if (!left_in_lane) l = sload<K, C>(src + (0 * 5 + k) * plane + (long long)y * L.pitch + xl);
        if (!right_in_lane) rr = sload<K, C>(src + (2 * 5 + k) * plane + (long long)y * L.pitch + xr);
        P0[k][0] = l;
#pragma unroll
        for (int e = 1; e < V; ++e) P0[k][e] = own0[k][e - 1];
#pragma unroll
        for (int e = 0; e < V - 1; ++e) P2[k][e] = own2[k][e + 1];
        P2[k][V - 1] = rr;
    }
    if (!dir && x0 + V > nx && x0 <= nx - 1) {
        const int e = nx - 1 - x0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const M r0 = sload<K, C>(src + (2 * 5 + k) * plane + (long long)y * L.pitch + 0);
#pragma unroll
            for (int q = 0; q < V; ++q)
                if (q == e) P2[k][q] = r0;
        }
    }
    const M a = M(L.a), b = M(L.b);
    M out[4][5][V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int x = x0 + e;
        M f[4][5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            f[0][k] = P0[k][e];
            f[1][k] = P1[k][e];
            f[2][k] = P2[k][e];
            f[3][k] = P3[k][e];
        }
        if (dir) {
            // homogeneous Dirichlet: f_ij = D f*_{-i,-j}(x), D = diag(-1,-1,1,1,1), in FP64
            const double Dk[5] = {-1.0, -1.0, 1.0, 1.0, 1.0};
            if (x == 0)
#pragma unroll
                for (int k = 0; k < 5; ++k) f[0][k] = M(Dk[k] * (double)own2[k][e]);
            if (x == nx - 1)
#pragma unroll
                for (int k = 0; k < 5; ++k) f[2][k] = M(Dk[k] * (double)own0[k][e]);
            if (bot)
#pragma unroll
                for (int k = 0; k < 5; ++k) f[1][k] = M(Dk[k] * (double)P1[k][e]);
            if (top)
#pragma unroll
                for (int k = 0; k < 5; ++k) f[3][k] = M(Dk[k] * (double)P3[k][e]);
        }
        M U[5], rx[5], ry[5];
        M o[4][5];
        if constexpr (K == K_F64) {
            // FP64: the fixed-point node update, the single-lattice default, where the lattice's
            // multipliers allow it (uniform over the tile: one lattice per tile), else the exact
            // integer-pipe sums of split level 1
            if (LBM_BATCH_F64_FIXED && lbmfx::mul_ok(L.a) && lbmfx::mul_ok(L.b))
                collide_split<kSplitFixed>(f, a, b, U, o);
            else collide_split<kSplitDefaultMask>(f, a, b, U, o);
        } else {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                rx[k] = f[1][k] + f[3][k];
                ry[k] = f[0][k] + f[2][k];
                U[k] = rx[k] + ry[k];
            }
            collide<M>(f, U, rx, ry, a, b, o);
        }
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int k = 0; k < 5; ++k) out[d][k][e] = o[d][k];
    }
    if (!active) return;
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k) vstore<K, V>(dst + (d * 5 + k) * plane + row, out[d][k]);
}

// batch mode 3 (FP64, staged rows, lbm_batch_f64.cu): one step over one tile list
struct BatchF64Args {
    const LatDesc* lat;
    const int4* tiles;            // {lattice, first column (a multiple of 128), first row, 0}
    const double* src;            // arena read by this step
    double* dst;                  // arena written
    int rows;                     // rows per tile
};

template <int K, int V, bool PERSISTENT>
__global__ void __launch_bounds__(256, K == K_F64 ? LBM_SPLIT_MIN_BLOCKS : 2) batch_step_kernel(BatchArgs A)
{
    using E = typename Fmt<K>::E;
    const E* a = static_cast<const E*>(A.arenaA);
    const E* b = static_cast<const E*>(A.arenaB);
    for (int s = 0; s < A.steps; ++s) {
        const bool fromA = ((A.parity + s) & 1) == 0;
        const E* src = fromA ? a : b;
        E* dst = const_cast<E*>(fromA ? b : a);
        for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
            const LatDesc L = A.lat[A.tile_lat[t]];
            batch_tile<K, V, PERSISTENT>(L, t - L.first_tile, src, dst);
        }
        if (PERSISTENT && s + 1 < A.steps) {
            if (!grid_barrier(A)) return;
        }
    }
}

}  // namespace lbmk

namespace lbmh {

// list 0 / 1: periodic / Dirichlet lattices on the fixed-point node update; 2 / 3: the same on
// the IEEE sequence of split level 1.  ntiles == 0 launches nothing.
cudaError_t batch_f64_staged_step(const lbmk::BatchF64Args& A, int list, int ntiles, cudaStream_t s);

}  // namespace lbmh
