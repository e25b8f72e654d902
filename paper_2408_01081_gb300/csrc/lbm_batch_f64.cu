// FP64 batches on staged rows (batch mode 3): one step per launch over tiles of 128 columns
// x `rows` rows of every lattice, each tile run by one block of 128 threads in the manner of
// the single-lattice FP64 staged step (lbm_f64stage.cuh): thread t computes column t of the
// tile's rows one after the other, and the 20 populations its node pulls for the next row are
// copied into shared memory by cp.async (8 bytes each) while the current row is collided, so
// the loads occupy no registers.  The pull, the homogeneous Dirichlet reflection
// f_ij = D f*_{-i,-j} (b = 0, no wall data) and the node update are those of batch_tile
// (lbm_batch.cuh), so results equal batch mode 0 bit for bit.
//
// The node update is chosen per lattice as in batch_tile: the fixed-point update (split level
// 12) where both multipliers cK/c and cmu/c allow it, else the IEEE operation sequence of split
// level 1.  The host keeps four tile lists (periodic / Dirichlet x fixed point / level 1) and
// launches each non-empty one, so every block runs one instantiation.
#include <cuda_runtime.h>

#include "lbm_batch.cuh"
#include "lbm_f64stage.cuh"

namespace lbmk {

template <bool DIRICHLET, unsigned long long SPLIT>
__global__ void __launch_bounds__(SA_THREADS, (SPLIT & kSplitFixed) ? LBM_SA_FX_MIN_BLOCKS : LBM_SA_MIN_BLOCKS)
    batch_f64_staged_kernel(BatchF64Args A)
{
    __shared__ __align__(16) double slot[SA_SLOTS][SA_THREADS];
    const int4 tile = A.tiles[blockIdx.x];             // {lattice, first column, first row, 0}
    const LatDesc& L = A.lat[tile.x];
    const int t = threadIdx.x;
    const int nx = L.nx, ny = L.ny;
    const int xg = tile.y + t;
    const bool active = xg < nx;
    const int x = active ? xg : nx - 1;                // lanes past nx mirror column nx - 1
    const int y0 = tile.z;
    const int y1 = min(ny, y0 + A.rows);
    const long long plane = L.plane, pitch = L.pitch;
    const double* __restrict__ src = A.src + L.off;
    double* __restrict__ dst = A.dst + L.off;
    const double a = L.a, b = L.b;
    const int xl = (x == 0) ? nx - 1 : x - 1, xr = (x == nx - 1) ? 0 : x + 1;
    const bool le = DIRICHLET && x == 0, ri = DIRICHLET && x == nx - 1;
    const uint32_t s0 = lbmt::smem_u32(&slot[0][t]);
    constexpr uint32_t SL = SA_THREADS * 8;            // bytes from one slot to the next

    // slot d * 5 + k <- the population of direction d, component k that node (x, y) pulls; on a
    // Dirichlet edge the missing link's slot gets the node's own opposite population
    auto issue = [&](int y) {
        const int ym = (y == 0) ? ny - 1 : y - 1, yp = (y == ny - 1) ? 0 : y + 1;
        const bool bot = DIRICHLET && y == 0, top = DIRICHLET && y == ny - 1;
        const long long r = (long long)y * pitch;
        const double* p[4];
        p[0] = src + (le ? 10 * plane + r + x : r + xl);
        p[1] = src + (bot ? 15 * plane + r + x : 5 * plane + (long long)ym * pitch + x);
        p[2] = src + (ri ? r + x : 10 * plane + r + xr);
        p[3] = src + (top ? 5 * plane + r + x : 15 * plane + (long long)yp * pitch + x);
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int d = 0; d < 4; ++d) cp_async8(s0 + (d * 5 + k) * SL, p[d] + k * plane);
    };

    // one commit group per row; y0 < y1 for every listed tile
    issue(y0);
    cp_async_commit();
    for (int y = y0; y < y1; ++y) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        double f[4][5];
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int k = 0; k < 5; ++k) f[d][k] = lds_f64(s0 + (d * 5 + k) * SL);
        // each thread reads only its own slots: the copies of row y + 1 may overwrite them now
        __syncwarp();
        if (y + 1 < y1) issue(y + 1);
        cp_async_commit();
        if (DIRICHLET) {
            // homogeneous Dirichlet: f_ij = D f*_{-i,-j}(x), D = diag(-1, -1, 1, 1, 1)
            const bool bot = y == 0, top = y == ny - 1;
            const double Dk[5] = {-1.0, -1.0, 1.0, 1.0, 1.0};
            if (le)
#pragma unroll
                for (int k = 0; k < 5; ++k) f[0][k] = Dk[k] * f[0][k];
            if (ri)
#pragma unroll
                for (int k = 0; k < 5; ++k) f[2][k] = Dk[k] * f[2][k];
            if (bot)
#pragma unroll
                for (int k = 0; k < 5; ++k) f[1][k] = Dk[k] * f[1][k];
            if (top)
#pragma unroll
                for (int k = 0; k < 5; ++k) f[3][k] = Dk[k] * f[3][k];
        }
        double U[5], o[4][5];
        collide_split<SPLIT>(f, a, b, U, o);
        if (active) {
            const long long off = (long long)y * pitch + x;
#pragma unroll
            for (int d = 0; d < 4; ++d)
#pragma unroll
                for (int k = 0; k < 5; ++k) dst[(d * 5 + k) * plane + off] = o[d][k];
        }
    }
    // no copy is left in flight: the group committed after the last row is empty
}

}  // namespace lbmk

namespace lbmh {

cudaError_t batch_f64_staged_step(const lbmk::BatchF64Args& A, int list, int ntiles, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const dim3 grid((unsigned)ntiles), block(lbmk::SA_THREADS);
    switch (list) {
    case 0: lbmk::batch_f64_staged_kernel<false, lbmk::kSplitFixed><<<grid, block, 0, s>>>(A); break;
    case 1: lbmk::batch_f64_staged_kernel<true, lbmk::kSplitFixed><<<grid, block, 0, s>>>(A); break;
    case 2: lbmk::batch_f64_staged_kernel<false, lbmk::kSplitDefaultMask><<<grid, block, 0, s>>>(A); break;
    case 3: lbmk::batch_f64_staged_kernel<true, lbmk::kSplitDefaultMask><<<grid, block, 0, s>>>(A); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbmh
