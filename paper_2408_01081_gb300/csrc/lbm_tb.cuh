// Two time steps per pass over memory (temporal blocking) for the population
// formats stored in FP32 / BF16 / FP16 (FP32 arithmetic), periodic or
// homogeneous-Dirichlet lattices without body load (omega = 2).
//
// Each warp owns a strip of 32 columns and streams down a block of rows.  Lane l
// computes the intermediate state S1 = f*(t+dt) at column x0 + l for every row r
// of the block plus one row above and below, straight from the stored state
// S0 = f*(t) (pull + collision, as in step_kernel), and keeps the rows r-1, r-2
// it still needs in registers.  From them it computes S2 = f*(t+2dt) of row r-1
// (pull along x by warp shuffles, along y from the kept rows) and writes it.  S2
// needs S1 one column beyond each side, so strips overlap by two columns and a
// warp writes the 30 inner columns.  S1 never leaves the registers, so one pass
// reads and writes the state once for two steps.  With FP32 storage the result
// is bit-identical to two single steps; with 16-bit storage S1 is not rounded to
// 16 bits, which is more accurate than two single steps.
#pragma once

#include "lbm_kernels.cuh"

namespace lbmk {

struct TbArgs {
    const void* src;
    void* dst;
    int nx, ny, pitch;
    long long plane;
    double a, b;
    float af, bf;         // a, b in FP32, converted on the host
    int rows;             // rows per block (gridDim.y blocks of rows)
};

constexpr int TB_OUT = 30;   // output columns per 32-lane strip

// S0 inputs of S1(r) at one lane's column: own (1,0) and (-1,0) values of row r (the
// x-neighbours come from the adjacent lanes), the halo values lanes 0 and 31 need,
// and the pulled (0,1) / (0,-1) values (own opposite plane on a Dirichlet edge row)
struct TbRow {
    float o0[5], o2[5], hl[5], hr[5], fy1[5], fy3[5];
};

template <int K, bool DIRICHLET>
__device__ __forceinline__ void tb_load_row(const typename Fmt<K>::E* __restrict__ src, const TbArgs& A, int r, int xc,
                                            int lane, TbRow& L)
{
    const int nx = A.nx, ny = A.ny;
    const long long plane = A.plane;
    const bool row_ok = DIRICHLET ? (r >= 0 && r < ny) : true;
    const int ry = row_ok ? (r < 0 ? r + ny : (r >= ny ? r - ny : r)) : 0;   // r in [-1, ny]
    const long long rowoff = (long long)ry * A.pitch;
    const int rm = (ry == 0) ? ny - 1 : ry - 1, rp = (ry == ny - 1) ? 0 : ry + 1;
    const bool bot = DIRICHLET && ry == 0, top = DIRICHLET && ry == ny - 1;
    const int xl = DIRICHLET ? max(xc - 1, 0) : (xc == 0 ? nx - 1 : xc - 1);
    const int xr = DIRICHLET ? min(xc + 1, nx - 1) : (xc == nx - 1 ? 0 : xc + 1);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        L.o0[k] = sload<K>(src + (0 * 5 + k) * plane + rowoff + xc);
        L.o2[k] = sload<K>(src + (2 * 5 + k) * plane + rowoff + xc);
        L.hl[k] = (lane == 0) ? sload<K>(src + (0 * 5 + k) * plane + rowoff + xl) : 0.f;
        L.hr[k] = (lane == 31) ? sload<K>(src + (2 * 5 + k) * plane + rowoff + xr) : 0.f;
        L.fy1[k] = bot ? sload<K>(src + (3 * 5 + k) * plane + rowoff + xc)
                       : sload<K>(src + (1 * 5 + k) * plane + (long long)rm * A.pitch + xc);
        L.fy3[k] = top ? sload<K>(src + (1 * 5 + k) * plane + rowoff + xc)
                       : sload<K>(src + (3 * 5 + k) * plane + (long long)rp * A.pitch + xc);
    }
}

#ifndef LBM_TB_MIN_BLOCKS
#define LBM_TB_MIN_BLOCKS 1
#endif

template <int K, bool DIRICHLET>
__global__ void __launch_bounds__(128, LBM_TB_MIN_BLOCKS) tb2_kernel(TbArgs A)
{
    using E = typename Fmt<K>::E;
    const E* __restrict__ src = static_cast<const E*>(A.src);
    E* __restrict__ dst = static_cast<E*>(A.dst);
    const int lane = threadIdx.x & 31;
    const int strip = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nx = A.nx, ny = A.ny;
    const long long plane = A.plane;
    const int nstrip = (nx + TB_OUT - 1) / TB_OUT;
    if (strip >= nstrip) return;                          // whole warp leaves together
    const int xs = strip * TB_OUT - 1 + lane;             // this lane's column (may be -1 or >= nx)
    const bool inside = (xs >= 0) && (xs < nx);
    const int xc = DIRICHLET ? (xs < 0 ? 0 : (xs >= nx ? nx - 1 : xs)) : ((xs % nx) + nx) % nx;
    const bool out_lane = (lane >= 1) && (lane <= TB_OUT) && inside;
    const int y0 = blockIdx.y * A.rows;
    const int y1 = min(ny, y0 + A.rows);
    const float fa = A.af, fb = A.bf;
    const float Dk[5] = {-1.f, -1.f, 1.f, 1.f, 1.f};

    float keep_py[5];          // S1(r-2), direction (0,1)
    float prev[4][5];          // S1(r-1), all directions
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        keep_py[k] = 0.f;
#pragma unroll
        for (int d = 0; d < 4; ++d) prev[d][k] = 0.f;
    }
    TbRow cur_in, next_in;
    tb_load_row<K, DIRICHLET>(src, A, y0 - 1, xc, lane, cur_in);

    for (int r = y0 - 1; r <= y1; ++r) {
        if (r < y1) tb_load_row<K, DIRICHLET>(src, A, r + 1, xc, lane, next_in);   // in flight during the math
        // ---- S1(r) at column xc ----
        float cur[4][5];
        const bool row_ok = DIRICHLET ? (r >= 0 && r < ny) : true;
        {
            float f[4][5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                float l = __shfl_up_sync(0xffffffffu, cur_in.o0[k], 1);
                float rr = __shfl_down_sync(0xffffffffu, cur_in.o2[k], 1);
                f[0][k] = (lane == 0) ? cur_in.hl[k] : l;
                f[2][k] = (lane == 31) ? cur_in.hr[k] : rr;
                f[1][k] = cur_in.fy1[k];
                f[3][k] = cur_in.fy3[k];
            }
            if (DIRICHLET) {
                const int ry = row_ok ? r : 0;
                const bool bot = ry == 0, top = ry == ny - 1;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if (xc == 0) f[0][k] = Dk[k] * cur_in.o2[k];
                    if (xc == nx - 1) f[2][k] = Dk[k] * cur_in.o0[k];
                    if (bot) f[1][k] = Dk[k] * f[1][k];
                    if (top) f[3][k] = Dk[k] * f[3][k];
                }
            }
            float U[5], rx[5], ry2[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                rx[k] = f[1][k] + f[3][k];
                ry2[k] = f[0][k] + f[2][k];
                U[k] = rx[k] + ry2[k];
            }
            collide<float>(f, U, rx, ry2, fa, fb, cur);
            if (!row_ok)
#pragma unroll
                for (int d = 0; d < 4; ++d)
#pragma unroll
                    for (int k = 0; k < 5; ++k) cur[d][k] = 0.f;
        }
        // ---- S2(r-1) from S1(r-2), S1(r-1), S1(r) ----
        const int q = r - 1;
        if (q >= y0) {
            const bool bot = DIRICHLET && q == 0, top = DIRICHLET && q == ny - 1;
            float f[4][5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                f[0][k] = __shfl_up_sync(0xffffffffu, prev[0][k], 1);
                f[2][k] = __shfl_down_sync(0xffffffffu, prev[2][k], 1);
                f[1][k] = bot ? Dk[k] * prev[3][k] : keep_py[k];
                f[3][k] = top ? Dk[k] * prev[1][k] : cur[3][k];
                if (DIRICHLET && xs == 0) f[0][k] = Dk[k] * prev[2][k];
                if (DIRICHLET && xs == nx - 1) f[2][k] = Dk[k] * prev[0][k];
            }
            float U[5], rx[5], ry2[5], o[4][5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                rx[k] = f[1][k] + f[3][k];
                ry2[k] = f[0][k] + f[2][k];
                U[k] = rx[k] + ry2[k];
            }
            collide<float>(f, U, rx, ry2, fa, fb, o);
            if (out_lane) {
                const long long off = (long long)q * A.pitch + xs;
#pragma unroll
                for (int d = 0; d < 4; ++d)
#pragma unroll
                    for (int k = 0; k < 5; ++k) dst[(d * 5 + k) * plane + off] = Fmt<K>::st(o[d][k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            keep_py[k] = prev[1][k];
#pragma unroll
            for (int d = 0; d < 4; ++d) prev[d][k] = cur[d][k];
        }
        cur_in = next_in;
    }
}

}  // namespace lbmk
