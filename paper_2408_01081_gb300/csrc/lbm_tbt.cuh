// Two time steps per pass with the input rows staged in shared memory by tensor
// copies (TMA), for the population formats stored in FP32 / BF16 / FP16 (FP32
// arithmetic), periodic or homogeneous-Dirichlet lattices without body load,
// omega = 2.  Same arithmetic as tb2_kernel (lbm_tb.cuh), so FP32 results are
// bit-identical to two single steps.
//
// Block = 4 compute warps + 1 producer warp over a tile of 120 output columns and
// `rows` output rows.  The producer's elected lane streams the input rows
// y0-2 .. y1+1 of all 20 planes, columns [X0 - HL, X0 + 120 + HL), into a ring of
// shared-memory stages, one tensor copy per row (lbm_tma.cuh), as far ahead as the
// ring allows; the compute warps never wait on registers for global loads.  Compute
// warp w owns the S1 columns X0 - 1 + 30 w + lane: S1 = f*(t+dt) of row r from the
// staged rows r-1, r, r+1 (pull + collision), then S2 = f*(t+2dt) of row r-1 from S1
// of rows r-2, r-1, r kept in registers (x-neighbours by warp shuffles), written by
// lanes 1..30.  A staged row is released (empty barrier) as soon as S1 of the row
// above it is done.
//
// Periodic lattices: a lane whose S1 column or its x-neighbours wrap around the
// lattice (only at x = 0 and x = nx - 1) reads those values from global memory;
// every other read comes from shared memory.  Dirichlet lattices need no wrap:
// the edge reflections use the node's own staged values, and rows outside the
// lattice are not loaded (their stages complete without data).
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_ms.cuh"
#include "lbm_tb.cuh"
#include "lbm_tma.cuh"

namespace lbmk {

// r modulo ny in [0, ny) for r within three rows of the lattice (the staged rows of the
// three-step kernels): one wrap suffices unless ny = 2, where the remainder is taken
__device__ __forceinline__ int wrap_row(int r, int ny)
{
    if (r < 0) r += ny;
    else if (r >= ny) r -= ny;
    if ((unsigned)r >= (unsigned)ny) {
        const int q = r % ny;
        r = q < 0 ? q + ny : q;
    }
    return r;
}

struct TbtArgs {
    const void* src;       // f*(t) planes (wrapped edge columns are read here)
    void* dst;             // f*(t+2dt) planes
    int nx, ny, pitch;
    long long plane;
    float af, bf;          // cK/c, cmu/c in FP32
    int rows;              // output rows per block
    int* timeout;          // device flag: set when a bounded wait ran out
    int withhold;          // test hook: staged input row the producer never copies (-1: none)
    float scale, inv_s;    // moment-space storage: scale of the stored deviations and its reciprocal
    int* sat;              // moment space, block floating point: set when a stored block saturated
    int l2_ahead;          // rows prefetched into L2 ahead of the row the ring loads (0: none)
};

// stages of the row ring: FP32 rows (10 KB), 16-bit rows (5.4 KB), moment-space rows (6.8 KB).
// Measured at 8192^2 (GB300): 4 to 12 stages change the rate by a few per cent at most; FP32
// is fastest with 7, the 16-bit and moment-space formats with 4 (the shallow ring leaves the
// register file, not shared memory, as the occupancy limit)
#ifndef LBM_TBT_NST4
#define LBM_TBT_NST4 7
#endif
#ifndef LBM_TBT_NST2
#define LBM_TBT_NST2 4
#endif
#ifndef LBM_TBT_NSTMS
#define LBM_TBT_NSTMS 4
#endif

constexpr int TBT_WARPS = 4;                  // compute warps per block
constexpr int TBT_L2_AHEAD = 0;               // default rows the producer prefetches into L2 beyond the ring
                                              // (measured: any prefetch distance made the kernels slower)
constexpr int TBT_OUT = TBT_WARPS * TB_OUT;   // output columns per block (120)
constexpr int TBT_THREADS = 32 * (TBT_WARPS + 1);

template <int ES>
struct TbtGeom {
    static constexpr int HL = 16 / ES;                                 // staged columns left of the tile
    static constexpr int WIN = HL + TBT_OUT + HL;                      // staged columns per row
    static constexpr int ROW_BYTES = 20 * WIN * ES;                    // one row of the 20 planes
    static constexpr int STAGE_BYTES = (ROW_BYTES + 127) / 128 * 128;  // stage starts 128-byte aligned
    static constexpr int NST = (ES == 4) ? LBM_TBT_NST4 : LBM_TBT_NST2; // stages in the ring
    static constexpr int SMEM = NST * STAGE_BYTES + 128;               // dynamic shared memory per block
                                                                       // (+128: the ring starts 128-B aligned)
    static_assert((WIN * ES) % 16 == 0, "staged row width must be a multiple of 16 bytes");
    static_assert(WIN <= 256, "tensor-copy box width");
};

template <int K, bool DIRICHLET>
__global__ void __launch_bounds__(TBT_THREADS, 3) tbt_kernel(const __grid_constant__ CUtensorMap map, TbtArgs A)
{
    using E = typename Fmt<K>::E;
    using G = TbtGeom<(int)sizeof(E)>;
    constexpr int NST = G::NST, WIN = G::WIN, HL = G::HL;
    extern __shared__ __align__(128) unsigned char tbt_smem_raw[];
    __shared__ __align__(8) unsigned long long full_bar[NST], empty_bar[NST];
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = A.nx, ny = A.ny;
    const int X0 = blockIdx.x * TBT_OUT;
    const int y0 = blockIdx.y * A.rows;
    const int y1 = min(ny, y0 + A.rows);
    const int nin = (y1 - y0) + 4;                   // staged input rows y0-2 .. y1+1
    const uint32_t raw = lbmt::smem_u32(tbt_smem_raw);
    const uint32_t sbase = (raw + 127u) & ~127u;                    // 128-byte aligned ring

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            lbmt::mbar_init(lbmt::smem_u32(&full_bar[s]), 1);
            lbmt::mbar_init(lbmt::smem_u32(&empty_bar[s]), TBT_WARPS);
        }
        abort_flag = 0;
        lbmt::fence_mbar_init();
    }
    __syncthreads();

    if (warp == TBT_WARPS) {
        // ---- producer: one tensor copy per input row, as far ahead as the ring allows ----
        if (lane == 0) {
            lbmt::prefetch_map(&map);
            for (int jp = NST; jp < NST + A.l2_ahead && jp < nin; ++jp) {
                const int yp = y0 - 2 + jp;
                if (!DIRICHLET || (yp >= 0 && yp < ny))
                    lbmt::tma_prefetch_3d(&map, X0 - HL, (yp < 0) ? yp + ny : (yp >= ny ? yp - ny : yp), 0);
            }
            int j = 0;
            for (; j < nin; ++j) {
                const int s = j % NST;
                const uint32_t fb = lbmt::smem_u32(&full_bar[s]);
                if (j == A.withhold) continue;               // test hook: this row never arrives
                if (j >= NST && !lbmt::mbar_wait(lbmt::smem_u32(&empty_bar[s]), ((j / NST) - 1) & 1, &abort_flag))
                    break;
                {
                    // the row the ring will reach l2_ahead copies later: into L2 now
                    const int jp = j + A.l2_ahead;
                    const int yp = y0 - 2 + jp;
                    if (j >= NST && A.l2_ahead > 0 && jp < nin && (!DIRICHLET || (yp >= 0 && yp < ny)))
                        lbmt::tma_prefetch_3d(&map, X0 - HL, (yp < 0) ? yp + ny : (yp >= ny ? yp - ny : yp), 0);
                }
                int y = y0 - 2 + j;
                if (DIRICHLET && (y < 0 || y >= ny)) {
                    lbmt::mbar_arrive(fb);                   // row outside the lattice: never read
                    continue;
                }
                if (!DIRICHLET) y = (y < 0) ? y + ny : (y >= ny ? y - ny : y);
                lbmt::mbar_arrive_expect_tx(fb, G::ROW_BYTES);
                lbmt::tma_load_3d(sbase + s * G::STAGE_BYTES, &map, X0 - HL, y, 0, fb);
            }
            // every copy issued has landed before the block leaves
            for (int q = (j > NST ? j - NST : 0); q < j; ++q)
                if (q != A.withhold) lbmt::mbar_drain(lbmt::smem_u32(&full_bar[q % NST]), (q / NST) & 1);
            if (abort_flag) atomicExch(A.timeout, 1);
        }
        return;
    }

    // ---- compute warps ----
    const E* __restrict__ src = static_cast<const E*>(A.src);
    E* __restrict__ dst = static_cast<E*>(A.dst);
    const long long plane = A.plane;
    const int xs = X0 - 1 + TB_OUT * warp + lane;        // this lane's S1 column (may be -1 or >= nx)
    const int xc = DIRICHLET ? (xs < 0 ? 0 : (xs >= nx ? nx - 1 : xs)) : ((xs % nx) + nx) % nx;
    const bool out_lane = (lane >= 1) && (lane <= TB_OUT) && (xs >= 0) && (xs < nx);
    const bool staged = DIRICHLET || (xs >= 1 && xs + 1 <= nx - 1);   // all three columns in the tile
    const int xl = (xc == 0) ? nx - 1 : xc - 1, xr = (xc == nx - 1) ? 0 : xc + 1;
    const int idx = xs - X0 + HL;                        // shared-memory column of xs
    const float fa = A.af, fb = A.bf;
    const float Dk[5] = {-1.f, -1.f, 1.f, 1.f, 1.f};

    float keep_py[5], prev[4][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        keep_py[k] = 0.f;
#pragma unroll
        for (int d = 0; d < 4; ++d) prev[d][k] = 0.f;
    }
    bool ok = lbmt::mbar_wait(lbmt::smem_u32(&full_bar[0]), 0, &abort_flag) &&
              lbmt::mbar_wait(lbmt::smem_u32(&full_bar[1 % NST]), (1 / NST) & 1, &abort_flag);
    for (int i = 0; i + 2 < nin; ++i) {
        const int r = y0 - 1 + i;                        // S1 row, from staged rows i, i+1, i+2
        {
            const int j = i + 2;
            ok = ok && lbmt::mbar_wait(lbmt::smem_u32(&full_bar[j % NST]), (j / NST) & 1, &abort_flag);
        }
        if (!__all_sync(0xffffffffu, ok)) break;
        // shared addresses of this lane's column in the staged rows r-1, r, r+1
        constexpr uint32_t ES = sizeof(E), PL = WIN * sizeof(E);
        const uint32_t rm = sbase + (i % NST) * G::STAGE_BYTES + idx * ES;
        const uint32_t rc = sbase + ((i + 1) % NST) * G::STAGE_BYTES + idx * ES;
        const uint32_t rp = sbase + ((i + 2) % NST) * G::STAGE_BYTES + idx * ES;
        // ---- S1(r) at column xc ----
        float cur[4][5];
        const bool row_ok = DIRICHLET ? (r >= 0 && r < ny) : true;
        {
            float f[4][5];
            if (staged) {
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    f[0][k] = Fmt<K>::ld(lbmt::lds<E>(rc + (0 * 5 + k) * PL - ES));
                    f[2][k] = Fmt<K>::ld(lbmt::lds<E>(rc + (2 * 5 + k) * PL + ES));
                    f[1][k] = Fmt<K>::ld(lbmt::lds<E>(rm + (1 * 5 + k) * PL));
                    f[3][k] = Fmt<K>::ld(lbmt::lds<E>(rp + (3 * 5 + k) * PL));
                }
            } else {
                // periodic wrap around x = 0 / x = nx - 1: read the wrapped columns directly
                const int ry = (r < 0) ? r + ny : (r >= ny ? r - ny : r);
                const int rmy = (ry == 0) ? ny - 1 : ry - 1, rpy = (ry == ny - 1) ? 0 : ry + 1;
                const long long o = (long long)ry * A.pitch;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    f[0][k] = sload<K>(src + (0 * 5 + k) * plane + o + xl);
                    f[2][k] = sload<K>(src + (2 * 5 + k) * plane + o + xr);
                    f[1][k] = sload<K>(src + (1 * 5 + k) * plane + (long long)rmy * A.pitch + xc);
                    f[3][k] = sload<K>(src + (3 * 5 + k) * plane + (long long)rpy * A.pitch + xc);
                }
            }
            if (DIRICHLET) {
                const bool bot = r == 0, top = r == ny - 1;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if (xc == 0) f[0][k] = Dk[k] * Fmt<K>::ld(lbmt::lds<E>(rc + (2 * 5 + k) * PL));
                    if (xc == nx - 1) f[2][k] = Dk[k] * Fmt<K>::ld(lbmt::lds<E>(rc + (0 * 5 + k) * PL));
                    if (bot) f[1][k] = Dk[k] * Fmt<K>::ld(lbmt::lds<E>(rc + (3 * 5 + k) * PL));
                    if (top) f[3][k] = Dk[k] * Fmt<K>::ld(lbmt::lds<E>(rc + (1 * 5 + k) * PL));
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
        // staged row i (row r-1) is not read again
        __syncwarp();
        if (lane == 0) lbmt::mbar_arrive(lbmt::smem_u32(&empty_bar[i % NST]));
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
    }
    if (lane == 0 && abort_flag) atomicExch(A.timeout, 1);
}

// ---------------------------------------------------------------------------
// Moment-space storage (lbm_ms.cuh): the same two-step pass over a state of 5 FP32
// planes m0 followed by 15 16-bit planes (dx[5], dy[5], dd[5]) of deviations scaled
// by s.  Each staged row holds columns [X0 - 8, X0 + 128) of both parts (two tensor
// copies, one barrier); populations are rebuilt from the moments on the fly.  The
// intermediate step S1 stays in FP32 registers (not rounded to 16 bits); S2 is
// stored as moments.
// ---------------------------------------------------------------------------
struct TbtMsGeom {
    static constexpr int HL = 8;                                       // 16 bytes of 16-bit values
    static constexpr int WIN = HL + TBT_OUT + HL;                      // 136 staged columns
    static constexpr int M0_BYTES = 5 * WIN * 4;                       // FP32 part of a row
    static constexpr int DEV_OFF = (M0_BYTES + 127) / 128 * 128;       // 16-bit part starts 128-B aligned
    static constexpr int DEV_BYTES = 15 * WIN * 2;
    static constexpr int ROW_BYTES = M0_BYTES + DEV_BYTES;             // bytes the two copies bring
    static constexpr int STAGE_BYTES = (DEV_OFF + DEV_BYTES + 127) / 128 * 128;
    static constexpr int NST = LBM_TBT_NSTMS;
    static constexpr int SMEM = NST * STAGE_BYTES + 128;
    static_assert((WIN * 4) % 16 == 0 && (WIN * 2) % 16 == 0, "staged row width must be a multiple of 16 bytes");
};

// the four moment sets of one node from a staged row (column c of the window)
// or from global memory (column c of row y), deviations unscaled
struct MsNode {
    float m0[5], dx[5], dy[5], dd[5];
};

template <int K>
__device__ __forceinline__ void ms_node_smem(uint32_t stage, int c, float inv_s, MsNode& n)
{
    using Codec = typename Ms<K>::C;
    constexpr uint32_t W = TbtMsGeom::WIN;
    const uint32_t m0 = stage + 4u * c, dv = stage + TbtMsGeom::DEV_OFF + 2u * c;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        n.m0[k] = lbmt::lds_f32(m0 + 4u * W * k);
        Codec::decode(lbmt::lds_u16(dv + 2u * W * k), lbmt::lds_u16(dv + 2u * W * (5 + k)),
                      lbmt::lds_u16(dv + 2u * W * (10 + k)), inv_s, n.dx[k], n.dy[k], n.dd[k]);
    }
}

template <int K>
__device__ __forceinline__ void ms_node_global(const void* S, long long plane, long long off, float inv_s, MsNode& n)
{
    using Codec = typename Ms<K>::C;
    const float* m0 = static_cast<const float*>(S);
    const unsigned short* dv = reinterpret_cast<const unsigned short*>(m0 + 5 * plane);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        n.m0[k] = __ldg(m0 + k * plane + off);
        Codec::decode(__ldg(dv + k * plane + off), __ldg(dv + (5 + k) * plane + off),
                      __ldg(dv + (10 + k) * plane + off), inv_s, n.dx[k], n.dy[k], n.dd[k]);
    }
}

__device__ __forceinline__ void ms_node_dir(const MsNode& n, int d, float a, float b, float (&f)[5])
{
    ms_dir(d, n.m0, (d == 0 || d == 2) ? n.dx : n.dy, n.dd, a, b, f);
}

template <int K, bool DIRICHLET>
__global__ void __launch_bounds__(TBT_THREADS, 3) tbt_ms_kernel(const __grid_constant__ CUtensorMap map32,
                                                                const __grid_constant__ CUtensorMap map16, TbtArgs A)
{
    const float scale = A.scale, inv_s = A.inv_s;
    using Codec = typename Ms<K>::C;
    using G = TbtMsGeom;
    constexpr int NST = G::NST, HL = G::HL;
    extern __shared__ __align__(128) unsigned char tbt_smem_raw[];
    __shared__ __align__(8) unsigned long long full_bar[NST], empty_bar[NST];
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = A.nx, ny = A.ny;
    const int X0 = blockIdx.x * TBT_OUT;
    const int y0 = blockIdx.y * A.rows;
    const int y1 = min(ny, y0 + A.rows);
    const int nin = (y1 - y0) + 4;
    const uint32_t raw = lbmt::smem_u32(tbt_smem_raw);
    const uint32_t sbase = (raw + 127u) & ~127u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            lbmt::mbar_init(lbmt::smem_u32(&full_bar[s]), 1);
            lbmt::mbar_init(lbmt::smem_u32(&empty_bar[s]), TBT_WARPS);
        }
        abort_flag = 0;
        lbmt::fence_mbar_init();
    }
    __syncthreads();

    if (warp == TBT_WARPS) {
        if (lane == 0) {
            lbmt::prefetch_map(&map32);
            lbmt::prefetch_map(&map16);
            auto l2_row = [&](int jp) {
                const int yp = y0 - 2 + jp;
                if (jp < nin && (!DIRICHLET || (yp >= 0 && yp < ny))) {
                    const int yw = (yp < 0) ? yp + ny : (yp >= ny ? yp - ny : yp);
                    lbmt::tma_prefetch_3d(&map32, X0 - HL, yw, 0);
                    lbmt::tma_prefetch_3d(&map16, X0 - HL, yw, 0);
                }
            };
            for (int jp = NST; jp < NST + A.l2_ahead; ++jp) l2_row(jp);
            int j = 0;
            for (; j < nin; ++j) {
                const int s = j % NST;
                const uint32_t fb = lbmt::smem_u32(&full_bar[s]);
                if (j == A.withhold) continue;
                if (j >= NST && !lbmt::mbar_wait(lbmt::smem_u32(&empty_bar[s]), ((j / NST) - 1) & 1, &abort_flag))
                    break;
                if (j >= NST && A.l2_ahead > 0) l2_row(j + A.l2_ahead);
                int y = y0 - 2 + j;
                if (DIRICHLET && (y < 0 || y >= ny)) {
                    lbmt::mbar_arrive(fb);
                    continue;
                }
                if (!DIRICHLET) y = (y < 0) ? y + ny : (y >= ny ? y - ny : y);
                const uint32_t st = sbase + s * G::STAGE_BYTES;
                lbmt::mbar_arrive_expect_tx(fb, G::ROW_BYTES);
                lbmt::tma_load_3d(st, &map32, X0 - HL, y, 0, fb);
                lbmt::tma_load_3d(st + G::DEV_OFF, &map16, X0 - HL, y, 0, fb);
            }
            for (int q = (j > NST ? j - NST : 0); q < j; ++q)
                if (q != A.withhold) lbmt::mbar_drain(lbmt::smem_u32(&full_bar[q % NST]), (q / NST) & 1);
            if (abort_flag) atomicExch(A.timeout, 1);
        }
        return;
    }

    const long long plane = A.plane;
    const int xs = X0 - 1 + TB_OUT * warp + lane;
    const int xc = DIRICHLET ? (xs < 0 ? 0 : (xs >= nx ? nx - 1 : xs)) : ((xs % nx) + nx) % nx;
    const bool out_lane = (lane >= 1) && (lane <= TB_OUT) && (xs >= 0) && (xs < nx);
    const bool own_staged = DIRICHLET || (xs >= 0 && xs < nx);         // own column inside the lattice
    const int xl = (xc == 0) ? nx - 1 : xc - 1, xr = (xc == nx - 1) ? 0 : xc + 1;
    const bool left_staged = DIRICHLET || (xs - 1 >= 0 && xs - 1 < nx);
    const bool right_staged = DIRICHLET || (xs + 1 >= 0 && xs + 1 < nx);
    const int idx = xs - X0 + HL;
    const float fa = A.af, fb = A.bf;
    const float Dk[5] = {-1.f, -1.f, 1.f, 1.f, 1.f};

    // S1 rows r-2 (direction (0,1)), r-1; f*_(0,1)(t) of row r-1; f*(t) of all four directions of
    // the own column in row r, rebuilt from its moments once, as the row above of row r-1
    float keep_py[5], prev[4][5], d1_prev[5], ft[4][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        keep_py[k] = 0.f;
        d1_prev[k] = 0.f;
#pragma unroll
        for (int d = 0; d < 4; ++d) prev[d][k] = ft[d][k] = 0.f;
    }
    auto row_of = [&](int r) { return (r < 0) ? r + ny : (r >= ny ? r - ny : r); };
    bool ok = lbmt::mbar_wait(lbmt::smem_u32(&full_bar[0]), 0, &abort_flag) &&
              lbmt::mbar_wait(lbmt::smem_u32(&full_bar[1 % NST]), (1 / NST) & 1, &abort_flag);
    if (__all_sync(0xffffffffu, ok)) {
        // f*_(0,1)(t) of the own column in staged row 0 (row y0-2): the pull source of row y0-1
        MsNode n;
        if (own_staged) ms_node_smem<K>(sbase, idx, inv_s, n);
        else ms_node_global<K>(A.src, plane, (long long)row_of(y0 - 2) * A.pitch + xc, inv_s, n);
        ms_node_dir(n, 1, fa, fb, d1_prev);
        const uint32_t s1 = sbase + (1 % NST) * G::STAGE_BYTES;
        if (own_staged) ms_node_smem<K>(s1, idx, inv_s, n);
        else ms_node_global<K>(A.src, plane, (long long)row_of(y0 - 1) * A.pitch + xc, inv_s, n);
#pragma unroll
        for (int d = 0; d < 4; ++d) ms_node_dir(n, d, fa, fb, ft[d]);
    }
    for (int i = 0; i + 2 < nin; ++i) {
        const int r = y0 - 1 + i;
        {
            const int j = i + 2;
            ok = ok && lbmt::mbar_wait(lbmt::smem_u32(&full_bar[j % NST]), (j / NST) & 1, &abort_flag);
        }
        if (!__all_sync(0xffffffffu, ok)) break;
        const uint32_t sc = sbase + ((i + 1) % NST) * G::STAGE_BYTES;   // row r
        const uint32_t sp = sbase + ((i + 2) % NST) * G::STAGE_BYTES;   // row r+1
        float cur[4][5];
        const bool row_ok = DIRICHLET ? (r >= 0 && r < ny) : true;
        {
            // own node of row r (all four directions, from the previous iteration) and row r+1
            // (rebuilt here, kept for the next)
            float o0[5], o1[5], o2[5], o3[5], nt[4][5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                o0[k] = ft[0][k];
                o1[k] = ft[1][k];
                o2[k] = ft[2][k];
                o3[k] = ft[3][k];
            }
            {
                MsNode np;
                if (own_staged) ms_node_smem<K>(sp, idx, inv_s, np);
                else ms_node_global<K>(A.src, plane, (long long)row_of(r + 1) * A.pitch + xc, inv_s, np);
#pragma unroll
                for (int d = 0; d < 4; ++d) ms_node_dir(np, d, fa, fb, nt[d]);
            }
            const float (&p3)[5] = nt[3];
            float hl[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, hr[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            if (lane == 0) {
                MsNode h;
                if (left_staged) ms_node_smem<K>(sc, idx - 1, inv_s, h);
                else ms_node_global<K>(A.src, plane, (long long)row_of(r) * A.pitch + xl, inv_s, h);
                ms_node_dir(h, 0, fa, fb, hl);
            }
            if (lane == 31) {
                MsNode h;
                if (right_staged) ms_node_smem<K>(sc, idx + 1, inv_s, h);
                else ms_node_global<K>(A.src, plane, (long long)row_of(r) * A.pitch + xr, inv_s, h);
                ms_node_dir(h, 2, fa, fb, hr);
            }
            float f[4][5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const float l = __shfl_up_sync(0xffffffffu, o0[k], 1);
                const float rr = __shfl_down_sync(0xffffffffu, o2[k], 1);
                f[0][k] = (lane == 0) ? hl[k] : l;
                f[2][k] = (lane == 31) ? hr[k] : rr;
                f[1][k] = d1_prev[k];
                f[3][k] = p3[k];
            }
            if (DIRICHLET) {
                const bool bot = r == 0, top = r == ny - 1;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if (xc == 0) f[0][k] = Dk[k] * o2[k];
                    if (xc == nx - 1) f[2][k] = Dk[k] * o0[k];
                    if (bot) f[1][k] = Dk[k] * o3[k];
                    if (top) f[3][k] = Dk[k] * o1[k];
                }
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                d1_prev[k] = o1[k];
#pragma unroll
                for (int d = 0; d < 4; ++d) ft[d][k] = nt[d][k];
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
        __syncwarp();
        if (lane == 0) lbmt::mbar_arrive(lbmt::smem_u32(&empty_bar[i % NST]));
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
                float m0[5], dx[5], dy[5], dd[5];
                ms_moments(o, fa, fb, m0, dx, dy, dd);
                float* m0p = static_cast<float*>(A.dst);
                unsigned short* dv = reinterpret_cast<unsigned short*>(m0p + 5 * plane);
                const long long off = (long long)q * A.pitch + xs;
                bool sat = false;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    m0p[k * plane + off] = m0[k];
                    unsigned short wx, wy, wz;
                    Codec::encode(dx[k] * scale, dy[k] * scale, dd[k] * scale, wx, wy, wz, sat);
                    dv[k * plane + off] = wx;
                    dv[(5 + k) * plane + off] = wy;
                    dv[(10 + k) * plane + off] = wz;
                }
                if (sat && A.sat) atomicOr(A.sat, 1);
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            keep_py[k] = prev[1][k];
#pragma unroll
            for (int d = 0; d < 4; ++d) prev[d][k] = cur[d][k];
        }
    }
    if (lane == 0 && abort_flag) atomicExch(A.timeout, 1);
}


// ---------------------------------------------------------------------------
// Moment-space storage, three steps per pass (tbt3_ms_kernel).  The same staging as
// tbt_ms_kernel with one more level in registers: S1 = f*(t+dt) of row r from the
// staged rows, S2 = f*(t+2dt) of row r-1 from S1 rows r-2..r, S3 = f*(t+3dt) of row
// r-2 from S2 rows r-3..r-1, stored as moments.  Each level needs one more column
// on each side than the next, so a warp's S1 columns are X0 - 2 + 28 w + lane and
// lanes 2..29 store (112 columns per block), and the staged rows run from y0 - 3 to
// y1 + 2.  The deviations are rounded to 16 bits once per three steps.
// ---------------------------------------------------------------------------
constexpr int TB3_OUT = 28;                    // output columns per warp
constexpr int TBT3_OUT = TBT_WARPS * TB3_OUT;  // output columns per block (112)

struct Tbt3MsGeom {
    static constexpr int HL = 8;
    static constexpr int WIN = HL + TBT3_OUT + HL;                     // 128 staged columns
    static constexpr int M0_BYTES = 5 * WIN * 4;
    static constexpr int DEV_OFF = (M0_BYTES + 127) / 128 * 128;
    static constexpr int DEV_BYTES = 15 * WIN * 2;
    static constexpr int ROW_BYTES = M0_BYTES + DEV_BYTES;
    static constexpr int STAGE_BYTES = (DEV_OFF + DEV_BYTES + 127) / 128 * 128;
    static constexpr int NST = LBM_TBT_NSTMS;
    static constexpr int SMEM = NST * STAGE_BYTES + 128;
    static_assert((WIN * 4) % 16 == 0 && (WIN * 2) % 16 == 0, "staged row width must be a multiple of 16 bytes");
};

template <int K>
__device__ __forceinline__ void ms3_node_smem(uint32_t stage, int c, float inv_s, MsNode& n)
{
    using Codec = typename Ms<K>::C;
    constexpr uint32_t W = Tbt3MsGeom::WIN;
    const uint32_t m0 = stage + 4u * c, dv = stage + Tbt3MsGeom::DEV_OFF + 2u * c;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        n.m0[k] = lbmt::lds_f32(m0 + 4u * W * k);
        Codec::decode(lbmt::lds_u16(dv + 2u * W * k), lbmt::lds_u16(dv + 2u * W * (5 + k)),
                      lbmt::lds_u16(dv + 2u * W * (10 + k)), inv_s, n.dx[k], n.dy[k], n.dd[k]);
    }
}

// one collide-and-pull level on rows kept in registers: f*(q) from the rows below (kb: the
// (0,1) direction of row q-1), at (p: all directions of row q, x-neighbours by shuffles)
// and above (ka: the (0,-1) direction of row q+1); walls as in tbt_kernel
template <bool DIRICHLET>
__device__ __forceinline__ void level_step(const float (&p)[4][5], const float (&kb)[5], const float (&ka)[5], int q,
                                           int xs, int nx, int ny, float fa, float fb, float (&o)[4][5])
{
    const float Dk[5] = {-1.f, -1.f, 1.f, 1.f, 1.f};
    const bool bot = DIRICHLET && q == 0, top = DIRICHLET && q == ny - 1;
    float f[4][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        f[0][k] = __shfl_up_sync(0xffffffffu, p[0][k], 1);
        f[2][k] = __shfl_down_sync(0xffffffffu, p[2][k], 1);
        f[1][k] = bot ? Dk[k] * p[3][k] : kb[k];
        f[3][k] = top ? Dk[k] * p[1][k] : ka[k];
        if (DIRICHLET && xs == 0) f[0][k] = Dk[k] * p[2][k];
        if (DIRICHLET && xs == nx - 1) f[2][k] = Dk[k] * p[0][k];
    }
    float U[5], rx[5], ry2[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        rx[k] = f[1][k] + f[3][k];
        ry2[k] = f[0][k] + f[2][k];
        U[k] = rx[k] + ry2[k];
    }
    collide<float>(f, U, rx, ry2, fa, fb, o);
}

#ifndef LBM_TBT3MS_MIN_BLOCKS
#define LBM_TBT3MS_MIN_BLOCKS 3     // 128 registers (a few values spilled): 3 blocks per SM measured
                                    // faster than 2 at 164 registers
#endif

template <int K, bool DIRICHLET>
__global__ void __launch_bounds__(TBT_THREADS, LBM_TBT3MS_MIN_BLOCKS) tbt3_ms_kernel(const __grid_constant__ CUtensorMap map32,
                                                                 const __grid_constant__ CUtensorMap map16, TbtArgs A)
{
    using Codec = typename Ms<K>::C;
    using G = Tbt3MsGeom;
    constexpr int NST = G::NST, HL = G::HL;
    const float scale = A.scale, inv_s = A.inv_s;
    extern __shared__ __align__(128) unsigned char tbt_smem_raw[];
    __shared__ __align__(8) unsigned long long full_bar[NST], empty_bar[NST];
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = A.nx, ny = A.ny;
    const int X0 = blockIdx.x * TBT3_OUT;
    const int y0 = blockIdx.y * A.rows;
    const int y1 = min(ny, y0 + A.rows);
    const int nin = (y1 - y0) + 6;                   // staged input rows y0-3 .. y1+2
    const uint32_t raw = lbmt::smem_u32(tbt_smem_raw);
    const uint32_t sbase = (raw + 127u) & ~127u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            lbmt::mbar_init(lbmt::smem_u32(&full_bar[s]), 1);
            lbmt::mbar_init(lbmt::smem_u32(&empty_bar[s]), TBT_WARPS);
        }
        abort_flag = 0;
        lbmt::fence_mbar_init();
    }
    __syncthreads();

    if (warp == TBT_WARPS) {
        if (lane == 0) {
            lbmt::prefetch_map(&map32);
            lbmt::prefetch_map(&map16);
            int j = 0;
            for (; j < nin; ++j) {
                const int s = j % NST;
                const uint32_t fb = lbmt::smem_u32(&full_bar[s]);
                if (j == A.withhold) continue;
                if (j >= NST && !lbmt::mbar_wait(lbmt::smem_u32(&empty_bar[s]), ((j / NST) - 1) & 1, &abort_flag))
                    break;
                int y = y0 - 3 + j;
                if (DIRICHLET && (y < 0 || y >= ny)) {
                    lbmt::mbar_arrive(fb);
                    continue;
                }
                if (!DIRICHLET) y = wrap_row(y, ny);   // rows y0 - 3 .. y1 + 2: more than one wrap when ny = 2
                const uint32_t st = sbase + s * G::STAGE_BYTES;
                lbmt::mbar_arrive_expect_tx(fb, G::ROW_BYTES);
                lbmt::tma_load_3d(st, &map32, X0 - HL, y, 0, fb);
                lbmt::tma_load_3d(st + G::DEV_OFF, &map16, X0 - HL, y, 0, fb);
            }
            for (int q = (j > NST ? j - NST : 0); q < j; ++q)
                if (q != A.withhold) lbmt::mbar_drain(lbmt::smem_u32(&full_bar[q % NST]), (q / NST) & 1);
            if (abort_flag) atomicExch(A.timeout, 1);
        }
        return;
    }

    const long long plane = A.plane;
    const int xs = X0 - 2 + TB3_OUT * warp + lane;   // this lane's S1 column
    const int xc = DIRICHLET ? (xs < 0 ? 0 : (xs >= nx ? nx - 1 : xs)) : ((xs % nx) + nx) % nx;
    const bool out_lane = (lane >= 2) && (lane < 2 + TB3_OUT) && (xs >= 0) && (xs < nx);
    const bool own_staged = DIRICHLET || (xs >= 0 && xs < nx);
    const int xl = (xc == 0) ? nx - 1 : xc - 1, xr = (xc == nx - 1) ? 0 : xc + 1;
    const bool left_staged = DIRICHLET || (xs - 1 >= 0 && xs - 1 < nx);
    const bool right_staged = DIRICHLET || (xs + 1 >= 0 && xs + 1 < nx);
    const int idx = xs - X0 + HL;
    const float fa = A.af, fb = A.bf;
    const float Dk[5] = {-1.f, -1.f, 1.f, 1.f, 1.f};

    // S1 rows r-1 (p1, all directions) and r-2 (k1: (0,1)); S2 rows r-2 (p2) and r-3 (k2: (0,1));
    // f*_(0,1)(t) of the own column in the staged row below the current one (d1), and
    // f*(t) of all four directions of the own column in the current staged row (ft), rebuilt
    // from its moments once, as the row above of the previous S1 row
    float p1[4][5], k1[5], p2[4][5], k2[5], d1[5], ft[4][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        k1[k] = k2[k] = d1[k] = 0.f;
#pragma unroll
        for (int d = 0; d < 4; ++d) p1[d][k] = p2[d][k] = ft[d][k] = 0.f;
    }
    auto row_of = [&](int r) { return wrap_row(r, ny); };   // r in y0 - 3 .. y1 + 2
    bool ok = lbmt::mbar_wait(lbmt::smem_u32(&full_bar[0]), 0, &abort_flag) &&
              lbmt::mbar_wait(lbmt::smem_u32(&full_bar[1 % NST]), (1 / NST) & 1, &abort_flag);
    if (__all_sync(0xffffffffu, ok)) {
        MsNode n;
        if (own_staged) ms3_node_smem<K>(sbase, idx, inv_s, n);
        else ms_node_global<K>(A.src, plane, (long long)row_of(y0 - 3) * A.pitch + xc, inv_s, n);
        ms_node_dir(n, 1, fa, fb, d1);
        const uint32_t s1 = sbase + (1 % NST) * G::STAGE_BYTES;
        if (own_staged) ms3_node_smem<K>(s1, idx, inv_s, n);
        else ms_node_global<K>(A.src, plane, (long long)row_of(y0 - 2) * A.pitch + xc, inv_s, n);
#pragma unroll
        for (int d = 0; d < 4; ++d) ms_node_dir(n, d, fa, fb, ft[d]);
    }
    for (int i = 0; i + 2 < nin; ++i) {
        const int r = y0 - 2 + i;                    // S1 row, from staged rows i, i+1, i+2
        {
            const int j = i + 2;
            ok = ok && lbmt::mbar_wait(lbmt::smem_u32(&full_bar[j % NST]), (j / NST) & 1, &abort_flag);
        }
        if (!__all_sync(0xffffffffu, ok)) break;
        const uint32_t sc = sbase + ((i + 1) % NST) * G::STAGE_BYTES;   // row r
        const uint32_t sp = sbase + ((i + 2) % NST) * G::STAGE_BYTES;   // row r+1
        float c1[4][5];
        {
            // own column: row r from the previous iteration, row r+1 rebuilt here (kept for the next)
            float o0[5], o1[5], o2[5], o3[5], nt[4][5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                o0[k] = ft[0][k];
                o1[k] = ft[1][k];
                o2[k] = ft[2][k];
                o3[k] = ft[3][k];
            }
            {
                MsNode np;
                if (own_staged) ms3_node_smem<K>(sp, idx, inv_s, np);
                else ms_node_global<K>(A.src, plane, (long long)row_of(r + 1) * A.pitch + xc, inv_s, np);
#pragma unroll
                for (int d = 0; d < 4; ++d) ms_node_dir(np, d, fa, fb, nt[d]);
            }
            const float (&p3)[5] = nt[3];
            float hl[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, hr[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            if (lane == 0) {
                MsNode h;
                if (left_staged) ms3_node_smem<K>(sc, idx - 1, inv_s, h);
                else ms_node_global<K>(A.src, plane, (long long)row_of(r) * A.pitch + xl, inv_s, h);
                ms_node_dir(h, 0, fa, fb, hl);
            }
            if (lane == 31) {
                MsNode h;
                if (right_staged) ms3_node_smem<K>(sc, idx + 1, inv_s, h);
                else ms_node_global<K>(A.src, plane, (long long)row_of(r) * A.pitch + xr, inv_s, h);
                ms_node_dir(h, 2, fa, fb, hr);
            }
            float f[4][5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const float l = __shfl_up_sync(0xffffffffu, o0[k], 1);
                const float rr = __shfl_down_sync(0xffffffffu, o2[k], 1);
                f[0][k] = (lane == 0) ? hl[k] : l;
                f[2][k] = (lane == 31) ? hr[k] : rr;
                f[1][k] = d1[k];
                f[3][k] = p3[k];
            }
            if (DIRICHLET) {
                const bool bot = r == 0, top = r == ny - 1;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if (xc == 0) f[0][k] = Dk[k] * o2[k];
                    if (xc == nx - 1) f[2][k] = Dk[k] * o0[k];
                    if (bot) f[1][k] = Dk[k] * o3[k];
                    if (top) f[3][k] = Dk[k] * o1[k];
                }
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                d1[k] = o1[k];
#pragma unroll
                for (int d = 0; d < 4; ++d) ft[d][k] = nt[d][k];
            }
            float U[5], rx[5], ry2[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                rx[k] = f[1][k] + f[3][k];
                ry2[k] = f[0][k] + f[2][k];
                U[k] = rx[k] + ry2[k];
            }
            collide<float>(f, U, rx, ry2, fa, fb, c1);
            if (DIRICHLET && !(r >= 0 && r < ny))
#pragma unroll
                for (int d = 0; d < 4; ++d)
#pragma unroll
                    for (int k = 0; k < 5; ++k) c1[d][k] = 0.f;
        }
        __syncwarp();
        if (lane == 0) lbmt::mbar_arrive(lbmt::smem_u32(&empty_bar[i % NST]));
        // ---- S2(r-1) from S1 rows r-2 (k1), r-1 (p1), r (c1) ----
        const int q2 = r - 1;
        float c2[4][5];
        const bool has2 = q2 >= y0 - 1;
        if (has2) {
            level_step<DIRICHLET>(p1, k1, c1[3], q2, xs, nx, ny, fa, fb, c2);
            if (DIRICHLET && !(q2 >= 0 && q2 < ny))
#pragma unroll
                for (int d = 0; d < 4; ++d)
#pragma unroll
                    for (int k = 0; k < 5; ++k) c2[d][k] = 0.f;
            // ---- S3(r-2) from S2 rows r-3 (k2), r-2 (p2), r-1 (c2) ----
            const int q3 = r - 2;
            if (q3 >= y0) {
                float o[4][5];
                level_step<DIRICHLET>(p2, k2, c2[3], q3, xs, nx, ny, fa, fb, o);
                if (out_lane) {
                    float m0[5], dx[5], dy[5], dd[5];
                    ms_moments(o, fa, fb, m0, dx, dy, dd);
                    float* m0p = static_cast<float*>(A.dst);
                    unsigned short* dv = reinterpret_cast<unsigned short*>(m0p + 5 * plane);
                    const long long off = (long long)q3 * A.pitch + xs;
                    bool sat = false;
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        m0p[k * plane + off] = m0[k];
                        unsigned short wx, wy, wz;
                        Codec::encode(dx[k] * scale, dy[k] * scale, dd[k] * scale, wx, wy, wz, sat);
                        dv[k * plane + off] = wx;
                        dv[(5 + k) * plane + off] = wy;
                        dv[(10 + k) * plane + off] = wz;
                    }
                    if (sat && A.sat) atomicOr(A.sat, 1);
                }
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                k2[k] = p2[1][k];
#pragma unroll
                for (int d = 0; d < 4; ++d) p2[d][k] = c2[d][k];
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            k1[k] = p1[1][k];
#pragma unroll
            for (int d = 0; d < 4; ++d) p1[d][k] = c1[d][k];
        }
    }
    if (lane == 0 && abort_flag) atomicExch(A.timeout, 1);
}


// ---------------------------------------------------------------------------
// Population formats, three steps per pass (tbt3_kernel): tbt_kernel's staging with the
// three register levels of tbt3_ms_kernel (S1 from the staged rows, S2, S3 stored by
// lanes 2..29 of each warp, 112 columns per block, staged rows y0 - 3 .. y1 + 2).  Same
// arithmetic as single steps, so FP32 results stay bit-identical to them.
// ---------------------------------------------------------------------------
#ifndef LBM_TBT3_NST4
#define LBM_TBT3_NST4 7
#endif
#ifndef LBM_TBT3_NST2
#define LBM_TBT3_NST2 4
#endif

template <int ES>
struct Tbt3Geom {
    static constexpr int HL = 16 / ES;                                 // >= 3 staged columns each side
    static constexpr int WIN = HL + TBT3_OUT + HL;
    static constexpr int ROW_BYTES = 20 * WIN * ES;
    static constexpr int STAGE_BYTES = (ROW_BYTES + 127) / 128 * 128;
    static constexpr int NST = (ES == 4) ? LBM_TBT3_NST4 : LBM_TBT3_NST2;
    static constexpr int SMEM = NST * STAGE_BYTES + 128;
    static_assert((WIN * ES) % 16 == 0 && HL >= 3, "staged row geometry");
};

#ifndef LBM_TBT3_MIN_BLOCKS
#define LBM_TBT3_MIN_BLOCKS 3       // 116-127 registers
#endif

// One block's work: output columns X0 .. X0 + TBT3_OUT - 1 and rows y0 .. y0 + A.rows - 1 of
// the lattice A describes, its rows staged through `map` (a generic address: a kernel
// parameter or a map in global memory).
template <int K, bool DIRICHLET>
__device__ __forceinline__ void tbt3_body(const CUtensorMap* mapp, const TbtArgs& A, int X0, int y0)
{
    using E = typename Fmt<K>::E;
    using G = Tbt3Geom<(int)sizeof(E)>;
    constexpr int NST = G::NST, WIN = G::WIN, HL = G::HL;
    extern __shared__ __align__(128) unsigned char tbt_smem_raw[];
    __shared__ __align__(8) unsigned long long full_bar[NST], empty_bar[NST];
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = A.nx, ny = A.ny;
    const int y1 = min(ny, y0 + A.rows);
    const int nin = (y1 - y0) + 6;                   // staged input rows y0-3 .. y1+2
    const uint32_t raw = lbmt::smem_u32(tbt_smem_raw);
    const uint32_t sbase = (raw + 127u) & ~127u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            lbmt::mbar_init(lbmt::smem_u32(&full_bar[s]), 1);
            lbmt::mbar_init(lbmt::smem_u32(&empty_bar[s]), TBT_WARPS);
        }
        abort_flag = 0;
        lbmt::fence_mbar_init();
    }
    __syncthreads();

    if (warp == TBT_WARPS) {
        if (lane == 0) {
            lbmt::prefetch_map(mapp);
            int j = 0;
            for (; j < nin; ++j) {
                const int s = j % NST;
                const uint32_t fb = lbmt::smem_u32(&full_bar[s]);
                if (j == A.withhold) continue;
                if (j >= NST && !lbmt::mbar_wait(lbmt::smem_u32(&empty_bar[s]), ((j / NST) - 1) & 1, &abort_flag))
                    break;
                int y = y0 - 3 + j;
                if (DIRICHLET && (y < 0 || y >= ny)) {
                    lbmt::mbar_arrive(fb);
                    continue;
                }
                if (!DIRICHLET) y = wrap_row(y, ny);   // rows y0 - 3 .. y1 + 2: more than one wrap when ny = 2
                lbmt::mbar_arrive_expect_tx(fb, G::ROW_BYTES);
                lbmt::tma_load_3d(sbase + s * G::STAGE_BYTES, mapp, X0 - HL, y, 0, fb);
            }
            for (int q = (j > NST ? j - NST : 0); q < j; ++q)
                if (q != A.withhold) lbmt::mbar_drain(lbmt::smem_u32(&full_bar[q % NST]), (q / NST) & 1);
            if (abort_flag) atomicExch(A.timeout, 1);
        }
        return;
    }

    const E* __restrict__ src = static_cast<const E*>(A.src);
    E* __restrict__ dst = static_cast<E*>(A.dst);
    const long long plane = A.plane;
    const int xs = X0 - 2 + TB3_OUT * warp + lane;   // this lane's S1 column
    const int xc = DIRICHLET ? (xs < 0 ? 0 : (xs >= nx ? nx - 1 : xs)) : ((xs % nx) + nx) % nx;
    const bool out_lane = (lane >= 2) && (lane < 2 + TB3_OUT) && (xs >= 0) && (xs < nx);
    const bool staged = DIRICHLET || (xs >= 1 && xs + 1 <= nx - 1);
    const int xl = (xc == 0) ? nx - 1 : xc - 1, xr = (xc == nx - 1) ? 0 : xc + 1;
    const int idx = xs - X0 + HL;
    const float fa = A.af, fb = A.bf;
    const float Dk[5] = {-1.f, -1.f, 1.f, 1.f, 1.f};

    float p1[4][5], k1[5], p2[4][5], k2[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        k1[k] = k2[k] = 0.f;
#pragma unroll
        for (int d = 0; d < 4; ++d) p1[d][k] = p2[d][k] = 0.f;
    }
    bool ok = lbmt::mbar_wait(lbmt::smem_u32(&full_bar[0]), 0, &abort_flag) &&
              lbmt::mbar_wait(lbmt::smem_u32(&full_bar[1 % NST]), (1 / NST) & 1, &abort_flag);
    for (int i = 0; i + 2 < nin; ++i) {
        const int r = y0 - 2 + i;                    // S1 row, from staged rows i, i+1, i+2
        {
            const int j = i + 2;
            ok = ok && lbmt::mbar_wait(lbmt::smem_u32(&full_bar[j % NST]), (j / NST) & 1, &abort_flag);
        }
        if (!__all_sync(0xffffffffu, ok)) break;
        constexpr uint32_t ES = sizeof(E), PL = WIN * sizeof(E);
        const uint32_t rm = sbase + (i % NST) * G::STAGE_BYTES + idx * ES;
        const uint32_t rc = sbase + ((i + 1) % NST) * G::STAGE_BYTES + idx * ES;
        const uint32_t rp = sbase + ((i + 2) % NST) * G::STAGE_BYTES + idx * ES;
        float c1[4][5];
        {
            float f[4][5];
            if (staged) {
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    f[0][k] = Fmt<K>::ld(lbmt::lds<E>(rc + (0 * 5 + k) * PL - ES));
                    f[2][k] = Fmt<K>::ld(lbmt::lds<E>(rc + (2 * 5 + k) * PL + ES));
                    f[1][k] = Fmt<K>::ld(lbmt::lds<E>(rm + (1 * 5 + k) * PL));
                    f[3][k] = Fmt<K>::ld(lbmt::lds<E>(rp + (3 * 5 + k) * PL));
                }
            } else {
                const int ry = (r < 0) ? r + ny : (r >= ny ? r - ny : r);
                const int rmy = (ry == 0) ? ny - 1 : ry - 1, rpy = (ry == ny - 1) ? 0 : ry + 1;
                const long long o = (long long)ry * A.pitch;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    f[0][k] = sload<K>(src + (0 * 5 + k) * plane + o + xl);
                    f[2][k] = sload<K>(src + (2 * 5 + k) * plane + o + xr);
                    f[1][k] = sload<K>(src + (1 * 5 + k) * plane + (long long)rmy * A.pitch + xc);
                    f[3][k] = sload<K>(src + (3 * 5 + k) * plane + (long long)rpy * A.pitch + xc);
                }
            }
            if (DIRICHLET) {
                const bool bot = r == 0, top = r == ny - 1;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if (xc == 0) f[0][k] = Dk[k] * Fmt<K>::ld(lbmt::lds<E>(rc + (2 * 5 + k) * PL));
                    if (xc == nx - 1) f[2][k] = Dk[k] * Fmt<K>::ld(lbmt::lds<E>(rc + (0 * 5 + k) * PL));
                    if (bot) f[1][k] = Dk[k] * Fmt<K>::ld(lbmt::lds<E>(rc + (3 * 5 + k) * PL));
                    if (top) f[3][k] = Dk[k] * Fmt<K>::ld(lbmt::lds<E>(rc + (1 * 5 + k) * PL));
                }
            }
            float U[5], rx[5], ry2[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                rx[k] = f[1][k] + f[3][k];
                ry2[k] = f[0][k] + f[2][k];
                U[k] = rx[k] + ry2[k];
            }
            collide<float>(f, U, rx, ry2, fa, fb, c1);
            if (DIRICHLET && !(r >= 0 && r < ny))
#pragma unroll
                for (int d = 0; d < 4; ++d)
#pragma unroll
                    for (int k = 0; k < 5; ++k) c1[d][k] = 0.f;
        }
        __syncwarp();
        if (lane == 0) lbmt::mbar_arrive(lbmt::smem_u32(&empty_bar[i % NST]));
        const int q2 = r - 1;
        if (q2 >= y0 - 1) {
            float c2[4][5];
            level_step<DIRICHLET>(p1, k1, c1[3], q2, xs, nx, ny, fa, fb, c2);
            if (DIRICHLET && !(q2 >= 0 && q2 < ny))
#pragma unroll
                for (int d = 0; d < 4; ++d)
#pragma unroll
                    for (int k = 0; k < 5; ++k) c2[d][k] = 0.f;
            const int q3 = r - 2;
            if (q3 >= y0) {
                float o[4][5];
                level_step<DIRICHLET>(p2, k2, c2[3], q3, xs, nx, ny, fa, fb, o);
                if (out_lane) {
                    const long long off = (long long)q3 * A.pitch + xs;
#pragma unroll
                    for (int d = 0; d < 4; ++d)
#pragma unroll
                        for (int k = 0; k < 5; ++k) dst[(d * 5 + k) * plane + off] = Fmt<K>::st(o[d][k]);
                }
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                k2[k] = p2[1][k];
#pragma unroll
                for (int d = 0; d < 4; ++d) p2[d][k] = c2[d][k];
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            k1[k] = p1[1][k];
#pragma unroll
            for (int d = 0; d < 4; ++d) p1[d][k] = c1[d][k];
        }
    }
    if (lane == 0 && abort_flag) atomicExch(A.timeout, 1);
}

template <int K, bool DIRICHLET>
__global__ void __launch_bounds__(TBT_THREADS, LBM_TBT3_MIN_BLOCKS) tbt3_kernel(const __grid_constant__ CUtensorMap map, TbtArgs A)
{
    tbt3_body<K, DIRICHLET>(&map, A, blockIdx.x * TBT3_OUT, blockIdx.y * A.rows);
}

// ---------------------------------------------------------------------------
// Batches of lattices, three steps per pass (lbm_batch.cu, mode 2): one block per tile
// {lattice, X0, y0} of a flat list, each running tbt3_body on its lattice with that
// lattice's row map of the source arena.  The maps live in global memory, written by the
// host before the launch; a lattice's planes sit at its element offset in each arena.
// ---------------------------------------------------------------------------
struct BatchLatT3 {
    long long off;         // element offset of plane 0 in each arena
    long long plane;       // elements per plane = ny * pitch
    int nx, ny, pitch;
    float af, bf;          // cK / c, cmu / c in FP32
    int pad_;
};

struct BatchTbtArgs {
    const int4* tiles;          // {lattice, X0, y0, 0} per block
    const BatchLatT3* lat;
    const CUtensorMap* maps;    // [lattice][arena]: row maps (box width Tbt3Geom::WIN)
    void* arenaA;
    void* arenaB;
    int parity;                 // 0: read arena A, write arena B
    int rows;                   // output rows per tile
    int* timeout;               // set when a bounded wait ran out
};

template <int K, bool DIRICHLET>
__global__ void __launch_bounds__(TBT_THREADS, LBM_TBT3_MIN_BLOCKS) batch_tbt3_kernel(BatchTbtArgs B)
{
    using E = typename Fmt<K>::E;
    const int4 t = B.tiles[blockIdx.x];
    const BatchLatT3 L = B.lat[t.x];
    E* a = static_cast<E*>(B.arenaA) + L.off;
    E* b = static_cast<E*>(B.arenaB) + L.off;
    TbtArgs A;
    A.src = B.parity ? b : a;
    A.dst = B.parity ? a : b;
    A.nx = L.nx;
    A.ny = L.ny;
    A.pitch = L.pitch;
    A.plane = L.plane;
    A.af = L.af;
    A.bf = L.bf;
    A.rows = B.rows;
    A.timeout = B.timeout;
    A.withhold = -1;
    A.scale = 1.f;
    A.inv_s = 1.f;
    A.sat = nullptr;
    A.l2_ahead = 0;
    tbt3_body<K, DIRICHLET>(B.maps + 2 * t.x + B.parity, A, t.y, t.z);
}

}  // namespace lbmk
