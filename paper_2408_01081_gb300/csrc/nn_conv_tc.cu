// 3x3 circular convolution of the surrogate as an implicit GEMM on the fifth-
// generation tensor cores: tcgen05.mma (kind::f16, BF16 operands from shared
// memory, FP32 accumulator in tensor memory), issued by one elected lane of a warp.
//
// Tiling.  A CTA computes MT tiles of 128 output pixels (each 16 rows x 8 columns;
// the MT tiles side by side) for BN output channels: the accumulator
// D[pixel][co] of tile j sits in tensor-memory lanes 0..127 (lane = pixel) and
// columns j BN .. j BN + BN - 1 (two such accumulators, alternating between output
// blocks).  The input block with its one-pixel halo ((16 + 2) x (8 MT + 2) pixels)
// is staged per 16-channel chunk as two planes of 8 channels, one 16-byte row per
// pixel: the K-major operand layout without swizzle, whose 8-row core matrices are
// then 8 consecutive pixels of one image row.  A stencil tap (dy, dx) is a
// descriptor into that same block, started dy halo rows and dx pixels further on,
// with the stride between 8-row groups (SBO) = one halo row and between the two K
// halves (LBO) = one plane; no im2col copy is made.  The weights of a chunk's nine
// taps are copied (cp.async) into the same layout with output channels as rows;
// they stay resident for the whole kernel when all chunks fit in shared memory.
//
// Precision is that of the mma.sync kernels: activations split into BF16 hi + lo
// (two MMAs per tap; one with act_bf16), BF16 weights, FP32 accumulation.
//
// Pipeline (conv3_tc_kernel below): persistent CTAs, one per SM, with warp roles.
// Producer warps copy the FP32 chunks a few steps ahead with cp.async and convert
// them into the BF16 operand buffers; one warp issues the MMAs; four warps read the
// accumulators (tcgen05.ld), add the bias, apply ReLU and store FP32 (or add into
// the destination); one warp streams the weights when they are not resident.  The
// roles hand buffers and accumulators to each other through mbarriers.
//
// Every wait is bounded (about two seconds of SM clock).  A wait that runs out
// sets a device flag (read by conv3_tc_take_timeout) and makes every role leave its
// loop; the MMA warp waits (bounded) for the MMAs it has in flight, and the CTA
// frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nn_conv_tc.h"

#ifndef LBM_CONV_TC_STAGES
#define LBM_CONV_TC_STAGES 0    // BF16 operand buffers; 0 = three
#endif
#ifndef LBM_CONV_TC_RAWD
#define LBM_CONV_TC_RAWD 3      // FP32 chunks in flight per producer thread
#endif

namespace {

__device__ int g_tc_timeout;

constexpr int kMaxStages = 4;
constexpr long long kWaitCycles = 4000000000LL;
constexpr int kSmemLimit = 227 * 1024 - 1024;   // dynamic shared memory per CTA (static part kept below 1 KB)
constexpr int kTmemColumns = 512;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading-dimension (K) byte offset
// and stride-dimension (M / N) byte offset, each >> 4 in 14 bits; descriptor
// version 1 at bits 46-47; base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), no negation, both K-major (bits 15, 16 = 0), dense,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (+)= A B^T with A, B in shared memory (descriptors) and D in tensor memory.  Executed by a
// whole converged warp: one lane (elect.sync) issues the instruction, so that the operands can
// stay in warp-uniform registers.
__device__ __forceinline__ void mma_bf16_ss_elect(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                                  uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
        "}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on the mbarrier once every tcgen05 operation issued so far by the elected lane has completed
__device__ __forceinline__ void mma_commit_elect(uint32_t bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t"
        "}\n" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t"
        "}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// wait for the completion of the barrier's phase with this parity; false after ~2 s
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) { return *reinterpret_cast<const uint32_t*>(&v); }

template <int BN, int MT, bool LO>
struct TcShape {
    static constexpr int TH = 16, TW = 8 * MT;               // output block (MT tiles of 16 x 8)
    static constexpr int HWD = TW + 2, HP = (TH + 2) * HWD;  // halo block width, pixels
    static constexpr int NQ = (HP * 4 + 255) / 256;          // 16-byte copies per producer thread per chunk
    static constexpr int RAW_BYTES = HP * 64;                // one FP32 chunk of the halo block (16 channels)
    static constexpr int PLANE = HP * 16;                    // 8 channels of every halo pixel (BF16)
    static constexpr int A_HALF = 2 * PLANE;                 // one BF16 half of a 16-channel chunk
    static constexpr int A_BYTES = (LO ? 2 : 1) * A_HALF;
    static constexpr int B_PLANE = BN * 16;                  // 8 input channels of BN weight rows
    static constexpr int B_TAP = 2 * B_PLANE;
    static constexpr int B_BYTES = 9 * B_TAP;                // weights of one 16-channel chunk
    static constexpr int ACC = MT * BN;                      // accumulator columns of one block
    static constexpr int COLS = 2 * ACC <= 32 ? 32 : 2 * ACC <= 64 ? 64 : 2 * ACC <= 128 ? 128
                                : 2 * ACC <= 256 ? 256 : 512;   // two accumulators
    static constexpr uint32_t IDESC = idesc_bf16_f32(128, BN);
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 128 && MT >= 1 && MT <= 2, "tile");
};

// warp roles
constexpr int kProducerWarps = 8;       // warps 0-7: activations (cp.async FP32 -> BF16 hi / lo)
constexpr int kEpilogueWarp0 = 8;       // warps 8-11: accumulator -> global (TMEM lanes 32 (w % 4) ..)
constexpr int kMmaWarp = 12;            // warp 12: tensor-memory allocation; the MMA loop (elected lane issues)
constexpr int kWeightWarp = 13;         // warp 13: weights per chunk when they are not resident
constexpr int kThreads = 14 * 32;
constexpr int kProducers = kProducerWarps * 32;
static_assert(kEpilogueWarp0 % 4 == 0 && kEpilogueWarp0 + 4 == kMmaWarp && kProducers == 256, "warp roles");

struct TcConf {
    int stages;     // BF16 operand buffers (and weight buffers when not resident)
    int rawd;       // FP32 chunks in flight per producer thread
    int resident;   // the weights of all chunks stay in shared memory
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// bounded wait that also gives up once another role has given up (`abort_flag`)
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void cp_async_wait_upto(int n)   // at most n of this thread's groups pending
{
    if (n <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else if (n == 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else asm volatile("cp.async.wait_group 3;" ::: "memory");
}

// Persistent, warp-specialised.  CTA b takes the output blocks b, b + gridDim.x, ...
// (output channels of blockIdx.y) and walks their 16-channel chunks as one sequence
// g = 0 .. G-1.  Barriers: full[s] (operands of the chunk in buffer s staged: one
// arrival per producer warp, and one from the weight warp when weights stream), empty[s] (the MMAs that
// read buffer s completed: tcgen05.commit), acc_full[b] (the MMAs of the block in
// accumulator b completed), acc_empty[b] (the epilogue warps have read accumulator b:
// one arrival per warp).
// Shared memory: [BF16 operand buffers][FP32 chunk ring][weights].
template <int BN, int MT, bool LO>
__global__ void __launch_bounds__(kThreads, 1) conv3_tc_kernel(ConvTcArgs a, TcConf cf)
{
    using S = TcShape<BN, MT, LO>;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    volatile int* abort_v = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = a.W / S::TW, tiles_y = a.H / S::TH;
    const int ntiles = a.B * tiles_x * tiles_y;
    const int co0 = blockIdx.y * BN;
    const int Cin = a.C1 + a.C2;
    const int nchunk = Cin / 16;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int G = my_tiles * nchunk;
    const int stages = cf.stages, rawd = cf.rawd;
    uint8_t* const ring = smem;
    uint8_t* const raw = smem + stages * S::A_BYTES;
    uint8_t* const wts = raw + rawd * S::RAW_BYTES;

    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"((uint32_t)S::COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        abort_flag = 0;
        for (int i = 0; i < stages; ++i) {
            mbar_init(smem_addr(&full[i]), kProducerWarps + (cf.resident ? 0 : 1));   // one arrival per warp
            mbar_init(smem_addr(&empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_addr(&acc_full[i]), 1);
            mbar_init(smem_addr(&acc_empty[i]), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights of one chunk c into `dst`: row co, plane p = input channels 16 c + 8 p .. + 7, nine taps
    auto copy_b = [&](int c, uint8_t* dst, int first, int step) {
        const uint32_t bs = smem_addr(dst);
        const int ci0 = c * 16;
        for (int q = first; q < 9 * BN * 2; q += step) {
            const int plane = q & 1, r = q >> 1;         // r = co * 9 + tap
            const int co = r / 9, tap = r - co * 9;
            cp_async16(bs + tap * S::B_TAP + plane * S::B_PLANE + co * 16,
                       a.w + ((long long)(co0 + co) * 9 + tap) * Cin + ci0 + plane * 8);
        }
    };
    if (cf.resident && G > 0) {
        for (int c = 0; c < nchunk; ++c) copy_b(c, wts + c * S::B_BYTES, tid, kThreads);
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    auto tile_of = [&](int t, int& n, int& ty0, int& tx0) {
        const int tile = (int)blockIdx.x + t * (int)gridDim.x;
        n = tile / (tiles_x * tiles_y);
        ty0 = ((tile / tiles_x) % tiles_y) * S::TH;
        tx0 = (tile % tiles_x) * S::TW;
    };

    if (warp < kProducerWarps) {
        // ---- activations: FP32 chunk g + rawd copied while chunk g is converted ----
        // pixel indices of this thread's halo elements in the block being copied, the same for
        // every channel chunk of the block: full resolution, and halved for an x1 stored at half size
        int cached_t = -1;
        uint32_t pix_full[S::NQ], pix_half[S::NQ];
        auto issue_raw = [&](int g) {
            const int t = g / nchunk, ci0 = (g - t * nchunk) * 16;
            if (t != cached_t) {
                int n, ty0, tx0;
                tile_of(t, n, ty0, tx0);
#pragma unroll
                for (int i = 0; i < S::NQ; ++i) {
                    const int hp = (tid + kProducers * i) >> 2;
                    const int hy = hp / S::HWD, hx = hp - hy * S::HWD;
                    const int sy = (ty0 + hy - 1) & (a.H - 1), sx = (tx0 + hx - 1) & (a.W - 1);
                    pix_full[i] = ((uint32_t)n * (uint32_t)a.H + (uint32_t)sy) * (uint32_t)a.W + (uint32_t)sx;
                    pix_half[i] = ((uint32_t)n * (uint32_t)(a.H >> 1) + (uint32_t)(sy >> 1)) * (uint32_t)(a.W >> 1) +
                                  (uint32_t)(sx >> 1);
                }
                cached_t = t;
            }
            const bool from1 = ci0 < a.C1;
            const float* base = from1 ? a.x1 + ci0 : a.x2 + (ci0 - a.C1);
            const size_t cstride = (size_t)(from1 ? a.C1 : a.C2);
            const bool half = from1 && a.x1_half;          // nearest upsampling of a half-size x1
            const uint32_t dst = smem_addr(raw + (g % rawd) * S::RAW_BYTES);
#pragma unroll
            for (int i = 0; i < S::NQ; ++i) {
                const int q = tid + kProducers * i;
                if (q < S::HP * 4)
                    cp_async16(dst + q * 16, base + (size_t)(half ? pix_half[i] : pix_full[i]) * cstride + (q & 3) * 4);
            }
        };
        for (int d = 0; d < rawd; ++d) {
            if (d < G) issue_raw(d);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        for (int g = 0; g < G; ++g) {
            const int s = g % stages;
            // (warp-uniform, so that the whole warp leaves together after an abort)
            if (g >= stages &&
                !__all_sync(0xffffffffu,
                            wait_or_abort(smem_addr(&empty[s]), (uint32_t)((g / stages - 1) & 1), abort_v)))
                break;
            cp_async_wait_upto(rawd - 1);                  // this thread's copies of chunk g have landed
            const uint8_t* src = raw + (g % rawd) * S::RAW_BYTES;
            uint8_t* st = ring + s * S::A_BYTES;
#pragma unroll
            for (int i = 0; i < S::NQ; ++i) {
                const int q = tid + kProducers * i;
                if (q < S::HP * 4) {
                    const int hp = q >> 2, c4 = q & 3;
                    const float4 v = *reinterpret_cast<const float4*>(src + q * 16);
                    const int off = (c4 >> 1) * S::PLANE + hp * 16 + (c4 & 1) * 8;
                    const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
                    *reinterpret_cast<uint2*>(st + off) = make_uint2(bf16x2_bits(h01), bf16x2_bits(h23));
                    if constexpr (LO) {
                        const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
                        const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
                        const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
                        *reinterpret_cast<uint2*>(st + S::A_HALF + off) =
                            make_uint2(bf16x2_bits(l01), bf16x2_bits(l23));
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> tensor core
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&full[s]));              // for the whole warp
            if (g + rawd < G) issue_raw(g + rawd);          // into the ring slot just converted (own elements)
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else if (warp < kEpilogueWarp0 + 4) {
        // ---- epilogue: accumulator of block t -> bias, ReLU, FP32 stores ----
        const int q = warp & 3;
        const int m = q * 32 + lane;                        // pixel of a 128-pixel tile = TMEM lane
        for (int t = 0; t < my_tiles; ++t) {
            const bool ok = wait_or_abort(smem_addr(&acc_full[t & 1]), (uint32_t)((t >> 1) & 1), abort_v);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            int n, ty0, tx0;
            tile_of(t, n, ty0, tx0);
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                const int oy = ty0 + (m >> 3), ox = tx0 + 8 * j + (m & 7);
                const long long p = ((long long)n * a.H + oy) * a.W + ox;
                const uint32_t col0 = (uint32_t)((t & 1) * S::ACC + j * BN);
#pragma unroll 1
                for (int cc = 0; cc < BN; cc += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + col0 + (uint32_t)cc, v);
                    const int co = co0 + cc;                // 16 channels, all in y1 or all in y2
                    float* dst = co < a.Co1 ? a.y1 + p * a.Co1 + co : a.y2 + p * (a.Cout - a.Co1) + (co - a.Co1);
#pragma unroll
                    for (int e = 0; e < 16; e += 4) {
                        float4 r = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                        if (a.bias) {
                            const float4 b = __ldg(reinterpret_cast<const float4*>(a.bias + co + e));
                            r.x += b.x; r.y += b.y; r.z += b.z; r.w += b.w;
                        }
                        if (a.relu) {
                            r.x = fmaxf(r.x, 0.f); r.y = fmaxf(r.y, 0.f); r.z = fmaxf(r.z, 0.f); r.w = fmaxf(r.w, 0.f);
                        }
                        float4* d4 = reinterpret_cast<float4*>(dst + e);
                        if (a.beta) {
                            const float4 o = *d4;
                            r.x += o.x; r.y += o.y; r.z += o.z; r.w += o.w;
                        }
                        *d4 = r;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&acc_empty[t & 1]));
        }
    } else if (warp == kMmaWarp) {
        // ---- MMAs: the whole warp runs the loop (warp-uniform control flow and operands),
        //      one elected lane issues each instruction ----
        int last = -1;
        for (int g = 0; g < G; ++g) {
            const int t = g / nchunk, c = g - t * nchunk, s = g % stages;
            // accumulator t & 1 was last read by the epilogue of block t - 2
            if (c == 0 && t >= 2 &&
                !__all_sync(0xffffffffu, wait_or_abort(smem_addr(&acc_empty[t & 1]),
                                                       (uint32_t)(((t >> 1) - 1) & 1), abort_v)))
                break;
            if (!__all_sync(0xffffffffu, wait_or_abort(smem_addr(&full[s]), (uint32_t)((g / stages) & 1), abort_v)))
                break;
            tc_fence_after();
            const uint32_t ab = smem_addr(ring + s * S::A_BYTES);
            const uint32_t bb = smem_addr(wts + (cf.resident ? c : s) * S::B_BYTES);
            const uint32_t acc = tmem + (uint32_t)((t & 1) * S::ACC);
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap - dy * 3;
                const uint64_t bd = smem_desc(bb + tap * S::B_TAP, S::B_PLANE, 128);
#pragma unroll
                for (int j = 0; j < MT; ++j) {
                    const uint32_t aoff = (uint32_t)((dy * S::HWD + 8 * j + dx) * 16);
                    const uint32_t d = acc + (uint32_t)(j * BN);
                    mma_bf16_ss_elect(d, smem_desc(ab + aoff, S::PLANE, S::HWD * 16), bd, S::IDESC,
                                      (c | tap) != 0);
                    if constexpr (LO)
                        mma_bf16_ss_elect(d, smem_desc(ab + S::A_HALF + aoff, S::PLANE, S::HWD * 16), bd,
                                          S::IDESC, 1u);
                }
            }
            mma_commit_elect(smem_addr(&empty[s]));
            if (c == nchunk - 1) mma_commit_elect(smem_addr(&acc_full[t & 1]));
            last = g;
        }
        // after an abort: wait (bounded) for the MMAs in flight before the memory is freed
        if (*abort_v && last >= 0) mbar_wait(smem_addr(&empty[last % stages]), (uint32_t)((last / stages) & 1));
        __syncwarp();
    } else if (warp == kWeightWarp && !cf.resident) {
        // ---- weights of chunk g + 1 copied while chunk g is consumed ----
        if (G > 0) copy_b(0, wts, lane, 32);
        asm volatile("cp.async.commit_group;" ::: "memory");
        for (int g = 0; g < G; ++g) {
            const int s = g % stages;
            bool ok = true;
            if (g + 1 < G) {
                const int g1 = g + 1, s1 = g1 % stages;
                if (g1 >= stages)
                    ok = __all_sync(0xffffffffu,
                                    wait_or_abort(smem_addr(&empty[s1]), (uint32_t)((g1 / stages - 1) & 1), abort_v));
                if (ok) copy_b(g1 % nchunk, wts + s1 * S::B_BYTES, lane, 32);
            }
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 1;" ::: "memory");   // chunk g landed
            if (!ok) break;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&full[s]));
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort_v) atomicExch(&g_tc_timeout, 1);
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)S::COLS)
                     : "memory");
    }
}

constexpr int kMaxDevices = 64;

struct VariantInfo {
    int ready;          // attributes set and read
    int regs_per_cta;   // registers allocated to one CTA (per-warp granularity of 256)
    int static_smem;
};
// filled on the first launch of a variant on a device; first launches racing from several host
// threads write the same values
VariantInfo g_var[kMaxDevices][12];
int g_sms[kMaxDevices], g_smem_sm[kMaxDevices], g_smem_reserved[kMaxDevices];

// CTAs that fit on one SM with `smem` bytes of dynamic shared memory: the limits of
// threads, registers and shared memory (carveout at its maximum, which the variant requests)
int ctas_per_sm(const VariantInfo& v, int dev, long long smem)
{
    int k = 2048 / kThreads;
    const int by_regs = 65536 / v.regs_per_cta;
    if (by_regs < k) k = by_regs;
    const long long by_smem = g_smem_sm[dev] / (smem + v.static_smem + g_smem_reserved[dev]);
    if (by_smem < k) k = (int)by_smem;
    return k;
}

template <int BN, int MT, bool LO>
bool launch_variant(const ConvTcArgs& a, cudaStream_t s, int stages, int slot)
{
    using S = TcShape<BN, MT, LO>;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
    VariantInfo& v = g_var[dev][slot];
    if (!v.ready) {
        cudaFuncAttributes fa;
        if (cudaFuncSetAttribute(conv3_tc_kernel<BN, MT, LO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemLimit) != cudaSuccess ||
            cudaFuncSetAttribute(conv3_tc_kernel<BN, MT, LO>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, conv3_tc_kernel<BN, MT, LO>) != cudaSuccess ||
            cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&g_smem_sm[dev], cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&g_smem_reserved[dev], cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
                cudaSuccess)
            return false;
        v.regs_per_cta = (kThreads / 32) * ((fa.numRegs * 32 + 255) / 256 * 256);
        v.static_smem = (int)fa.sharedSizeBytes;
        v.ready = 1;
    }
    const int nchunk = (a.C1 + a.C2) / 16;
    TcConf cf{stages > 0 ? stages : 3, LBM_CONV_TC_RAWD, 1};
    if (cf.stages < 2 || cf.stages > kMaxStages || cf.rawd < 1 || cf.rawd > 4) return false;
    // largest configuration that fits: resident weights first, then fewer FP32 chunks in
    // flight, then fewer operand buffers
    long long smem = 0;
    for (;;) {
        const long long base = (long long)cf.stages * S::A_BYTES + (long long)cf.rawd * S::RAW_BYTES;
        const long long res = base + (long long)nchunk * S::B_BYTES;
        const long long str = base + (long long)cf.stages * S::B_BYTES;
        if (res <= kSmemLimit) { cf.resident = 1; smem = res; break; }
        if (str <= kSmemLimit) { cf.resident = 0; smem = str; break; }
        if (cf.rawd > 2) --cf.rawd;
        else if (cf.stages > 2) --cf.stages;
        else return false;
    }
    const int per_sm = ctas_per_sm(v, dev, smem);
    // the CTAs resident on one SM must fit in its tensor memory together, so that no
    // allocation ever waits for another CTA
    if (per_sm < 1 || per_sm * S::COLS > kTmemColumns) return false;
    const long long ntiles = (long long)a.B * (a.H / S::TH) * (a.W / S::TW);
    const int cob = a.Cout / BN;
    long long gx = ((long long)per_sm * g_sms[dev] + cob - 1) / cob;
    if (gx > ntiles) gx = ntiles;
    if (gx < 1) gx = 1;
    conv3_tc_kernel<BN, MT, LO><<<dim3((unsigned)gx, (unsigned)cob), kThreads, (size_t)smem, s>>>(a, cf);
    return true;
}

template <int BN>
bool launch_bn(const ConvTcArgs& a, cudaStream_t s, int stages, int mt)
{
    const int base = (BN == 128 ? 8 : BN == 64 ? 4 : 0);
    if (mt == 2) return a.act_bf16 ? launch_variant<BN, 2, false>(a, s, stages, base + 0)
                                   : launch_variant<BN, 2, true>(a, s, stages, base + 1);
    return a.act_bf16 ? launch_variant<BN, 1, false>(a, s, stages, base + 2)
                      : launch_variant<BN, 1, true>(a, s, stages, base + 3);
}

}  // namespace

bool conv3_tc_launch(const ConvTcArgs& a, cudaStream_t s, int stages)
{
    const auto aligned = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    if (a.H < 16 || a.W < 8 || a.C1 % 32 || a.C2 % 32 || a.Co1 % 16 || a.Cout % 32 || a.Co1 > a.Cout ||
        a.B <= 0 || (long long)a.B * a.H * a.W > (1LL << 31) - 1 || !aligned(a.x1) || !aligned(a.x2) ||
        !aligned(a.w) || !aligned(a.bias) || !aligned(a.y1) || !aligned(a.y2))
        return false;
    if (stages <= 0) stages = LBM_CONV_TC_STAGES;
    const int bn = a.Cout % 128 == 0 ? 128 : a.Cout % 64 == 0 ? 64 : 32;
#ifdef LBM_CONV_TC_MT
    const int mt = (LBM_CONV_TC_MT == 2 && a.W >= 16) ? 2 : 1;
#else
    // two 128-pixel tiles per CTA (one B operand for both) wherever the width allows
    const int mt = a.W >= 16 ? 2 : 1;
#endif
    if (bn == 128) return launch_bn<128>(a, s, stages, mt);
    if (bn == 64) return launch_bn<64>(a, s, stages, mt);
    return launch_bn<32>(a, s, stages, mt);
}

bool conv3_tc_take_timeout(cudaStream_t s)
{
    int v = 0, zero = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_tc_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return false;
    if (cudaStreamSynchronize(s) != cudaSuccess) return false;
    if (v) {
        cudaMemcpyToSymbolAsync(g_tc_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
    }
    return v != 0;
}
