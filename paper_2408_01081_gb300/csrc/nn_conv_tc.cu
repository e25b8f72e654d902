// 3x3 circular convolution of the surrogate as an implicit GEMM on the fifth-
// generation tensor cores: tcgen05.mma (kind::f16, BF16 operands from shared
// memory, FP32 accumulator in tensor memory), one thread issuing for the CTA.
//
// Tiling.  A CTA computes MT tiles of 128 output pixels (each 16 rows x 8 columns;
// the MT tiles side by side) for BN output channels: the accumulator
// D[pixel][co] of tile j sits in tensor-memory lanes 0..127 (lane = pixel) and
// columns j BN .. j BN + BN - 1.  The input block with its one-pixel halo
// ((16 + 2) x (8 MT + 2) pixels) is staged per 16-channel chunk as two planes of
// 8 channels, one 16-byte row per pixel: the K-major operand layout without
// swizzle, whose 8-row core matrices are then 8 consecutive pixels of one image
// row.  A stencil tap (dy, dx) is a descriptor into that same block, started dy
// halo rows and dx pixels further on, with the stride between 8-row groups (SBO)
// = one halo row and between the two K halves (LBO) = one plane; no im2col copy
// is made.  The weights of the chunk's nine taps are copied (cp.async) into the
// same layout with output channels as rows.
//
// Precision is that of the mma.sync kernels: activations split into BF16 hi + lo
// (two MMAs per tap; one with act_bf16), BF16 weights, FP32 accumulation.
//
// Pipeline.  `stages` buffers.  All 256 threads stage chunk c (FP32 loads, BF16
// split, shared stores; weights by cp.async) while the tensor core works on the
// previous chunks; after a proxy fence and a barrier one thread issues the
// chunk's 9 MT (hi/lo) MMAs and commits them to the buffer's mbarrier, which the
// threads wait on before they refill that buffer.  Epilogue: warp w reads lanes
// 32 (w % 4) .. of the accumulator (tcgen05.ld), adds the bias, applies ReLU and
// stores FP32 (or adds into the destination).
//
// Every wait is bounded (about two seconds of SM clock).  A wait that runs out
// sets a device flag (read by conv3_tc_take_timeout); the CTA then stops issuing,
// waits (bounded) for the MMAs it has in flight, frees its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nn_conv_tc.h"

#ifndef LBM_CONV_TC_STAGES
#define LBM_CONV_TC_STAGES 0    // pipeline depth; 0 = chosen per variant
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

__device__ __forceinline__ void mma_bf16_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
        "}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on the mbarrier once every tcgen05 operation issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
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
    static constexpr int NQ = (HP * 4 + 255) / 256;          // 16-byte loads per thread per chunk
    static constexpr int PLANE = HP * 16;                    // 8 channels of every halo pixel
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

// Persistent CTAs: CTA b takes the output blocks b, b + gridDim.x, ... (all with the
// output channels of blockIdx.y), and walks their 16-channel chunks as one sequence
// g = 0 .. G-1, so the pipeline runs on across blocks.  Per chunk g: the input chunk
// loaded into registers one step earlier is converted and stored (buffer g % stages);
// the loads of chunk g + 1 are issued; the weights of chunk g + 1 are copied (unless
// all chunks' weights are resident); one thread issues the MMAs of chunk g into
// accumulator (block & 1).  The epilogue of block t - 1 runs right after the first
// MMAs of block t are issued, so it overlaps them.
// CTAs per SM the register budget is sized for (shared and tensor memory allow as many)
constexpr int tc_min_blocks(int BN, int MT) { return BN == 32 ? 3 : (BN == 128 && MT == 2) ? 1 : 2; }

template <int BN, int MT, bool LO>
__global__ void __launch_bounds__(256, tc_min_blocks(BN, MT)) conv3_tc_kernel(ConvTcArgs a, int stages, int resident)
{
    using S = TcShape<BN, MT, LO>;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar[kMaxStages];   // buffer s: MMAs of its latest chunk done
    __shared__ __align__(8) uint64_t accbar[2];          // accumulator b: MMAs of its latest block done
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = a.W / S::TW, tiles_y = a.H / S::TH;
    const int ntiles = a.B * tiles_x * tiles_y;
    const int co0 = blockIdx.y * BN;
    const int Cin = a.C1 + a.C2;
    const int nchunk = Cin / 16;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int G = my_tiles * nchunk;
    uint8_t* const ring = smem;                            // stages x A_BYTES
    uint8_t* const wts = smem + stages * S::A_BYTES;       // resident: nchunk x B_BYTES, else stages x B_BYTES

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"((uint32_t)S::COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < stages; ++i) mbar_init(smem_addr(&mbar[i]), 1);
        mbar_init(smem_addr(&accbar[0]), 1);
        mbar_init(smem_addr(&accbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
    // chunk g of the halo block into registers: pixel hp = hy * HWD + hx at image
    // (ty0 + hy - 1, tx0 + hx - 1), periodic; four channels per load
    auto load_a = [&](int g, float4 (&v)[S::NQ]) {
        const int t = g / nchunk, ci0 = (g - t * nchunk) * 16;
        int n, ty0, tx0;
        tile_of(t, n, ty0, tx0);
        const bool from1 = ci0 < a.C1;
        const float* base = from1 ? a.x1 : a.x2;
        const int cstride = from1 ? a.C1 : a.C2;
        const int coff = from1 ? ci0 : ci0 - a.C1;
        const int half = (from1 && a.x1_half) ? 1 : 0;     // nearest upsampling of a half-size x1
        const int hs = a.H >> half, ws = a.W >> half;
#pragma unroll
        for (int i = 0; i < S::NQ; ++i) {
            const int q = tid + 256 * i;
            if (q < S::HP * 4) {
                const int hp = q >> 2, c4 = q & 3;
                const int hy = hp / S::HWD, hx = hp - hy * S::HWD;
                const int sy = (ty0 + hy - 1) & (a.H - 1), sx = (tx0 + hx - 1) & (a.W - 1);
                const long long spix = ((long long)n * hs + (sy >> half)) * ws + (sx >> half);
                v[i] = __ldg(reinterpret_cast<const float4*>(base + spix * cstride + coff + c4 * 4));
            }
        }
    };
    // registers -> BF16 hi (and lo) planes of one buffer
    auto store_a = [&](const float4 (&v)[S::NQ], uint8_t* st) {
#pragma unroll
        for (int i = 0; i < S::NQ; ++i) {
            const int q = tid + 256 * i;
            if (q < S::HP * 4) {
                const int hp = q >> 2, c4 = q & 3;
                const int off = (c4 >> 1) * S::PLANE + hp * 16 + (c4 & 1) * 8;
                const __nv_bfloat162 h01 = __floats2bfloat162_rn(v[i].x, v[i].y);
                const __nv_bfloat162 h23 = __floats2bfloat162_rn(v[i].z, v[i].w);
                *reinterpret_cast<uint2*>(st + off) = make_uint2(bf16x2_bits(h01), bf16x2_bits(h23));
                if constexpr (LO) {
                    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
                    const __nv_bfloat162 l01 = __floats2bfloat162_rn(v[i].x - f01.x, v[i].y - f01.y);
                    const __nv_bfloat162 l23 = __floats2bfloat162_rn(v[i].z - f23.x, v[i].w - f23.y);
                    *reinterpret_cast<uint2*>(st + S::A_HALF + off) =
                        make_uint2(bf16x2_bits(l01), bf16x2_bits(l23));
                }
            }
        }
    };
    // weights of chunk c: row co, plane p = input channels 16 c + 8 p .. + 7, all nine taps
    auto load_b = [&](int c, uint8_t* dst) {
        const uint32_t bs = smem_addr(dst);
        const int ci0 = c * 16;
        for (int q = tid; q < 9 * BN * 2; q += 256) {
            const int plane = q & 1, r = q >> 1;         // r = co * 9 + tap
            const int co = r / 9, tap = r - co * 9;
            cp_async16(bs + tap * S::B_TAP + plane * S::B_PLANE + co * 16,
                       a.w + ((long long)(co0 + co) * 9 + tap) * Cin + ci0 + plane * 8);
        }
    };
    // accumulator of block t -> bias, ReLU, FP32 stores; false if the wait ran out
    auto epilogue = [&](int t) -> bool {
        if (!mbar_wait(smem_addr(&accbar[t & 1]), (uint32_t)((t >> 1) & 1))) return false;
        tc_fence_after();
        int n, ty0, tx0;
        tile_of(t, n, ty0, tx0);
        const int q = warp & 3, hw = warp >> 2;
        const int j = MT == 2 ? hw : 0;                     // 128-pixel tile of this warp
        constexpr int NCW = MT == 2 ? BN : BN / 2;          // accumulator columns per warp
        const int cb = MT == 2 ? 0 : hw * NCW;
        const int m = q * 32 + lane;                        // pixel of the tile = TMEM lane
        const int oy = ty0 + (m >> 3), ox = tx0 + 8 * j + (m & 7);
        const long long p = ((long long)n * a.H + oy) * a.W + ox;
        const uint32_t col0 = (uint32_t)((t & 1) * S::ACC + j * BN + cb);
#pragma unroll 1
        for (int cc = 0; cc < NCW; cc += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + col0 + (uint32_t)cc, v);
            const int co = co0 + cb + cc;                   // 16 channels, all in y1 or all in y2
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
        tc_fence_before();
        return true;
    };

    if (G > 0) {
        if (resident)
            for (int c = 0; c < nchunk; ++c) load_b(c, wts + c * S::B_BYTES);
        else
            load_b(0, wts);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    float4 v[S::NQ];
    if (G > 0) load_a(0, v);
    int bad = 0, issued = -1;     // a wait ran out; last chunk whose MMAs were issued
    for (int g = 0; g < G; ++g) {
        const int t = g / nchunk, c = g - t * nchunk, s = g % stages;
        uint8_t* st = ring + s * S::A_BYTES;
        store_a(v, st);
        if (g + 1 < G) {
            load_a(g + 1, v);
            // buffer (g + 1) % stages was last read by the MMAs of chunk g + 1 - stages
            const int g1 = g + 1, s1 = g1 % stages;
            if (g1 >= stages && !mbar_wait(smem_addr(&mbar[s1]), (uint32_t)((g1 / stages - 1) & 1))) bad = 1;
            if (!resident && !bad) load_b(g1 % nchunk, wts + s1 * S::B_BYTES);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");            // the weights of chunk g have landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> tensor core
        bad = __syncthreads_or(bad);
        if (bad) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t ab = smem_addr(st);
            const uint32_t bb = smem_addr(wts + (resident ? c : s) * S::B_BYTES);
            const uint32_t acc = tmem + (uint32_t)((t & 1) * S::ACC);
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap - dy * 3;
                const uint64_t bd = smem_desc(bb + tap * S::B_TAP, S::B_PLANE, 128);
#pragma unroll
                for (int j = 0; j < MT; ++j) {
                    const uint32_t aoff = (uint32_t)((dy * S::HWD + 8 * j + dx) * 16);
                    const uint32_t d = acc + (uint32_t)(j * BN);
                    mma_bf16_ss(d, smem_desc(ab + aoff, S::PLANE, S::HWD * 16), bd, S::IDESC, (c | tap) != 0);
                    if constexpr (LO)
                        mma_bf16_ss(d, smem_desc(ab + S::A_HALF + aoff, S::PLANE, S::HWD * 16), bd, S::IDESC, 1u);
                }
            }
            mma_commit(smem_addr(&mbar[s]));
            if (c == nchunk - 1) mma_commit(smem_addr(&accbar[t & 1]));
        }
        issued = g;
        if (c == 0 && t > 0 && !epilogue(t - 1)) bad = 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    bad = __syncthreads_or(bad);
    if (!bad && my_tiles > 0 && !epilogue(my_tiles - 1)) bad = 1;
    bad = __syncthreads_or(bad);
    if (bad) {
        // stop: wait (bounded) for the MMAs in flight before the tensor memory is freed
        if (issued >= 0) mbar_wait(smem_addr(&mbar[issued % stages]), (uint32_t)((issued / stages) & 1));
        if (tid == 0) atomicExch(&g_tc_timeout, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)S::COLS)
                     : "memory");
    }
}

constexpr int kMaxDevices = 64;
constexpr int kResidentLimit = 112 * 1024;      // resident weights while two CTAs still fit on an SM

struct VariantInfo {
    int ready;          // attributes set and read
    int regs_per_cta;   // registers allocated to one CTA (per-warp granularity of 256)
    int static_smem;
};
VariantInfo g_var[kMaxDevices][12];
int g_sms[kMaxDevices], g_smem_sm[kMaxDevices], g_smem_reserved[kMaxDevices];

// CTAs of 256 threads that fit on one SM with `smem` bytes of dynamic shared memory:
// the limits of threads, registers and shared memory (with the shared-memory carveout
// at its maximum, which the variant requests)
int ctas_per_sm(const VariantInfo& v, int dev, long long smem)
{
    int k = 2048 / 256;
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
        v.regs_per_cta = 8 * ((fa.numRegs * 32 + 255) / 256 * 256);
        v.static_smem = (int)fa.sharedSizeBytes;
        v.ready = 1;
    }
    const int nchunk = (a.C1 + a.C2) / 16;
    if (stages <= 0) stages = 2;
    if (stages > kMaxStages) return false;
    const long long res_smem = (long long)stages * S::A_BYTES + (long long)nchunk * S::B_BYTES;
    const int resident = res_smem <= kResidentLimit ? 1 : 0;
    const long long smem = resident ? res_smem : (long long)stages * (S::A_BYTES + S::B_BYTES);
    if (smem > kSmemLimit) return false;
    const int per_sm = ctas_per_sm(v, dev, smem);
    // the CTAs resident on one SM must fit in its tensor memory together, so that no
    // allocation ever waits for another CTA
    if (per_sm < 1 || per_sm * S::COLS > kTmemColumns) return false;
    const long long ntiles = (long long)a.B * (a.H / S::TH) * (a.W / S::TW);
    const int cob = a.Cout / BN;
    long long gx = ((long long)per_sm * g_sms[dev] + cob - 1) / cob;
    if (gx > ntiles) gx = ntiles;
    if (gx < 1) gx = 1;
    conv3_tc_kernel<BN, MT, LO><<<dim3((unsigned)gx, (unsigned)cob), 256, (size_t)smem, s>>>(a, stages, resident);
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
    // two tiles per CTA when that still gives two CTAs per SM on 152 SMs
    const long long ctas2 = a.W >= 16 ? (long long)a.B * (a.H / 16) * (a.W / 16) * (a.Cout / bn) : 0;
    const int mt = ctas2 >= 2 * 152 ? 2 : 1;
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
