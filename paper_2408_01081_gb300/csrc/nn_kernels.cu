// Kernels of the convolutional surrogate (U-Net neural operator) and their C ABI.
//
// Activations are FP32, channels-last [B][H][W][C]; H and W are powers of two
// and every convolution pads circularly (the lattices are periodic).  Weights
// are BF16, [Cout][KS][KS][Cin], with FP32 master copies for the optimiser.
//
// 3x3 forward convolutions go to the tcgen05 kernel of nn_conv_tc.cu where its tiling
// applies; the kernels here are implicit GEMMs with mma.sync m16n8k16 (BF16 inputs,
// FP32 accumulation) for the forward sizes that tiling does not take (the data
// gradient is a forward convolution too) and for the weight gradients.  An FP32
// activation a is split into
// a_hi = bf16(a) and a_lo = bf16(a - a_hi); products use both halves, so the
// only rounding of the forward pass is the BF16 weights themselves:
//   forward / data gradient: W x (a_hi + a_lo)           (2 MMAs per tile)
//   weight gradient:        dY_hi X_hi + dY_hi X_lo + dY_lo X_hi (3 MMAs)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "lbm_nn.h"
#include "nn_conv_tc.h"

namespace {

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// v -> hi = bf16(v), lo = bf16(v - hi), four values packed in pairs (cvt.rn.bf16x2)
__device__ __forceinline__ void split_bf16x4(const float4 v, uint2& hi, uint2& lo)
{
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
    hi = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
    lo = make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ---------------------------------------------------------------------------
// convolution forward (also the data gradient, with flipped/transposed weights)
// ---------------------------------------------------------------------------
struct ConvArgs {
    const float* x1;            // first input, C1 channels
    const float* x2;            // second input (concatenated after x1), C2 channels, or null
    int C1, C2;
    const __nv_bfloat16* w;     // [Cout][KS][KS][C1+C2]
    const float* bias;          // [Cout] or null
    float* y1;                  // output channels [0, Co1)
    float* y2;                  // output channels [Co1, Cout), or null
    int Co1, Cout;
    int B, H, W;                // H, W powers of two
    int relu;                   // apply max(0, .) to the output
    int beta;                   // 1: add into the output instead of overwriting
    int x1_half;                // x1 is stored at (H/2, W/2) and read nearest-upsampled
    int act_bf16;               // activations as one BF16 value (no lo half)
};

constexpr int CBM = 128;        // pixels per CTA tile
constexpr int CKC = 32;         // K chunk (channels of one tap)
constexpr int CPAD = 8;

template <int BN, int KS>
__global__ void __launch_bounds__(256) conv_fwd_kernel(ConvArgs a)
{
    __shared__ __align__(16) __nv_bfloat16 As_hi[CBM][CKC + CPAD];
    __shared__ __align__(16) __nv_bfloat16 As_lo[CBM][CKC + CPAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][CKC + CPAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int wm = warp & 3;                 // 4 warps along M (32 pixels each)
    const int wn = warp >> 2;                // 2 warps along N
    constexpr int WN = BN / 2;               // columns per warp
    constexpr int NT = WN / 8;               // n-tiles per warp
    const int P = a.B * a.H * a.W;
    const int p0 = blockIdx.x * CBM;
    const int co0 = blockIdx.y * BN;
    const int Cin = a.C1 + a.C2;
    const int HW = a.H * a.W;
    const int R = KS / 2;

    float acc[2][NT][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    // this thread stages half a row of A: pixel p0 + tid/2, channels (tid&1)*16 .. +16
    const int ap = p0 + (tid >> 1);
    const int ahalf = (tid & 1) * 16;
    const bool avalid = ap < P;
    int an = 0, ay = 0, ax = 0;
    if (avalid) {
        an = ap / HW;
        ay = (ap / a.W) & (a.H - 1);
        ax = ap & (a.W - 1);
    }

    for (int tap = 0; tap < KS * KS; ++tap) {
        const int dy = tap / KS - R, dx = tap % KS - R;
        const int sy = (ay + dy) & (a.H - 1), sx = (ax + dx) & (a.W - 1);
        const long long spix = ((long long)an * a.H + sy) * a.W + sx;
        const long long spix1 = a.x1_half ? ((long long)an * (a.H >> 1) + (sy >> 1)) * (a.W >> 1) + (sx >> 1) : spix;
        for (int ci0 = 0; ci0 < Cin; ci0 += CKC) {
            // --- stage A (FP32 -> bf16 hi / lo) ---
            {
                float v[16];
                if (avalid) {
                    const float* src;
                    if (ci0 < a.C1) src = a.x1 + spix1 * a.C1 + ci0 + ahalf;
                    else src = a.x2 + spix * a.C2 + (ci0 - a.C1) + ahalf;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 f = *reinterpret_cast<const float4*>(src + 4 * q);
                        v[4 * q] = f.x;
                        v[4 * q + 1] = f.y;
                        v[4 * q + 2] = f.z;
                        v[4 * q + 3] = f.w;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = 0.f;
                }
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * q]);
                    const __nv_bfloat16 h1 = __float2bfloat16_rn(v[2 * q + 1]);
                    const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * q] - __bfloat162float(h0));
                    const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * q + 1] - __bfloat162float(h1));
                    hi[q] = pack_bf16(h0, h1);
                    lo[q] = pack_bf16(l0, l1);
                }
                uint4* dh = reinterpret_cast<uint4*>(&As_hi[tid >> 1][ahalf]);
                uint4* dl = reinterpret_cast<uint4*>(&As_lo[tid >> 1][ahalf]);
                dh[0] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                dh[1] = make_uint4(hi[4], hi[5], hi[6], hi[7]);
                dl[0] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                dl[1] = make_uint4(lo[4], lo[5], lo[6], lo[7]);
            }
            // --- stage B: BN output channels x 32 inputs of this tap (64 bytes per row) ---
            for (int q = tid; q < BN * 4; q += 256) {
                const int n = q >> 2, part = q & 3;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (co0 + n < a.Cout)
                    val = *reinterpret_cast<const uint4*>(a.w + ((long long)(co0 + n) * KS * KS + tap) * Cin + ci0 +
                                                          part * 8);
                *reinterpret_cast<uint4*>(&Bs[n][part * 8]) = val;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < CKC; kk += 16) {
                uint32_t fh[2][4], fl[2][4];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int r = wm * 32 + i * 16 + g;
                    fh[i][0] = *reinterpret_cast<const uint32_t*>(&As_hi[r][kk + 2 * t4]);
                    fh[i][1] = *reinterpret_cast<const uint32_t*>(&As_hi[r + 8][kk + 2 * t4]);
                    fh[i][2] = *reinterpret_cast<const uint32_t*>(&As_hi[r][kk + 8 + 2 * t4]);
                    fh[i][3] = *reinterpret_cast<const uint32_t*>(&As_hi[r + 8][kk + 8 + 2 * t4]);
                    fl[i][0] = *reinterpret_cast<const uint32_t*>(&As_lo[r][kk + 2 * t4]);
                    fl[i][1] = *reinterpret_cast<const uint32_t*>(&As_lo[r + 8][kk + 2 * t4]);
                    fl[i][2] = *reinterpret_cast<const uint32_t*>(&As_lo[r][kk + 8 + 2 * t4]);
                    fl[i][3] = *reinterpret_cast<const uint32_t*>(&As_lo[r + 8][kk + 8 + 2 * t4]);
                }
#pragma unroll
                for (int j = 0; j < NT; ++j) {
                    const int n = wn * WN + j * 8 + g;
                    uint32_t fb[2];
                    fb[0] = *reinterpret_cast<const uint32_t*>(&Bs[n][kk + 2 * t4]);
                    fb[1] = *reinterpret_cast<const uint32_t*>(&Bs[n][kk + 8 + 2 * t4]);
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        mma_bf16(acc[i][j], fh[i], fb);
                        if (!a.act_bf16) mma_bf16(acc[i][j], fl[i], fb);
                    }
                }
            }
            __syncthreads();
        }
    }
    // --- epilogue: bias, activation, store (optionally accumulate) ---
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int p = p0 + wm * 32 + i * 16 + g + 8 * h;
            if (p >= P) continue;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int co = co0 + wn * WN + j * 8 + 2 * t4;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int c = co + e;
                    if (c >= a.Cout) continue;
                    float v = acc[i][j][2 * h + e];
                    if (a.bias) v += a.bias[c];
                    if (a.relu) v = fmaxf(v, 0.f);
                    float* dst = (c < a.Co1) ? a.y1 + (long long)p * a.Co1 + c
                                             : a.y2 + (long long)p * (a.Cout - a.Co1) + (c - a.Co1);
                    *dst = a.beta ? *dst + v : v;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 3x3 convolution on an 8 x 16 pixel tile (H >= 8, W >= 16): the input tile with
// its one-pixel halo (10 x 18 pixels) is staged once per 32-channel chunk as
// BF16 hi / lo, the weights of all nine taps once per chunk, and every tap reads
// its A fragments from the halo tile at the tap's offset (ldmatrix).  Same
// arithmetic as conv_fwd_kernel; warps: 4 along the tile rows (2 rows = 2 m16
// tiles each) x 2 along the output channels.
// ---------------------------------------------------------------------------
constexpr int TW = 16;                          // output tile width (pixels); height TH is 8 or 16
constexpr int HW2 = TW + 2;                     // halo tile width
constexpr int KROW = CKC + CPAD;                // smem row: 40 bf16 = 80 bytes

// 16-byte global -> shared copy that bypasses the registers (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(__nv_bfloat16* smem_dst, const __nv_bfloat16* gmem_src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const __nv_bfloat16* p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a)
                 : "memory");
}

template <int BN, int TH>
constexpr int conv3_tile_smem_bytes()
{
    return (2 * (TH + 2) * HW2 + 9 * BN) * KROW * (int)sizeof(__nv_bfloat16);
}

// TH = 8: warps 4 (row pairs) x 2 (channel halves); TH = 16: 8 row pairs x all BN channels
template <int BN, bool LO, int TH>
__global__ void __launch_bounds__(256) conv3_tile_kernel(ConvArgs a)
{
    constexpr int HH = TH + 2;               // halo tile height
    constexpr int WR = TH / 2;               // warps along the tile rows (2 rows each)
    constexpr int WC = 8 / WR;               // warps along the output channels
    extern __shared__ __align__(16) __nv_bfloat16 smem[];
    __nv_bfloat16* Ah = smem;                            // [HH*HW2][KROW]
    __nv_bfloat16* Al = Ah + HH * HW2 * KROW;            // [HH*HW2][KROW]
    __nv_bfloat16* Bs = Al + HH * HW2 * KROW;            // [9][BN][KROW]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int wm = warp % WR;                // tile rows 2 wm, 2 wm + 1
    const int wn = warp / WR;                // output-channel group
    constexpr int WN = BN / WC;
    constexpr int NT = WN / 8;               // n8 tiles per warp (even)
    const int tiles_x = a.W / TW, tiles_y = a.H / TH;
    const int tile = blockIdx.x;
    const int n = tile / (tiles_x * tiles_y);
    const int ty0 = ((tile / tiles_x) % tiles_y) * TH, tx0 = (tile % tiles_x) * TW;
    const int co0 = blockIdx.y * BN;
    const int Cin = a.C1 + a.C2;

    float acc[2][NT][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    for (int ci0 = 0; ci0 < Cin; ci0 += CKC) {
        // --- stage the weights of the nine taps: BN x 32 inputs each (asynchronous copies,
        //     issued first so that they overlap the halo staging; the launcher guarantees
        //     co0 + BN <= Cout) ---
        for (int q = tid; q < 9 * BN * 4; q += 256) {
            const int tap = q / (BN * 4), r = q % (BN * 4);
            const int nn = r >> 2, part = r & 3;
            cp_async16(Bs + (tap * BN + nn) * KROW + part * 8,
                       a.w + ((long long)(co0 + nn) * 9 + tap) * Cin + ci0 + part * 8);
        }
        // --- stage the halo tile: (TH + 2) x 18 pixels x 32 channels, FP32 -> BF16 hi / lo ---
        const bool from1 = ci0 < a.C1;
        const float* base = from1 ? a.x1 : a.x2;
        const int cstride = from1 ? a.C1 : a.C2;
        const int coff = from1 ? ci0 : ci0 - a.C1;
        const int half = (from1 && a.x1_half) ? 1 : 0;     // nearest upsampling of a half-size x1
#pragma unroll 4
        for (int q = tid; q < HH * HW2 * (CKC / 4); q += 256) {
            const int hp = q >> 3, c4 = (q & 7) * 4;
            const int hy = hp / HW2, hx = hp % HW2;
            const int sy = (ty0 + hy - 1) & (a.H - 1), sx = (tx0 + hx - 1) & (a.W - 1);
            const long long spix = ((long long)n * (a.H >> half) + (sy >> half)) * (a.W >> half) + (sx >> half);
            const float4 v = *reinterpret_cast<const float4*>(base + spix * cstride + coff + c4);
            if constexpr (LO) {
                uint2 hi, lo;
                split_bf16x4(v, hi, lo);
                *reinterpret_cast<uint2*>(Ah + hp * KROW + c4) = hi;
                *reinterpret_cast<uint2*>(Al + hp * KROW + c4) = lo;
            } else {
                const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
                *reinterpret_cast<uint2*>(Ah + hp * KROW + c4) =
                    make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
            }
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3;     // halo offsets (0..2)
#pragma unroll
            for (int kk = 0; kk < CKC; kk += 16) {
                uint32_t fh[2][4], fl[2][4];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int hp = (2 * wm + i + dy) * HW2 + (lane & 15) + dx;
                    const int kc = kk + (lane >> 4) * 8;
                    ldsm_x4(fh[i], Ah + hp * KROW + kc);
                    if constexpr (LO) ldsm_x4(fl[i], Al + hp * KROW + kc);
                }
#pragma unroll
                for (int j = 0; j < NT; j += 2) {
                    uint32_t fb[4];
                    const int nn = wn * WN + j * 8 + (lane & 7) + ((lane >> 4) << 3);
                    ldsm_x4(fb, Bs + (tap * BN + nn) * KROW + kk + ((lane >> 3) & 1) * 8);
                    const uint32_t b0[2] = {fb[0], fb[1]}, b1[2] = {fb[2], fb[3]};
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        mma_bf16(acc[i][j], fh[i], b0);
                        mma_bf16(acc[i][j + 1], fh[i], b1);
                        if constexpr (LO) {
                            mma_bf16(acc[i][j], fl[i], b0);
                            mma_bf16(acc[i][j + 1], fl[i], b1);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    // --- epilogue: bias, activation, store (optionally accumulate) ---
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int oy = ty0 + 2 * wm + i, ox = tx0 + g + 8 * h;
            const long long p = ((long long)n * a.H + oy) * a.W + ox;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int co = co0 + wn * WN + j * 8 + 2 * t4;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int c = co + e;
                    if (c >= a.Cout) continue;
                    float v = acc[i][j][2 * h + e];
                    if (a.bias) v += a.bias[c];
                    if (a.relu) v = fmaxf(v, 0.f);
                    float* dst = (c < a.Co1) ? a.y1 + p * a.Co1 + c : a.y2 + p * (a.Cout - a.Co1) + (c - a.Co1);
                    *dst = a.beta ? *dst + v : v;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// weight gradient: dW[co][tap][ci] = sum_p dY[p][co] X[p + tap][ci]
// CTA tile 64 (co) x 64 (ci of one tap), K = pixels in chunks of 64, split over
// pixel ranges (gridDim.z); partial[split][co][tap][ci] reduced in fixed order.
// ---------------------------------------------------------------------------
struct WgradArgs {
    const float* dy;          // [P][Cout]
    const float* x1;          // [P][C1]
    const float* x2;          // [P][C2] or null
    int C1, C2, Cout;
    int B, H, W, KS;
    int pix_per_split;
    float* partial;           // [splits][Cout][KS*KS][Cin]
    int lw, lhw;              // log2(W), log2(H W)
    int x1_half;              // x1 stored at (H/2, W/2), read nearest-upsampled
};

constexpr int WK = 64;                 // pixels per staged chunk
constexpr int WROW = 64 + 8;           // smem row of 64 channels (+8 pad): 144 bytes

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const __nv_bfloat16* p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a)
                 : "memory");
}

// staging of one 64-pixel chunk: dY[p][co0 .. co0+63] and X[p + tap][ci0 .. ci0+63] as
// BF16 hi / lo in their natural [pixel][channel] layout (16-byte vector loads); the
// MMA fragments are read transposed with ldmatrix.trans
__global__ void __launch_bounds__(256) conv_wgrad_kernel(WgradArgs a)
{
    __shared__ __align__(16) __nv_bfloat16 Yh[WK][WROW];
    __shared__ __align__(16) __nv_bfloat16 Yl[WK][WROW];
    __shared__ __align__(16) __nv_bfloat16 Xh[WK][WROW];
    __shared__ __align__(16) __nv_bfloat16 Xl[WK][WROW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int wm = warp & 1;                 // 2 warps along M (32 co each)
    const int wn = warp >> 1;                // 4 warps along N (16 ci each)
    const int Cin = a.C1 + a.C2;
    const int co0 = blockIdx.x * 64;
    const int ntap = a.KS * a.KS;
    const int nci = (Cin + 63) / 64;
    const int tap = blockIdx.y / nci;
    const int ci0 = (blockIdx.y % nci) * 64;
    const int R = a.KS / 2;
    const int dy = tap / a.KS - R, dx = tap % a.KS - R;
    const int P = a.B * a.H * a.W;
    const int pbeg = blockIdx.z * a.pix_per_split;
    const int pend = min(P, pbeg + a.pix_per_split);

    float acc[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    // 64 pixels x 16 float4 per tensor per chunk: 4 of each per thread, loaded one
    // chunk ahead into registers while the tensor cores work on the current one
    float4 ry[4], rx[4];
    auto load_chunk = [&](int pc) {
#pragma unroll
        for (int rep = 0; rep < 4; ++rep) {
            const int q = tid + rep * 256;
            const int pk = q >> 4, c4 = (q & 15) * 4;
            const int p = pc + pk;
            ry[rep] = make_float4(0.f, 0.f, 0.f, 0.f);
            rx[rep] = ry[rep];
            if (p < pend) {
                if (co0 + c4 < a.Cout)
                    ry[rep] = *reinterpret_cast<const float4*>(a.dy + (long long)p * a.Cout + co0 + c4);
                const int ci = ci0 + c4;
                if (ci < Cin) {
                    const int n = p >> a.lhw, y = (p >> a.lw) & (a.H - 1), x = p & (a.W - 1);
                    const long long sp =
                        (((long long)n << a.lhw) | ((long long)((y + dy) & (a.H - 1)) << a.lw)) | ((x + dx) & (a.W - 1));
                    if (ci < a.C1) {
                        const long long s1 = a.x1_half ? (((long long)n << (a.lhw - 2)) |
                                                          ((long long)(((y + dy) & (a.H - 1)) >> 1) << (a.lw - 1)) |
                                                          (((x + dx) & (a.W - 1)) >> 1))
                                                       : sp;
                        rx[rep] = *reinterpret_cast<const float4*>(a.x1 + s1 * a.C1 + ci);
                    } else {
                        rx[rep] = *reinterpret_cast<const float4*>(a.x2 + sp * a.C2 + (ci - a.C1));
                    }
                }
            }
        }
    };
    if (pbeg < pend) load_chunk(pbeg);
    for (int pc = pbeg; pc < pend; pc += WK) {
#pragma unroll
        for (int rep = 0; rep < 4; ++rep) {
            const int q = tid + rep * 256;
            const int pk = q >> 4, c4 = (q & 15) * 4;
            uint2 yh, yl, xh, xl;
            split_bf16x4(ry[rep], yh, yl);
            split_bf16x4(rx[rep], xh, xl);
            *reinterpret_cast<uint2*>(&Yh[pk][c4]) = yh;
            *reinterpret_cast<uint2*>(&Yl[pk][c4]) = yl;
            *reinterpret_cast<uint2*>(&Xh[pk][c4]) = xh;
            *reinterpret_cast<uint2*>(&Xl[pk][c4]) = xl;
        }
        if (pc + WK < pend) load_chunk(pc + WK);
        __syncthreads();
        const int mi = lane >> 3, r8 = lane & 7;
#pragma unroll
        for (int kk = 0; kk < WK; kk += 16) {
            // A = dY^T (co x pixel): matrices (m, k), (m+8, k), (m, k+8), (m+8, k+8)
            uint32_t fah[2][4], fal[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int m0 = wm * 32 + i * 16 + (mi & 1) * 8;
                const int k0 = kk + (mi >> 1) * 8 + r8;
                ldsm_x4_trans(fah[i], &Yh[k0][m0]);
                ldsm_x4_trans(fal[i], &Yl[k0][m0]);
            }
            // B = X (pixel x ci): matrices (k, n), (k+8, n), (k, n+8), (k+8, n+8)
            uint32_t fbh[4], fbl[4];
            {
                const int n0 = wn * 16 + (mi >> 1) * 8;
                const int k0 = kk + (mi & 1) * 8 + r8;
                ldsm_x4_trans(fbh, &Xh[k0][n0]);
                ldsm_x4_trans(fbl, &Xl[k0][n0]);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const uint32_t bh[2] = {fbh[2 * j], fbh[2 * j + 1]}, bl[2] = {fbl[2 * j], fbl[2 * j + 1]};
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    mma_bf16(acc[i][j], fah[i], bh);
                    mma_bf16(acc[i][j], fah[i], bl);
                    mma_bf16(acc[i][j], fal[i], bh);
                }
            }
        }
        __syncthreads();
    }
    float* out = a.partial + (long long)blockIdx.z * a.Cout * ntap * Cin;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int co = co0 + wm * 32 + i * 16 + g + 8 * h;
            if (co >= a.Cout) continue;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int ci = ci0 + wn * 16 + j * 8 + 2 * t4 + e;
                    if (ci < Cin) out[((long long)co * ntap + tap) * Cin + ci] = acc[i][j][2 * h + e];
                }
        }
}

// ---------------------------------------------------------------------------
// 3x3 weight gradient on 16 x 16 pixel blocks (H, W >= 16; Cin, Cout multiples of 32).
// A CTA takes 32 output x 32 input channels and all nine taps.  Per block it stages dY
// (256 pixels) and X with its one-pixel halo (18 x 18 pixels) once, as BF16 hi / lo in
// [pixel][channel] rows, and warp w accumulates tap w: its B fragments are read
// (ldmatrix.trans, one row address per lane) from the halo block at the tap's offset,
// so nothing is staged per tap.  Products as in conv_wgrad_kernel (dY_hi X_hi +
// dY_hi X_lo + dY_lo X_hi); split over ranges of blocks (gridDim.z),
// partial[split][co][tap][ci] reduced in fixed order by sum_splits_kernel.
// ---------------------------------------------------------------------------
struct Wgrad3Args {
    const float* dy;          // [B][H][W][Cout]
    const float* x1;          // [B][H][W][C1] (or [B][H/2][W/2][C1] with x1_half)
    const float* x2;          // [B][H][W][C2] or null
    int C1, C2, Cout;
    int B, H, W;
    int blocks_per_split;
    float* partial;           // [splits][Cout][9][Cin]
    int x1_half;
};

constexpr int G3ROW = 40;                 // smem row: 32 channels + 8 pad (80 bytes, conflict-free ldmatrix)
constexpr int G3Y = 256, G3X = 18 * 18;   // pixels of the dY block and of the X halo block
constexpr int G3THREADS = 9 * 32;         // one warp per tap
constexpr int conv_wgrad3_smem_bytes() { return 2 * (G3Y + G3X) * G3ROW * (int)sizeof(__nv_bfloat16); }

__global__ void __launch_bounds__(G3THREADS, 2) conv_wgrad3_tile_kernel(Wgrad3Args a)
{
    extern __shared__ __align__(16) __nv_bfloat16 sm3[];
    __nv_bfloat16* Yh = sm3;                      // [256][G3ROW]
    __nv_bfloat16* Yl = Yh + G3Y * G3ROW;
    __nv_bfloat16* Xh = Yl + G3Y * G3ROW;         // [324][G3ROW]
    __nv_bfloat16* Xl = Xh + G3X * G3ROW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;   // warp = tap
    const int g = lane >> 2, t4 = lane & 3, mi = lane >> 3, r8 = lane & 7;
    const int dy = warp / 3, dx = warp - 3 * (warp / 3);              // halo offsets 0..2
    const int Cin = a.C1 + a.C2;
    const int co0 = blockIdx.x * 32, ci0 = blockIdx.y * 32;
    const int bx = a.W / 16, by = a.H / 16;
    const int nblocks = a.B * by * bx;
    const int b0 = blockIdx.z * a.blocks_per_split;
    const int b1 = min(nblocks, b0 + a.blocks_per_split);
    // input channels ci0 .. ci0 + 31 lie in x1 or in x2 (C1 is a multiple of 32)
    const bool from1 = ci0 < a.C1;
    const float* xs = from1 ? a.x1 : a.x2;
    const int xstride = from1 ? a.C1 : a.C2;
    const int xoff = from1 ? ci0 : ci0 - a.C1;
    const int half = (from1 && a.x1_half) ? 1 : 0;      // nearest upsampling of a half-size x1
    const int hs = a.H >> half, ws = a.W >> half;

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    for (int b = b0; b < b1; ++b) {
        const int n = b / (by * bx), ty0 = ((b / bx) % by) * 16, tx0 = (b % bx) * 16;
#pragma unroll 4
        for (int q = tid; q < G3Y * 8; q += G3THREADS) {            // dY: 256 pixels x 8 float4
            const int pk = q >> 3, c4 = (q & 7) * 4;
            const long long p = ((long long)n * a.H + ty0 + (pk >> 4)) * a.W + tx0 + (pk & 15);
            uint2 h, l;
            split_bf16x4(__ldg(reinterpret_cast<const float4*>(a.dy + p * a.Cout + co0 + c4)), h, l);
            *reinterpret_cast<uint2*>(Yh + pk * G3ROW + c4) = h;
            *reinterpret_cast<uint2*>(Yl + pk * G3ROW + c4) = l;
        }
#pragma unroll 4
        for (int q = tid; q < G3X * 8; q += G3THREADS) {            // X: 18 x 18 halo pixels, periodic
            const int hp = q >> 3, c4 = (q & 7) * 4;
            const int hy = hp / 18, hx = hp - hy * 18;
            const int sy = (ty0 + hy - 1) & (a.H - 1), sx = (tx0 + hx - 1) & (a.W - 1);
            const long long sp = ((long long)n * hs + (sy >> half)) * ws + (sx >> half);
            uint2 h, l;
            split_bf16x4(__ldg(reinterpret_cast<const float4*>(xs + sp * xstride + xoff + c4)), h, l);
            *reinterpret_cast<uint2*>(Xh + hp * G3ROW + c4) = h;
            *reinterpret_cast<uint2*>(Xl + hp * G3ROW + c4) = l;
        }
        __syncthreads();
#pragma unroll 2
        for (int r = 0; r < 16; ++r) {            // K step: row r of the block (16 pixels)
            // A = dY^T (co x pixel): matrices (m, k), (m+8, k), (m, k+8), (m+8, k+8)
            uint32_t fah[2][4], fal[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int m0 = i * 16 + (mi & 1) * 8;
                const int k0 = r * 16 + (mi >> 1) * 8 + r8;
                ldsm_x4_trans(fah[i], Yh + k0 * G3ROW + m0);
                ldsm_x4_trans(fal[i], Yl + k0 * G3ROW + m0);
            }
            // B = X (pixel x ci): pixel (r, c) of the block is halo pixel (r + dy, c + dx)
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                uint32_t fbh[4], fbl[4];
                const int n0 = jj * 16 + (mi >> 1) * 8;
                const int hp = (r + dy) * 18 + (mi & 1) * 8 + r8 + dx;
                ldsm_x4_trans(fbh, Xh + hp * G3ROW + n0);
                ldsm_x4_trans(fbl, Xl + hp * G3ROW + n0);
#pragma unroll
                for (int j2 = 0; j2 < 2; ++j2) {
                    const uint32_t bh[2] = {fbh[2 * j2], fbh[2 * j2 + 1]}, bl[2] = {fbl[2 * j2], fbl[2 * j2 + 1]};
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        mma_bf16(acc[i][jj * 2 + j2], fah[i], bh);
                        mma_bf16(acc[i][jj * 2 + j2], fah[i], bl);
                        mma_bf16(acc[i][jj * 2 + j2], fal[i], bh);
                    }
                }
            }
        }
        __syncthreads();
    }
    float* out = a.partial + (long long)blockIdx.z * a.Cout * 9 * Cin;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int co = co0 + i * 16 + g + 8 * h;
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    out[((long long)co * 9 + warp) * Cin + ci0 + j * 8 + 2 * t4 + e] = acc[i][j][2 * h + e];
        }
}

// sum the split partials in order into dW (FP32)
__global__ void sum_splits_kernel(const float* __restrict__ partial, int splits, long long n, float* __restrict__ out,
                                  int beta)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < splits; ++k) s += partial[(long long)k * n + i];
        out[i] = beta ? out[i] + s : s;
    }
}

// db[c] = sum_p dY[p][c] in two fixed-order passes.  Pass 1: block b sums the
// pixels [b ppb, (b+1) ppb); within a block thread t handles channel c0 + t % cc
// and every (256 / cc)-th pixel (a warp reads consecutive channels of one pixel)
// into four interleaved partial sums, then the per-thread sums are added in
// thread order.  Pass 2: one block per channel adds the blocks' partials in a
// fixed strided order and a fixed tree.
__global__ void bias_grad_partial_kernel(const float* __restrict__ dy, long long P, int C, long long ppb,
                                         float* __restrict__ partial)
{
    __shared__ float red[256];
    const int t = threadIdx.x;
    const long long p0 = blockIdx.x * ppb, p1 = min(P, p0 + ppb);
    for (int c0 = 0; c0 < C; c0 += 256) {
        const int cc = min(256, C - c0);
        const int rows = 256 / cc;
        const int c = t % cc, r = t / cc;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        if (r < rows) {
            long long p = p0 + r;
            for (; p + 3 * rows < p1; p += 4 * rows) {
                s0 += dy[p * C + c0 + c];
                s1 += dy[(p + rows) * C + c0 + c];
                s2 += dy[(p + 2 * rows) * C + c0 + c];
                s3 += dy[(p + 3 * rows) * C + c0 + c];
            }
            for (; p < p1; p += rows) s0 += dy[p * C + c0 + c];
        }
        red[t] = (s0 + s1) + (s2 + s3);
        __syncthreads();
        if (t < cc) {
            float acc = 0.f;
            for (int q = 0; q < rows; ++q) acc += red[q * cc + t];
            partial[(long long)blockIdx.x * C + c0 + t] = acc;
        }
        __syncthreads();
    }
}

__global__ void bias_grad_finish_kernel(const float* __restrict__ partial, int nblk, int C, float* __restrict__ db)
{
    __shared__ float red[256];
    const int c = blockIdx.x, t = threadIdx.x;
    float acc = 0.f;
    for (int b = t; b < nblk; b += 256) acc += partial[(long long)b * C + c];
    red[t] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    if (t == 0) db[c] = red[0];
}

// pixels per block: about 32 per thread
long long bias_grad_ppb(long long P, int C)
{
    const int cc = C < 256 ? C : 256;
    long long ppb = 32LL * (256 / cc);
    const long long nb = (P + ppb - 1) / ppb;
    if (nb > 8192) ppb = (P + 8191) / 8192;
    return ppb;
}

int bias_grad_blocks(long long P, int C)
{
    const long long ppb = bias_grad_ppb(P, C);
    return (int)((P + ppb - 1) / ppb);
}

// Wt[ci][tap'][co] = W[co][KS*KS-1-tap'][ci]: weights of the data-gradient convolution
__global__ void weight_flip_kernel(const __nv_bfloat16* __restrict__ w, int Cout, int Cin, int KS,
                                   __nv_bfloat16* __restrict__ wt)
{
    const int ntap = KS * KS;
    const long long n = (long long)Cout * ntap * Cin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % Cin);
        const int tap = (int)((i / Cin) % ntap);
        const int co = (int)(i / ((long long)Cin * ntap));
        wt[((long long)ci * ntap + (ntap - 1 - tap)) * Cout + co] = w[i];
    }
}

__global__ void relu_backward_kernel(float* __restrict__ dy, const float* __restrict__ y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(y[i] > 0.f)) dy[i] = 0.f;
}

// 2x2 average pooling, [B][H][W][C] -> [B][H/2][W/2][C]
__global__ void pool_kernel(const float* __restrict__ x, int B, int H, int W, int C, float* __restrict__ y)
{
    const int Ho = H / 2, Wo = W / 2;
    const long long n = (long long)B * Ho * Wo * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long pix = i / C;
        const int xo = (int)(pix % Wo), yo = (int)((pix / Wo) % Ho), b = (int)(pix / ((long long)Wo * Ho));
        const long long base = (((long long)b * H + 2 * yo) * W + 2 * xo) * C + c;
        y[i] = 0.25f * (x[base] + x[base + C] + x[base + (long long)W * C] + x[base + (long long)W * C + C]);
    }
}

__global__ void pool_backward_kernel(const float* __restrict__ dy, int B, int H, int W, int C, float* __restrict__ dx,
                                     int beta)
{
    const long long n = (long long)B * H * W * C;
    const int Ho = H / 2, Wo = W / 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long pix = i / C;
        const int x = (int)(pix % W), y = (int)((pix / W) % H), b = (int)(pix / ((long long)W * H));
        const float v = 0.25f * dy[(((long long)b * Ho + y / 2) * Wo + x / 2) * C + c];
        dx[i] = beta ? dx[i] + v : v;
    }
}

// Fast paths of pooling and upsampling for power-of-two H, W and C / 4: one thread
// per output pixel and 4 channels (16-byte accesses), index arithmetic by shifts.
__global__ void pool4_kernel(const float4* __restrict__ x, int lho, int lwo, int lc4, long long n,
                             float4* __restrict__ y)
{
    const int C4 = 1 << lc4, Wo = 1 << lwo, Ho = 1 << lho;
    const long long rowin = 2LL * Wo * C4;           // one input row
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i & (C4 - 1));
        const long long pix = i >> lc4;
        const int xo = (int)(pix & (Wo - 1)), yo = (int)((pix >> lwo) & (Ho - 1));
        const long long b = pix >> (lwo + lho);
        const long long base = ((b * 2 * Ho + 2 * yo) * 2 * Wo + 2 * xo) * C4 + c;
        const float4 a0 = x[base], a1 = x[base + C4], a2 = x[base + rowin], a3 = x[base + rowin + C4];
        y[i] = make_float4(0.25f * (a0.x + a1.x + a2.x + a3.x), 0.25f * (a0.y + a1.y + a2.y + a3.y),
                           0.25f * (a0.z + a1.z + a2.z + a3.z), 0.25f * (a0.w + a1.w + a2.w + a3.w));
    }
}

__global__ void upsample4_kernel(const float4* __restrict__ x, int lho, int lwo, int lc4, long long n,
                                 float4* __restrict__ y)
{
    const int C4 = 1 << lc4, Wo = 1 << lwo, Ho = 1 << lho;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i & (C4 - 1));
        const long long pix = i >> lc4;
        const int xo = (int)(pix & (Wo - 1)), yo = (int)((pix >> lwo) & (Ho - 1));
        const long long b = pix >> (lwo + lho);
        y[i] = x[((b * (Ho >> 1) + (yo >> 1)) * (Wo >> 1) + (xo >> 1)) * C4 + c];
    }
}

// nearest 2x upsampling, [B][H][W][C] -> [B][2H][2W][C]
__global__ void upsample_kernel(const float* __restrict__ x, int B, int H, int W, int C, float* __restrict__ y)
{
    const int Ho = 2 * H, Wo = 2 * W;
    const long long n = (long long)B * Ho * Wo * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long pix = i / C;
        const int xo = (int)(pix % Wo), yo = (int)((pix / Wo) % Ho), b = (int)(pix / ((long long)Wo * Ho));
        y[i] = x[(((long long)b * H + yo / 2) * W + xo / 2) * C + c];
    }
}

__global__ void upsample_backward_kernel(const float* __restrict__ dy, int B, int H, int W, int C,
                                         float* __restrict__ dx, int beta)
{
    const long long n = (long long)B * H * W * C;
    const int Wo = 2 * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long pix = i / C;
        const int x = (int)(pix % W), y = (int)((pix / W) % H), b = (int)(pix / ((long long)W * H));
        const long long base = (((long long)b * 2 * H + 2 * y) * Wo + 2 * x) * C + c;
        const float v = dy[base] + dy[base + C] + dy[base + (long long)Wo * C] + dy[base + (long long)Wo * C + C];
        dx[i] = beta ? dx[i] + v : v;
    }
}

// loss = sum over pixels and the first `cvalid` channels of (out - tgt)^2; d = 2 (out - tgt) * scale
__global__ void mse_kernel(const float* __restrict__ out, const float* __restrict__ tgt, long long P, int C, int cvalid,
                           float scale, float* __restrict__ dout, double* __restrict__ partial)
{
    __shared__ double red[256];
    double s = 0.0;
    const long long n = P * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        float d = 0.f;
        if (c < cvalid) {
            d = out[i] - tgt[i];
            s += (double)d * d;
        }
        if (dout) dout[i] = 2.f * d * scale;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void sum_double_kernel(const double* __restrict__ partial, int n, double* __restrict__ out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Adam on FP32 master weights, then the BF16 working copy
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ gw, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2, __nv_bfloat16* __restrict__ wb)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float g = gw[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ x, long long n, __nv_bfloat16* __restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// network input: U fields [B][nf][H][W] (FP64, field-major per sample) scaled by 1/scale[c], plus a
// constant channel per sample, into [B][H][W][C] FP32 with zero padding channels
__global__ void pack_input_kernel(const double* __restrict__ U, long long sample_stride, int nf, const double* __restrict__ scale,
                                  const float* __restrict__ extra, int B, int H, int W, int C, float* __restrict__ x)
{
    // one thread per pixel: the nf fields (coalesced across the warp), the extra
    // channel, zeros up to C; 16-byte stores when C is a multiple of 4
    const long long HW = (long long)H * W;
    const long long npix = (long long)B * HW;
    for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < npix;
         pix += (long long)gridDim.x * blockDim.x) {
        const long long b = pix / HW, q = pix - b * HW;
        float* dst = x + pix * C;
        if ((C & 3) == 0) {
            for (int c0 = 0; c0 < C; c0 += 4) {
                float v[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = c0 + e;
                    v[e] = c < nf ? (float)(U[b * sample_stride + c * HW + q] / scale[c])
                                  : (c == nf && extra) ? extra[b] : 0.f;
                }
                *reinterpret_cast<float4*>(dst + c0) = make_float4(v[0], v[1], v[2], v[3]);
            }
        } else {
            for (int c = 0; c < C; ++c)
                dst[c] = c < nf ? (float)(U[b * sample_stride + c * HW + q] / scale[c])
                                : (c == nf && extra) ? extra[b] : 0.f;
        }
    }
}

// prediction: U_out[b][c] = U_in[b][c] + scale[c] * net[b][.][.][c] for c < nf (FP64, field-major)
__global__ void residual_output_kernel(const double* __restrict__ Uin, long long in_stride, const float* __restrict__ net,
                                       int C, const double* __restrict__ scale, int nf, int B, int H, int W,
                                       double* __restrict__ Uout, long long out_stride)
{
    const long long HW = (long long)H * W;
    const long long n = (long long)B * nf * HW;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i % HW;
        const int c = (int)((i / HW) % nf);
        const int b = (int)(i / (HW * nf));
        Uout[(long long)b * out_stride + c * HW + q] =
            Uin[(long long)b * in_stride + c * HW + q] + scale[c] * (double)net[((long long)b * HW + q) * C + c];
    }
}

// training target in network units: (U_next - U_now) / scale, [B][H][W][C] (channels >= nf zero)
__global__ void pack_target_kernel(const double* __restrict__ Unow, const double* __restrict__ Unext, long long stride,
                                   int nf, const double* __restrict__ scale, int B, int H, int W, int C,
                                   float* __restrict__ t)
{
    // one thread per pixel (field reads coalesced across the warp), zeros up to C
    const long long HW = (long long)H * W;
    const long long npix = (long long)B * HW;
    for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < npix;
         pix += (long long)gridDim.x * blockDim.x) {
        const long long b = pix / HW, q = pix - b * HW;
        float* dst = t + pix * C;
        for (int c = 0; c < C; ++c) {
            float v = 0.f;
            if (c < nf) {
                const long long o = b * stride + c * HW + q;
                v = (float)((Unext[o] - Unow[o]) / scale[c]);
            }
            dst[c] = v;
        }
    }
}

// second-order periodic central differences of [B][nf][H][W] FP64 fields (spacing dx)
__global__ void gradient_kernel(const double* __restrict__ U, long long stride, int nf, int B, int H, int W, double dx,
                                double* __restrict__ dUx, double* __restrict__ dUy)
{
    const long long HW = (long long)H * W;
    const long long n = (long long)B * nf * HW;
    const double s = 0.5 / dx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % W);
        const int y = (int)((i / W) % H);
        const long long fld = i / HW;
        const int c = (int)(fld % nf), b = (int)(fld / nf);
        const double* u = U + (long long)b * stride + c * HW;
        const long long o = (long long)b * stride + c * HW + (long long)y * W + x;
        dUx[o] = s * (u[(long long)y * W + ((x + 1) % W)] - u[(long long)y * W + ((x + W - 1) % W)]);
        dUy[o] = s * (u[(long long)((y + 1) % H) * W + x] - u[(long long)((y + H - 1) % H) * W + x]);
    }
}

int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(long long v)
{
    int l = 0;
    while ((1LL << l) < v) ++l;
    return l;
}

// dynamic shared-memory opt-in of the tile convolution, set once per device and variant
// (setting it twice from racing threads is harmless)
constexpr int kMaxDevices = 64;
bool g_conv3_attr[kMaxDevices][8] = {};
bool g_wgrad3_attr[kMaxDevices] = {};

// pixels per split of the weight gradient: enough splits for about four blocks per
// SM (a block walks its pixels serially), at least 1024 pixels (16 chunks) each
long long wgrad_pixels_per_split(int Cin, int Cout, long long P, int KS)
{
    const long long tiles = (long long)((Cout + 63) / 64) * KS * KS * ((Cin + 63) / 64);
    long long splits = (4 * 152 + tiles - 1) / tiles;
    const long long max_splits = (P + 1023) / 1024;
    if (splits > max_splits) splits = max_splits;
    if (splits < 1) splits = 1;
    long long pps = (P + splits - 1) / splits;
    return (pps + 63) / 64 * 64;
}

// convolutions launched since the library was loaded: forward [0] tcgen05, [1] mma.sync;
// weight gradient [2] block-tiled, [3] per tap
std::atomic<long long> g_conv_launches[4];

// the block-tiled 3x3 weight gradient applies (C1, C2 are multiples of 32 already)
bool wgrad3_applies(int Cout, int H, int W, int KS) { return KS == 3 && H >= 16 && W >= 16 && Cout % 32 == 0; }

// 16 x 16 pixel blocks per split of the block-tiled kernel: about four CTAs per SM
long long wgrad3_blocks_per_split(int Cin, int Cout, int B, int H, int W)
{
    const long long nblocks = (long long)B * (H / 16) * (W / 16);
    const long long tiles = (long long)(Cout / 32) * (Cin / 32);
    long long splits = (4 * 152 + tiles - 1) / tiles;
    if (splits > nblocks) splits = nblocks;
    if (splits < 1) splits = 1;
    return (nblocks + splits - 1) / splits;
}

lbm_status launch_status()
{
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace

extern "C" {

lbm_status lbm_nn_conv_forward(const float* x1, int32_t C1, const float* x2, int32_t C2, const void* w_bf16,
                               const float* bias, float* y1, int32_t Co1, float* y2, int32_t Cout, int32_t B,
                               int32_t H, int32_t W, int32_t KS, int32_t flags, void* stream)
{
    if (!x1 || !w_bf16 || !y1 || C1 <= 0 || C1 % 32 || C2 < 0 || C2 % 32 || (C2 > 0 && !x2) || Cout <= 0 ||
        Cout % 8 || Co1 <= 0 || Co1 > Cout || (Co1 < Cout && !y2) || B <= 0 || !pow2(H) || !pow2(W) ||
        (KS != 1 && KS != 3) || (flags & ~31) || ((flags & LBM_NN_X1_HALF) && (H < 2 || W < 2)))
        return LBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (KS == 3 && !(flags & LBM_NN_MMA_SYNC)) {
        // tcgen05 kernel where its tiling applies (H >= 16, W >= 8, Cout a multiple of 32)
        const ConvTcArgs t{x1, x2, C1, C2, static_cast<const uint16_t*>(w_bf16), bias, y1, y2, Co1, Cout, B, H, W,
                           (flags & LBM_NN_RELU) ? 1 : 0, (flags & LBM_NN_ACCUMULATE) ? 1 : 0,
                           (flags & LBM_NN_X1_HALF) ? 1 : 0, (flags & LBM_NN_ACT_BF16) ? 1 : 0};
        if (conv3_tc_launch(t, s, 0)) {
            g_conv_launches[0].fetch_add(1, std::memory_order_relaxed);
            return launch_status();
        }
    }
    g_conv_launches[1].fetch_add(1, std::memory_order_relaxed);
    ConvArgs a{x1, x2, C1, C2, static_cast<const __nv_bfloat16*>(w_bf16), bias, y1, y2, Co1, Cout, B, H, W,
               (flags & LBM_NN_RELU) ? 1 : 0, (flags & LBM_NN_ACCUMULATE) ? 1 : 0, (flags & LBM_NN_X1_HALF) ? 1 : 0,
               (flags & LBM_NN_ACT_BF16) ? 1 : 0};
    const long long P = (long long)B * H * W;
    if (KS == 3 && H >= 8 && W >= TW && Cout % 32 == 0) {
        // halo-tiled kernel: BN = 64 when it divides Cout, else 32; 16-row tiles when H allows
        const bool lo = !a.act_bf16;
        const int th = H >= 16 ? 16 : 8;
        const long long tiles = (long long)B * (H / th) * (W / TW);
        const int bn = (Cout % 64 == 0) ? 64 : 32;
        const dim3 grid((unsigned)tiles, (unsigned)(Cout / bn));
        int dev = 0;
        cudaGetDevice(&dev);
#define LBM_CONV3(BNV, LOV, THV)                                                                     \
    do {                                                                                             \
        constexpr int smem = conv3_tile_smem_bytes<BNV, THV>();                                      \
        constexpr int slot = (BNV == 64 ? 4 : 0) + (LOV ? 2 : 0) + (THV == 16 ? 1 : 0);              \
        if (dev >= 0 && dev < kMaxDevices && !g_conv3_attr[dev][slot]) {                             \
            cudaFuncSetAttribute(conv3_tile_kernel<BNV, LOV, THV>,                                   \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);                 \
            g_conv3_attr[dev][slot] = true;                                                          \
        }                                                                                            \
        conv3_tile_kernel<BNV, LOV, THV><<<grid, 256, smem, s>>>(a);                                 \
    } while (0)
        if (bn == 64) {
            if (th == 16) { if (lo) LBM_CONV3(64, true, 16); else LBM_CONV3(64, false, 16); }
            else { if (lo) LBM_CONV3(64, true, 8); else LBM_CONV3(64, false, 8); }
        } else {
            if (th == 16) { if (lo) LBM_CONV3(32, true, 16); else LBM_CONV3(32, false, 16); }
            else { if (lo) LBM_CONV3(32, true, 8); else LBM_CONV3(32, false, 8); }
        }
#undef LBM_CONV3
        return launch_status();
    }
    const int BN = Cout >= 64 ? 64 : (Cout >= 32 ? 32 : 16);
    dim3 grid((unsigned)((P + CBM - 1) / CBM), (unsigned)((Cout + BN - 1) / BN));
    if (KS == 3) {
        if (BN == 64) conv_fwd_kernel<64, 3><<<grid, 256, 0, s>>>(a);
        else if (BN == 32) conv_fwd_kernel<32, 3><<<grid, 256, 0, s>>>(a);
        else conv_fwd_kernel<16, 3><<<grid, 256, 0, s>>>(a);
    } else {
        if (BN == 64) conv_fwd_kernel<64, 1><<<grid, 256, 0, s>>>(a);
        else if (BN == 32) conv_fwd_kernel<32, 1><<<grid, 256, 0, s>>>(a);
        else conv_fwd_kernel<16, 1><<<grid, 256, 0, s>>>(a);
    }
    return launch_status();
}

lbm_status lbm_nn_conv_counts(int64_t* out)
{
    if (!out) return LBM_ERR_ARG;
    for (int i = 0; i < 4; ++i) out[i] = g_conv_launches[i].load(std::memory_order_relaxed);
    return LBM_OK;
}

lbm_status lbm_nn_check(void* stream)
{
    return conv3_tc_take_timeout(static_cast<cudaStream_t>(stream)) ? LBM_ERR_TIMEOUT : launch_status();
}

int64_t lbm_nn_wgrad_workspace_bytes(int32_t Cin, int32_t Cout, int32_t B, int32_t H, int32_t W, int32_t KS)
{
    const long long P = (long long)B * H * W;
    const long long pps = wgrad_pixels_per_split(Cin, Cout, P, KS);
    long long splits = (P + pps - 1) / pps;
    if (wgrad3_applies(Cout, H, W, KS)) {       // either kernel may run: room for the larger split count
        const long long nblocks = (long long)B * (H / 16) * (W / 16);
        const long long bps = wgrad3_blocks_per_split(Cin, Cout, B, H, W);
        const long long s3 = (nblocks + bps - 1) / bps;
        if (s3 > splits) splits = s3;
    }
    return splits * (long long)Cout * KS * KS * Cin * (long long)sizeof(float);
}

lbm_status lbm_nn_conv_backward_weight(const float* dy, int32_t Cout, const float* x1, int32_t C1, const float* x2,
                                       int32_t C2, int32_t B, int32_t H, int32_t W, int32_t KS, float* dw,
                                       int32_t flags, void* workspace, int64_t workspace_bytes, void* stream)
{
    if (!dy || !x1 || !dw || !workspace || C1 <= 0 || C1 % 32 || C2 < 0 || C2 % 32 || (C2 > 0 && !x2) ||
        Cout <= 0 || Cout % 8 || B <= 0 || !pow2(H) || !pow2(W) || (KS != 1 && KS != 3) ||
        (flags & ~(LBM_NN_ACCUMULATE | LBM_NN_X1_HALF | LBM_NN_WGRAD_PER_TAP)) ||
        ((flags & LBM_NN_X1_HALF) && (H < 2 || W < 2)))
        return LBM_ERR_ARG;
    const int beta = (flags & LBM_NN_ACCUMULATE) ? 1 : 0;
    const int Cin = C1 + C2;
    if (workspace_bytes < lbm_nn_wgrad_workspace_bytes(Cin, Cout, B, H, W, KS)) return LBM_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (wgrad3_applies(Cout, H, W, KS) && !(flags & LBM_NN_WGRAD_PER_TAP)) {
        const long long nblocks = (long long)B * (H / 16) * (W / 16);
        const int bps = (int)wgrad3_blocks_per_split(Cin, Cout, B, H, W);
        const int splits = (int)((nblocks + bps - 1) / bps);
        Wgrad3Args g3{dy, x1, x2, C1, C2, Cout, B, H, W, bps, static_cast<float*>(workspace),
                      (flags & LBM_NN_X1_HALF) ? 1 : 0};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < kMaxDevices && !g_wgrad3_attr[dev]) {
            cudaFuncSetAttribute(conv_wgrad3_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 conv_wgrad3_smem_bytes());
            g_wgrad3_attr[dev] = true;
        }
        conv_wgrad3_tile_kernel<<<dim3((unsigned)(Cout / 32), (unsigned)(Cin / 32), (unsigned)splits), G3THREADS,
                                  conv_wgrad3_smem_bytes(), st>>>(g3);
        const long long n = (long long)Cout * 9 * Cin;
        sum_splits_kernel<<<grid_for(n), 256, 0, st>>>(static_cast<const float*>(workspace), splits, n, dw, beta);
        g_conv_launches[2].fetch_add(1, std::memory_order_relaxed);
        return launch_status();
    }
    g_conv_launches[3].fetch_add(1, std::memory_order_relaxed);
    const long long P = (long long)B * H * W;
    const int pps = (int)wgrad_pixels_per_split(Cin, Cout, P, KS);
    const int splits = (int)((P + pps - 1) / pps);
    WgradArgs a{dy, x1, x2, C1, C2, Cout, B, H, W, KS, pps, static_cast<float*>(workspace), ilog2(W), ilog2(H * W),
                (flags & LBM_NN_X1_HALF) ? 1 : 0};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dim3 grid((unsigned)((Cout + 63) / 64), (unsigned)(KS * KS * ((Cin + 63) / 64)), (unsigned)splits);
    conv_wgrad_kernel<<<grid, 256, 0, s>>>(a);
    const long long n = (long long)Cout * KS * KS * Cin;
    sum_splits_kernel<<<grid_for(n), 256, 0, s>>>(static_cast<const float*>(workspace), splits, n, dw, beta);
    return launch_status();
}

int64_t lbm_nn_bias_grad_workspace_bytes(int64_t P, int32_t C)
{
    if (P <= 0 || C <= 0) return 0;
    return (int64_t)bias_grad_blocks(P, C) * C * (int64_t)sizeof(float);
}

lbm_status lbm_nn_bias_grad(const float* dy, int64_t P, int32_t C, float* db, void* workspace,
                            int64_t workspace_bytes, void* stream)
{
    if (!dy || !db || !workspace || P <= 0 || C <= 0) return LBM_ERR_ARG;
    if (workspace_bytes < lbm_nn_bias_grad_workspace_bytes(P, C)) return LBM_ERR_ARG;
    const int nblk = bias_grad_blocks(P, C);
    const long long ppb = bias_grad_ppb(P, C);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* part = static_cast<float*>(workspace);
    bias_grad_partial_kernel<<<nblk, 256, 0, s>>>(dy, P, C, ppb, part);
    bias_grad_finish_kernel<<<C, 256, 0, s>>>(part, nblk, C, db);
    return launch_status();
}

lbm_status lbm_nn_weight_flip(const void* w_bf16, int32_t Cout, int32_t Cin, int32_t KS, void* wt_bf16, void* stream)
{
    if (!w_bf16 || !wt_bf16 || Cout <= 0 || Cin <= 0 || (KS != 1 && KS != 3)) return LBM_ERR_ARG;
    const long long n = (long long)Cout * KS * KS * Cin;
    weight_flip_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16*>(w_bf16), Cout, Cin, KS, static_cast<__nv_bfloat16*>(wt_bf16));
    return launch_status();
}

lbm_status lbm_nn_relu_backward(float* dy, const float* y, int64_t n, void* stream)
{
    if (!dy || !y || n < 0) return LBM_ERR_ARG;
    relu_backward_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(dy, y, n);
    return launch_status();
}

lbm_status lbm_nn_pool(const float* x, int32_t B, int32_t H, int32_t W, int32_t C, float* y, void* stream)
{
    if (!x || !y || B <= 0 || H < 2 || W < 2 || (H & 1) || (W & 1) || C <= 0) return LBM_ERR_ARG;
    if (pow2(H) && pow2(W) && C % 4 == 0 && pow2(C / 4)) {
        const long long n = (long long)B * (H / 2) * (W / 2) * (C / 4);
        pool4_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
            reinterpret_cast<const float4*>(x), ilog2(H / 2), ilog2(W / 2), ilog2(C / 4), n, reinterpret_cast<float4*>(y));
        return launch_status();
    }
    pool_kernel<<<grid_for((long long)B * H * W * C / 4), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, B, H, W, C, y);
    return launch_status();
}

lbm_status lbm_nn_pool_backward(const float* dy, int32_t B, int32_t H, int32_t W, int32_t C, float* dx, int32_t beta,
                                void* stream)
{
    if (!dy || !dx || B <= 0 || H < 2 || W < 2 || (H & 1) || (W & 1) || C <= 0) return LBM_ERR_ARG;
    pool_backward_kernel<<<grid_for((long long)B * H * W * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        dy, B, H, W, C, dx, beta);
    return launch_status();
}

lbm_status lbm_nn_upsample(const float* x, int32_t B, int32_t H, int32_t W, int32_t C, float* y, void* stream)
{
    if (!x || !y || B <= 0 || H <= 0 || W <= 0 || C <= 0) return LBM_ERR_ARG;
    if (pow2(H) && pow2(W) && C % 4 == 0 && pow2(C / 4)) {
        const long long n = (long long)B * (2 * H) * (2 * W) * (C / 4);
        upsample4_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
            reinterpret_cast<const float4*>(x), ilog2(2 * H), ilog2(2 * W), ilog2(C / 4), n, reinterpret_cast<float4*>(y));
        return launch_status();
    }
    upsample_kernel<<<grid_for((long long)B * H * W * C * 4), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, B, H, W,
                                                                                                           C, y);
    return launch_status();
}

lbm_status lbm_nn_upsample_backward(const float* dy, int32_t B, int32_t H, int32_t W, int32_t C, float* dx,
                                    int32_t beta, void* stream)
{
    if (!dy || !dx || B <= 0 || H <= 0 || W <= 0 || C <= 0) return LBM_ERR_ARG;
    upsample_backward_kernel<<<grid_for((long long)B * H * W * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        dy, B, H, W, C, dx, beta);
    return launch_status();
}

lbm_status lbm_nn_mse(const float* out, const float* tgt, int64_t P, int32_t C, int32_t cvalid, float grad_scale,
                      float* dout, double* workspace, double* loss_out, void* stream)
{
    if (!out || !tgt || !workspace || !loss_out || P <= 0 || C <= 0 || cvalid < 0 || cvalid > C) return LBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    mse_kernel<<<512, 256, 0, s>>>(out, tgt, P, C, cvalid, grad_scale, dout, workspace);
    sum_double_kernel<<<1, 256, 0, s>>>(workspace, 512, loss_out);
    return launch_status();
}

lbm_status lbm_nn_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                       float eps, int64_t step, void* w_bf16, void* stream)
{
    if (!w || !g || !m || !v || n <= 0 || step < 1) return LBM_ERR_ARG;
    const float c1 = 1.f / (1.f - powf(beta1, (float)step));
    const float c2 = 1.f / (1.f - powf(beta2, (float)step));
    adam_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        w, g, m, v, n, lr, beta1, beta2, eps, c1, c2, static_cast<__nv_bfloat16*>(w_bf16));
    return launch_status();
}

lbm_status lbm_nn_to_bf16(const float* x, int64_t n, void* y_bf16, void* stream)
{
    if (!x || !y_bf16 || n <= 0) return LBM_ERR_ARG;
    to_bf16_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n,
                                                                               static_cast<__nv_bfloat16*>(y_bf16));
    return launch_status();
}

lbm_status lbm_nn_pack_input(const double* U, int64_t sample_stride, int32_t nf, const double* scale,
                             const float* extra, int32_t B, int32_t H, int32_t W, int32_t C, float* x, void* stream)
{
    if (!U || !scale || !x || nf <= 0 || C < nf + (extra ? 1 : 0) || B <= 0 || H <= 0 || W <= 0) return LBM_ERR_ARG;
    pack_input_kernel<<<grid_for((long long)B * H * W), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        U, sample_stride, nf, scale, extra, B, H, W, C, x);
    return launch_status();
}

lbm_status lbm_nn_pack_target(const double* Unow, const double* Unext, int64_t sample_stride, int32_t nf,
                              const double* scale, int32_t B, int32_t H, int32_t W, int32_t C, float* t, void* stream)
{
    if (!Unow || !Unext || !scale || !t || nf <= 0 || C < nf || B <= 0 || H <= 0 || W <= 0) return LBM_ERR_ARG;
    pack_target_kernel<<<grid_for((long long)B * H * W), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        Unow, Unext, sample_stride, nf, scale, B, H, W, C, t);
    return launch_status();
}

lbm_status lbm_nn_residual_output(const double* Uin, int64_t in_stride, const float* net, int32_t C,
                                  const double* scale, int32_t nf, int32_t B, int32_t H, int32_t W, double* Uout,
                                  int64_t out_stride, void* stream)
{
    if (!Uin || !net || !scale || !Uout || nf <= 0 || C < nf || B <= 0 || H <= 0 || W <= 0) return LBM_ERR_ARG;
    residual_output_kernel<<<grid_for((long long)B * nf * H * W), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        Uin, in_stride, net, C, scale, nf, B, H, W, Uout, out_stride);
    return launch_status();
}

lbm_status lbm_nn_gradient(const double* U, int64_t sample_stride, int32_t nf, int32_t B, int32_t H, int32_t W,
                           double dx, double* dUx, double* dUy, void* stream)
{
    if (!U || !dUx || !dUy || nf <= 0 || B <= 0 || H < 3 || W < 3 || !(dx > 0)) return LBM_ERR_ARG;
    gradient_kernel<<<grid_for((long long)B * nf * H * W), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        U, sample_stride, nf, B, H, W, dx, dUx, dUy);
    return launch_status();
}

}  // extern "C"
