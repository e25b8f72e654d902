// Launch table of one storage format: every kernel of lbm_kernels.cuh is
// instantiated once per format in lbm_kind.cu (compiled four times with
// LBM_KIND = 0..3) and reached through these function pointers.
#pragma once

#include <cuda_runtime.h>

#include "lbm_batch.cuh"
#include "lbm_f64stage.cuh"
#include "lbm_kernels.cuh"
#include "lbm_ms.cuh"
#include "lbm_tb.cuh"
#include "lbm_tbt.cuh"

namespace lbmh {

// step variant bits; bits 4-7 hold the FP64 split level (0 = every addition on the FP64 pipe)
enum { STEP_DIRICHLET = 1, STEP_FORCING = 2, STEP_TRACK = 4, STEP_OMEGA = 8, STEP_SPLIT_SHIFT = 4,
       STEP_SPLIT_LEVELS = 13, STEP_SPLIT_FIXED = 12 };

// additions moved to the integer pipes at split level 1..7, as bit masks over the
// node's 35 additions (bit layout of lbmk::collide_split): 0-4 f*_(-1,0), 5-9
// f*_(0,-1), 10-14 y-pair sums, 15-19 x-pair sums, 20-24 U, 25-29 / 30-34 U/2 + t.
// On GB300 at 8192^2 (three 256-thread blocks per SM) level 1 ran at 1.36x the
// FP64-pipe-only step, levels 2-5 at 1.30-1.34x, 6 at 1.12x, 7 at 1.23x.
constexpr unsigned long long split_mask(int level)
{
    return level == 1 ? lbmk::kSplitDefaultMask    // 15: the pair sums and U (fastest measured, the default)
         : level == 2 ? 0x001F07C1Full    // 15: f*_(-1,0), y-pair sums, U
         : level == 3 ? 0x001F0FC1Full    // 16: f*_(-1,0), y-pair sums, U, x-pair sum 0
         : level == 4 ? 0x001F003FFull    // 15: f*_(-1,0), f*_(0,-1), U
         : level == 5 ? 0x000F07C1Full    // 14: f*_(-1,0), y-pair sums, U 0-3
         : level == 6 ? 0x001FFFC1Full    // 20: f*_(-1,0), pair sums, U
         : level == 7 ? 0x007F07C1Full    // 17: f*_(-1,0), y-pair sums, U, U/2 + t of (1,0) 0-1
         // levels 8-11: faithfully rounded integer-pipe additions (emu_add_faithful_bits)
         : level == 8 ? (lbmk::kSplitDefaultMask | lbmk::kSplitFaithful)   // 15: pair sums, U
         : level == 9 ? lbmk::kSplitFastMask                               // 16: + f*_(-1,0) 0
         : level == 10 ? (0x001FFFC03ull | lbmk::kSplitFaithful)           // 17: + f*_(-1,0) 0-1
         : level == 11 ? (0x001FFFC1Full | lbmk::kSplitFaithful)           // 20: + f*_(-1,0)
         // level 12: the whole node in exact fixed-point arithmetic (lbm_f64fx.cuh)
         : level == 12 ? lbmk::kSplitFixed
                      : 0ull;
}

constexpr int split_adds(int level)
{
    int n = 0;
    for (unsigned long long m = split_mask(level) & ~(lbmk::kSplitFaithful | lbmk::kSplitFixed); m; m >>= 1)
        n += (int)(m & 1);
    return n;
}

struct KindOps {
    int kind;
    int vec;                       // nodes per thread in the step kernel
    int elem_bytes;
    int state_bytes_per_node;      // bytes of one node in one state buffer
    cudaError_t (*step)(const lbmk::StepArgs&, int variant, dim3 grid, dim3 block, cudaStream_t s);
    cudaError_t (*init)(const lbmk::NodeArgs&, const double* U0, const double* Ux, const double* Uy,
                        const double* B0, const double* u0, dim3 grid, dim3 block, cudaStream_t s);
    cudaError_t (*moments)(const lbmk::NodeArgs&, double* out, dim3 grid, dim3 block, cudaStream_t s);
    cudaError_t (*get_pop)(const lbmk::NodeArgs&, double* f, double* ustar, dim3 grid, dim3 block, cudaStream_t s);
    cudaError_t (*set_pop)(const lbmk::NodeArgs&, const double* f, const double* ustar, dim3 grid, dim3 block,
                           cudaStream_t s);
    cudaError_t (*energy)(const lbmk::NodeArgs&, double* partial, dim3 grid, dim3 block, cudaStream_t s);
    cudaError_t (*error)(const lbmk::NodeArgs&, const double* exact, double* partial, dim3 grid, dim3 block,
                         cudaStream_t s);
    cudaError_t (*finite)(const lbmk::NodeArgs&, int* flag, dim3 grid, dim3 block, cudaStream_t s);
    // batch: one launch of `grid` blocks x 256 threads; persistent launches are cooperative
    cudaError_t (*batch_step)(const lbmk::BatchArgs&, bool persistent, int grid, cudaStream_t s);
    cudaError_t (*batch_occupancy)(int* blocks_per_sm);
    // two fused steps (FP32 / BF16 / FP16 populations only; others return cudaErrorNotSupported)
    cudaError_t (*tb2_step)(const lbmk::TbArgs&, bool dirichlet, dim3 grid, dim3 block, cudaStream_t s);
    // two fused steps with the input rows staged by tensor copies (FP32 / BF16 / FP16 populations
    // and the moment-space formats); maps: the row maps of the source buffer, one for the
    // population formats (box {TbtGeom::WIN, 1, 20}), two for moment space (FP32 part, 16-bit part)
    cudaError_t (*tbt_step)(const CUtensorMap* maps, const lbmk::TbtArgs&, bool dirichlet, dim3 grid, cudaStream_t s);
    // three fused steps (maps with box width Tbt3Geom::WIN, or Tbt3MsGeom::WIN for moment space)
    cudaError_t (*tbt3_step)(const CUtensorMap* maps, const lbmk::TbtArgs&, bool dirichlet, dim3 grid, cudaStream_t s);
    // one FP64 step at split level 1 or 12 with the rows staged by asynchronous copies, `rows`
    // rows per block (other formats and variants return cudaErrorNotSupported)
    cudaError_t (*step_staged)(const lbmk::StepArgs&, int variant, int rows, cudaStream_t s);
    // three fused steps over the tiles of a batch (FP32 / BF16 / FP16; others return
    // cudaErrorNotSupported): `ntiles` blocks, all of periodic or all of Dirichlet lattices
    cudaError_t (*batch_tbt3_step)(const lbmk::BatchTbtArgs&, bool dirichlet, int ntiles, cudaStream_t s);
    int vec_split;                 // nodes per thread of the FP64 split-level step kernels
    int batch_vec;                 // nodes per thread of the batch kernel
};

extern const KindOps kind_ops_0;  // FP64
extern const KindOps kind_ops_1;  // FP32
extern const KindOps kind_ops_2;  // BF16
extern const KindOps kind_ops_3;  // FP16
extern const KindOps kind_ops_4;  // moment space, BF16 deviations
extern const KindOps kind_ops_5;  // moment space, FP16 deviations
extern const KindOps kind_ops_6;  // moment space, block-floating-point deviations

// 3D row map of a lattice buffer (x = column, y = row, z = plane; box {box_w, 1, nplanes},
// out-of-range elements read as zero), defined in lbm_capi.cu
bool encode_rows_map(CUtensorMap* m, void* base, int esize, int nx, int ny, int pitch, long long plane,
                     int nplanes, int box_w);

// reduction tails (format independent), defined in lbm_capi.cu
cudaError_t finish_sum1(const double* partial, int nblk, double* out, cudaStream_t s);
cudaError_t finish_err30(const double* partial, int nblk, double* out, cudaStream_t s);

}  // namespace lbmh
