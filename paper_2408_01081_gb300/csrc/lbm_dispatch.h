// Launch table of one storage format: every kernel of lbm_kernels.cuh is
// instantiated once per format in lbm_kind.cu (compiled four times with
// LBM_KIND = 0..3) and reached through these function pointers.
#pragma once

#include <cuda_runtime.h>

#include "lbm_batch.cuh"
#include "lbm_kernels.cuh"
#include "lbm_ms.cuh"
#include "lbm_tb.cuh"

namespace lbmh {

// step variant bits
enum { STEP_DIRICHLET = 1, STEP_FORCING = 2, STEP_TRACK = 4, STEP_OMEGA = 8 };

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
};

extern const KindOps kind_ops_0;  // FP64
extern const KindOps kind_ops_1;  // FP32
extern const KindOps kind_ops_2;  // BF16
extern const KindOps kind_ops_3;  // FP16
extern const KindOps kind_ops_4;  // moment space, BF16 deviations
extern const KindOps kind_ops_5;  // moment space, FP16 deviations

// reduction tails (format independent), defined in lbm_capi.cu
cudaError_t finish_sum1(const double* partial, int nblk, double* out, cudaStream_t s);
cudaError_t finish_err30(const double* partial, int nblk, double* out, cudaStream_t s);

}  // namespace lbmh
