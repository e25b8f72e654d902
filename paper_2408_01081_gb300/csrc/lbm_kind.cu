// Instantiates every kernel for one storage format; compiled once per format
// with -DLBM_KIND=<0|1|2|3> (FP64, FP32, BF16, FP16).
#include "lbm_dispatch.h"

#ifndef LBM_KIND
#error "LBM_KIND must be defined"
#endif

namespace {

#ifndef LBM_VEC_F64
#define LBM_VEC_F64 2
#endif
#ifndef LBM_VEC_F32
#define LBM_VEC_F32 4
#endif
#ifndef LBM_VEC_F16
#define LBM_VEC_F16 4
#endif

constexpr int K = LBM_KIND;
// nodes per thread in the step kernel (one vector access per plane and thread)
constexpr int V = (K == lbmk::K_F64) ? LBM_VEC_F64 : (K == lbmk::K_F32) ? LBM_VEC_F32 : LBM_VEC_F16;

template <bool D, bool F, bool T>
cudaError_t step_v(const lbmk::StepArgs& a, dim3 g, dim3 b, cudaStream_t s)
{
    lbmk::step_kernel<K, V, D, F, T><<<g, b, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t step(const lbmk::StepArgs& a, int variant, dim3 g, dim3 b, cudaStream_t s)
{
    switch (variant & 7) {
    case 0: return step_v<false, false, false>(a, g, b, s);
    case 1: return step_v<true, false, false>(a, g, b, s);
    case 2: return step_v<false, true, false>(a, g, b, s);
    case 3: return step_v<true, true, false>(a, g, b, s);
    case 4: return step_v<false, false, true>(a, g, b, s);
    case 5: return step_v<true, false, true>(a, g, b, s);
    case 6: return step_v<false, true, true>(a, g, b, s);
    default: return step_v<true, true, true>(a, g, b, s);
    }
}

cudaError_t init(const lbmk::NodeArgs& a, const double* U0, const double* Ux, const double* Uy,
                 const double* B0, const double* u0, dim3 g, dim3 b, cudaStream_t s)
{
    lbmk::init_kernel<K><<<g, b, 0, s>>>(a, U0, Ux, Uy, B0, u0);
    return cudaGetLastError();
}

cudaError_t moments(const lbmk::NodeArgs& a, double* out, dim3 g, dim3 b, cudaStream_t s)
{
    lbmk::moments_kernel<K><<<g, b, 0, s>>>(a, out);
    return cudaGetLastError();
}

cudaError_t get_pop(const lbmk::NodeArgs& a, double* f, double* ustar, dim3 g, dim3 b, cudaStream_t s)
{
    lbmk::get_populations_kernel<K><<<g, b, 0, s>>>(a, f, ustar);
    return cudaGetLastError();
}

cudaError_t set_pop(const lbmk::NodeArgs& a, const double* f, const double* ustar, dim3 g, dim3 b,
                    cudaStream_t s)
{
    lbmk::set_populations_kernel<K><<<g, b, 0, s>>>(a, f, ustar);
    return cudaGetLastError();
}

cudaError_t energy(const lbmk::NodeArgs& a, double* partial, dim3 g, dim3 b, cudaStream_t s)
{
    lbmk::energy_kernel<K><<<g, b, 0, s>>>(a, partial);
    return cudaGetLastError();
}

cudaError_t error(const lbmk::NodeArgs& a, const double* exact, double* partial, dim3 g, dim3 b,
                  cudaStream_t s)
{
    lbmk::error_kernel<K><<<g, b, 0, s>>>(a, exact, partial);
    return cudaGetLastError();
}

cudaError_t finite(const void* S, int nx, int ny, int pitch, long long plane, int* flag, dim3 g, dim3 b,
                   cudaStream_t s)
{
    lbmk::finite_kernel<K><<<g, b, 0, s>>>(S, nx, ny, pitch, plane, flag);
    return cudaGetLastError();
}

cudaError_t batch_step(const lbmk::BatchArgs& a, bool persistent, int grid, cudaStream_t s)
{
    if (!persistent) {
        lbmk::batch_step_kernel<K, V, false><<<grid, 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, lbmk::batch_step_kernel<K, V, true>, a);
}

cudaError_t batch_occupancy(int* n)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, lbmk::batch_step_kernel<K, V, true>, 256, 0);
}

}  // namespace

namespace lbmh {

#define LBM_OPS_NAME2(k) kind_ops_##k
#define LBM_OPS_NAME(k) LBM_OPS_NAME2(k)

const KindOps LBM_OPS_NAME(LBM_KIND) = {
    K, V, (int)sizeof(typename lbmk::Fmt<K>::E),
    step, init, moments, get_pop, set_pop, energy, error, finite, batch_step, batch_occupancy,
};

}  // namespace lbmh
