// Instantiates every kernel for one storage format; compiled once per format
// with -DLBM_KIND=<0..6> (FP64, FP32, BF16, FP16, and moment space with BF16, FP16
// or block-floating-point deviations).
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
#ifndef LBM_VEC_SPLIT
#define LBM_VEC_SPLIT 1
#endif

constexpr int K = LBM_KIND;
constexpr bool MS = (K >= lbmk::K_MSBF16);
// nodes per thread in the step kernel (one vector access per plane and thread)
constexpr int V = (K == lbmk::K_F64) ? LBM_VEC_F64 : (K == lbmk::K_F32) ? LBM_VEC_F32 : MS ? 4 : LBM_VEC_F16;
constexpr int ELEM = (K == lbmk::K_F64) ? 8 : (K == lbmk::K_F32) ? 4 : 2;
// nodes per thread in the batch kernel (FP64 runs the split collision, at its width)
constexpr int VB = (K == lbmk::K_F64) ? LBM_VEC_SPLIT : V;
constexpr int NODE_BYTES = MS ? 5 * 4 + 15 * 2 : 20 * ELEM;

template <bool D, bool F, bool T, bool O, unsigned long long SPLIT = 0>
cudaError_t step_v(const lbmk::StepArgs& a, dim3 g, dim3 b, cudaStream_t s)
{
    if constexpr (MS) lbmk::ms_step_kernel<K, V, D, F, T, O><<<g, b, 0, s>>>(a);
    else if constexpr (SPLIT > 0) lbmk::step_kernel<K, LBM_VEC_SPLIT, D, F, T, O, SPLIT><<<g, b, 0, s>>>(a);
    else lbmk::step_kernel<K, V, D, F, T, O><<<g, b, 0, s>>>(a);
    return cudaGetLastError();
}

// FP64 without body load and with omega = 2: the number of the node's 35
// additions computed on the integer pipes (lbmh::split_adds of the level)
template <bool D, bool T>
cudaError_t step_split(const lbmk::StepArgs& a, int level, dim3 g, dim3 b, cudaStream_t s)
{
    if constexpr (K != lbmk::K_F64) {
        return cudaErrorNotSupported;
    } else {
        switch (level) {
        case 1: return step_v<D, false, T, false, lbmh::split_mask(1)>(a, g, b, s);
        case 2: return step_v<D, false, T, false, lbmh::split_mask(2)>(a, g, b, s);
        case 3: return step_v<D, false, T, false, lbmh::split_mask(3)>(a, g, b, s);
        case 4: return step_v<D, false, T, false, lbmh::split_mask(4)>(a, g, b, s);
        case 5: return step_v<D, false, T, false, lbmh::split_mask(5)>(a, g, b, s);
        case 6: return step_v<D, false, T, false, lbmh::split_mask(6)>(a, g, b, s);
        case 7: return step_v<D, false, T, false, lbmh::split_mask(7)>(a, g, b, s);
        case 8: return step_v<D, false, T, false, lbmh::split_mask(8)>(a, g, b, s);
        case 9: return step_v<D, false, T, false, lbmh::split_mask(9)>(a, g, b, s);
        case 10: return step_v<D, false, T, false, lbmh::split_mask(10)>(a, g, b, s);
        case 11: return step_v<D, false, T, false, lbmh::split_mask(11)>(a, g, b, s);
        case 12: return step_v<D, false, T, false, lbmh::split_mask(12)>(a, g, b, s);
        default: return cudaErrorInvalidValue;
        }
    }
}

#ifndef LBM_SA_MASK
#define LBM_SA_MASK lbmh::split_mask(1)   // the additions of split level 1 on the integer pipes
#endif

// FP64 at split level 1 or 12 with the rows staged by asynchronous copies (lbm_f64stage.cuh);
// other formats, levels and variants return cudaErrorNotSupported
template <bool D, bool T, unsigned long long M>
cudaError_t step_staged_dt(const lbmk::StepArgs& a, int rows, cudaStream_t s)
{
    if constexpr (K != lbmk::K_F64) {
        return cudaErrorNotSupported;
    } else {
        const dim3 g((a.nx + lbmk::SA_THREADS - 1) / lbmk::SA_THREADS, (a.ny + rows - 1) / rows);
        lbmk::step_f64_staged_kernel<D, T, M><<<g, lbmk::SA_THREADS, 0, s>>>(a, rows);
        return cudaGetLastError();
    }
}

template <unsigned long long M>
cudaError_t step_staged_m(const lbmk::StepArgs& a, bool d, bool t, int rows, cudaStream_t s)
{
    return d ? (t ? step_staged_dt<true, true, M>(a, rows, s) : step_staged_dt<true, false, M>(a, rows, s))
             : (t ? step_staged_dt<false, true, M>(a, rows, s) : step_staged_dt<false, false, M>(a, rows, s));
}

// split levels 1 (LBM_SA_MASK) and 12 (fixed point)
cudaError_t step_staged(const lbmk::StepArgs& a, int variant, int rows, cudaStream_t s)
{
    const int level = (variant >> lbmh::STEP_SPLIT_SHIFT) & 15;
    if ((level != 1 && level != lbmh::STEP_SPLIT_FIXED) || (variant & (lbmh::STEP_FORCING | lbmh::STEP_OMEGA)) ||
        rows < 1)
        return cudaErrorNotSupported;
    const bool d = variant & lbmh::STEP_DIRICHLET, t = variant & lbmh::STEP_TRACK;
    return level == 1 ? step_staged_m<LBM_SA_MASK>(a, d, t, rows, s)
                      : step_staged_m<lbmh::split_mask(lbmh::STEP_SPLIT_FIXED)>(a, d, t, rows, s);
}

template <bool O>
cudaError_t step_o(const lbmk::StepArgs& a, int variant, dim3 g, dim3 b, cudaStream_t s)
{
    switch (variant & 7) {
    case 0: return step_v<false, false, false, O>(a, g, b, s);
    case 1: return step_v<true, false, false, O>(a, g, b, s);
    case 2: return step_v<false, true, false, O>(a, g, b, s);
    case 3: return step_v<true, true, false, O>(a, g, b, s);
    case 4: return step_v<false, false, true, O>(a, g, b, s);
    case 5: return step_v<true, false, true, O>(a, g, b, s);
    case 6: return step_v<false, true, true, O>(a, g, b, s);
    default: return step_v<true, true, true, O>(a, g, b, s);
    }
}

// FP64 with a body load at split level 12 (omega = 2): the fixed-point node update with it
template <bool D, bool T>
cudaError_t step_fixed_forced(const lbmk::StepArgs& a, dim3 g, dim3 b, cudaStream_t s)
{
    if constexpr (K != lbmk::K_F64) {
        return cudaErrorNotSupported;
    } else {
        return step_v<D, true, T, false, lbmh::split_mask(lbmh::STEP_SPLIT_FIXED)>(a, g, b, s);
    }
}

cudaError_t step(const lbmk::StepArgs& a, int variant, dim3 g, dim3 b, cudaStream_t s)
{
    const int level = (variant >> lbmh::STEP_SPLIT_SHIFT) & 15;
    if (level == lbmh::STEP_SPLIT_FIXED && (variant & lbmh::STEP_FORCING) && !(variant & lbmh::STEP_OMEGA)) {
        const bool d = variant & lbmh::STEP_DIRICHLET, t = variant & lbmh::STEP_TRACK;
        return d ? (t ? step_fixed_forced<true, true>(a, g, b, s) : step_fixed_forced<true, false>(a, g, b, s))
                 : (t ? step_fixed_forced<false, true>(a, g, b, s) : step_fixed_forced<false, false>(a, g, b, s));
    }
    if (level && !(variant & (lbmh::STEP_FORCING | lbmh::STEP_OMEGA))) {
        const bool d = variant & lbmh::STEP_DIRICHLET, t = variant & lbmh::STEP_TRACK;
        return d ? (t ? step_split<true, true>(a, level, g, b, s) : step_split<true, false>(a, level, g, b, s))
                 : (t ? step_split<false, true>(a, level, g, b, s) : step_split<false, false>(a, level, g, b, s));
    }
    return (variant & lbmh::STEP_OMEGA) ? step_o<true>(a, variant, g, b, s) : step_o<false>(a, variant, g, b, s);
}

cudaError_t init(const lbmk::NodeArgs& a, const double* U0, const double* Ux, const double* Uy,
                 const double* B0, const double* u0, dim3 g, dim3 b, cudaStream_t s)
{
    if (B0) lbmk::init_kernel<K, true><<<g, b, 0, s>>>(a, U0, Ux, Uy, B0, u0);
    else lbmk::init_kernel<K, false><<<g, b, 0, s>>>(a, U0, Ux, Uy, B0, u0);
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

cudaError_t finite(const lbmk::NodeArgs& a, int* flag, dim3 g, dim3 b, cudaStream_t s)
{
    lbmk::finite_kernel<K><<<g, b, 0, s>>>(a, flag);
    return cudaGetLastError();
}

template <int KK>
cudaError_t batch_step_t(const lbmk::BatchArgs& a, bool persistent, int grid, cudaStream_t s)
{
    if constexpr (KK >= lbmk::K_MSBF16) {
        return cudaErrorNotSupported;        // batches use the population formats only
    } else {
        if (!persistent) {
            lbmk::batch_step_kernel<KK, VB, false><<<grid, 256, 0, s>>>(a);
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
        return cudaLaunchKernelEx(&cfg, lbmk::batch_step_kernel<KK, VB, true>, a);
    }
}

template <int KK>
cudaError_t batch_occupancy_t(int* n)
{
    if constexpr (KK >= lbmk::K_MSBF16) {
        *n = 1;
        return cudaSuccess;
    } else {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, lbmk::batch_step_kernel<KK, VB, true>, 256, 0);
    }
}

cudaError_t batch_step(const lbmk::BatchArgs& a, bool persistent, int grid, cudaStream_t s)
{
    return batch_step_t<K>(a, persistent, grid, s);
}

template <int KK>
cudaError_t tb2_t(const lbmk::TbArgs& a, bool dirichlet, dim3 g, dim3 b, cudaStream_t s)
{
    if constexpr (KK == lbmk::K_F32 || KK == lbmk::K_BF16 || KK == lbmk::K_F16) {
        if (dirichlet) lbmk::tb2_kernel<KK, true><<<g, b, 0, s>>>(a);
        else lbmk::tb2_kernel<KK, false><<<g, b, 0, s>>>(a);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

cudaError_t tb2_step(const lbmk::TbArgs& a, bool dirichlet, dim3 g, dim3 b, cudaStream_t s)
{
    return tb2_t<K>(a, dirichlet, g, b, s);
}

template <int KK>
cudaError_t tbt_t(const CUtensorMap* maps, const lbmk::TbtArgs& a, bool dirichlet, dim3 g, cudaStream_t s)
{
    if constexpr (KK == lbmk::K_F32 || KK == lbmk::K_BF16 || KK == lbmk::K_F16) {
        using G = lbmk::TbtGeom<(int)sizeof(typename lbmk::Fmt<KK>::E)>;
        void (*kern)(CUtensorMap, lbmk::TbtArgs) = dirichlet ? lbmk::tbt_kernel<KK, true> : lbmk::tbt_kernel<KK, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        kern<<<g, lbmk::TBT_THREADS, G::SMEM, s>>>(maps[0], a);
        return cudaGetLastError();
    } else if constexpr (KK == lbmk::K_MSBF16 || KK == lbmk::K_MSF16 || KK == lbmk::K_MSBFP) {
        using G = lbmk::TbtMsGeom;
        void (*kern)(CUtensorMap, CUtensorMap, lbmk::TbtArgs) =
            dirichlet ? lbmk::tbt_ms_kernel<KK, true> : lbmk::tbt_ms_kernel<KK, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        kern<<<g, lbmk::TBT_THREADS, G::SMEM, s>>>(maps[0], maps[1], a);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

cudaError_t tbt_step(const CUtensorMap* maps, const lbmk::TbtArgs& a, bool dirichlet, dim3 g, cudaStream_t s)
{
    return tbt_t<K>(maps, a, dirichlet, g, s);
}

template <int KK>
cudaError_t tbt3_t(const CUtensorMap* maps, const lbmk::TbtArgs& a, bool dirichlet, dim3 g, cudaStream_t s)
{
    if constexpr (KK == lbmk::K_F32 || KK == lbmk::K_BF16 || KK == lbmk::K_F16) {
        using G = lbmk::Tbt3Geom<(int)sizeof(typename lbmk::Fmt<KK>::E)>;
        void (*kern)(CUtensorMap, lbmk::TbtArgs) = dirichlet ? lbmk::tbt3_kernel<KK, true> : lbmk::tbt3_kernel<KK, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        kern<<<g, lbmk::TBT_THREADS, G::SMEM, s>>>(maps[0], a);
        return cudaGetLastError();
    } else if constexpr (KK == lbmk::K_MSBF16 || KK == lbmk::K_MSF16 || KK == lbmk::K_MSBFP) {
        using G = lbmk::Tbt3MsGeom;
        void (*kern)(CUtensorMap, CUtensorMap, lbmk::TbtArgs) =
            dirichlet ? lbmk::tbt3_ms_kernel<KK, true> : lbmk::tbt3_ms_kernel<KK, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        kern<<<g, lbmk::TBT_THREADS, G::SMEM, s>>>(maps[0], maps[1], a);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

cudaError_t tbt3_step(const CUtensorMap* maps, const lbmk::TbtArgs& a, bool dirichlet, dim3 g, cudaStream_t s)
{
    return tbt3_t<K>(maps, a, dirichlet, g, s);
}

template <int KK>
cudaError_t batch_tbt3_t(const lbmk::BatchTbtArgs& a, bool dirichlet, int ntiles, cudaStream_t s)
{
    if constexpr (KK == lbmk::K_F32 || KK == lbmk::K_BF16 || KK == lbmk::K_F16) {
        using G = lbmk::Tbt3Geom<(int)sizeof(typename lbmk::Fmt<KK>::E)>;
        if (ntiles <= 0) return cudaSuccess;
        void (*kern)(lbmk::BatchTbtArgs) =
            dirichlet ? lbmk::batch_tbt3_kernel<KK, true> : lbmk::batch_tbt3_kernel<KK, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        kern<<<ntiles, lbmk::TBT_THREADS, G::SMEM, s>>>(a);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

cudaError_t batch_tbt3_step(const lbmk::BatchTbtArgs& a, bool dirichlet, int ntiles, cudaStream_t s)
{
    return batch_tbt3_t<K>(a, dirichlet, ntiles, s);
}

cudaError_t batch_occupancy(int* n)
{
    return batch_occupancy_t<K>(n);
}

}  // namespace

namespace lbmh {

#define LBM_OPS_NAME2(k) kind_ops_##k
#define LBM_OPS_NAME(k) LBM_OPS_NAME2(k)

const KindOps LBM_OPS_NAME(LBM_KIND) = {
    K, V, ELEM, NODE_BYTES,
    step, init, moments, get_pop, set_pop, energy, error, finite, batch_step, batch_occupancy, tb2_step, tbt_step,
    tbt3_step, step_staged, batch_tbt3_step,
    LBM_VEC_SPLIT, VB,
};

}  // namespace lbmh
