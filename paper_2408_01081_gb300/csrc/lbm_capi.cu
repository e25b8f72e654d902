// Host side of the C ABI declared in include/lbm.h: argument checks, device
// memory, data tables and kernel launches for one lattice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "lbm.h"
#include "lbm_dispatch.h"

using lbmh::KindOps;
using lbmh::encode_rows_map;

namespace {

__global__ void to_float_kernel(const double* __restrict__ x, long long n, float* __restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

// expand separable wall tables into g[m][c][e] for m in [0, nt)
__global__ void wall_tables_kernel(int R, const double* __restrict__ Xn, const double* __restrict__ Xw,
                                   const double* __restrict__ Yn, const double* __restrict__ Yw,
                                   const double* __restrict__ T, long long nt, int nx, int ny, double* __restrict__ g)
{
    const int nwall = 2 * (nx + ny);
    const long long n = nt * nwall;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(id % nwall);
        const long long m = id / nwall;
        double gx = 0.0, gy = 0.0;
        for (int r = 0; r < R; ++r) {
            double xy;
            if (e < ny) xy = Xw[r * 2 + 0] * Yn[(long long)r * ny + e];                        // left wall
            else if (e < 2 * ny) xy = Xw[r * 2 + 1] * Yn[(long long)r * ny + (e - ny)];        // right wall
            else if (e < 2 * ny + nx) xy = Xn[(long long)r * nx + (e - 2 * ny)] * Yw[r * 2 + 0];  // bottom
            else xy = Xn[(long long)r * nx + (e - 2 * ny - nx)] * Yw[r * 2 + 1];                // top
            gx = fma(xy, T[(m * 2 + 0) * R + r], gx);
            gy = fma(xy, T[(m * 2 + 1) * R + r], gy);
        }
        g[(m * 2 + 0) * nwall + e] = gx;
        g[(m * 2 + 1) * nwall + e] = gy;
    }
}


// one row of five planes (first plane p0, consecutive) <-> a dense [5][nx] message
template <typename T>
__global__ void halo_copy_kernel(T* __restrict__ state, long long plane, int pitch, int row, int p0,
                                 T* __restrict__ msg, int nx, bool to_msg)
{
    const int n = 5 * nx;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = i / nx, x = i - k * nx;
        T* s = state + (long long)(p0 + k) * plane + (long long)row * pitch + x;
        if (to_msg) msg[i] = *s;
        else *s = msg[i];
    }
}

cudaError_t halo_copy(int es, void* state, long long plane, int pitch, int row, int p0, void* msg, int nx,
                      bool to_msg, cudaStream_t s)
{
    const int blocks = (5 * nx + 255) / 256 < 152 * 4 ? (5 * nx + 255) / 256 : 152 * 4;
    if (es == 8)
        halo_copy_kernel<unsigned long long><<<blocks, 256, 0, s>>>(static_cast<unsigned long long*>(state), plane,
                                                                    pitch, row, p0,
                                                                    static_cast<unsigned long long*>(msg), nx, to_msg);
    else if (es == 4)
        halo_copy_kernel<unsigned int><<<blocks, 256, 0, s>>>(static_cast<unsigned int*>(state), plane, pitch, row, p0,
                                                              static_cast<unsigned int*>(msg), nx, to_msg);
    else
        halo_copy_kernel<unsigned short><<<blocks, 256, 0, s>>>(static_cast<unsigned short*>(state), plane, pitch, row,
                                                                p0, static_cast<unsigned short*>(msg), nx, to_msg);
    return cudaGetLastError();
}

thread_local std::string g_create_error;

const KindOps* ops_for(int storage)
{
    switch (storage) {
    case LBM_F64: return &lbmh::kind_ops_0;
    case LBM_F32: return &lbmh::kind_ops_1;
    case LBM_BF16: return &lbmh::kind_ops_2;
    case LBM_F16: return &lbmh::kind_ops_3;
    case LBM_MS_BF16: return &lbmh::kind_ops_4;
    case LBM_MS_F16: return &lbmh::kind_ops_5;
    case LBM_MS_BFP: return &lbmh::kind_ops_6;
    default: return nullptr;
    }
}

constexpr int kRedBlocks = 152 * 4;   // blocks of the FP64 reductions (one partial each)
constexpr int kMaxR = 16;
constexpr int kTimeoutSlot = kRedBlocks * 30 + 56;   // scratch double index of the staged kernel's timeout flag
constexpr int kSatSlot = kRedBlocks * 30 + 58;       // scratch double index of the block-floating-point saturation flag
constexpr int kEnergyThrSlot = kRedBlocks * 30 + 60; // energy monitor: growth x the energy when it was armed
constexpr int kUnstableSlot = kRedBlocks * 30 + 62;  // energy monitor: set when the energy exceeded it

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point (no link to libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

}  // namespace

namespace lbmh {

// 3D map of a lattice buffer: x = column (extent nx), y = row (extent ny), z = plane
// (extent nplanes); box {box_w, 1, nplanes}, out-of-range elements read as zero
bool encode_rows_map(CUtensorMap* m, void* base, int esize, int nx, int ny, int pitch, long long plane,
                     int nplanes, int box_w)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nplanes};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * esize, (cuuint64_t)plane * esize};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, 1u, (cuuint32_t)nplanes};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace lbmh

namespace {

// 5x5 inverse by Gauss-Jordan elimination with partial pivoting (FP64)
bool invert5(const double (&a_in)[25], double (&inv)[25])
{
    double a[5][10];
    for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 10; ++c) a[r][c] = (c < 5) ? a_in[r * 5 + c] : (c - 5 == r ? 1.0 : 0.0);
    for (int col = 0; col < 5; ++col) {
        int piv = col;
        for (int r = col + 1; r < 5; ++r)
            if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return false;
        if (piv != col)
            for (int c = 0; c < 10; ++c) std::swap(a[piv][c], a[col][c]);
        const double d = a[col][col];
        for (int c = 0; c < 10; ++c) a[col][c] /= d;
        for (int r = 0; r < 5; ++r) {
            if (r == col) continue;
            const double m = a[r][col];
            if (m != 0.0)
                for (int c = 0; c < 10; ++c) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c) inv[r * 5 + c] = a[r][c + 5];
    return true;
}

}  // namespace

struct lbm_ctx {
    lbm_params p{};
    cudaStream_t s = nullptr;
    const KindOps* ops = nullptr;
    int pitch = 0;
    long long plane = 0;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    double* w = nullptr;
    int R = 0;
    double* fX = nullptr;
    double* fY = nullptr;
    double* fT = nullptr;
    float* fXf = nullptr;        // FP32 copies of the body-load tables for the reduced formats
    float* fYf = nullptr;
    float* fTf = nullptr;
    long long fnt = 0;
    double* g = nullptr;
    long long gnt = 0;
    int nwall = 0;
    double* scratch = nullptr;   // kRedBlocks * 30 partials + 32 results + flag
    long long m = 0;
    bool ready = false;
    lbm_status sticky = LBM_OK;
    std::string err;
    double a = 0, b = 0, c = 0;
    double k[4][25] = {};
    double omega = 2.0;
    double neq_scale = 1.0;      // moment-space storage: scale of the stored deviations
    int fuse = 1;                // steps per pass over memory when the fused kernel applies
    int tb_rows = 16;            // rows per block of the fused kernels and the staged FP64 step
    bool rows_set = false;       // tb_rows given by lbm_set_step_fusion (else the staged FP64 step's
                                 // rows per block follow its split level)
    int split = 1;               // FP64: split level (which additions run on the integer pipes; 12:
                                 // the fixed-point node update, the default where it applies)
    int echeck_every = 0;        // energy monitor (lbm_set_energy_check): steps between checks, 0 = off
    int echeck_since = 0;        // steps since the last check
    int staging = 1;             // 1 = rows staged in shared memory (tensor copies for the fused kernels,
                                 // asynchronous copies for the FP64 step), 0 = register loads
    int l2_ahead = lbmk::TBT_L2_AHEAD;   // staged kernel: rows prefetched into L2 ahead of the ring
                                         // (environment LBM_TBT_L2_AHEAD, 0..64, read at lbm_create)
    int nyi = 0;                 // rows of the lattice's own (a slab: without its halo rows)
    int yo = 0;                  // storage row of own row 0 (1 when a halo row sits below)
    bool slab = false;           // a row slab of a larger lattice (lbm_create_slab)
    int halo_lo = 0, halo_hi = 0;  // halo rows below / above the slab's own rows (0 or 1)
    bool maps_ok = false;        // row maps of both buffers encoded (all formats but FP64)
    CUtensorMap map[2][2];       // row maps of buf[0], buf[1] for the staged fused kernel
                                 // ([buffer][part]; moment space: FP32 part, 16-bit part)
    CUtensorMap map3[2][2];      // row maps of the three-step kernels (narrower box)
};

namespace {

lbm_status fail(lbm_ctx* ctx, lbm_status st, const std::string& msg)
{
    if (ctx) {
        ctx->err = msg;
        if (st == LBM_ERR_CUDA) ctx->sticky = LBM_ERR_CUDA;
    }
    return st;
}

lbm_status cuda_fail(lbm_ctx* ctx, cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) {
        // a refused allocation leaves the context usable (not sticky); the runtime keeps it as
        // its last error, which the launch checks of later calls would otherwise report as theirs
        cudaGetLastError();
        return fail(ctx, LBM_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return fail(ctx, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(ctx, call)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

#define LBM_CHECK_CTX(ctx)                                               \
    do {                                                                 \
        if (!(ctx)) return LBM_ERR_ARG;                                  \
        if ((ctx)->sticky != LBM_OK) return (ctx)->sticky;               \
    } while (0)

lbmk::NodeArgs node_args(const lbm_ctx* ctx, long long m_time)
{
    lbmk::NodeArgs A;
    A.S = ctx->buf[ctx->cur];
    A.Sout = ctx->buf[ctx->cur];
    A.w = ctx->w;
    A.nx = ctx->p.nx;
    A.ny = ctx->nyi;
    A.yo = ctx->yo;
    A.pitch = ctx->pitch;
    A.plane = ctx->plane;
    A.a = ctx->a;
    A.b = ctx->b;
    A.cK = ctx->p.cK;
    A.cmu = ctx->p.cmu;
    A.dt = ctx->p.dt;
    A.c = ctx->c;
    A.R = 0;
    A.X = A.Y = A.T = nullptr;
    if (ctx->R > 0 && m_time >= 0 && m_time < ctx->fnt) {
        A.R = ctx->R;
        A.X = ctx->fX;
        A.Y = ctx->fY;
        A.T = ctx->fT + m_time * 2 * ctx->R;
    }
    std::memcpy(A.k, ctx->k, sizeof(A.k));
    A.omega = ctx->omega;
    A.neq_scale = ctx->neq_scale;
    A.measure = nullptr;
    A.sat = reinterpret_cast<int*>(ctx->scratch + kSatSlot);
    return A;
}

void node_grid(const lbm_ctx* ctx, dim3& grid, dim3& block)
{
    const long long n = (long long)ctx->p.nx * ctx->nyi;
    long long nb = (n + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    grid = dim3((unsigned)nb);
    block = dim3(256);
}

// The device address of pinned (page-locked) host memory, which kernels read and write in place
// (over NVLink-C2C on GB300), or nullptr for pageable memory.
void* pinned_view(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost) return nullptr;
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, const_cast<void*>(p), 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return d;
}

// a device-readable view of a host or device FP64 array of n values: device memory and pinned
// host memory as they are, pageable host memory copied into a fresh device buffer (stream ordered)
lbm_status stage_in(lbm_ctx* ctx, const double* src, size_t n, int on_device, const double** dev, double** owned)
{
    *owned = nullptr;
    if (!src) {
        *dev = nullptr;
        return LBM_OK;
    }
    if (on_device) {
        *dev = src;
        return LBM_OK;
    }
    if (const void* v = pinned_view(src)) {
        *dev = static_cast<const double*>(v);
        return LBM_OK;
    }
    double* d = nullptr;
    LBM_CUDA(ctx, cudaMallocAsync((void**)&d, n * sizeof(double), ctx->s));
    cudaError_t e = cudaMemcpyAsync(d, src, n * sizeof(double), cudaMemcpyHostToDevice, ctx->s);
    if (e != cudaSuccess) {
        cudaFreeAsync(d, ctx->s);
        return cuda_fail(ctx, e, "cudaMemcpyAsync H2D");
    }
    *dev = d;
    *owned = d;
    return LBM_OK;
}

lbm_status check_ready(lbm_ctx* ctx)
{
    if (!ctx->ready) return fail(ctx, LBM_ERR_STATE, "state not initialised: call lbm_init or lbm_set_populations");
    return LBM_OK;
}

}  // namespace

// Moment-space storage: pick the power-of-two scale of the stored deviations from the
// largest deviation the state about to be stored has (run the storing kernel once with
// `measure` set), so that the 16-bit values use their full precision and stay far from
// overflow (largest stored value about 2048).
template <typename Launch>
lbm_status choose_neq_scale(lbm_ctx* ctx, Launch launch)
{
    if (ctx->p.storage < LBM_MS_BF16) return LBM_OK;
    float* meas = reinterpret_cast<float*>(ctx->scratch + kRedBlocks * 30 + 48);
    LBM_CUDA(ctx, cudaMemsetAsync(meas, 0, sizeof(float), ctx->s));
    lbmk::NodeArgs A = node_args(ctx, -1);
    A.measure = meas;
    LBM_CUDA(ctx, launch(A));
    float mx = 0.f;
    LBM_CUDA(ctx, cudaMemcpyAsync(&mx, meas, sizeof(float), cudaMemcpyDeviceToHost, ctx->s));
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    double s = 1.0;
    if (mx > 0.f && std::isfinite(mx)) {
        const int e = (int)std::floor(std::log2(2048.0 / (double)mx));
        s = std::ldexp(1.0, std::max(-60, std::min(60, e)));
    }
    ctx->neq_scale = s;
    return LBM_OK;
}

extern "C" {

lbm_status lbm_create(const lbm_params* p, lbm_ctx** out)
{
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return LBM_ERR_ARG;
    }
    *out = nullptr;
    if (!p) {
        g_create_error = "params is NULL";
        return LBM_ERR_ARG;
    }
    if (p->nx < 2 || p->ny < 2 || p->ny > 65535 || p->nx > (1 << 24)) {
        g_create_error = "nx must be in [2, 2^24] and ny in [2, 65535]";
        return LBM_ERR_ARG;
    }
    if (p->bc != LBM_PERIODIC && p->bc != LBM_DIRICHLET) {
        g_create_error = "bc must be LBM_PERIODIC or LBM_DIRICHLET";
        return LBM_ERR_ARG;
    }
    if (!ops_for(p->storage)) {
        g_create_error = "unknown storage format";
        return LBM_ERR_ARG;
    }
    if ((p->track_displacement != 0 && p->track_displacement != 1) || p->reserved != 0) {
        g_create_error = "track_displacement must be 0 or 1 and reserved 0";
        return LBM_ERR_ARG;
    }
    if (!(p->dx > 0.0) || !(p->dt > 0.0) || !std::isfinite(p->dx) || !std::isfinite(p->dt) ||
        !(p->cK > 0.0) || !(p->cmu >= 0.0) || !std::isfinite(p->cK) || !std::isfinite(p->cmu)) {
        g_create_error = "dx, dt, cK must be positive and finite, cmu >= 0";
        return LBM_ERR_ARG;
    }
    const double c = p->dx / p->dt;
    if (!(2.0 * std::sqrt(p->cK * p->cK + p->cmu * p->cmu) < c)) {
        g_create_error = "CFL-like condition 2 sqrt(cK^2 + cmu^2) < dx/dt violated";
        return LBM_ERR_CFL;
    }
    lbm_ctx* ctx = new (std::nothrow) lbm_ctx();
    if (!ctx) {
        g_create_error = "host allocation failed";
        return LBM_ERR_OOM;
    }
    ctx->p = *p;
    ctx->nyi = p->ny;
    if (const char* v = std::getenv("LBM_TBT_L2_AHEAD")) {
        const int a = std::atoi(v);
        if (a >= 0 && a <= 64) ctx->l2_ahead = a;
    }
    ctx->s = static_cast<cudaStream_t>(p->stream);
    ctx->ops = ops_for(p->storage);
    ctx->pitch = (p->nx + 63) / 64 * 64;
    ctx->plane = (long long)ctx->pitch * p->ny;
    ctx->c = c;
    ctx->a = p->cK / c;
    ctx->b = p->cmu / c;
    ctx->nwall = 2 * (p->nx + p->ny);
    // three steps per pass for every reduced format (measured faster than one or two steps for each
    // of them at 8192^2, and fewer roundings to the storage format); rows per block measured best
    // per format
    ctx->fuse = (p->storage == LBM_F64) ? 1 : 3;
    ctx->tb_rows = (p->storage == LBM_F64) ? 2 : (p->storage == LBM_F32) ? 12 : 64;
    // FP64: the fixed-point node update by default (within FP64 accuracy, bound by memory
    // instead of the FP64 pipe); the exact integer-pipe sums where its multipliers do not fit
    ctx->split = (lbmfx::mul_ok(ctx->a) && lbmfx::mul_ok(ctx->b)) ? lbmh::STEP_SPLIT_FIXED : 1;
    // symmetrizer blocks k_ij = g_ij^{-1}, g_ij = 1/4 I + (i A_x + j A_y)/(2c)  (Eq. stability_linear)
    const int VI[4] = {1, 0, -1, 0}, VJ[4] = {0, 1, 0, -1};
    for (int d = 0; d < 4; ++d) {
        double Ax[25] = {0}, Ay[25] = {0}, gm[25];
        Ax[0 * 5 + 2] = Ax[2 * 5 + 0] = p->cK;
        Ax[0 * 5 + 3] = Ax[3 * 5 + 0] = p->cmu;
        Ax[1 * 5 + 4] = Ax[4 * 5 + 1] = p->cmu;
        Ay[0 * 5 + 4] = Ay[4 * 5 + 0] = p->cmu;
        Ay[1 * 5 + 2] = Ay[2 * 5 + 1] = p->cK;
        Ay[1 * 5 + 3] = Ay[3 * 5 + 1] = -p->cmu;
        for (int q = 0; q < 25; ++q)
            gm[q] = (q % 6 == 0 ? 0.25 : 0.0) + (VI[d] * Ax[q] + VJ[d] * Ay[q]) / (2.0 * c);
        if (!invert5(gm, ctx->k[d])) {
            delete ctx;
            g_create_error = "singular g_ij";
            return LBM_ERR_CFL;
        }
    }
    const size_t state_bytes = (size_t)ctx->plane * ctx->ops->state_bytes_per_node;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&ctx->buf[i], state_bytes);
    if (e == cudaSuccess && p->track_displacement) e = cudaMalloc((void**)&ctx->w, (size_t)2 * ctx->plane * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->scratch, (size_t)(kRedBlocks * 30 + 64) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->buf[0], 0, state_bytes, ctx->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->buf[1], 0, state_bytes, ctx->s);
    if (e == cudaSuccess && ctx->w) e = cudaMemsetAsync(ctx->w, 0, (size_t)2 * ctx->plane * sizeof(double), ctx->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->scratch, 0, (size_t)(kRedBlocks * 30 + 64) * sizeof(double), ctx->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->s);
    if (e == cudaSuccess && (p->storage == LBM_F32 || p->storage == LBM_BF16 || p->storage == LBM_F16)) {
        const int es = ctx->ops->elem_bytes;
        const int win = es == 4 ? lbmk::TbtGeom<4>::WIN : lbmk::TbtGeom<2>::WIN;
        const int win3 = es == 4 ? lbmk::Tbt3Geom<4>::WIN : lbmk::Tbt3Geom<2>::WIN;
        ctx->maps_ok = true;
        for (int i = 0; i < 2; ++i)
            ctx->maps_ok = ctx->maps_ok &&
                           encode_rows_map(&ctx->map[i][0], ctx->buf[i], es, p->nx, p->ny, ctx->pitch, ctx->plane, 20,
                                           win) &&
                           encode_rows_map(&ctx->map3[i][0], ctx->buf[i], es, p->nx, p->ny, ctx->pitch, ctx->plane, 20,
                                           win3);
    }
    if (e == cudaSuccess && (p->storage == LBM_MS_BF16 || p->storage == LBM_MS_F16 || p->storage == LBM_MS_BFP)) {
        const int win = lbmk::TbtMsGeom::WIN;
        ctx->maps_ok = true;
        for (int i = 0; i < 2; ++i) {
            char* b = static_cast<char*>(ctx->buf[i]);
            const int win3 = lbmk::Tbt3MsGeom::WIN;
            ctx->maps_ok = ctx->maps_ok &&
                           encode_rows_map(&ctx->map[i][0], b, 4, p->nx, p->ny, ctx->pitch, ctx->plane, 5, win) &&
                           encode_rows_map(&ctx->map[i][1], b + 20 * ctx->plane, 2, p->nx, p->ny, ctx->pitch,
                                           ctx->plane, 15, win) &&
                           encode_rows_map(&ctx->map3[i][0], b, 4, p->nx, p->ny, ctx->pitch, ctx->plane, 5, win3) &&
                           encode_rows_map(&ctx->map3[i][1], b + 20 * ctx->plane, 2, p->nx, p->ny, ctx->pitch,
                                           ctx->plane, 15, win3);
        }
    }
    if (e != cudaSuccess) {
        g_create_error = std::string("device allocation failed: ") + cudaGetErrorString(e);
        lbm_destroy(ctx);
        // a refused allocation is not sticky, but the runtime keeps it as its last error, which
        // the launch checks of later calls (cudaGetLastError) would otherwise report as theirs
        if (e == cudaErrorMemoryAllocation) cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
    }
    *out = ctx;
    return LBM_OK;
}

lbm_status lbm_create_slab(const lbm_params* p, int32_t y_begin, int32_t rows, lbm_ctx** out)
{
    g_create_error.clear();
    if (!out || !p) {
        g_create_error = "params and out are required";
        return LBM_ERR_ARG;
    }
    *out = nullptr;
    if (p->ny < 2 || y_begin < 0 || rows < 1 || (long long)y_begin + rows > p->ny) {
        g_create_error = "slab rows [y_begin, y_begin + rows) must lie in [0, ny), ny >= 2";
        return LBM_ERR_ARG;
    }
    if (p->storage == LBM_MS_BF16 || p->storage == LBM_MS_F16 || p->storage == LBM_MS_BFP) {
        g_create_error = "slabs take the population formats (the moment-space scale is chosen per context)";
        return LBM_ERR_ARG;
    }
    const bool dir = p->bc == LBM_DIRICHLET;
    const int lo = (dir && y_begin == 0) ? 0 : 1;               // no neighbour below the bottom wall
    const int hi = (dir && y_begin + rows == p->ny) ? 0 : 1;    // nor above the top wall
    lbm_params q = *p;
    q.ny = rows + lo + hi;
    lbm_status st = lbm_create(&q, out);
    if (st != LBM_OK) return st;
    lbm_ctx* ctx = *out;
    ctx->slab = true;
    ctx->nyi = rows;
    ctx->yo = lo;
    ctx->halo_lo = lo;
    ctx->halo_hi = hi;
    ctx->fuse = 1;
    return LBM_OK;
}

lbm_status lbm_halo_bytes(const lbm_ctx* ctx, int64_t* nbytes)
{
    if (!ctx || !nbytes) return LBM_ERR_ARG;
    *nbytes = ctx->slab ? (int64_t)5 * ctx->p.nx * ctx->ops->elem_bytes : 0;
    return LBM_OK;
}

lbm_status lbm_halo_pack(lbm_ctx* ctx, void* to_lower, void* to_upper)
{
    LBM_CHECK_CTX(ctx);
    if (!ctx->slab) return fail(ctx, LBM_ERR_ARG, "not a slab");
    if ((to_lower != nullptr) != (ctx->halo_lo == 1) || (to_upper != nullptr) != (ctx->halo_hi == 1))
        return fail(ctx, LBM_ERR_ARG, "a message buffer is needed exactly for each neighbour of the slab");
    lbm_status st = check_ready(ctx);
    if (st != LBM_OK) return st;
    const int es = ctx->ops->elem_bytes;
    // pull scheme: the lower neighbour's top row pulls f*_(0,-1) of our first row, the upper
    // neighbour's bottom row pulls f*_(0,1) of our last row
    if (to_lower)
        LBM_CUDA(ctx, halo_copy(es, ctx->buf[ctx->cur], ctx->plane, ctx->pitch, ctx->yo, 3 * 5, to_lower, ctx->p.nx,
                                true, ctx->s));
    if (to_upper)
        LBM_CUDA(ctx, halo_copy(es, ctx->buf[ctx->cur], ctx->plane, ctx->pitch, ctx->yo + ctx->nyi - 1, 1 * 5,
                                to_upper, ctx->p.nx, true, ctx->s));
    return LBM_OK;
}

lbm_status lbm_halo_unpack(lbm_ctx* ctx, const void* from_lower, const void* from_upper)
{
    LBM_CHECK_CTX(ctx);
    if (!ctx->slab) return fail(ctx, LBM_ERR_ARG, "not a slab");
    if ((from_lower != nullptr) != (ctx->halo_lo == 1) || (from_upper != nullptr) != (ctx->halo_hi == 1))
        return fail(ctx, LBM_ERR_ARG, "a message buffer is needed exactly for each neighbour of the slab");
    const int es = ctx->ops->elem_bytes;
    if (from_lower)
        LBM_CUDA(ctx, halo_copy(es, ctx->buf[ctx->cur], ctx->plane, ctx->pitch, 0, 1 * 5, const_cast<void*>(from_lower),
                                ctx->p.nx, false, ctx->s));
    if (from_upper)
        LBM_CUDA(ctx, halo_copy(es, ctx->buf[ctx->cur], ctx->plane, ctx->pitch, ctx->yo + ctx->nyi, 3 * 5,
                                const_cast<void*>(from_upper), ctx->p.nx, false, ctx->s));
    return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx* ctx)
{
    if (!ctx) return LBM_OK;
    cudaStreamSynchronize(ctx->s);
    cudaFree(ctx->buf[0]);
    cudaFree(ctx->buf[1]);
    cudaFree(ctx->w);
    cudaFree(ctx->fX);
    cudaFree(ctx->fY);
    cudaFree(ctx->fT);
    cudaFree(ctx->fXf);
    cudaFree(ctx->fYf);
    cudaFree(ctx->fTf);
    cudaFree(ctx->g);
    cudaFree(ctx->scratch);
    delete ctx;
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

lbm_status lbm_time_step(const lbm_ctx* ctx, int64_t* m)
{
    if (!ctx || !m) return LBM_ERR_ARG;
    *m = ctx->m;
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_ctx* ctx)
{
    LBM_CHECK_CTX(ctx);
    int* flag = reinterpret_cast<int*>(ctx->scratch + kTimeoutSlot);
    int h = 0;
    LBM_CUDA(ctx, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    if (h) {
        LBM_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->s));
        LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
        return fail(ctx, LBM_ERR_TIMEOUT, "a bounded wait of the staged two-step kernel ran out; the state is "
                                          "undefined until re-initialised");
    }
    if (ctx->echeck_every > 0) {
        int* uflag = reinterpret_cast<int*>(ctx->scratch + kUnstableSlot);
        LBM_CUDA(ctx, cudaMemcpyAsync(&h, uflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
        LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
        if (h) {
            LBM_CUDA(ctx, cudaMemsetAsync(uflag, 0, sizeof(int), ctx->s));
            LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
            return fail(ctx, LBM_ERR_UNSTABLE, "the energy ||f||_P exceeded the growth bound of lbm_set_energy_check "
                                               "(or is not finite)");
        }
    }
    return LBM_OK;
}

lbm_status lbm_set_staging(lbm_ctx* ctx, int32_t mode)
{
    LBM_CHECK_CTX(ctx);
    if (mode < 0 || mode > 2) return fail(ctx, LBM_ERR_ARG, "staging mode must be 0, 1 or 2");
    ctx->staging = mode;
    return LBM_OK;
}

lbm_status lbm_set_step_fusion(lbm_ctx* ctx, int32_t steps_per_pass, int32_t rows_per_block)
{
    LBM_CHECK_CTX(ctx);
    if (steps_per_pass < 1 || steps_per_pass > 3 || rows_per_block < 0 || rows_per_block > 65535)
        return fail(ctx, LBM_ERR_ARG, "steps_per_pass must be 1, 2 or 3 and rows_per_block in [0, 65535]");
    ctx->fuse = steps_per_pass;
    if (rows_per_block > 0) {
        ctx->tb_rows = rows_per_block;
        ctx->rows_set = true;
    }
    return LBM_OK;
}

lbm_status lbm_set_fp64_split(lbm_ctx* ctx, int32_t level)
{
    LBM_CHECK_CTX(ctx);
    if (level < 0 || level >= lbmh::STEP_SPLIT_LEVELS) return fail(ctx, LBM_ERR_ARG, "split level must be in [0, 12]");
    if (level == lbmh::STEP_SPLIT_FIXED && (!lbmfx::mul_ok(ctx->a) || !lbmfx::mul_ok(ctx->b)))
        return fail(ctx, LBM_ERR_ARG, "split level 12 needs cK/c and cmu/c in [2^-60, 1/2) (or cmu = 0)");
    ctx->split = level;
    return LBM_OK;
}

lbm_status lbm_set_relaxation(lbm_ctx* ctx, double omega)
{
    LBM_CHECK_CTX(ctx);
    if (!(omega > 0.0) || omega > 2.0 || omega == 1.0)
        return fail(ctx, LBM_ERR_ARG, "omega must be in (0, 1) or (1, 2]");
    ctx->omega = omega;
    return LBM_OK;
}

lbm_status lbm_set_forcing(lbm_ctx* ctx, int32_t R, const double* X, const double* Y, const double* T,
                           int64_t nt, int32_t on_device)
{
    LBM_CHECK_CTX(ctx);
    if (R < 0 || R > kMaxR) return fail(ctx, LBM_ERR_ARG, "R must be in [0, 16]");
    if (ctx->slab && R > 0) return fail(ctx, LBM_ERR_ARG, "a slab has no body load");
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    cudaFree(ctx->fX);
    cudaFree(ctx->fY);
    cudaFree(ctx->fT);
    cudaFree(ctx->fXf);
    cudaFree(ctx->fYf);
    cudaFree(ctx->fTf);
    ctx->fX = ctx->fY = ctx->fT = nullptr;
    ctx->fXf = ctx->fYf = ctx->fTf = nullptr;
    ctx->R = 0;
    ctx->fnt = 0;
    if (R == 0) return LBM_OK;
    if (!X || !Y || !T || nt < 1) return fail(ctx, LBM_ERR_ARG, "forcing tables missing or nt < 1");
    const size_t nX = (size_t)R * ctx->p.nx, nY = (size_t)R * ctx->p.ny, nT = (size_t)nt * 2 * R;
    LBM_CUDA(ctx, cudaMalloc((void**)&ctx->fX, nX * sizeof(double)));
    LBM_CUDA(ctx, cudaMalloc((void**)&ctx->fY, nY * sizeof(double)));
    LBM_CUDA(ctx, cudaMalloc((void**)&ctx->fT, nT * sizeof(double)));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LBM_CUDA(ctx, cudaMemcpyAsync(ctx->fX, X, nX * sizeof(double), kind, ctx->s));
    LBM_CUDA(ctx, cudaMemcpyAsync(ctx->fY, Y, nY * sizeof(double), kind, ctx->s));
    LBM_CUDA(ctx, cudaMemcpyAsync(ctx->fT, T, nT * sizeof(double), kind, ctx->s));
    if (ctx->p.storage != LBM_F64) {
        LBM_CUDA(ctx, cudaMalloc((void**)&ctx->fXf, nX * sizeof(float)));
        LBM_CUDA(ctx, cudaMalloc((void**)&ctx->fYf, nY * sizeof(float)));
        LBM_CUDA(ctx, cudaMalloc((void**)&ctx->fTf, nT * sizeof(float)));
        to_float_kernel<<<256, 256, 0, ctx->s>>>(ctx->fX, (long long)nX, ctx->fXf);
        to_float_kernel<<<256, 256, 0, ctx->s>>>(ctx->fY, (long long)nY, ctx->fYf);
        to_float_kernel<<<256, 256, 0, ctx->s>>>(ctx->fT, (long long)nT, ctx->fTf);
        LBM_CUDA(ctx, cudaGetLastError());
    }
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    ctx->R = R;
    ctx->fnt = nt;
    return LBM_OK;
}

lbm_status lbm_set_dirichlet(lbm_ctx* ctx, const double* g, int64_t nt, int32_t on_device)
{
    LBM_CHECK_CTX(ctx);
    if (ctx->p.bc != LBM_DIRICHLET) return fail(ctx, LBM_ERR_ARG, "lattice is periodic");
    if (ctx->slab && g) return fail(ctx, LBM_ERR_ARG, "a slab takes homogeneous Dirichlet data only");
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    cudaFree(ctx->g);
    ctx->g = nullptr;
    ctx->gnt = 0;
    if (!g) return LBM_OK;
    if (nt < 1) return fail(ctx, LBM_ERR_ARG, "nt < 1");
    const size_t n = (size_t)nt * 2 * ctx->nwall;
    LBM_CUDA(ctx, cudaMalloc((void**)&ctx->g, n * sizeof(double)));
    LBM_CUDA(ctx, cudaMemcpyAsync(ctx->g, g, n * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->s));
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    ctx->gnt = nt;
    return LBM_OK;
}

lbm_status lbm_set_dirichlet_separable(lbm_ctx* ctx, int32_t R, const double* Xn, const double* Xw, const double* Yn,
                                       const double* Yw, const double* T, int64_t nt, int32_t on_device)
{
    LBM_CHECK_CTX(ctx);
    if (ctx->p.bc != LBM_DIRICHLET) return fail(ctx, LBM_ERR_ARG, "lattice is periodic");
    if (ctx->slab) return fail(ctx, LBM_ERR_ARG, "a slab takes homogeneous Dirichlet data only");
    if (R < 1 || R > kMaxR || !Xn || !Xw || !Yn || !Yw || !T || nt < 1)
        return fail(ctx, LBM_ERR_ARG, "R must be in [1, 16], tables non-NULL and nt >= 1");
    const int nx = ctx->p.nx, ny = ctx->p.ny;
    const double *dXn, *dXw, *dYn, *dYw, *dT;
    double *o1, *o2, *o3, *o4, *o5;
    lbm_status st;
    if ((st = stage_in(ctx, Xn, (size_t)R * nx, on_device, &dXn, &o1)) != LBM_OK) return st;
    if ((st = stage_in(ctx, Xw, (size_t)R * 2, on_device, &dXw, &o2)) != LBM_OK) return st;
    if ((st = stage_in(ctx, Yn, (size_t)R * ny, on_device, &dYn, &o3)) != LBM_OK) return st;
    if ((st = stage_in(ctx, Yw, (size_t)R * 2, on_device, &dYw, &o4)) != LBM_OK) return st;
    if ((st = stage_in(ctx, T, (size_t)nt * 2 * R, on_device, &dT, &o5)) != LBM_OK) return st;
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    cudaFree(ctx->g);
    ctx->g = nullptr;
    ctx->gnt = 0;
    const size_t n = (size_t)nt * 2 * ctx->nwall;
    LBM_CUDA(ctx, cudaMalloc((void**)&ctx->g, n * sizeof(double)));
    long long nb = ((long long)nt * ctx->nwall + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    wall_tables_kernel<<<(unsigned)nb, 256, 0, ctx->s>>>(R, dXn, dXw, dYn, dYw, dT, nt, nx, ny, ctx->g);
    cudaError_t e = cudaGetLastError();
    for (double* o : {o1, o2, o3, o4, o5})
        if (o) cudaFreeAsync(o, ctx->s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "wall tables kernel");
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    ctx->gnt = nt;
    return LBM_OK;
}

lbm_status lbm_init(lbm_ctx* ctx, const double* U0, const double* dU0dx, const double* dU0dy,
                    const double* B0, const double* u0, int32_t on_device)
{
    LBM_CHECK_CTX(ctx);
    if (!U0 || !dU0dx || !dU0dy) return fail(ctx, LBM_ERR_ARG, "U0, dU0dx and dU0dy are required");
    const size_t n = (size_t)ctx->p.nx * ctx->nyi;
    const double *dU0, *dUx, *dUy, *dB0, *du0;
    double *o1, *o2, *o3, *o4, *o5;
    lbm_status st;
    if ((st = stage_in(ctx, U0, 5 * n, on_device, &dU0, &o1)) != LBM_OK) return st;
    if ((st = stage_in(ctx, dU0dx, 5 * n, on_device, &dUx, &o2)) != LBM_OK) return st;
    if ((st = stage_in(ctx, dU0dy, 5 * n, on_device, &dUy, &o3)) != LBM_OK) return st;
    if ((st = stage_in(ctx, B0, 2 * n, on_device, &dB0, &o4)) != LBM_OK) return st;
    if ((st = stage_in(ctx, ctx->w ? u0 : nullptr, 2 * n, on_device, &du0, &o5)) != LBM_OK) return st;
    dim3 grid, block;
    node_grid(ctx, grid, block);
    st = choose_neq_scale(ctx, [&](const lbmk::NodeArgs& M) {
        return ctx->ops->init(M, dU0, dUx, dUy, dB0, du0, grid, block, ctx->s);
    });
    if (st != LBM_OK) return st;
    lbmk::NodeArgs A = node_args(ctx, -1);
    cudaError_t e = ctx->ops->init(A, dU0, dUx, dUy, dB0, du0, grid, block, ctx->s);
    for (double* o : {o1, o2, o3, o4, o5})
        if (o) cudaFreeAsync(o, ctx->s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "init kernel");
    if (!on_device) LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    ctx->m = 0;
    ctx->ready = true;
    return LBM_OK;
}

// n > 0 steps, arguments checked by lbm_step
static lbm_status step_n(lbm_ctx* ctx, int64_t n)
{
    const KindOps* ops = ctx->ops;
    // the split levels apply without body load; the fixed-point update (level 12) with one too
    const bool split = ctx->p.storage == LBM_F64 && ctx->split > 0 &&
                       (ctx->R == 0 || ctx->split == lbmh::STEP_SPLIT_FIXED) && ctx->omega == 2.0;
    const int vec = split ? ops->vec_split : ops->vec;
    const int nchunk = (ctx->p.nx + vec - 1) / vec;
    int bx = (nchunk + 31) / 32 * 32;
    if (bx > 256) bx = 256;
    const dim3 block(bx), grid((nchunk + bx - 1) / bx, ctx->p.ny);
    lbmk::StepArgs A;
    A.w = ctx->w;
    A.nx = ctx->p.nx;
    A.ny = ctx->p.ny;
    A.pitch = ctx->pitch;
    A.plane = ctx->plane;
    A.a = ctx->a;
    A.b = ctx->b;
    A.dt = ctx->p.dt;
    A.R = ctx->R;
    A.X = ctx->fX;
    A.Y = ctx->fY;
    A.Xf = ctx->fXf;
    A.Yf = ctx->fYf;
    A.nwall = ctx->nwall;
    A.omega = ctx->omega;
    A.neq_scale = ctx->neq_scale;
    A.af = (float)ctx->a;
    A.bf = (float)ctx->b;
    A.scale_f = (float)ctx->neq_scale;
    A.inv_scale_f = (float)(1.0 / ctx->neq_scale);
    A.sat = reinterpret_cast<int*>(ctx->scratch + kSatSlot);
    const int variant = (ctx->p.bc == LBM_DIRICHLET ? lbmh::STEP_DIRICHLET : 0) |
                        (ctx->R > 0 ? lbmh::STEP_FORCING : 0) | (ctx->w ? lbmh::STEP_TRACK : 0) |
                        (ctx->omega != 2.0 ? lbmh::STEP_OMEGA : 0) |
                        (split ? ctx->split << lbmh::STEP_SPLIT_SHIFT : 0);
    // two steps per pass: population formats in FP32 / BF16 / FP16 (and the moment-space formats
    // with staged rows), omega = 2, no body load, no displacement tracking, periodic or
    // homogeneous Dirichlet
    const bool ms = ctx->p.storage == LBM_MS_BF16 || ctx->p.storage == LBM_MS_F16 || ctx->p.storage == LBM_MS_BFP;
    const bool fusable = ctx->fuse >= 2 && !ctx->slab &&
                         (ctx->p.storage == LBM_F32 || ctx->p.storage == LBM_BF16 || ctx->p.storage == LBM_F16 ||
                          (ms && ctx->staging >= 1)) &&
                         ctx->omega == 2.0 && ctx->R == 0 && !ctx->w && !(ctx->p.bc == LBM_DIRICHLET && ctx->g);
    if (fusable) {
        lbmk::TbArgs T;
        T.nx = ctx->p.nx;
        T.ny = ctx->p.ny;
        T.pitch = ctx->pitch;
        T.plane = ctx->plane;
        T.a = ctx->a;
        T.b = ctx->b;
        T.af = (float)ctx->a;
        T.bf = (float)ctx->b;
        T.rows = ctx->tb_rows;
        const int nstrip = (ctx->p.nx + lbmk::TB_OUT - 1) / lbmk::TB_OUT;
        const dim3 tblock(128), tgrid((nstrip + 3) / 4, (ctx->p.ny + T.rows - 1) / T.rows);
        if (ctx->staging >= 1) {
            if (!ctx->maps_ok) return fail(ctx, LBM_ERR_CUDA, "tensor maps of the state buffers could not be encoded");
            lbmk::TbtArgs Q;
            Q.nx = ctx->p.nx;
            Q.ny = ctx->p.ny;
            Q.pitch = ctx->pitch;
            Q.plane = ctx->plane;
            Q.af = (float)ctx->a;
            Q.bf = (float)ctx->b;
            Q.rows = ctx->tb_rows;
            Q.timeout = reinterpret_cast<int*>(ctx->scratch + kTimeoutSlot);
            Q.withhold = ctx->staging == 2 ? 2 : -1;
            Q.l2_ahead = ctx->l2_ahead;
            Q.scale = (float)ctx->neq_scale;
            Q.inv_s = (float)(1.0 / ctx->neq_scale);
            Q.sat = reinterpret_cast<int*>(ctx->scratch + kSatSlot);
            if (ctx->fuse == 3) {
                // three steps per pass: the remainder below runs as one pair or a single step
                const dim3 q3grid((ctx->p.nx + lbmk::TBT3_OUT - 1) / lbmk::TBT3_OUT, (ctx->p.ny + Q.rows - 1) / Q.rows);
                while (n >= 3) {
                    Q.src = ctx->buf[ctx->cur];
                    Q.dst = ctx->buf[ctx->cur ^ 1];
                    cudaError_t e = ops->tbt3_step(ctx->map3[ctx->cur], Q, ctx->p.bc == LBM_DIRICHLET, q3grid, ctx->s);
                    if (e != cudaSuccess) return cuda_fail(ctx, e, "staged three-step kernel");
                    ctx->cur ^= 1;
                    ctx->m += 3;
                    n -= 3;
                }
            }
            const dim3 qgrid((ctx->p.nx + lbmk::TBT_OUT - 1) / lbmk::TBT_OUT, (ctx->p.ny + Q.rows - 1) / Q.rows);
            while (n >= 2) {
                Q.src = ctx->buf[ctx->cur];
                Q.dst = ctx->buf[ctx->cur ^ 1];
                cudaError_t e = ops->tbt_step(ctx->map[ctx->cur], Q, ctx->p.bc == LBM_DIRICHLET, qgrid, ctx->s);
                if (e == cudaErrorNotSupported) return fail(ctx, LBM_ERR_ARG, "no staged two-step kernel for this format");
                if (e != cudaSuccess) return cuda_fail(ctx, e, "staged two-step kernel");
                ctx->cur ^= 1;
                ctx->m += 2;
                n -= 2;
            }
        }
        while (n >= 2) {
            T.src = ctx->buf[ctx->cur];
            T.dst = ctx->buf[ctx->cur ^ 1];
            cudaError_t e = ops->tb2_step(T, ctx->p.bc == LBM_DIRICHLET, tgrid, tblock, ctx->s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "fused two-step kernel");
            ctx->cur ^= 1;
            ctx->m += 2;
            n -= 2;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        const long long m = ctx->m;
        A.src = ctx->buf[ctx->cur];
        A.dst = ctx->buf[ctx->cur ^ 1];
        A.T = ctx->R > 0 ? ctx->fT + (m + 1) * 2 * ctx->R : nullptr;
        A.Tf = (ctx->R > 0 && ctx->fTf) ? ctx->fTf + (m + 1) * 2 * ctx->R : nullptr;
        A.g = ctx->g ? ctx->g + m * 2 * ctx->nwall : nullptr;
        // FP64 at split level 1: rows staged by asynchronous copies unless staging is off
        cudaError_t e = cudaErrorNotSupported;
        if (split && (ctx->split == 1 || ctx->split == lbmh::STEP_SPLIT_FIXED) && ctx->staging >= 1) {
            // rows per block measured best at 8192^2: 2 at level 1, 4 for the fixed-point update
            const int rows = ctx->rows_set ? ctx->tb_rows : (ctx->split == 1 ? 2 : 4);
            e = ops->step_staged(A, variant, rows, ctx->s);
        }
        if (e == cudaErrorNotSupported) e = ops->step(A, variant, grid, block, ctx->s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "step kernel");
        ctx->cur ^= 1;
        ctx->m = m + 1;
    }
    return LBM_OK;
}

__global__ void energy_threshold_kernel(const double* e, double growth, double* thr) { *thr = growth * e[0]; }

// sets the flag when the energy exceeds the threshold or is not finite
__global__ void energy_guard_kernel(const double* e, const double* thr, int* flag)
{
    if (!(e[0] <= thr[0])) *flag = 1;
}

// ||f||_P of the current state into the scratch result slot, on the stream, no host wait
static lbm_status energy_on_device(lbm_ctx* ctx)
{
    double* partial = ctx->scratch;
    double* result = ctx->scratch + kRedBlocks * 30;
    LBM_CUDA(ctx, ctx->ops->energy(node_args(ctx, ctx->m), partial, dim3(kRedBlocks), dim3(256), ctx->s));
    LBM_CUDA(ctx, lbmh::finish_sum1(partial, kRedBlocks, result, ctx->s));
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int64_t n)
{
    LBM_CHECK_CTX(ctx);
    if (n < 0) return fail(ctx, LBM_ERR_ARG, "n < 0");
    if (n == 0) return LBM_OK;
    lbm_status st = check_ready(ctx);
    if (st != LBM_OK) return st;
    if (ctx->R > 0 && ctx->m + n >= ctx->fnt)
        return fail(ctx, LBM_ERR_STATE, "body-load table has no row for the requested time");
    if (ctx->g && ctx->m + n > ctx->gnt)
        return fail(ctx, LBM_ERR_STATE, "Dirichlet table has no row for the requested step");
    if (ctx->echeck_every <= 0) return step_n(ctx, n);
    // energy monitor: the steps run in chunks that end where a check is due
    while (n > 0) {
        const int64_t m = std::min<int64_t>(n, ctx->echeck_every - ctx->echeck_since);
        if ((st = step_n(ctx, m)) != LBM_OK) return st;
        n -= m;
        ctx->echeck_since += (int)m;
        if (ctx->echeck_since == ctx->echeck_every) {
            ctx->echeck_since = 0;
            if ((st = energy_on_device(ctx)) != LBM_OK) return st;
            energy_guard_kernel<<<1, 1, 0, ctx->s>>>(ctx->scratch + kRedBlocks * 30, ctx->scratch + kEnergyThrSlot,
                                                     reinterpret_cast<int*>(ctx->scratch + kUnstableSlot));
            LBM_CUDA(ctx, cudaGetLastError());
        }
    }
    return LBM_OK;
}

lbm_status lbm_set_energy_check(lbm_ctx* ctx, int32_t every, double growth)
{
    LBM_CHECK_CTX(ctx);
    if (every < 0) return fail(ctx, LBM_ERR_ARG, "every must be >= 0");
    if (every > 0 && !(growth > 0.0 && std::isfinite(growth)))
        return fail(ctx, LBM_ERR_ARG, "growth must be positive and finite");
    ctx->echeck_every = 0;
    ctx->echeck_since = 0;
    if (every == 0) return LBM_OK;
    lbm_status st = check_ready(ctx);
    if (st != LBM_OK) return st;
    if ((st = energy_on_device(ctx)) != LBM_OK) return st;
    energy_threshold_kernel<<<1, 1, 0, ctx->s>>>(ctx->scratch + kRedBlocks * 30, growth, ctx->scratch + kEnergyThrSlot);
    LBM_CUDA(ctx, cudaGetLastError());
    LBM_CUDA(ctx, cudaMemsetAsync(ctx->scratch + kUnstableSlot, 0, sizeof(int), ctx->s));
    ctx->echeck_every = every;
    return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx* ctx, double* out, int32_t on_device)
{
    LBM_CHECK_CTX(ctx);
    if (!out) return fail(ctx, LBM_ERR_ARG, "out is NULL");
    lbm_status st = check_ready(ctx);
    if (st != LBM_OK) return st;
    const size_t n = (size_t)ctx->p.nx * ctx->nyi;
    double* dst = out;
    // pinned host memory is written in place by the kernel; pageable memory through a device buffer
    double* view = on_device ? nullptr : static_cast<double*>(pinned_view(out));
    const bool staged = !on_device && !view;
    if (view) dst = view;
    if (staged) LBM_CUDA(ctx, cudaMallocAsync((void**)&dst, 10 * n * sizeof(double), ctx->s));
    dim3 grid, block;
    node_grid(ctx, grid, block);
    cudaError_t e = ctx->ops->moments(node_args(ctx, ctx->m), dst, grid, block, ctx->s);
    if (e == cudaSuccess && staged)
        e = cudaMemcpyAsync(out, dst, 10 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->s);
    if (staged) cudaFreeAsync(dst, ctx->s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "moments");
    if (!on_device) LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    return LBM_OK;
}

lbm_status lbm_energy(lbm_ctx* ctx, double* out)
{
    LBM_CHECK_CTX(ctx);
    if (!out) return fail(ctx, LBM_ERR_ARG, "out is NULL");
    lbm_status st = check_ready(ctx);
    if (st != LBM_OK) return st;
    double* partial = ctx->scratch;
    double* result = ctx->scratch + kRedBlocks * 30;
    LBM_CUDA(ctx, ctx->ops->energy(node_args(ctx, ctx->m), partial, dim3(kRedBlocks), dim3(256), ctx->s));
    LBM_CUDA(ctx, lbmh::finish_sum1(partial, kRedBlocks, result, ctx->s));
    LBM_CUDA(ctx, cudaMemcpyAsync(out, result, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    return LBM_OK;
}

lbm_status lbm_error_sums(lbm_ctx* ctx, const double* exact, int32_t on_device, double* out)
{
    LBM_CHECK_CTX(ctx);
    if (!exact || !out) return fail(ctx, LBM_ERR_ARG, "exact and out are required");
    lbm_status st = check_ready(ctx);
    if (st != LBM_OK) return st;
    const size_t n = (size_t)ctx->p.nx * ctx->nyi;
    const double* dex;
    double* owned;
    if ((st = stage_in(ctx, exact, 10 * n, on_device, &dex, &owned)) != LBM_OK) return st;
    double* partial = ctx->scratch;
    double* result = ctx->scratch + kRedBlocks * 30;
    cudaError_t e = ctx->ops->error(node_args(ctx, ctx->m), dex, partial, dim3(kRedBlocks), dim3(256), ctx->s);
    if (e == cudaSuccess) e = lbmh::finish_err30(partial, kRedBlocks, result, ctx->s);
    if (owned) cudaFreeAsync(owned, ctx->s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error sums");
    LBM_CUDA(ctx, cudaMemcpyAsync(out, result, 30 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* ctx, double* f, double* ustar, int32_t on_device)
{
    LBM_CHECK_CTX(ctx);
    if (!f) return fail(ctx, LBM_ERR_ARG, "f is NULL");
    lbm_status st = check_ready(ctx);
    if (st != LBM_OK) return st;
    const size_t n = (size_t)ctx->p.nx * ctx->nyi;
    double *df = f, *du = ustar;
    if (!on_device) {
        LBM_CUDA(ctx, cudaMallocAsync((void**)&df, 22 * n * sizeof(double), ctx->s));
        du = ustar ? df + 20 * n : nullptr;
    }
    dim3 grid, block;
    node_grid(ctx, grid, block);
    cudaError_t e = ctx->ops->get_pop(node_args(ctx, ctx->m), df, du, grid, block, ctx->s);
    if (!on_device) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(f, df, 20 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->s);
        if (e == cudaSuccess && ustar)
            e = cudaMemcpyAsync(ustar, du, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->s);
        cudaFreeAsync(df, ctx->s);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "get_populations");
    if (!on_device) LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* ctx, const double* f, const double* ustar, int64_t m, int32_t on_device)
{
    LBM_CHECK_CTX(ctx);
    if (!f || m < 0) return fail(ctx, LBM_ERR_ARG, "f is NULL or m < 0");
    if (ctx->R > 0 && m >= ctx->fnt) return fail(ctx, LBM_ERR_STATE, "body-load table has no row for step m");
    const size_t n = (size_t)ctx->p.nx * ctx->nyi;
    const double *df, *du;
    double *o1, *o2;
    lbm_status st;
    if ((st = stage_in(ctx, f, 20 * n, on_device, &df, &o1)) != LBM_OK) return st;
    if ((st = stage_in(ctx, ctx->w ? ustar : nullptr, 2 * n, on_device, &du, &o2)) != LBM_OK) return st;
    dim3 grid, block;
    node_grid(ctx, grid, block);
    st = choose_neq_scale(ctx, [&](const lbmk::NodeArgs& M0) {
        lbmk::NodeArgs M = node_args(ctx, m);
        M.measure = M0.measure;
        return ctx->ops->set_pop(M, df, du, grid, block, ctx->s);
    });
    if (st != LBM_OK) return st;
    cudaError_t e = ctx->ops->set_pop(node_args(ctx, m), df, du, grid, block, ctx->s);
    if (o1) cudaFreeAsync(o1, ctx->s);
    if (o2) cudaFreeAsync(o2, ctx->s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_populations");
    if (!on_device) LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    ctx->m = m;
    ctx->ready = true;
    return LBM_OK;
}

lbm_status lbm_check_finite(lbm_ctx* ctx)
{
    LBM_CHECK_CTX(ctx);
    lbm_status st = check_ready(ctx);
    if (st != LBM_OK) return st;
    int* flag = reinterpret_cast<int*>(ctx->scratch + kRedBlocks * 30 + 40);
    LBM_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->s));
    LBM_CUDA(ctx, ctx->ops->finite(node_args(ctx, ctx->m), flag, dim3(152 * 8), dim3(256), ctx->s));
    int h = 0, sat = 0;
    int* satp = reinterpret_cast<int*>(ctx->scratch + kSatSlot);
    LBM_CUDA(ctx, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    LBM_CUDA(ctx, cudaMemcpyAsync(&sat, satp, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    if (h) return fail(ctx, LBM_ERR_UNSTABLE, "non-finite population found");
    if (sat) {
        LBM_CUDA(ctx, cudaMemsetAsync(satp, 0, sizeof(int), ctx->s));
        LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
        return fail(ctx, LBM_ERR_UNSTABLE, "a stored block of deviations exceeded the block-floating-point range "
                                           "(at least 8x the largest deviation at initialisation) and was clamped");
    }
    return LBM_OK;
}

lbm_status lbm_state_bytes(const lbm_ctx* ctx, int64_t* nbytes)
{
    if (!ctx || !nbytes) return LBM_ERR_ARG;
    *nbytes = (int64_t)ctx->plane * ctx->ops->state_bytes_per_node + (ctx->w ? (int64_t)2 * ctx->plane * 8 : 0);
    return LBM_OK;
}

lbm_status lbm_save_state(lbm_ctx* ctx, void* dst, int32_t on_device)
{
    LBM_CHECK_CTX(ctx);
    if (!dst) return fail(ctx, LBM_ERR_ARG, "dst is NULL");
    lbm_status st = check_ready(ctx);
    if (st != LBM_OK) return st;
    const size_t sb = (size_t)ctx->plane * ctx->ops->state_bytes_per_node;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    LBM_CUDA(ctx, cudaMemcpyAsync(dst, ctx->buf[ctx->cur], sb, kind, ctx->s));
    if (ctx->w)
        LBM_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(dst) + sb, ctx->w, (size_t)2 * ctx->plane * 8, kind, ctx->s));
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_ctx* ctx, const void* src, int64_t m, int32_t on_device)
{
    LBM_CHECK_CTX(ctx);
    if (!src || m < 0) return fail(ctx, LBM_ERR_ARG, "src is NULL or m < 0");
    const size_t sb = (size_t)ctx->plane * ctx->ops->state_bytes_per_node;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LBM_CUDA(ctx, cudaMemcpyAsync(ctx->buf[ctx->cur], src, sb, kind, ctx->s));
    if (ctx->w)
        LBM_CUDA(ctx, cudaMemcpyAsync(ctx->w, static_cast<const char*>(src) + sb, (size_t)2 * ctx->plane * 8, kind,
                                      ctx->s));
    LBM_CUDA(ctx, cudaStreamSynchronize(ctx->s));
    ctx->m = m;
    ctx->ready = true;
    return LBM_OK;
}

}  // extern "C"

namespace lbmh {

cudaError_t finish_sum1(const double* partial, int nblk, double* out, cudaStream_t s)
{
    lbmk::finish_kernel<1><<<1, 256, 0, s>>>(partial, nblk, 1, out);
    return cudaGetLastError();
}

cudaError_t finish_err30(const double* partial, int nblk, double* out, cudaStream_t s)
{
    lbmk::finish_kernel<30><<<1, 256, 0, s>>>(partial, nblk, 20, out);
    return cudaGetLastError();
}

}  // namespace lbmh

namespace lbmh {

// message for lbm_last_error(NULL) from context-free entry points in other files
void set_thread_error(const char* msg)
{
    g_create_error = msg ? msg : "";
}

}  // namespace lbmh
