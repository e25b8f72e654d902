// lbm_energy_noalloc: the weighted-norm reduction of lbm_energy for callers that
// cannot allocate device memory.  It needs no context; its scratch (one partial
// sum per lattice row plus a result slot) lives in a file-scope __device__ array
// that every GPU loading this library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "lbm.h"

namespace {

constexpr int kNoAllocMaxRows = 16384;   // rows the static scratch can hold
constexpr int kMaxDevices = 64;

// [0, kNoAllocMaxRows): per-row partial sums; [kNoAllocMaxRows]: result for host output
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxRows + 32];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device

struct KBlocks {
    double k[4][25];
};

// 5x5 inverse, Gauss-Jordan with partial pivoting
bool inverse5(const double (&a_in)[25], double (&inv)[25])
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
            for (int c = 0; c < 10; ++c) {
                const double t = a[piv][c];
                a[piv][c] = a[col][c];
                a[col][c] = t;
            }
        const double d = a[col][col];
        for (int c = 0; c < 10; ++c) a[col][c] /= d;
        for (int r = 0; r < 5; ++r) {
            if (r == col) continue;
            const double m = a[r][col];
            for (int c = 0; c < 10; ++c) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c) inv[r * 5 + c] = a[r][c + 5];
    return true;
}

__device__ __forceinline__ double nwarp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over a block of 256 threads; result valid in thread 0
__device__ __forceinline__ double nblock_sum(double v)
{
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = nwarp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) t = nwarp_sum(lane < 8 ? red[lane] : 0.0);
    __syncthreads();
    return t;
}

// one partial per row: rows[y] = sum_x sum_d f_d^T k_d f_d (f dense [4][5][ny][nx])
__global__ void __launch_bounds__(256) noalloc_rows_kernel(const double* __restrict__ f, int nx, int ny,
                                                           KBlocks K, double* __restrict__ rows)
{
    const long long n = (long long)nx * ny;
    for (int y = blockIdx.x; y < ny; y += gridDim.x) {
        double acc = 0.0;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const long long id = (long long)y * nx + x;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                double v[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) v[q] = f[(d * 5 + q) * n + id];
#pragma unroll
                for (int p = 0; p < 5; ++p) {
                    double kv = 0.0;
#pragma unroll
                    for (int q = 0; q < 5; ++q) kv = fma(K.k[d][p * 5 + q], v[q], kv);
                    acc = fma(v[p], kv, acc);
                }
            }
        }
        acc = nblock_sum(acc);
        if (threadIdx.x == 0) rows[y] = acc;
    }
}

// fixed-order sum of the row partials into *out
__global__ void __launch_bounds__(256) noalloc_final_kernel(const double* __restrict__ rows, int ny,
                                                            double* __restrict__ out)
{
    double acc = 0.0;
    for (int y = threadIdx.x; y < ny; y += blockDim.x) acc += rows[y];
    acc = nblock_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

}  // namespace

namespace lbmh {
void set_thread_error(const char* msg);
}

extern "C" lbm_status lbm_energy_noalloc(const double* f, int32_t nx, int32_t ny, double dx, double dt, double cK,
                                         double cmu, double* out, int32_t out_on_device, void* stream)
{
    if (!f || !out) {
        lbmh::set_thread_error("lbm_energy_noalloc: f and out are required");
        return LBM_ERR_ARG;
    }
    if (nx < 1 || ny < 1 || ny > kNoAllocMaxRows) {
        lbmh::set_thread_error("lbm_energy_noalloc: ny must be in [1, 16384] (one static partial per row), nx >= 1");
        return LBM_ERR_ARG;
    }
    if (!(dx > 0.0) || !(dt > 0.0) || !(cK > 0.0) || !(cmu >= 0.0)) {
        lbmh::set_thread_error("lbm_energy_noalloc: dx, dt, cK must be positive, cmu >= 0");
        return LBM_ERR_ARG;
    }
    const double c = dx / dt;
    if (!(2.0 * std::sqrt(cK * cK + cmu * cmu) < c)) {
        lbmh::set_thread_error("lbm_energy_noalloc: CFL-like condition violated, k_ij not SPD");
        return LBM_ERR_CFL;
    }
    // k_ij = g_ij^{-1} with g_ij = 1/4 I + (i A_x + j A_y) / (2c)
    KBlocks K;
    const int VI[4] = {1, 0, -1, 0}, VJ[4] = {0, 1, 0, -1};
    for (int d = 0; d < 4; ++d) {
        double g[25] = {0};
        for (int q = 0; q < 5; ++q) g[q * 6] = 0.25;
        const double s = 1.0 / (2.0 * c);
        g[0 * 5 + 2] += s * VI[d] * cK;  g[2 * 5 + 0] += s * VI[d] * cK;
        g[0 * 5 + 3] += s * VI[d] * cmu; g[3 * 5 + 0] += s * VI[d] * cmu;
        g[1 * 5 + 4] += s * VI[d] * cmu; g[4 * 5 + 1] += s * VI[d] * cmu;
        g[0 * 5 + 4] += s * VJ[d] * cmu; g[4 * 5 + 0] += s * VJ[d] * cmu;
        g[1 * 5 + 2] += s * VJ[d] * cK;  g[2 * 5 + 1] += s * VJ[d] * cK;
        g[1 * 5 + 3] -= s * VJ[d] * cmu; g[3 * 5 + 1] -= s * VJ[d] * cmu;
        if (!inverse5(g, K.k[d])) {
            lbmh::set_thread_error("lbm_energy_noalloc: singular g_ij");
            return LBM_ERR_CFL;
        }
    }
    // set-up once per device, with that device current: the device address of the scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        lbmh::set_thread_error("lbm_energy_noalloc: no usable current device");
        return LBM_ERR_CUDA;
    }
    // the scratch address and the launch belong to the current device: f (and a device
    // result) must be device memory of that device (or managed memory)
    for (int i = 0; i < (out_on_device ? 2 : 1); ++i) {
        cudaPointerAttributes at{};
        const cudaError_t e = cudaPointerGetAttributes(&at, i == 0 ? static_cast<const void*>(f)
                                                                   : static_cast<const void*>(out));
        const bool here = (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
        if (e != cudaSuccess || !here) {
            cudaGetLastError();   // a failed query leaves no sticky error behind
            lbmh::set_thread_error(i == 0 ? "lbm_energy_noalloc: f is not device memory of the current device"
                                          : "lbm_energy_noalloc: out is not device memory of the current device");
            return LBM_ERR_ARG;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!out_on_device) {
        // a host result needs a wait for the stream, which a capturing stream does not allow
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            lbmh::set_thread_error("lbm_energy_noalloc: out_on_device = 0 waits for the stream, which is not "
                                   "allowed while the stream is being captured");
            return LBM_ERR_ARG;
        }
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                lbmh::set_thread_error((std::string("lbm_energy_noalloc: cudaGetSymbolAddress: ") +
                                        cudaGetErrorString(e)).c_str());
                return LBM_ERR_CUDA;
            }
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    int blocks = ny < 152 * 8 ? ny : 152 * 8;
    noalloc_rows_kernel<<<blocks, 256, 0, s>>>(f, nx, ny, K, scratch);
    double* dst = out_on_device ? out : scratch + kNoAllocMaxRows;
    noalloc_final_kernel<<<1, 256, 0, s>>>(scratch, ny, dst);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !out_on_device) {
        e = cudaMemcpyAsync(out, scratch + kNoAllocMaxRows, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        lbmh::set_thread_error((std::string("lbm_energy_noalloc: ") + cudaGetErrorString(e)).c_str());
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
