// Host side of the batch API (include/lbm.h): arena layout, tile work-list,
// CUDA-graph replay of many steps, persistent cooperative launches, and the
// autotuner that picks a tile width per size class by timing them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_dispatch.h"

namespace {

thread_local std::string g_batch_create_error;

const lbmh::KindOps* batch_ops_for(int storage)
{
    switch (storage) {
    case LBM_F64: return &lbmh::kind_ops_0;
    case LBM_F32: return &lbmh::kind_ops_1;
    case LBM_BF16: return &lbmh::kind_ops_2;
    case LBM_F16: return &lbmh::kind_ops_3;
    default: return nullptr;
    }
}

const char* storage_name(int s)
{
    static const char* n[4] = {"f64", "f32", "bf16", "f16"};
    return (s >= 0 && s < 4) ? n[s] : "?";
}

constexpr int kRed = 152 * 4;
constexpr int kMinTpr = 8, kMaxTpr = 256;

int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// size class of a lattice: ceil(log2(chunks per row)), clamped to [3, 12]
int size_class(int nchunk)
{
    int c = 0;
    while ((1 << c) < nchunk) ++c;
    return std::min(12, std::max(3, c));
}

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
            for (int c = 0; c < 10; ++c) std::swap(a[piv][c], a[col][c]);
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

}  // namespace

struct lbm_batch {
    int count = 0;
    int storage = 0;
    const lbmh::KindOps* ops = nullptr;
    cudaStream_t s = nullptr;
    std::vector<lbm_lattice_desc> in;
    std::vector<lbmk::LatDesc> lat;      // host copy
    std::vector<int> cls;                // size class per lattice
    std::map<int, int> tpr_of_class;     // tuned threads per row
    lbmk::LatDesc* d_lat = nullptr;
    int* d_tile = nullptr;
    int ntiles = 0;
    size_t tile_cap = 0;
    void* arena[2] = {nullptr, nullptr};
    long long total_elems = 0;
    long long nodes = 0;
    int cur = 0;                          // arena holding the current state
    unsigned int* d_bar = nullptr;        // [0] count, [1] generation, [2] error flag
    double* scratch = nullptr;
    int mode = 0;
    int graph_steps = 100;
    int persistent_grid = 0;
    unsigned long long timeout_ns = 2000000000ull;
    unsigned int extra_arrivals = 0;
    bool own_stream = false;              // created here because the caller gave the legacy stream
    // mode 2: three steps per pass with staged rows (FP32 / BF16 / FP16)
    bool t3_ok = false;                   // row maps encoded and tile lists built
    int t3_rows = 0;                      // output rows per tile
    lbmk::BatchLatT3* d_lat3 = nullptr;
    CUtensorMap* d_maps = nullptr;        // [lattice][arena]
    int4* d_t3 = nullptr;                 // periodic tiles, then Dirichlet tiles
    int nt3[2] = {0, 0};                  // tile counts: periodic, Dirichlet
    // mode 3: FP64 on staged rows, one step per launch (lbm_batch_f64.cu)
    bool f64s_ok = false;                 // tile lists built (FP64 storage)
    int4* d_f64s = nullptr;               // the four lists, one after the other
    int nf64s[4] = {0, 0, 0, 0};          // periodic / Dirichlet x fixed point / split level 1
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    bool initialised = false;
    bool sticky = false;
    std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status st, const std::string& m)
{
    b->err = m;
    if (st == LBM_ERR_CUDA) b->sticky = true;
    return st;
}

#define B_CUDA(b, call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

void drop_graph(lbm_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_valid = false;
}

// (re)build the tile list from the tile widths of the size classes
lbm_status build_tiles(lbm_batch* b)
{
    const int V = b->ops->batch_vec;
    int first = 0;
    std::vector<int> tile_lat;
    for (int i = 0; i < b->count; ++i) {
        lbmk::LatDesc& L = b->lat[i];
        const int nchunk = (L.nx + V - 1) / V;
        int tpr = b->tpr_of_class.count(b->cls[i]) ? b->tpr_of_class[b->cls[i]] : std::min(64, next_pow2(nchunk));
        tpr = std::max(kMinTpr, std::min(kMaxTpr, tpr));
        L.tpr = tpr;
        L.rpt = 256 / tpr;
        L.tiles_x = (nchunk + tpr - 1) / tpr;
        L.tiles_y = (L.ny + L.rpt - 1) / L.rpt;
        L.first_tile = first;
        const int nt = L.tiles_x * L.tiles_y;
        tile_lat.insert(tile_lat.end(), (size_t)nt, i);
        first += nt;
    }
    b->ntiles = first;
    if (b->tile_cap < (size_t)first) {
        cudaFree(b->d_tile);
        b->d_tile = nullptr;
        B_CUDA(b, cudaMalloc((void**)&b->d_tile, (size_t)first * sizeof(int)));
        b->tile_cap = first;
    }
    B_CUDA(b, cudaMemcpyAsync(b->d_lat, b->lat.data(), b->lat.size() * sizeof(lbmk::LatDesc),
                              cudaMemcpyHostToDevice, b->s));
    B_CUDA(b, cudaMemcpyAsync(b->d_tile, tile_lat.data(), (size_t)first * sizeof(int), cudaMemcpyHostToDevice, b->s));
    B_CUDA(b, cudaStreamSynchronize(b->s));
    drop_graph(b);
    return LBM_OK;
}

#ifndef LBM_BATCH_T3_ROWS4
#define LBM_BATCH_T3_ROWS4 12     // output rows per mode-2 tile, FP32 (the single-lattice default)
#endif
#ifndef LBM_BATCH_T3_ROWS2
#define LBM_BATCH_T3_ROWS2 64     // the same for BF16 / FP16
#endif

// Row maps (box width Tbt3Geom::WIN, both arenas) and tile lists of mode 2, for the
// population formats FP32 / BF16 / FP16 and lattices of at least 2 x 2 nodes; leaves
// t3_ok false (mode 2 unavailable) where a map cannot be encoded
lbm_status setup_t3(lbm_batch* b)
{
    if (b->storage != LBM_F32 && b->storage != LBM_BF16 && b->storage != LBM_F16) return LBM_OK;
    const int es = b->ops->elem_bytes;
    const int win = es == 4 ? lbmk::Tbt3Geom<4>::WIN : lbmk::Tbt3Geom<2>::WIN;
    b->t3_rows = es == 4 ? LBM_BATCH_T3_ROWS4 : LBM_BATCH_T3_ROWS2;
    std::vector<CUtensorMap> maps((size_t)2 * b->count);
    std::vector<lbmk::BatchLatT3> l3((size_t)b->count);
    std::vector<int4> tiles[2];
    for (int i = 0; i < b->count; ++i) {
        const lbmk::LatDesc& L = b->lat[i];
        for (int a = 0; a < 2; ++a) {
            void* base = static_cast<char*>(b->arena[a]) + (size_t)L.off * es;
            if (!lbmh::encode_rows_map(&maps[(size_t)2 * i + a], base, es, L.nx, L.ny, L.pitch, L.plane, 20, win))
                return LBM_OK;
        }
        lbmk::BatchLatT3& q = l3[i];
        q.off = L.off;
        q.plane = L.plane;
        q.nx = L.nx;
        q.ny = L.ny;
        q.pitch = L.pitch;
        q.af = (float)L.a;
        q.bf = (float)L.b;
        q.pad_ = 0;
        for (int y = 0; y < L.ny; y += b->t3_rows)
            for (int x = 0; x < L.nx; x += lbmk::TBT3_OUT) tiles[L.bc ? 1 : 0].push_back(make_int4(i, x, y, 0));
    }
    b->nt3[0] = (int)tiles[0].size();
    b->nt3[1] = (int)tiles[1].size();
    std::vector<int4> all(tiles[0]);
    all.insert(all.end(), tiles[1].begin(), tiles[1].end());
    B_CUDA(b, cudaMalloc((void**)&b->d_lat3, l3.size() * sizeof(lbmk::BatchLatT3)));
    B_CUDA(b, cudaMalloc((void**)&b->d_maps, maps.size() * sizeof(CUtensorMap)));
    B_CUDA(b, cudaMalloc((void**)&b->d_t3, std::max<size_t>(1, all.size()) * sizeof(int4)));
    B_CUDA(b, cudaMemcpy(b->d_lat3, l3.data(), l3.size() * sizeof(lbmk::BatchLatT3), cudaMemcpyHostToDevice));
    B_CUDA(b, cudaMemcpy(b->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    if (!all.empty())
        B_CUDA(b, cudaMemcpy(b->d_t3, all.data(), all.size() * sizeof(int4), cudaMemcpyHostToDevice));
    b->t3_ok = true;
    return LBM_OK;
}

#ifndef LBM_BATCH_F64S_ROWS_FX
#define LBM_BATCH_F64S_ROWS_FX 4     // rows per mode-3 tile on the fixed-point update (single-lattice default)
#endif
#ifndef LBM_BATCH_F64S_ROWS_L1
#define LBM_BATCH_F64S_ROWS_L1 2     // the same on the IEEE sequence of split level 1
#endif

int f64s_rows(int list)
{
    return list < 2 ? LBM_BATCH_F64S_ROWS_FX : LBM_BATCH_F64S_ROWS_L1;
}

// Tile lists of mode 3 for FP64 storage: 128 columns x f64s_rows(list) rows, row bands of a
// lattice one after the other, each lattice in the list of its boundary and node update
// (the fixed-point update where both multipliers allow it, as batch_tile decides per lattice)
lbm_status setup_f64s(lbm_batch* b)
{
    if (b->storage != LBM_F64) return LBM_OK;
    std::vector<int4> tiles[4];
    for (int i = 0; i < b->count; ++i) {
        const lbmk::LatDesc& L = b->lat[i];
        const bool fixed = LBM_BATCH_F64_FIXED && lbmfx::mul_ok(L.a) && lbmfx::mul_ok(L.b);
        const int list = (fixed ? 0 : 2) + (L.bc ? 1 : 0);
        const int rows = f64s_rows(list);
        for (int y = 0; y < L.ny; y += rows)
            for (int x = 0; x < L.nx; x += lbmk::SA_THREADS) tiles[list].push_back(make_int4(i, x, y, 0));
    }
    std::vector<int4> all;
    for (int l = 0; l < 4; ++l) {
        b->nf64s[l] = (int)tiles[l].size();
        all.insert(all.end(), tiles[l].begin(), tiles[l].end());
    }
    B_CUDA(b, cudaMalloc((void**)&b->d_f64s, std::max<size_t>(1, all.size()) * sizeof(int4)));
    if (!all.empty())
        B_CUDA(b, cudaMemcpy(b->d_f64s, all.data(), all.size() * sizeof(int4), cudaMemcpyHostToDevice));
    b->f64s_ok = true;
    return LBM_OK;
}

lbmk::BatchArgs batch_args(const lbm_batch* b, int steps, int parity)
{
    lbmk::BatchArgs A;
    A.lat = b->d_lat;
    A.tile_lat = b->d_tile;
    A.ntiles = b->ntiles;
    A.arenaA = b->arena[0];
    A.arenaB = b->arena[1];
    A.steps = steps;
    A.parity = parity;
    A.bar_count = b->d_bar;
    A.bar_gen = b->d_bar + 1;
    A.err = reinterpret_cast<int*>(b->d_bar + 2);
    A.timeout_ns = b->timeout_ns;
    A.extra_arrivals = b->extra_arrivals;
    return A;
}

// arena swaps of `steps` steps: one per launch (a three-step pass of mode 2 is one launch pair)
int swaps_of(const lbm_batch* b, long long steps)
{
    return (int)((b->mode == 2 ? steps / 3 + steps % 3 : steps) & 1);
}

// enqueue `steps` steps starting from arena `parity` (no graph)
cudaError_t enqueue_steps(lbm_batch* b, int steps, int parity)
{
    if (b->mode == 1) {
        return b->ops->batch_step(batch_args(b, steps, parity), true, b->persistent_grid, b->s);
    }
    if (b->mode == 3) {
        // one launch per non-empty tile list and step
        lbmk::BatchF64Args F;
        F.lat = b->d_lat;
        for (int i = 0; i < steps; ++i) {
            F.src = static_cast<const double*>(b->arena[parity]);
            F.dst = static_cast<double*>(b->arena[parity ^ 1]);
            const int4* t = b->d_f64s;
            for (int l = 0; l < 4; ++l) {
                F.tiles = t;
                F.rows = f64s_rows(l);
                cudaError_t e = lbmh::batch_f64_staged_step(F, l, b->nf64s[l], b->s);
                if (e != cudaSuccess) return e;
                t += b->nf64s[l];
            }
            parity ^= 1;
        }
        return cudaSuccess;
    }
    int i = 0;
    if (b->mode == 2) {
        // three steps per pass: the periodic tiles and the Dirichlet tiles, one launch each
        lbmk::BatchTbtArgs T;
        T.lat = b->d_lat3;
        T.maps = b->d_maps;
        T.arenaA = b->arena[0];
        T.arenaB = b->arena[1];
        T.rows = b->t3_rows;
        T.timeout = reinterpret_cast<int*>(b->d_bar + 2);
        for (; i + 3 <= steps; i += 3) {
            T.parity = parity;
            T.tiles = b->d_t3;
            cudaError_t e = b->ops->batch_tbt3_step(T, false, b->nt3[0], b->s);
            if (e != cudaSuccess) return e;
            T.tiles = b->d_t3 + b->nt3[0];
            e = b->ops->batch_tbt3_step(T, true, b->nt3[1], b->s);
            if (e != cudaSuccess) return e;
            parity ^= 1;
        }
    }
    for (; i < steps; ++i) {
        cudaError_t e = b->ops->batch_step(batch_args(b, 1, parity), false, b->ntiles, b->s);
        if (e != cudaSuccess) return e;
        parity ^= 1;
    }
    return cudaSuccess;
}

lbm_status ensure_graph(lbm_batch* b)
{
    if (b->graph_valid) return LBM_OK;
    cudaGraph_t g = nullptr;
    B_CUDA(b, cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_steps(b, b->graph_steps, 0);
    cudaError_t e2 = cudaStreamEndCapture(b->s, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        b->err = std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
        return LBM_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph = nullptr;
        b->err = std::string("graph instantiate: ") + cudaGetErrorString(e);
        return LBM_ERR_CUDA;
    }
    b->graph_valid = true;
    return LBM_OK;
}

lbm_status run_steps(lbm_batch* b, long long n)
{
    while (n > 0) {
        if (b->cur == 0 && n >= b->graph_steps) {
            lbm_status st = ensure_graph(b);
            if (st != LBM_OK) return st;
            B_CUDA(b, cudaGraphLaunch(b->graph, b->s));
            n -= b->graph_steps;           // an even number of swaps: the state returns to arena 0
            continue;
        }
        const int k = (int)std::min<long long>(n, b->cur == 0 ? (n % b->graph_steps) : 1);
        const int kk = std::max(1, k);
        B_CUDA(b, enqueue_steps(b, kk, b->cur));
        b->cur = (b->cur + swaps_of(b, kk)) & 1;
        n -= kk;
    }
    return LBM_OK;
}

lbmk::NodeArgs lattice_node_args(const lbm_batch* b, int i)
{
    const lbmk::LatDesc& L = b->lat[i];
    const lbm_lattice_desc& D = b->in[i];
    lbmk::NodeArgs A;
    char* base = static_cast<char*>(b->arena[b->cur]) + (size_t)L.off * b->ops->elem_bytes;
    A.S = base;
    A.Sout = base;
    A.w = nullptr;
    A.nx = L.nx;
    A.ny = L.ny;
    A.pitch = L.pitch;
    A.plane = L.plane;
    A.a = L.a;
    A.b = L.b;
    A.cK = D.cK;
    A.cmu = D.cmu;
    A.dt = D.dt;
    A.c = D.dx / D.dt;
    A.R = 0;
    A.X = A.Y = A.T = nullptr;
    A.omega = 2.0;
    const int VI[4] = {1, 0, -1, 0}, VJ[4] = {0, 1, 0, -1};
    for (int d = 0; d < 4; ++d) {
        double gm[25] = {0};
        for (int q = 0; q < 5; ++q) gm[q * 6] = 0.25;
        const double s = 1.0 / (2.0 * A.c);
        gm[0 * 5 + 2] += s * VI[d] * D.cK;  gm[2 * 5 + 0] += s * VI[d] * D.cK;
        gm[0 * 5 + 3] += s * VI[d] * D.cmu; gm[3 * 5 + 0] += s * VI[d] * D.cmu;
        gm[1 * 5 + 4] += s * VI[d] * D.cmu; gm[4 * 5 + 1] += s * VI[d] * D.cmu;
        gm[0 * 5 + 4] += s * VJ[d] * D.cmu; gm[4 * 5 + 0] += s * VJ[d] * D.cmu;
        gm[1 * 5 + 2] += s * VJ[d] * D.cK;  gm[2 * 5 + 1] += s * VJ[d] * D.cK;
        gm[1 * 5 + 3] -= s * VJ[d] * D.cmu; gm[3 * 5 + 1] -= s * VJ[d] * D.cmu;
        inverse5(gm, A.k[d]);
    }
    return A;
}

void node_grid_for(long long n, dim3& grid, dim3& block)
{
    long long nb = (n + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    grid = dim3((unsigned)std::max(1LL, nb));
    block = dim3(256);
}

// time `steps` steps of the current configuration (events on the batch stream), ms per step
lbm_status time_config(lbm_batch* b, int steps, float* ms_per_step)
{
    lbm_status st = build_tiles(b);
    if (st != LBM_OK) return st;
    cudaEvent_t e0, e1;
    B_CUDA(b, cudaEventCreate(&e0));
    B_CUDA(b, cudaEventCreate(&e1));
    st = run_steps(b, 2);
    if (st == LBM_OK) {
        cudaEventRecord(e0, b->s);
        st = run_steps(b, steps);
        cudaEventRecord(e1, b->s);
    }
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBM_OK) return st;
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("tuning timer: ") + cudaGetErrorString(e));
    unsigned int flag = 0;
    B_CUDA(b, cudaMemcpy(&flag, b->d_bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost));
    if (flag) {
        unsigned int z[3] = {0, 0, 0};
        cudaMemcpy(b->d_bar, z, sizeof(z), cudaMemcpyHostToDevice);
        return bfail(b, LBM_ERR_TIMEOUT, "grid barrier timed out while tuning");
    }
    *ms_per_step = ms / steps;
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(int32_t count, const lbm_lattice_desc* lats, int32_t storage, void* stream,
                            lbm_batch** out)
{
    g_batch_create_error.clear();
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (count < 1 || count > 65536 || !lats) {
        g_batch_create_error = "count must be in [1, 65536] and lattices non-NULL";
        return LBM_ERR_ARG;
    }
    const lbmh::KindOps* ops = batch_ops_for(storage);
    if (!ops) {
        g_batch_create_error = "unknown storage format";
        return LBM_ERR_ARG;
    }
    for (int i = 0; i < count; ++i) {
        const lbm_lattice_desc& d = lats[i];
        char msg[160];
        if (d.nx < 2 || d.ny < 2 || d.ny > 65535 || d.nx > (1 << 24) || (d.bc != 0 && d.bc != 1) || d.reserved != 0 ||
            !(d.dx > 0) || !(d.dt > 0) || !(d.cK > 0) || !(d.cmu >= 0)) {
            std::snprintf(msg, sizeof(msg), "lattice %d: invalid size, bc or parameters", i);
            g_batch_create_error = msg;
            return LBM_ERR_ARG;
        }
        if (!(2.0 * std::sqrt(d.cK * d.cK + d.cmu * d.cmu) < d.dx / d.dt)) {
            std::snprintf(msg, sizeof(msg), "lattice %d: CFL-like condition 2 sqrt(cK^2+cmu^2) < dx/dt violated", i);
            g_batch_create_error = msg;
            return LBM_ERR_CFL;
        }
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->count = count;
    b->storage = storage;
    b->ops = ops;
    b->s = static_cast<cudaStream_t>(stream);
    if (!b->s) {
        // stream capture is not possible on the legacy stream; a blocking stream keeps its ordering
        if (cudaStreamCreate(&b->s) != cudaSuccess) {
            delete b;
            g_batch_create_error = "could not create a stream";
            return LBM_ERR_CUDA;
        }
        b->own_stream = true;
    }
    b->in.assign(lats, lats + count);
    b->lat.resize(count);
    b->cls.resize(count);
    long long off = 0;
    for (int i = 0; i < count; ++i) {
        const lbm_lattice_desc& d = lats[i];
        lbmk::LatDesc& L = b->lat[i];
        std::memset(&L, 0, sizeof(L));
        L.nx = d.nx;
        L.ny = d.ny;
        L.pitch = (d.nx + 63) / 64 * 64;
        L.plane = (long long)L.pitch * d.ny;
        L.off = off;
        L.bc = d.bc;
        const double c = d.dx / d.dt;
        L.a = d.cK / c;
        L.b = d.cmu / c;
        off += 20 * L.plane;
        b->nodes += (long long)d.nx * d.ny;
        b->cls[i] = size_class((d.nx + ops->batch_vec - 1) / ops->batch_vec);
    }
    b->total_elems = off;
    const size_t bytes = (size_t)off * ops->elem_bytes;
    cudaError_t e = cudaMalloc(&b->arena[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->arena[1], bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_lat, (size_t)count * sizeof(lbmk::LatDesc));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_bar, 4 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->scratch, (kRed + 8) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->arena[0], 0, bytes, b->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->arena[1], 0, bytes, b->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, 4 * sizeof(unsigned int), b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    int occ = 0, sms = 0, dev = 0;
    if (e == cudaSuccess) e = ops->batch_occupancy(&occ);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        g_batch_create_error = std::string("device allocation or query failed: ") + cudaGetErrorString(e);
        lbm_batch_destroy(b);
        // a refused allocation is not sticky; clear the runtime's last error so that later launch
        // checks do not report it as theirs
        if (e == cudaErrorMemoryAllocation) cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
    }
    b->persistent_grid = std::max(1, occ) * sms;
    if (build_tiles(b) != LBM_OK || setup_t3(b) != LBM_OK || setup_f64s(b) != LBM_OK) {
        g_batch_create_error = b->err;
        lbm_batch_destroy(b);
        return LBM_ERR_CUDA;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b)
{
    if (!b) return LBM_OK;
    cudaStreamSynchronize(b->s);
    drop_graph(b);
    cudaFree(b->arena[0]);
    cudaFree(b->arena[1]);
    cudaFree(b->d_lat);
    cudaFree(b->d_tile);
    cudaFree(b->d_bar);
    cudaFree(b->scratch);
    cudaFree(b->d_lat3);
    cudaFree(b->d_maps);
    cudaFree(b->d_t3);
    cudaFree(b->d_f64s);
    if (b->own_stream) cudaStreamDestroy(b->s);
    delete b;
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b)
{
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

lbm_status lbm_batch_set_mode(lbm_batch* b, int32_t mode, int32_t graph_steps)
{
    if (!b) return LBM_ERR_ARG;
    if (b->sticky) return LBM_ERR_CUDA;
    // a graph must return the state to arena 0, an even number of arena swaps: graph_steps even
    // (in mode 2, 3q + r steps swap q + r times, even exactly when 3q + r is)
    if (mode < 0 || mode > 3 || graph_steps < 2 || graph_steps > 10000 || (graph_steps & 1))
        return bfail(b, LBM_ERR_ARG, "mode must be 0, 1, 2 or 3 and graph_steps even in [2, 10000]");
    if (mode == 2 && !b->t3_ok)
        return bfail(b, LBM_ERR_ARG, "mode 2 needs FP32, BF16 or FP16 storage");
    if (mode == 3 && !b->f64s_ok)
        return bfail(b, LBM_ERR_ARG, "mode 3 needs FP64 storage");
    b->mode = mode;
    b->graph_steps = graph_steps;
    drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_set_barrier(lbm_batch* b, double timeout_s, int32_t extra_arrivals)
{
    if (!b) return LBM_ERR_ARG;
    if (!(timeout_s > 0.0) || timeout_s > 600.0 || extra_arrivals < 0)
        return bfail(b, LBM_ERR_ARG, "timeout must be in (0, 600] s and extra_arrivals >= 0");
    b->timeout_ns = (unsigned long long)(timeout_s * 1e9);
    b->extra_arrivals = (unsigned int)extra_arrivals;
    drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_init(lbm_batch* b, int32_t index, const double* U0, const double* dU0dx, const double* dU0dy,
                          int32_t on_device)
{
    if (!b) return LBM_ERR_ARG;
    if (b->sticky) return LBM_ERR_CUDA;
    if (index < 0 || index >= b->count || !U0 || !dU0dx || !dU0dy)
        return bfail(b, LBM_ERR_ARG, "index out of range or input missing");
    const size_t n = (size_t)b->lat[index].nx * b->lat[index].ny;
    const double* src[3] = {U0, dU0dx, dU0dy};
    const double* dev[3] = {U0, dU0dx, dU0dy};
    double* stage = nullptr;
    if (!on_device) {
        B_CUDA(b, cudaMallocAsync((void**)&stage, 15 * n * sizeof(double), b->s));
        for (int q = 0; q < 3; ++q) {
            cudaError_t e = cudaMemcpyAsync(stage + q * 5 * n, src[q], 5 * n * sizeof(double),
                                            cudaMemcpyHostToDevice, b->s);
            if (e != cudaSuccess) {
                cudaFreeAsync(stage, b->s);
                return bfail(b, LBM_ERR_CUDA, std::string("init copy: ") + cudaGetErrorString(e));
            }
            dev[q] = stage + q * 5 * n;
        }
    }
    dim3 grid, block;
    node_grid_for((long long)n, grid, block);
    cudaError_t e = b->ops->init(lattice_node_args(b, index), dev[0], dev[1], dev[2], nullptr, nullptr, grid, block, b->s);
    if (stage) cudaFreeAsync(stage, b->s);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch init: ") + cudaGetErrorString(e));
    if (!on_device) B_CUDA(b, cudaStreamSynchronize(b->s));
    b->initialised = true;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t n)
{
    if (!b) return LBM_ERR_ARG;
    if (b->sticky) return LBM_ERR_CUDA;
    if (n < 0) return bfail(b, LBM_ERR_ARG, "n < 0");
    return run_steps(b, n);
}

lbm_status lbm_batch_synchronize(lbm_batch* b)
{
    if (!b) return LBM_ERR_ARG;
    if (b->sticky) return LBM_ERR_CUDA;
    B_CUDA(b, cudaStreamSynchronize(b->s));
    unsigned int flag = 0;
    B_CUDA(b, cudaMemcpy(&flag, b->d_bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost));
    if (flag) {
        unsigned int z[3] = {0, 0, 0};
        B_CUDA(b, cudaMemcpy(b->d_bar, z, sizeof(z), cudaMemcpyHostToDevice));
        return bfail(b, LBM_ERR_TIMEOUT, "a grid barrier wait ran out; populations are undefined");
    }
    return LBM_OK;
}

lbm_status lbm_batch_moments(lbm_batch* b, int32_t index, double* out, int32_t on_device)
{
    if (!b) return LBM_ERR_ARG;
    if (b->sticky) return LBM_ERR_CUDA;
    if (index < 0 || index >= b->count || !out) return bfail(b, LBM_ERR_ARG, "index out of range or out NULL");
    const size_t n = (size_t)b->lat[index].nx * b->lat[index].ny;
    double* dst = out;
    if (!on_device) B_CUDA(b, cudaMallocAsync((void**)&dst, 10 * n * sizeof(double), b->s));
    dim3 grid, block;
    node_grid_for((long long)n, grid, block);
    cudaError_t e = b->ops->moments(lattice_node_args(b, index), dst, grid, block, b->s);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(out, dst, 10 * n * sizeof(double), cudaMemcpyDeviceToHost, b->s);
    if (!on_device) cudaFreeAsync(dst, b->s);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch moments: ") + cudaGetErrorString(e));
    if (!on_device) B_CUDA(b, cudaStreamSynchronize(b->s));
    return LBM_OK;
}

lbm_status lbm_batch_energy(lbm_batch* b, int32_t index, double* out)
{
    if (!b) return LBM_ERR_ARG;
    if (b->sticky) return LBM_ERR_CUDA;
    if (index < 0 || index >= b->count || !out) return bfail(b, LBM_ERR_ARG, "index out of range or out NULL");
    B_CUDA(b, b->ops->energy(lattice_node_args(b, index), b->scratch, dim3(kRed), dim3(256), b->s));
    B_CUDA(b, lbmh::finish_sum1(b->scratch, kRed, b->scratch + kRed, b->s));
    B_CUDA(b, cudaMemcpyAsync(out, b->scratch + kRed, sizeof(double), cudaMemcpyDeviceToHost, b->s));
    B_CUDA(b, cudaStreamSynchronize(b->s));
    return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch* b, int32_t index, int64_t* nodes, int64_t* state_bytes, int32_t* ntiles,
                          int32_t* tile_width)
{
    if (!b) return LBM_ERR_ARG;
    if (nodes) *nodes = b->nodes;
    if (state_bytes) *state_bytes = 2 * b->total_elems * b->ops->elem_bytes;
    if (ntiles) *ntiles = b->ntiles;
    if (tile_width) {
        if (index < 0 || index >= b->count) return LBM_ERR_ARG;
        *tile_width = b->lat[index].tpr * b->ops->batch_vec;
    }
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch* b, const char* cache_path)
{
    if (!b) return LBM_ERR_ARG;
    if (b->sticky) return LBM_ERR_CUDA;
    if (b->initialised) return bfail(b, LBM_ERR_STATE, "tune before lbm_batch_init (tuning steps the state)");
    int dev = 0;
    cudaDeviceProp prop;
    B_CUDA(b, cudaGetDevice(&dev));
    B_CUDA(b, cudaGetDeviceProperties(&prop, dev));
    std::string gpu = prop.name;
    for (char& ch : gpu)
        if (ch == ' ' || ch == '|') ch = '_';
    const std::string key = gpu + "|" + storage_name(b->storage) + "|";
    // classes present, largest node share first
    std::map<int, long long> share;
    for (int i = 0; i < b->count; ++i) share[b->cls[i]] += (long long)b->lat[i].nx * b->lat[i].ny;
    std::vector<std::pair<long long, int>> order;
    for (auto& kv : share) order.push_back({-kv.second, kv.first});
    std::sort(order.begin(), order.end());
    // cached results
    std::map<std::string, int> cache;
    if (cache_path) {
        std::ifstream f(cache_path);
        std::string line;
        while (std::getline(f, line)) {
            const size_t p = line.rfind('|');
            if (p == std::string::npos) continue;
            cache[line.substr(0, p)] = std::atoi(line.c_str() + p + 1);
        }
    }
    std::vector<std::string> fresh;
    bool all_cached = cache.count(key + "mode") > 0;
    for (auto& o : order) {
        const std::string k = key + "class" + std::to_string(o.second);
        if (cache.count(k)) b->tpr_of_class[o.second] = cache[k];
        else all_cached = false;
    }
    if (all_cached) {
        b->mode = cache[key + "mode"];
        if (b->mode < 0 || b->mode > 3 || (b->mode == 2 && !b->t3_ok) || (b->mode == 3 && !b->f64s_ok)) b->mode = 0;
        return build_tiles(b);
    }
    const int V = b->ops->batch_vec;
    const int steps = 6;
    const int saved_graph = b->graph_steps;
    b->graph_steps = 2;
    const std::map<int, int> start = b->tpr_of_class;
    std::map<int, int> tpr_mode[4];
    float mode_ms[4] = {1e30f, 1e30f, 1e30f, 1e30f};
    for (int mode = 0; mode < 2; ++mode) {
        b->mode = mode;
        b->tpr_of_class = start;
        bool failed = false;
        for (auto& o : order) {
            const int c = o.second;
            if (cache.count(key + "class" + std::to_string(c))) continue;
            int maxc = 0;
            for (int i = 0; i < b->count; ++i)
                if (b->cls[i] == c) maxc = std::max(maxc, (b->lat[i].nx + V - 1) / V);
            const int hi = std::min(kMaxTpr, std::max(kMinTpr, next_pow2(maxc)));
            int best_t = std::min(64, hi);
            float best = 1e30f;
            for (int t = kMinTpr; t <= hi && !failed; t <<= 1) {
                b->tpr_of_class[c] = t;
                float ms = 0.f;
                lbm_status st = time_config(b, steps, &ms);
                if (st == LBM_ERR_TIMEOUT || (st == LBM_ERR_CUDA && !b->sticky && mode == 1)) {
                    failed = true;     // this launch mode is not usable here
                    break;
                }
                if (st != LBM_OK) {
                    b->graph_steps = saved_graph;
                    return st;
                }
                if (ms < best) {
                    best = ms;
                    best_t = t;
                }
            }
            b->tpr_of_class[c] = best_t;
        }
        if (failed) continue;
        // the modes are compared at the caller's graph length (the launch overhead per step
        // depends on it), best of two runs of two graphs each
        b->graph_steps = saved_graph;
        for (int rep = 0; rep < 2; ++rep) {
            float ms = 0.f;
            lbm_status st = time_config(b, 2 * saved_graph, &ms);
            if (st != LBM_OK) {
                if (mode == 1 && !b->sticky) break;
                return st;
            }
            mode_ms[mode] = std::min(mode_ms[mode], ms);
        }
        b->graph_steps = 2;
        tpr_mode[mode] = b->tpr_of_class;
    }
    // mode 2 (three steps per pass, FP32 / 16 bits) and mode 3 (FP64 on staged rows) run over
    // fixed tiles; mode 2's remainder steps use mode 0's widths
    for (int m = 2; m < 4; ++m) {
        if (!(m == 2 ? b->t3_ok : b->f64s_ok)) continue;
        b->mode = m;
        b->tpr_of_class = tpr_mode[0];
        b->graph_steps = saved_graph;
        for (int rep = 0; rep < 2; ++rep) {
            float ms = 0.f;
            lbm_status st = time_config(b, 2 * saved_graph, &ms);
            if (st != LBM_OK) {
                b->graph_steps = saved_graph;
                return st;
            }
            mode_ms[m] = std::min(mode_ms[m], ms);
        }
        b->graph_steps = 2;
        tpr_mode[m] = tpr_mode[0];
    }
    int best_mode = 0;
    for (int m = 1; m < 4; ++m)
        if (mode_ms[m] < mode_ms[best_mode]) best_mode = m;
    b->tpr_of_class = tpr_mode[best_mode];
    b->graph_steps = saved_graph;
    b->mode = best_mode;
    lbm_status st = build_tiles(b);
    if (st != LBM_OK) return st;
    // the timing runs stepped the (zero) state; start again from zeros
    const size_t bytes = (size_t)b->total_elems * b->ops->elem_bytes;
    B_CUDA(b, cudaMemsetAsync(b->arena[0], 0, bytes, b->s));
    B_CUDA(b, cudaMemsetAsync(b->arena[1], 0, bytes, b->s));
    B_CUDA(b, cudaStreamSynchronize(b->s));
    b->cur = 0;
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        for (auto& o : order) {
            const std::string k = key + "class" + std::to_string(o.second);
            if (!cache.count(k)) f << k << "|" << b->tpr_of_class[o.second] << "\n";
        }
        if (!cache.count(key + "mode")) f << key << "mode|" << b->mode << "\n";
    }
    return LBM_OK;
}

}  // extern "C"
