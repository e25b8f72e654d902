/*
 * lbm.h -- C ABI of the GB300 vectorial lattice Boltzmann library for 2D linear
 * elastodynamics (D2Q4^5 scheme of Boolakee, Geier and De Lorenzis, arXiv 2408.01081).
 *
 * Problem (Sec. 2): d2u/dt2 = div(sigma) + b on a rectangle, periodic on both
 * axes or u = u_D on all four edges, with u(0) = u0 and du/dt(0) = v0.  The
 * library advances the first-order system of Eq. system, U = [v_x, v_y, j_s,
 * j_d, j_xy], with 4 vector populations per node (Eq. index_vel).  All
 * quantities are dimensionless (Sec. 2.3): lattice spacing dx, time step dt,
 * lattice speed c = dx/dt, wave speeds cK and cmu.
 *
 * Conventions shared by every call
 *   - Field arrays are dense, field-major and row-major: [field][y][x], x fastest,
 *     FP64.  Node (k, l) sits at ((k + 1/2) dx, (l + 1/2) dx).
 *   - Population arrays are [d][k][y][x] with d = 0..3 the velocities
 *     (1,0), (0,1), (-1,0), (0,-1) and k = 0..4 the components of U.
 *   - `on_device` = 1: the pointer is CUDA device memory (e.g. a torch tensor's
 *     data_ptr); 0: host memory.  Host pointers are copied synchronously with
 *     respect to the context's stream; the caller keeps ownership of every buffer
 *     it passes and may free it when the call returns.  Pinned host memory
 *     (cudaHostAlloc / cudaHostRegister, e.g. a pinned torch tensor) is read and
 *     written by the kernels in place, without a device copy; pageable host memory
 *     goes through a temporary device buffer.
 *   - The context owns all device memory it allocates (created by lbm_create,
 *     released by lbm_destroy).  Work is enqueued on the stream given at creation.
 *   - No call aborts.  Errors return a status; LBM_ERR_CUDA is sticky: every later
 *     call on the same context returns it.  lbm_last_error() gives a message.
 *   - Calls on one context are not thread-safe; distinct contexts are independent.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,       /* invalid argument: NULL pointer, size, enum, table too short  */
    LBM_ERR_CFL = 2,       /* 2 sqrt(cK^2 + cmu^2) >= c: some g_ij is not SPD (Eq. stab_cond) */
    LBM_ERR_OOM = 3,       /* a device allocation was refused (not sticky: the context and
                              the device stay usable)                                       */
    LBM_ERR_CUDA = 4,      /* a CUDA runtime call or launch failed (sticky)                 */
    LBM_ERR_UNSTABLE = 5,  /* lbm_check_finite found a non-finite value, or the energy
                              monitor of lbm_set_energy_check found growth beyond its bound */
    LBM_ERR_TIMEOUT = 6,   /* a bounded device-side wait ran out                            */
    LBM_ERR_STATE = 7      /* call order: stepping before lbm_init, data for step m missing */
} lbm_status;

typedef enum { LBM_PERIODIC = 0, LBM_DIRICHLET = 1 } lbm_bc;

/* Storage of the state.  LBM_F64 stores in FP64 and computes to FP64 accuracy (by
 * default the node update in exact fixed point with one binary64 rounding per output,
 * lbm_set_fp64_split); LBM_F32 / BF16 /
 * F16 store the populations in that format and compute in FP32.  LBM_MS_BF16 /
 * LBM_MS_F16 store per node the zeroth moment U (FP32) and the 15 deviations of
 * the other moments from their local-equilibrium values (Eq. cond_eq) in BF16 /
 * FP16, scaled by a power of two chosen at lbm_init / lbm_set_populations
 * (50 bytes per node instead of 80 for 16-bit populations).  LBM_MS_BFP stores
 * the same 15 deviations in 16-bit words as block floating point: the three
 * deviations of one component of one node share a 3-bit exponent (one bit in
 * each word) and keep 15-bit mantissas, about 8 times finer than FP16 for the
 * largest of the three.  Its range holds deviations at least 8 times the largest
 * one at initialisation; a block beyond it is clamped and lbm_check_finite then
 * returns LBM_ERR_UNSTABLE.  In every reduced format the initialisation, the
 * Dirichlet reconstruction and all reductions stay in FP64.  Batches accept
 * formats 0..3. */
typedef enum {
    LBM_F64 = 0, LBM_F32 = 1, LBM_BF16 = 2, LBM_F16 = 3, LBM_MS_BF16 = 4, LBM_MS_F16 = 5, LBM_MS_BFP = 6
} lbm_storage;

typedef struct {
    int32_t nx, ny;              /* nodes per row / number of rows, each >= 2            */
    int32_t bc;                  /* lbm_bc                                               */
    int32_t storage;             /* lbm_storage                                          */
    double dx, dt;               /* lattice spacing and time step, > 0 (Sec. 3.1)        */
    double cK, cmu;              /* dimensionless wave speeds c~_K > 0, c~_mu >= 0       */
    int32_t track_displacement;  /* 1: keep u* and update it every step (Eq. trapezoidal) */
    int32_t reserved;            /* must be 0                                            */
    void* stream;                /* cudaStream_t for all work; NULL = legacy stream      */
} lbm_params;

/* Create a context: validates the parameters (LBM_ERR_ARG), the CFL-like
 * condition 2 sqrt(cK^2 + cmu^2) < dx/dt (Eq. stab_cond; LBM_ERR_CFL) and
 * allocates two population buffers (plus u* when tracked).  No kernel runs.
 * On failure *out is set to NULL and nothing is leaked. */
lbm_status lbm_create(const lbm_params* p, lbm_ctx** out);

/* Second-order initialisation, Eq. ic_second, evaluated per node in FP64.
 *   U0, dU0dx, dU0dy : [5][ny][nx] initial U (Eq. ic_vector) and its x / y derivatives
 *   B0               : [2][ny][nx] body load b at t = 0, or NULL for b = 0
 *   u0               : [2][ny][nx] initial displacement, or NULL for 0 (only read
 *                      when displacement tracking is on; u^num(0) = u0, Eq. trapezoidal)
 * Resets the step counter to m = 0 (t = 0). */
lbm_status lbm_init(lbm_ctx* ctx, const double* U0, const double* dU0dx, const double* dU0dy,
                    const double* B0, const double* u0, int32_t on_device);

/* Steps per pass over memory: 1, 2 or 3 (3 is the default for every format but
 * LBM_F64, whose step is bound by arithmetic, not memory).  With 2 lbm_step advances
 * pairs of steps with one kernel that keeps the intermediate state on chip (halving
 * the memory traffic per step), with 3 triples, whenever the lattice stores FP32 / BF16 / FP16
 * populations (or moment-space deviations, with staged rows: lbm_set_staging),
 * omega = 2, there is no body load and no displacement tracking, and the
 * boundary is periodic or homogeneous Dirichlet; otherwise, and for an odd last
 * step, one kernel per step runs.  FP32 results are bit-identical to single
 * steps; 16-bit and moment-space results skip one rounding per pair and are more
 * accurate.  Three steps per kernel need staged rows (lbm_set_staging 1; with 0 pairs
 * run instead); a remainder of one or two steps runs as a single step or a pair.
 * rows_per_block sets the rows each thread block streams through (0 keeps the
 * format's default: 12 for LBM_F32, 64 for the other reduced formats; for the
 * staged LBM_F64 step of lbm_set_staging 4 at split level 12 and 2 at level 1).
 * steps_per_pass = 1 always uses one kernel per step. */
lbm_status lbm_set_step_fusion(lbm_ctx* ctx, int32_t steps_per_pass, int32_t rows_per_block);

/* How the multi-step kernels of lbm_set_step_fusion and the LBM_F64 step at split
 * level 1 read their input (no counterpart in the paper; results are identical
 * either way).  1 (the default): each multi-step block's input rows are copied into
 * a ring of shared-memory stages by tensor copies (TMA) issued by one producer warp,
 * as far ahead as the ring allows; each thread of the FP64 step copies the 20
 * populations its node pulls into shared memory by asynchronous copies, one row
 * ahead of the row it computes.  0: each thread loads into registers (the two-step
 * kernel prefetches the next row there).  A bounded wait of the staged
 * kernel that runs out (about 2 s) makes the next lbm_synchronize return
 * LBM_ERR_TIMEOUT.  Mode 2 is a test hook: staged, but the producer withholds one
 * input row of every block, so that the compute warps' waits run out and the
 * bounded-wait path is exercised (the state is then undefined).  Other modes
 * return LBM_ERR_ARG. */
lbm_status lbm_set_staging(lbm_ctx* ctx, int32_t mode);

/* FP64 arithmetic split (LBM_F64 storage only; no counterpart in the paper, whose
 * scheme this does not change).  The FP64 step needs 35 additions and 12 fused
 * multiply-adds per node and GB300 issues FP64 operations at 2 per clock per SM,
 * so the step is bound by the FP64 pipe.  At level > 0 a set of the additions is
 * computed on the integer pipes, in parallel with the FP64 pipe.  Levels 1..7
 * compute them exactly (IEEE 754 binary64, round to nearest even): results are
 * bit-identical to level 0 (level 1: the 10 pair sums and the 5 sums U, the
 * fastest of them).  Levels 8..11 round them faithfully, within (1/2 + 2^-9) ulp
 * of the exact sum, with fewer integer instructions: the 15 sums of level 1, plus
 * 1, 2 or 5 of the f*_(-1,0) subtractions; results stay within FP64 accuracy of
 * level 0 but are not bit-identical, and the rounding is biased (half up, no sticky
 * bit): over 10^5 steps the discrete energy drifts by about 3e-12 instead of 4e-16.
 * Lanes whose operands leave the integer path (subnormal, infinite or NaN results)
 * recompute on the FP64 pipe.  Level 12 (the default where it applies) computes the
 * whole node update (Eqs. cond_eq, feq, collision) in exact 64-bit fixed-point
 * arithmetic on the integer pipes: each input as an integer multiple of
 * rho = 2^-57 times the power of two just above the node's largest input (exact
 * within 2^5 of it), the sums exactly, the seven products by cK / c and cmu / c
 * rounded to a multiple of rho, and one round-to-nearest-even conversion to
 * binary64 per output.  Every output is then within half an ulp plus 10 rho of the
 * exact update of its inputs, a tighter bound than the FP64 operation sequence's,
 * but the bits differ from level 0.  The state stays binary64; the step is bound by
 * memory instead of the FP64 pipe.  Nodes whose largest input is below about
 * 2^-964, at or above about 2^1019, or not finite run the level-1 sequence instead
 * (the choice depends on the node's own inputs only).  Level 12 needs cK / c and
 * cmu / c in [2^-60, 1/2) (cmu may be 0); otherwise it returns LBM_ERR_ARG and
 * level 1 is the default.  Level 0 runs every operation on the FP64 pipe.  Levels
 * 1..11 apply to steps without body load, level 12 also to steps with one (U of the
 * two velocity components gains dt/2 b, rounded once in FP64, as another input of the
 * exact update); all need omega = 2, and other steps use the FP64 pipe only.  A
 * level outside [0, 12] returns LBM_ERR_ARG. */
lbm_status lbm_set_fp64_split(lbm_ctx* ctx, int32_t level);

/* Relaxation rate of the BGK collision (Eq. collision); the paper's scheme is
 * omega = 2 (the default), the only value with second-order consistency
 * (Sec. 4.1).  Other values give a first-order, dissipative control scheme whose
 * forcing weight is W_ij = 1/8 (the value that adds dt B to the zeroth moment
 * per step).  omega in (0, 1) or (1, 2]; omega = 1 is rejected (LBM_ERR_ARG)
 * because the pre-collision populations cannot be recovered from f^eq. */
lbm_status lbm_set_relaxation(lbm_ctx* ctx, double omega);

/* Body load as a separable sum (the library copies the tables):
 *   b_c(x_k, y_l, t_m) = sum_{r<R} X[r][k] * Y[r][l] * T[m][c][r],   c = 0 (b_x), 1 (b_y)
 * X: [R][nx], Y: [R][ny], T: [nt][2][R]; m = 0 .. nt-1 indexes t = m dt.
 * 1 <= R <= 16.  R = 0 (pointers ignored) removes the body load.  Stepping to a
 * time whose row is missing returns LBM_ERR_STATE.  (Eq. lbe uses B at time t.) */
lbm_status lbm_set_forcing(lbm_ctx* ctx, int32_t R, const double* X, const double* Y,
                           const double* T, int64_t nt, int32_t on_device);

/* Dirichlet data (only for LBM_DIRICHLET): d/dt u_D at the wall midpoints x_b at
 * time t_m + dt/2 for the step m -> m+1 (Eq. bc_ansatz with q = 1/2, Eq. bc_q).
 * g: [nt][2][2(nx+ny)], the last axis ordered [left wall rows 0..ny-1 | right wall
 * rows | bottom wall columns 0..nx-1 | top wall columns].  g = NULL (nt ignored)
 * selects homogeneous data u_D = const.  Stepping past row nt-1 returns LBM_ERR_STATE. */
lbm_status lbm_set_dirichlet(lbm_ctx* ctx, const double* g, int64_t nt, int32_t on_device);

/* Dirichlet data given as a separable sum, expanded on the device into the
 * per-step table of lbm_set_dirichlet (which it replaces):
 *   g_c(x_b, t_m + dt/2) = sum_{r<R} X(x_b)[r] * Y(y_b)[r] * T[m][c][r]
 * with X evaluated at the node columns Xn [R][nx] (bottom and top walls) and at the
 * two side walls Xw [R][2] (x = 0, x = nx dx), Y at the node rows Yn [R][ny] (left and
 * right walls) and at Yw [R][2] (y = 0, y = ny dx); T: [nt][2][R], 1 <= R <= 16.
 * Device memory of nt * 2 * 2(nx+ny) doubles is allocated for the expanded table. */
lbm_status lbm_set_dirichlet_separable(lbm_ctx* ctx, int32_t R, const double* Xn, const double* Xw, const double* Yn,
                                       const double* Yw, const double* T, int64_t nt, int32_t on_device);

/* Advance n >= 0 time steps (Sec. 3.6: collision, streaming, boundary rule,
 * displacement update), asynchronously on the context's stream. */
lbm_status lbm_step(lbm_ctx* ctx, int64_t n);

/* The ten output fields at the current time t = m dt, FP64, [10][ny][nx]:
 *   v_x, v_y, j_s, j_d, j_xy  (U^num, Eq. cond_eq),
 *   u_x, u_y                  (u^num = u* + dt/2 v^num; zeros when not tracked),
 *   sigma_xx, sigma_yy, sigma_xy  (Eq. sigma_num with V = 1).
 * With a host pointer the call waits for the stream. */
lbm_status lbm_moments(lbm_ctx* ctx, double* out, int32_t on_device);

/* Weighted grid norm squared ||f||_P^2 = sum_x sum_ij f_ij^T k_ij f_ij of the
 * pre-collision populations at the current time, k_ij = g_ij^{-1}
 * (Definition grid_norm, Eq. def_symmetrizer), reduced in FP64.  Writes one
 * double to host memory *out; waits for the stream. */
lbm_status lbm_energy(lbm_ctx* ctx, double* out);

/* Error sums against a caller-supplied exact field set, FP64 reductions:
 *   exact: [10][ny][nx] in the layout of lbm_moments (on_device as given)
 *   out (host): [3][10] = per field sum (num - exact)^2, sum exact^2, max |num - exact|.
 * Waits for the stream.  (Error norms of Sec. 6.1.) */
lbm_status lbm_error_sums(lbm_ctx* ctx, const double* exact, int32_t on_device, double* out);

/* Pre-collision populations f(x, t) at the current time, FP64 [4][5][ny][nx],
 * and the displacement helper u*(t) [2][ny][nx] (NULL to skip). */
lbm_status lbm_get_populations(lbm_ctx* ctx, double* f, double* ustar, int32_t on_device);

/* Replace the state: pre-collision populations f at step m (t = m dt) and u*(t)
 * (NULL = zeros).  Values are rounded to the storage precision. */
lbm_status lbm_set_populations(lbm_ctx* ctx, const double* f, const double* ustar, int64_t m,
                               int32_t on_device);

/* LBM_ERR_UNSTABLE if any stored population is NaN or infinite, or (LBM_MS_BFP) if a
 * block of deviations was clamped since the last call; else LBM_OK (waits). */
lbm_status lbm_check_finite(lbm_ctx* ctx);

/* Current step counter m (t = m dt). */
lbm_status lbm_time_step(const lbm_ctx* ctx, int64_t* m);

/* Energy monitor (failure detection; Sec. 6.2 takes growth of ||f||_P, Definition
 * grid_norm, as the sign of instability).  With every > 0, lbm_step evaluates the
 * discrete energy ||f||_P^2 on the device after each `every` steps (counted from this
 * call) and compares it with growth times its value at this call; a larger or
 * non-finite energy sets a device flag that the next lbm_synchronize reports as
 * LBM_ERR_UNSTABLE (and clears).  Nothing waits on the host: the check is two
 * small kernels on the context's stream.  Without body load or wall data the energy
 * is conserved up to the storage format's rounding (FP64: 4e-16 relative over 10^5
 * steps on 512 x 256; the reduced formats round the state every pass), so a growth
 * just above 1 plus that drift detects an instability; with data the energy may grow
 * legitimately and growth is the caller's bound.  The steps run
 * in chunks that end where a check is due, which changes how steps group into the
 * multi-step kernels of lbm_set_step_fusion (FP32 and FP64 results are unchanged;
 * 16-bit formats round once per pass, so choose every as a multiple of 3 there).
 * every = 0 turns it off.  Errors: LBM_ERR_ARG for every < 0 or a growth that is not
 * positive and finite; LBM_ERR_STATE before lbm_init. */
lbm_status lbm_set_energy_check(lbm_ctx* ctx, int32_t every, double growth);

/* Wait until all work enqueued by this context has finished; LBM_ERR_TIMEOUT if a
 * bounded device-side wait of the staged two-step kernel ran out since the last call,
 * else LBM_ERR_UNSTABLE if the energy monitor (lbm_set_energy_check) found the energy
 * above its bound since the last call. */
lbm_status lbm_synchronize(lbm_ctx* ctx);

/* Release all device memory of the context; NULL is accepted. */
lbm_status lbm_destroy(lbm_ctx* ctx);

/* Message describing the last error on ctx (never NULL; "" when none).  With
 * ctx = NULL: the last error of a failed lbm_create or lbm_energy_noalloc in
 * this thread. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Raw storage-format state for bit-exact checkpoints: bytes needed, copy out, copy in. */
lbm_status lbm_state_bytes(const lbm_ctx* ctx, int64_t* nbytes);
lbm_status lbm_save_state(lbm_ctx* ctx, void* dst, int32_t on_device);
lbm_status lbm_load_state(lbm_ctx* ctx, const void* src, int64_t m, int32_t on_device);

/* ------------------------------------------------------------------------
 * Row slabs: one lattice split across devices or processes (no counterpart in
 * the paper; the step itself is unchanged).  In the pull form of Eq. streaming
 * the only values that cross a horizontal cut are the populations moving along
 * y: a node of row y pulls f*_(0,1) from row y-1 and f*_(0,-1) from row y+1.
 * A slab therefore keeps one halo row on each side that has a neighbour slab,
 * and before every step receives 5 values per column from each neighbour:
 *   lbm_halo_pack    writes f*_(0,-1) of its first row (for the slab below) and
 *                    f*_(0,1) of its last row (for the slab above),
 *   (the caller moves the messages: NCCL send/recv, a peer copy, ...)
 *   lbm_halo_unpack  stores the neighbours' messages into the halo rows,
 *   lbm_step(ctx, 1) advances the slab's own rows.
 * A periodic lattice wraps: the slab holding row 0 has the slab holding row
 * ny - 1 below it (a single periodic slab is its own neighbour on both sides).
 * A Dirichlet lattice has no neighbour below row 0 or above row ny - 1.  The
 * own rows of all slabs together follow exactly the trajectory of the whole
 * lattice (same arithmetic per node).
 * Restrictions: population formats (LBM_F64 / F32 / BF16 / F16), no body load,
 * homogeneous Dirichlet data, one kernel per step (lbm_set_step_fusion is
 * ignored).  Every other call works on the slab's own rows: field arrays of
 * lbm_init, lbm_moments, lbm_error_sums, lbm_get/set_populations are
 * [.][rows][nx], and lbm_energy sums the own rows (add the slabs' values for the
 * whole lattice).
 * ------------------------------------------------------------------------ */

/* Rows [y_begin, y_begin + rows) of the lattice described by p (p->ny = the
 * whole lattice's rows), 1 <= rows, 0 <= y_begin, y_begin + rows <= p->ny.  As
 * lbm_create otherwise (the halo rows add at most 2 rows of device memory). */
lbm_status lbm_create_slab(const lbm_params* p, int32_t y_begin, int32_t rows, lbm_ctx** out);

/* Bytes of one halo message: 5 * nx elements of the storage type, [5][nx]
 * (components of U, x fastest); 0 for a context that is not a slab. */
lbm_status lbm_halo_bytes(const lbm_ctx* ctx, int64_t* nbytes);

/* Write the messages for the neighbours into device buffers of lbm_halo_bytes
 * each: to_lower for the slab below, to_upper for the slab above.  A pointer must
 * be given exactly when that neighbour exists (LBM_ERR_ARG otherwise).  Stream
 * ordered on the context's stream; no wait. */
lbm_status lbm_halo_pack(lbm_ctx* ctx, void* to_lower, void* to_upper);

/* Store the neighbours' messages (device buffers: from_lower = the to_upper
 * message of the slab below, from_upper = the to_lower message of the slab
 * above) into the halo rows; same pointer rule and ordering as lbm_halo_pack. */
lbm_status lbm_halo_unpack(lbm_ctx* ctx, const void* from_lower, const void* from_upper);

/* ------------------------------------------------------------------------
 * Batches: many independent lattices of uneven size and material advanced
 * together.  Every lattice of a batch has b = 0; a Dirichlet lattice has
 * homogeneous data (u_D constant in time).  All lattices share one storage
 * format.  The per-node arithmetic is the single-lattice step's, so a batch
 * lattice follows exactly the trajectory it would follow alone.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

typedef struct {
    int32_t nx, ny;      /* >= 2, ny <= 65535 */
    int32_t bc;          /* lbm_bc */
    int32_t reserved;    /* must be 0 */
    double dx, dt, cK, cmu;
} lbm_lattice_desc;

/* Lay out `count` lattices (1 <= count <= 65536) in two device arenas and build
 * the tile work-list with the default tile widths.  Validates every lattice like
 * lbm_create (LBM_ERR_ARG / LBM_ERR_CFL, message names the lattice index).  All
 * populations start at zero. */
lbm_status lbm_batch_create(int32_t count, const lbm_lattice_desc* lattices, int32_t storage, void* stream,
                            lbm_batch** out);

/* Eq. ic_second for lattice `index` (b = 0, no displacement tracking): U0, dU0dx,
 * dU0dy are [5][ny][nx] FP64 as in lbm_init. */
lbm_status lbm_batch_init(lbm_batch* b, int32_t index, const double* U0, const double* dU0dx,
                          const double* dU0dy, int32_t on_device);

/* Choose the tile width of every size class and the launch mode (0, 1, and 2 or 3
 * where the storage allows) by timing them on this GPU, before any lbm_batch_init
 * (tuning steps the zero state; returns
 * LBM_ERR_STATE afterwards).  cache_path (or NULL): a text file of earlier
 * results keyed by GPU name, storage format and size class; found entries are
 * used without timing, new ones are appended. */
lbm_status lbm_batch_tune(lbm_batch* b, const char* cache_path);

/* Launch mode: 0 = one launch per step; 1 = one persistent launch per
 * `graph_steps` steps with a grid barrier between steps (cooperative launch);
 * 2 = three steps per pass (FP32 / BF16 / FP16 storage only, LBM_ERR_ARG otherwise):
 * every lattice is cut into tiles of 112 columns and 12 (FP32) or 64 (16-bit) rows,
 * one block per tile stages the tile's input rows with tensor copies and keeps the
 * two intermediate steps on chip (the single-lattice three-step kernel of
 * lbm_set_step_fusion), one launch for the periodic and one for the Dirichlet
 * tiles per pass; steps beyond a multiple of three run as mode 0;
 * 3 = one step per launch on staged rows (FP64 storage only, LBM_ERR_ARG otherwise):
 * tiles of 128 columns and 4 rows (2 for a lattice on the level-1 sequence), one
 * block per tile copying each node's 20 inputs into shared memory one row ahead
 * (the single-lattice FP64 staged step), one launch per non-empty list of periodic
 * and Dirichlet lattices on the fixed-point update and on the level-1 sequence.
 * FP32 and FP64 results are bit-identical in every mode; 16-bit formats round the
 * state once per pass in mode 2.  graph_steps (even, 2..10000): steps captured in
 * one CUDA graph and replayed. */
lbm_status lbm_batch_set_mode(lbm_batch* b, int32_t mode, int32_t graph_steps);

/* Advance every lattice n >= 0 steps, asynchronously.  Barrier time-outs of the
 * persistent mode are reported by lbm_batch_synchronize. */
lbm_status lbm_batch_step(lbm_batch* b, int64_t n);

/* Wait for the batch's stream; LBM_ERR_TIMEOUT if a grid barrier wait ran out
 * (the flag is cleared; the populations are then undefined until re-initialised). */
lbm_status lbm_batch_synchronize(lbm_batch* b);

/* Ten output fields of lattice `index` ([10][ny][nx], as lbm_moments; u fields 0). */
lbm_status lbm_batch_moments(lbm_batch* b, int32_t index, double* out, int32_t on_device);

/* ||f||_P^2 of lattice `index` (as lbm_energy), written to host *out. */
lbm_status lbm_batch_energy(lbm_batch* b, int32_t index, double* out);

/* Sizes: total nodes, state bytes (both arenas), tiles, and the current tile
 * width in nodes of lattice `index` (any pointer may be NULL). */
lbm_status lbm_batch_info(const lbm_batch* b, int32_t index, int64_t* nodes, int64_t* state_bytes,
                          int32_t* ntiles, int32_t* tile_width);

/* Barrier wait limit of the persistent mode (seconds, > 0; default 2) and a test
 * hook: extra_arrivals > 0 makes every barrier wait for arrivals that never come,
 * so the limit expires and lbm_batch_synchronize reports LBM_ERR_TIMEOUT. */
lbm_status lbm_batch_set_barrier(lbm_batch* b, double timeout_s, int32_t extra_arrivals);

lbm_status lbm_batch_destroy(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

/* ||f||_P^2 of caller-supplied populations, allocating no device memory.
 *
 * Same quantity as lbm_energy, for callers that cannot call cudaMalloc: a host
 * process whose device memory is entirely owned by another allocator (a caching
 * allocator that reserved the pool), or a time-critical loop that cannot afford
 * the implicit device-wide synchronisation of cudaFree.  The paper has no
 * counterpart; this is a library service.
 *   f      : device pointer, pre-collision populations [4][5][ny][nx], FP64 (for
 *            example written by lbm_get_populations with on_device = 1)
 *   nx, ny : lattice size, nx >= 1 and 1 <= ny <= 16384; larger ny is rejected with
 *            LBM_ERR_ARG because the scratch holds one partial sum per row
 *   dx, dt, cK, cmu : as in lbm_params; LBM_ERR_CFL if 2 sqrt(cK^2+cmu^2) >= dx/dt
 *   out    : one double; device memory when out_on_device = 1 (written in stream
 *            order, no wait), else host memory (the call waits for the stream)
 *   stream : cudaStream_t to run on (NULL = legacy stream)
 * The call works on the current device: f, and out when out_on_device = 1, must be
 * device memory of that device (or managed memory), else LBM_ERR_ARG.  The size of
 * the buffer behind f cannot be checked here: it must hold 20 * nx * ny doubles.
 * With out_on_device = 0 the call waits for the stream; on a stream that is being
 * captured that wait is not allowed, and such a call returns LBM_ERR_ARG.
 * Scratch: a static 128 KB array (16384 + 32 doubles) in the library's device
 * image, held by every GPU that loads the library until the process exits.  The
 * first call on each device looks up its device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents; every row
 * partial is rewritten before it is read, so nothing needs clearing.  Calls
 * whose work overlaps on the GPU (different streams, or different host threads
 * on one device) race on the array and must be serialised by the caller. */
lbm_status lbm_energy_noalloc(const double* f, int32_t nx, int32_t ny, double dx, double dt, double cK,
                              double cmu, double* out, int32_t out_on_device, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
