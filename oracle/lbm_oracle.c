/*
 * Plain FP64 CPU oracle of the vectorial lattice Boltzmann scheme (D2Q4^5)
 * for 2D linear elastodynamics (Boolakee, Geier, De Lorenzis, arXiv 2408.01081).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or table with the
 * CUDA library: every formula below is written out again from the paper.
 *
 * Conventions (all quantities dimensionless, Sec. 2.3):
 *   velocity index d = 0..3 is (i,j) = (1,0), (0,1), (-1,0), (0,-1)   (Eq. index_vel)
 *   component  k = 0..4 is U = [v_x, v_y, j_s, j_d, j_xy]             (Eq. system)
 *   populations f[d][k][y][x], x fastest; lattice nx * ny nodes.
 *   c = dx / dt (Sec. 3.1), cK and cmu are the dimensionless wave speeds.
 *
 * The step is written the way the paper states it (Sec. 3.6 summary):
 *   1(a) U^num = sum_ij f_ij + dt/2 B                     (Eq. cond_eq)
 *   1(c) f^eq_ij = 1/4 [U + 2/c (i Phi_x(U) + j Phi_y(U))] (Eq. feq)
 *   1(d) f*_ij = omega f^eq + (1-omega) f + dt (2-omega) W B (Eq. collision)
 *   2(a) f_ij(x + c_ij dt) = f*_ij(x)                      (Eq. streaming)
 *   2(b) periodic wrap (Sec. 3.4.1) or the Dirichlet rule
 *        f_ij(x, t+dt) = D f*_{-i,-j}(x, t) + S_ij(x_b, t+dt/2)  (Eqs. bc_ansatz-bc_q)
 *   2(c) u* <- u* + dt v  (Eq. trapezoidal and step 2(c))
 * Streaming is evaluated per destination node so that the Dirichlet rule,
 * which the paper states per destination, reads literally.
 *
 * No FMA contraction: build with -ffp-contract=off.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t nx, ny;
    int32_t dirichlet;   /* 0: periodic on both axes, 1: Dirichlet on all four edges */
    int32_t pad_;
    double dx, dt;       /* lattice spacing and time step */
    double cK, cmu;      /* dimensionless wave speeds c~_K, c~_mu */
    double omega;        /* BGK relaxation rate; the paper's scheme uses 2 */
    double W;            /* forcing weight W_ij (only used when omega != 2) */
} orc_params;

static const int VI[4] = {1, 0, -1, 0};
static const int VJ[4] = {0, 1, 0, -1};

/* Eq. system: flux Phi_x(U) */
static void phi_x(const double U[5], double cK, double cmu, double out[5])
{
    out[0] = cK * U[2] + cmu * U[3];
    out[1] = cmu * U[4];
    out[2] = cK * U[0];
    out[3] = cmu * U[0];
    out[4] = cmu * U[1];
}

/* Eq. system: flux Phi_y(U) */
static void phi_y(const double U[5], double cK, double cmu, double out[5])
{
    out[0] = cmu * U[4];
    out[1] = cK * U[2] - cmu * U[3];
    out[2] = cK * U[1];
    out[3] = -cmu * U[1];
    out[4] = cmu * U[0];
}

static size_t idx(const orc_params* p, int d, int k, int y, int x)
{
    return (((size_t)d * 5 + (size_t)k) * (size_t)p->ny + (size_t)y) * (size_t)p->nx + (size_t)x;
}

static size_t fld(const orc_params* p, int k, int y, int x)
{
    return ((size_t)k * (size_t)p->ny + (size_t)y) * (size_t)p->nx + (size_t)x;
}

/* Eq. feq: equilibrium population of direction d for the moment vector U. */
void orc_equilibrium(const orc_params* p, const double U[5], int d, double feq[5])
{
    const double c = p->dx / p->dt;
    double px[5], py[5];
    phi_x(U, p->cK, p->cmu, px);
    phi_y(U, p->cK, p->cmu, py);
    for (int k = 0; k < 5; ++k)
        feq[k] = 0.25 * (U[k] + (2.0 / c) * ((double)VI[d] * px[k] + (double)VJ[d] * py[k]));
}

/* Zeroth moment plus forcing, Eq. cond_eq: U^num = sum f + dt/2 B.
 * B holds the two body-load fields b_x, b_y ([2][ny][nx]) or is NULL. */
static void node_moment(const orc_params* p, const double* f, const double* B, int y, int x, double U[5])
{
    for (int k = 0; k < 5; ++k) {
        double s = 0.0;
        for (int d = 0; d < 4; ++d) s += f[idx(p, d, k, y, x)];
        U[k] = s;
    }
    if (B) {
        U[0] += 0.5 * p->dt * B[fld(p, 0, y, x)];
        U[1] += 0.5 * p->dt * B[fld(p, 1, y, x)];
    }
}

/* Post-collision populations at one node, Eq. collision. */
static void node_collide(const orc_params* p, const double* f, const double* B, int y, int x,
                         double fstar[4][5], double U[5])
{
    node_moment(p, f, B, y, x, U);
    for (int d = 0; d < 4; ++d) {
        double feq[5];
        orc_equilibrium(p, U, d, feq);
        for (int k = 0; k < 5; ++k) {
            double force = 0.0;
            if (B && k < 2) force = p->dt * (2.0 - p->omega) * p->W * B[fld(p, k, y, x)];
            fstar[d][k] = p->omega * feq[k] + (1.0 - p->omega) * f[idx(p, d, k, y, x)] + force;
        }
    }
}

/* Eq. bc_s with the wall data g = d/dt u_D at x_b.  The last three rows carry
 * the factor 1/c that the equilibrium difference f^eq_ij - f^eq_{-i,-j} =
 * (i Phi_x + j Phi_y)/c produces (leading-order bounce-back balance, Eq. bb0);
 * the printed matrix omits it. */
static void wall_source(const orc_params* p, int d, double gx, double gy, double S[5])
{
    const double c = p->dx / p->dt;
    const double i = (double)VI[d], j = (double)VJ[d];
    S[0] = 0.5 * gx;
    S[1] = 0.5 * gy;
    S[2] = (p->cK / c) * (i * gx + j * gy);
    S[3] = (p->cmu / c) * (i * gx - j * gy);
    S[4] = (p->cmu / c) * (j * gx + i * gy);
}

/* Index of the wall midpoint x_b that the missing population (d at node x,y)
 * crosses, in the edge array layout [left rows | right rows | bottom cols | top cols]. */
static int wall_index(const orc_params* p, int d, int y, int x)
{
    switch (d) {
    case 0: return y;                              /* (1,0) missing on the left column  */
    case 2: return p->ny + y;                      /* (-1,0) missing on the right column */
    case 1: return 2 * p->ny + x;                  /* (0,1) missing on the bottom row   */
    default: return 2 * p->ny + p->nx + x;         /* (0,-1) missing on the top row     */
    }
}

/*
 * One time step t -> t+dt.
 *   f_in   pre-collision populations at t, [4][5][ny][nx]
 *   f_out  pre-collision populations at t+dt (distinct buffer)
 *   B      body load at t, [2][ny][nx], or NULL for b = 0
 *   g      d/dt u_D at the wall midpoints at t + dt/2, [2][2(nx+ny)], or NULL (homogeneous)
 *   ustar  displacement helper u*, [2][ny][nx], updated in place, or NULL
 *   fstar  scratch [4][5][ny][nx] for the post-collision state
 */
void orc_step(const orc_params* p, const double* f_in, double* f_out, const double* B,
              const double* g, double* ustar, double* fstar)
{
    const int nx = p->nx, ny = p->ny;
    const double dt = p->dt;
    const size_t nwall = 2 * ((size_t)nx + (size_t)ny);

    /* 1. collision at every node (and step 2(c) for the displacement helper) */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double fs[4][5], U[5];
            node_collide(p, f_in, B, y, x, fs, U);
            for (int d = 0; d < 4; ++d)
                for (int k = 0; k < 5; ++k) fstar[idx(p, d, k, y, x)] = fs[d][k];
            if (ustar) {
                ustar[fld(p, 0, y, x)] += dt * U[0];
                ustar[fld(p, 1, y, x)] += dt * U[1];
            }
        }
    }

    /* 2. streaming, evaluated per destination node */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            for (int d = 0; d < 4; ++d) {
                int xs = x - VI[d], ys = y - VJ[d];      /* source node x - c_ij dt */
                int inside = (xs >= 0 && xs < nx && ys >= 0 && ys < ny);
                if (inside || !p->dirichlet) {
                    xs = (xs + nx) % nx;                 /* periodic wrap, Sec. 3.4.1 */
                    ys = (ys + ny) % ny;
                    for (int k = 0; k < 5; ++k)
                        f_out[idx(p, d, k, y, x)] = fstar[idx(p, d, k, ys, xs)];
                } else {
                    /* (i,j) in D_x: Dirichlet rule with q = 1/2, Eq. bc_ansatz */
                    const int dbar = (d + 2) % 4;
                    double gx = 0.0, gy = 0.0, S[5];
                    if (g) {
                        const int w = wall_index(p, d, y, x);
                        gx = g[w];
                        gy = g[nwall + (size_t)w];
                    }
                    wall_source(p, d, gx, gy, S);
                    const double Dm[5] = {-1.0, -1.0, 1.0, 1.0, 1.0};   /* Eq. bc_d */
                    for (int k = 0; k < 5; ++k)
                        f_out[idx(p, d, k, y, x)] = Dm[k] * fstar[idx(p, dbar, k, y, x)] + S[k];
                }
            }
        }
    }
}

/*
 * Second-order initialisation, Eq. ic_second, at every node.
 *   U0, dU0dx, dU0dy : [5][ny][nx] initial moment vector and its derivatives (Eq. ic_vector)
 *   B0               : [2][ny][nx] body load at t = 0, or NULL
 *   f                : output [4][5][ny][nx]
 */
void orc_init(const orc_params* p, const double* U0, const double* dU0dx, const double* dU0dy,
              const double* B0, double* f)
{
    const int nx = p->nx, ny = p->ny;
    const double c = p->dx / p->dt, dt = p->dt, cK = p->cK, cmu = p->cmu;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double U[5], Ux[5], Uy[5], Bv[5] = {0, 0, 0, 0, 0};
            for (int k = 0; k < 5; ++k) {
                U[k] = U0[fld(p, k, y, x)];
                Ux[k] = dU0dx[fld(p, k, y, x)];
                Uy[k] = dU0dy[fld(p, k, y, x)];
            }
            if (B0) {
                Bv[0] = B0[fld(p, 0, y, x)];
                Bv[1] = B0[fld(p, 1, y, x)];
            }
            double pxU[5], pyU[5], pxB[5], pyB[5], pxUx[5], pyUy[5];
            double pxpxUx[5], pypxUx[5], pxpyUy[5], pypyUy[5];
            phi_x(U, cK, cmu, pxU);
            phi_y(U, cK, cmu, pyU);
            phi_x(Bv, cK, cmu, pxB);
            phi_y(Bv, cK, cmu, pyB);
            phi_x(Ux, cK, cmu, pxUx);
            phi_y(Uy, cK, cmu, pyUy);
            phi_x(pxUx, cK, cmu, pxpxUx);
            phi_y(pxUx, cK, cmu, pypxUx);
            phi_x(pyUy, cK, cmu, pxpyUy);
            phi_y(pyUy, cK, cmu, pypyUy);
            for (int d = 0; d < 4; ++d) {
                const double i = (double)VI[d], j = (double)VJ[d];
                for (int k = 0; k < 5; ++k) {
                    const double eq = 0.25 * (U[k] + (2.0 / c) * (i * pxU[k] + j * pyU[k]));
                    const double tb = Bv[k] + (2.0 / c) * (i * pxB[k] + j * pyB[k]);
                    const double tx = c * (i * Ux[k] + ((2.0 * i * i - 1.0) / c) * pxUx[k]
                                           - (2.0 / (c * c)) * (i * pxpxUx[k] + j * pypxUx[k]));
                    const double ty = c * (j * Uy[k] + ((2.0 * j * j - 1.0) / c) * pyUy[k]
                                           - (2.0 / (c * c)) * (i * pxpyUy[k] + j * pypyUy[k]));
                    f[idx(p, d, k, y, x)] = eq - (dt / 8.0) * (tb + tx + ty);
                }
            }
        }
    }
}

/* U^num at every node, Eq. cond_eq: out [5][ny][nx]; B at the same time or NULL. */
void orc_moments(const orc_params* p, const double* f, const double* B, double* out)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double U[5];
            node_moment(p, f, B, y, x, U);
            for (int k = 0; k < 5; ++k) out[fld(p, k, y, x)] = U[k];
        }
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
