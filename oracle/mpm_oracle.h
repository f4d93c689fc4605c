/*
 * mpm_oracle.h -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, serial FP64 CPU implementation of the compressible-gas
 * Material Point Method step (Baioni et al., "Portable, Massively Parallel
 * Implementation of a Material Point Method for Compressible Flows",
 * Sec. 2-3, Algorithm 1).  It exists only so that the tests, the smoke check
 * and the benchmark's CPU-baseline leg can check and time the CUDA path.
 * It shares no code, header, table or helper with the CUDA library; only the
 * seeded input generators are common to both.
 *
 * Conventions shared with the CUDA path by necessity (they define the
 * results that are compared, not how they are computed):
 *   - node storage layout and the tile-major span numbering used as the
 *     sort key (see mpm_oracle.c, "geometry");
 *   - Philox-4x32-10 as the counter-based generator for particle recycling.
 * Every function returns 0 on success or a positive error code.
 */
#ifndef MPM_ORACLE_H
#define MPM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ESTATE = 4,
       OR_ENONFINITE = 5, OR_ECFL = 8 };
enum { OR_BC_WALL = 0, OR_BC_PERIODIC = 1, OR_BC_INFLOW = 2, OR_BC_OUTFLOW = 3 };

/* Field ids for oracle_read (the product's read call uses the same numbers
 * for the fields both have; VBAR is the oracle's alone).  GEN = how many times
 * each particle has been re-created at the inflow. */
enum { OR_F_X = 0, OR_F_V = 1, OR_F_M = 2, OR_F_RHO = 3, OR_F_E = 4, OR_F_P = 5,
       OR_F_Q = 6, OR_F_ID = 7, OR_F_KEY = 8, OR_F_CELLSTART = 9,
       OR_F_GRID_M = 10, OR_F_GRID_MV = 11, OR_F_GRID_F = 12, OR_F_GRID_MV2 = 13,
       OR_F_CLOCK = 14, OR_F_VBAR = 15, OR_F_GEN = 16 };

typedef struct {
    int dim;              /* 2 or 3 */
    int n[3];             /* cells per axis (n[2] ignored in 2D) */
    double h;             /* square cell edge */
    double origin[3];
    double gamma, c0, c1; /* EOS and artificial-viscosity constants */
    int degree;           /* 1 = bilinear/trilinear (Q1), 2 = quadratic B-spline */
    int bc[6];            /* faces -x,+x,-y,+y,-z,+z */
    double inflow_rho, inflow_p, inflow_v[3];
    double cfl;
    int sort_interval;    /* re-order every k steps (0 = never) */
    uint64_t seed;        /* recycling generator key */
    int tile[3];          /* span-tile edge per axis for the key numbering
                             (0: 16 x 8 x 4 in 3D, 32 x 8 in 2D) */
} oracle_config;

typedef struct oracle_sim oracle_sim;

int  oracle_create(const oracle_config* cfg, oracle_sim** out);
void oracle_destroy(oracle_sim* s);
int  oracle_add_particles(oracle_sim* s, int64_t n, const double* x, const double* v,
                          const double* mass, const double* rho, const double* e);
int  oracle_set_obstacle_mask(oracle_sim* s, const uint8_t* node_mask, const double* normals);
int  oracle_cfl_dt(oracle_sim* s, double* dt_out);
/* nsteps steps; dt > 0 fixes the step, dt <= 0 uses the CFL rule; t_end > 0
 * clips the last step so that t reaches t_end exactly and stops there. */
int  oracle_step(oracle_sim* s, int64_t nsteps, double dt, double t_end);
int  oracle_read(oracle_sim* s, int field, double* out, int64_t count);
int64_t oracle_field_size(oracle_sim* s, int field);
int  oracle_conservation(oracle_sim* s, double out[5]);
int  oracle_sizes(oracle_sim* s, int64_t out[4]); /* particles, nodes, spans(keys), steps */

/* ---- standalone pieces used by the pins and the unit-level parity tests ---- */

/* Degree-p B-spline weights/derivatives (per unit of xi) at offset fx of the
 * particle from its first support node. */
void oracle_bspline(int degree, double fx, double w[3], double dw[3]);
/* Closed-form 1D B-spline N(r) and N'(r) as functions of the signed distance
 * r (in cells) from the node; used for the brute-force pins. */
double oracle_bspline_dense(int degree, double r, double* dN);

/* Sort keys of n positions (SoA, dim x n) with the span/tile numbering of cfg.
 * prec32 != 0 evaluates the span in binary32 exactly as the storage-precision
 * rule prescribes; positions must then be binary32 values. */
int oracle_keys(const oracle_config* cfg, int64_t n, const double* x, int prec32, uint32_t* keys);
/* Stable sort by key: perm[j] = old index placed at j; start[K+1]. */
int oracle_stable_sort(int64_t n, const uint32_t* keys, int64_t nkeys, int64_t* perm, int64_t* start);
/* The per-step re-order (Sec. 3 step xii): particles in their current order
 * go to the list of their key; those re-created at the inflow during the step
 * (recycled[k] != 0, Sec. 4.1) follow the other particles of their key, by
 * id.  perm[j] = current index placed at j; start[K] (nkeys + 1 entries). */
int oracle_reorder(int64_t n, const uint32_t* keys, const uint8_t* recycled, const int64_t* ids,
                   int64_t nkeys, int64_t* perm, int64_t* start);

/* P2G of m, M V, (P+Q) M/rho grad(phi) for a particle set (FP64, plain loop). */
int oracle_p2g(const oracle_config* cfg, int64_t n, const double* x, const double* v,
               const double* mass, const double* rho, const double* e, const double* q,
               double* grid_m, double* grid_mv, double* grid_f);
/* Same sums by dense O(N_p N_n) evaluation of the closed-form basis. */
int oracle_p2g_dense(const oracle_config* cfg, int64_t n, const double* x, const double* v,
                     const double* mass, const double* rho, const double* e, const double* q,
                     double* grid_m, double* grid_mv, double* grid_f);
/* Fixed-point P2G: every particle-node contribution evaluated in binary32 in
 * the documented order, quantised to round(value * 2^32/unit) and summed in
 * int64.  unit[3] = mass, momentum, force units. */
int oracle_p2g_fixed32(const oracle_config* cfg, int64_t n, const float* x, const float* v,
                       const float* mass, const float* rho, const float* e, const float* q,
                       const double unit[3], int64_t* grid_m, int64_t* grid_mv, int64_t* grid_f);

/* Obstacle projection of one vector (eqs. normali1/normali2). */
void oracle_obstacle_project(int dim, const double* x, const double* n, double* out);
/* Obstacle of a 2D problem from closed loops of boundary points (Eq. sdf):
 * loop l has loop_len[l] >= 3 points, pts = all x then all y (SoA, 2 x total).
 * Per stored node: sd[node] (negative inside, even-odd rule), mask[node] = 1
 * on the corner nodes of cells with a corner at sd <= 0, normals (2 x nodes,
 * SoA) = grad sd on masked nodes, 0 elsewhere. */
int oracle_obstacle_profile(const oracle_config* cfg, int64_t nloops, const int64_t* loop_len, const double* pts,
                            uint8_t* mask, double* normals, double* sd);

/* Philox-4x32-10 block function. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Exact solution of the 1D Riemann problem for an ideal gas, sampled at
 * x/t = s[i]: writes rho, u, p.  Also returns p* and u* in star[2]. */
int oracle_riemann_exact(double gamma, double rl, double ul, double pl,
                         double rr, double ur, double pr,
                         int64_t n, const double* s, double* rho, double* u, double* p,
                         double star[2]);

#ifdef __cplusplus
}
#endif
#endif
