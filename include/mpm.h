/*
 * mpm.h -- C ABI of the B300 (sm_103a) compressible-gas Material Point Method
 * hot path (Baioni, Benacchio, Capone, de Falco, "Portable, Massively
 * Parallel Implementation of a Material Point Method for Compressible Flows").
 *
 * One time step (Sec. 3, Algorithm 1) runs entirely on the GPU:
 *   a1 stable re-order of the particles by the tile-major number of the basis
 *      span that holds them (step xii; keys from step x),
 *   a2 P2G of mass and momentum and P2GD of the pressure force (step ii),
 *   a3 grid boundary conditions / obstacle projection (eqs. normali1-2) and
 *      the momentum update mv' = mv + dt f (steps iii-iv),
 *   a4 G2P of the acceleration, velocity update, momentum P2G (steps v-vii),
 *   a5 boundary conditions on the new momentum (step vii),
 *   a6 G2PD of the velocity divergence, energy / density / EOS / artificial
 *      viscosity update (step viii, eqs. pressures, muart), move with Vbar
 *      (step ix) and the new connectivity (step x),
 *   a7 the CFL reduction and time advance (step xiii, eq. CFL).
 *
 * Conventions (all entry points):
 *   - every call returns an mpm_status; nothing aborts, prints or exits;
 *   - pointers to arrays are HOST pointers owned by the caller; inputs are
 *     copied before the call returns, outputs are written before it returns;
 *     the library never keeps a caller pointer;
 *   - particle arrays are structure-of-arrays: x[a*n + k] is component a of
 *     particle k; node arrays use the storage layout described below;
 *   - device memory is owned by the simulation and released by mpm_destroy;
 *   - a failing device check (non-finite state, a particle moving more than
 *     one span in a step, an inconsistent tile) poisons the simulation: the
 *     status is returned by the call that observes it (mpm_step, mpm_sync or
 *     a read) and every later call except mpm_last_error/mpm_destroy returns
 *     MPM_ESTATE.
 *
 * Grid layout.  d = dim, p = degree, n_a cells of edge h along axis a on
 * [origin_a, origin_a + n_a h].  A non-periodic axis stores n_a + 2p - 1
 * nodes, storage index i <-> node at origin_a + (i - (p - 1)) h (degree 2 has
 * one ghost node beyond each face); a periodic axis stores n_a nodes.  Node
 * (i0, i1, i2) is stored at (i2 N1 + i1) N0 + i0.
 *
 * Span and key.  A particle at xi = (x - origin)/h lies in span
 * c = floor(xi) (degree 1, the grid cell) or c = floor(xi + 1/2) (degree 2, the
 * dual cell around the nearest node), clamped to the axis (periodic: wrapped).
 * Spans are grouped in tiles of tile[a] spans per axis; the key is
 * tile_index * tile_volume + local_index, both x-fastest.  Keys are evaluated
 * in the storage precision with one rounding per operation, so a given
 * binary32 (binary64) position always gets the same key.
 */
#ifndef MPM_H
#define MPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_sim mpm_sim;   /* opaque; owned by the library */

typedef enum {
    MPM_OK = 0,
    MPM_EINVAL = 1,        /* bad argument, size or configuration */
    MPM_ENOMEM = 2,        /* device or host allocation failed */
    MPM_ECUDA = 3,         /* a CUDA runtime call failed (see mpm_last_error) */
    MPM_ESTATE = 4,        /* call not allowed in the current state / poisoned */
    MPM_ENONFINITE = 5,    /* non-finite state or 1 + dt div(v) <= 0 */
    MPM_ETIMEOUT = 6,      /* a bounded device wait expired */
    MPM_EUNSUPPORTED = 7,  /* valid request the library does not support */
    MPM_ECFL = 8           /* a particle crossed more than one span in a step */
} mpm_status;

typedef enum { MPM_BC_WALL = 0, MPM_BC_PERIODIC = 1, MPM_BC_INFLOW = 2, MPM_BC_OUTFLOW = 3 } mpm_bc;
/* MPM_FP32: float atomics on the grid (fastest; the order of the float
 *   sums into a node varies between runs).
 * MPM_FP32_FIXED64: binary32 contributions quantised to int64 (exact,
 *   order-independent sums: bit-reproducible).
 * MPM_FP64: everything in binary64 (float atomics).
 * MPM_FP32_COLOURED: MPM_FP32 arithmetic, with the two node-scattering
 *   kernels run in colour passes over the tiles (tile coordinate parities;
 *   a third colour for the last tile of an odd periodic axis) whose node
 *   windows never overlap, so each node receives its sums in a fixed order:
 *   bit-reproducible FP32 without fixed point (the grid colouring that
 *   Sec. 5, Discussion and conclusion, proposes, on tiles instead of cells).  Needs every tile edge >= degree and a
 *   periodic axis to hold at least two whole tiles (MPM_EUNSUPPORTED), and
 *   cannot join a batch. */
typedef enum { MPM_FP32 = 0, MPM_FP32_FIXED64 = 1, MPM_FP64 = 2, MPM_FP32_COLOURED = 3 } mpm_precision;

/* Fields for mpm_read_state / mpm_field_size. */
enum {
    MPM_FIELD_X = 0, MPM_FIELD_V = 1, MPM_FIELD_M = 2, MPM_FIELD_RHO = 3, MPM_FIELD_E = 4,
    MPM_FIELD_P = 5, MPM_FIELD_Q = 6, MPM_FIELD_ID = 7, MPM_FIELD_KEY = 8,
    MPM_FIELD_CELLSTART = 9, MPM_FIELD_GRID_M = 10, MPM_FIELD_GRID_MV = 11,
    MPM_FIELD_GRID_F = 12, MPM_FIELD_GRID_MV2 = 13, MPM_FIELD_CLOCK = 14, MPM_FIELD_GEN = 16
};

typedef struct {
    int dim;                 /* 2 or 3 */
    int n[3];                /* cells per axis (n[2] ignored for dim 2) */
    double h;                /* cell edge (square cells) */
    double origin[3];
    double gamma, c0, c1;    /* ideal-gas ratio (eq. pressures), AV constants (eq. muart) */
    int degree;              /* 1: the paper's Q1 basis; 2: quadratic B-spline (Sec. 5) */
    int precision;           /* mpm_precision */
    double fixed_unit[3];    /* MPM_FP32_FIXED64: mass, momentum, force unit U; a
                                contribution c is stored as round(c 2^32 / U) in int64.
                                0 selects U = 1. */
    int bc[6];               /* mpm_bc of faces -x,+x,-y,+y,-z,+z; periodic in pairs */
    double inflow_rho, inflow_p, inflow_v[3];   /* inflow faces and recycled particles */
    double cfl;              /* dt = cfl h / (max|v| + max c) (eq. CFL, Sec. 4.1) */
    int sort_interval;       /* must be 1: the tiled kernels need ordered particles */
    uint64_t seed;           /* Philox-4x32-10 key of particle recycling: a particle
                                leaving through an outflow face for the g-th time draws
                                from counter (g, 0, id, 0) */
    int tile[3];             /* spans per tile per axis, powers of two <= 64; 0 selects
                                16 x 8 x 4 (3D) / 32 x 8 (2D).  The tiles define the
                                key numbering, so they fix the KEY and CELLSTART
                                outputs (see "Span and key" above) */
    void* stream;            /* cudaStream_t to run on; NULL: the library's own stream */
    /* Optional device allocator (e.g. a framework's caching allocator):
       alloc(bytes, ctx) returns device memory or NULL; free(ptr, ctx).
       NULL: cudaMalloc/cudaFree. Memory is allocated only by create,
       add_particles and set_obstacle_mask, never by step. */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* alloc_ctx;
} mpm_config;

/* Create an empty simulation on the current CUDA device (Sec. 3 step 2: the
 * object is built once).  cfg is copied.  *out receives the handle, or NULL
 * on error.  Errors: MPM_EINVAL (bad configuration), MPM_ENOMEM, MPM_ECUDA. */
mpm_status mpm_create(const mpm_config* cfg, mpm_sim** out);

/* Append n particles (Sec. 3 step 2: the one host-to-device copy of the
 * initial state).  x, v: dim x n SoA; mass, rho, e (specific internal
 * energy): n values; all host pointers.  Positions must lie in the domain
 * (closed, or half-open along periodic axes); mass, rho > 0.  The particles
 * are converted to the storage precision, numbered (id = running count) and
 * ordered by key.  Allowed only before the first mpm_step (MPM_ESTATE). */
mpm_status mpm_add_particles(mpm_sim* sim, int64_t n, const double* x, const double* v,
                             const double* mass, const double* rho, const double* e);

/* mpm_add_particles with the initial state in binary32 (Sec. 3 step 2),
 * for callers whose state is already single precision: the same layout,
 * checks, errors, numbering and ordering, and half the bytes over the host
 * link.  The FP32 modes store the values as given; MPM_FP64 widens them
 * exactly, so either call gives the same state for binary32 values. */
mpm_status mpm_add_particles_f32(mpm_sim* sim, int64_t n, const float* x, const float* v,
                                 const float* mass, const float* rho, const float* e);

/* Obstacle nodes (Sec. 2.2, eqs. normali1-2, sdf): node_mask[i] != 0 marks
 * node i; normals is dim x nodes (outward unit normals, used on marked nodes
 * only).  Both host arrays of the full node count.  When the -x or +x face
 * is an inflow face, marked nodes within p+1 nodes of it are rejected
 * (MPM_EINVAL): recycled particles are placed there. */
mpm_status mpm_set_obstacle_mask(mpm_sim* sim, const uint8_t* node_mask, const double* normals);

/* Obstacle of a 2D problem from closed loops of boundary points (the
 * aerofoil case of Sec. 4.1 reads its profile from a point file; Eq. sdf).
 *   nloops       >= 1
 *   loop_len     nloops counts, each >= 3; at most 2^24 points in all
 *   pts          host, 2 x total points: all x, then all y; loop l is the
 *                next loop_len[l] points, its edges join consecutive points
 *                and the last to the first (either orientation)
 *   mask_out     optional host output (NULL: not returned), one byte per
 *                stored node: the mask that was installed
 *   normals_out  optional, 2 x nodes doubles (SoA): the normals installed
 *   sd_out       optional, nodes doubles: the signed distance
 * Computed on the device in binary64, every operation rounded separately:
 * per stored node, sd = distance to the nearest point of the edges (the
 * first edge wins ties), negative inside by the even-odd rule (inner loops
 * are holes); cells with a corner at sd <= 0 are obstacle cells and their
 * corner nodes are masked; normals = grad sd on masked nodes, (X - Q)/|X - Q|
 * outside and (Q - X)/|X - Q| inside for the nearest boundary point Q (so
 * they point out of the obstacle), 0 on the boundary and on unmasked nodes.
 * Along a periodic axis the profile is not repeated.  The result replaces
 * the obstacle as mpm_set_obstacle_mask would, with the same checks.
 * Synchronous.  Errors: MPM_EINVAL (fewer than 3 points in a loop,
 * non-finite points, obstacle nodes next to an inflow face),
 * MPM_EUNSUPPORTED (3D), MPM_ENOMEM, MPM_ECUDA, MPM_ESTATE. */
mpm_status mpm_set_obstacle_profile(mpm_sim* sim, int64_t nloops, const int64_t* loop_len, const double* pts,
                                    uint8_t* mask_out, double* normals_out, double* sd_out);

/* The CFL step (eq. CFL with Sec. 4.1's form) for the next step: from the
 * initial state before the first step, else from the last step. */
mpm_status mpm_cfl_dt(mpm_sim* sim, double* dt_out);

/* Advance nsteps steps of Algorithm 1.  dt > 0 fixes the step; dt <= 0 uses
 * the CFL rule.  t_end > 0 clips the last step so that t reaches t_end exactly
 * and turns the remaining steps into no-ops.  Waits for completion and
 * reports device-side errors. */
mpm_status mpm_step(mpm_sim* sim, int64_t nsteps, double dt, double t_end);
/* Same, but only enqueues the work on the simulation's stream; device
 * errors are reported by the next mpm_sync or read. */
mpm_status mpm_step_async(mpm_sim* sim, int64_t nsteps, double dt, double t_end);
/* Wait for queued work; report device errors. */
mpm_status mpm_sync(mpm_sim* sim);

/* Copy a field to the host buffer out: the outputs of the time loop (the
 * device-to-host copies of Sec. 3 step xi and of the final output after
 * Algorithm 1; KEY and CELLSTART are the connectivity of step x in the
 * order of the re-order of step xii).  out holds count doubles, at least
 * mpm_field_size(sim, field), else MPM_EINVAL.
 *   X, V           dim x n, structure of arrays
 *   M, RHO, E, Q   mass, density, specific internal energy, artificial
 *                  viscosity (eq. muart) of each particle
 *   P              pressure of the ideal-gas law (eq. pressures),
 *                  (gamma - 1) rho e, evaluated on the device in the storage
 *                  precision exactly as the step kernels evaluate it, then
 *                  widened to double
 *   ID             the input numbering (running count of mpm_add_particles)
 *   KEY            span key of each particle (tile-major, see above)
 *   CELLSTART      keys + 1 entries: first position of each key
 *   GEN            times each particle has been re-created at the inflow
 *                  (Sec. 4.1); the counter g of its next Philox draw
 *   GRID_*         the raw P2G sums of the last step before boundary
 *                  conditions (GRID_MV2 the second momentum P2G)
 *   CLOCK          {t, dt_next, steps, relayouts}: relayouts counts the steps
 *                  whose re-order gave every tile a new region (a tile had
 *                  outgrown its own)
 * Particle fields are in the current (key) order.  Synchronous.  Errors:
 * MPM_EINVAL (unknown field, short buffer, NULL out), MPM_ESTATE (poisoned
 * or in a batch), MPM_ENOMEM, MPM_ECUDA, or the device error the call
 * observes. */
mpm_status mpm_read_state(mpm_sim* sim, int field, double* out, int64_t count);
/* Raw int64 grid sums of the fixed-point mode (GRID_M/MV/F/MV2 only). */
mpm_status mpm_read_grid_fixed(mpm_sim* sim, int field, int64_t* out, int64_t count);
/* Number of doubles a field needs, or -1. */
int64_t mpm_field_size(const mpm_sim* sim, int field);

/* Conservation diagnostics of the state (mass, total energy and momentum,
 * the quantities whose balance Sec. 2.1's equations state): FP64 sums over
 * particles {sum M, sum M (e + |V|^2/2), sum M V_x, _y, _z}, reduced on the
 * device in a fixed order, so repeated calls on the same state agree bit for
 * bit.  Synchronous.  Errors as for mpm_read_state. */
mpm_status mpm_conservation(mpm_sim* sim, double out[5]);
/* {particles, nodes, keys, steps done}. */
mpm_status mpm_sizes(const mpm_sim* sim, int64_t out[4]);

/* Per-phase device timing: enable (1) or disable (0).  When enabled each step
 * records CUDA events around its phases on the simulation's stream; times
 * accumulate until read.  out[8] = ms of {P2G, grid+G2P+P2G, G2PD+update,
 * time advance, re-order, whole steps, -, -}; counts[8] = launches of this
 * library's kernels in the same phases. */
mpm_status mpm_profile(mpm_sim* sim, int enable);
mpm_status mpm_profile_read(mpm_sim* sim, double out[8], int64_t counts[8], int reset);

/* Stable sort of caller-supplied span keys that allocates no device memory.
 * The paper has no counterpart: this is the library's re-order step (a1)
 * offered to callers that must not call cudaMalloc -- components confined to
 * another framework's memory pool, which must not grow the device footprint
 * behind its back, or latency-critical loops where an allocation could
 * synchronise the device.  Its scratch lives in fixed device arrays inside
 * the library (3.1 MiB per GPU that loads the library, held until the
 * process exits), so the input size is capped.
 *   keys        device pointer, n keys, each < nkeys (not modified)
 *   n           0 <= n <= MPM_SORT_STATIC_MAX_KEYS, else MPM_EINVAL
 *   nkeys       1 <= nkeys <= MPM_SORT_STATIC_MAX_SPANS, else MPM_EINVAL
 *   perm        device pointer, n entries: perm[j] = index of the key placed
 *               at position j (equal keys keep their input order)
 *   cell_start  device pointer, nkeys + 1 entries: first position of each
 *               key; cell_start[nkeys] = n.  If some key is >= nkeys the
 *               call writes 0xffffffff to cell_start[nkeys] instead (the
 *               check runs on the device); perm and the other cell starts
 *               are then unspecified
 *   stream      cudaStream_t the work is queued on (NULL: the default stream)
 * The call only queues kernels and returns; the outputs are valid once the
 * stream reaches them.  The first call on a device looks up the scratch
 * addresses and keeps them for the life of the process, so the call must not
 * be used after cudaDeviceReset.  All calls on a device share the scratch,
 * which keeps the last call's contents: calls whose work overlaps on the GPU
 * (other streams, other threads) race and must be serialised by the
 * caller. */
#define MPM_SORT_STATIC_MAX_KEYS 262144
#define MPM_SORT_STATIC_MAX_SPANS 16777216
mpm_status mpm_sort_keys_static(const uint32_t* keys, int64_t n, int64_t nkeys, uint32_t* perm,
                                uint32_t* cell_start, void* stream);

/* Self-check of the fixed-point quantiser (MPM_FP32_FIXED64).  That mode
 * turns every binary32 P2G contribution c into the int64 round(c * S), ties
 * to even.  Where a particle's quantised contributions are bounded by 2^31
 * in magnitude the kernels round with the 32-bit float-to-int conversion
 * (the 64-bit one is much slower).  This call evaluates both conversions on
 * every binary32 bit pattern v with |v| < 2^31 on the current device and
 * returns, in host memory, the number of patterns where they differ
 * (*mismatches) and the smallest such pattern (*first, 0xffffffff if
 * none).  Synchronous; allocates 16 bytes
 * of device memory for the call.  Errors: MPM_EINVAL (NULL pointer),
 * MPM_ENOMEM, MPM_ECUDA. */
mpm_status mpm_check_fixed_rounding(uint64_t* mismatches, uint32_t* first);

/* ---- Batched execution of independent simulations (serving) ----
 * The paper solves one problem at a time; a batch advances many resident
 * simulations together: each stage of the step (Algorithm 1) is one launch
 * over a flattened list of (simulation, tile) pairs, and one step of the whole
 * batch is recorded once as a CUDA graph and replayed.  Every member runs the
 * same tile code with its own geometry, clock and CFL time step, so its
 * results equal those of mpm_step on that simulation alone (bit for bit in
 * the fixed-point mode).
 *   mpm_batch_create  stream: cudaStream_t the batch runs on (NULL: its own).
 *   mpm_batch_add     sim joins (it must have particles and not be in a
 *                     batch); it takes at most nsteps further steps in batched
 *                     runs (nsteps > 0), with dt and t_end as in mpm_step.
 *                     While a member, the sim accepts only mpm_batch_remove,
 *                     mpm_stream, mpm_last_error and mpm_destroy; other calls
 *                     return MPM_ESTATE.  The batch's stream waits for the
 *                     sim's queued work.
 *   mpm_batch_remove  sim leaves; its stream waits for the batch's queued
 *                     work, after which all calls on the sim are valid again.
 *   mpm_batch_step_async  queue nsteps steps of every member (a member whose
 *                     step budget or t_end is reached idles).  Changing the
 *                     members re-records the graph at the next call.
 *   mpm_batch_sync    wait for the batch's work and return the status of
 *                     the first member whose kernels raised an error (its
 *                     further batched steps do nothing); that member reports
 *                     its own status at its first call after it leaves the
 *                     batch, and is poisoned from then on.
 *   mpm_batch_destroy removes all members and releases the batch.
 * Members are grouped by kernel variant (dimension, degree, precision,
 * periodicity); each group's stages are single launches. */
typedef struct mpm_batch mpm_batch;
mpm_status mpm_batch_create(void* stream, mpm_batch** out);
mpm_status mpm_batch_add(mpm_batch* batch, mpm_sim* sim, int64_t nsteps, double dt, double t_end);
mpm_status mpm_batch_remove(mpm_batch* batch, mpm_sim* sim);
mpm_status mpm_batch_step_async(mpm_batch* batch, int64_t nsteps);
mpm_status mpm_batch_sync(mpm_batch* batch);
/* {members, groups, launches per batched step, graph recordings so far}. */
mpm_status mpm_batch_info(const mpm_batch* batch, int64_t out[4]);
/* The batch's stream (cudaStream_t). */
void* mpm_batch_stream(const mpm_batch* batch);
const char* mpm_batch_last_error(const mpm_batch* batch);
void mpm_batch_destroy(mpm_batch* batch);

/* The simulation's stream (cudaStream_t). */
void* mpm_stream(const mpm_sim* sim);
/* Message of the last error of this handle (static storage if sim is NULL). */
const char* mpm_last_error(const mpm_sim* sim);
/* Release everything; NULL is allowed. Waits for queued work. */
void mpm_destroy(mpm_sim* sim);

#ifdef __cplusplus
}
#endif
#endif /* MPM_H */
