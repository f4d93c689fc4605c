/*
 * mpm_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * Plain serial FP64 reference of the compressible-gas MPM time step of
 * Baioni et al. (Sec. 3, Algorithm 1), written for reading, not for speed:
 * every mapping of the paper (P2G, P2GD, G2P, G2PD, eqs. p2g_gen..g2pd_gen)
 * is its own loop over particles, in the order the algorithm lists them.
 * Only the tests, the smoke check and the benchmark CPU-baseline leg use it.
 *
 * Readings of the paper that this file fixes (the CUDA path follows them):
 *   - degree 1 = the paper's Q1 basis (Sec. 2.2); degree 2 = the quadratic
 *     B-spline named as the higher-order option (Sec. 5);
 *   - a particle's "cell" (the connectivity map of Sec. 3 step x and the
 *     reordering of step xii) is the knot span of the basis that contains it:
 *     the grid cell for degree 1, the cell of the dual grid centred on the
 *     nearest node for degree 2.  Particles in one span share their support;
 *   - spans are numbered tile-major (tiles of tile[a] spans, tiles and spans
 *     inside a tile both x-fastest);
 *   - grid BC on a node: obstacle projection (eqs. normali1, normali2) if the
 *     node is masked, then the domain faces: a slip wall zeroes the normal
 *     component, an inflow face imposes m*v_in on momentum and zero force;
 *   - theta(a, m) = a/m, and 0 where m == 0 (node with no mass);
 *   - artificial viscosity (eq. muart) evaluated with the updated rho, p and
 *     this step's div(v); the energy update uses the old p, q, rho;
 *   - dt = cfl*h/(max|v| + max c) (Sec. 3 step xiii, Sec. 4.1): v over the
 *     moving velocity Vbar and the updated velocity V' of every particle
 *     (plus the inflow speed when a particle is recycled), c from the state
 *     after the step;
 *   - a particle leaving through an outflow face is re-created in the first
 *     cell layer of the inflow face with the inflow state (Sec. 4.1),
 *     positions drawn from Philox-4x32-10 keyed by (seed, step, id).
 */
#include "mpm_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ geometry */

typedef struct {
    int dim, p;
    int n[3], per[3], S[3], N[3], g[3], T[3], nt[3];
    int64_t nkey, nnode;
    double h, inv_h, lo[3], hi[3];
} geom;

static int geom_init(const oracle_config* c, geom* G)
{
    memset(G, 0, sizeof(*G));
    if (!c || (c->dim != 2 && c->dim != 3) || (c->degree != 1 && c->degree != 2)) return OR_EINVAL;
    if (!(c->h > 0.0)) return OR_EINVAL;
    G->dim = c->dim; G->p = c->degree; G->h = c->h; G->inv_h = 1.0 / c->h;
    for (int a = 0; a < 3; ++a) {
        if (a >= c->dim) {
            G->n[a] = 1; G->S[a] = 1; G->N[a] = 1; G->T[a] = 1; G->nt[a] = 1;
            continue;
        }
        int bl = c->bc[2 * a], bh = c->bc[2 * a + 1];
        if (bl < 0 || bl > 3 || bh < 0 || bh > 3) return OR_EINVAL;
        if ((bl == OR_BC_PERIODIC) != (bh == OR_BC_PERIODIC)) return OR_EINVAL;
        if (c->n[a] < 1) return OR_EINVAL;
        G->n[a] = c->n[a];
        G->per[a] = (bl == OR_BC_PERIODIC);
        G->S[a] = G->per[a] ? c->n[a] : (G->p == 2 ? c->n[a] + 1 : c->n[a]);
        G->N[a] = G->per[a] ? c->n[a] : c->n[a] + 2 * G->p - 1;
        G->g[a] = G->per[a] ? 0 : G->p - 1;
        static const int def3[3] = {16, 8, 4}, def2[3] = {32, 8, 1};
        G->T[a] = c->tile[a] > 0 ? c->tile[a] : (c->dim == 3 ? def3[a] : def2[a]);
        G->nt[a] = (G->S[a] + G->T[a] - 1) / G->T[a];
        G->lo[a] = c->origin[a];
        G->hi[a] = c->origin[a] + c->n[a] * c->h;
    }
    G->nkey = (int64_t)G->nt[0] * G->nt[1] * G->nt[2] * G->T[0] * G->T[1] * G->T[2];
    G->nnode = (int64_t)G->N[0] * G->N[1] * G->N[2];
    return OR_OK;
}

static int64_t imod(int64_t a, int64_t n) { int64_t r = a % n; return r < 0 ? r + n : r; }

/* Span number of a particle along axis a from xi = (x - lo)/h (FP64). */
static int64_t span_of_xi(const geom* G, int a, double xi)
{
    int64_t c = (G->p == 2) ? (int64_t)floor(xi + 0.5) : (int64_t)floor(xi);
    if (G->per[a]) return c;                 /* unwrapped; caller wraps */
    if (c < 0) c = 0;
    if (c > G->S[a] - 1) c = G->S[a] - 1;
    return c;
}

static uint32_t key_of_spans(const geom* G, const int64_t sp[3])
{
    int64_t t[3], l[3];
    for (int a = 0; a < 3; ++a) { t[a] = sp[a] / G->T[a]; l[a] = sp[a] % G->T[a]; }
    int64_t tile = (t[2] * G->nt[1] + t[1]) * G->nt[0] + t[0];
    int64_t loc = (l[2] * G->T[1] + l[1]) * G->T[0] + l[0];
    return (uint32_t)(tile * (int64_t)(G->T[0] * G->T[1] * G->T[2]) + loc);
}

/* ------------------------------------------------------------------ basis */

void oracle_bspline(int degree, double fx, double w[3], double dw[3])
{
    if (degree == 1) {               /* hat functions of the Q1 basis, Sec. 2.2 */
        w[0] = 1.0 - fx; w[1] = fx; w[2] = 0.0;
        dw[0] = -1.0; dw[1] = 1.0; dw[2] = 0.0;
    } else {                         /* quadratic B-spline, fx in [0.5, 1.5) */
        double a = 1.5 - fx, b = fx - 1.0, c = fx - 0.5;
        w[0] = 0.5 * a * a; w[1] = 0.75 - b * b; w[2] = 0.5 * c * c;
        dw[0] = -a; dw[1] = -2.0 * b; dw[2] = c;
    }
}

double oracle_bspline_dense(int degree, double r, double* dN)
{
    double ar = fabs(r), s = (r < 0) ? -1.0 : 1.0;
    if (degree == 1) {
        if (ar >= 1.0) { *dN = 0.0; return 0.0; }
        *dN = -s; return 1.0 - ar;
    }
    if (ar < 0.5) { *dN = -2.0 * r; return 0.75 - r * r; }
    if (ar < 1.5) { *dN = -s * (1.5 - ar); return 0.5 * (1.5 - ar) * (1.5 - ar); }
    *dN = 0.0; return 0.0;
}

/* Support of one particle: storage index, weight and gradient of each of the
 * (p+1)^d nodes whose basis function is non-zero at x. */
typedef struct { int cnt; int64_t node[27]; double w[27]; double gw[27][3]; int64_t span[3]; } support;

static void particle_support(const geom* G, const double* xk, support* sp)
{
    int64_t idx[3][3]; double w[3][3], dw[3][3]; int ns[3];
    for (int a = 0; a < 3; ++a) {
        if (a >= G->dim) { idx[a][0] = 0; w[a][0] = 1.0; dw[a][0] = 0.0; ns[a] = 1; sp->span[a] = 0; continue; }
        double xi = (xk[a] - G->lo[a]) * G->inv_h;
        int64_t c = span_of_xi(G, a, xi);
        double fx = xi - (double)(c - (G->p == 2 ? 1 : 0));
        oracle_bspline(G->p, fx, w[a], dw[a]);
        ns[a] = G->p + 1;
        for (int k = 0; k < ns[a]; ++k) {
            int64_t phys = c - (G->p == 2 ? 1 : 0) + k;
            idx[a][k] = G->per[a] ? imod(phys, G->n[a]) : phys + G->g[a];
        }
        sp->span[a] = G->per[a] ? imod(c, G->n[a]) : c;
    }
    sp->cnt = 0;
    for (int kz = 0; kz < ns[2]; ++kz)
        for (int ky = 0; ky < ns[1]; ++ky)
            for (int kx = 0; kx < ns[0]; ++kx) {
                int j = sp->cnt++;
                sp->node[j] = (idx[2][kz] * G->N[1] + idx[1][ky]) * G->N[0] + idx[0][kx];
                sp->w[j] = w[0][kx] * w[1][ky] * w[2][kz];
                sp->gw[j][0] = dw[0][kx] * w[1][ky] * w[2][kz] * G->inv_h;
                sp->gw[j][1] = w[0][kx] * dw[1][ky] * w[2][kz] * G->inv_h;
                sp->gw[j][2] = w[0][kx] * w[1][ky] * dw[2][kz] * G->inv_h;
            }
}

/* ------------------------------------------------------- the four mappings */

/* P2G(F, A; x_i) = sum_k F(A_k) phi_i(X_k)  (eq. p2g_gen); coef[k] = F(A_k). */
static void p2g(const geom* G, int64_t np, double* const x[3], const double* coef, double* out)
{
    support sp; double xk[3];
    for (int64_t k = 0; k < np; ++k) {
        for (int a = 0; a < 3; ++a) xk[a] = (a < G->dim) ? x[a][k] : 0.0;
        particle_support(G, xk, &sp);
        for (int j = 0; j < sp.cnt; ++j) out[sp.node[j]] += coef[k] * sp.w[j];
    }
}

/* P2GD(G, A; x_i) = sum_k G(A_k) . grad phi_i(X_k)  (eq. p2gd_gen) for the
 * functors zeta/eta/(z-analogue): G = coef[k] e_a, one output per component. */
static void p2gd(const geom* G, int64_t np, double* const x[3], const double* coef, double* out[3])
{
    support sp; double xk[3];
    for (int64_t k = 0; k < np; ++k) {
        for (int a = 0; a < 3; ++a) xk[a] = (a < G->dim) ? x[a][k] : 0.0;
        particle_support(G, xk, &sp);
        for (int j = 0; j < sp.cnt; ++j)
            for (int a = 0; a < G->dim; ++a) out[a][sp.node[j]] += coef[k] * sp.gw[j][a];
    }
}

/* G2P(F, a; X_k) = sum_i F(a_i) phi_i(X_k)  (eq. g2p_gen); fa[i] = F(a_i). */
static void g2p(const geom* G, int64_t np, double* const x[3], const double* fa, double* out)
{
    support sp; double xk[3];
    for (int64_t k = 0; k < np; ++k) {
        for (int a = 0; a < 3; ++a) xk[a] = (a < G->dim) ? x[a][k] : 0.0;
        particle_support(G, xk, &sp);
        double s = 0.0;
        for (int j = 0; j < sp.cnt; ++j) s += fa[sp.node[j]] * sp.w[j];
        out[k] = s;
    }
}

/* G2PD(F, a; X_k) = sum_i F(a_i) grad phi_i(X_k)  (eq. g2pd_gen). */
static void g2pd(const geom* G, int64_t np, double* const x[3], const double* fa, double* out[3])
{
    support sp; double xk[3];
    for (int64_t k = 0; k < np; ++k) {
        for (int a = 0; a < 3; ++a) xk[a] = (a < G->dim) ? x[a][k] : 0.0;
        particle_support(G, xk, &sp);
        double s[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < sp.cnt; ++j)
            for (int a = 0; a < G->dim; ++a) s[a] += fa[sp.node[j]] * sp.gw[j][a];
        for (int a = 0; a < G->dim; ++a) out[a][k] = s[a];
    }
}

/* theta(a, m) = a / m of Sec. 3, with 0 on nodes that carry no mass. */
static void theta(int64_t nn, const double* a, const double* m, double* out)
{
    for (int64_t i = 0; i < nn; ++i) out[i] = (m[i] != 0.0) ? a[i] / m[i] : 0.0;
}

/* ------------------------------------------------------------- simulation */

struct oracle_sim {
    oracle_config cfg;
    geom G;
    int64_t np;
    double *x[3], *v[3], *vbar[3], *M, *rho, *E, *Q;
    int64_t* id;
    uint32_t* gen;       /* times each particle has been recycled */
    uint8_t* recyc;      /* re-created at the inflow in the current step */
    uint32_t* key;
    int64_t* cellstart;
    double *gm, *gmv[3], *gf[3], *gmv2[3];     /* raw P2G sums of the last step */
    double *bmv[3], *bf[3], *bmv2[3];          /* the same after the grid BC */
    double *tmp_node, *tmp_p[3], *coef;
    uint8_t* mask; double* nrm[3];
    double t, dt_next, vmax_step;
    int64_t step;
    int started, poisoned;
};

static void* zalloc(size_t n) { return calloc(n ? n : 1, 1); }

static void free_particles(oracle_sim* s)
{
    for (int a = 0; a < 3; ++a) { free(s->x[a]); free(s->v[a]); free(s->vbar[a]); free(s->tmp_p[a]);
                                  s->x[a] = s->v[a] = s->vbar[a] = s->tmp_p[a] = NULL; }
    free(s->M); free(s->rho); free(s->E); free(s->Q); free(s->id); free(s->key); free(s->coef); free(s->gen);
    free(s->recyc);
    s->M = s->rho = s->E = s->Q = s->coef = NULL; s->id = NULL; s->key = NULL; s->gen = NULL; s->recyc = NULL;
}

void oracle_destroy(oracle_sim* s)
{
    if (!s) return;
    free_particles(s);
    free(s->gm); free(s->tmp_node); free(s->mask); free(s->cellstart);
    for (int a = 0; a < 3; ++a) { free(s->gmv[a]); free(s->gf[a]); free(s->gmv2[a]); free(s->bmv[a]);
                                  free(s->bf[a]); free(s->bmv2[a]); free(s->nrm[a]); }
    free(s);
}

int oracle_create(const oracle_config* cfg, oracle_sim** out)
{
    if (!out) return OR_EINVAL;
    *out = NULL;
    geom G;
    int st = geom_init(cfg, &G);
    if (st) return st;
    if (!(cfg->gamma > 1.0) || !(cfg->cfl > 0.0) || cfg->sort_interval < 0) return OR_EINVAL;
    oracle_sim* s = (oracle_sim*)zalloc(sizeof(oracle_sim));
    if (!s) return OR_ENOMEM;
    s->cfg = *cfg; s->G = G;
    size_t nb = (size_t)G.nnode * sizeof(double);
    s->gm = zalloc(nb); s->tmp_node = zalloc(nb); s->mask = zalloc((size_t)G.nnode);
    s->cellstart = zalloc((size_t)(G.nkey + 1) * sizeof(int64_t));
    int ok = s->gm && s->tmp_node && s->mask && s->cellstart;
    for (int a = 0; a < 3; ++a) {
        s->gmv[a] = zalloc(nb); s->gf[a] = zalloc(nb); s->gmv2[a] = zalloc(nb);
        s->bmv[a] = zalloc(nb); s->bf[a] = zalloc(nb); s->bmv2[a] = zalloc(nb); s->nrm[a] = zalloc(nb);
        ok = ok && s->gmv[a] && s->gf[a] && s->gmv2[a] && s->bmv[a] && s->bf[a] && s->bmv2[a] && s->nrm[a];
    }
    if (!ok) { oracle_destroy(s); return OR_ENOMEM; }
    *out = s;
    return OR_OK;
}

static int sort_particles(oracle_sim* s);

int oracle_add_particles(oracle_sim* s, int64_t n, const double* x, const double* v,
                         const double* mass, const double* rho, const double* e)
{
    if (!s || n < 0 || (n > 0 && (!x || !v || !mass || !rho || !e))) return OR_EINVAL;
    if (s->started) return OR_ESTATE;
    const geom* G = &s->G;
    int64_t np = s->np + n;
    for (int64_t k = 0; k < n; ++k) {          /* inputs must lie in the domain */
        if (!(mass[k] > 0.0) || !(rho[k] > 0.0) || !isfinite(e[k])) return OR_EINVAL;
        for (int a = 0; a < G->dim; ++a) {
            double xa = x[a * n + k];
            if (!(xa >= G->lo[a]) || !(xa <= G->hi[a]) || !isfinite(v[a * n + k])) return OR_EINVAL;
            if (G->per[a] && !(xa < G->hi[a])) return OR_EINVAL;
        }
    }
    double* nx[3] = {0}; double* nv[3] = {0}; double* nvb[3] = {0}; double* ntp[3] = {0};
    double *nM = realloc(s->M, np * sizeof(double) + 8), *nR = NULL, *nE = NULL, *nQ = NULL, *nc = NULL;
    if (nM) s->M = nM;
    nR = realloc(s->rho, np * sizeof(double) + 8); if (nR) s->rho = nR;
    nE = realloc(s->E, np * sizeof(double) + 8); if (nE) s->E = nE;
    nQ = realloc(s->Q, np * sizeof(double) + 8); if (nQ) s->Q = nQ;
    nc = realloc(s->coef, np * sizeof(double) + 8); if (nc) s->coef = nc;
    int64_t* nid = realloc(s->id, np * sizeof(int64_t) + 8); if (nid) s->id = nid;
    uint32_t* nk = realloc(s->key, np * sizeof(uint32_t) + 8); if (nk) s->key = nk;
    uint32_t* ng = realloc(s->gen, np * sizeof(uint32_t) + 8); if (ng) s->gen = ng;
    uint8_t* nrc = realloc(s->recyc, np + 8); if (nrc) s->recyc = nrc;
    int ok = nM && nR && nE && nQ && nc && nid && nk && ng && nrc;
    for (int a = 0; a < 3; ++a) {
        nx[a] = realloc(s->x[a], np * sizeof(double) + 8); if (nx[a]) s->x[a] = nx[a];
        nv[a] = realloc(s->v[a], np * sizeof(double) + 8); if (nv[a]) s->v[a] = nv[a];
        nvb[a] = realloc(s->vbar[a], np * sizeof(double) + 8); if (nvb[a]) s->vbar[a] = nvb[a];
        ntp[a] = realloc(s->tmp_p[a], np * sizeof(double) + 8); if (ntp[a]) s->tmp_p[a] = ntp[a];
        ok = ok && nx[a] && nv[a] && nvb[a] && ntp[a];
    }
    if (!ok) return OR_ENOMEM;
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = s->np + k;
        for (int a = 0; a < 3; ++a) {
            s->x[a][j] = (a < G->dim) ? x[a * n + k] : 0.0;
            s->v[a][j] = (a < G->dim) ? v[a * n + k] : 0.0;
            s->vbar[a][j] = s->v[a][j];
        }
        s->M[j] = mass[k]; s->rho[j] = rho[k]; s->E[j] = e[k]; s->Q[j] = 0.0; s->id[j] = j; s->gen[j] = 0;
        s->recyc[j] = 0;
    }
    s->np = np;
    return sort_particles(s);
}

int oracle_set_obstacle_mask(oracle_sim* s, const uint8_t* mask, const double* normals)
{
    if (!s || !mask || !normals) return OR_EINVAL;
    const int64_t nn = s->G.nnode;
    for (int64_t i = 0; i < nn; ++i) {
        s->mask[i] = mask[i] ? 1 : 0;
        for (int a = 0; a < 3; ++a) s->nrm[a][i] = (a < s->G.dim) ? normals[a * nn + i] : 0.0;
    }
    return OR_OK;
}

/* ------------------------------------------- obstacle from a point profile */

/* Signed distance of the point (X, Y) to the boundary made of closed loops of
 * points (Eq. sdf): the boundary is the union of the loops' edges (vertex k
 * to vertex k+1, the last back to the first); |sd| is the distance to its
 * nearest point (*qx, *qy), found edge by edge, the first edge winning ties;
 * sd < 0 inside, where a ray towards +x crosses the edges an odd number of
 * times (even-odd rule, so inner loops are holes). */
static double profile_sd(int64_t nloops, const int64_t* len, const double* px, const double* py, double X,
                         double Y, double* qx, double* qy)
{
    double best = INFINITY;
    int inside = 0;
    int64_t base = 0;
    *qx = X;
    *qy = Y;
    for (int64_t l = 0; l < nloops; ++l) {
        for (int64_t k = 0; k < len[l]; ++k) {
            int64_t a = base + k, b = base + (k + 1) % len[l];
            double ex = px[b] - px[a], ey = py[b] - py[a];
            double wx = X - px[a], wy = Y - py[a];
            /* nearest point of the edge: a + t (b - a), t clamped to [0, 1] */
            double L2 = ex * ex + ey * ey;
            double t = L2 > 0.0 ? (wx * ex + wy * ey) / L2 : 0.0;
            if (t < 0.0) t = 0.0;
            if (t > 1.0) t = 1.0;
            double cx = px[a] + t * ex, cy = py[a] + t * ey;
            double dx = X - cx, dy = Y - cy;
            double d2 = dx * dx + dy * dy;
            if (d2 < best) { best = d2; *qx = cx; *qy = cy; }
            /* crossing of the ray y = Y, x > X with this edge */
            if ((py[a] > Y) != (py[b] > Y)) {
                double xc = px[a] + (Y - py[a]) * ex / ey;
                if (X < xc) inside ^= 1;
            }
        }
        base += len[l];
    }
    double d = sqrt(best);
    return inside ? -d : d;
}

int oracle_obstacle_profile(const oracle_config* cfg, int64_t nloops, const int64_t* loop_len, const double* pts,
                            uint8_t* mask, double* normals, double* sd)
{
    geom G;
    int st = geom_init(cfg, &G);
    if (st != OR_OK) return st;
    if (G.dim != 2 || nloops < 1 || !loop_len || !pts || !mask || !normals || !sd) return OR_EINVAL;
    int64_t np = 0;
    for (int64_t l = 0; l < nloops; ++l) {
        if (loop_len[l] < 3) return OR_EINVAL;
        np += loop_len[l];
    }
    const double* px = pts;
    const double* py = pts + np;
    for (int64_t k = 0; k < 2 * np; ++k)
        if (!isfinite(pts[k])) return OR_EINVAL;
    const int64_t nn = G.nnode;
    double* qx = (double*)malloc((size_t)nn * sizeof(double));
    double* qy = (double*)malloc((size_t)nn * sizeof(double));
    if (!qx || !qy) { free(qx); free(qy); return OR_ENOMEM; }
    /* 1. sd at every stored node, node i at lo + (i - g) h per axis */
    for (int64_t j = 0; j < G.N[1]; ++j)
        for (int64_t i = 0; i < G.N[0]; ++i) {
            int64_t node = j * G.N[0] + i;
            double X = G.lo[0] + (double)(i - G.g[0]) * G.h;
            double Y = G.lo[1] + (double)(j - G.g[1]) * G.h;
            sd[node] = profile_sd(nloops, loop_len, px, py, X, Y, &qx[node], &qy[node]);
        }
    /* 2. obstacle cells: a corner with sd <= 0; their corner nodes are masked */
    memset(mask, 0, (size_t)nn);
    for (int64_t cy = 0; cy < G.n[1]; ++cy)
        for (int64_t cx = 0; cx < G.n[0]; ++cx) {
            int64_t corner[4];
            int hit = 0;
            for (int c = 0; c < 4; ++c) {
                int64_t ix = cx + (c & 1), iy = cy + (c >> 1);
                ix = G.per[0] ? imod(ix, G.n[0]) : ix + G.g[0];
                iy = G.per[1] ? imod(iy, G.n[1]) : iy + G.g[1];
                corner[c] = iy * G.N[0] + ix;
                if (sd[corner[c]] <= 0.0) hit = 1;
            }
            if (hit)
                for (int c = 0; c < 4; ++c) mask[corner[c]] = 1;
        }
    /* 3. n = grad sd on masked nodes: (X - Q)/|X - Q| outside, (Q - X)/|X - Q|
     *    inside (pointing out of the obstacle); 0 on the boundary itself */
    for (int64_t j = 0; j < G.N[1]; ++j)
        for (int64_t i = 0; i < G.N[0]; ++i) {
            int64_t node = j * G.N[0] + i;
            double nx = 0.0, ny = 0.0;
            double d = fabs(sd[node]);
            if (mask[node] && d > 0.0) {
                double X = G.lo[0] + (double)(i - G.g[0]) * G.h;
                double Y = G.lo[1] + (double)(j - G.g[1]) * G.h;
                double s = sd[node] < 0.0 ? -1.0 : 1.0;
                nx = s * ((X - qx[node]) / d);
                ny = s * ((Y - qy[node]) / d);
            }
            normals[node] = nx;
            normals[nn + node] = ny;
        }
    free(qx);
    free(qy);
    return OR_OK;
}

/* Obstacle projection, eqs. normali1/normali2: subtract the inward part. */
void oracle_obstacle_project(int dim, const double* x, const double* n, double* out)
{
    double xn = 0.0;
    for (int a = 0; a < dim; ++a) xn += x[a] * n[a];
    double c = 0.5 * (xn - fabs(xn));
    for (int a = 0; a < dim; ++a) out[a] = x[a] - c * n[a];
}

/* Grid boundary conditions on one vector field of the nodes (Sec. 3 steps
 * iii and vii): kind 0 = momentum, 1 = force. */
static void grid_bc(oracle_sim* s, double* f[3], int kind)
{
    const geom* G = &s->G;
    const oracle_config* c = &s->cfg;
    for (int64_t i = 0; i < G->nnode; ++i) {
        int64_t ix[3] = { i % G->N[0], (i / G->N[0]) % G->N[1], i / ((int64_t)G->N[0] * G->N[1]) };
        if (s->mask[i]) {
            double vin[3], nn[3], vo[3];
            for (int a = 0; a < 3; ++a) { vin[a] = f[a][i]; nn[a] = s->nrm[a][i]; }
            oracle_obstacle_project(G->dim, vin, nn, vo);
            for (int a = 0; a < G->dim; ++a) f[a][i] = vo[a];
        }
        for (int a = 0; a < G->dim; ++a) {
            if (G->per[a]) continue;
            int64_t phys = ix[a] - G->g[a];
            for (int side = 0; side < 2; ++side) {
                int on = side == 0 ? (phys <= 0) : (phys >= G->n[a]);
                if (!on) continue;
                int bc = c->bc[2 * a + side];
                if (bc == OR_BC_WALL) {
                    f[a][i] = 0.0;
                } else if (bc == OR_BC_INFLOW) {
                    for (int b = 0; b < G->dim; ++b)
                        f[b][i] = (kind == 0) ? s->gm[i] * c->inflow_v[b] : 0.0;
                }
            }
        }
    }
}

static double pressure(const oracle_sim* s, int64_t k)
{
    return (s->cfg.gamma - 1.0) * s->rho[k] * s->E[k];
}

/* dt for the next step: after a step use_step_vmax = 1 takes the velocity
 * maximum recorded during the step; before the first step Vbar := V. */
static void cfl_from_state(oracle_sim* s, int use_step_vmax)
{
    double vmax = 0.0, cmax = 0.0;
    for (int64_t k = 0; k < s->np; ++k) {
        double v2 = 0.0;
        for (int a = 0; a < s->G.dim; ++a) v2 += s->v[a][k] * s->v[a][k];
        if (!use_step_vmax && sqrt(v2) > vmax) vmax = sqrt(v2);
        double c2 = s->cfg.gamma * pressure(s, k) / s->rho[k];
        double cs = sqrt(c2 > 0.0 ? c2 : 0.0);
        if (cs > cmax) cmax = cs;
    }
    if (use_step_vmax) vmax = s->vmax_step;
    double den = vmax + cmax;
    s->dt_next = den > 0.0 ? s->cfg.cfl * s->G.h / den : 0.0;
}

static double norm_d(double* const v[3], int d, int64_t k)
{
    double s = 0.0;
    for (int a = 0; a < d; ++a) s += v[a][k] * v[a][k];
    return sqrt(s);
}

int oracle_cfl_dt(oracle_sim* s, double* dt_out)
{
    if (!s || !dt_out) return OR_EINVAL;
    if (!s->started) cfl_from_state(s, 0);
    *dt_out = s->dt_next;
    return OR_OK;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* Salmon et al., SC'11: ten rounds of the Philox S-box on 4x32-bit words. */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static int first_inflow_face(const oracle_sim* s)
{
    for (int f = 0; f < 2 * s->G.dim; ++f)
        if (s->cfg.bc[f] == OR_BC_INFLOW) return f;
    return -1;
}

/* Particle recycling (Sec. 4.1, cylinder case): new position in the first
 * cell layer of the inflow face, other coordinates uniform; inflow state.
 * The draw is keyed by the particle's own recycle count, so a particle that
 * leaves one step earlier or later lands at the same place. */
static void recycle(oracle_sim* s, int64_t k, int face)
{
    const geom* G = &s->G; const oracle_config* c = &s->cfg;
    uint32_t ctr[4] = { s->gen[k], 0u, (uint32_t)s->id[k], (uint32_t)((uint64_t)s->id[k] >> 32) };
    s->gen[k] += 1;
    uint32_t key[2] = { (uint32_t)c->seed, (uint32_t)(c->seed >> 32) }, r[4];
    oracle_philox4x32_10(ctr, key, r);
    int af = face / 2, side = face % 2;
    for (int a = 0; a < G->dim; ++a) {
        double u = (double)(r[a] >> 8) * (1.0 / 16777216.0);
        if (a == af) s->x[a][k] = side == 0 ? G->lo[a] + u * G->h : G->hi[a] - G->h + u * G->h;
        else s->x[a][k] = G->lo[a] + u * (G->hi[a] - G->lo[a]);
        s->v[a][k] = c->inflow_v[a];
    }
    s->rho[k] = c->inflow_rho;
    s->E[k] = c->inflow_p / ((c->gamma - 1.0) * c->inflow_rho);
    s->Q[k] = 0.0;
}

static void keys_of_particles(oracle_sim* s)
{
    support sp; double xk[3];
    for (int64_t k = 0; k < s->np; ++k) {
        for (int a = 0; a < 3; ++a) xk[a] = (a < s->G.dim) ? s->x[a][k] : 0.0;
        particle_support(&s->G, xk, &sp);
        s->key[k] = key_of_spans(&s->G, sp.span);
    }
}

int oracle_stable_sort(int64_t n, const uint32_t* keys, int64_t nkeys, int64_t* perm, int64_t* start)
{
    /* Counting sort: count per key, exclusive prefix sum, then place particles
     * in their current order -- the per-cell lists of Sec. 3 step xii. */
    if (n < 0 || nkeys < 1 || !perm || !start) return OR_EINVAL;
    for (int64_t i = 0; i <= nkeys; ++i) start[i] = 0;
    for (int64_t k = 0; k < n; ++k) {
        if ((int64_t)keys[k] >= nkeys) return OR_EINVAL;
        start[keys[k] + 1]++;
    }
    for (int64_t i = 0; i < nkeys; ++i) start[i + 1] += start[i];
    int64_t* cur = (int64_t*)malloc((size_t)nkeys * sizeof(int64_t) + 8);
    if (!cur) return OR_ENOMEM;
    memcpy(cur, start, (size_t)nkeys * sizeof(int64_t));
    for (int64_t k = 0; k < n; ++k) perm[cur[keys[k]]++] = k;
    free(cur);
    return OR_OK;
}

/* Sec. 3 step xii: the per-cell lists rebuilt from the cells the particles
 * are now in.  Walk the particles in their current order and append each to
 * the list of its key; a particle re-created at the inflow during the step
 * (Sec. 4.1) is new in its cell and goes after the cell's other particles,
 * several of them by id.  perm[j] = current index of the particle placed at
 * j; start[K] = first position of key K (nkeys + 1 entries). */
int oracle_reorder(int64_t n, const uint32_t* keys, const uint8_t* recycled, const int64_t* ids,
                   int64_t nkeys, int64_t* perm, int64_t* start)
{
    if (n < 0 || nkeys < 1 || !perm || !start || (n > 0 && (!keys || !recycled || !ids))) return OR_EINVAL;
    for (int64_t i = 0; i <= nkeys; ++i) start[i] = 0;
    for (int64_t k = 0; k < n; ++k) {
        if ((int64_t)keys[k] >= nkeys) return OR_EINVAL;
        start[keys[k] + 1]++;
    }
    for (int64_t i = 0; i < nkeys; ++i) start[i + 1] += start[i];
    int64_t* cur = (int64_t*)malloc((size_t)nkeys * sizeof(int64_t) + 8);
    if (!cur) return OR_ENOMEM;
    memcpy(cur, start, (size_t)nkeys * sizeof(int64_t));
    /* the cell's stayers in current order */
    for (int64_t k = 0; k < n; ++k)
        if (!recycled[k]) perm[cur[keys[k]]++] = k;
    /* then its re-created particles: each goes after those of its cell with a
     * smaller id (insertion into the cell's tail, which is short) */
    for (int64_t k = 0; k < n; ++k) {
        if (!recycled[k]) continue;
        const uint32_t K = keys[k];
        int64_t j = cur[K]++;
        while (j > start[K] && recycled[perm[j - 1]] && ids[perm[j - 1]] > ids[k]) {
            perm[j] = perm[j - 1];
            --j;
        }
        perm[j] = k;
    }
    free(cur);
    return OR_OK;
}

static void permute_d(double* a, const int64_t* perm, int64_t n, double* tmp)
{
    for (int64_t j = 0; j < n; ++j) tmp[j] = a[perm[j]];
    memcpy(a, tmp, (size_t)n * sizeof(double));
}

/* Re-order the particle state by the lists of oracle_reorder. */
static int sort_particles(oracle_sim* s)
{
    keys_of_particles(s);
    int64_t n = s->np;
    int64_t* perm = (int64_t*)malloc((size_t)n * sizeof(int64_t) + 8);
    double* tmp = (double*)malloc((size_t)n * sizeof(double) + 8);
    if (!perm || !tmp) { free(perm); free(tmp); return OR_ENOMEM; }
    int st = oracle_reorder(n, s->key, s->recyc, s->id, s->G.nkey, perm, s->cellstart);
    if (st) { free(perm); free(tmp); return st; }
    for (int a = 0; a < 3; ++a) { permute_d(s->x[a], perm, n, tmp); permute_d(s->v[a], perm, n, tmp);
                                  permute_d(s->vbar[a], perm, n, tmp); }
    permute_d(s->M, perm, n, tmp); permute_d(s->rho, perm, n, tmp);
    permute_d(s->E, perm, n, tmp); permute_d(s->Q, perm, n, tmp);
    int64_t* ti = (int64_t*)tmp;   /* same width as double */
    for (int64_t j = 0; j < n; ++j) ti[j] = s->id[perm[j]];
    memcpy(s->id, ti, (size_t)n * sizeof(int64_t));
    uint32_t* tk = (uint32_t*)tmp;
    for (int64_t j = 0; j < n; ++j) tk[j] = s->key[perm[j]];
    memcpy(s->key, tk, (size_t)n * sizeof(uint32_t));
    for (int64_t j = 0; j < n; ++j) tk[j] = s->gen[perm[j]];
    memcpy(s->gen, tk, (size_t)n * sizeof(uint32_t));
    memset(s->recyc, 0, (size_t)n);
    free(perm); free(tmp);
    return OR_OK;
}

/* One pass of Algorithm 1 with time step dt. */
static int one_step(oracle_sim* s, double dt)
{
    const geom* G = &s->G; const oracle_config* c = &s->cfg;
    const int64_t np = s->np, nn = G->nnode;
    const int d = G->dim;
    const double gam = c->gamma;
    double* A[3] = { s->tmp_p[0], s->tmp_p[1], s->tmp_p[2] };

    /* (i) grid reset */
    memset(s->gm, 0, (size_t)nn * sizeof(double));
    for (int a = 0; a < 3; ++a) {
        memset(s->gmv[a], 0, (size_t)nn * sizeof(double));
        memset(s->gf[a], 0, (size_t)nn * sizeof(double));
        memset(s->gmv2[a], 0, (size_t)nn * sizeof(double));
    }
    /* (ii) m = P2G(I, M); mv_a = P2G(I, M V_a); f = P2GD(zeta/eta, P, Q, M, rho) */
    p2g(G, np, s->x, s->M, s->gm);
    for (int a = 0; a < d; ++a) {
        for (int64_t k = 0; k < np; ++k) s->coef[k] = s->M[k] * s->v[a][k];
        p2g(G, np, s->x, s->coef, s->gmv[a]);
    }
    for (int64_t k = 0; k < np; ++k) s->coef[k] = (pressure(s, k) + s->Q[k]) * s->M[k] / s->rho[k];
    p2gd(G, np, s->x, s->coef, s->gf);
    /* (iii) boundary conditions and obstacle treatment on mv and f */
    for (int a = 0; a < 3; ++a) {
        memcpy(s->bmv[a], s->gmv[a], (size_t)nn * sizeof(double));
        memcpy(s->bf[a], s->gf[a], (size_t)nn * sizeof(double));
    }
    grid_bc(s, s->bmv, 0);
    grid_bc(s, s->bf, 1);
    /* (iv) momentum update on the grid: mv' = mv + dt f */
    for (int a = 0; a < d; ++a)
        for (int64_t i = 0; i < nn; ++i) s->bmv[a][i] = s->bmv[a][i] + dt * s->bf[a][i];
    /* (v) Vbar = G2P(theta, mv', m); A = G2P(theta, f, m) */
    for (int a = 0; a < d; ++a) {
        theta(nn, s->bmv[a], s->gm, s->tmp_node);
        g2p(G, np, s->x, s->tmp_node, s->vbar[a]);
        theta(nn, s->bf[a], s->gm, s->tmp_node);
        g2p(G, np, s->x, s->tmp_node, A[a]);
    }
    /* (vi) V' = V + dt A */
    for (int a = 0; a < d; ++a)
        for (int64_t k = 0; k < np; ++k) s->v[a][k] = s->v[a][k] + dt * A[a][k];
    s->vmax_step = 0.0;
    for (int64_t k = 0; k < np; ++k) {
        double vb = norm_d(s->vbar, d, k), vn = norm_d(s->v, d, k);
        if (vb > s->vmax_step) s->vmax_step = vb;
        if (vn > s->vmax_step) s->vmax_step = vn;
    }
    /* (vii) mv = P2G(I, M V') */
    for (int a = 0; a < d; ++a) {
        for (int64_t k = 0; k < np; ++k) s->coef[k] = s->M[k] * s->v[a][k];
        p2g(G, np, s->x, s->coef, s->gmv2[a]);
    }
    /* (viii) boundary conditions on the new mv */
    for (int a = 0; a < 3; ++a) memcpy(s->bmv2[a], s->gmv2[a], (size_t)nn * sizeof(double));
    grid_bc(s, s->bmv2, 0);
    /* (ix) grad V_a = G2PD(theta, mv_a, m); then E, rho, p, q on particles */
    double* div = s->coef;
    for (int64_t k = 0; k < np; ++k) div[k] = 0.0;
    for (int a = 0; a < d; ++a) {
        theta(nn, s->bmv2[a], s->gm, s->tmp_node);
        g2pd(G, np, s->x, s->tmp_node, A);      /* A now holds grad V_a */
        for (int64_t k = 0; k < np; ++k) div[k] += A[a][k];
    }
    for (int64_t k = 0; k < np; ++k) {
        double P = pressure(s, k), Q = s->Q[k], rho = s->rho[k];
        double Enew = s->E[k] + dt * (-(P + Q) / rho) * div[k];
        double den = 1.0 + dt * div[k];
        if (!(den > 0.0)) return OR_ENONFINITE;
        double rnew = rho / den;
        double Pnew = (gam - 1.0) * rnew * Enew;
        double qnew = 0.0;
        if (div[k] < 0.0) {
            double c2 = gam * Pnew / rnew;
            double cs = sqrt(c2 > 0.0 ? c2 : 0.0);
            /* eq. muart read as the von Neumann-Richtmyer and Landshoff
             * terms it names, both proportional to the density */
            double t1 = G->h * div[k];
            qnew = rnew * (c->c0 * t1 * t1 - c->c1 * G->h * cs * div[k]);
        }
        s->E[k] = Enew; s->rho[k] = rnew; s->Q[k] = qnew;
        if (!isfinite(Enew) || !isfinite(rnew) || !isfinite(qnew)) return OR_ENONFINITE;
    }
    /* (x) move X' = X + dt Vbar, and (xi) the connectivity: particles that
     * leave the domain are wrapped (periodic), held at the wall, or recycled. */
    int inflow = first_inflow_face(s);
    for (int64_t k = 0; k < np; ++k) {
        double xo[3], xn[3];
        for (int a = 0; a < 3; ++a) { xo[a] = s->x[a][k]; xn[a] = xo[a]; }
        for (int a = 0; a < d; ++a) xn[a] = xo[a] + dt * s->vbar[a][k];
        for (int a = 0; a < d; ++a)
            if (!isfinite(xn[a])) return OR_ENONFINITE;
        /* a particle may cross at most one span per axis per step (Sec. 4.1) */
        for (int a = 0; a < d; ++a) {
            int64_t c0s = span_of_xi(G, a, (xo[a] - G->lo[a]) * G->inv_h);
            int64_t c1s = span_of_xi(G, a, (xn[a] - G->lo[a]) * G->inv_h);
            int64_t dd = c1s - c0s;
            if (dd < -1 || dd > 1) return OR_ECFL;
        }
        int out = 0;
        for (int a = 0; a < d; ++a) {
            if (G->per[a]) continue;
            if (xn[a] < G->lo[a] && c->bc[2 * a] == OR_BC_OUTFLOW) out = 1;
            if (xn[a] >= G->hi[a] && c->bc[2 * a + 1] == OR_BC_OUTFLOW) out = 1;
        }
        for (int a = 0; a < d; ++a) s->x[a][k] = xn[a];
        if (out && inflow >= 0) {
            recycle(s, k, inflow);
            s->recyc[k] = 1;
            double vi = norm_d(s->v, d, k);
            if (vi > s->vmax_step) s->vmax_step = vi;
            continue;
        }
        for (int a = 0; a < d; ++a) {
            double lo = G->lo[a], hi = G->hi[a], L = hi - lo;
            if (G->per[a]) {
                if (s->x[a][k] < lo) s->x[a][k] += L;
                else if (s->x[a][k] >= hi) s->x[a][k] -= L;
            } else {
                if (s->x[a][k] < lo) s->x[a][k] = lo;
                if (s->x[a][k] > hi) s->x[a][k] = hi;
            }
        }
    }
    return OR_OK;
}

int oracle_step(oracle_sim* s, int64_t nsteps, double dt, double t_end)
{
    if (!s || nsteps < 0) return OR_EINVAL;
    if (s->poisoned) return OR_ESTATE;
    if (!s->started) { cfl_from_state(s, 0); s->started = 1; }
    for (int64_t i = 0; i < nsteps; ++i) {
        if (t_end > 0.0 && s->t >= t_end) break;
        double h = dt > 0.0 ? dt : s->dt_next;
        if (!(h > 0.0)) { s->poisoned = 1; return OR_ENONFINITE; }
        int last = 0;
        if (t_end > 0.0 && s->t + h >= t_end) { h = t_end - s->t; last = 1; }
        int st = one_step(s, h);
        if (st) { s->poisoned = 1; return st; }
        s->step += 1;
        s->t = last ? t_end : s->t + h;
        /* (xii) optional reorder, (xiii) CFL check and time advance */
        if (s->cfg.sort_interval > 0 && s->step % s->cfg.sort_interval == 0) {
            st = sort_particles(s);
            if (st) { s->poisoned = 1; return st; }
        } else {
            keys_of_particles(s);
        }
        cfl_from_state(s, 1);
    }
    return OR_OK;
}

int64_t oracle_field_size(oracle_sim* s, int field)
{
    if (!s) return -1;
    int d = s->G.dim;
    switch (field) {
    case OR_F_X: case OR_F_V: case OR_F_VBAR: return d * s->np;
    case OR_F_M: case OR_F_RHO: case OR_F_E: case OR_F_P: case OR_F_Q: case OR_F_ID: case OR_F_KEY:
    case OR_F_GEN: return s->np;
    case OR_F_CELLSTART: return s->G.nkey + 1;
    case OR_F_GRID_M: return s->G.nnode;
    case OR_F_GRID_MV: case OR_F_GRID_F: case OR_F_GRID_MV2: return d * s->G.nnode;
    case OR_F_CLOCK: return 3;
    }
    return -1;
}

int oracle_read(oracle_sim* s, int field, double* out, int64_t count)
{
    if (!s || !out) return OR_EINVAL;
    int64_t need = oracle_field_size(s, field);
    if (need < 0 || count < need) return OR_EINVAL;
    int d = s->G.dim; int64_t np = s->np, nn = s->G.nnode;
    switch (field) {
    case OR_F_X: for (int a = 0; a < d; ++a) memcpy(out + a * np, s->x[a], np * sizeof(double)); break;
    case OR_F_V: for (int a = 0; a < d; ++a) memcpy(out + a * np, s->v[a], np * sizeof(double)); break;
    case OR_F_VBAR: for (int a = 0; a < d; ++a) memcpy(out + a * np, s->vbar[a], np * sizeof(double)); break;
    case OR_F_M: memcpy(out, s->M, np * sizeof(double)); break;
    case OR_F_RHO: memcpy(out, s->rho, np * sizeof(double)); break;
    case OR_F_E: memcpy(out, s->E, np * sizeof(double)); break;
    case OR_F_P: for (int64_t k = 0; k < np; ++k) out[k] = pressure(s, k); break;
    case OR_F_Q: memcpy(out, s->Q, np * sizeof(double)); break;
    case OR_F_ID: for (int64_t k = 0; k < np; ++k) out[k] = (double)s->id[k]; break;
    case OR_F_KEY: for (int64_t k = 0; k < np; ++k) out[k] = (double)s->key[k]; break;
    case OR_F_GEN: for (int64_t k = 0; k < np; ++k) out[k] = (double)s->gen[k]; break;
    case OR_F_CELLSTART: for (int64_t i = 0; i <= s->G.nkey; ++i) out[i] = (double)s->cellstart[i]; break;
    case OR_F_GRID_M: memcpy(out, s->gm, nn * sizeof(double)); break;
    case OR_F_GRID_MV: for (int a = 0; a < d; ++a) memcpy(out + a * nn, s->gmv[a], nn * sizeof(double)); break;
    case OR_F_GRID_F: for (int a = 0; a < d; ++a) memcpy(out + a * nn, s->gf[a], nn * sizeof(double)); break;
    case OR_F_GRID_MV2: for (int a = 0; a < d; ++a) memcpy(out + a * nn, s->gmv2[a], nn * sizeof(double)); break;
    case OR_F_CLOCK: out[0] = s->t; out[1] = s->started ? s->dt_next : 0.0; out[2] = (double)s->step;
        if (!s->started) { cfl_from_state(s, 0); out[1] = s->dt_next; } break;
    }
    return OR_OK;
}

int oracle_conservation(oracle_sim* s, double out[5])
{
    if (!s || !out) return OR_EINVAL;
    double m = 0.0, en = 0.0, mv[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k < s->np; ++k) {
        double v2 = 0.0;
        for (int a = 0; a < s->G.dim; ++a) { v2 += s->v[a][k] * s->v[a][k]; mv[a] += s->M[k] * s->v[a][k]; }
        m += s->M[k];
        en += s->M[k] * (s->E[k] + 0.5 * v2);
    }
    out[0] = m; out[1] = en; out[2] = mv[0]; out[3] = mv[1]; out[4] = mv[2];
    return OR_OK;
}

int oracle_sizes(oracle_sim* s, int64_t out[4])
{
    if (!s || !out) return OR_EINVAL;
    out[0] = s->np; out[1] = s->G.nnode; out[2] = s->G.nkey; out[3] = s->step;
    return OR_OK;
}

/* ------------------------------------------------- standalone unit pieces */

int oracle_keys(const oracle_config* cfg, int64_t n, const double* x, int prec32, uint32_t* keys)
{
    geom G;
    int st = geom_init(cfg, &G);
    if (st) return st;
    for (int64_t k = 0; k < n; ++k) {
        int64_t sp[3] = {0, 0, 0};
        for (int a = 0; a < G.dim; ++a) {
            int64_t c;
            if (prec32) {
                /* binary32: xi = (x - o) * (1/h), then floor(xi + 1/2) or floor(xi) */
                volatile float xf = (float)x[a * n + k], of = (float)G.lo[a], ih = (float)G.inv_h;
                volatile float d0 = xf - of;
                volatile float xi = d0 * ih;
                volatile float xs = (G.p == 2) ? xi + 0.5f : xi;
                c = (int64_t)floorf(xs);
                if (!G.per[a]) { if (c < 0) c = 0; if (c > G.S[a] - 1) c = G.S[a] - 1; }
            } else {
                c = span_of_xi(&G, a, (x[a * n + k] - G.lo[a]) * G.inv_h);
            }
            sp[a] = G.per[a] ? imod(c, G.n[a]) : c;
        }
        keys[k] = key_of_spans(&G, sp);
    }
    return OR_OK;
}

int oracle_p2g(const oracle_config* cfg, int64_t n, const double* x, const double* v,
               const double* mass, const double* rho, const double* e, const double* q,
               double* grid_m, double* grid_mv, double* grid_f)
{
    geom G;
    int st = geom_init(cfg, &G);
    if (st) return st;
    int d = G.dim; int64_t nn = G.nnode;
    double* xp[3] = { (double*)x, (double*)(x + n), (double*)(d == 3 ? x + 2 * n : x) };
    double* coef = (double*)malloc((size_t)n * sizeof(double) + 8);
    if (!coef) return OR_ENOMEM;
    memset(grid_m, 0, nn * sizeof(double));
    memset(grid_mv, 0, d * nn * sizeof(double));
    memset(grid_f, 0, d * nn * sizeof(double));
    p2g(&G, n, xp, mass, grid_m);
    for (int a = 0; a < d; ++a) {
        for (int64_t k = 0; k < n; ++k) coef[k] = mass[k] * v[a * n + k];
        p2g(&G, n, xp, coef, grid_mv + a * nn);
    }
    for (int64_t k = 0; k < n; ++k)
        coef[k] = ((cfg->gamma - 1.0) * rho[k] * e[k] + (q ? q[k] : 0.0)) * mass[k] / rho[k];
    double* fo[3] = { grid_f, grid_f + nn, d == 3 ? grid_f + 2 * nn : grid_f };
    p2gd(&G, n, xp, coef, fo);
    free(coef);
    return OR_OK;
}

/* Physical coordinate of a node from its storage index along axis a. */
static double node_coord(const geom* G, int a, int64_t i)
{
    return G->lo[a] + (double)(i - G->g[a]) * G->h;
}

int oracle_p2g_dense(const oracle_config* cfg, int64_t n, const double* x, const double* v,
                     const double* mass, const double* rho, const double* e, const double* q,
                     double* grid_m, double* grid_mv, double* grid_f)
{
    geom G;
    int st = geom_init(cfg, &G);
    if (st) return st;
    int d = G.dim; int64_t nn = G.nnode;
    for (int64_t i = 0; i < nn; ++i) {
        int64_t ix[3] = { i % G.N[0], (i / G.N[0]) % G.N[1], i / ((int64_t)G.N[0] * G.N[1]) };
        double sm = 0.0, smv[3] = {0, 0, 0}, sf[3] = {0, 0, 0};
        for (int64_t k = 0; k < n; ++k) {
            double N1[3], D1[3];
            for (int a = 0; a < 3; ++a) {
                if (a >= d) { N1[a] = 1.0; D1[a] = 0.0; continue; }
                double r = (x[a * n + k] - node_coord(&G, a, ix[a])) * G.inv_h;
                if (G.per[a]) r -= G.n[a] * floor(r / G.n[a] + 0.5);   /* nearest image */
                N1[a] = oracle_bspline_dense(G.p, r, &D1[a]);
            }
            double w = N1[0] * N1[1] * N1[2];
            if (w == 0.0 && D1[0] == 0.0 && D1[1] == 0.0 && D1[2] == 0.0) continue;
            double gw[3] = { D1[0] * N1[1] * N1[2] * G.inv_h, N1[0] * D1[1] * N1[2] * G.inv_h,
                             N1[0] * N1[1] * D1[2] * G.inv_h };
            double F = ((cfg->gamma - 1.0) * rho[k] * e[k] + (q ? q[k] : 0.0)) * mass[k] / rho[k];
            sm += mass[k] * w;
            for (int a = 0; a < d; ++a) { smv[a] += mass[k] * v[a * n + k] * w; sf[a] += F * gw[a]; }
        }
        grid_m[i] = sm;
        for (int a = 0; a < d; ++a) { grid_mv[a * nn + i] = smv[a]; grid_f[a * nn + i] = sf[a]; }
    }
    return OR_OK;
}

int oracle_p2g_fixed32(const oracle_config* cfg, int64_t n, const float* x, const float* v,
                       const float* mass, const float* rho, const float* e, const float* q,
                       const double unit[3], int64_t* grid_m, int64_t* grid_mv, int64_t* grid_f)
{
    /* The binary32 evaluation order of each contribution is part of the
     * fixed-point contract: xi = (x-o)*ih; span and offset fx; weights
     * t0=1.5-fx, w0=(t0*t0)*0.5, dw0=-t0; t1=fx-1, w1=0.75-t1*t1, dw1=-2*t1;
     * t2=fx-0.5, w2=(t2*t2)*0.5, dw2=t2 (degree 1: w=(1-fx, fx), dw=(-1, 1));
     * P=((g-1)*rho)*e, vol=M/rho, F=((P+q)*vol)*ih; yz=wy*wz, w=wx*yz,
     * gx=dwx*yz, gy=wx*(dwy*wz), gz=wx*(wy*dwz) (2D: w=wx*wy, gx=dwx*wy,
     * gy=wx*dwy); contributions M*w, (M*V_a)*w, F*g_a, each quantised as
     * llrintf(c * S) with S = (float)(2^32/unit). */
    geom G;
    int st = geom_init(cfg, &G);
    if (st) return st;
    int d = G.dim; int64_t nn = G.nnode;
    memset(grid_m, 0, nn * sizeof(int64_t));
    memset(grid_mv, 0, d * nn * sizeof(int64_t));
    memset(grid_f, 0, d * nn * sizeof(int64_t));
    volatile float Sm = (float)(4294967296.0 / unit[0]);
    volatile float Sv = (float)(4294967296.0 / unit[1]);
    volatile float Sf = (float)(4294967296.0 / unit[2]);
    volatile float ih = (float)G.inv_h, gm1 = (float)(cfg->gamma - 1.0);
    for (int64_t k = 0; k < n; ++k) {
        float w[3][3], dw[3][3]; int64_t idx[3][3]; int ns[3];
        for (int a = 0; a < 3; ++a) {
            if (a >= d) { ns[a] = 1; w[a][0] = 1.0f; dw[a][0] = 0.0f; idx[a][0] = 0; continue; }
            volatile float of = (float)G.lo[a];
            volatile float t = x[a * n + k] - of;
            volatile float xi = t * ih;
            volatile float xs = (G.p == 2) ? xi + 0.5f : xi;
            int64_t c = (int64_t)floorf(xs);
            if (!G.per[a]) { if (c < 0) c = 0; if (c > G.S[a] - 1) c = G.S[a] - 1; }
            int64_t b = c - (G.p == 2 ? 1 : 0);
            volatile float fx = xi - (float)b;
            if (G.p == 2) {
                volatile float t0 = 1.5f - fx, t1 = fx - 1.0f, t2 = fx - 0.5f;
                volatile float s0 = t0 * t0, s1 = t1 * t1, s2 = t2 * t2;
                w[a][0] = s0 * 0.5f; w[a][1] = 0.75f - s1; w[a][2] = s2 * 0.5f;
                dw[a][0] = -t0; dw[a][1] = -2.0f * t1; dw[a][2] = t2;
            } else {
                w[a][0] = 1.0f - fx; w[a][1] = fx; dw[a][0] = -1.0f; dw[a][1] = 1.0f;
            }
            ns[a] = G.p + 1;
            for (int j = 0; j < ns[a]; ++j) {
                int64_t phys = b + j;
                idx[a][j] = G.per[a] ? imod(phys, G.n[a]) : phys + G.g[a];
            }
        }
        volatile float M = mass[k], r = rho[k];
        volatile float P0 = gm1 * r;
        volatile float P = P0 * e[k];
        volatile float PQ = P + (q ? q[k] : 0.0f);
        volatile float vol = M / r;
        volatile float F0 = PQ * vol;
        volatile float F = F0 * ih;
        float MV[3];
        for (int a = 0; a < d; ++a) { volatile float t = M * v[a * n + k]; MV[a] = t; }
        for (int kz = 0; kz < ns[2]; ++kz)
            for (int ky = 0; ky < ns[1]; ++ky)
                for (int kx = 0; kx < ns[0]; ++kx) {
                    int64_t node = (idx[2][kz] * G.N[1] + idx[1][ky]) * G.N[0] + idx[0][kx];
                    volatile float wgt, g[3];
                    if (d == 3) {
                        volatile float yz = w[1][ky] * w[2][kz];
                        volatile float dyz = dw[1][ky] * w[2][kz];
                        volatile float ydz = w[1][ky] * dw[2][kz];
                        wgt = w[0][kx] * yz;
                        g[0] = dw[0][kx] * yz; g[1] = w[0][kx] * dyz; g[2] = w[0][kx] * ydz;
                    } else {
                        wgt = w[0][kx] * w[1][ky];
                        g[0] = dw[0][kx] * w[1][ky]; g[1] = w[0][kx] * dw[1][ky]; g[2] = 0.0f;
                    }
                    volatile float cm = M * wgt;
                    volatile float qm = cm * Sm;
                    grid_m[node] += llrintf(qm);
                    for (int a = 0; a < d; ++a) {
                        volatile float cv = MV[a] * wgt;
                        volatile float qv = cv * Sv;
                        grid_mv[a * nn + node] += llrintf(qv);
                        volatile float cf = F * g[a];
                        volatile float qf = cf * Sf;
                        grid_f[a * nn + node] += llrintf(qf);
                    }
                }
    }
    return OR_OK;
}

/* ------------------------------------------------ exact Riemann (Toro ch. 4) */

typedef struct { double r, u, p, c; } gstate;

/* Pressure function f_K(p) and derivative for side K: shock if p > p_K,
 * rarefaction otherwise. */
static double fK(double p, const gstate* K, double g, double* dfd)
{
    if (p > K->p) {
        double A = 2.0 / ((g + 1.0) * K->r), B = (g - 1.0) / (g + 1.0) * K->p;
        double q = sqrt(A / (p + B));
        *dfd = q * (1.0 - 0.5 * (p - K->p) / (B + p));
        return (p - K->p) * q;
    }
    double e = (g - 1.0) / (2.0 * g);
    *dfd = 1.0 / (K->r * K->c) * pow(p / K->p, -(g + 1.0) / (2.0 * g));
    return 2.0 * K->c / (g - 1.0) * (pow(p / K->p, e) - 1.0);
}

int oracle_riemann_exact(double g, double rl, double ul, double pl, double rr, double ur, double pr,
                         int64_t n, const double* s, double* rho, double* u, double* p, double star[2])
{
    gstate L = { rl, ul, pl, sqrt(g * pl / rl) }, R = { rr, ur, pr, sqrt(g * pr / rr) };
    if (2.0 / (g - 1.0) * (L.c + R.c) <= ur - ul) return OR_EINVAL;   /* vacuum */
    /* Newton iteration on f(p) = f_L(p) + f_R(p) + (u_R - u_L) = 0 from the
     * two-rarefaction estimate. */
    double e = (g - 1.0) / (2.0 * g);
    double ps = pow((L.c + R.c - 0.5 * (g - 1.0) * (ur - ul)) / (L.c / pow(pl, e) + R.c / pow(pr, e)), 1.0 / e);
    if (!(ps > 0.0)) ps = 1e-8;
    for (int it = 0; it < 100; ++it) {
        double dl, dr;
        double f = fK(ps, &L, g, &dl) + fK(ps, &R, g, &dr) + (ur - ul);
        double pn = ps - f / (dl + dr);
        if (pn < 1e-14) pn = 1e-14;
        double ch = 2.0 * fabs(pn - ps) / (pn + ps);
        ps = pn;
        if (ch < 1e-15) break;
    }
    double dl, dr;
    double us = 0.5 * (ul + ur) + 0.5 * (fK(ps, &R, g, &dr) - fK(ps, &L, g, &dl));
    star[0] = ps; star[1] = us;
    double gp = (g + 1.0) / (2.0 * g), gm = (g - 1.0) / (2.0 * g), gr = (g - 1.0) / (g + 1.0);
    for (int64_t i = 0; i < n; ++i) {
        double S = s[i], rr0, uu, pp;
        if (S <= us) {                          /* left of the contact */
            if (ps > pl) {                      /* left shock */
                double SL = ul - L.c * sqrt(gp * ps / pl + gm);
                if (S <= SL) { rr0 = rl; uu = ul; pp = pl; }
                else { rr0 = rl * (ps / pl + gr) / (gr * ps / pl + 1.0); uu = us; pp = ps; }
            } else {                            /* left rarefaction */
                double csl = L.c * pow(ps / pl, gm);
                double SHL = ul - L.c, STL = us - csl;
                if (S <= SHL) { rr0 = rl; uu = ul; pp = pl; }
                else if (S >= STL) { rr0 = rl * pow(ps / pl, 1.0 / g); uu = us; pp = ps; }
                else {
                    double f = 2.0 / (g + 1.0) + gr / L.c * (ul - S);
                    rr0 = rl * pow(f, 2.0 / (g - 1.0));
                    uu = 2.0 / (g + 1.0) * (L.c + 0.5 * (g - 1.0) * ul + S);
                    pp = pl * pow(f, 1.0 / e);
                }
            }
        } else {                                /* right of the contact */
            if (ps > pr) {                      /* right shock */
                double SR = ur + R.c * sqrt(gp * ps / pr + gm);
                if (S >= SR) { rr0 = rr; uu = ur; pp = pr; }
                else { rr0 = rr * (ps / pr + gr) / (gr * ps / pr + 1.0); uu = us; pp = ps; }
            } else {                            /* right rarefaction */
                double csr = R.c * pow(ps / pr, gm);
                double SHR = ur + R.c, STR = us + csr;
                if (S >= SHR) { rr0 = rr; uu = ur; pp = pr; }
                else if (S <= STR) { rr0 = rr * pow(ps / pr, 1.0 / g); uu = us; pp = ps; }
                else {
                    double f = 2.0 / (g + 1.0) - gr / R.c * (ur - S);
                    rr0 = rr * pow(f, 2.0 / (g - 1.0));
                    uu = 2.0 / (g + 1.0) * (-R.c + 0.5 * (g - 1.0) * ur + S);
                    pp = pr * pow(f, 1.0 / e);
                }
            }
        }
        rho[i] = rr0; u[i] = uu; p[i] = pp;
    }
    return OR_OK;
}
