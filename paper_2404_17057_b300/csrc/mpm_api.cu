// mpm_api.cu -- the C ABI of include/mpm.h on top of the sm_103a kernels.
//
// Host side only: argument checks, device memory, the order of the launches
// of one step (Algorithm 1), CUDA-graph replay of whole steps, and reads.
// Every arithmetic step of the method runs in the kernels of
// mpm_kernels.cuh / mpm_sort.cuh.
#include "mpm.h"
#include "mpm_kernels.cuh"
#include "mpm_fast.cuh"
#include "mpm_sort.cuh"
#include "mpm_reorder.cuh"
#include "mpm_batch_kernels.cuh"

#include <cuda_runtime.h>

#include <type_traits>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace mpm;

namespace {

constexpr int kThreads = 256;
constexpr int kPhases = 5;   // P2G, grid+G2P+P2G, G2PD+update, time advance, re-order

struct Buffers {             // one copy of the particle state (type-erased)
    void* x[3] = {nullptr, nullptr, nullptr};
    void* v[3] = {nullptr, nullptr, nullptr};
    void* M = nullptr;
    void* rho = nullptr;
    void* E = nullptr;
    void* Q = nullptr;
    uint32_t* id = nullptr;
    uint32_t* key = nullptr;
    uint32_t* gen = nullptr;
};

struct ProfStep {
    cudaEvent_t ev[kPhases + 1];
};

}  // namespace

struct Vtbl;

struct mpm_sim {
    mpm_config cfg;
    Geom G;
    const Vtbl* vt = nullptr;
    size_t rsize = 4, asize = 4;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int sms = 148;                 // streaming multiprocessors of the device
    int64_t np = 0;
    int cur = 0;
    Buffers buf[2];
    void* grid = nullptr;          // m, mv[d], f[d], mv2[d] of type A, contiguous
    size_t grid_bytes = 0;
    uint8_t* mask = nullptr;
    void* nrm = nullptr;           // d x nodes of type R
    Clock* clk = nullptr;
    uint32_t* cs[2] = {nullptr, nullptr};   // per-tile cell starts of the tiles in buffer b
    uint8_t* tpar[2] = {nullptr, nullptr};  // buffer of each tile before step parity 0 / 1
    uint32_t* tbase = nullptr;              // tile regions (ntiles + 1 slots)
    uint32_t* tbase_next = nullptr;         // regions of a relayout
    uint32_t* tcount = nullptr;             // particles of each tile after a step
    uint32_t* dirty = nullptr;              // tiles whose span lists change in a step
    uint32_t* toff = nullptr;               // particles before each tile (reads; ntiles + 1)
    int64_t nslots = 0;                     // slots of each particle buffer
    uint32_t* col_tiles = nullptr;          // colour passes: tiles grouped by colour
    std::vector<int> col_off;               // colour c: col_tiles[col_off[c] .. col_off[c+1])
    uint32_t* count = nullptr;              // particles per new span (step re-order)
    uint32_t* cscan_part = nullptr;         // scan partials over the tiles
    uint2* far = nullptr;                   // recycled particles of a step
    uint32_t far_cap = 0;
    unsigned long long* ring = nullptr;     // per tile: ring parts entered in a step
    int mwords = 0;
    double* cons_part = nullptr;
    double* cons_out = nullptr;
    bool started = false, poisoned = false, stepped = false, cfl_done = false;
    std::vector<void*> allocs;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool graph_ok = true;
    bool profiling = false;
    std::vector<ProfStep> prof;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[8] = {0};
    int64_t prof_launch[8] = {0};
    int64_t launches = 0;
    std::string err;
    mpm_batch* batch = nullptr;     // set while the simulation is a member of a batch
};

namespace {

thread_local std::string g_static_err;

mpm_status fail(mpm_sim* s, mpm_status st, const std::string& msg)
{
    if (s) s->err = msg; else g_static_err = msg;
    return st;
}

mpm_status cuda_fail(mpm_sim* s, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (s) s->poisoned = true;
    return fail(s, MPM_ECUDA, m);
}

#define CK(call, what)                                 \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, what); \
    } while (0)

void* dalloc(mpm_sim* s, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (s->cfg.alloc) {
        p = s->cfg.alloc(bytes, s->cfg.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) s->allocs.push_back(p);
    return p;
}

void dfree(mpm_sim* s, void* p)
{
    if (!p) return;
    for (size_t i = 0; i < s->allocs.size(); ++i)
        if (s->allocs[i] == p) { s->allocs.erase(s->allocs.begin() + i); break; }
    if (s->cfg.free) s->cfg.free(p, s->cfg.alloc_ctx);
    else cudaFree(p);
}

unsigned nblk(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

__global__ void k_zero(uint4* p, int64_t n16, const int* active)
{
    if (active && !*active) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_uint4(0, 0, 0, 0);
}

}  // namespace

// ------------------------------------------------------ per-type dispatch

struct Vtbl {
    void (*step_kernels)(mpm_sim* s, int phase_mask_first, cudaStream_t st);
    void (*keys)(mpm_sim* s, int b, cudaStream_t st);
    void (*gather)(mpm_sim* s, int from, const uint32_t* perm, const uint32_t* skeys, const int* active,
                   cudaStream_t st);
    void (*cfl_init)(mpm_sim* s, cudaStream_t st);
    void (*cons)(mpm_sim* s, cudaStream_t st);
    // the particle field `f` (0 x, 1 v, 2 M, 3 rho, 4 E, 5 Q, 6 id, 7 gen;
    // component a) in key order into out (device); needs s->toff
    void (*compact)(mpm_sim* s, int f, int a, void* out, cudaStream_t st);
    void (*tile_counts)(mpm_sim* s, uint32_t* counts, cudaStream_t st);
    void (*spread)(mpm_sim* s, const uint32_t* cc, cudaStream_t st);
    void (*from_double)(const double* in, void* out, int64_t n, cudaStream_t st);
    void (*from_float)(const float* in, void* out, int64_t n, cudaStream_t st);
    cudaError_t (*set_smem)(const Geom& G);
    size_t (*smem)(const Geom& G, int kernel);
    void (*reorder)(mpm_sim* s, cudaStream_t st);
    // batched execution: descriptor of a member, stage launches of a group
    size_t bdesc_size;
    void (*bdesc_fill)(const mpm_sim* s, void* out);
    void (*blaunch)(int stage, const void* desc, const TileRef* tl, int ntl, size_t smem, int flags, cudaStream_t st);
    cudaError_t (*bset_smem)(const size_t smem[4]);
};

namespace {

template <class R>
Particles<R> parts(const Buffers& b)
{
    Particles<R> p;
    for (int a = 0; a < 3; ++a) {
        p.x[a] = (R*)b.x[a];
        p.v[a] = (R*)b.v[a];
    }
    p.M = (R*)b.M;
    p.rho = (R*)b.rho;
    p.E = (R*)b.E;
    p.Q = (R*)b.Q;
    p.id = b.id;
    p.key = b.key;
    p.gen = b.gen;
    return p;
}

template <class A, class R>
Grid<A, R> grid_view(const mpm_sim* s)
{
    Grid<A, R> g;
    const int64_t nn = s->G.nnode_p;
    const int d = s->G.dim;
    A* base = (A*)s->grid;
    g.m = base;
    for (int a = 0; a < 3; ++a) {
        g.mv[a] = a < d ? base + (1 + a) * nn : nullptr;
        g.f[a] = a < d ? base + (1 + d + a) * nn : nullptr;
        g.mv2[a] = a < d ? base + (1 + 2 * d + a) * nn : nullptr;
        g.nrm[a] = (s->nrm && a < d) ? (const R*)s->nrm + a * nn : nullptr;
    }
    g.mask = s->mask;
    return g;
}

void order_offsets(mpm_sim* s, cudaStream_t st);

// The particle state with the tile-buffer table of step parity b.
template <class R>
TileState<R> tstate(const mpm_sim* s, int b)
{
    TileState<R> ts;
    ts.pt = parts<R>(s->buf[0]);
    ts.cs[0] = s->cs[0];
    ts.cs[1] = s->cs[1];
    ts.tpar = s->tpar[b];
    return ts;
}

// Colour passes of a coloured simulation (one pass over all tiles otherwise).
int ncolours(const mpm_sim* s) { return s->col_off.empty() ? 1 : (int)s->col_off.size() - 1; }
const uint32_t* colour_tiles(const mpm_sim* s, int c) { return s->col_off.empty() ? nullptr : s->col_tiles + s->col_off[c]; }
unsigned colour_blocks(const mpm_sim* s, int c)
{
    return s->col_off.empty() ? (unsigned)s->G.ntiles : (unsigned)(s->col_off[c + 1] - s->col_off[c]);
}

template <int D, int P, class R, class A>
struct Impl {
    // The single-precision float-atomic path (and its colour passes) runs the
    // span-per-thread kernels of mpm_fast.cuh; the fixed-point and FP64 paths
    // run the 2D span kernels below, or the generic ones (3D, small grids).
    static constexpr bool kFast = std::is_same<R, float>::value && std::is_same<A, float>::value;
    // G2PD reads the grid once into its window, so the fixed-point mode runs
    // the single-precision kernel too (the int64 sums are converted there)
    static constexpr bool kFast3 = std::is_same<R, float>::value;
    // 2D fixed point and FP64: P2G and grid + G2P + P2G by the span-per-lane
    // kernels with 64-bit register sums
    static constexpr bool kSpan2d = D == 2 && ((std::is_same<R, float>::value && std::is_same<A, long long>::value) ||
                                               (std::is_same<R, double>::value && std::is_same<A, double>::value));
    static_assert(!(kSpan2d && kFast), "one P2G kernel per mode");
    // ... always in fixed point; in FP64 on grids of at least two tiles per
    // SM (smaller FP64 grids keep the particle-parallel generic kernels, whose
    // 256 threads finish a tile sooner; fixed point gains at every size)
    static bool span2d(const mpm_sim* s) { return std::is_same<A, long long>::value || s->G.ntiles >= 2 * s->sms; }
    static size_t smem(const Geom& G, int kernel)
    {
        const size_t W = (size_t)G.Wvol;
        if (kernel == 2 && kFast3) return (D == 3 ? 24 : 16) * W;
        if (kFast) {
            if (kernel == 0) return (1 + 2 * D) * W * sizeof(float);
            return (K2Cfg<D>::kHeadFloats + tile_cs_words(G)) * sizeof(float) + 2 * D * W * sizeof(float);
        }
        if (kernel == 0) return (1 + 2 * D) * W * sizeof(A);
        if (kernel == 1) return align16(D * W * sizeof(R)) + D * W * sizeof(A);
        return 2 * D * W * sizeof(R);
    }
    // Shared-memory limits of the single-problem kernels: the device's whole
    // shared memory (a limit, not an allocation), so that simulations with
    // different tiles never lower each other's limit; G's needs must fit.
    static cudaError_t set_smem(const Geom& G)
    {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        auto allow = [&](const void* f, size_t need) -> cudaError_t {
            cudaFuncAttributes fa;
            cudaError_t e = cudaFuncGetAttributes(&fa, f);
            if (e != cudaSuccess) return e;
            const int room = optin - (int)fa.sharedSizeBytes;
            if ((int)need > room) return cudaErrorInvalidValue;
            return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
        };
        cudaError_t e = allow((const void*)k_reorder<D, R>, reorder_smem(G));
        if (e != cudaSuccess) return e;
        if constexpr (kFast3) e = allow((const void*)k_g2pd_fast<D, P, A>, smem(G, 2));
        else e = allow((const void*)k_g2pd<D, P, R, A>, smem(G, 2));
        if (e != cudaSuccess) return e;
        if constexpr (kFast3 && D == 3 && P == 2) {
            const int shape = static_tile(G);
            const bool wl = all_walls(G);
            if (shape == 1)
                e = allow(wl ? (const void*)k_g2pd_fast<3, 2, A, 8, 8, 8, true> : (const void*)k_g2pd_fast<3, 2, A, 8, 8, 8>,
                          smem(G, 2));
            if (shape == 2)
                e = allow(wl ? (const void*)k_g2pd_fast<3, 2, A, 16, 8, 4, true> : (const void*)k_g2pd_fast<3, 2, A, 16, 8, 4>,
                          smem(G, 2));
            if (e != cudaSuccess) return e;
        }
        if constexpr (kFast) {
            const void* f[6] = {(const void*)k_p2g_span<D, P, true, true>, (const void*)k_p2g_span<D, P, false, true>,
                                (const void*)k_p2g_span<D, P, true, false>, (const void*)k_p2g_span<D, P, false, false>,
                                (const void*)k_grid_g2p_span<D, P, true>, (const void*)k_grid_g2p_span<D, P, false>};
            const size_t z[6] = {smem(G, 0), smem(G, 0), smem(G, 0), smem(G, 0), smem(G, 1), smem(G, 1)};
            for (int i = 0; i < 6; ++i)
                if ((e = allow(f[i], z[i])) != cudaSuccess) return e;
            if constexpr (D == 3 && P == 2) {
                const void* g[8] = {(const void*)k_p2g_span<3, 2, true, true, 8, 8, 8>,
                                    (const void*)k_p2g_span<3, 2, false, true, 8, 8, 8>,
                                    (const void*)k_grid_g2p_span<3, 2, true, 8, 8, 8>,
                                    (const void*)k_grid_g2p_span<3, 2, false, 8, 8, 8>,
                                    (const void*)k_p2g_span<3, 2, true, true, 16, 8, 4>,
                                    (const void*)k_p2g_span<3, 2, false, true, 16, 8, 4>,
                                    (const void*)k_grid_g2p_span<3, 2, true, 16, 8, 4>,
                                    (const void*)k_grid_g2p_span<3, 2, false, 16, 8, 4>};
                const int st = static_tile(G);
                for (int i = 0; i < 4 && st > 0; ++i)
                    if ((e = allow(g[4 * (st - 1) + i], smem(G, i < 2 ? 0 : 1))) != cudaSuccess) return e;
            }
            return cudaSuccess;
        } else {
            if constexpr (kSpan2d) {
                if ((e = allow((const void*)k_p2g_span2d<P, R, A>, smem(G, 0))) != cudaSuccess) return e;
                if ((e = allow((const void*)k_grid_g2p_span2d<P, R, A>, smem(G, 1))) != cudaSuccess) return e;
            }
            if ((e = allow((const void*)k_p2g<D, P, R, A>, smem(G, 0))) != cudaSuccess) return e;
            return allow((const void*)k_grid_g2p<D, P, R, A>, smem(G, 1));
        }
    }
    // which bit 0: zero + P2G, bit 1: grid + G2P + P2G, bit 2: G2PD + update
    static void step_kernels(mpm_sim* s, int which, cudaStream_t st)
    {
        const Geom& G = s->G;
        const TileState<R> ts = tstate<R>(s, s->cur);
        Grid<A, R> gr = grid_view<A, R>(s);
        const Reorder ro = {s->count, s->far, s->far_cap, s->mwords, s->ring, s->dirty};
        if (which & 1) {
            k_zero<<<std::min<int64_t>(nblk(s->grid_bytes / 16), s->sms * 8), kThreads, 0, st>>>(
                (uint4*)s->grid, (int64_t)(s->grid_bytes / 16), &s->clk->active);
            if constexpr (kFast) {
                const FieldPtrs o = p2g_fields(gr);
                const bool per = G.per[0] | G.per[1] | G.per[2];
                for (int c = 0; c < ncolours(s); ++c) {
                    const uint32_t* tl = colour_tiles(s, c);
                    const unsigned nb = colour_blocks(s, c);
                    if (nb == 0) continue;
                    const bool col = p2g_columns(G);
                    if constexpr (D == 3 && P == 2) {
                        // compile-time tile edges for the common shapes
                        const int shape = static_tile(G);
                        if (shape == 1 && per)
                            k_p2g_span<3, 2, true, true, 8, 8, 8><<<nb, kP2GThreads, smem(G, 0), st>>>(G, ts, o, s->clk, tl);
                        else if (shape == 1)
                            k_p2g_span<3, 2, false, true, 8, 8, 8><<<nb, kP2GThreads, smem(G, 0), st>>>(G, ts, o, s->clk, tl);
                        else if (shape == 2 && per)
                            k_p2g_span<3, 2, true, true, 16, 8, 4><<<nb, kP2GThreads, smem(G, 0), st>>>(G, ts, o, s->clk, tl);
                        else if (shape == 2)
                            k_p2g_span<3, 2, false, true, 16, 8, 4><<<nb, kP2GThreads, smem(G, 0), st>>>(G, ts, o, s->clk, tl);
                        if (shape > 0) continue;
                    }
                    if (per && col) k_p2g_span<D, P, true, true><<<nb, kP2GThreads, smem(G, 0), st>>>(G, ts, o, s->clk, tl);
                    else if (col) k_p2g_span<D, P, false, true><<<nb, kP2GThreads, smem(G, 0), st>>>(G, ts, o, s->clk, tl);
                    else if (per) k_p2g_span<D, P, true, false><<<nb, kP2GThreads, smem(G, 0), st>>>(G, ts, o, s->clk, tl);
                    else k_p2g_span<D, P, false, false><<<nb, kP2GThreads, smem(G, 0), st>>>(G, ts, o, s->clk, tl);
                }
                s->launches += ncolours(s) - 1;
            } else if (kSpan2d && span2d(s)) {
                k_p2g_span2d<P, R, A><<<G.ntiles, kP2GSpan2dThreads, smem(G, 0), st>>>(G, ts, gr, s->clk);
            } else {
                k_p2g<D, P, R, A><<<G.ntiles, kThreads, smem(G, 0), st>>>(G, ts, gr, s->clk);
            }
            s->launches += 2;
        }
        if (which & 2) {
            if constexpr (kFast) {
                const FieldPtrs o = g2p_fields(gr);
                const bool per = G.per[0] | G.per[1] | G.per[2];
                for (int c = 0; c < ncolours(s); ++c) {
                    const uint32_t* tl = colour_tiles(s, c);
                    const unsigned nb = colour_blocks(s, c);
                    if (nb == 0) continue;
                    if constexpr (D == 3 && P == 2) {
                        // compile-time tile edges for the common shapes
                        const int shape = static_tile(G);
                        const unsigned nt = K2Cfg<3>::kThreads;
                        if (shape == 1 && per)
                            k_grid_g2p_span<3, 2, true, 8, 8, 8><<<nb, nt, smem(G, 1), st>>>(G, ts, gr, o, s->clk, tl);
                        else if (shape == 1)
                            k_grid_g2p_span<3, 2, false, 8, 8, 8><<<nb, nt, smem(G, 1), st>>>(G, ts, gr, o, s->clk, tl);
                        else if (shape == 2 && per)
                            k_grid_g2p_span<3, 2, true, 16, 8, 4><<<nb, nt, smem(G, 1), st>>>(G, ts, gr, o, s->clk, tl);
                        else if (shape == 2)
                            k_grid_g2p_span<3, 2, false, 16, 8, 4><<<nb, nt, smem(G, 1), st>>>(G, ts, gr, o, s->clk, tl);
                        if (shape > 0) continue;
                    }
                    if (per)
                        k_grid_g2p_span<D, P, true><<<nb, K2Cfg<D>::kThreads, smem(G, 1), st>>>(G, ts, gr, o, s->clk,
                                                                                                tl);
                    else
                        k_grid_g2p_span<D, P, false><<<nb, K2Cfg<D>::kThreads, smem(G, 1), st>>>(G, ts, gr, o, s->clk,
                                                                                                 tl);
                }
                s->launches += ncolours(s) - 1;
            } else if (kSpan2d && span2d(s)) {
                k_grid_g2p_span2d<P, R, A><<<G.ntiles, kG2PSpan2dThreads, smem(G, 1), st>>>(G, ts, gr, s->clk);
            } else {
                k_grid_g2p<D, P, R, A><<<G.ntiles, kThreads, smem(G, 1), st>>>(G, ts, gr, s->clk);
            }
            s->launches += 1;
        }
        if (which & 4) {
            int shape = 0;
            if constexpr (kFast3 && D == 3 && P == 2) {
                // compile-time tile edges for the common shapes
                shape = static_tile(G);
                const bool wl = all_walls(G);
                if (shape == 1 && wl)
                    k_g2pd_fast<3, 2, A, 8, 8, 8, true><<<G.ntiles, kG2PDThreads, smem(G, 2), st>>>(G, ts, gr, s->clk, ro);
                else if (shape == 1)
                    k_g2pd_fast<3, 2, A, 8, 8, 8><<<G.ntiles, kG2PDThreads, smem(G, 2), st>>>(G, ts, gr, s->clk, ro);
                else if (shape == 2 && wl)
                    k_g2pd_fast<3, 2, A, 16, 8, 4, true><<<G.ntiles, kG2PDThreads, smem(G, 2), st>>>(G, ts, gr, s->clk, ro);
                else if (shape == 2)
                    k_g2pd_fast<3, 2, A, 16, 8, 4><<<G.ntiles, kG2PDThreads, smem(G, 2), st>>>(G, ts, gr, s->clk, ro);
            }
            if (shape == 0) {
                if constexpr (kFast3)
                    k_g2pd_fast<D, P, A><<<G.ntiles, kG2PDThreads, smem(G, 2), st>>>(G, ts, gr, s->clk, ro);
                else
                    k_g2pd<D, P, R, A><<<G.ntiles, kThreads, smem(G, 2), st>>>(G, ts, gr, s->clk, ro);
            }
            s->launches += 1;
        }
    }
    static ReorderArgs<R> rargs(const mpm_sim* s, int b)
    {
        ReorderArgs<R> a;
        a.pt = parts<R>(s->buf[0]);
        a.nslots = (uint32_t)s->nslots;
        a.cs[0] = s->cs[0];
        a.cs[1] = s->cs[1];
        a.tpar_old = s->tpar[b];
        a.tpar_new = s->tpar[1 - b];
        a.tbase = s->tbase;
        a.tbase_next = s->tbase_next;
        a.tcount = s->tcount;
        a.ro = {s->count, s->far, s->far_cap, s->mwords, s->ring, s->dirty};
        a.clk = s->clk;
        return a;
    }
    // Pass 0 over the changed tiles; the relayout kernels return at once
    // unless a tile overflowed its region.
    static void reorder(mpm_sim* s, cudaStream_t st)
    {
        const Geom& G = s->G;
        const ReorderArgs<R> a = rargs(s, s->cur);
        const unsigned nb = (unsigned)std::min<int64_t>(G.ntiles, (int64_t)s->sms * kReorderBlocksPerSM);
        k_reorder<D, R><<<nb, kReorderThreads, reorder_smem(G), st>>>(G, a, 0);
        k_consolidate<D, R><<<nb, kReorderThreads, 0, st>>>(G, a);
        k_relayout_bases<<<1, 1024, 0, st>>>(s->tcount, G.ntiles, s->tbase_next, s->clk);
        k_reorder<D, R><<<nb, kReorderThreads, reorder_smem(G), st>>>(G, a, 1);
        k_reorder_done<<<nblk(G.ntiles * 32), kThreads, 0, st>>>(G, a.ro, s->clk, s->tbase, s->tbase_next);
        s->launches += 5;
    }
    // m, mv[D], f[D] (P2G) and mv2[D] (grid + G2P + P2G) are consecutive
    // arrays of nnode_p nodes in the grid allocation (grid_view)
    static FieldPtrs p2g_fields(const Grid<A, R>& gr)
    {
        return FieldPtrs{(float*)gr.m, (int64_t)(gr.mv[0] - gr.m)};
    }
    static FieldPtrs g2p_fields(const Grid<A, R>& gr)
    {
        return FieldPtrs{(float*)gr.mv2[0], (int64_t)(gr.mv2[1] - gr.mv2[0])};
    }
    static void bdesc_fill(const mpm_sim* s, void* out)
    {
        BatchProb<R, A> d;
        memset(&d, 0, sizeof d);
        d.G = s->G;
        d.pt = parts<R>(s->buf[0]);
        d.gr = grid_view<A, R>(s);
        if constexpr (kFast) {
            d.p2g_out = p2g_fields(d.gr);
            d.g2p_out = g2p_fields(d.gr);
        }
        d.nslots = (uint32_t)s->nslots;
        d.cs[0] = s->cs[0];
        d.cs[1] = s->cs[1];
        d.tpar[0] = s->tpar[0];
        d.tpar[1] = s->tpar[1];
        d.tbase = s->tbase;
        d.tbase_next = s->tbase_next;
        d.tcount = s->tcount;
        d.ro = {s->count, s->far, s->far_cap, s->mwords, s->ring, s->dirty};
        d.np = s->np;
        d.clk = s->clk;
        memcpy(out, &d, sizeof d);
    }
    // stage 0: P2G, 1: grid + G2P + P2G, 2: G2PD + update, 3: re-order of
    // the changed tiles, 4 and 5: relayout (consolidation, rebuild).
    // flags: 1 = a periodic axis, 2 = P2G walks span columns (p2g_columns)
    static void blaunch(int stage, const void* dv, const TileRef* tl, int ntl, size_t sm, int flags, cudaStream_t st)
    {
        const bool per = (flags & 1) != 0;
        const BatchProb<R, A>* d = static_cast<const BatchProb<R, A>*>(dv);
        if (ntl <= 0) return;
        if (stage == 3 || stage == 5) {
            kb_reorder<D, R, A><<<ntl, kReorderThreads, sm, st>>>(d, tl, stage == 5 ? 1 : 0);
            return;
        }
        if (stage == 4) {
            kb_consolidate<D, R, A><<<ntl, kReorderThreads, 0, st>>>(d, tl);
            return;
        }
        if (stage == 2) {
            if constexpr (kFast3) kb_g2pd_fast<D, P, A><<<ntl, kG2PDThreads, sm, st>>>(d, tl);
            else kb_g2pd<D, P, R, A><<<ntl, kThreads, sm, st>>>(d, tl);
            return;
        }
        if constexpr (kFast) {
            if (stage == 0) {
                const bool col = (flags & 2) != 0;
                if (per && col) kb_p2g_span<D, P, true, true><<<ntl, kP2GThreads, sm, st>>>(d, tl);
                else if (col) kb_p2g_span<D, P, false, true><<<ntl, kP2GThreads, sm, st>>>(d, tl);
                else if (per) kb_p2g_span<D, P, true, false><<<ntl, kP2GThreads, sm, st>>>(d, tl);
                else kb_p2g_span<D, P, false, false><<<ntl, kP2GThreads, sm, st>>>(d, tl);
            } else {
                if (per) kb_grid_g2p_span<D, P, true><<<ntl, K2Cfg<D>::kThreads, sm, st>>>(d, tl);
                else kb_grid_g2p_span<D, P, false><<<ntl, K2Cfg<D>::kThreads, sm, st>>>(d, tl);
            }
        } else if constexpr (kSpan2d) {
            if (stage == 0) kb_p2g_span2d<P, R, A><<<ntl, kP2GSpan2dThreads, sm, st>>>(d, tl);
            else kb_grid_g2p_span2d<P, R, A><<<ntl, kG2PSpan2dThreads, sm, st>>>(d, tl);
        } else {
            if (stage == 0) kb_p2g<D, P, R, A><<<ntl, kThreads, sm, st>>>(d, tl);
            else kb_grid_g2p<D, P, R, A><<<ntl, kThreads, sm, st>>>(d, tl);
        }
    }
    // Allow every batched kernel the device's whole shared memory (a limit,
    // not an allocation: each launch asks for what its group needs), so that
    // groups and batches with different tiles never undercut each other;
    // fails if a group needs more than a kernel can have.
    static cudaError_t bset_smem(const size_t sm[4])
    {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        auto allow = [&](const void* f, size_t need) -> cudaError_t {
            cudaFuncAttributes fa;
            cudaError_t e = cudaFuncGetAttributes(&fa, f);
            if (e != cudaSuccess) return e;
            const int room = optin - (int)fa.sharedSizeBytes;
            if ((int)need > room) return cudaErrorInvalidValue;
            return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
        };
        cudaError_t e = allow((const void*)kb_reorder<D, R, A>, sm[3]);
        if (e != cudaSuccess) return e;
        if constexpr (kFast3) e = allow((const void*)kb_g2pd_fast<D, P, A>, sm[2]);
        else e = allow((const void*)kb_g2pd<D, P, R, A>, sm[2]);
        if (e != cudaSuccess) return e;
        if constexpr (kFast) {
            const void* f[6] = {(const void*)kb_p2g_span<D, P, true, true>, (const void*)kb_p2g_span<D, P, false, true>,
                                (const void*)kb_p2g_span<D, P, true, false>, (const void*)kb_p2g_span<D, P, false, false>,
                                (const void*)kb_grid_g2p_span<D, P, true>, (const void*)kb_grid_g2p_span<D, P, false>};
            const size_t z[6] = {sm[0], sm[0], sm[0], sm[0], sm[1], sm[1]};
            for (int i = 0; i < 6; ++i)
                if ((e = allow(f[i], z[i])) != cudaSuccess) return e;
            return cudaSuccess;
        } else {
            if constexpr (kSpan2d) {
                if ((e = allow((const void*)kb_p2g_span2d<P, R, A>, sm[0])) != cudaSuccess) return e;
                return allow((const void*)kb_grid_g2p_span2d<P, R, A>, sm[1]);
            }
            if ((e = allow((const void*)kb_p2g<D, P, R, A>, sm[0])) != cudaSuccess) return e;
            return allow((const void*)kb_grid_g2p<D, P, R, A>, sm[1]);
        }
    }
    static void keys(mpm_sim* s, int b, cudaStream_t st)
    {
        if (s->np == 0) return;
        k_keys<D, P, R><<<nblk(s->np), kThreads, 0, st>>>(s->G, parts<R>(s->buf[b]), s->np);
        s->launches += 1;
    }
    static void gather(mpm_sim* s, int from, const uint32_t* perm, const uint32_t* sk, const int* active,
                       cudaStream_t st)
    {
        if (s->np == 0) return;
        k_gather<D, R><<<nblk(s->np), kThreads, 0, st>>>(parts<R>(s->buf[from]), parts<R>(s->buf[1 - from]), perm,
                                                         sk, s->np, active);
        s->launches += 1;
    }
    static void cfl_init(mpm_sim* s, cudaStream_t st)
    {
        unsigned nb = std::max(1u, std::min(nblk(s->np), (unsigned)s->sms * 8u));
        order_offsets(s, st);
        k_cfl_init<D, R><<<nb, kThreads, 0, st>>>(s->G, tstate<R>(s, s->cur), s->toff, s->np, s->clk);
        k_cfl_init_finish<<<1, 1, 0, st>>>(s->clk, s->G.cfl * s->G.h);
        s->launches += 2;
    }
    static void cons(mpm_sim* s, cudaStream_t st)
    {
        const int nb = 1024;
        order_offsets(s, st);
        k_cons_partial<D, R><<<nb, 256, 0, st>>>(s->G, tstate<R>(s, s->cur), s->toff, s->np, s->cons_part);
        k_cons_final<<<1, kConsThreads, 0, st>>>(s->cons_part, nb, s->cons_out);
        s->launches += 2;
    }
    static void from_double(const double* in, void* out, int64_t n, cudaStream_t st)
    {
        if (n > 0) k_from_double<R><<<nblk(n), kThreads, 0, st>>>(in, (R*)out, n);
    }
    static void from_float(const float* in, void* out, int64_t n, cudaStream_t st)
    {
        if (n > 0) k_from_float<R><<<nblk(n), kThreads, 0, st>>>(in, (R*)out, n);
    }
    static void compact(mpm_sim* s, int f, int a, void* out, cudaStream_t st)
    {
        const TileState<R> ts = tstate<R>(s, s->cur);
        const unsigned nb = std::max(1u, std::min(nblk(s->np), (unsigned)s->sms * 16u));
        const Particles<R>& p = ts.pt;
        if (f <= 5) {
            const R* src = f == 0 ? p.x[a] : f == 1 ? p.v[a] : f == 2 ? p.M : f == 3 ? p.rho : f == 4 ? p.E : p.Q;
            k_compact<R, R><<<nb, kThreads, 0, st>>>(s->G, ts, s->toff, src, (R*)out, s->np);
        } else {
            k_compact<uint32_t, R><<<nb, kThreads, 0, st>>>(s->G, ts, s->toff, f == 6 ? p.id : p.gen, (uint32_t*)out,
                                                            s->np);
        }
        s->launches += 1;
    }
    static void tile_counts(mpm_sim* s, uint32_t* counts, cudaStream_t st)
    {
        k_tile_counts<R><<<nblk(s->G.ntiles), kThreads, 0, st>>>(s->G, tstate<R>(s, s->cur), counts);
        s->launches += 1;
    }
    // the compact sorted state of buffer 1 (cell starts cc) into the regions
    // of buffer 0; every tile in buffer 0
    static void spread(mpm_sim* s, const uint32_t* cc, cudaStream_t st)
    {
        const unsigned nb = (unsigned)std::min<int64_t>(s->G.ntiles, (int64_t)s->sms * 8);
        k_spread<D, R><<<nb, kThreads, 0, st>>>(s->G, parts<R>(s->buf[1]), parts<R>(s->buf[0]), cc, s->tbase,
                                                s->cs[0]);   // compact order at the start of buffer 1 -> regions of 0
        s->launches += 1;
    }
};

template <int D, int P, class R, class A>
const Vtbl* vtbl_of()
{
    typedef Impl<D, P, R, A> I;
    static const Vtbl v = {I::step_kernels, I::keys,    I::gather,          I::cfl_init,
                           I::cons,         I::compact, I::tile_counts,     I::spread,
                           I::from_double,  I::from_float, I::set_smem, I::smem, I::reorder,
                           sizeof(BatchProb<R, A>), I::bdesc_fill, I::blaunch, I::bset_smem};
    return &v;
}

template <int D, int P>
const Vtbl* vtbl_prec(int prec)
{
    if (prec == MPM_FP32 || prec == MPM_FP32_COLOURED) return vtbl_of<D, P, float, float>();
    if (prec == MPM_FP32_FIXED64) return vtbl_of<D, P, float, long long>();
    return vtbl_of<D, P, double, double>();
}

const Vtbl* select_vtbl(int d, int p, int prec)
{
    if (d == 2) return p == 1 ? vtbl_prec<2, 1>(prec) : vtbl_prec<2, 2>(prec);
    return p == 1 ? vtbl_prec<3, 1>(prec) : vtbl_prec<3, 2>(prec);
}

// ------------------------------------------------------------- geometry

mpm_status make_geom(const mpm_config* c, Geom* G, std::string* why)
{
    memset(G, 0, sizeof(*G));
    if (c->dim != 2 && c->dim != 3) { *why = "dim must be 2 or 3"; return MPM_EINVAL; }
    if (c->degree != 1 && c->degree != 2) { *why = "degree must be 1 or 2"; return MPM_EINVAL; }
    if (!(c->h > 0.0) || !std::isfinite(c->h)) { *why = "h must be > 0"; return MPM_EINVAL; }
    if (!(c->gamma > 1.0)) { *why = "gamma must be > 1"; return MPM_EINVAL; }
    if (!(c->cfl > 0.0)) { *why = "cfl must be > 0"; return MPM_EINVAL; }
    if (c->precision < 0 || c->precision > 3) { *why = "bad precision"; return MPM_EINVAL; }
    if (c->sort_interval != 1) { *why = "sort_interval must be 1 (tiled kernels need key order)"; return MPM_EUNSUPPORTED; }
    G->dim = c->dim;
    G->p = c->degree;
    G->h = c->h;
    G->inv_h = 1.0 / c->h;
    int64_t nkey = 1, nnode = 1;
    int tvol = 1, wvol = 1, ntiles = 1;
    for (int a = 0; a < 3; ++a) {
        if (a >= c->dim) {
            G->n[a] = G->S[a] = G->N[a] = G->T[a] = G->nt[a] = G->W[a] = 1;
            continue;
        }
        int bl = c->bc[2 * a], bh = c->bc[2 * a + 1];
        if (bl < 0 || bl > 3 || bh < 0 || bh > 3) { *why = "bad boundary condition"; return MPM_EINVAL; }
        if ((bl == MPM_BC_PERIODIC) != (bh == MPM_BC_PERIODIC)) { *why = "periodic faces come in pairs"; return MPM_EINVAL; }
        if (c->n[a] < 1 || c->n[a] > (1 << 20)) { *why = "bad cell count"; return MPM_EINVAL; }
        G->n[a] = c->n[a];
        G->per[a] = bl == MPM_BC_PERIODIC;
        if (G->per[a] && G->p == 2 && c->n[a] < 2) { *why = "a periodic axis needs 2 cells for degree 2"; return MPM_EINVAL; }
        G->S[a] = G->per[a] ? c->n[a] : (G->p == 2 ? c->n[a] + 1 : c->n[a]);
        G->N[a] = G->per[a] ? c->n[a] : c->n[a] + 2 * G->p - 1;
        G->g[a] = G->per[a] ? 0 : G->p - 1;
        static const int def3[3] = {16, 8, 4}, def2[3] = {32, 8, 1};
        G->T[a] = c->tile[a] > 0 ? c->tile[a] : (c->dim == 3 ? def3[a] : def2[a]);
        if (G->T[a] > 64 || (G->T[a] & (G->T[a] - 1))) { *why = "tile edges must be powers of two <= 64"; return MPM_EINVAL; }
        while ((1 << G->tsh[a]) < G->T[a]) ++G->tsh[a];
        G->nt[a] = (G->S[a] + G->T[a] - 1) / G->T[a];
        G->W[a] = G->T[a] + G->p;
        if (c->precision == MPM_FP32_COLOURED) {
            // same-colour tiles are two apart: their windows (tile + degree
            // nodes) must not meet, nor may a window wrap onto itself
            if (G->T[a] < G->p) { *why = "colouring needs tile edges >= degree"; return MPM_EUNSUPPORTED; }
            if (G->per[a] && (G->n[a] % G->T[a] != 0 || G->n[a] < 2 * G->T[a])) {
                *why = "colouring needs a periodic axis of at least two whole tiles";
                return MPM_EUNSUPPORTED;
            }
        }
        G->lo[a] = c->origin[a];
        G->hi[a] = c->origin[a] + c->n[a] * c->h;
    }
    G->inv_w[0] = 1.0f / (float)G->W[0];
    G->inv_w[1] = 1.0f / (float)G->W[1];
    for (int a = 0; a < 3; ++a) {
        tvol *= G->T[a];
        wvol *= G->W[a];
        ntiles *= G->nt[a];
        nnode *= G->N[a];
    }
    nkey = (int64_t)ntiles * tvol;
    if (nkey >= (int64_t)0x7FFFFFFFLL) { *why = "too many spans for 31-bit keys"; return MPM_EINVAL; }
    if (tvol < 32) { *why = "a tile must hold at least 32 spans"; return MPM_EINVAL; }
    G->Tvol = tvol;
    G->Wvol = wvol;
    G->ntiles = ntiles;
    G->nkey = nkey;
    G->nnode = nnode;
    G->pitch = (G->N[0] + 3) & ~3;
    G->nnode_p = (int64_t)G->pitch * G->N[1] * G->N[2];
    for (int f = 0; f < 6; ++f) G->bc[f] = f < 2 * c->dim ? c->bc[f] : MPM_BC_WALL;
    G->inflow_face = -1;
    for (int f = 0; f < 2 * c->dim; ++f)
        if (c->bc[f] == MPM_BC_INFLOW) { G->inflow_face = f; break; }
    G->gamma = c->gamma;
    G->c0 = c->c0;
    G->c1 = c->c1;
    G->cfl = c->cfl;
    G->inflow_rho = c->inflow_rho;
    G->inflow_p = c->inflow_p;
    for (int a = 0; a < 3; ++a) G->inflow_v[a] = a < c->dim ? c->inflow_v[a] : 0.0;
    if (G->inflow_face >= 0) {
        if (!(c->inflow_rho > 0.0)) { *why = "inflow_rho must be > 0"; return MPM_EINVAL; }
        G->inflow_e = c->inflow_p / ((c->gamma - 1.0) * c->inflow_rho);
    }
    G->seed = c->seed;
    for (int i = 0; i < 3; ++i) {
        double u = c->fixed_unit[i] > 0.0 ? c->fixed_unit[i] : 1.0;
        G->qscale[i] = (float)(4294967296.0 / u);
        G->dqscale[i] = (float)(u / 4294967296.0);
    }
    return MPM_OK;
}

// Two buffers of n slots per field, in one array of 2 n (buffer 1 from slot
// n), so that absolute slots address either buffer.
mpm_status alloc_particles(mpm_sim* s, int64_t n, Buffers nb[2])
{
    const int d = s->G.dim;
    const size_t rb = (size_t)n * s->rsize, ub = (size_t)n * 4;
    auto two = [&](void*& p0, void*& p1, size_t bytes) {
        p0 = dalloc(s, 2 * bytes);
        p1 = p0 ? (void*)((char*)p0 + bytes) : nullptr;
        return p0 != nullptr;
    };
    bool ok = true;
    for (int a = 0; a < d; ++a) {
        ok = ok && two(nb[0].x[a], nb[1].x[a], rb);
        ok = ok && two(nb[0].v[a], nb[1].v[a], rb);
    }
    ok = ok && two(nb[0].M, nb[1].M, rb) && two(nb[0].rho, nb[1].rho, rb) && two(nb[0].E, nb[1].E, rb) &&
         two(nb[0].Q, nb[1].Q, rb);
    void *i0 = nullptr, *i1 = nullptr, *k0 = nullptr, *k1 = nullptr, *g0 = nullptr, *g1 = nullptr;
    ok = ok && two(i0, i1, ub) && two(k0, k1, ub) && two(g0, g1, ub);
    nb[0].id = (uint32_t*)i0;
    nb[1].id = (uint32_t*)i1;
    nb[0].key = (uint32_t*)k0;
    nb[1].key = (uint32_t*)k1;
    nb[0].gen = (uint32_t*)g0;
    nb[1].gen = (uint32_t*)g1;
    return ok ? MPM_OK : MPM_ENOMEM;
}

// Buffer 1 lives inside buffer 0's allocations.
void free_particles(mpm_sim* s, Buffers b[2])
{
    for (int a = 0; a < 3; ++a) { dfree(s, b[0].x[a]); dfree(s, b[0].v[a]); }
    dfree(s, b[0].M); dfree(s, b[0].rho); dfree(s, b[0].E); dfree(s, b[0].Q);
    dfree(s, b[0].id); dfree(s, b[0].key); dfree(s, b[0].gen);
    b[0] = Buffers();
    b[1] = Buffers();
}

void drop_graphs(mpm_sim* s)
{
    for (int b = 0; b < 2; ++b)
        if (s->graph[b]) { cudaGraphExecDestroy(s->graph[b]); s->graph[b] = nullptr; }
}

// Scratch of the LSD radix sort used for the arbitrary initial order.
struct RadixScratch {
    uint32_t* skeys[2] = {nullptr, nullptr};
    uint32_t* sidx[2] = {nullptr, nullptr};
    uint32_t* hist = nullptr;
    uint32_t* part = nullptr;
    int passes = 0, bits = 0;
};

// Particles before each tile in key order (s->toff, ntiles + 1 entries).
void order_offsets(mpm_sim* s, cudaStream_t st)
{
    s->vt->tile_counts(s, s->toff, st);
    scan_exclusive(s->toff, s->toff, s->G.ntiles, s->cscan_part, 1, st, &s->launches);
}

// Regions for the tile counts in s->tcount: region_slots each, in tile order.
__global__ void k_region_bases(const uint32_t* tcount, int ntiles, uint32_t* tbase)
{
    relayout_bases_block(tcount, ntiles, tbase);
}

// Initial order of the particles of buffer 0 (any order, slots [0, n)): LSD
// radix passes over (key, index), a gather into buffer 1 (compact key order)
// and its cell starts cc (nkey + 1 entries), then every tile spread into its
// region of buffer 0.
void launch_sort(mpm_sim* s, const RadixScratch& rs, uint32_t* cc, cudaStream_t st)
{
    const int64_t n = s->np;
    const Geom& G = s->G;
    if (n > 0) {
        const unsigned nb = (unsigned)((n + kSortTile - 1) / kSortTile);
        const uint32_t* kin = s->buf[0].key;
        const uint32_t* iin = nullptr;
        int o = 0;
        for (int pass = 0; pass < rs.passes; ++pass) {
            const int shift = pass * rs.bits;
            k_radix_hist<<<nb, kSortThreads, 0, st>>>(kin, n, shift, rs.bits, rs.hist, nullptr);
            scan_exclusive(rs.hist, rs.hist, (int64_t)(1 << rs.bits) * nb, rs.part, 0, st, &s->launches);
            k_radix_scatter<<<nb, kSortThreads, 0, st>>>(kin, iin, rs.skeys[o], rs.sidx[o], n, shift, rs.bits, rs.hist,
                                                          nullptr, pass == 0);
            s->launches += 2;
            kin = rs.skeys[o];
            iin = rs.sidx[o];
            o ^= 1;
        }
        s->vt->gather(s, 0, iin, nullptr, nullptr, st);
        k_cell_start<<<nblk(n + 1), kThreads, 0, st>>>(kin, n, G.nkey, cc, nullptr);
    } else {
        k_cell_start<<<1, kThreads, 0, st>>>(nullptr, 0, G.nkey, cc, nullptr);
    }
    k_tile_counts_compact<<<nblk(G.ntiles), kThreads, 0, st>>>(cc, G.ntiles, G.Tvol, s->tcount);
    k_region_bases<<<1, 1024, 0, st>>>(s->tcount, G.ntiles, s->tbase);
    s->vt->spread(s, cc, st);
    cudaMemsetAsync(s->tpar[0], 0, (size_t)G.ntiles, st);
    cudaMemsetAsync(s->tpar[1], 0, (size_t)G.ntiles, st);
    s->launches += 3;
    s->cur = 0;
}

// Per-step re-order (Sec. 3 step xii): the G2PD step has written each
// particle's new key, counted the particles of every new span and marked the
// changed tiles; every changed tile moves into its other buffer (or the
// whole state is laid out again if one outgrew its region).  Swaps s->cur
// (the tile-buffer table in use).
void launch_reorder(mpm_sim* s, cudaStream_t st)
{
    if (s->np == 0) return;
    s->vt->reorder(s, st);
    s->cur ^= 1;
}

// One whole step (Algorithm 1) on the stream; phase events if profiling.
void launch_step(mpm_sim* s, cudaStream_t st, ProfStep* ps)
{
    if (ps) cudaEventRecord(ps->ev[0], st);
    k_prepare<<<1, 1, 0, st>>>(s->clk);
    s->launches += 1;
    s->vt->step_kernels(s, 1, st);
    if (ps) cudaEventRecord(ps->ev[1], st);
    s->vt->step_kernels(s, 2, st);
    if (ps) cudaEventRecord(ps->ev[2], st);
    s->vt->step_kernels(s, 4, st);
    if (ps) cudaEventRecord(ps->ev[3], st);
    k_finalize<<<1, 1, 0, st>>>(s->clk, s->G.cfl * s->G.h);
    s->launches += 1;
    if (ps) cudaEventRecord(ps->ev[4], st);
    launch_reorder(s, st);
    if (ps) cudaEventRecord(ps->ev[5], st);
}

mpm_status check_device_errors(mpm_sim* s)
{
    Clock c;
    CK(cudaMemcpyAsync(&c, s->clk, sizeof(Clock), cudaMemcpyDeviceToHost, s->stream), "read clock");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    if (c.err) {
        s->poisoned = true;
        if (c.err & ERR_CFL) return fail(s, MPM_ECFL, "a particle crossed more than one span in one step");
        if (c.err & ERR_NONFINITE) return fail(s, MPM_ENONFINITE, "non-finite state or 1 + dt div(v) <= 0");
        if (c.err & ERR_TIMEOUT) return fail(s, MPM_ETIMEOUT, "a bounded device wait expired");
        return fail(s, MPM_ESTATE, "internal: particle outside its tile (order lost)");
    }
    return MPM_OK;
}

cudaEvent_t pool_event(mpm_sim* s)
{
    if (!s->ev_pool.empty()) {
        cudaEvent_t e = s->ev_pool.back();
        s->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

mpm_status collect_profile(mpm_sim* s)
{
    if (s->prof.empty()) return MPM_OK;
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    for (auto& ps : s->prof) {
        float ms;
        for (int k = 0; k < kPhases; ++k) {
            if (cudaEventElapsedTime(&ms, ps.ev[k], ps.ev[k + 1]) == cudaSuccess) s->prof_ms[k] += ms;
        }
        if (cudaEventElapsedTime(&ms, ps.ev[0], ps.ev[kPhases]) == cudaSuccess) s->prof_ms[5] += ms;
        for (int k = 0; k <= kPhases; ++k) s->ev_pool.push_back(ps.ev[k]);
    }
    s->prof.clear();
    cudaGetLastError();
    return MPM_OK;
}

// Colour passes of MPM_FP32_COLOURED: the tiles grouped by the parities of
// their coordinates, so that two tiles of one colour are at least two tiles
// apart along some axis and their node windows (tile + degree nodes) never
// meet; on a periodic axis with an odd tile count the last tile takes a
// third colour (tile 0 is its neighbour across the seam).  Empty colours are
// dropped; each list is in tile order.
mpm_status build_colours(mpm_sim* s)
{
    const Geom& G = s->G;
    int nc[3];
    for (int a = 0; a < 3; ++a) nc[a] = G.nt[a] < 2 ? 1 : ((G.per[a] && (G.nt[a] & 1)) ? 3 : 2);
    auto colour = [&](int a, int t) { return nc[a] == 1 ? 0 : (nc[a] == 3 && t == G.nt[a] - 1 ? 2 : (t & 1)); };
    std::vector<std::vector<uint32_t>> lists((size_t)nc[0] * nc[1] * nc[2]);
    for (int tz = 0; tz < G.nt[2]; ++tz)
        for (int ty = 0; ty < G.nt[1]; ++ty)
            for (int tx = 0; tx < G.nt[0]; ++tx) {
                const int c = (colour(2, tz) * nc[1] + colour(1, ty)) * nc[0] + colour(0, tx);
                lists[c].push_back((uint32_t)((tz * G.nt[1] + ty) * G.nt[0] + tx));
            }
    std::vector<uint32_t> flat;
    flat.reserve(G.ntiles);
    s->col_off.assign(1, 0);
    for (const auto& l : lists) {
        if (l.empty()) continue;
        flat.insert(flat.end(), l.begin(), l.end());
        s->col_off.push_back((int)flat.size());
    }
    s->col_tiles = (uint32_t*)dalloc(s, flat.size() * 4);
    if (!s->col_tiles) return fail(s, MPM_ENOMEM, "device allocation failed");
    CK(cudaMemcpy(s->col_tiles, flat.data(), flat.size() * 4, cudaMemcpyHostToDevice), "colour list");
    return MPM_OK;
}

}  // namespace

static mpm_status set_obstacle(mpm_sim* s, const uint8_t* mask, const double* normals);

// ================================================================== ABI

extern "C" {

mpm_status mpm_create(const mpm_config* cfg, mpm_sim** out)
{
    if (!out) return fail(nullptr, MPM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, MPM_EINVAL, "cfg is NULL");
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
        return fail(nullptr, MPM_EINVAL, "alloc and free hooks come together");
    mpm_sim* s = new (std::nothrow) mpm_sim();
    if (!s) return fail(nullptr, MPM_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    std::string why;
    mpm_status st = make_geom(cfg, &s->G, &why);
    if (st != MPM_OK) { delete s; return fail(nullptr, st, why); }
    s->vt = select_vtbl(cfg->dim, cfg->degree, cfg->precision);
    s->rsize = cfg->precision == MPM_FP64 ? 8 : 4;
    s->asize = (cfg->precision == MPM_FP32 || cfg->precision == MPM_FP32_COLOURED) ? 4 : 8;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(nullptr, MPM_ECUDA, "no CUDA device");
    }
    if (cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess || s->sms < 1) {
        cudaGetLastError();
        s->sms = 148;
    }
    if (cfg->stream) {
        s->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return fail(nullptr, MPM_ECUDA, "stream creation failed");
        }
        s->own_stream = true;
    }
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    for (int k = 0; k < 3; ++k)
        if ((int)s->vt->smem(s->G, k) > smem_optin) {
            mpm_destroy(s);
            return fail(nullptr, MPM_EINVAL, "tile too large for shared memory");
        }
    if ((int)reorder_smem(s->G) + 128 > smem_optin || reorder_ranges(s->G) > kReorderMaxRanges) {
        mpm_destroy(s);
        return fail(nullptr, MPM_EINVAL, "tile too large for the re-order");
    }
    cudaError_t e = s->vt->set_smem(s->G);
    if (e != cudaSuccess) {
        mpm_destroy(s);
        return fail(nullptr, MPM_ECUDA, std::string("shared memory attribute: ") + cudaGetErrorString(e));
    }
    const int d = s->G.dim;
    s->grid_bytes = align16((size_t)(1 + 3 * d) * (size_t)s->G.nnode_p * s->asize);
    s->grid = dalloc(s, s->grid_bytes);
    s->clk = (Clock*)dalloc(s, sizeof(Clock));
    const int64_t nt = s->G.ntiles;
    const size_t csb = (size_t)(tile_cs0(s->G, nt) + 1) * 4;
    const size_t ntb = (size_t)(nt + 1) * 4;
    s->cs[0] = (uint32_t*)dalloc(s, csb);
    s->cs[1] = (uint32_t*)dalloc(s, csb);
    s->count = (uint32_t*)dalloc(s, (size_t)(s->G.nkey + 1) * 4);
    s->cscan_part = (uint32_t*)dalloc(s, (size_t)scan_blocks(nt + 1) * 4);
    s->tpar[0] = (uint8_t*)dalloc(s, (size_t)nt);
    s->tpar[1] = (uint8_t*)dalloc(s, (size_t)nt);
    s->tbase = (uint32_t*)dalloc(s, ntb);
    s->tbase_next = (uint32_t*)dalloc(s, ntb);
    s->tcount = (uint32_t*)dalloc(s, ntb);
    s->dirty = (uint32_t*)dalloc(s, ntb);
    s->toff = (uint32_t*)dalloc(s, ntb);
    s->mwords = (reorder_ranges(s->G) + 63) / 64;
    const size_t ringb = (size_t)s->G.ntiles * s->mwords * 8;
    s->ring = (unsigned long long*)dalloc(s, ringb);
    s->cons_part = (double*)dalloc(s, 1024 * 5 * sizeof(double));
    s->cons_out = (double*)dalloc(s, 8 * sizeof(double));
    if (!s->grid || !s->clk || !s->cs[0] || !s->cs[1] || !s->count || !s->cscan_part || !s->ring ||
        !s->cons_part || !s->cons_out || !s->tpar[0] || !s->tpar[1] || !s->tbase || !s->tbase_next || !s->tcount ||
        !s->dirty || !s->toff) {
        mpm_destroy(s);
        return fail(nullptr, MPM_ENOMEM, "device allocation failed");
    }
    if (cudaMemsetAsync(s->grid, 0, s->grid_bytes, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->clk, 0, sizeof(Clock), s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->cs[0], 0, csb, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->cs[1], 0, csb, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->count, 0, (size_t)(s->G.nkey + 1) * 4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->tpar[0], 0, (size_t)nt, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->tpar[1], 0, (size_t)nt, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->tbase, 0, ntb, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->tcount, 0, ntb, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->dirty, 0, ntb, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->ring, 0, ringb, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess) {
        cudaGetLastError();
        mpm_destroy(s);
        return fail(nullptr, MPM_ECUDA, "device initialisation failed");
    }
    if (cfg->precision == MPM_FP32_COLOURED) {
        st = build_colours(s);
        if (st != MPM_OK) {
            const std::string m = s->err;
            mpm_destroy(s);
            return fail(nullptr, st, m);
        }
    }
    *out = s;
    return MPM_OK;
}

namespace {

// mpm_add_particles and mpm_add_particles_f32: the host arrays hold doubles,
// or floats when f32.
mpm_status add_particles(mpm_sim* s, int64_t n, const void* x, const void* v, const void* mass, const void* rho,
                         const void* e, bool f32)
{
    if (!s) return fail(nullptr, MPM_EINVAL, "sim is NULL");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    if (s->poisoned) return fail(s, MPM_ESTATE, "simulation is poisoned: " + s->err);
    if (s->started) return fail(s, MPM_ESTATE, "particles can only be added before the first step");
    if (n < 0) return fail(s, MPM_EINVAL, "n < 0");
    if (n == 0) return MPM_OK;
    if (!x || !v || !mass || !rho || !e) return fail(s, MPM_EINVAL, "NULL input array");
    if (s->np + n > (int64_t)0x7FFFFFFF) return fail(s, MPM_EINVAL, "too many particles");
    const Geom& G = s->G;
    const int d = G.dim;
    const int64_t np = s->np + n;
    // every tile's region holds region_slots(its count) <= 2 count + 95
    // slots, now and after any relayout: buffers of 2 np + 95 ntiles slots
    const int64_t nslots = (2 * np + 95 * (int64_t)G.ntiles + 31) & ~(int64_t)31;
    if (2 * nslots > (int64_t)0xFFFFFFFF) return fail(s, MPM_EINVAL, "too many particles");
    Buffers nb[2];
    mpm_status st = alloc_particles(s, nslots, nb);
    if (st != MPM_OK) { free_particles(s, nb); return fail(s, st, "device allocation failed"); }
    const size_t rs = s->rsize;
    cudaStream_t S = s->stream;
    // keep the particles already there at the front, in key order
    if (s->np > 0) {
        order_offsets(s, S);
        for (int a = 0; a < d; ++a) {
            s->vt->compact(s, 0, a, nb[0].x[a], S);
            s->vt->compact(s, 1, a, nb[0].v[a], S);
        }
        s->vt->compact(s, 2, 0, nb[0].M, S);
        s->vt->compact(s, 3, 0, nb[0].rho, S);
        s->vt->compact(s, 4, 0, nb[0].E, S);
        s->vt->compact(s, 5, 0, nb[0].Q, S);
        s->vt->compact(s, 6, 0, nb[0].id, S);
        s->vt->compact(s, 7, 0, nb[0].gen, S);
        CK(cudaGetLastError(), "compact");
    }
    // stage the new values on the device, check them there and convert them
    // to the storage precision; stream order keeps the staging buffer safe to
    // reuse (each copy into it follows the previous array's kernels)
    const size_t es = f32 ? sizeof(float) : sizeof(double);
    void* stage = dalloc(s, (size_t)n * es);
    unsigned* bad = (unsigned*)dalloc(s, sizeof(unsigned));
    if (!stage || !bad) {
        dfree(s, stage);
        dfree(s, bad);
        free_particles(s, nb);
        return fail(s, MPM_ENOMEM, "device allocation failed");
    }
    enum { kBadState = 1, kBadPlace = 2, kBadSeam = 4 };
    // axis >= 0: a position component (inside the domain, below hi on a
    // periodic axis); otherwise a value checked by `mode` that sets `bit`
    auto check = [&](int mode, double lo, double hi, unsigned bit) {
        if (f32) k_check_values<<<nblk(n), kThreads, 0, S>>>((const float*)stage, n, mode, lo, hi, bit, bad);
        else k_check_values<<<nblk(n), kThreads, 0, S>>>((const double*)stage, n, mode, lo, hi, bit, bad);
    };
    auto up = [&](const void* src, void* dst, int mode, unsigned bit, int axis) -> cudaError_t {
        cudaError_t r = cudaMemcpyAsync(stage, src, n * es, cudaMemcpyHostToDevice, S);
        if (r != cudaSuccess) return r;
        if (axis < 0) {
            check(mode, 0.0, 0.0, bit);
        } else {
            check(2, G.lo[axis], G.hi[axis], kBadPlace);
            if (G.per[axis]) check(3, G.lo[axis], G.hi[axis], kBadSeam);
        }
        if (f32) s->vt->from_float((const float*)stage, (char*)dst + s->np * rs, n, S);
        else s->vt->from_double((const double*)stage, (char*)dst + s->np * rs, n, S);
        return cudaGetLastError();
    };
    // component a of a dim x n SoA host array
    auto comp = [&](const void* p, int a) { return (const void*)((const char*)p + (size_t)a * n * es); };
    cudaError_t ue = cudaMemsetAsync(bad, 0, sizeof(unsigned), S);
    for (int a = 0; a < d && ue == cudaSuccess; ++a) {
        ue = up(comp(x, a), nb[0].x[a], 2, kBadPlace, a);
        if (ue == cudaSuccess) ue = up(comp(v, a), nb[0].v[a], 0, kBadPlace, -1);
    }
    if (ue == cudaSuccess) ue = up(mass, nb[0].M, 1, kBadState, -1);
    if (ue == cudaSuccess) ue = up(rho, nb[0].rho, 1, kBadState, -1);
    if (ue == cudaSuccess) ue = up(e, nb[0].E, 0, kBadState, -1);
    unsigned hbad = 0;
    if (ue == cudaSuccess) ue = cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, S);
    if (ue == cudaSuccess) ue = cudaStreamSynchronize(S);
    dfree(s, stage);
    dfree(s, bad);
    if (ue != cudaSuccess) { free_particles(s, nb); return cuda_fail(s, ue, "upload"); }
    if (hbad) {
        free_particles(s, nb);
        if (hbad & kBadState) return fail(s, MPM_EINVAL, "mass and rho must be > 0, e finite");
        if (hbad & kBadPlace) return fail(s, MPM_EINVAL, "particle outside the domain or non-finite velocity");
        return fail(s, MPM_EINVAL, "periodic axis: x must be < hi");
    }
    CK(cudaMemsetAsync((char*)nb[0].Q + s->np * rs, 0, n * rs, S), "zero q");
    CK(cudaMemsetAsync(nb[0].gen + s->np, 0, n * 4, S), "zero gen");
    k_iota<<<nblk(n), kThreads, 0, S>>>(nb[0].id + s->np, n, (uint32_t)s->np);
    // replace the old buffers and the sort scratch
    free_particles(s, s->buf);
    s->buf[0] = nb[0];
    s->buf[1] = nb[1];
    s->cur = 0;
    s->np = np;
    s->nslots = nslots;
    dfree(s, s->far);
    s->far = nullptr;
    s->far_cap = G.inflow_face >= 0 ? (uint32_t)np : 0u;
    if (s->far_cap) {
        s->far = (uint2*)dalloc(s, (size_t)np * sizeof(uint2));
        if (!s->far) return fail(s, MPM_ENOMEM, "device allocation failed");
    }
    // radix scratch for the initial order only
    RadixScratch sc;
    int bits = 1;
    while (((int64_t)1 << bits) < G.nkey) ++bits;
    sc.passes = (bits + kRadixBitsMax - 1) / kRadixBitsMax;
    sc.bits = (bits + sc.passes - 1) / sc.passes;
    const int64_t nblocks = (np + kSortTile - 1) / kSortTile;
    const int64_t nhist = nblocks * ((int64_t)1 << sc.bits);
    for (int b = 0; b < 2; ++b) {
        sc.skeys[b] = (uint32_t*)dalloc(s, (size_t)np * 4);
        sc.sidx[b] = (uint32_t*)dalloc(s, (size_t)np * 4);
    }
    sc.hist = (uint32_t*)dalloc(s, (size_t)nhist * 4);
    sc.part = (uint32_t*)dalloc(s, (size_t)std::max<int64_t>(scan_blocks(nhist), 1) * 4);
    uint32_t* cc = (uint32_t*)dalloc(s, (size_t)(G.nkey + 1) * 4);
    auto free_sc = [&]() {
        for (int b = 0; b < 2; ++b) { dfree(s, sc.skeys[b]); dfree(s, sc.sidx[b]); }
        dfree(s, sc.hist);
        dfree(s, sc.part);
        dfree(s, cc);
    };
    if (!sc.skeys[0] || !sc.skeys[1] || !sc.sidx[0] || !sc.sidx[1] || !sc.hist || !sc.part || !cc) {
        free_sc();
        return fail(s, MPM_ENOMEM, "device allocation failed");
    }
    drop_graphs(s);
    s->cfl_done = false;
    // initial order: keys from the positions, then the stable re-order into
    // the tile regions
    s->vt->keys(s, 0, S);
    launch_sort(s, sc, cc, S);
    cudaError_t le = cudaGetLastError();
    cudaError_t se = cudaStreamSynchronize(S);
    free_sc();
    CK(le, "launch");
    CK(se, "synchronize");
    return MPM_OK;
}

}  // namespace

mpm_status mpm_add_particles(mpm_sim* s, int64_t n, const double* x, const double* v, const double* mass,
                             const double* rho, const double* e)
{
    return add_particles(s, n, x, v, mass, rho, e, false);
}

mpm_status mpm_add_particles_f32(mpm_sim* s, int64_t n, const float* x, const float* v, const float* mass,
                                 const float* rho, const float* e)
{
    return add_particles(s, n, x, v, mass, rho, e, true);
}

mpm_status mpm_set_obstacle_mask(mpm_sim* s, const uint8_t* mask, const double* normals)
{
    if (!s) return fail(nullptr, MPM_EINVAL, "sim is NULL");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    if (s->poisoned) return fail(s, MPM_ESTATE, "simulation is poisoned: " + s->err);
    if (!mask || !normals) return fail(s, MPM_EINVAL, "NULL input array");
    return set_obstacle(s, mask, normals);
}

}  // extern "C"

// Checks a host node mask and normals (stored-node order) and installs them.
static mpm_status set_obstacle(mpm_sim* s, const uint8_t* mask, const double* normals)
{
    const Geom& G = s->G;
    const int64_t nn = G.nnode;
    const int d = G.dim;
    if (G.inflow_face >= 0) {
        const int af = G.inflow_face / 2, side = G.inflow_face % 2;
        for (int64_t i = 0; i < nn; ++i) {
            if (!mask[i]) continue;
            int64_t ia = af == 0 ? i % G.N[0] : af == 1 ? (i / G.N[0]) % G.N[1] : i / ((int64_t)G.N[0] * G.N[1]);
            int64_t phys = ia - G.g[af];
            bool near = side == 0 ? phys <= G.p : phys >= G.n[af] - G.p;
            if (near) return fail(s, MPM_EINVAL, "obstacle nodes next to the inflow face");
        }
    }
    for (int64_t i = 0; i < (int64_t)d * nn; ++i)
        if (!std::isfinite(normals[i])) return fail(s, MPM_EINVAL, "non-finite normal");
    const int64_t np_ = G.nnode_p;
    if (!s->mask) {
        s->mask = (uint8_t*)dalloc(s, (size_t)np_);
        s->nrm = dalloc(s, (size_t)d * np_ * s->rsize);
        if (!s->mask || !s->nrm) return fail(s, MPM_ENOMEM, "device allocation failed");
    }
    // expand to the device layout (rows padded to G.pitch)
    std::vector<uint8_t> m(np_, 0);
    std::vector<double> nv((size_t)d * np_, 0.0);
    for (int64_t i = 0; i < nn; ++i) {
        const int64_t row = i / G.N[0], x0 = i % G.N[0];
        const int64_t j = row * G.pitch + x0;
        m[j] = mask[i] ? 1 : 0;
        for (int a = 0; a < d; ++a) nv[(size_t)a * np_ + j] = normals[(size_t)a * nn + i];
    }
    CK(cudaMemcpyAsync(s->mask, m.data(), np_, cudaMemcpyHostToDevice, s->stream), "upload mask");
    double* stage = (double*)dalloc(s, (size_t)d * np_ * sizeof(double));
    if (!stage) return fail(s, MPM_ENOMEM, "device allocation failed");
    CK(cudaMemcpyAsync(stage, nv.data(), (size_t)d * np_ * sizeof(double), cudaMemcpyHostToDevice, s->stream),
       "upload");
    s->vt->from_double(stage, s->nrm, (int64_t)d * np_, s->stream);
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    dfree(s, stage);
    drop_graphs(s);
    return MPM_OK;
}

extern "C" {

static mpm_status ensure_cfl(mpm_sim* s)
{
    if (s->cfl_done) return MPM_OK;
    if (s->np == 0) return fail(s, MPM_ESTATE, "no particles");
    s->vt->cfl_init(s, s->stream);
    CK(cudaGetLastError(), "launch");
    s->cfl_done = true;
    return MPM_OK;
}

mpm_status mpm_cfl_dt(mpm_sim* s, double* dt_out)
{
    if (!s || !dt_out) return fail(s, MPM_EINVAL, "NULL argument");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    if (s->poisoned) return fail(s, MPM_ESTATE, "simulation is poisoned: " + s->err);
    mpm_status st = ensure_cfl(s);
    if (st != MPM_OK) return st;
    Clock c;
    CK(cudaMemcpyAsync(&c, s->clk, sizeof(Clock), cudaMemcpyDeviceToHost, s->stream), "read clock");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    *dt_out = c.dt_next;
    return MPM_OK;
}

static mpm_status capture_graph(mpm_sim* s, int b)
{
    // the step reads buffer b and leaves the sorted state in 1 - b
    cudaStream_t st = s->stream;
    cudaGraph_t g = nullptr;
    const int saved = s->cur;
    const int64_t saved_l = s->launches;
    s->cur = b;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        s->cur = saved;
        return MPM_ECUDA;
    }
    launch_step(s, st, nullptr);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    s->cur = saved;
    s->launches = saved_l;
    if (e != cudaSuccess || !g) { cudaGetLastError(); return MPM_ECUDA; }
    e = cudaGraphInstantiate(&s->graph[b], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { cudaGetLastError(); s->graph[b] = nullptr; return MPM_ECUDA; }
    return MPM_OK;
}

static int64_t step_launch_count(const mpm_sim* s)
{
    // prepare, zero, 3 step kernels, finalize; re-order: changed tiles,
    // consolidation, region bases, relayout pass, marks (the last three return
    // at once unless a tile outgrew its region)
    // a coloured simulation launches the two scattering kernels once per colour
    const int extra = s->col_off.empty() ? 0 : 2 * ((int)s->col_off.size() - 2);
    return 6 + 5 + extra;
}

mpm_status mpm_step_async(mpm_sim* s, int64_t nsteps, double dt, double t_end)
{
    if (!s) return fail(nullptr, MPM_EINVAL, "sim is NULL");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    if (s->poisoned) return fail(s, MPM_ESTATE, "simulation is poisoned: " + s->err);
    if (nsteps < 0 || !std::isfinite(dt) || !std::isfinite(t_end)) return fail(s, MPM_EINVAL, "bad step arguments");
    mpm_status st = ensure_cfl(s);
    if (st != MPM_OK) return st;
    s->started = true;
    k_set_params<<<1, 1, 0, s->stream>>>(s->clk, dt > 0.0 ? dt : 0.0, t_end > 0.0 ? t_end : 0.0);
    s->launches += 1;
    for (int64_t i = 0; i < nsteps; ++i) {
        if (s->profiling) {
            ProfStep ps;
            for (int k = 0; k <= kPhases; ++k) ps.ev[k] = pool_event(s);
            const int64_t l0 = s->launches;
            launch_step(s, s->stream, &ps);
            s->prof_launch[5] += s->launches - l0;
            s->prof.push_back(ps);
        } else {
            const int b = s->cur;
            if (!s->graph[b] && s->graph_ok && capture_graph(s, b) != MPM_OK) s->graph_ok = false;
            if (s->graph[b]) {
                CK(cudaGraphLaunch(s->graph[b], s->stream), "graph launch");
                s->cur ^= 1;
                s->launches += step_launch_count(s);
            } else {
                launch_step(s, s->stream, nullptr);
            }
        }
    }
    CK(cudaGetLastError(), "launch");
    s->stepped = true;
    return MPM_OK;
}

mpm_status mpm_sync(mpm_sim* s)
{
    if (!s) return fail(nullptr, MPM_EINVAL, "sim is NULL");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    if (s->poisoned) return fail(s, MPM_ESTATE, "simulation is poisoned: " + s->err);
    return check_device_errors(s);
}

mpm_status mpm_step(mpm_sim* s, int64_t nsteps, double dt, double t_end)
{
    mpm_status st = mpm_step_async(s, nsteps, dt, t_end);
    if (st != MPM_OK) return st;
    return check_device_errors(s);
}

int64_t mpm_field_size(const mpm_sim* s, int field)
{
    if (!s) return -1;
    const int d = s->G.dim;
    switch (field) {
    case MPM_FIELD_X: case MPM_FIELD_V: return d * s->np;
    case MPM_FIELD_M: case MPM_FIELD_RHO: case MPM_FIELD_E: case MPM_FIELD_P: case MPM_FIELD_Q:
    case MPM_FIELD_ID: case MPM_FIELD_KEY: case MPM_FIELD_GEN: return s->np;
    case MPM_FIELD_CELLSTART: return s->G.nkey + 1;
    case MPM_FIELD_GRID_M: return s->G.nnode;
    case MPM_FIELD_GRID_MV: case MPM_FIELD_GRID_F: case MPM_FIELD_GRID_MV2: return d * s->G.nnode;
    case MPM_FIELD_CLOCK: return 4;
    }
    return -1;
}

static mpm_status read_real(mpm_sim* s, const void* src, int64_t n, double* out)
{
    if (n == 0) return MPM_OK;
    if (s->rsize == 8) {
        CK(cudaMemcpyAsync(out, src, n * 8, cudaMemcpyDeviceToHost, s->stream), "read");
        CK(cudaStreamSynchronize(s->stream), "synchronize");
        return MPM_OK;
    }
    // widen on the device and copy straight into the caller's array, in
    // chunks (stream order protects the staging buffer)
    const int64_t chunk = std::min<int64_t>(n, (int64_t)1 << 25);
    double* stage = (double*)dalloc(s, (size_t)chunk * 8);
    if (stage) {
        cudaError_t e = cudaSuccess;
        for (int64_t off = 0; off < n && e == cudaSuccess; off += chunk) {
            const int64_t m = std::min(chunk, n - off);
            k_to_double<float><<<nblk(m), kThreads, 0, s->stream>>>((const float*)src + off, stage, m);
            e = cudaMemcpyAsync(out + off, stage, m * 8, cudaMemcpyDeviceToHost, s->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        dfree(s, stage);
        CK(e, "read");
        return MPM_OK;
    }
    std::vector<float> t(n);
    CK(cudaMemcpyAsync(t.data(), src, n * 4, cudaMemcpyDeviceToHost, s->stream), "read");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    for (int64_t i = 0; i < n; ++i) out[i] = (double)t[i];
    return MPM_OK;
}

static mpm_status read_u32(mpm_sim* s, const uint32_t* src, int64_t n, double* out)
{
    std::vector<uint32_t> t(n);
    if (n) {
        CK(cudaMemcpyAsync(t.data(), src, n * 4, cudaMemcpyDeviceToHost, s->stream), "read");
        CK(cudaStreamSynchronize(s->stream), "synchronize");
    }
    for (int64_t i = 0; i < n; ++i) out[i] = (double)t[i];
    return MPM_OK;
}

mpm_status mpm_read_state(mpm_sim* s, int field, double* out, int64_t count)
{
    if (!s) return fail(nullptr, MPM_EINVAL, "sim is NULL");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    if (s->poisoned) return fail(s, MPM_ESTATE, "simulation is poisoned: " + s->err);
    if (!out) return fail(s, MPM_EINVAL, "out is NULL");
    const int64_t need = mpm_field_size(s, field);
    if (need < 0) return fail(s, MPM_EINVAL, "unknown field");
    if (count < need) return fail(s, MPM_EINVAL, "output buffer too short");
    mpm_status st = check_device_errors(s);
    if (st != MPM_OK) return st;
    const int d = s->G.dim;
    const int64_t np = s->np, nn = s->G.nnode;
    const bool particle_field = field <= MPM_FIELD_CELLSTART || field == MPM_FIELD_GEN;
    if (particle_field && np > 0) order_offsets(s, s->stream);
    // a particle field gathered into key order on the device, then read
    auto real_field = [&](int f, int a, double* dst) -> mpm_status {
        void* tmp = dalloc(s, (size_t)np * s->rsize);
        if (!tmp) return fail(s, MPM_ENOMEM, "device allocation failed");
        s->vt->compact(s, f, a, tmp, s->stream);
        const mpm_status r = read_real(s, tmp, np, dst);
        dfree(s, tmp);
        return r;
    };
    auto u32_field = [&](int f, double* dst) -> mpm_status {
        uint32_t* tmp = (uint32_t*)dalloc(s, (size_t)np * 4);
        if (!tmp) return fail(s, MPM_ENOMEM, "device allocation failed");
        s->vt->compact(s, f, 0, tmp, s->stream);
        const mpm_status r = read_u32(s, tmp, np, dst);
        dfree(s, tmp);
        return r;
    };
    // the cell starts of the key order without the regions' gaps
    auto compact_starts = [&](uint32_t* dst) {
        k_compact_starts<<<std::min<int64_t>(nblk(s->G.nkey + 1), s->sms * 16), kThreads, 0, s->stream>>>(
            s->G, s->cs[0], s->cs[1], s->tpar[s->cur], s->toff, dst);
    };
    if (np == 0 && particle_field && field != MPM_FIELD_CELLSTART) return MPM_OK;
    switch (field) {
    case MPM_FIELD_X:
        for (int a = 0; a < d; ++a) if ((st = real_field(0, a, out + a * np))) return st;
        return MPM_OK;
    case MPM_FIELD_V:
        for (int a = 0; a < d; ++a) if ((st = real_field(1, a, out + a * np))) return st;
        return MPM_OK;
    case MPM_FIELD_M: return real_field(2, 0, out);
    case MPM_FIELD_RHO: return real_field(3, 0, out);
    case MPM_FIELD_E: return real_field(4, 0, out);
    case MPM_FIELD_Q: return real_field(5, 0, out);
    case MPM_FIELD_P: {
        // evaluated on the device from the stored density and energy, as
        // the step kernels evaluate it
        char* tmp = (char*)dalloc(s, (size_t)np * s->rsize * 3);
        if (!tmp) return fail(s, MPM_ENOMEM, "device allocation failed");
        void* tr = tmp;
        void* te = tmp + np * s->rsize;
        void* tp = tmp + 2 * np * s->rsize;
        s->vt->compact(s, 3, 0, tr, s->stream);
        s->vt->compact(s, 4, 0, te, s->stream);
        if (s->rsize == 8)
            k_pressure<double><<<nblk(np), kThreads, 0, s->stream>>>((const double*)tr, (const double*)te,
                                                                    s->G.gamma - 1.0, (double*)tp, np);
        else
            k_pressure<float><<<nblk(np), kThreads, 0, s->stream>>>((const float*)tr, (const float*)te,
                                                                   (float)(s->G.gamma - 1.0), (float*)tp, np);
        st = read_real(s, tp, np, out);
        dfree(s, tmp);
        return st;
    }
    case MPM_FIELD_ID: return u32_field(6, out);
    case MPM_FIELD_GEN:
        // the recycle counts move with the particles only where recycling
        // exists (an inflow face); elsewhere they are all 0
        if (s->G.inflow_face < 0) {
            for (int64_t k = 0; k < np; ++k) out[k] = 0.0;
            return MPM_OK;
        }
        return u32_field(7, out);
    case MPM_FIELD_KEY: {
        // keys of the current order, expanded from its cell starts
        uint32_t* tcs = (uint32_t*)dalloc(s, (size_t)(s->G.nkey + 1) * 4);
        uint32_t* tk = (uint32_t*)dalloc(s, (size_t)np * 4);
        if (!tcs || !tk) {
            dfree(s, tcs);
            dfree(s, tk);
            return fail(s, MPM_ENOMEM, "device allocation failed");
        }
        compact_starts(tcs);
        k_keys_from_start<<<std::min<int64_t>(nblk(s->G.nkey), s->sms * 16), kThreads, 0, s->stream>>>(
            tcs, s->G.nkey, tk);
        st = read_u32(s, tk, np, out);
        dfree(s, tcs);
        dfree(s, tk);
        return st;
    }
    case MPM_FIELD_CELLSTART: {
        if (np == 0) {
            for (int64_t k = 0; k <= s->G.nkey; ++k) out[k] = 0.0;
            return MPM_OK;
        }
        uint32_t* tcs = (uint32_t*)dalloc(s, (size_t)(s->G.nkey + 1) * 4);
        if (!tcs) return fail(s, MPM_ENOMEM, "device allocation failed");
        compact_starts(tcs);
        st = read_u32(s, tcs, s->G.nkey + 1, out);
        dfree(s, tcs);
        return st;
    }
    case MPM_FIELD_CLOCK: {
        Clock c;
        CK(cudaMemcpyAsync(&c, s->clk, sizeof(Clock), cudaMemcpyDeviceToHost, s->stream), "read clock");
        CK(cudaStreamSynchronize(s->stream), "synchronize");
        out[0] = c.t;
        out[1] = c.dt_next;
        out[2] = (double)c.step;
        out[3] = (double)c.relayouts;
        if (!s->started) {
            double dt0 = 0.0;
            if ((st = mpm_cfl_dt(s, &dt0))) return st;
            out[1] = dt0;
        }
        return MPM_OK;
    }
    default: break;
    }
    // grid fields: copy the padded rows, then drop the padding
    const int64_t npd = s->G.nnode_p;
    const int comps = field == MPM_FIELD_GRID_M ? 1 : d;
    int64_t off = field == MPM_FIELD_GRID_M ? 0 : field == MPM_FIELD_GRID_MV ? npd
                : field == MPM_FIELD_GRID_F ? (1 + d) * npd : (1 + 2 * d) * npd;
    std::vector<double> tmp((size_t)comps * npd);
    if (s->cfg.precision == MPM_FP32_FIXED64) {
        std::vector<long long> t((size_t)comps * npd);
        CK(cudaMemcpyAsync(t.data(), (long long*)s->grid + off, t.size() * 8, cudaMemcpyDeviceToHost, s->stream),
           "read");
        CK(cudaStreamSynchronize(s->stream), "synchronize");
        const int kind = field == MPM_FIELD_GRID_M ? 0 : field == MPM_FIELD_GRID_F ? 2 : 1;
        const double u = s->cfg.fixed_unit[kind] > 0.0 ? s->cfg.fixed_unit[kind] : 1.0;
        for (size_t i = 0; i < t.size(); ++i) tmp[i] = (double)t[i] * (u / 4294967296.0);
    } else {
        if ((st = read_real(s, (char*)s->grid + off * s->asize, (int64_t)tmp.size(), tmp.data()))) return st;
    }
    for (int c = 0; c < comps; ++c)
        for (int64_t i = 0; i < nn; ++i) {
            const int64_t row = i / s->G.N[0], x0 = i % s->G.N[0];
            out[(size_t)c * nn + i] = tmp[(size_t)c * npd + row * s->G.pitch + x0];
        }
    return MPM_OK;
}

mpm_status mpm_read_grid_fixed(mpm_sim* s, int field, int64_t* out, int64_t count)
{
    if (!s) return fail(nullptr, MPM_EINVAL, "sim is NULL");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    if (s->poisoned) return fail(s, MPM_ESTATE, "simulation is poisoned: " + s->err);
    if (s->cfg.precision != MPM_FP32_FIXED64) return fail(s, MPM_EINVAL, "not a fixed-point simulation");
    if (!out || field < MPM_FIELD_GRID_M || field > MPM_FIELD_GRID_MV2) return fail(s, MPM_EINVAL, "bad field");
    const int64_t need = mpm_field_size(s, field);
    if (count < need) return fail(s, MPM_EINVAL, "output buffer too short");
    const int d = s->G.dim;
    const int64_t nn = s->G.nnode, npd = s->G.nnode_p;
    const int comps = field == MPM_FIELD_GRID_M ? 1 : d;
    int64_t off = field == MPM_FIELD_GRID_M ? 0 : field == MPM_FIELD_GRID_MV ? npd
                : field == MPM_FIELD_GRID_F ? (1 + d) * npd : (1 + 2 * d) * npd;
    std::vector<long long> t((size_t)comps * npd);
    CK(cudaMemcpyAsync(t.data(), (long long*)s->grid + off, t.size() * 8, cudaMemcpyDeviceToHost, s->stream), "read");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    for (int c = 0; c < comps; ++c)
        for (int64_t i = 0; i < nn; ++i) {
            const int64_t row = i / s->G.N[0], x0 = i % s->G.N[0];
            out[(size_t)c * nn + i] = t[(size_t)c * npd + row * s->G.pitch + x0];
        }
    return MPM_OK;
}

mpm_status mpm_conservation(mpm_sim* s, double out[5])
{
    if (!s || !out) return fail(s, MPM_EINVAL, "NULL argument");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    if (s->poisoned) return fail(s, MPM_ESTATE, "simulation is poisoned: " + s->err);
    mpm_status st = check_device_errors(s);
    if (st != MPM_OK) return st;
    if (s->np == 0) { for (int i = 0; i < 5; ++i) out[i] = 0.0; return MPM_OK; }
    s->vt->cons(s, s->stream);
    CK(cudaGetLastError(), "launch");
    double t[5];
    CK(cudaMemcpyAsync(t, s->cons_out, sizeof(t), cudaMemcpyDeviceToHost, s->stream), "read");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    for (int i = 0; i < 5; ++i) out[i] = t[i];
    if (s->G.dim == 2) out[4] = 0.0;
    return MPM_OK;
}

mpm_status mpm_sizes(const mpm_sim* s, int64_t out[4])
{
    if (!s || !out) return MPM_EINVAL;
    if (s->batch) return MPM_ESTATE;
    Clock c;
    memset(&c, 0, sizeof(c));
    if (cudaMemcpyAsync(&c, s->clk, sizeof(Clock), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        cudaGetLastError();
    out[0] = s->np;
    out[1] = s->G.nnode;
    out[2] = s->G.nkey;
    out[3] = c.step;
    return MPM_OK;
}

mpm_status mpm_profile(mpm_sim* s, int enable)
{
    if (!s) return fail(nullptr, MPM_EINVAL, "sim is NULL");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    s->profiling = enable != 0;
    return MPM_OK;
}

mpm_status mpm_profile_read(mpm_sim* s, double out[8], int64_t counts[8], int reset)
{
    if (!s) return fail(nullptr, MPM_EINVAL, "sim is NULL");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    mpm_status st = collect_profile(s);
    if (st != MPM_OK) return st;
    // launches per phase of one step, times the profiled steps
    for (int i = 0; i < 8; ++i) {
        if (out) out[i] = s->prof_ms[i];
        if (counts) counts[i] = s->prof_launch[i];
    }
    if (counts) {
        // per-step launch counts of each phase (fixed by the configuration)
        const int ncol = s->col_off.empty() ? 1 : (int)s->col_off.size() - 1;
        counts[0] = 1 + ncol;   // zero + P2G
        counts[1] = ncol;
        counts[2] = 1;
        counts[3] = 1;   // finalize (prepare counted with the step)
        counts[4] = 4 + (s->far_cap ? 1 : 0);
        counts[6] = s->launches;
    }
    if (reset) {
        for (int i = 0; i < 8; ++i) { s->prof_ms[i] = 0.0; s->prof_launch[i] = 0; }
    }
    return MPM_OK;
}

void* mpm_stream(const mpm_sim* s) { return s ? (void*)s->stream : nullptr; }

const char* mpm_last_error(const mpm_sim* s)
{
    return s ? s->err.c_str() : g_static_err.c_str();
}

void mpm_destroy(mpm_sim* s)
{
    if (!s) return;
    if (s->batch) mpm_batch_remove(s->batch, s);
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graphs(s);
    for (auto& ps : s->prof)
        for (int k = 0; k <= kPhases; ++k) cudaEventDestroy(ps.ev[k]);
    for (auto e : s->ev_pool) cudaEventDestroy(e);
    std::vector<void*> a = s->allocs;
    for (void* p : a) dfree(s, p);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    cudaGetLastError();
    delete s;
}

}  // extern "C"

// The allocation-free re-order entry point (same translation unit).
#include "mpm_noalloc.cu"
#include "mpm_selfcheck.cu"
#include "mpm_obstacle.cu"
#include "mpm_batch.cu"
