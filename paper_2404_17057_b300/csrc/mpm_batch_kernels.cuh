// mpm_batch_kernels.cuh -- one launch per stage of the step for many
// independent problems at once.
//
// Every block of a batched launch looks up its (problem, tile) pair in a
// flattened list, copies that problem's descriptor into shared memory and runs
// the same tile body as the single-problem kernel, so a problem computes
// exactly what it computes alone.  Each problem keeps its own clock (time
// step, CFL maxima, step budget) and the parity of the buffer holding its
// state, which the last launch of every step flips.
#pragma once
#include "mpm_kernels.cuh"
#include "mpm_fast.cuh"
#include "mpm_sort.cuh"
#include "mpm_reorder.cuh"

namespace mpm {

struct TileRef {
    int prob, tile;
};

// Type-independent view of a member (clock, grid storage, re-order arrays).
struct BatchCommon {
    Clock* clk;
    uint4* grid16;
    int64_t n16;
    uint32_t* count;
    int64_t nkey;
    int ntiles, mwords, tvol;
    uint32_t* dirty;
    unsigned long long* ring;
    uint32_t* tbase;
    uint32_t* tbase_next;
    uint32_t* tcount;
    double cfl_h;
};

template <class R, class A>
struct BatchProb {
    Geom G;
    Particles<R> pt;                // both buffers (absolute slots)
    uint32_t nslots;
    Grid<A, R> gr;
    FieldPtrs p2g_out, g2p_out;     // single-precision kernels: grid fields they add into
    uint32_t* cs[2];
    uint8_t* tpar[2];               // buffer of each tile, by step parity
    uint32_t* tbase;
    uint32_t* tbase_next;
    uint32_t* tcount;
    Reorder ro;
    int64_t np;
    Clock* clk;
};

constexpr int kZeroChunk = 256 * 16;    // 16-byte words cleared per block

template <class T>
__device__ __forceinline__ void load_shared(T& dst, const T& src)
{
    static_assert(sizeof(T) % 4 == 0, "descriptor size");
    const uint32_t* s = reinterpret_cast<const uint32_t*>(&src);
    uint32_t* d = reinterpret_cast<uint32_t*>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
}

// ---------------------------------------------------------- per member

__global__ void kb_prepare(const BatchCommon* __restrict__ c, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) prepare_clock(*c[i].clk);
}

__global__ void kb_finalize(const BatchCommon* __restrict__ c, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) finalize_clock(*c[i].clk, c[i].cfl_h);
}

__global__ void kb_flip(const BatchCommon* __restrict__ c, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) c[i].clk->par ^= 1;
}

__global__ void kb_zero(const BatchCommon* __restrict__ c, const TileRef* __restrict__ zl)
{
    const TileRef r = zl[blockIdx.x];
    const BatchCommon& d = c[r.prob];
    if (!d.clk->active) return;
    const int64_t b = (int64_t)r.tile * kZeroChunk, e = min(b + (int64_t)kZeroChunk, d.n16);
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) d.grid16[i] = make_uint4(0, 0, 0, 0);
}

// Relayout of a member whose tile outgrew its region: the new regions (one
// block per member).
__global__ void __launch_bounds__(1024) kb_relayout_bases(const BatchCommon* __restrict__ c)
{
    const BatchCommon& d = c[blockIdx.x];
    if (!d.clk->overflow) return;
    relayout_bases_block(d.tcount, d.ntiles, d.tbase_next);
}

// End of a member's step: block (member, k) finishes the re-order of the
// tiles [k, k + 1) * kScanTile (marks cleared, the regions of a relayout
// installed).
__global__ void __launch_bounds__(kScanThreads) kb_step_end(const BatchCommon* __restrict__ c,
                                                           const TileRef* __restrict__ bl)
{
    const TileRef r = bl[blockIdx.x];
    const BatchCommon& d = c[r.prob];
    const int64_t b = (int64_t)r.tile * kScanTile;
    const Reorder ro = {d.count, nullptr, 0u, d.mwords, d.ring, d.dirty};
    for (int64_t t = b + (threadIdx.x >> 5); t < min(b + (int64_t)kScanTile, (int64_t)d.ntiles); t += blockDim.x >> 5)
        reorder_done_tile(d.tvol, ro, d.clk, d.tbase, d.tbase_next, (int)t, d.ntiles, threadIdx.x & 31);
}

// ------------------------------------------------------------ per tile

#define MPM_BATCH_PROLOGUE(R, A)                 \
    __shared__ BatchProb<R, A> p;                \
    const TileRef r = tl[blockIdx.x];            \
    load_shared(p, bp[r.prob]);                  \
    __syncthreads();                             \
    const int par = p.clk->par;                  \
    const uint32_t* csp = p.cs[p.tpar[par][r.tile]];

template <int D, int P, class R, class A>
__global__ void __launch_bounds__(256) kb_p2g(const BatchProb<R, A>* __restrict__ bp, const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    p2g_tile<D, P, R, A>(p.G, p.pt, p.gr, csp, p.clk, r.tile);
}

template <int D, int P, class R, class A>
__global__ void __launch_bounds__(256) kb_grid_g2p(const BatchProb<R, A>* __restrict__ bp,
                                                   const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    grid_g2p_tile<D, P, R, A>(p.G, p.pt, p.gr, csp, p.clk, r.tile);
}

template <int D, int P, class R, class A>
__global__ void __launch_bounds__(256) kb_g2pd(const BatchProb<R, A>* __restrict__ bp, const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    g2pd_tile<D, P, R, A>(p.G, p.pt, p.gr, csp, p.clk, p.ro, r.tile);
}

template <int D, int P, bool PER, bool COL>
__global__ void __launch_bounds__(kP2GThreads, 6) kb_p2g_span(const BatchProb<float, float>* __restrict__ bp,
                                                              const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(float, float)
    p2g_span_tile<D, P, PER, COL>(p.G, p.pt, p.p2g_out, csp, p.clk, r.tile);
}

template <int P, class R, class A>
__global__ void __launch_bounds__(kP2GSpan2dThreads, 6) kb_p2g_span2d(const BatchProb<R, A>* __restrict__ bp,
                                                                      const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    p2g_span2d_tile<P, R, A>(p.G, p.pt, p.gr, csp, p.clk, r.tile);
}

template <int P, class R, class A>
__global__ void __launch_bounds__(kG2PSpan2dThreads, 4)
    kb_grid_g2p_span2d(const BatchProb<R, A>* __restrict__ bp, const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    grid_g2p_span2d_tile<P, R, A>(p.G, p.pt, p.gr, csp, p.clk, r.tile);
}

template <int D, int P, bool PER>
__global__ void __launch_bounds__(K2Cfg<D>::kThreads, 5)
    kb_grid_g2p_span(const BatchProb<float, float>* __restrict__ bp, const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(float, float)
    grid_g2p_span_tile<D, P, PER>(p.G, p.pt, p.gr, p.g2p_out, csp, p.clk, r.tile);
}

template <int D, int P, class A>
__global__ void __launch_bounds__(kG2PDThreads, g2pd_blocks<D>()) kb_g2pd_fast(const BatchProb<float, A>* __restrict__ bp,
                                                             const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(float, A)
    g2pd_fast_tile<D, P, A>(p.G, p.pt, p.gr, csp, p.clk, p.ro, r.tile);
}

// The re-order arguments of member p at step parity par.
template <class R, class A>
__device__ __forceinline__ void batch_reorder_args(const BatchProb<R, A>& p, int par, ReorderArgs<R>& a)
{
    a.pt = p.pt;
    a.nslots = p.nslots;
    a.cs[0] = p.cs[0];
    a.cs[1] = p.cs[1];
    a.tpar_old = p.tpar[par];
    a.tpar_new = p.tpar[1 - par];
    a.tbase = p.tbase;
    a.tbase_next = p.tbase_next;
    a.tcount = p.tcount;
    a.ro = p.ro;
    a.clk = p.clk;
}

// mode 0: the member's changed tiles; mode 1: its relayout (if a tile
// overflowed)
template <int D, class R, class A>
__global__ void __launch_bounds__(kReorderThreads, kReorderBlocksPerSM) kb_reorder(const BatchProb<R, A>* __restrict__ bp,
                                                                 const TileRef* __restrict__ tl, int mode)
{
    MPM_BATCH_PROLOGUE(R, A)
    (void)csp;
    __shared__ ReorderArgs<R> a;
    if (threadIdx.x == 0) batch_reorder_args(p, par, a);
    __syncthreads();
    if (mode == 1 && !p.clk->overflow) return;
    reorder_tile<D, R>(p.G, a, mode, r.tile);
}

template <int D, class R, class A>
__global__ void __launch_bounds__(kReorderThreads) kb_consolidate(const BatchProb<R, A>* __restrict__ bp,
                                                                  const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    (void)csp;
    if (!p.clk->overflow) return;
    __shared__ ReorderArgs<R> a;
    if (threadIdx.x == 0) batch_reorder_args(p, par, a);
    __syncthreads();
    consolidate_tile<D, R>(p.G, a, r.tile);
}

#undef MPM_BATCH_PROLOGUE

}  // namespace mpm
