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
    uint32_t* cs[2];
    uint32_t* cscan_part;
    int64_t nkey;
    uint2* far;
    uint32_t far_cap;
    uint32_t* perm;
    double cfl_h;
};

template <class R, class A>
struct BatchProb {
    Geom G;
    Particles<R> pt[2];
    Grid<A, R> gr;
    FieldPtrs p2g_out, g2p_out;     // single-precision kernels: grid fields they add into
    uint32_t* cs[2];
    Reorder ro;
    uint32_t* perm;
    int64_t np;
    Clock* clk;
};

constexpr int kZeroChunk = 256 * 16;    // 16-byte words cleared per block
constexpr int kFarBlocks = 8;           // blocks placing one member's recycled particles

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

// Counts of the new spans -> cell starts of the other buffer, per member.
__global__ void __launch_bounds__(kScanThreads) kb_scan_reduce(const BatchCommon* __restrict__ c,
                                                              const TileRef* __restrict__ bl)
{
    const TileRef r = bl[blockIdx.x];
    const BatchCommon& d = c[r.prob];
    scan_reduce_block(d.count, d.nkey, d.cscan_part, r.tile);
}

__global__ void __launch_bounds__(kScanThreads) kb_scan_partials(const BatchCommon* __restrict__ c)
{
    const BatchCommon& d = c[blockIdx.x];
    scan_partials_block(d.cscan_part, scan_blocks(d.nkey));
}

__global__ void __launch_bounds__(kScanThreads) kb_scan_down(const BatchCommon* __restrict__ c,
                                                            const TileRef* __restrict__ bl)
{
    const TileRef r = bl[blockIdx.x];
    const BatchCommon& d = c[r.prob];
    scan_down_block(d.count, d.nkey, d.cscan_part, d.cs[1 - d.clk->par], 1, r.tile);
}

__global__ void kb_far_place(const BatchCommon* __restrict__ c, const TileRef* __restrict__ bl)
{
    const TileRef r = bl[blockIdx.x];
    const BatchCommon& d = c[r.prob];
    far_place_block(d.far, d.far_cap, d.count, d.cs[1 - d.clk->par], d.perm, d.clk, (unsigned)r.tile, kFarBlocks);
}

// ------------------------------------------------------------ per tile

#define MPM_BATCH_PROLOGUE(R, A)                 \
    __shared__ BatchProb<R, A> p;                \
    const TileRef r = tl[blockIdx.x];            \
    load_shared(p, bp[r.prob]);                  \
    __syncthreads();                             \
    const int par = p.clk->par;

template <int D, int P, class R, class A>
__global__ void __launch_bounds__(256) kb_p2g(const BatchProb<R, A>* __restrict__ bp, const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    p2g_tile<D, P, R, A>(p.G, p.pt[par], p.gr, p.cs[par], p.clk, r.tile);
}

template <int D, int P, class R, class A>
__global__ void __launch_bounds__(256) kb_grid_g2p(const BatchProb<R, A>* __restrict__ bp,
                                                   const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    grid_g2p_tile<D, P, R, A>(p.G, p.pt[par], p.gr, p.cs[par], p.clk, r.tile);
}

template <int D, int P, class R, class A>
__global__ void __launch_bounds__(256) kb_g2pd(const BatchProb<R, A>* __restrict__ bp, const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    g2pd_tile<D, P, R, A>(p.G, p.pt[par], p.gr, p.cs[par], p.clk, p.ro, r.tile);
}

template <int D, int P, bool PER>
__global__ void __launch_bounds__(kP2GThreads, 6) kb_p2g_span(const BatchProb<float, float>* __restrict__ bp,
                                                              const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(float, float)
    p2g_span_tile<D, P, PER>(p.G, p.pt[par], p.p2g_out, p.cs[par], p.clk, r.tile);
}

template <int P, class R, class A>
__global__ void __launch_bounds__(kP2GSpan2dThreads, 6) kb_p2g_span2d(const BatchProb<R, A>* __restrict__ bp,
                                                                      const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    p2g_span2d_tile<P, R, A>(p.G, p.pt[par], p.gr, p.cs[par], p.clk, r.tile);
}

template <int P, class R, class A>
__global__ void __launch_bounds__(kG2PSpan2dThreads, 4)
    kb_grid_g2p_span2d(const BatchProb<R, A>* __restrict__ bp, const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    grid_g2p_span2d_tile<P, R, A>(p.G, p.pt[par], p.gr, p.cs[par], p.clk, r.tile);
}

template <int D, int P, bool PER>
__global__ void __launch_bounds__(K2Cfg<D>::kThreads, 3)
    kb_grid_g2p_span(const BatchProb<float, float>* __restrict__ bp, const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(float, float)
    grid_g2p_span_tile<D, P, PER>(p.G, p.pt[par], p.gr, p.g2p_out, p.cs[par], p.clk, r.tile);
}

template <int D, int P, class A>
__global__ void __launch_bounds__(kG2PDThreads, kG2PDBlocks) kb_g2pd_fast(const BatchProb<float, A>* __restrict__ bp,
                                                             const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(float, A)
    g2pd_fast_tile<D, P, A>(p.G, p.pt[par], p.gr, p.cs[par], p.clk, p.ro, r.tile);
}

template <int D, class R, class A>
__global__ void __launch_bounds__(kReorderThreads, 3) kb_reorder(const BatchProb<R, A>* __restrict__ bp,
                                                                 const TileRef* __restrict__ tl)
{
    MPM_BATCH_PROLOGUE(R, A)
    reorder_tile<D, R>(p.G, p.pt[par], p.pt[1 - par], p.cs[par], p.cs[1 - par], p.ro.count, p.perm, p.np, p.ro.ring,
                       p.ro.mwords, p.clk, r.tile);
}

#undef MPM_BATCH_PROLOGUE

}  // namespace mpm
