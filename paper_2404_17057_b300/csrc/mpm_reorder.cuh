// mpm_reorder.cuh -- per-step stable re-order of the particles (Sec. 3 step xii).
//
// After the G2PD step every particle carries its new span key, and the
// particles of every new span have been counted.  The time-step rule of
// Sec. 4.1 (checked by the G2PD step) keeps every particle within one span of
// where it was, so the particles that end up in a tile all come from the
// tile's old spans and one ring of old spans around it.  One CTA per tile:
//
//   1. lists the old index ranges of that neighbourhood (one range per row of
//      spans inside the tile, single spans outside it), ordered by old index;
//   2. streams the keys of those ranges (coalesced) and compacts the particles
//      whose new key lies in the tile into shared memory, in old order;
//   3. ranks them per new span with per-warp counters (stable: a span keeps
//      its particles' previous order) and copies each particle's state from
//      the old buffer straight to its slot in the new one;
//   4. appends the particles recycled at the inflow during the step (they
//      were given the tail slots of their span by k_far_place), ordered by id.
//
// Scan of the counts into the new cell starts happens before (mpm_sort.cuh).
#pragma once
#include "mpm_kernels.cuh"

namespace mpm {

constexpr int kReorderThreads = 256;
constexpr int kReorderWarps = kReorderThreads / 32;
constexpr int kReorderItems = 8;                                  // keys per thread per chunk
constexpr int kReorderChunk = kReorderThreads * kReorderItems;
constexpr int kReorderCap = 6144;                                 // compacted particles per flush
constexpr int kReorderMaxRanges = 1024;

__host__ inline size_t reorder_smem(const Geom& G)
{
    const size_t T = (size_t)G.Tvol, nr = (size_t)reorder_ranges(G);
    return ((kReorderWarps + 2) * T + kReorderCap + 4 * nr + 2 + kReorderWarps) * 4 + kReorderCap * 2;
}

// The recycle count (gen) is read only by recycling, so problems without an
// inflow face do not move it.
template <class R>
__device__ __forceinline__ void copy_particle(const Particles<R>& in, const Particles<R>& out, int D, uint32_t q,
                                              uint32_t j, bool with_gen)
{
    R xv[6];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (a < D) { xv[a] = in.x[a][q]; xv[3 + a] = in.v[a][q]; }
    const R M = in.M[q], rho = in.rho[q], E = in.E[q], Q = in.Q[q];
    const uint32_t id = in.id[q], gen = with_gen ? in.gen[q] : 0u;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (a < D) { out.x[a][j] = xv[a]; out.v[a][j] = xv[3 + a]; }
    out.M[j] = M;
    out.rho[j] = rho;
    out.E[j] = E;
    out.Q[j] = Q;
    out.id[j] = id;
    if (with_gen) out.gen[j] = gen;
}

// Copy kB particles per lane, q[u] -> j[u] where ok[u]: all loads first, so
// that 12 kB independent loads per lane are in flight.
template <int kB, class R>
__device__ __forceinline__ void copy_batch(const Particles<R>& in, const Particles<R>& out, int D, const uint32_t* q,
                                           const uint32_t* j, const bool* ok, bool with_gen)
{
    R xv[kB][6], M[kB], rho[kB], E[kB], Q[kB];
    uint32_t id[kB], gen[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
        if (!ok[u]) continue;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a < D) { xv[u][a] = in.x[a][q[u]]; xv[u][3 + a] = in.v[a][q[u]]; }
        M[u] = in.M[q[u]];
        rho[u] = in.rho[q[u]];
        E[u] = in.E[q[u]];
        Q[u] = in.Q[q[u]];
        id[u] = in.id[q[u]];
        gen[u] = with_gen ? in.gen[q[u]] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
        if (!ok[u]) continue;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a < D) { out.x[a][j[u]] = xv[u][a]; out.v[a][j[u]] = xv[u][3 + a]; }
        out.M[j[u]] = M[u];
        out.rho[j[u]] = rho[u];
        out.E[j[u]] = E[u];
        out.Q[j[u]] = Q[u];
        out.id[j[u]] = id[u];
        if (with_gen) out.gen[j[u]] = gen[u];
    }
}

// Recycled particles may land anywhere: each takes a slot at the end of its
// new span's segment (count[K] counts down to the span's stayers); their
// order inside the span is fixed by k_reorder (by id).
__device__ __forceinline__ void far_place_block(const uint2* __restrict__ far, uint32_t far_cap,
                                                uint32_t* __restrict__ count, const uint32_t* __restrict__ cs_new,
                                                uint32_t* __restrict__ perm, const Clock* clk, unsigned blk,
                                                unsigned nblk)
{
    if (!clk->active) return;
    const unsigned F = min(clk->nfar, far_cap);
    for (unsigned i = blk * blockDim.x + threadIdx.x; i < F; i += nblk * blockDim.x) {
        const uint2 e = far[i];
        const uint32_t r = atomicSub(&count[e.x], 1u) - 1u;
        const uint32_t pos = cs_new[e.x] + r;
        if (pos < cs_new[e.x + 1]) perm[pos] = e.y;
    }
}

__global__ void k_far_place(const uint2* __restrict__ far, uint32_t far_cap, uint32_t* __restrict__ count,
                            const uint32_t* __restrict__ cs_new, uint32_t* __restrict__ perm, const Clock* clk)
{
    far_place_block(far, far_cap, count, cs_new, perm, clk, blockIdx.x, gridDim.x);
}

template <int D, class R>
__device__ __forceinline__ void reorder_tile(const Geom& G, const Particles<R>& in, const Particles<R>& out,
                                             const uint32_t* __restrict__ cs_old, uint32_t* cs_new,
                                             uint32_t* __restrict__ count, uint32_t* perm, int64_t n,
                                             unsigned long long* __restrict__ ring, int mwords, Clock* clk, const int t)
{
    extern __shared__ __align__(16) uint32_t reorder_sm[];
    const int Tvol = G.Tvol;
    const int nrmax = reorder_ranges(G);
    uint32_t* cnt = reorder_sm;                                 // [warp][span of tile]
    uint32_t* base = cnt + kReorderWarps * Tvol;          // next slot of each span
    uint32_t* endv = base + Tvol;                         // end of each span's stayers
    uint32_t* list_q = endv + Tvol;                       // compacted old indices
    uint32_t* ustart = list_q + kReorderCap;              // ranges as listed
    uint32_t* ulen = ustart + nrmax;
    uint32_t* sstart = ulen + nrmax;                      // ranges by old index
    uint32_t* soff = sstart + nrmax;                      // exclusive prefix of lengths (nrmax + 1)
    uint32_t* wsum = soff + nrmax + 1;                    // per-warp totals (+1 spare)
    uint16_t* list_k = reinterpret_cast<uint16_t*>(wsum + kReorderWarps + 1);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t K0 = (int64_t)t * Tvol;

    if (!clk->active) {
        // no step was taken: same order, same cell starts
        const uint32_t b = cs_old[K0], e = cs_old[K0 + Tvol];
        for (uint32_t j = b + tid; j < e; j += kReorderThreads) copy_particle(in, out, D, j, j, G.inflow_face >= 0);
        const int last = (t == G.ntiles - 1) ? 1 : 0;
        for (int k = tid; k < Tvol + last; k += kReorderThreads) cs_new[K0 + k] = cs_old[K0 + k];
        return;
    }

    // tile position and its real spans
    const int tx = t % G.nt[0], ty = (t / G.nt[0]) % G.nt[1], tz = t / (G.nt[0] * G.nt[1]);
    int lo[3], hi[3], ex[3][2], nex[3];
    {
        const int tc[3] = {tx, ty, tz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = tc[a] * G.T[a];
            hi[a] = min(lo[a] + G.T[a], G.S[a]) - 1;
            nex[a] = axis_ring(G, a, lo[a], hi[a], ex[a]);
        }
    }
    const int ny = hi[1] - lo[1] + 1 + nex[1], nz = hi[2] - lo[2] + 1 + nex[2];
    const int nrows = ny * nz;
    int nr = 3 * nrows;
    // ring parts that particles entered this tile from (set by the G2PD step)
    __shared__ unsigned long long rbits[kReorderMaxRanges / 64];
    for (int w = tid; w < kReorderMaxRanges / 64; w += kReorderThreads)
        rbits[w] = w < mwords ? ring[(int64_t)t * mwords + w] : 0ull;

    for (int k = tid; k < kReorderWarps * Tvol; k += kReorderThreads) cnt[k] = 0u;
    int err = 0;
    for (int k = tid; k < Tvol; k += kReorderThreads) {
        const uint32_t s0 = cs_new[K0 + k], s1 = cs_new[K0 + k + 1];
        uint32_t stay = count[K0 + k];
        if (stay > s1 - s0) { err |= ERR_TILE; stay = 0; }
        base[k] = s0;
        endv[k] = s0 + stay;
    }
    __syncthreads();
    // 1. old index ranges of the tile's rows and of the ring parts entered
    for (int row = tid; row < nrows; row += kReorderThreads) {
        const int iy = row % ny, iz = row / ny;
        const bool inner = iy <= hi[1] - lo[1] && iz <= hi[2] - lo[2];
        const int y = iy <= hi[1] - lo[1] ? lo[1] + iy : ex[1][iy - (hi[1] - lo[1] + 1)];
        const int z = iz <= hi[2] - lo[2] ? lo[2] + iz : ex[2][iz - (hi[2] - lo[2] + 1)];
        auto marked = [&](int bit) { return ((rbits[bit >> 6] >> (bit & 63)) & 1ull) != 0ull; };
        {
            uint32_t b = 0, l = 0;
            if (inner || marked(3 * row)) {
                const int a0[3] = {lo[0], y, z}, a1[3] = {hi[0], y, z};
                b = cs_old[key_of<float>(G, a0)];
                l = cs_old[key_of<float>(G, a1) + 1] - b;
            }
            ustart[3 * row] = b;
            ulen[3 * row] = l;
        }
        for (int j = 0; j < 2; ++j) {
            uint32_t b = 0, l = 0;
            if (j < nex[0] && marked(3 * row + 1 + j)) {
                const int sp[3] = {ex[0][j], y, z};
                const uint32_t k = key_of<float>(G, sp);
                b = cs_old[k];
                l = cs_old[k + 1] - b;
            }
            ustart[3 * row + 1 + j] = b;
            ulen[3 * row + 1 + j] = l;
        }
    }
    __syncthreads();
    // the non-empty ranges, ordered by old index (one warp: typically the
    // tile's own rows and a few ring parts)
    __shared__ int nr_used;
    if (warp == 0) {
        const uint32_t lt = (1u << lane) - 1u;
        int k = 0;
        for (int b = 0; b < nr; b += 32) {
            // in place: an entry moves to a position at or before its own
            const int i = b + lane;
            const uint32_t st = i < nr ? ustart[i] : 0u, ln = i < nr ? ulen[i] : 0u;
            const uint32_t m = __ballot_sync(0xffffffffu, ln > 0u);
            if (ln > 0u) {
                ustart[k + __popc(m & lt)] = st;
                ulen[k + __popc(m & lt)] = ln;
            }
            k += __popc(m);
        }
        __syncwarp();
        // non-empty ranges are disjoint: their starts differ
        for (int i = lane; i < k; i += 32) {
            const uint32_t si = ustart[i];
            int rank = 0;
            for (int j = 0; j < k; ++j) rank += ustart[j] < si ? 1 : 0;
            sstart[rank] = si;
            soff[rank] = ulen[i];    // length for now; prefix below
        }
        __syncwarp();
        uint32_t carry = 0;
        for (int b = 0; b < k; b += 32) {
            const int i = b + lane;
            const uint32_t v = i < k ? soff[i] : 0u;
            uint32_t s = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += u;
            }
            if (i < k) soff[i] = carry + s - v;
            carry += __shfl_sync(0xffffffffu, s, 31);
        }
        if (lane == 0) {
            soff[k] = carry;
            nr_used = k;
        }
    }
    __syncthreads();
    nr = nr_used;
    const uint32_t C = soff[nr];
    const int lsh = G.tsh[0] + G.tsh[1] + G.tsh[2];
    const uint32_t lmask = (uint32_t)Tvol - 1u;

    uint32_t L = 0;
    for (uint32_t cb = 0; cb < C; cb += kReorderChunk) {
        // 2. keys of this chunk of candidates; keep the tile's particles
        uint32_t myq[kReorderItems], mykl[kReorderItems], bal[kReorderItems];
        uint32_t wtot = 0;
        int r = -1;
#pragma unroll
        for (int i = 0; i < kReorderItems; ++i) {
            const uint32_t c = cb + (uint32_t)(warp * 32 * kReorderItems + i * 32 + lane);
            bool hit = false;
            myq[i] = 0u;
            mykl[i] = 0u;
            if (c < C) {
                if (r < 0) {
                    int lo_r = 0, hi_r = nr - 1;     // last range with soff <= c
                    while (lo_r < hi_r) {
                        const int mid = (lo_r + hi_r + 1) >> 1;
                        if (soff[mid] <= c) lo_r = mid; else hi_r = mid - 1;
                    }
                    r = lo_r;
                } else {
                    while (soff[r + 1] <= c) ++r;
                }
                const uint32_t q = sstart[r] + (c - soff[r]);
                const uint32_t k = in.key[q];
                hit = (k >> lsh) == (uint32_t)t;
                myq[i] = q;
                mykl[i] = k & lmask;
            }
            bal[i] = __ballot_sync(0xffffffffu, hit);
            wtot += __popc(bal[i]);
        }
        if (lane == 0) wsum[warp] = wtot;
        __syncthreads();
        uint32_t off = L, tot = 0;
#pragma unroll
        for (int w = 0; w < kReorderWarps; ++w) {
            const uint32_t v = wsum[w];
            off += w < warp ? v : 0u;
            tot += v;
        }
        const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
        for (int i = 0; i < kReorderItems; ++i) {
            if ((bal[i] >> lane) & 1u) {
                const uint32_t at = off + __popc(bal[i] & lt);
                list_q[at] = myq[i];
                list_k[at] = (uint16_t)mykl[i];
            }
            off += __popc(bal[i]);
        }
        L += tot;
        __syncthreads();
        if (L + kReorderChunk <= (uint32_t)kReorderCap && cb + kReorderChunk < C) continue;

        // 3. stable placement of the compacted particles
        const uint32_t per = (L + kReorderWarps - 1) / kReorderWarps;
        const uint32_t wb = min(L, per * warp), we = min(L, wb + per);
        uint32_t* wc = cnt + warp * Tvol;
        for (uint32_t j0 = wb; j0 < we; j0 += 32) {
            const uint32_t j = j0 + lane;
            const bool valid = j < we;
            const uint32_t kl = valid ? list_k[j] : 0xffffffffu;
            const uint32_t peers = __match_any_sync(0xffffffffu, kl);
            if (valid && lane == __ffs(peers) - 1) wc[kl] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        for (int k = tid; k < Tvol; k += kReorderThreads) {
            uint32_t run = base[k];
#pragma unroll
            for (int w = 0; w < kReorderWarps; ++w) {
                const uint32_t v = cnt[w * Tvol + k];
                cnt[w * Tvol + k] = run;
                run += v;
            }
            base[k] = run;
        }
        __syncthreads();
        constexpr int kB = sizeof(R) == 4 ? 4 : 2;     // particles per lane per batch
        for (uint32_t j0 = wb; j0 < we; j0 += 32 * kB) {
            uint32_t qv[kB], pv[kB];
            bool okv[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const uint32_t j = j0 + u * 32 + lane;
                const bool valid = j < we;
                const uint32_t kl = valid ? list_k[j] : 0xffffffffu;
                const uint32_t peers = __match_any_sync(0xffffffffu, kl);
                const int leader = __ffs(peers) - 1;
                uint32_t bv = 0;
                if (valid && lane == leader) bv = wc[kl];
                bv = __shfl_sync(0xffffffffu, bv, leader);
                const uint32_t pos = bv + __popc(peers & lt);
                okv[u] = valid && pos < endv[kl];
                if (valid && !okv[u]) err |= ERR_TILE;
                qv[u] = valid ? list_q[j] : 0u;
                pv[u] = pos;
                __syncwarp();
                if (valid && lane == leader) wc[kl] = bv + __popc(peers);
                __syncwarp();
            }
            copy_batch<kB>(in, out, D, qv, pv, okv, G.inflow_face >= 0);
        }
        __syncthreads();
        for (int k = tid; k < kReorderWarps * Tvol; k += kReorderThreads) cnt[k] = 0u;
        L = 0;
        __syncthreads();
    }

    for (int w = tid; w < mwords; w += kReorderThreads) ring[(int64_t)t * mwords + w] = 0ull;
    // 4. every span got exactly its stayers; then its recycled particles by id
    for (int k = tid; k < Tvol; k += kReorderThreads) {
        const int64_t K = K0 + k;
        if (count[K]) count[K] = 0u;
        if (base[k] != endv[k]) { err |= ERR_TILE; continue; }
        const uint32_t fb = endv[k], fe = cs_new[K + 1];
        if (fb == fe) continue;
        if (fb > fe || perm == nullptr) { err |= ERR_TILE; continue; }
        bool ok = true;
        for (uint32_t i = fb; i < fe; ++i) ok = ok && (int64_t)perm[i] < n;
        if (!ok) { err |= ERR_TILE; continue; }
        for (uint32_t i = fb + 1; i < fe; ++i) {
            const uint32_t v = perm[i], vid = in.id[v];
            uint32_t j = i;
            while (j > fb && in.id[perm[j - 1]] > vid) { perm[j] = perm[j - 1]; --j; }
            perm[j] = v;
        }
        for (uint32_t i = fb; i < fe; ++i) copy_particle(in, out, D, perm[i], i, true);
    }
    if (err) atomicOr(&clk->err, err);
}

template <int D, class R>
__global__ void __launch_bounds__(kReorderThreads, 3) k_reorder(Geom G, Particles<R> in, Particles<R> out,
                                                             const uint32_t* __restrict__ cs_old, uint32_t* cs_new,
                                                             uint32_t* __restrict__ count, uint32_t* perm, int64_t n,
                                                             unsigned long long* __restrict__ ring, int mwords,
                                                             Clock* clk)
{
    reorder_tile<D, R>(G, in, out, cs_old, cs_new, count, perm, n, ring, mwords, clk, blockIdx.x);
}

// Sorted keys from the cell-start table (for reading the state back).
__global__ void k_keys_from_start(const uint32_t* cs, int64_t nkey, uint32_t* out)
{
    for (int64_t K = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; K < nkey; K += (int64_t)gridDim.x * blockDim.x)
        for (uint32_t j = cs[K]; j < cs[K + 1]; ++j) out[j] = (uint32_t)K;
}

}  // namespace mpm
