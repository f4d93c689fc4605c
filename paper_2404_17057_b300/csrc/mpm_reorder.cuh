// mpm_reorder.cuh -- per-step stable re-order of the particles (Sec. 3 step xii)
// on tiles that own regions of the particle buffers.
//
// Tile t's particles occupy the first n_t slots of its region [tbase[t],
// tbase[t + 1]) in buffer tpar[t], span after span; its cell starts are the
// entries tile_cs0(t) .. tile_cs0(t) + Tvol of cs[tpar[t]].  The G2PD step
// writes each particle's new key, moves one count from the old span to the
// new one of every particle that changes span, marks the tiles whose lists
// change (a particle left or entered one of their spans) and the ring parts
// particles entered a tile from, and lists the particles recycled at the
// inflow.  The time-step rule of Sec. 4.1 (checked
// by the G2PD step) keeps every other particle within one span of where it
// was, so the particles that end up in a tile come from the tile's old spans
// and one ring of spans around it.
//
// Pass 0, one tile at a time per CTA:
//   - a tile whose lists did not change keeps its particles where they are
//     (most of a domain at rest costs nothing);
//   - a changed tile lists the old slot ranges of that neighbourhood, streams
//     their keys, compacts the particles that now belong to it in old order,
//     ranks them per new span (stable: a span keeps its particles' previous
//     order) and copies each into its new slot in the same region of the
//     other buffer; the particles recycled into it follow the others of
//     their span, ordered by id; then it switches to that buffer;
//   - a tile that would outgrow its region raises the clock's overflow flag
//     and writes nothing.
// If any tile overflowed, the state is laid out again: every tile's old
// particles are first brought into buffer 0 (k_consolidate), regions are
// sized anew from the new counts (k_relayout_bases), and pass 1 rebuilds
// every tile from buffer 0 into buffer 1.  k_reorder_done clears the step's
// marks and installs the new regions.
#pragma once
#include "mpm_kernels.cuh"
#include "mpm_sort.cuh"

namespace mpm {

constexpr int kReorderThreads = 128;
constexpr int kReorderWarps = kReorderThreads / 32;
constexpr int kReorderItems = 8;                                  // keys per thread per chunk
constexpr int kReorderChunk = kReorderThreads * kReorderItems;
constexpr int kReorderCap = 1024;                                 // compacted particles per flush
constexpr int kReorderMaxRanges = 1024;
constexpr int kReorderFarCap = 512;                               // recycled arrivals per tile
// Resident re-order blocks per SM: a tile's re-order is a chain of short
// dependent phases, so many small blocks hide each other's latency.
constexpr int kReorderBlocksPerSM = 8;

// Region of a tile with n particles: room for twice as many plus 64, in
// multiples of 32 slots (128-byte aligned starts in single precision).
__host__ __device__ inline uint32_t region_slots(uint32_t n) { return (2u * n + 64u + 31u) & ~31u; }

__host__ inline size_t reorder_smem(const Geom& G)
{
    const size_t T = (size_t)G.Tvol, nr = (size_t)reorder_ranges(G);
    return ((kReorderWarps + 3) * T + kReorderCap + 4 * nr + 2 + kReorderWarps) * 4 + kReorderCap * 2 +
           (size_t)kReorderFarCap * 8;
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

// Copy kB particles per lane, slot q[u] -> slot j[u], where ok[u]: all loads
// first, so that up to 12 kB independent loads per lane are in flight.
template <int kB, class R>
__device__ __forceinline__ void copy_batch(const Particles<R>& s, const Particles<R>& out, int D, const uint32_t* q,
                                           const uint32_t* j, const bool* ok, bool with_gen)
{
    R xv[kB][6], M[kB], rho[kB], E[kB], Q[kB];
    uint32_t id[kB], gen[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
        if (!ok[u]) continue;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a < D) { xv[u][a] = s.x[a][q[u]]; xv[u][3 + a] = s.v[a][q[u]]; }
        M[u] = s.M[q[u]];
        rho[u] = s.rho[q[u]];
        E[u] = s.E[q[u]];
        Q[u] = s.Q[q[u]];
        id[u] = s.id[q[u]];
        gen[u] = with_gen ? s.gen[q[u]] : 0u;
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

// What one re-order pass needs of a simulation.
template <class R>
struct ReorderArgs {
    Particles<R> pt;                // both buffers (absolute slots; buffer 1 from nslots)
    uint32_t nslots;
    uint32_t* cs[2];
    const uint8_t* tpar_old;        // buffer of each tile during the step
    uint8_t* tpar_new;              // ... after the re-order
    const uint32_t* tbase;          // regions (ntiles + 1 entries)
    uint32_t* tbase_next;           // regions of a relayout
    uint32_t* tcount;               // particles of each tile after the step
    Reorder ro;
    Clock* clk;
};

// Tile t, pass `mode` (0: changed tiles into their other buffer; 1: relayout,
// every tile from buffer 0 into buffer 1, only if a tile overflowed).
template <int D, class R>
__device__ __forceinline__ void reorder_tile(const Geom& G, const ReorderArgs<R>& A, const int mode, const int t)
{
    extern __shared__ __align__(16) uint32_t reorder_sm[];
    const int Tvol = G.Tvol;
    const int nrmax = reorder_ranges(G);
    uint32_t* cnt = reorder_sm;                           // [warp][span of tile]
    uint32_t* base = cnt + kReorderWarps * Tvol;          // next slot of each span
    uint32_t* endv = base + Tvol;                         // end of each span's stayers
    uint32_t* news = endv + Tvol;                         // new start of each span
    uint32_t* list_q = news + Tvol;                       // compacted slots
    uint32_t* ustart = list_q + kReorderCap;              // ranges as listed
    uint32_t* ulen = ustart + nrmax;
    uint32_t* sstart = ulen + nrmax;                      // ranges by old slot
    uint32_t* soff = sstart + nrmax;                      // exclusive prefix of lengths (nrmax + 1)
    uint32_t* wsum = soff + nrmax + 1;                    // per-warp totals (+1 spare)
    uint16_t* list_k = reinterpret_cast<uint16_t*>(wsum + kReorderWarps + 1);
    uint2* farl = reinterpret_cast<uint2*>(list_k + kReorderCap);   // {local span, slot}, by id

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t K0 = (int64_t)t * Tvol;
    const int64_t C0 = tile_cs0(G, t);
    Clock* clk = A.clk;
    const bool relayout = mode == 1;
    const int tp = relayout ? 0 : A.tpar_old[t];
    __shared__ int s_skip;

    if (!relayout) {
        // an unchanged tile (and every tile of a step that was not taken)
        if (!clk->active || !A.ro.dirty[t]) {
            if (tid == 0) {
                A.tpar_new[t] = (uint8_t)tp;
                A.tcount[t] = A.cs[tp][C0 + Tvol] - A.cs[tp][C0];
            }
            return;
        }
    }
    const int dst = relayout ? 1 : 1 - tp;
    const uint32_t* rb = relayout ? A.tbase_next : A.tbase;
    const uint32_t rbeg = (dst ? A.nslots : 0u) + rb[t], rcap = rb[t + 1] - rb[t];
    const uint32_t NS = A.nslots;
    int err = 0;

    // new span counts (old counts plus the step's changes) -> new starts
    // (block scan), and the tile's total
    const uint32_t* cso = A.cs[tp];          // the tile's old cell starts (relayout: consolidated)
    uint32_t total = 0;
    for (int k0 = 0; k0 < Tvol; k0 += kReorderThreads) {
        const int k = k0 + tid;
        const uint32_t c = k < Tvol ? cso[C0 + k + 1] - cso[C0 + k] + A.ro.count[K0 + k] : 0u;
        const uint32_t inc = block_inclusive_scan(c, wsum);
        if (k < Tvol) news[k] = rbeg + total + inc - c;
        if (tid == kReorderThreads - 1) wsum[kReorderWarps] = inc;
        __syncthreads();
        total += wsum[kReorderWarps];
        __syncthreads();
    }
    if (tid == 0) {
        s_skip = 0;
        if (!relayout) A.tcount[t] = total;
        if (total > rcap) {
            if (!relayout) atomicOr(&clk->overflow, 1u);
            else atomicOr(&clk->err, ERR_TILE);
            s_skip = 1;
            A.tpar_new[t] = (uint8_t)tp;
        }
    }
    __syncthreads();
    if (s_skip) return;

    // particles recycled into this tile (they may come from anywhere)
    const int lsh = G.tsh[0] + G.tsh[1] + G.tsh[2];
    const uint32_t lmask = (uint32_t)Tvol - 1u;
    __shared__ uint32_t s_nfar;
    if (tid == 0) s_nfar = 0;
    for (int k = tid; k < Tvol; k += kReorderThreads) {
        endv[k] = 0u;
#pragma unroll
        for (int w = 0; w < kReorderWarps; ++w) cnt[w * Tvol + k] = 0u;
    }
    __syncthreads();
    const uint32_t F = A.ro.far_cap ? min(clk->nfar, A.ro.far_cap) : 0u;
    for (uint32_t i = tid; i < F; i += kReorderThreads) {
        const uint2 e = A.ro.far[i];
        if ((e.x >> lsh) != (uint32_t)t) continue;
        const uint32_t at = atomicAdd(&s_nfar, 1u);
        if (at < (uint32_t)kReorderFarCap) {
            // (a relayout reads every old particle from buffer 0)
            farl[at] = make_uint2(e.x & lmask, relayout && e.y >= NS ? e.y - NS : e.y);
            atomicAdd(&endv[e.x & lmask], 1u);      // recycled arrivals per span (for now)
        } else {
            err |= ERR_TILE;
        }
    }
    __syncthreads();
    const uint32_t nfar = min(s_nfar, (uint32_t)kReorderFarCap);
    for (int k = tid; k < Tvol; k += kReorderThreads) {
        const uint32_t nf = endv[k];
        const uint32_t c = (k + 1 < Tvol ? news[k + 1] : rbeg + total) - news[k];
        if (nf > c) err |= ERR_TILE;
        base[k] = news[k];
        endv[k] = news[k] + (nf > c ? 0u : c - nf);
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
    const int mwords = A.ro.mwords;
    __shared__ unsigned long long rbits[kReorderMaxRanges / 64];
    for (int w = tid; w < kReorderMaxRanges / 64; w += kReorderThreads)
        rbits[w] = w < mwords ? A.ro.ring[(int64_t)t * mwords + w] : 0ull;
    __syncthreads();
    // old slot range of the spans a0..a1 of one row (one tile)
    auto range = [&](const int a0[3], const int a1[3], uint32_t& b, uint32_t& l) {
        const uint32_t k0 = key_of<float>(G, a0), k1 = key_of<float>(G, a1);
        const uint32_t* cso = A.cs[relayout ? 0 : A.tpar_old[k0 >> lsh]];
        b = cso[cs_index(G, k0)];
        l = cso[cs_index(G, k1) + 1] - b;
    };
    // 1. old slot ranges of the tile's rows and of the ring parts entered
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
                range(a0, a1, b, l);
            }
            ustart[3 * row] = b;
            ulen[3 * row] = l;
        }
        for (int j = 0; j < 2; ++j) {
            uint32_t b = 0, l = 0;
            if (j < nex[0] && marked(3 * row + 1 + j)) {
                const int sp[3] = {ex[0][j], y, z};
                range(sp, sp, b, l);
            }
            ustart[3 * row + 1 + j] = b;
            ulen[3 * row + 1 + j] = l;
        }
    }
    __syncthreads();
    // the non-empty ranges in old key order (one warp: typically the tile's
    // own rows and a few ring parts)
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
        // non-empty ranges are disjoint.  Regions lie in tile order at the
        // same places of both buffers, so the slot within its buffer gives
        // the old key order
        for (int i = lane; i < k; i += 32) {
            const uint32_t si = ustart[i];
            const uint32_t sv = si >= NS ? si - NS : si;
            int rank = 0;
            for (int j = 0; j < k; ++j) {
                const uint32_t vj = ustart[j] >= NS ? ustart[j] - NS : ustart[j];
                rank += (vj < sv) ? 1 : 0;
            }
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
    const bool with_gen = G.inflow_face >= 0;

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
                const uint32_t k = A.pt.key[q];
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
        constexpr int kB = 2;                          // particles per lane per batch
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
                uint32_t b0 = 0;
                if (valid && lane == leader) b0 = wc[kl];
                b0 = __shfl_sync(0xffffffffu, b0, leader);
                const uint32_t pos = b0 + __popc(peers & lt);
                okv[u] = valid && pos < endv[kl];
                if (valid && !okv[u]) err |= ERR_TILE;
                qv[u] = valid ? list_q[j] : 0u;
                pv[u] = pos;
                __syncwarp();
                if (valid && lane == leader) wc[kl] = b0 + __popc(peers);
                __syncwarp();
            }
            copy_batch<kB>(A.pt, A.pt, D, qv, pv, okv, with_gen);
        }
        __syncthreads();
        for (int k = tid; k < kReorderWarps * Tvol; k += kReorderThreads) cnt[k] = 0u;
        L = 0;
        __syncthreads();
    }

    // 4. every span got exactly its stayers; then its recycled particles by
    // id (the tile's recycled arrivals, sorted by (span, id): few)
    if (nfar > 0) {
        if (tid == 0) {
            for (uint32_t i = 1; i < nfar; ++i) {
                const uint2 v = farl[i];
                const uint32_t vid = A.pt.id[v.y];
                uint32_t j = i;
                while (j > 0) {
                    const uint2 u = farl[j - 1];
                    const uint32_t uid = A.pt.id[u.y];
                    if (u.x < v.x || (u.x == v.x && uid < vid)) break;
                    farl[j] = u;
                    --j;
                }
                farl[j] = v;
            }
        }
        __syncthreads();
        // arrivals of one span are consecutive in farl: place each after the
        // span's stayers
        for (uint32_t i = tid; i < nfar; i += kReorderThreads) {
            const uint2 v = farl[i];
            uint32_t first = i;
            while (first > 0 && farl[first - 1].x == v.x) --first;
            const uint32_t pos = endv[v.x] + (i - first);
            if (pos < (v.x + 1 < (uint32_t)Tvol ? news[v.x + 1] : rbeg + total))
                copy_particle(A.pt, A.pt, D, v.y, pos, true);
            else
                err |= ERR_TILE;
        }
    }
    for (int k = tid; k < Tvol; k += kReorderThreads)
        if (base[k] != endv[k]) err |= ERR_TILE;
    // the new cell starts, and the tile's buffer
    uint32_t* csn = A.cs[dst];
    for (int k = tid; k < Tvol; k += kReorderThreads) csn[C0 + k] = news[k];
    if (tid == 0) {
        csn[C0 + Tvol] = rbeg + total;
        A.tpar_new[t] = (uint8_t)dst;
    }
    if (err) atomicOr(&clk->err, err);
}

// Pass `mode` over the tiles of one simulation (persistent CTAs).
template <int D, class R>
__global__ void __launch_bounds__(kReorderThreads, kReorderBlocksPerSM) k_reorder(Geom G, ReorderArgs<R> A, int mode)
{
    if (mode == 1 && !A.clk->overflow) return;
    for (int t = blockIdx.x; t < G.ntiles; t += gridDim.x) {
        reorder_tile<D, R>(G, A, mode, t);
        __syncthreads();
    }
}

// Relayout, step 1: the old particles (with the new keys the G2PD step gave
// them) and the cell starts of every tile in buffer 1 are copied to the same
// slots / entries of buffer 0.
template <int D, class R>
__device__ __forceinline__ void consolidate_tile(const Geom& G, const ReorderArgs<R>& A, const int t)
{
    if (A.tpar_old[t] != 1) return;
    const int64_t C0 = tile_cs0(G, t);
    const uint32_t b = A.cs[1][C0], e = A.cs[1][C0 + G.Tvol], NS = A.nslots;
    for (uint32_t j = b + threadIdx.x; j < e; j += blockDim.x) {
        copy_particle(A.pt, A.pt, D, j, j - NS, true);
        A.pt.key[j - NS] = A.pt.key[j];
    }
    for (int k = threadIdx.x; k <= G.Tvol; k += blockDim.x) A.cs[0][C0 + k] = A.cs[1][C0 + k] - NS;
}

template <int D, class R>
__global__ void __launch_bounds__(kReorderThreads) k_consolidate(Geom G, ReorderArgs<R> A)
{
    if (!A.clk->overflow) return;
    for (int t = blockIdx.x; t < G.ntiles; t += gridDim.x) consolidate_tile<D, R>(G, A, t);
}

// Relayout, step 2: regions sized for the new counts (one block).
__device__ __forceinline__ void relayout_bases_block(const uint32_t* tcount, int ntiles, uint32_t* tbase_next)
{
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b = 0; b < ntiles; b += blockDim.x) {
        const int i = b + threadIdx.x;
        const uint32_t v = i < ntiles ? region_slots(tcount[i]) : 0u;
        const uint32_t inc = block_inclusive_scan(v, ws);
        const uint32_t c = carry;
        if (i < ntiles) tbase_next[i] = c + inc - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) tbase_next[ntiles] = carry;
}

__global__ void __launch_bounds__(1024) k_relayout_bases(const uint32_t* tcount, int ntiles, uint32_t* tbase_next,
                                                         const Clock* clk)
{
    if (!clk->overflow) return;
    relayout_bases_block(tcount, ntiles, tbase_next);
}

// End of the re-order: clear the changed tiles' marks, install the regions of
// a relayout.  One warp per tile (a changed tile clears Tvol counts).
__device__ __forceinline__ void reorder_done_tile(int tvol, const Reorder& ro, Clock* clk, uint32_t* tbase,
                                                  const uint32_t* tbase_next, int t, int ntiles, int lane)
{
    // only a changed tile has count changes and ring marks
    if (ro.dirty[t]) {
        for (int w = lane; w < ro.mwords; w += 32) ro.ring[(int64_t)t * ro.mwords + w] = 0ull;
        uint4* c4 = reinterpret_cast<uint4*>(ro.count + (int64_t)t * tvol);
        for (int k = lane; k < tvol / 4; k += 32) c4[k] = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();                       // every lane has read the mark
        if (lane == 0) ro.dirty[t] = 0u;
    }
    if (lane == 0 && clk->overflow) {
        tbase[t] = tbase_next[t];
        if (t == ntiles - 1) tbase[ntiles] = tbase_next[ntiles];
        if (t == 0) clk->relayouts += 1;
    }
}

__global__ void k_reorder_done(Geom G, Reorder ro, Clock* clk, uint32_t* tbase, const uint32_t* tbase_next)
{
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = w0; t < G.ntiles; t += nw)
        reorder_done_tile(G.Tvol, ro, clk, tbase, tbase_next, (int)t, G.ntiles, threadIdx.x & 31);
}

// Initial layout: the particles of a compact key order (cell starts cc[key],
// nkey + 1 entries, of buffer `from`) spread into the regions tbase of buffer
// `to`, with the per-tile cell starts cs_to.
template <int D, class R>
__global__ void k_spread(Geom G, Particles<R> from, Particles<R> to, const uint32_t* cc, const uint32_t* tbase,
                         uint32_t* cs_to)
{
    for (int t = blockIdx.x; t < G.ntiles; t += gridDim.x) {
        const int64_t K0 = (int64_t)t * G.Tvol, C0 = tile_cs0(G, t);
        const uint32_t b = cc[K0], e = cc[K0 + G.Tvol], rb = tbase[t];
        for (uint32_t j = b + threadIdx.x; j < e; j += blockDim.x) copy_particle(from, to, D, j, rb + (j - b), true);
        for (int k = threadIdx.x; k <= G.Tvol; k += blockDim.x) cs_to[C0 + k] = rb + (cc[K0 + k] - b);
    }
}

// Particles of each tile from a compact cell-start table (nkey + 1 entries).
__global__ void k_tile_counts_compact(const uint32_t* cc, int64_t ntiles, int tvol, uint32_t* counts)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x)
        counts[t] = cc[(t + 1) * tvol] - cc[t * tvol];
}

// Compact cell starts (key order without gaps) from the per-tile table:
// out[key] = toff[t] + (start of the span - start of the tile), out[nkey] = n.
__global__ void k_compact_starts(Geom G, const uint32_t* cs0, const uint32_t* cs1, const uint8_t* tpar,
                                 const uint32_t* toff, uint32_t* out)
{
    for (int64_t key = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; key <= G.nkey;
         key += (int64_t)gridDim.x * blockDim.x) {
        if (key == G.nkey) { out[key] = toff[G.ntiles]; continue; }
        const int64_t t = key / G.Tvol;
        const uint32_t* cs = tpar[t] ? cs1 : cs0;
        const int64_t C0 = tile_cs0(G, t);
        out[key] = toff[t] + (cs[C0 + (key - t * G.Tvol)] - cs[C0]);
    }
}

// Sorted keys from a compact cell-start table (for reading the state back).
__global__ void k_keys_from_start(const uint32_t* cs, int64_t nkey, uint32_t* out)
{
    for (int64_t K = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; K < nkey; K += (int64_t)gridDim.x * blockDim.x)
        for (uint32_t j = cs[K]; j < cs[K + 1]; ++j) out[j] = (uint32_t)K;
}

}  // namespace mpm
