// mpm_kernels.cuh -- sm_103a kernels of one MPM time step (Sec. 3, Algorithm 1).
//
// The particles are kept in key order, so the particles of one tile of spans
// are contiguous.  Each kernel below gives one CTA one tile: the CTA stages
// the tile's node window (tile + p halo nodes per axis) in shared memory,
// works on the tile's particles from there, and touches global node memory
// once per window node.
//   k_p2g       steps ii   : P2G of m and M V, P2GD of (P+Q) M/rho
//   k_grid_g2p  steps iii-vi: BC + momentum update at window load, G2P of f/m,
//                             V' = V + dt A, momentum P2G of M V'
//   k_g2pd      steps vii-x: BC on the new momentum, G2PD div V, E/rho/P/Q
//                             update, move with Vbar, recycling, new key
//   k_finalize  step xiii  : time advance and the CFL step for the next step
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>

namespace mpm {

enum : int { ERR_NONFINITE = 1, ERR_CFL = 2, ERR_TILE = 4, ERR_TIMEOUT = 8 };

constexpr uint32_t kFarFlag = 0x80000000u;   // key bit of a particle recycled this step

// Per-step re-order bookkeeping written by the G2PD step.
struct Reorder {
    uint32_t* count;               // per span: particles gained minus lost in the step (mod 2^32)
    uint2* far;                    // particles recycled this step: {new key, old slot}
    uint32_t far_cap;              // entries of far (0: the problem has no inflow face)
    int mwords;                    // words of ring bits per tile
    unsigned long long* ring;      // per tile: parts of its one-span ring that particles entered from
    uint32_t* dirty;               // per tile: its span lists change in this step
};

struct Geom {
    int dim, p;
    int n[3], per[3], S[3], N[3], g[3], T[3], nt[3], W[3];
    int tsh[3];                     // log2 of the tile edges (powers of two)
    int Tvol, Wvol, ntiles;
    int pitch;                      // stored x-extent of a node row (N[0] rounded up to 4)
    int64_t nnode, nnode_p, nkey;   // nodes, stored nodes (padded rows), keys
    int bc[6];
    int inflow_face;                // -1: none
    double h, inv_h, lo[3], hi[3];
    double gamma, c0, c1, cfl, inflow_rho, inflow_p, inflow_v[3], inflow_e;
    uint64_t seed;
    float qscale[3];                // fixed point: 2^32 / unit (mass, momentum, force)
    float dqscale[3];               // unit / 2^32
    float inv_w[2];                 // 1 / W[0], 1 / W[1] (window slot decoding)
};

struct Clock {
    double t, t_end, dt_fixed, dt_next, dt_cur;
    long long step;
    int active, done, last, err;
    unsigned long long vmax_bits, cmax_bits;   // bits of non-negative doubles
    unsigned nfar;                             // recycled particles this step
    int par;                                   // batched runs: parity of the step (tile-buffer table in use)
    long long step_end;                        // > 0: no step starts at or after this count
    unsigned overflow;                         // a tile outgrew its region in this step's re-order
    long long relayouts;                       // steps whose re-order laid the state out again
};

// Tiles own regions of the particle buffers: tile t's particles occupy the
// first n_t slots of its region in buffer tpar[t], span after span, and its
// cell starts are the Tvol + 1 entries tile_cs0(t) .. tile_cs0(t) + Tvol of
// cs[tpar[t]] (the start of each span and the end of the tile's particles).
// The two buffers of a field are one array of 2 nslots slots (buffer b from
// slot b nslots), and cell starts hold absolute slots: a kernel reaches a
// tile's particles through the buffer-0 pointers whichever buffer they are in.
__host__ __device__ inline int64_t tile_cs0(const Geom& G, int64_t t) { return t * (int64_t)(G.Tvol + 1); }
// Entry of the cell-start table of the span with key `key`.
__host__ __device__ inline int64_t cs_index(const Geom& G, uint32_t key)
{
    return (int64_t)key + (int64_t)(key >> (G.tsh[0] + G.tsh[1] + G.tsh[2]));
}


// Rows of spans (y, z) of a tile and its one-span ring, times three x-parts
// (the tile's own x-range and the span before and after it).
__host__ __device__ inline int reorder_ranges(const Geom& G)
{
    return 3 * (G.T[1] + 2) * (G.dim == 3 ? G.T[2] + 2 : 1);
}

// The real spans [lo, hi] of a tile along axis a, plus the up to two span
// coordinates next to them (wrapped on a periodic axis), without repeats.
__device__ __forceinline__ int axis_ring(const Geom& G, int a, int lo, int hi, int ex[2])
{
    int m = 0;
    if (a >= G.dim) return 0;
    int l = lo - 1, r = hi + 1;
    if (G.per[a]) {
        l = l < 0 ? l + G.n[a] : l;
        r = r >= G.n[a] ? r - G.n[a] : r;
    }
    if (l >= 0 && l < G.S[a] && (l < lo || l > hi)) ex[m++] = l;
    if (r >= 0 && r < G.S[a] && (r < lo || r > hi) && (m == 0 || ex[0] != r)) ex[m++] = r;
    return m;
}

// Ring part of tile t that contains span `old` (numbered as the re-order
// lists them: 3 * (iz * ny + iy) + x part), or -1 if it is not next to t.
__device__ __forceinline__ int ring_bit(const Geom& G, uint32_t t, const int old[3])
{
    const int tc[3] = {(int)(t % (uint32_t)G.nt[0]), (int)((t / (uint32_t)G.nt[0]) % (uint32_t)G.nt[1]),
                       (int)(t / (uint32_t)(G.nt[0] * G.nt[1]))};
    int idx[3] = {0, 0, 0}, ny = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= G.dim) continue;
        const int lo = tc[a] * G.T[a], hi = min(lo + G.T[a], G.S[a]) - 1;
        int ex[2];
        const int m = axis_ring(G, a, lo, hi, ex);
        if (a == 1) ny = hi - lo + 1 + m;
        if (old[a] >= lo && old[a] <= hi) {
            idx[a] = a == 0 ? 0 : old[a] - lo;
        } else {
            int f = -1;
            for (int j = 0; j < m; ++j)
                if (ex[j] == old[a]) f = j;
            if (f < 0) return -1;
            idx[a] = a == 0 ? 1 + f : hi - lo + 1 + f;
        }
    }
    return 3 * (idx[2] * ny + idx[1]) + idx[0];
}

__device__ __forceinline__ void tile_origin(const Geom& G, int tile, int so[3]);

// New key of particle k (absolute slot k), whose old key was okey (a span
// of `tile`).  A particle that changes span moves one count from its old span
// to its new one (most particles keep their span and cost nothing here) and
// marks the tile it leaves and the tile it enters as changed; one that enters
// another tile marks the ring part it comes from.  Recycled particles go to
// the far list (they may jump anywhere) and carry the flag bit.
__device__ __forceinline__ uint32_t record_key(const Geom& G, const Reorder& ro, Clock* clk, uint32_t key,
                                               bool recycled, uint32_t k, int tile, uint32_t okey, int& err)
{
    const int lsh = G.tsh[0] + G.tsh[1] + G.tsh[2];
    const uint32_t nt = key >> lsh;
    if (recycled || key != okey) {
        atomicAdd(&ro.count[key], 1u);
        atomicSub(&ro.count[okey], 1u);
        ro.dirty[tile] = 1u;
        ro.dirty[nt] = 1u;
        if (recycled) {
            const unsigned slot = atomicAdd(&clk->nfar, 1u);
            if (slot < ro.far_cap) ro.far[slot] = make_uint2(key, k);
            else err |= ERR_TILE;
            return key | kFarFlag;
        }
        // a particle that enters another tile: mark the ring part it comes from
        if (nt != (uint32_t)tile) {
            const uint32_t l = okey & ((uint32_t)G.Tvol - 1u);
            int old[3];
            tile_origin(G, tile, old);
            old[0] += (int)(l & (uint32_t)(G.T[0] - 1));
            old[1] += (int)((l >> G.tsh[0]) & (uint32_t)(G.T[1] - 1));
            old[2] += (int)(l >> (G.tsh[0] + G.tsh[1]));
            const int bit = ring_bit(G, nt, old);
            if (bit >= 0) atomicOr(&ro.ring[(int64_t)nt * ro.mwords + (bit >> 6)], 1ull << (bit & 63));
        }
    }
    return key;
}

template <class R>
struct Particles {
    R* x[3];
    R* v[3];
    R* M;
    R* rho;
    R* E;
    R* Q;
    uint32_t* id;
    uint32_t* key;
    uint32_t* gen;   // times the particle has been recycled (keys its Philox draw)
};

// The particle state seen by the tile kernels.
template <class R>
struct TileState {
    Particles<R> pt;               // both buffers (absolute slots)
    uint32_t* cs[2];
    const uint8_t* tpar;           // buffer of each tile
};

template <class A, class R>
struct Grid {
    A* m;
    A* mv[3];
    A* f[3];
    A* mv2[3];
    const uint8_t* mask;
    const R* nrm[3];
};

// ----------------------------------------------------- rounding-exact ops
template <class R> struct Op;
template <> struct Op<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float dvd(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float sqr(float a) { return __fsqrt_rn(a); }
    static __device__ __forceinline__ float flr(float a) { return floorf(a); }
};
template <> struct Op<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double dvd(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double sqr(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double flr(double a) { return floor(a); }
};

// ---------------------------------------------------- accumulator types
template <class A> struct Acc;
template <> struct Acc<float> {
    static constexpr bool kFixed = false;
    static __device__ __forceinline__ float from(float c, float) { return c; }
    template <bool>
    static __device__ __forceinline__ float from_t(float c, float) { return c; }
    static __device__ __forceinline__ void add(float* p, float v) { atomicAdd(p, v); }
    static __device__ __forceinline__ float to_real(float a, float) { return a; }
};
template <> struct Acc<double> {
    static constexpr bool kFixed = false;
    static __device__ __forceinline__ double from(double c, float) { return c; }
    template <bool>
    static __device__ __forceinline__ double from_t(double c, float) { return c; }
    static __device__ __forceinline__ void add(double* p, double v) { atomicAdd(p, v); }
    static __device__ __forceinline__ double to_real(double a, float) { return a; }
};
// Fixed-point rounding of a quantised value v = c * S to int64, ties to
// even.  The 64-bit conversion issues at a small fraction of the 32-bit
// rate, so values known to lie below 2^31 in magnitude (SMALL) take the
// 32-bit conversion, which is exact there.
template <bool SMALL>
__device__ __forceinline__ long long round_ll(float v)
{
    if constexpr (SMALL) return (long long)__float2int_rn(v);
    else return __float2ll_rn(v);
}

template <> struct Acc<long long> {
    static constexpr bool kFixed = true;
    // Fixed point: a binary32 contribution c becomes round(c * 2^32/U).
    static __device__ __forceinline__ long long from(float c, float s) { return round_ll<false>(__fmul_rn(c, s)); }
    template <bool SMALL>
    static __device__ __forceinline__ long long from_t(float c, float s)
    {
        return round_ll<SMALL>(__fmul_rn(c, s));
    }
    static __device__ __forceinline__ void add(long long* p, long long v)
    {
        atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
    }
    static __device__ __forceinline__ float to_real(long long a, float ds) { return __fmul_rn(__ll2float_rn(a), ds); }
};

// --------------------------------------------------------------- basis

template <class R>
struct AxisSup {
    int l;          // local span inside the tile, or < 0 if the particle is not in it
    int c;          // unwrapped span
    R w[3], dw[3];  // weights and d/dxi of the p+1 support nodes
};

// Span of coordinate x along axis a evaluated in the storage precision R with
// one rounding per operation: xi = (x - lo) * (1/h); c = floor(xi [+ 1/2]).
// WALLS: the caller knows that no axis is periodic.
template <class R, int P, bool WALLS = false>
__device__ __forceinline__ int span_of(const Geom& G, int a, R x, R& xi)
{
    typedef Op<R> O;
    xi = O::mul(O::sub(x, (R)G.lo[a]), (R)G.inv_h);
    R s = (P == 2) ? O::add(xi, (R)0.5) : xi;
    int c = (int)O::flr(s);
    if (WALLS || !G.per[a]) c = min(max(c, 0), G.S[a] - 1);
    return c;
}

template <bool WALLS = false>
__device__ __forceinline__ int wrap_span(const Geom& G, int a, int c)
{
    if (WALLS || !G.per[a]) return c;
    const int n = G.n[a];
    // spans of positions in [lo, hi] and one span beyond wrap by one period
    int r = c >= n ? c - n : (c < 0 ? c + n : c);
    if ((unsigned)r >= (unsigned)n) {
        r = c % n;
        if (r < 0) r += n;
    }
    return r;
}

template <class R, int P>
__device__ __forceinline__ void axis_support(const Geom& G, int a, R x, int tile_span0, AxisSup<R>& s)
{
    typedef Op<R> O;
    R xi;
    int c = span_of<R, P>(G, a, x, xi);
    s.c = c;
    int b = c - (P == 2 ? 1 : 0);
    R fx = O::sub(xi, (R)b);
    if (P == 2) {
        R t0 = O::sub((R)1.5, fx), t1 = O::sub(fx, (R)1.0), t2 = O::sub(fx, (R)0.5);
        s.w[0] = O::mul(O::mul(t0, t0), (R)0.5);
        s.w[1] = O::sub((R)0.75, O::mul(t1, t1));
        s.w[2] = O::mul(O::mul(t2, t2), (R)0.5);
        s.dw[0] = -t0;
        s.dw[1] = O::mul((R)-2.0, t1);
        s.dw[2] = t2;
    } else {
        s.w[0] = O::sub((R)1.0, fx);
        s.w[1] = fx;
        s.w[2] = (R)0;
        s.dw[0] = (R)-1.0;
        s.dw[1] = (R)1.0;
        s.dw[2] = (R)0;
    }
    int l = wrap_span(G, a, c) - tile_span0;
    s.l = (l >= 0 && l < G.T[a]) ? l : -1;
}

// Largest |w| and |dw| over the support nodes of one axis.
template <int NS, class R>
__device__ __forceinline__ void axis_bounds(const AxisSup<R>& s, R& wm, R& dm)
{
    wm = fabs(s.w[0]);
    dm = fabs(s.dw[0]);
#pragma unroll
    for (int k = 1; k < NS; ++k) {
        wm = fmax(wm, fabs(s.w[k]));
        dm = fmax(dm, fabs(s.dw[k]));
    }
}

// Fixed point: a particle may round its contributions with the 32-bit
// conversion when each bound (|factor| x S x largest weight) is below 2^30,
// a factor 2 under 2^31 for the roundings of the contribution and of the
// bound itself.  NaN and infinity fail the comparison.
constexpr float kSmallQuanta = 1073741824.f;

__device__ __forceinline__ void tile_origin(const Geom& G, int tile, int so[3])
{
    int tx = tile % G.nt[0];
    int ty = (tile / G.nt[0]) % G.nt[1];
    int tz = tile / (G.nt[0] * G.nt[1]);
    so[0] = tx * G.T[0];
    so[1] = ty * G.T[1];
    so[2] = tz * G.T[2];
}

// w / d for 0 <= w < 2^21 from the float reciprocal of d: (w + 1/2) / d lies
// at least 1/(2d) from an integer, and the two float roundings move it by
// less than 2^-22 (w + 1/2) / d, which is smaller.
__device__ __forceinline__ int div_small(int w, float inv_d) { return (int)(((float)w + 0.5f) * inv_d); }

// Storage index of window slot w of the tile whose first span is so[], or -1.
// TX, TY > 0: the tile edges as compile-time constants (slot decoded by
// integer division by constants).
template <int P, int TX = 0, int TY = 0>
__device__ __forceinline__ int64_t slot_node(const Geom& G, const int so[3], int w, int idx[3])
{
    int ws[3];
    if constexpr (TX > 0) {
        constexpr unsigned W0 = TX + P, W1 = TY + P;
        const unsigned q = (unsigned)w / W0, q2 = q / W1;
        ws[0] = (int)((unsigned)w - q * W0);
        ws[2] = (int)q2;
        ws[1] = (int)(q - q2 * W1);
    } else {
        const int q = div_small(w, G.inv_w[0]);
        ws[0] = w - q * G.W[0];
        ws[2] = div_small(q, G.inv_w[1]);
        ws[1] = q - ws[2] * G.W[1];
    }
    for (int a = 0; a < 3; ++a) {
        if (a >= G.dim) { idx[a] = 0; continue; }
        int i = so[a] + ws[a];
        if (G.per[a]) {
            i -= (P == 2 ? 1 : 0);
            i %= G.n[a];
            if (i < 0) i += G.n[a];
        } else if (i >= G.N[a]) {
            return -1;
        }
        idx[a] = i;
    }
    return ((int64_t)idx[2] * G.N[1] + idx[1]) * G.pitch + idx[0];
}

// Grid boundary conditions of one node (Sec. 3 steps iii and vii): obstacle
// projection (eqs. normali1/normali2) on a masked node, then the domain
// faces -- slip wall: normal component 0; inflow: m v_in (momentum) or 0
// (force).  kind 0 = momentum, 1 = force.
template <class R, int D>
__device__ __forceinline__ void node_bc(const Geom& G, const uint8_t* mask, const R* const* nrm, int64_t node,
                                        const int idx[3], R m, R* vec, int kind)
{
    typedef Op<R> O;
    if (mask && mask[node]) {
        R n[3], xn = (R)0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            n[a] = nrm[a][node];
            xn = O::add(xn, O::mul(vec[a], n[a]));
        }
        R c = O::mul((R)0.5, O::sub(xn, fabs(xn)));
#pragma unroll
        for (int a = 0; a < D; ++a) vec[a] = O::sub(vec[a], O::mul(c, n[a]));
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (G.per[a]) continue;
        int phys = idx[a] - G.g[a];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            bool on = side == 0 ? (phys <= 0) : (phys >= G.n[a]);
            if (!on) continue;
            int bc = G.bc[2 * a + side];
            if (bc == 0) {
                vec[a] = (R)0;
            } else if (bc == 2) {
#pragma unroll
                for (int b = 0; b < D; ++b) vec[b] = kind == 0 ? O::mul(m, (R)G.inflow_v[b]) : (R)0;
            }
        }
    }
}

// Whether any node of the window of the tile at so[] needs node_bc: an
// obstacle mask exists, or the window reaches a node on or beyond a
// non-periodic face.
__device__ __forceinline__ bool window_has_bc(const Geom& G, const uint8_t* mask, const int so[3])
{
    if (mask) return true;
    for (int a = 0; a < G.dim; ++a) {
        if (G.per[a]) continue;
        if (so[a] <= G.g[a] || so[a] + G.W[a] - 1 >= G.n[a] + G.g[a]) return true;
    }
    return false;
}

template <class R>
__device__ __forceinline__ uint32_t key_of(const Geom& G, const int sp[3])
{
    const int t = ((sp[2] >> G.tsh[2]) * G.nt[1] + (sp[1] >> G.tsh[1])) * G.nt[0] + (sp[0] >> G.tsh[0]);
    const int l = (((sp[2] & (G.T[2] - 1)) << G.tsh[1]) + (sp[1] & (G.T[1] - 1))) << G.tsh[0] | (sp[0] & (G.T[0] - 1));
    return (uint32_t)t * (uint32_t)G.Tvol + (uint32_t)l;
}

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    // Salmon et al. (SC'11): ten rounds, multipliers 0xD2511F53/0xCD9E8D57,
    // Weyl key increments 0x9E3779B9/0xBB67AE85.
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

// Non-negative doubles order like their bit patterns as unsigned integers.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v)
{
    if (v > 0.0) atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

template <class R>
__device__ __forceinline__ R warp_max(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ------------------------------------------------------------------ P2G

// Weights of support node (kx, ky, kz) in the documented binary32 order.
template <class R, int D>
__device__ __forceinline__ void node_weights(const AxisSup<R>* s, int kx, int ky, int kz, R& w, R g[3])
{
    typedef Op<R> O;
    if (D == 3) {
        R yz = O::mul(s[1].w[ky], s[2].w[kz]);
        R dyz = O::mul(s[1].dw[ky], s[2].w[kz]);
        R ydz = O::mul(s[1].w[ky], s[2].dw[kz]);
        w = O::mul(s[0].w[kx], yz);
        g[0] = O::mul(s[0].dw[kx], yz);
        g[1] = O::mul(s[0].w[kx], dyz);
        g[2] = O::mul(s[0].w[kx], ydz);
    } else {
        w = O::mul(s[0].w[kx], s[1].w[ky]);
        g[0] = O::mul(s[0].dw[kx], s[1].w[ky]);
        g[1] = O::mul(s[0].w[kx], s[1].dw[ky]);
        g[2] = (R)0;
    }
}

template <int D, int P, class R, class A>
__device__ __forceinline__ void p2g_tile(const Geom& G, const Particles<R>& pt, const Grid<A, R>& gr,
                                         const uint32_t* cellstart, Clock* clk, const int tile)
{
    typedef Op<R> O;
    if (!clk->active) return;
    const uint32_t beg = cellstart[tile_cs0(G, tile)];
    const uint32_t end = cellstart[tile_cs0(G, tile) + G.Tvol];
    if (beg == end) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A* s = reinterpret_cast<A*>(smem_raw);
    const int W = G.Wvol;
    const int NF = 1 + 2 * D;
    for (int i = threadIdx.x; i < NF * W; i += blockDim.x) s[i] = A(0);
    __syncthreads();
    int so[3];
    tile_origin(G, tile, so);
    const R gm1 = (R)(G.gamma - 1.0), ih = (R)G.inv_h;
    constexpr int NS = P + 1;
    for (uint32_t k = beg + threadIdx.x; k < end; k += blockDim.x) {
        AxisSup<R> sx[3];
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            axis_support<R, P>(G, a, pt.x[a][k], so[a], sx[a]);
            ok = ok && sx[a].l >= 0;
        }
        if (!ok) { atomicOr(&clk->err, ERR_TILE); continue; }
        if (D == 2) { sx[2].l = 0; sx[2].w[0] = (R)1; sx[2].dw[0] = (R)0; }
        const R M = pt.M[k], rho = pt.rho[k];
        const R Pk = O::mul(O::mul(gm1, rho), pt.E[k]);
        const R vol = O::dvd(M, rho);
        const R F = O::mul(O::mul(O::add(Pk, pt.Q[k]), vol), ih);
        R MV[3];
#pragma unroll
        for (int a = 0; a < D; ++a) MV[a] = O::mul(M, pt.v[a][k]);
        auto scatter = [&](auto small) {
            constexpr bool SM = decltype(small)::value;
#pragma unroll
            for (int kz = 0; kz < (D == 3 ? NS : 1); ++kz)
#pragma unroll
                for (int ky = 0; ky < NS; ++ky)
#pragma unroll
                    for (int kx = 0; kx < NS; ++kx) {
                        R w, g[3];
                        node_weights<R, D>(sx, kx, ky, kz, w, g);
                        const int slot = ((sx[2].l + kz) * G.W[1] + sx[1].l + ky) * G.W[0] + sx[0].l + kx;
                        Acc<A>::add(&s[slot], Acc<A>::template from_t<SM>(O::mul(M, w), G.qscale[0]));
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            Acc<A>::add(&s[(1 + a) * W + slot],
                                        Acc<A>::template from_t<SM>(O::mul(MV[a], w), G.qscale[1]));
                            Acc<A>::add(&s[(1 + D + a) * W + slot],
                                        Acc<A>::template from_t<SM>(O::mul(F, g[a]), G.qscale[2]));
                        }
                    }
        };
        if constexpr (Acc<A>::kFixed) {
            R wm[3], dm[3];
#pragma unroll
            for (int a = 0; a < D; ++a) axis_bounds<NS>(sx[a], wm[a], dm[a]);
            R wb = wm[0], gb = (R)0, mvb = (R)0;
#pragma unroll
            for (int a = 1; a < D; ++a) wb *= wm[a];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                R ga = dm[a];
#pragma unroll
                for (int b = 0; b < D; ++b)
                    if (b != a) ga *= wm[b];
                gb = fmax(gb, ga);
                mvb = fmax(mvb, fabs(MV[a]));
            }
            const bool small = (M * G.qscale[0] * wb < kSmallQuanta) & (mvb * G.qscale[1] * wb < kSmallQuanta) &
                               (fabs(F) * G.qscale[2] * gb < kSmallQuanta);
            if (small) scatter(std::true_type{});
            else scatter(std::false_type{});
        } else {
            scatter(std::false_type{});
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        int idx[3];
        int64_t node = slot_node<P>(G, so, i, idx);
        if (node < 0) continue;
        A v = s[i];
        if (v != A(0)) Acc<A>::add(&gr.m[node], v);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            v = s[(1 + a) * W + i];
            if (v != A(0)) Acc<A>::add(&gr.mv[a][node], v);
            v = s[(1 + D + a) * W + i];
            if (v != A(0)) Acc<A>::add(&gr.f[a][node], v);
        }
    }
}

template <int D, int P, class R, class A>
__global__ void __launch_bounds__(256) k_p2g(Geom G, TileState<R> ts, Grid<A, R> gr, Clock* clk)
{
    const int t = blockIdx.x;
    p2g_tile<D, P, R, A>(G, ts.pt, gr, ts.tpar[t] ? ts.cs[1] : ts.cs[0], clk, t);
}

// ----------------------------------------------- grid update + G2P + P2G

// G2P window of a tile: the acceleration a = f/m after the force boundary
// conditions (D x W values), and the momentum accumulators set to zero.
template <int D, int P, class R, class A>
__device__ __forceinline__ void accel_window(const Geom& G, const Grid<A, R>& gr, const int so[3], R* sA, A* s2)
{
    typedef Op<R> O;
    const int W = G.Wvol;
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        int idx[3];
        int64_t node = slot_node<P>(G, so, i, idx);
        R f[3] = {(R)0, (R)0, (R)0};
        R m = (R)0;
        if (node >= 0) {
            m = Acc<A>::to_real(gr.m[node], G.dqscale[0]);
#pragma unroll
            for (int a = 0; a < D; ++a) f[a] = Acc<A>::to_real(gr.f[a][node], G.dqscale[2]);
            node_bc<R, D>(G, gr.mask, gr.nrm, node, idx, m, f, 1);
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            sA[a * W + i] = (m != (R)0) ? O::dvd(f[a], m) : (R)0;
            s2[a * W + i] = A(0);
        }
    }
}

template <int D, int P, class R, class A>
__device__ __forceinline__ void grid_g2p_tile(const Geom& G, const Particles<R>& pt, const Grid<A, R>& gr,
                                              const uint32_t* cellstart, Clock* clk, const int tile)
{
    typedef Op<R> O;
    if (!clk->active) return;
    const uint32_t beg = cellstart[tile_cs0(G, tile)];
    const uint32_t end = cellstart[tile_cs0(G, tile) + G.Tvol];
    if (beg == end) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int W = G.Wvol;
    R* sA = reinterpret_cast<R*>(smem_raw);                       // D x W: f/m after BC
    // D x W momentum P2G accumulators, 16-byte aligned (8-byte atomics)
    A* s2 = reinterpret_cast<A*>(smem_raw + ((sizeof(R) * D * W + 15) & ~size_t(15)));
    int so[3];
    tile_origin(G, tile, so);
    const R dt = (R)clk->dt_cur;
    accel_window<D, P, R, A>(G, gr, so, sA, s2);
    __syncthreads();
    constexpr int NS = P + 1;
    R vmax = (R)0;
    for (uint32_t k = beg + threadIdx.x; k < end; k += blockDim.x) {
        AxisSup<R> sx[3];
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            axis_support<R, P>(G, a, pt.x[a][k], so[a], sx[a]);
            ok = ok && sx[a].l >= 0;
        }
        if (!ok) { atomicOr(&clk->err, ERR_TILE); continue; }
        if (D == 2) { sx[2].l = 0; sx[2].w[0] = (R)1; sx[2].dw[0] = (R)0; }
        R acc[3] = {(R)0, (R)0, (R)0};
#pragma unroll
        for (int kz = 0; kz < (D == 3 ? NS : 1); ++kz)
#pragma unroll
            for (int ky = 0; ky < NS; ++ky)
#pragma unroll
                for (int kx = 0; kx < NS; ++kx) {
                    R w, g[3];
                    node_weights<R, D>(sx, kx, ky, kz, w, g);
                    const int slot = ((sx[2].l + kz) * G.W[1] + sx[1].l + ky) * G.W[0] + sx[0].l + kx;
#pragma unroll
                    for (int a = 0; a < D; ++a) acc[a] = O::add(acc[a], O::mul(w, sA[a * W + slot]));
                }
        const R M = pt.M[k];
        R MV[3], v2 = (R)0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            R vn = O::add(pt.v[a][k], O::mul(dt, acc[a]));
            pt.v[a][k] = vn;
            MV[a] = O::mul(M, vn);
            v2 = O::add(v2, O::mul(vn, vn));
        }
        vmax = fmax(vmax, O::sqr(v2));
        auto scatter = [&](auto small) {
            constexpr bool SM = decltype(small)::value;
#pragma unroll
            for (int kz = 0; kz < (D == 3 ? NS : 1); ++kz)
#pragma unroll
                for (int ky = 0; ky < NS; ++ky)
#pragma unroll
                    for (int kx = 0; kx < NS; ++kx) {
                        R w, g[3];
                        node_weights<R, D>(sx, kx, ky, kz, w, g);
                        const int slot = ((sx[2].l + kz) * G.W[1] + sx[1].l + ky) * G.W[0] + sx[0].l + kx;
#pragma unroll
                        for (int a = 0; a < D; ++a)
                            Acc<A>::add(&s2[a * W + slot], Acc<A>::template from_t<SM>(O::mul(MV[a], w), G.qscale[1]));
                    }
        };
        if constexpr (Acc<A>::kFixed) {
            R wb = (R)1, mvb = (R)0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                R wm, dm;
                axis_bounds<NS>(sx[a], wm, dm);
                wb *= wm;
                mvb = fmax(mvb, fabs(MV[a]));
            }
            if (mvb * G.qscale[1] * wb < kSmallQuanta) scatter(std::true_type{});
            else scatter(std::false_type{});
        } else {
            scatter(std::false_type{});
        }
    }
    // block max of |V'| for the CFL rule
    vmax = warp_max(vmax);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&clk->vmax_bits, (double)vmax);
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        int idx[3];
        int64_t node = slot_node<P>(G, so, i, idx);
        if (node < 0) continue;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            A v = s2[a * W + i];
            if (v != A(0)) Acc<A>::add(&gr.mv2[a][node], v);
        }
    }
}

template <int D, int P, class R, class A>
__global__ void __launch_bounds__(256) k_grid_g2p(Geom G, TileState<R> ts, Grid<A, R> gr, Clock* clk)
{
    const int t = blockIdx.x;
    grid_g2p_tile<D, P, R, A>(G, ts.pt, gr, ts.tpar[t] ? ts.cs[1] : ts.cs[0], clk, t);
}

// ------------------------------------ G2PD + particle update + move + key

template <int D, int P, class R, class A>
__device__ __forceinline__ void g2pd_tile(const Geom& G, const Particles<R>& pt, const Grid<A, R>& gr,
                                          const uint32_t* cellstart, Clock* clk, const Reorder& ro, const int tile)
{
    typedef Op<R> O;
    if (!clk->active) return;
    const uint32_t beg = cellstart[tile_cs0(G, tile)];
    const uint32_t end = cellstart[tile_cs0(G, tile) + G.Tvol];
    if (beg == end) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int W = G.Wvol;
    R* sVb = reinterpret_cast<R*>(smem_raw);   // D x W: mv'/m
    R* sV2 = sVb + D * W;                       // D x W: mv2/m after BC
    int so[3];
    tile_origin(G, tile, so);
    const R dt = (R)clk->dt_cur;
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        int idx[3];
        int64_t node = slot_node<P>(G, so, i, idx);
        R mv[3] = {(R)0, (R)0, (R)0}, f[3] = {(R)0, (R)0, (R)0}, m2[3] = {(R)0, (R)0, (R)0};
        R m = (R)0;
        if (node >= 0) {
            m = Acc<A>::to_real(gr.m[node], G.dqscale[0]);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                mv[a] = Acc<A>::to_real(gr.mv[a][node], G.dqscale[1]);
                f[a] = Acc<A>::to_real(gr.f[a][node], G.dqscale[2]);
                m2[a] = Acc<A>::to_real(gr.mv2[a][node], G.dqscale[1]);
            }
            node_bc<R, D>(G, gr.mask, gr.nrm, node, idx, m, mv, 0);
            node_bc<R, D>(G, gr.mask, gr.nrm, node, idx, m, f, 1);
            node_bc<R, D>(G, gr.mask, gr.nrm, node, idx, m, m2, 0);
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            R mvp = O::add(mv[a], O::mul(dt, f[a]));
            sVb[a * W + i] = (m != (R)0) ? O::dvd(mvp, m) : (R)0;
            sV2[a * W + i] = (m != (R)0) ? O::dvd(m2[a], m) : (R)0;
        }
    }
    __syncthreads();
    constexpr int NS = P + 1;
    const R gm1 = (R)(G.gamma - 1.0), gam = (R)G.gamma, ih = (R)G.inv_h, hh = (R)G.h;
    const R c0 = (R)G.c0, c1 = (R)G.c1;
    R vmax = (R)0, cmax = (R)0;
    int err = 0;
    for (uint32_t k = beg + threadIdx.x; k < end; k += blockDim.x) {
        AxisSup<R> sx[3];
        bool ok = true;
        R x[3];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            x[a] = pt.x[a][k];
            axis_support<R, P>(G, a, x[a], so[a], sx[a]);
            ok = ok && sx[a].l >= 0;
        }
        if (!ok) { err |= ERR_TILE; continue; }
        if (D == 2) { sx[2].l = 0; sx[2].w[0] = (R)1; sx[2].dw[0] = (R)0; }
        R vb[3] = {(R)0, (R)0, (R)0}, dv = (R)0;
#pragma unroll
        for (int kz = 0; kz < (D == 3 ? NS : 1); ++kz)
#pragma unroll
            for (int ky = 0; ky < NS; ++ky)
#pragma unroll
                for (int kx = 0; kx < NS; ++kx) {
                    R w, g[3];
                    node_weights<R, D>(sx, kx, ky, kz, w, g);
                    const int slot = ((sx[2].l + kz) * G.W[1] + sx[1].l + ky) * G.W[0] + sx[0].l + kx;
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        vb[a] = O::add(vb[a], O::mul(w, sVb[a * W + slot]));
                        dv = O::add(dv, O::mul(g[a], sV2[a * W + slot]));
                    }
                }
        dv = O::mul(dv, ih);   // node weights are per unit xi
        // step viii: energy, density, pressure, artificial viscosity
        const R rho = pt.rho[k], E = pt.E[k], Q = pt.Q[k];
        const R Pk = O::mul(O::mul(gm1, rho), E);
        const R En = O::add(E, O::mul(O::mul(dt, -O::dvd(O::add(Pk, Q), rho)), dv));
        const R den = O::add((R)1, O::mul(dt, dv));
        if (!(den > (R)0)) { err |= ERR_NONFINITE; continue; }
        const R rn = O::dvd(rho, den);
        const R Pn = O::mul(O::mul(gm1, rn), En);
        R c2 = O::dvd(O::mul(gam, Pn), rn);
        const R cs = O::sqr(c2 > (R)0 ? c2 : (R)0);
        R Qn = (R)0;
        if (dv < (R)0) {
            // eq. muart: von Neumann-Richtmyer and Landshoff terms, both
            // proportional to the density
            const R t1 = O::mul(hh, dv);
            Qn = O::mul(rn, O::sub(O::mul(O::mul(c0, t1), t1), O::mul(O::mul(O::mul(c1, hh), cs), dv)));
        }
        // step ix: move with Vbar; step x: connectivity (wrap, hold, recycle)
        R xn[3];
        R vb2 = (R)0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            xn[a] = O::add(x[a], O::mul(dt, vb[a]));
            vb2 = O::add(vb2, O::mul(vb[a], vb[a]));
        }
        bool out = false;
        bool fin = isfinite(En) && isfinite(rn) && isfinite(Qn);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            fin = fin && isfinite(xn[a]);
            R xi;
            int c_new = span_of<R, P>(G, a, xn[a], xi);
            int d = c_new - sx[a].c;
            if (d < -1 || d > 1) err |= ERR_CFL;
            if (!G.per[a]) {
                if (xn[a] < (R)G.lo[a] && G.bc[2 * a] == 3) out = true;
                if (xn[a] >= (R)G.hi[a] && G.bc[2 * a + 1] == 3) out = true;
            }
        }
        if (!fin) { err |= ERR_NONFINITE; continue; }
        R En_s = En, rn_s = rn, Qn_s = Qn;
        R cpart = cs;
        if (out && G.inflow_face >= 0) {
            const uint32_t gk = pt.gen[k];
            uint32_t c[4] = {gk, 0u, pt.id[k], 0u};
            philox4x32_10(c, (uint32_t)G.seed, (uint32_t)(G.seed >> 32));
            pt.gen[k] = gk + 1u;
            const int af = G.inflow_face / 2, side = G.inflow_face % 2;
            R vin2 = (R)0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                R u = O::mul((R)(c[a] >> 8), (R)(1.0 / 16777216.0));
                if (a == af)
                    xn[a] = side == 0 ? O::add((R)G.lo[a], O::mul(u, hh))
                                      : O::add(O::sub((R)G.hi[a], hh), O::mul(u, hh));
                else
                    xn[a] = O::add((R)G.lo[a], O::mul(u, O::sub((R)G.hi[a], (R)G.lo[a])));
                pt.v[a][k] = (R)G.inflow_v[a];
                vin2 = O::add(vin2, O::mul((R)G.inflow_v[a], (R)G.inflow_v[a]));
            }
            En_s = (R)G.inflow_e;
            rn_s = (R)G.inflow_rho;
            Qn_s = (R)0;
            R ci2 = O::dvd(O::mul(gam, O::mul(O::mul(gm1, rn_s), En_s)), rn_s);
            cpart = O::sqr(ci2 > (R)0 ? ci2 : (R)0);
            vmax = fmax(vmax, O::sqr(vin2));
        } else {
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const R lo = (R)G.lo[a], hi = (R)G.hi[a];
                if (G.per[a]) {
                    const R L = O::sub(hi, lo);
                    if (xn[a] < lo) xn[a] = O::add(xn[a], L);
                    else if (xn[a] >= hi) xn[a] = O::sub(xn[a], L);
                } else {
                    if (xn[a] < lo) xn[a] = lo;
                    if (xn[a] > hi) xn[a] = hi;
                }
            }
        }
        int sp[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            R xi;
            sp[a] = wrap_span(G, a, span_of<R, P>(G, a, xn[a], xi));
            pt.x[a][k] = xn[a];
        }
        int old[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) old[a] = wrap_span(G, a, sx[a].c);
        pt.key[k] = record_key(G, ro, clk, key_of<R>(G, sp), out && G.inflow_face >= 0, (uint32_t)k, tile,
                               key_of<R>(G, old), err);
        pt.E[k] = En_s;
        pt.rho[k] = rn_s;
        pt.Q[k] = Qn_s;
        vmax = fmax(vmax, O::sqr(vb2));
        cmax = fmax(cmax, cpart);
    }
    vmax = warp_max(vmax);
    cmax = warp_max(cmax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) err |= __shfl_xor_sync(0xffffffffu, err, o);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&clk->vmax_bits, (double)vmax);
        atomic_max_nonneg(&clk->cmax_bits, (double)cmax);
        if (err) atomicOr(&clk->err, err);
    }
}

template <int D, int P, class R, class A>
__global__ void __launch_bounds__(256) k_g2pd(Geom G, TileState<R> ts, Grid<A, R> gr, Clock* clk, Reorder ro)
{
    const int t = blockIdx.x;
    g2pd_tile<D, P, R, A>(G, ts.pt, gr, ts.tpar[t] ? ts.cs[1] : ts.cs[0], clk, ro, t);
}

// ---------------------------------------------------------- time control

// Decide this step's dt (fixed or CFL) and clip it to t_end (step xiii).
__device__ __forceinline__ void prepare_clock(Clock& c)
{
    c.nfar = 0u;
    c.overflow = 0u;
    if (c.done || c.err || (c.step_end > 0 && c.step >= c.step_end)) { c.active = 0; return; }
    double h = c.dt_fixed > 0.0 ? c.dt_fixed : c.dt_next;
    if (!(h > 0.0)) { c.err |= ERR_NONFINITE; c.active = 0; return; }
    c.last = 0;
    if (c.t_end > 0.0 && c.t + h >= c.t_end) { h = c.t_end - c.t; c.last = 1; }
    c.dt_cur = h;
    c.active = 1;
    c.vmax_bits = 0ull;
    c.cmax_bits = 0ull;
}

__global__ void k_prepare(Clock* clk) { prepare_clock(*clk); }

__device__ __forceinline__ void finalize_clock(Clock& c, double cfl_h)
{
    if (!c.active) return;
    c.t = c.last ? c.t_end : c.t + c.dt_cur;
    c.step += 1;
    const double v = __longlong_as_double((long long)c.vmax_bits);
    const double cs = __longlong_as_double((long long)c.cmax_bits);
    c.dt_next = (v + cs) > 0.0 ? cfl_h / (v + cs) : 0.0;
    if (c.last || (c.t_end > 0.0 && c.t >= c.t_end)) c.done = 1;
}

__global__ void k_finalize(Clock* clk, double cfl_h) { finalize_clock(*clk, cfl_h); }

// Step budget (from the current step) and buffer parity of a batch member.
__global__ void k_set_batch(Clock* clk, long long nsteps, int par)
{
    clk->step_end = nsteps > 0 ? clk->step + nsteps : 0;
    clk->par = par;
}

__global__ void k_set_params(Clock* clk, double dt_fixed, double t_end)
{
    Clock& c = *clk;
    c.dt_fixed = dt_fixed;
    if (t_end != c.t_end) {
        c.t_end = t_end;
        c.done = (t_end > 0.0 && c.t >= t_end) ? 1 : 0;
    }
}

// Particles of each tile (from its cell starts).
template <class R>
__global__ void k_tile_counts(Geom G, TileState<R> ts, uint32_t* counts)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < G.ntiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t* cs = ts.cs[ts.tpar[t]];
        counts[t] = cs[tile_cs0(G, t) + G.Tvol] - cs[tile_cs0(G, t)];
    }
}

// Slot of the particle at position j of the key order; toff[t] is the number
// of particles in the tiles before t (ntiles + 1 entries).
template <class R>
__device__ __forceinline__ uint32_t order_slot(const Geom& G, const TileState<R>& ts, const uint32_t* toff, int64_t j)
{
    int lo = 0, hi = G.ntiles - 1;      // the last tile whose first position is <= j
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)toff[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return ts.cs[ts.tpar[lo]][tile_cs0(G, lo)] + (uint32_t)(j - (int64_t)toff[lo]);
}

// out[j] = the field a (both buffers) of the particle at position j of the
// key order.
template <class T, class R>
__global__ void k_compact(Geom G, TileState<R> ts, const uint32_t* toff, const T* a, T* out, int64_t n)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = a[order_slot(G, ts, toff, j)];
}

// Initial CFL maxima over the particle state (Vbar := V before the first step).
template <int D, class R>
__global__ void k_cfl_init(Geom G, TileState<R> ts, const uint32_t* toff, int64_t n, Clock* clk)
{
    typedef Op<R> O;
    R vmax = (R)0, cmax = (R)0;
    const R gm1 = (R)(G.gamma - 1.0), gam = (R)G.gamma;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = order_slot(G, ts, toff, j);
        const Particles<R>& pt = ts.pt;
        R v2 = (R)0;
#pragma unroll
        for (int a = 0; a < D; ++a) v2 = O::add(v2, O::mul(pt.v[a][k], pt.v[a][k]));
        vmax = fmax(vmax, O::sqr(v2));
        R P = O::mul(O::mul(gm1, pt.rho[k]), pt.E[k]);
        R c2 = O::dvd(O::mul(gam, P), pt.rho[k]);
        cmax = fmax(cmax, O::sqr(c2 > (R)0 ? c2 : (R)0));
    }
    vmax = warp_max(vmax);
    cmax = warp_max(cmax);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&clk->vmax_bits, (double)vmax);
        atomic_max_nonneg(&clk->cmax_bits, (double)cmax);
    }
}

__global__ void k_cfl_init_finish(Clock* clk, double cfl_h)
{
    Clock& c = *clk;
    const double v = __longlong_as_double((long long)c.vmax_bits);
    const double cs = __longlong_as_double((long long)c.cmax_bits);
    c.dt_next = (v + cs) > 0.0 ? cfl_h / (v + cs) : 0.0;
    c.vmax_bits = 0ull;
    c.cmax_bits = 0ull;
}

// ----------------------------------------------------- keys and gathering

template <int D, int P, class R>
__global__ void k_keys(Geom G, Particles<R> pt, int64_t n)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int sp[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        R xi;
        sp[a] = wrap_span(G, a, span_of<R, P>(G, a, pt.x[a][k], xi));
    }
    pt.key[k] = key_of<R>(G, sp);
}

// out[j] = in[perm[j]] for every particle array; identity when inactive.
template <int D, class R>
__global__ void k_gather(Particles<R> in, Particles<R> out, const uint32_t* perm, const uint32_t* sorted_keys,
                         int64_t n, const int* active)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const bool act = active == nullptr || *active;
    uint32_t s = act ? perm[j] : (uint32_t)j;
    // a step that failed (reported through the clock's error bits) may leave
    // parts of perm unwritten: never follow an index out of the buffer
    if ((int64_t)s >= n) s = (uint32_t)j;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        out.x[a][j] = in.x[a][s];
        out.v[a][j] = in.v[a][s];
    }
    out.M[j] = in.M[s];
    out.rho[j] = in.rho[s];
    out.E[j] = in.E[s];
    out.Q[j] = in.Q[s];
    out.id[j] = in.id[s];
    out.gen[j] = in.gen[s];
    (void)sorted_keys;   // the sorted keys stay in the re-order's own buffer
}

// FP64 sums for the conservation diagnostics: one partial per block, summed
// by k_cons_final in a fixed order (deterministic).
template <int D, class R>
__global__ void __launch_bounds__(256) k_cons_partial(Geom G, TileState<R> ts, const uint32_t* toff, int64_t n,
                                                      double* partial)
{
    __shared__ double sh[5][256];
    double s[5] = {0, 0, 0, 0, 0};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = order_slot(G, ts, toff, j);
        const Particles<R>& pt = ts.pt;
        double M = (double)pt.M[k], v2 = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            double va = (double)pt.v[a][k];
            v2 += va * va;
            s[2 + a] += M * va;
        }
        s[0] += M;
        s[1] += M * ((double)pt.E[k] + 0.5 * v2);
    }
    for (int i = 0; i < 5; ++i) sh[i][threadIdx.x] = s[i];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int i = 0; i < 5; ++i) sh[i][threadIdx.x] += sh[i][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int i = 0; i < 5; ++i) partial[blockIdx.x * 5 + i] = sh[i][0];
}

// One block of kConsThreads: thread t adds partials t, t + kConsThreads, ...,
// then a fixed tree over the threads (a serial chain of dependent FP64 adds
// over all partials took longer than the partials themselves).
constexpr int kConsThreads = 256;

__global__ void __launch_bounds__(kConsThreads) k_cons_final(const double* partial, int nb, double* out)
{
    __shared__ double sh[5][kConsThreads];
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += kConsThreads)
        for (int i = 0; i < 5; ++i) s[i] += partial[b * 5 + i];
    for (int i = 0; i < 5; ++i) sh[i][threadIdx.x] = s[i];
    __syncthreads();
    for (int o = kConsThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int i = 0; i < 5; ++i) sh[i][threadIdx.x] += sh[i][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int i = 0; i < 5; ++i) out[i] = sh[i][0];
}

// Convert host-side doubles (or floats) to the storage precision.
template <class R>
__global__ void k_from_double(const double* in, R* out, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (R)in[i];
}

template <class R>
__global__ void k_from_float(const float* in, R* out, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (R)in[i];
}

template <class R>
__global__ void k_to_double(const R* in, double* out, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

// Pressure of the ideal-gas law (eq. pressures), P = (gamma - 1) rho e, in the
// storage precision with the operation order of the step kernels.
template <class R>
__global__ void k_pressure(const R* rho, const R* E, R gm1, R* out, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = Op<R>::mul(Op<R>::mul(gm1, rho[i]), E[i]);
}

// Checks of uploaded particle values (binary64 or binary32, compared in
// binary64, exactly); sets `bit` in *bad when one fails.
// mode 0: finite; 1: finite and > 0; 2: lo <= v <= hi; 3: lo <= v < hi.
template <class T>
__global__ void k_check_values(const T* in, int64_t n, int mode, double lo, double hi, unsigned bit, unsigned* bad)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = (double)in[i];
    bool ok;
    switch (mode) {
    case 0: ok = isfinite(v); break;
    case 1: ok = isfinite(v) && v > 0.0; break;
    case 2: ok = v >= lo && v <= hi; break;
    default: ok = v >= lo && v < hi; break;
    }
    if (!ok) atomicOr(bad, bit);
}

__global__ void k_iota(uint32_t* out, int64_t n, uint32_t base)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = base + (uint32_t)i;
}

}  // namespace mpm

