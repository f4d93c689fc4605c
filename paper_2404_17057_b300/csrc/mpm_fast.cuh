// mpm_fast.cuh -- single-precision kernels of the step, organised for sm_103a.
//
// P2G-type work (steps ii and vi of Algorithm 1) is a scatter: every particle
// adds (p+1)^d values per field to the grid.  All particles of one basis span
// share their support nodes, and the particles are stored span by span, so
// here one thread owns one span: it sums its particles' contributions in
// registers (tensor products of 1D weights, two fields per packed f32x2 FMA)
// and adds each node of the span once into the tile's shared-memory window.
// A warp owns 32 consecutive spans (one or more x-rows of the tile); the
// x-neighbours of a row are summed by shuffles first, so the adds never
// collide.  The window then goes to global memory once, as 16-byte vector
// reductions along the (padded, 16-byte aligned) node rows.
//
// G2P-type work (the gathers of steps iv-viii) keeps one thread per particle:
// lanes of one span read the same node records (a broadcast), and the sums
// are factored along the axes (x first, then y, then z).  K2 stages its row
// chunks of particles in shared memory with bulk copies and runs both kinds
// of work on them: the gather per particle, then the momentum scatter per
// span.
//
// The file also holds the 2D span-per-lane P2G and grid + G2P + P2G kernels
// of the fixed-point and FP64 modes (64-bit register sums), and the G2PD
// kernel that the fixed-point mode shares with FP32.
#pragma once
#include "mpm_kernels.cuh"
#include "mpm_tma.cuh"

namespace mpm {


template <int P>
__device__ __forceinline__ void weights1d(float fx, float* w, float* dw)
{
    if (P == 2) {
        const float t0 = 1.5f - fx, t1 = fx - 1.0f, t2 = fx - 0.5f;
        w[0] = 0.5f * t0 * t0;
        w[1] = 0.75f - t1 * t1;
        w[2] = 0.5f * t2 * t2;
        dw[0] = -t0;
        dw[1] = -2.0f * t1;
        dw[2] = t2;
    } else {
        w[0] = 1.0f - fx;
        w[1] = fx;
        dw[0] = -1.0f;
        dw[1] = 1.0f;
    }
}

// Offset and weights of a particle along one axis when its span is known
// (the thread's span, first support node cb): no float<->int conversion on
// the critical path.  Returns whether fx lies in the span's nominal interval
// (it may sit one ulp outside at a span edge); the P2G kernel ignores it: the
// G2PD step checks every particle's span against its tile.
template <int P, bool PER>
__device__ __forceinline__ bool axis_known(float x, float lo, float ih, float cb, float n, float* w, float* dw)
{
    const float xi = __fmul_rn(__fsub_rn(x, lo), ih);
    float fx = xi - cb;
    // degree 2, periodic: a particle at xi in [n - 1/2, n) belongs to span 0
    // (its nearest node wraps to 0); seen from span 0 its offset is fx + n
    if (PER && P == 2 && fx > 0.5f * n + 0.75f) fx -= n;
    weights1d<P>(fx, w, dw);
    return P == 2 ? (fx > 0.499f && fx < 1.501f) : (fx > -0.001f && fx < 1.001f);
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// axis_known for two axes at once (the x and y axes of a particle) in packed
// f32x2 arithmetic, with the same IEEE operations per axis: x - lo as
// x + (-lo), 1.5 - fx as fx (-1) + 1.5 (one rounding), and 0.75 - (fx - 1)^2
// as (fx - 1)(1 - fx) + 0.75 (one rounding; 1 - fx is -(fx - 1) exactly).
template <int P, bool PER>
__device__ __forceinline__ void axes2_known(float2 x, float2 nlo, float2 ih2, float2 ncb, float n0, float n1,
                                            float* wa, float* wb, float* dwa, float* dwb)
{
    float2 fx = __fadd2_rn(__fmul2_rn(__fadd2_rn(x, nlo), ih2), ncb);
    if (PER && P == 2) {
        if (fx.x > 0.5f * n0 + 0.75f) fx.x -= n0;
        if (fx.y > 0.5f * n1 + 0.75f) fx.y -= n1;
    }
    if constexpr (P == 2) {
        const float2 m1 = f2(-1.f, -1.f), hf = f2(0.5f, 0.5f);
        const float2 t0 = __ffma2_rn(fx, m1, f2(1.5f, 1.5f));
        const float2 t1 = __fadd2_rn(fx, m1);
        const float2 u1 = __ffma2_rn(fx, m1, f2(1.f, 1.f));
        const float2 t2 = __fadd2_rn(fx, f2(-0.5f, -0.5f));
        const float2 w0 = __fmul2_rn(__fmul2_rn(hf, t0), t0);
        const float2 w1 = __ffma2_rn(t1, u1, f2(0.75f, 0.75f));
        const float2 w2 = __fmul2_rn(__fmul2_rn(hf, t2), t2);
        wa[0] = w0.x; wa[1] = w1.x; wa[2] = w2.x;
        wb[0] = w0.y; wb[1] = w1.y; wb[2] = w2.y;
        dwa[0] = -t0.x; dwa[1] = 2.0f * u1.x; dwa[2] = t2.x;
        dwb[0] = -t0.y; dwb[1] = 2.0f * u1.y; dwb[2] = t2.y;
    } else {
        const float2 u = __ffma2_rn(fx, f2(-1.f, -1.f), f2(1.f, 1.f));
        wa[0] = u.x; wa[1] = fx.x;
        wb[0] = u.y; wb[1] = fx.y;
        dwa[0] = -1.f; dwa[1] = 1.f;
        dwb[0] = -1.f; dwb[1] = 1.f;
    }
}

// Add one node row of a span's contributions into the shared window with the
// neighbouring spans of the same x-row summed first.  Lane = span x in its
// row segment of T0 lanes (lx); v[a] = contribution to window node lx + a.
// Node lx gets v[0] of its own span, v[1] of span lx - 1 and v[2] of span
// lx - 2 (warp shuffles); the last two lanes of a segment also carry the
// halo nodes T0 and T0 + 1.  All lanes of the warp must call this together.
// Plain read-add-write: valid when no other warp writes this field of the
// window at the same time.  Within the instruction every lane writes a
// different node (lanes of different row segments use different node rows
// for the same (b, c)).
template <bool ATOMIC>
__device__ __forceinline__ void sh_add(float* p, float v)
{
    if constexpr (ATOMIC) atomicAdd(p, v);
    else *p += v;
}
template <bool ATOMIC>
__device__ __forceinline__ void sh_add(double* p, double v)
{
    if constexpr (ATOMIC) atomicAdd(p, v);
    else *p += v;
}
template <bool ATOMIC>
__device__ __forceinline__ void sh_add(long long* p, long long v)
{
    if constexpr (ATOMIC) atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
    else *p += v;
}

// ATOMIC: rows that other warps may update at the same time.
// Without ATOMIC the call starts with a warp barrier: lanes of different row
// segments (different y) reach the same node row in different calls.
template <int NS, class T, bool ATOMIC = false>
__device__ __forceinline__ void xrow_rmw(T* row, const T* v, int lx, int T0)
{
    if constexpr (!ATOMIC) __syncwarp();
    T s = v[0];
#pragma unroll
    for (int a = 1; a < NS; ++a) {
        const T u = __shfl_up_sync(0xffffffffu, v[a], a);
        if (lx >= a) s += u;
    }
    sh_add<ATOMIC>(row + lx, s);
    if (NS == 3) {
        const T u2 = __shfl_up_sync(0xffffffffu, v[2], 1);
        const T d2 = __shfl_down_sync(0xffffffffu, v[2], 1);
        if (lx >= T0 - 2) {
            const int o = lx == T0 - 1 ? T0 : T0 + 1;
            sh_add<ATOMIC>(row + o, lx == T0 - 1 ? v[1] + u2 : d2);
        }
    } else {
        if (lx == T0 - 1) sh_add<ATOMIC>(row + T0, v[NS - 1]);
    }
}

// Grid fields a kernel adds into: field f at p0 + f * stride (the fields of
// one kind are consecutive arrays of one allocation).
struct FieldPtrs {
    float* p0;
    int64_t stride;
};

// Add a tile's shared-memory window (nf fields of W floats) into global node
// rows.  Rows are padded to a multiple of 4 nodes and tiles start on a
// multiple of 4 spans, so x-chunks of 4 nodes are 16-byte aligned.
// TX, TY, TZ > 0: the tile edges as compile-time constants (3D); the
// chunk, row and field of a thread's item then come from integer divisions
// by constants.
template <int D, int P, int TX = 0, int TY = 0, int TZ = 0>
__device__ __forceinline__ void flush_window(const Geom& G, const int so[3], const float* sm, int nf,
                                             const FieldPtrs& dst)
{
    constexpr bool ST = TX > 0;
    static_assert(!ST || (D == 3 && TX % 4 == 0), "static windows: 3D tiles of a multiple of 4 spans in x");
    constexpr int SW0 = TX + P, SW1 = TY + P, SW2 = TZ + P, SNCH = (SW0 + 3) / 4;
    const int W0 = ST ? SW0 : G.W[0], W1 = ST ? SW1 : G.W[1];
    const int W = ST ? SW0 * SW1 * SW2 : G.Wvol;
    const int nch = ST ? SNCH : (W0 + 3) >> 2;
    const int nrow = ST ? SW1 * SW2 : W1 * G.W[2];
    const bool vec = !G.per[0] && (ST || G.T[0] % 4 == 0);
    // t < 7 * 66^2 * 17 < 2^21: exact quotients from float reciprocals
    const float inch = 1.0f / (float)nch, inrow = 1.0f / (float)nrow;
    for (int t = threadIdx.x; t < nf * nrow * nch; t += blockDim.x) {
        int q, f, wy, wz;
        if constexpr (ST) {
            const unsigned tq = (unsigned)t / SNCH, r = tq % (SW1 * SW2);
            q = (int)((unsigned)t - tq * SNCH);
            f = (int)(tq / (SW1 * SW2));
            wz = (int)(r / SW1);
            wy = (int)(r - (unsigned)wz * SW1);
        } else {
            const int tq = div_small(t, inch);
            q = t - tq * nch;
            f = div_small(tq, inrow);
            const int r = tq - f * nrow;
            wz = div_small(r, G.inv_w[1]);
            wy = r - wz * W1;
        }
        int iy = so[1] + wy, iz = D == 3 ? so[2] + wz : 0;
        if (G.per[1]) {
            iy -= (P == 2 ? 1 : 0);
            iy %= G.n[1];
            if (iy < 0) iy += G.n[1];
        } else if (iy >= G.N[1]) {
            continue;
        }
        if (D == 3) {
            if (G.per[2]) {
                iz -= (P == 2 ? 1 : 0);
                iz %= G.n[2];
                if (iz < 0) iz += G.n[2];
            } else if (iz >= G.N[2]) {
                continue;
            }
        }
        const float* src = sm + f * W + (wz * W1 + wy) * W0;
        float* row = dst.p0 + f * dst.stride + ((int64_t)iz * G.N[1] + iy) * G.pitch;
        const int x0 = 4 * q;
        if (vec) {
            const int gx = so[0] + x0;
            if (gx >= G.pitch) continue;
            float4 v;
            v.x = src[x0];
            v.y = x0 + 1 < W0 ? src[x0 + 1] : 0.f;
            v.z = x0 + 2 < W0 ? src[x0 + 2] : 0.f;
            v.w = x0 + 3 < W0 ? src[x0 + 3] : 0.f;
            if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
                atomicAdd(reinterpret_cast<float4*>(row + gx), v);
        } else {
            for (int j = x0; j < min(x0 + 4, W0); ++j) {
                int gx = so[0] + j;
                if (G.per[0]) {
                    gx -= (P == 2 ? 1 : 0);
                    gx %= G.n[0];
                    if (gx < 0) gx += G.n[0];
                } else if (gx >= G.N[0]) {
                    continue;
                }
                const float v = src[j];
                if (v != 0.f) atomicAdd(row + gx, v);
            }
        }
    }
}

// ---------------------------------------------------------------- K1: P2G

// Two warps per CTA: warp 0 sums m and M V, warp 1 the force (P + Q) M/rho
// grad(phi), each over all spans of the tile, 32 consecutive spans (one
// x-row for the default tiles) at a time; both read the same particles.
// Each warp is the only writer of its fields of the window, so the per-span
// sums go in with plain shared-memory adds.
constexpr int kP2GThreads = 64;

// 3D span columns: a lane walks the spans of one (x, y) column along z (rows
// of 32 spans are z-major in a tile).  Its sums hold the three node layers of
// the current span; after each span the lowest layer is complete and goes
// into the window, the two others move down and the top one starts at zero.
// (Rotating the layers through register slots instead of moving them, with
// the walk unrolled by three spans, was slower: three copies of the particle
// loop miss the instruction cache.)  GROUP 0 sums {m, mv_x, mv_y, mv_z},
// GROUP 1 {f_x, f_y, f_z}.  TX, TY, TZ > 0: the tile edges as compile-time constants
// (window offsets become immediates); 0: read from the geometry.
__host__ __device__ constexpr int clog2(int v) { return v <= 1 ? 0 : 1 + clog2(v >> 1); }

template <int P, int GROUP>
struct ZcolSums {
    static constexpr int NS = P + 1, L = NS * NS;
    // GROUP 0: qa = {m, mv_x}, qb = {mv_y, mv_z}; GROUP 1: qa = {f_y, f_z}, qc = f_x
    float2 qa[NS][L];
    float2 qb[GROUP == 0 ? NS : 1][GROUP == 0 ? L : 1];
    float qc[GROUP == 0 ? 1 : NS][GROUP == 0 ? 1 : L];
    __device__ __forceinline__ void clear(int s)
    {
#pragma unroll
        for (int n = 0; n < L; ++n) {
            qa[s][n] = f2(0.f, 0.f);
            if constexpr (GROUP == 0) qb[s][n] = f2(0.f, 0.f); else qc[s][n] = 0.f;
        }
    }
};

// The next particle of a column walk, loaded one particle ahead: the next of
// the same span, or, after a span's last particle, the first of the next
// span up the column (have: loaded).  GROUP 0 keeps {x, v, M}, GROUP 1
// {x, M, rho, E, Q} (u = rho, E, Q).
struct ZcolNext {
    float x[3], u[3], M;
    bool have;
};

template <int GROUP>
__device__ __forceinline__ void zcol_load(const Particles<float>& pt, uint32_t k, ZcolNext& N)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) N.x[a] = pt.x[a][k];
    N.M = pt.M[k];
    if constexpr (GROUP == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) N.u[a] = pt.v[a][k];
    } else {
        N.u[0] = pt.rho[k]; N.u[1] = pt.E[k]; N.u[2] = pt.Q[k];
    }
}

// One span of a column: its particles into the sums (layer c in slot c),
// then the completed layers into the window.  Returns whether it was the
// column's last span.
template <int P, bool PER, int GROUP, int TX, int TY, int TZ>
__device__ __forceinline__ bool zcol_span(const Geom& G, const Particles<float>& pt, const uint32_t* __restrict__ cs,
                                          int64_t kb, const int so[3], const float lo[3], const float nper[3],
                                          float ih, float gm1, float* sm, int lane, int yb, int rpl, int z, int nz,
                                          ZcolSums<P, GROUP>& S, ZcolNext& N)
{
    constexpr int NS = P + 1;
    constexpr bool ST = TX > 0;
    const int T0 = ST ? TX : G.T[0], T1 = ST ? TY : G.T[1];
    const int sh0 = ST ? clog2(TX) : G.tsh[0];
    const int W0 = ST ? TX + P : G.W[0], W1 = ST ? TY + P : G.W[1];
    const int W = ST ? (TX + P) * (TY + P) * (TZ + P) : G.Wvol;
    // a warp row of 32 spans: for tiles narrower than 32 spans, the y-rows
    // yb, yb + rpl, .. of the z-layer (lanes of different rows are rpl rows
    // apart); otherwise 32 consecutive spans of one x-row
    int lx, ly;
    if (T0 >= 32) {
        const int s0 = ((z * rpl + yb) << 5) + lane;
        lx = s0 & (T0 - 1);
        ly = (s0 >> sh0) & (T1 - 1);
    } else {
        lx = lane & (T0 - 1);
        ly = (lane >> sh0) * rpl + yb;
    }
    const int s = ((z * T1 + ly) << sh0) + lx;
    const uint32_t b = cs[kb + s], e = cs[kb + s + 1];
    const int base = (z * W1 + ly) * W0 + lx;
    const int sn = s + T0 * T1;                 // the next span up the column
    const bool up = z + 1 < nz;
    const uint32_t nb = up ? cs[kb + sn] : 0u, ne = up ? cs[kb + sn + 1] : 0u;
    const float cb0 = (float)(so[0] + lx - (P == 2 ? 1 : 0));
    const float cb1 = (float)(so[1] + ly - (P == 2 ? 1 : 0));
    const float cb2 = (float)(so[2] + z - (P == 2 ? 1 : 0));
    if constexpr (GROUP == 0) {
        if (!N.have && b < e) zcol_load<0>(pt, b, N);
        for (uint32_t k = b; k < e; ++k) {
            float x[3], v[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) { x[a] = N.x[a]; v[a] = N.u[a]; }
            const float M = N.M;
            if (k + 1 < e) zcol_load<0>(pt, k + 1, N);
            float w[3][3], dw[3][3];
            axes2_known<P, PER>(f2(x[0], x[1]), f2(-lo[0], -lo[1]), f2(ih, ih), f2(-cb0, -cb1), nper[0], nper[1],
                                w[0], w[1], dw[0], dw[1]);
            axis_known<P, PER>(x[2], lo[2], ih, cb2, nper[2], w[2], dw[2]);
            float2 c0[NS], c1[NS];
            const float mv0 = M * v[0], mv1 = M * v[1], mv2 = M * v[2];
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                const float wa = w[0][a];
                c0[a] = f2(M * wa, mv0 * wa);
                c1[a] = f2(mv1 * wa, mv2 * wa);
            }
#pragma unroll
            for (int c = 0; c < NS; ++c) {
#pragma unroll
                for (int bb = 0; bb < NS; ++bb) {
                    const float yz = w[1][bb] * w[2][c];
                    const float2 yy = f2(yz, yz);
                    const int sl = c;
#pragma unroll
                    for (int a = 0; a < NS; ++a) {
                        S.qa[sl][bb * NS + a] = __ffma2_rn(c0[a], yy, S.qa[sl][bb * NS + a]);
                        S.qb[sl][bb * NS + a] = __ffma2_rn(c1[a], yy, S.qb[sl][bb * NS + a]);
                    }
                }
            }
        }
    } else {
        if (!N.have && b < e) zcol_load<1>(pt, b, N);
        for (uint32_t k = b; k < e; ++k) {
            float x[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) x[a] = N.x[a];
            const float M = N.M, rho = N.u[0], E = N.u[1], Q = N.u[2];
            if (k + 1 < e) zcol_load<1>(pt, k + 1, N);
            float w[3][3], dw[3][3];
            axes2_known<P, PER>(f2(x[0], x[1]), f2(-lo[0], -lo[1]), f2(ih, ih), f2(-cb0, -cb1), nper[0], nper[1],
                                w[0], w[1], dw[0], dw[1]);
            axis_known<P, PER>(x[2], lo[2], ih, cb2, nper[2], w[2], dw[2]);
            const float F = fmaf(gm1 * rho, E, Q) * __fdividef(M, rho) * ih;
            float Fx[NS], Fd[NS];
#pragma unroll
            for (int a = 0; a < NS; ++a) { Fx[a] = F * w[0][a]; Fd[a] = F * dw[0][a]; }
#pragma unroll
            for (int c = 0; c < NS; ++c) {
#pragma unroll
                for (int bb = 0; bb < NS; ++bb) {
                    const float yz = w[1][bb] * w[2][c];
                    const float2 dd = f2(dw[1][bb] * w[2][c], w[1][bb] * dw[2][c]);
                    const int sl = c;
#pragma unroll
                    for (int a = 0; a < NS; ++a) {
                        S.qa[sl][bb * NS + a] = __ffma2_rn(f2(Fx[a], Fx[a]), dd, S.qa[sl][bb * NS + a]);
                        S.qc[sl][bb * NS + a] = fmaf(Fd[a], yz, S.qc[sl][bb * NS + a]);
                    }
                }
            }
        }
    }
    // the first particle of the next span up the column, loaded before this
    // span's layer adds
    N.have = nb < ne;
    if (N.have) zcol_load<GROUP>(pt, nb, N);
    // the completed node layers (the lowest, or all three after the column's
    // last span) go into the window in phases: in phase (a, g) lane (lx, ly)
    // adds its sums of the nodes (lx + a, ly + bb) with bb / ystep = g.  Lanes
    // of one y-row then write different nodes; lanes of two y-rows (rpl rows
    // apart, or adjacent when a warp row is one x-row) can meet only when
    // their bb differ by a multiple of that distance, which never happens
    // within one group.  A warp barrier separates the phases.
    const bool last = z + 1 == nz;
    float* sp = sm + base;
    const int ystep = T0 >= 32 ? NS : rpl;
#pragma unroll
    for (int a = 0; a < NS; ++a) {
#pragma unroll
        for (int g = 0; g < NS; ++g) {
            if (g * ystep >= NS) break;
            __syncwarp();
#pragma unroll
            for (int c = 0; c < NS; ++c) {
                if (c > 0 && !last) break;
                const int sl = c;
#pragma unroll
                for (int bb = 0; bb < NS; ++bb) {
                    if (bb / ystep != g) continue;
                    const int n = bb * NS + a;
                    float* r = sp + (c * W1 + bb) * W0 + a;
                    if constexpr (GROUP == 0) {
                        r[0] += S.qa[sl][n].x;
                        r[W] += S.qa[sl][n].y;
                        r[2 * W] += S.qb[sl][n].x;
                        r[3 * W] += S.qb[sl][n].y;
                    } else {
                        r[4 * W] += S.qc[sl][n];          // f_x
                        r[5 * W] += S.qa[sl][n].x;        // f_y
                        r[6 * W] += S.qa[sl][n].y;        // f_z
                    }
                }
            }
        }
    }
    __syncwarp();
    return last;
}

template <int P, bool PER, int GROUP, int TX, int TY, int TZ>
__device__ __forceinline__ void p2g_zcol(const Geom& G, const Particles<float>& pt, const uint32_t* __restrict__ cs,
                                         int64_t kb, const int so[3], const float lo[3], const float nper[3],
                                         float ih, float gm1, float* sm, int lane)
{
    constexpr int NS = P + 1;
    constexpr bool ST = TX > 0;
    const int T0 = ST ? TX : G.T[0], T1 = ST ? TY : G.T[1], T2 = ST ? TZ : G.T[2];
    const int sh0 = ST ? clog2(TX) : G.tsh[0];
    const int rpl = (T0 * T1) >> 5;
    // spans beyond the last one of an axis hold no particles: a tile at the
    // domain's end walks only its real z-layers and rows
    const int nz = min(T2, G.S[2] - so[2]);
    for (int yb = 0; yb < rpl; ++yb) {
        // the warp row's first span in its z-layer (its lowest y-row)
        const int r0 = T0 >= 32 ? yb << 5 : yb << sh0;
        if (so[1] + (r0 >> sh0) >= G.S[1] || so[0] + (r0 & (T0 - 1)) >= G.S[0]) continue;
        ZcolSums<P, GROUP> S;
#pragma unroll
        for (int sl = 0; sl < NS; ++sl) S.clear(sl);
        ZcolNext N;
        N.have = false;
        for (int z = 0; z < nz; ++z) {
            if (zcol_span<P, PER, GROUP, TX, TY, TZ>(G, pt, cs, kb, so, lo, nper, ih, gm1, sm, lane, yb, rpl, z, nz,
                                                    S, N)) break;
            // the layers move down; the new top layer starts at zero
#pragma unroll
            for (int sl = 0; sl + 1 < NS; ++sl) {
#pragma unroll
                for (int n = 0; n < NS * NS; ++n) {
                    S.qa[sl][n] = S.qa[sl + 1][n];
                    if constexpr (GROUP == 0) S.qb[sl][n] = S.qb[sl + 1][n]; else S.qc[sl][n] = S.qc[sl + 1][n];
                }
            }
            S.clear(NS - 1);
        }
    }
}


// 2D span columns: a lane walks the spans of one x along y (rows of 32 spans
// are x-rows of a tile at least 32 spans wide).  Its sums hold the three node
// rows of the current span; after each span the lowest row is complete and
// goes into the window in NS phases, the two others move down.  GROUP 0 sums
// {m, mv_x, mv_y}, GROUP 1 {f_x, f_y}.
template <int P, bool PER, int GROUP>
__device__ __forceinline__ void p2g_ycol(const Geom& G, const Particles<float>& pt, const uint32_t* __restrict__ cs,
                                         int64_t kb, const int so[3], const float lo[3], const float nper[3],
                                         float ih, float gm1, float* sm, int lane)
{
    constexpr int NS = P + 1, NN = NS * NS, L = NS;
    const int W = G.Wvol, W0 = G.W[0];
    const int rpl = G.T[0] >> 5;                       // rows of 32 spans per y-line
    const int ny = min(G.T[1], G.S[1] - so[1]);        // real y-lines of the tile
    for (int xb = 0; xb < rpl; ++xb) {
        if (so[0] + (xb << 5) >= G.S[0]) continue;
        // GROUP 0: qa = {m, mv_x}, qc = mv_y; GROUP 1: qa = {f_x, f_y}
        float2 qa[NN];
        float qc[GROUP == 0 ? NN : 1];
#pragma unroll
        for (int i = 0; i < NN; ++i) {
            qa[i] = f2(0.f, 0.f);
            if (GROUP == 0) qc[i] = 0.f;
        }
        for (int y = 0; y < ny; ++y) {
            const int s = ((y * rpl + xb) << 5) + lane;
            const uint32_t b = cs[kb + s], e = cs[kb + s + 1];
            const int lx = s & (G.T[0] - 1);
            const int base = y * W0 + lx;
            const float cb0 = (float)(so[0] + lx - (P == 2 ? 1 : 0));
            const float cb1 = (float)(so[1] + y - (P == 2 ? 1 : 0));
            if (GROUP == 0) {
                float nx[2] = {0.f, 0.f}, nv[2] = {0.f, 0.f}, nM = 0.f;
                if (b < e) {
#pragma unroll
                    for (int a = 0; a < 2; ++a) { nx[a] = pt.x[a][b]; nv[a] = pt.v[a][b]; }
                    nM = pt.M[b];
                }
                for (uint32_t k = b; k < e; ++k) {
                    float x[2], v[2];
#pragma unroll
                    for (int a = 0; a < 2; ++a) { x[a] = nx[a]; v[a] = nv[a]; }
                    const float M = nM;
                    if (k + 1 < e) {
#pragma unroll
                        for (int a = 0; a < 2; ++a) { nx[a] = pt.x[a][k + 1]; nv[a] = pt.v[a][k + 1]; }
                        nM = pt.M[k + 1];
                    }
                    float w[2][3], dw[2][3];
                    axis_known<P, PER>(x[0], lo[0], ih, cb0, nper[0], w[0], dw[0]);
                    axis_known<P, PER>(x[1], lo[1], ih, cb1, nper[1], w[1], dw[1]);
                    const float mv0 = M * v[0], mv1 = M * v[1];
                    float2 c0[NS];
                    float c3[NS];
#pragma unroll
                    for (int a = 0; a < NS; ++a) {
                        const float wa = w[0][a];
                        c0[a] = f2(M * wa, mv0 * wa);
                        c3[a] = mv1 * wa;
                    }
#pragma unroll
                    for (int j = 0; j < NS; ++j) {
                        const float yj = w[1][j];
#pragma unroll
                        for (int a = 0; a < NS; ++a) {
                            qa[j * NS + a] = __ffma2_rn(c0[a], f2(yj, yj), qa[j * NS + a]);
                            qc[j * NS + a] = fmaf(c3[a], yj, qc[j * NS + a]);
                        }
                    }
                }
            } else {
                float nx[2] = {0.f, 0.f}, nM = 0.f, nr = 1.f, nE = 0.f, nQ = 0.f;
                if (b < e) {
#pragma unroll
                    for (int a = 0; a < 2; ++a) nx[a] = pt.x[a][b];
                    nM = pt.M[b]; nr = pt.rho[b]; nE = pt.E[b]; nQ = pt.Q[b];
                }
                for (uint32_t k = b; k < e; ++k) {
                    float x[2];
#pragma unroll
                    for (int a = 0; a < 2; ++a) x[a] = nx[a];
                    const float M = nM, rho = nr, E = nE, Q = nQ;
                    if (k + 1 < e) {
#pragma unroll
                        for (int a = 0; a < 2; ++a) nx[a] = pt.x[a][k + 1];
                        nM = pt.M[k + 1]; nr = pt.rho[k + 1]; nE = pt.E[k + 1]; nQ = pt.Q[k + 1];
                    }
                    float w[2][3], dw[2][3];
                    axis_known<P, PER>(x[0], lo[0], ih, cb0, nper[0], w[0], dw[0]);
                    axis_known<P, PER>(x[1], lo[1], ih, cb1, nper[1], w[1], dw[1]);
                    const float F = fmaf(gm1 * rho, E, Q) * __fdividef(M, rho) * ih;
                    float2 cf[NS];
#pragma unroll
                    for (int a = 0; a < NS; ++a) cf[a] = f2(F * dw[0][a], F * w[0][a]);
#pragma unroll
                    for (int j = 0; j < NS; ++j) {
                        const float2 yd = f2(w[1][j], dw[1][j]);
#pragma unroll
                        for (int a = 0; a < NS; ++a) qa[j * NS + a] = __ffma2_rn(cf[a], yd, qa[j * NS + a]);
                    }
                }
            }
            // the completed node rows (the lowest, or all after the column's
            // last span) into the window in NS phases: in phase a lane lx
            // adds node lx + a, so the lanes of a phase write different nodes
            const bool last = y + 1 == ny;
            float* sp = sm + base;
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                __syncwarp();
#pragma unroll
                for (int j = 0; j < NS; ++j) {
                    if (j > 0 && !last) break;
                    const int i = j * NS + a;
                    float* r = sp + j * W0 + a;
                    if (GROUP == 0) {
                        r[0] += qa[i].x;
                        r[W] += qa[i].y;
                        r[2 * W] += qc[i];
                    } else {
                        r[3 * W] += qa[i].x;        // f_x
                        r[4 * W] += qa[i].y;        // f_y
                    }
                }
            }
            __syncwarp();
            if (last) break;
#pragma unroll
            for (int i = 0; i < NN; ++i) {
                if (i + L < NN) {
                    qa[i] = qa[i + L];
                    if (GROUP == 0) qc[i] = qc[i + L];
                } else {
                    qa[i] = f2(0.f, 0.f);
                    if (GROUP == 0) qc[i] = 0.f;
                }
            }
        }
    }
}

__host__ __device__ inline bool p2g_columns(const Geom& G)
{
    return G.dim == 3 ? G.T[0] * G.T[1] >= 32 : G.T[0] >= 32;
}

// COL: 3D tiles whose z-layers hold whole rows of 32 spans walk span columns
// (p2g_zcol); the others walk rows.  Separate instantiations keep each
// kernel's registers to its own path.
// TX, TY, TZ > 0 (3D span columns only): the tile edges as compile-time
// constants.
template <int D, int P, bool PER, bool COL, int TX = 0, int TY = 0, int TZ = 0>
__device__ __forceinline__ void p2g_span_tile(const Geom& G, const Particles<float>& pt, const FieldPtrs& out,
                                              const uint32_t* __restrict__ cs, Clock* clk, const int tile)
{
    constexpr bool ST = TX > 0;
    static_assert(!ST || (D == 3 && COL), "static tiles: 3D span columns");
    const int64_t kb = tile_cs0(G, tile);
    // compile-time tiles read the run state and the tile's particle range
    // while they clear their window, and return (uniformly) after that
    const int active = clk->active;
    const uint32_t pb = cs[kb], pe = cs[kb + (ST ? TX * TY * TZ : G.Tvol)];
    if (!ST && (!active || pb == pe)) return;
    extern __shared__ __align__(16) float sm[];
    constexpr int NS = P + 1, NF = 1 + 2 * D, NYZ = (D == 3) ? NS * NS : NS, NN = NYZ * NS;
    const int W = ST ? (TX + P) * (TY + P) * (TZ + P) : G.Wvol, W0 = G.W[0], W1 = G.W[1];
    for (int i = threadIdx.x; i < (NF * W) >> 2; i += blockDim.x)
        reinterpret_cast<float4*>(sm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = ((NF * W) & ~3) + threadIdx.x; i < NF * W; i += blockDim.x) sm[i] = 0.f;
    if (ST && (!active || pb == pe)) return;
    __syncthreads();
    int so[3];
    tile_origin(G, tile, so);
    const float gm1 = (float)(G.gamma - 1.0), ih = (float)G.inv_h;
    float lo[3], nper[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = (float)G.lo[a];
        nper[a] = G.per[a] ? (float)G.n[a] : 3.0e38f;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int group = warp & 1;
    if constexpr (COL) {
        if constexpr (D == 3) {
            if (group == 0) p2g_zcol<P, PER, 0, TX, TY, TZ>(G, pt, cs, kb, so, lo, nper, ih, gm1, sm, lane);
            else p2g_zcol<P, PER, 1, TX, TY, TZ>(G, pt, cs, kb, so, lo, nper, ih, gm1, sm, lane);
        } else {
            if (group == 0) p2g_ycol<P, PER, 0>(G, pt, cs, kb, so, lo, nper, ih, gm1, sm, lane);
            else p2g_ycol<P, PER, 1>(G, pt, cs, kb, so, lo, nper, ih, gm1, sm, lane);
        }
        __syncthreads();
        flush_window<D, P, TX, TY, TZ>(G, so, sm, NF, out);
        return;
    }
    const int nrows = G.Tvol >> 5;
    for (int r = 0; r < nrows; ++r) {
        const int s = (r << 5) + lane;
        // empty spans take part in the warp-wide row adds with zeros
        const uint32_t b = cs[kb + s], e = cs[kb + s + 1];
        const int lx = s & (G.T[0] - 1);
        const int ly = (s >> G.tsh[0]) & (G.T[1] - 1);
        const int lz = s >> (G.tsh[0] + G.tsh[1]);
        const int base = (lz * W1 + ly) * W0 + lx;
        const float cb0 = (float)(so[0] + lx - (P == 2 ? 1 : 0));
        const float cb1 = (float)(so[1] + ly - (P == 2 ? 1 : 0));
        const float cb2 = (float)(so[2] + lz - (P == 2 ? 1 : 0));
        if (__all_sync(0xffffffffu, b == e)) continue;
        // x-reduction segment: the spans of this warp chunk that share a row
        const int tseg = G.T[0] < 32 ? G.T[0] : 32;
        const int lxw = lane & (tseg - 1);
        if (group == 0) {
            // 3D: q0 = {m, mv_x}, q1 = {mv_y, mv_z}; 2D: q0 = {m, mv_x}, q3 = mv_y
            float2 q0[NN], q1[D == 3 ? NN : 1];
            float q3[D == 3 ? 1 : NN];
#pragma unroll
            for (int i = 0; i < NN; ++i) {
                q0[i] = f2(0.f, 0.f);
                if (D == 3) q1[i] = f2(0.f, 0.f); else q3[i] = 0.f;
            }
            float nx[3] = {0.f, 0.f, 0.f}, nv[3] = {0.f, 0.f, 0.f}, nM = 0.f;
            if (b < e) {
#pragma unroll
                for (int a = 0; a < D; ++a) { nx[a] = pt.x[a][b]; nv[a] = pt.v[a][b]; }
                nM = pt.M[b];
            }
            for (uint32_t k = b; k < e; ++k) {
                float x[3], v[3];
#pragma unroll
                for (int a = 0; a < D; ++a) { x[a] = nx[a]; v[a] = nv[a]; }
                const float M = nM;
                if (k + 1 < e) {
#pragma unroll
                    for (int a = 0; a < D; ++a) { nx[a] = pt.x[a][k + 1]; nv[a] = pt.v[a][k + 1]; }
                    nM = pt.M[k + 1];
                }
                float w[3][3], dw[3][3];
                axis_known<P, PER>(x[0], lo[0], ih, cb0, nper[0], w[0], dw[0]);
                axis_known<P, PER>(x[1], lo[1], ih, cb1, nper[1], w[1], dw[1]);
                if (D == 3) axis_known<P, PER>(x[2], lo[2], ih, cb2, nper[2], w[2], dw[2]);
                float2 c0[NS], c1[NS];
                float c3[NS];
                const float mv0 = M * v[0], mv1 = M * v[1], mv2 = D == 3 ? M * v[2] : 0.f;
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    const float wa = w[0][a];
                    c0[a] = f2(M * wa, mv0 * wa);
                    if (D == 3) c1[a] = f2(mv1 * wa, mv2 * wa); else c3[a] = mv1 * wa;
                }
#pragma unroll
                for (int j = 0; j < NYZ; ++j) {
                    const float yz = D == 3 ? w[1][j % NS] * w[2][j / NS] : w[1][j];
                    const float2 yy = f2(yz, yz);
#pragma unroll
                    for (int a = 0; a < NS; ++a) {
                        const int i = j * NS + a;
                        q0[i] = __ffma2_rn(c0[a], yy, q0[i]);
                        if (D == 3) q1[i] = __ffma2_rn(c1[a], yy, q1[i]);
                        else q3[i] = fmaf(c3[a], yz, q3[i]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < NYZ; ++j) {
                const int row = base - lxw + ((D == 3 ? j / NS : 0) * W1 + (D == 3 ? j % NS : j)) * W0;
                float v[NS];
#pragma unroll
                for (int a = 0; a < NS; ++a) v[a] = q0[j * NS + a].x;
                xrow_rmw<NS>(sm + row, v, lxw, tseg);
#pragma unroll
                for (int a = 0; a < NS; ++a) v[a] = q0[j * NS + a].y;
                xrow_rmw<NS>(sm + W + row, v, lxw, tseg);
#pragma unroll
                for (int a = 0; a < NS; ++a) v[a] = D == 3 ? q1[j * NS + a].x : q3[j * NS + a];
                xrow_rmw<NS>(sm + 2 * W + row, v, lxw, tseg);
                if (D == 3) {
#pragma unroll
                    for (int a = 0; a < NS; ++a) v[a] = q1[j * NS + a].y;
                    xrow_rmw<NS>(sm + 3 * W + row, v, lxw, tseg);
                }
            }
        } else {
            // 3D: q2 = {f_y, f_z}, q3 = f_x; 2D: q2 = {f_x, f_y}
            float2 q2[NN];
            float q3[D == 3 ? NN : 1];
#pragma unroll
            for (int i = 0; i < NN; ++i) {
                q2[i] = f2(0.f, 0.f);
                if (D == 3) q3[i] = 0.f;
            }
            float nx[3] = {0.f, 0.f, 0.f}, nM = 0.f, nr = 1.f, nE = 0.f, nQ = 0.f;
            if (b < e) {
#pragma unroll
                for (int a = 0; a < D; ++a) nx[a] = pt.x[a][b];
                nM = pt.M[b]; nr = pt.rho[b]; nE = pt.E[b]; nQ = pt.Q[b];
            }
            for (uint32_t k = b; k < e; ++k) {
                float x[3];
#pragma unroll
                for (int a = 0; a < D; ++a) x[a] = nx[a];
                const float M = nM, rho = nr, E = nE, Q = nQ;
                if (k + 1 < e) {
#pragma unroll
                    for (int a = 0; a < D; ++a) nx[a] = pt.x[a][k + 1];
                    nM = pt.M[k + 1]; nr = pt.rho[k + 1]; nE = pt.E[k + 1]; nQ = pt.Q[k + 1];
                }
                float w[3][3], dw[3][3];
                axis_known<P, PER>(x[0], lo[0], ih, cb0, nper[0], w[0], dw[0]);
                axis_known<P, PER>(x[1], lo[1], ih, cb1, nper[1], w[1], dw[1]);
                if (D == 3) axis_known<P, PER>(x[2], lo[2], ih, cb2, nper[2], w[2], dw[2]);
                const float F = fmaf(gm1 * rho, E, Q) * __fdividef(M, rho) * ih;
                if (D == 3) {
                    float Fx[NS], Fd[NS];
#pragma unroll
                    for (int a = 0; a < NS; ++a) { Fx[a] = F * w[0][a]; Fd[a] = F * dw[0][a]; }
#pragma unroll
                    for (int j = 0; j < NYZ; ++j) {
                        const int bb = j % NS, c = j / NS;
                        const float yz = w[1][bb] * w[2][c];
                        const float2 dd = f2(dw[1][bb] * w[2][c], w[1][bb] * dw[2][c]);
#pragma unroll
                        for (int a = 0; a < NS; ++a) {
                            const int i = j * NS + a;
                            q2[i] = __ffma2_rn(f2(Fx[a], Fx[a]), dd, q2[i]);
                            q3[i] = fmaf(Fd[a], yz, q3[i]);
                        }
                    }
                } else {
                    float2 cf[NS];
#pragma unroll
                    for (int a = 0; a < NS; ++a) cf[a] = f2(F * dw[0][a], F * w[0][a]);
#pragma unroll
                    for (int j = 0; j < NYZ; ++j) {
                        const float2 yd = f2(w[1][j], dw[1][j]);
#pragma unroll
                        for (int a = 0; a < NS; ++a) q2[j * NS + a] = __ffma2_rn(cf[a], yd, q2[j * NS + a]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < NYZ; ++j) {
                const int row = base - lxw + ((D == 3 ? j / NS : 0) * W1 + (D == 3 ? j % NS : j)) * W0;
                float v[NS];
                if (D == 3) {
#pragma unroll
                    for (int a = 0; a < NS; ++a) v[a] = q3[j * NS + a];
                    xrow_rmw<NS>(sm + 4 * W + row, v, lxw, tseg);     // f_x
                }
#pragma unroll
                for (int a = 0; a < NS; ++a) v[a] = q2[j * NS + a].x;
                xrow_rmw<NS>(sm + (D == 3 ? 5 : 3) * W + row, v, lxw, tseg);   // f_y (3D) / f_x (2D)
#pragma unroll
                for (int a = 0; a < NS; ++a) v[a] = q2[j * NS + a].y;
                xrow_rmw<NS>(sm + (D == 3 ? 6 : 4) * W + row, v, lxw, tseg);   // f_z (3D) / f_y (2D)
            }
        }
    }
    __syncthreads();
    flush_window<D, P>(G, so, sm, NF, out);
}

// tiles: the tiles of one colour pass (block b runs tiles[b]), or NULL (block
// b runs tile b)
template <int D, int P, bool PER, bool COL, int TX = 0, int TY = 0, int TZ = 0>
__global__ void __launch_bounds__(kP2GThreads, 6) k_p2g_span(Geom G, TileState<float> ts, FieldPtrs out, Clock* clk,
                                                              const uint32_t* __restrict__ tiles)
{
    const int t = tiles ? (int)tiles[blockIdx.x] : (int)blockIdx.x;
    p2g_span_tile<D, P, PER, COL, TX, TY, TZ>(G, ts.pt, out, ts.tpar[t] ? ts.cs[1] : ts.cs[0], clk, t);
}

// Tile shapes with compile-time variants of the 3D degree-2 FP32 span
// kernels: 1 = 8 x 8 x 8 spans, 2 = 16 x 8 x 4; 0 = none (edges read from the
// geometry).
__host__ __device__ inline int static_tile(const Geom& G)
{
    if (G.dim != 3 || G.p != 2) return 0;
    if (G.T[0] == 8 && G.T[1] == 8 && G.T[2] == 8) return 1;
    if (G.T[0] == 16 && G.T[1] == 8 && G.T[2] == 4) return 2;
    return 0;
}

// ------------------------------- 2D span-per-lane kernels, 64-bit sums
//
// P2G and grid + G2P + P2G of the 2D fixed-point and FP64 modes in the
// span-per-lane layout of K1: a lane takes the particles of its span one by
// one and sums their contributions to the span's (p+1)^2 support nodes in
// registers (int64 quanta, or binary64); each completed row of 32 spans goes
// into a shared window (x-neighbours summed by shuffles first), which is added
// to the grid once per node.  Every contribution is formed exactly as in the
// generic kernels (same weights, same operation order); fixed-point sums are
// exact and order independent, so they are bit-identical to the generic
// kernel's.  Registers bound this layout to two dimensions (3D needs
// 4 x 27 64-bit sums per lane); 3D keeps the generic kernels.
//
// Fixed point: rounding to int64 costs about as much as the rest of the
// kernel, so a particle whose every quantised contribution is bounded by 2^31
// in magnitude (checked from its largest weight, with a factor 2 margin for
// the roundings) takes the 32-bit conversion, which is exact there; the
// others take the 64-bit one.

// One particle's contributions into the lane sums: group 0 {M w, M V_x w,
// M V_y w} (a = {M, M V_x, M V_y}), group 1 {F g_x, F g_y} (a[0] = F).
template <int P, int GROUP, bool SMALL, class R, class A>
__device__ __forceinline__ void span2d_contribs(const Geom& G, const AxisSup<R>* sx, const R* a,
                                                A (&q)[GROUP == 0 ? 3 : 2][(P + 1) * (P + 1)])
{
    typedef Op<R> O;
    constexpr int NS = P + 1;
#pragma unroll
    for (int ky = 0; ky < NS; ++ky)
#pragma unroll
        for (int kx = 0; kx < NS; ++kx) {
            R w, g[3];
            node_weights<R, 2>(sx, kx, ky, 0, w, g);
            const int i = ky * NS + kx;
            if constexpr (GROUP == 0) {
                q[0][i] += Acc<A>::template from_t<SMALL>(O::mul(a[0], w), G.qscale[0]);
                q[1][i] += Acc<A>::template from_t<SMALL>(O::mul(a[1], w), G.qscale[1]);
                q[2][i] += Acc<A>::template from_t<SMALL>(O::mul(a[2], w), G.qscale[1]);
            } else {
                q[0][i] += Acc<A>::template from_t<SMALL>(O::mul(a[0], g[0]), G.qscale[2]);
                q[1][i] += Acc<A>::template from_t<SMALL>(O::mul(a[0], g[1]), G.qscale[2]);
            }
        }
}

template <int P, int GROUP, class R, class A>
__device__ __forceinline__ int p2g_span2d_group(const Geom& G, const Particles<R>& pt,
                                                const uint32_t* __restrict__ cs, int64_t kb, const int so[3], A* win)
{
    typedef Op<R> O;
    constexpr int NS = P + 1, NN = NS * NS, NQ = GROUP == 0 ? 3 : 2;
    const int W = G.Wvol, W0 = G.W[0];
    const int lane = threadIdx.x & 31;
    const R gm1 = (R)(G.gamma - 1.0), ih = (R)G.inv_h;
    const int nrows = G.Tvol >> 5;
    const int tseg = G.T[0] < 32 ? G.T[0] : 32;
    const int lxw = lane & (tseg - 1);
    int err = 0;
    for (int r = 0; r < nrows; ++r) {
        const int s = (r << 5) + lane;
        const uint32_t b = cs[kb + s], e = cs[kb + s + 1];
        const int lx = s & (G.T[0] - 1);
        const int ly = (s >> G.tsh[0]) & (G.T[1] - 1);
        if (__all_sync(0xffffffffu, b == e)) continue;
        A q[NQ][NN];
#pragma unroll
        for (int f = 0; f < NQ; ++f)
#pragma unroll
            for (int i = 0; i < NN; ++i) q[f][i] = A(0);
        for (uint32_t k = b; k < e; ++k) {
            AxisSup<R> sx[3];
            axis_support<R, P>(G, 0, pt.x[0][k], so[0], sx[0]);
            axis_support<R, P>(G, 1, pt.x[1][k], so[1], sx[1]);
            if (sx[0].l != lx || sx[1].l != ly) { err = 1; continue; }
            sx[2].l = 0;
            sx[2].w[0] = (R)1;
            sx[2].dw[0] = (R)0;
            const R M = pt.M[k];
            R a[3];
            if constexpr (GROUP == 0) {
                a[0] = M;
                a[1] = O::mul(M, pt.v[0][k]);
                a[2] = O::mul(M, pt.v[1][k]);
            } else {
                const R rho = pt.rho[k];
                const R Pk = O::mul(O::mul(gm1, rho), pt.E[k]);
                const R vol = O::dvd(M, rho);
                a[0] = O::mul(O::mul(O::add(Pk, pt.Q[k]), vol), ih);
                a[1] = a[2] = (R)0;
            }
            bool small = false;
            if constexpr (Acc<A>::kFixed) {
                R wm0, dm0, wm1, dm1;
                axis_bounds<NS>(sx[0], wm0, dm0);
                axis_bounds<NS>(sx[1], wm1, dm1);
                // NaN or infinity fails every comparison: full rounding
                if constexpr (GROUP == 0) {
                    const R wb = wm0 * wm1;
                    small = (M * G.qscale[0] * wb < kSmallQuanta) &
                            (fabs(a[1]) * G.qscale[1] * wb < kSmallQuanta) &
                            (fabs(a[2]) * G.qscale[1] * wb < kSmallQuanta);
                } else {
                    small = fabs(a[0]) * G.qscale[2] * fmax(dm0 * wm1, wm0 * dm1) < kSmallQuanta;
                }
            }
            if (small) span2d_contribs<P, GROUP, true>(G, sx, a, q);
            else span2d_contribs<P, GROUP, false>(G, sx, a, q);
        }
        const int base = ly * W0 + lx - lxw;
#pragma unroll
        for (int ky = 0; ky < NS; ++ky) {
#pragma unroll
            for (int f = 0; f < NQ; ++f) {
                A v[NS];
#pragma unroll
                for (int c = 0; c < NS; ++c) v[c] = q[f][ky * NS + c];
                // window fields: 0 m, 1 M V_x, 2 M V_y, 3 f_x, 4 f_y
                xrow_rmw<NS, A>(win + ((GROUP == 0 ? 0 : 3) + f) * W + base + ky * W0, v, lxw, tseg);
            }
        }
    }
    return err;
}

template <int P, class R, class A>
__device__ __forceinline__ void p2g_span2d_tile(const Geom& G, const Particles<R>& pt, const Grid<A, R>& gr,
                                                const uint32_t* __restrict__ cs, Clock* clk, const int tile)
{
    if (!clk->active) return;
    const int64_t kb = tile_cs0(G, tile);
    if (cs[kb] == cs[kb + G.Tvol]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A* swin = reinterpret_cast<A*>(smem_raw);
    constexpr int NF = 5;
    const int W = G.Wvol;
    for (int i = threadIdx.x; i < NF * W; i += blockDim.x) swin[i] = A(0);
    __syncthreads();
    int so[3];
    tile_origin(G, tile, so);
    // each warp is the only writer of its fields of the window
    const int err = (threadIdx.x >> 5) == 0 ? p2g_span2d_group<P, 0>(G, pt, cs, kb, so, swin)
                                            : p2g_span2d_group<P, 1>(G, pt, cs, kb, so, swin);
    if (err) atomicOr(&clk->err, ERR_TILE);
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        int idx[3];
        const int64_t node = slot_node<P>(G, so, i, idx);
        if (node < 0) continue;
        A* dst[NF] = {gr.m, gr.mv[0], gr.mv[1], gr.f[0], gr.f[1]};
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const A v = swin[f * W + i];
            if (v != A(0)) Acc<A>::add(dst[f] + node, v);
        }
    }
}

constexpr int kP2GSpan2dThreads = 64;

template <int P, class R, class A>
__global__ void __launch_bounds__(kP2GSpan2dThreads, 8) k_p2g_span2d(Geom G, TileState<R> ts, Grid<A, R> gr,
                                                                     Clock* clk)
{
    const int t = blockIdx.x;
    p2g_span2d_tile<P, R, A>(G, ts.pt, gr, ts.tpar[t] ? ts.cs[1] : ts.cs[0], clk, t);
}

// Grid update + G2P + P2G: the acceleration window is built as in the
// generic kernel; a lane then takes the particles of its span one by one --
// G2P sum in the generic node order, V' written back, M V' into 64-bit
// register sums for the span's support nodes -- and each warp adds its
// completed rows into the shared window with shared atomics (the rows of
// different warps overlap in y).
constexpr int kG2PSpan2dThreads = 128;

template <int P, class R, class A>
__device__ __forceinline__ void grid_g2p_span2d_tile(const Geom& G, const Particles<R>& pt, const Grid<A, R>& gr,
                                                     const uint32_t* __restrict__ cs, Clock* clk, const int tile)
{
    typedef Op<R> O;
    if (!clk->active) return;
    const int64_t kb = tile_cs0(G, tile);
    if (cs[kb] == cs[kb + G.Tvol]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int W = G.Wvol, W0 = G.W[0];
    R* sA = reinterpret_cast<R*>(smem_raw);
    A* s2 = reinterpret_cast<A*>(smem_raw + ((sizeof(R) * 2 * W + 15) & ~size_t(15)));
    int so[3];
    tile_origin(G, tile, so);
    accel_window<2, P, R, A>(G, gr, so, sA, s2);
    __syncthreads();
    constexpr int NS = P + 1, NN = NS * NS;
    const R dt = (R)clk->dt_cur;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int nrows = G.Tvol >> 5;
    const int tseg = G.T[0] < 32 ? G.T[0] : 32;
    const int lxw = lane & (tseg - 1);
    R vmax = (R)0;
    int err = 0;
    for (int r = warp; r < nrows; r += nwarps) {
        const int s = (r << 5) + lane;
        const uint32_t b = cs[kb + s], e = cs[kb + s + 1];
        const int lx = s & (G.T[0] - 1);
        const int ly = (s >> G.tsh[0]) & (G.T[1] - 1);
        if (__all_sync(0xffffffffu, b == e)) continue;
        A q[2][NN];
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
            for (int i = 0; i < NN; ++i) q[f][i] = A(0);
        for (uint32_t k = b; k < e; ++k) {
            AxisSup<R> sx[3];
            axis_support<R, P>(G, 0, pt.x[0][k], so[0], sx[0]);
            axis_support<R, P>(G, 1, pt.x[1][k], so[1], sx[1]);
            if (sx[0].l != lx || sx[1].l != ly) { err = 1; continue; }
            sx[2].l = 0;
            sx[2].w[0] = (R)1;
            sx[2].dw[0] = (R)0;
            R acc[2] = {(R)0, (R)0};
#pragma unroll
            for (int ky = 0; ky < NS; ++ky)
#pragma unroll
                for (int kx = 0; kx < NS; ++kx) {
                    R w, g[3];
                    node_weights<R, 2>(sx, kx, ky, 0, w, g);
                    const int slot = (ly + ky) * W0 + lx + kx;
                    acc[0] = O::add(acc[0], O::mul(w, sA[slot]));
                    acc[1] = O::add(acc[1], O::mul(w, sA[W + slot]));
                }
            const R M = pt.M[k];
            R MV[2], v2 = (R)0;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const R vn = O::add(pt.v[a][k], O::mul(dt, acc[a]));
                pt.v[a][k] = vn;
                MV[a] = O::mul(M, vn);
                v2 = O::add(v2, O::mul(vn, vn));
            }
            vmax = fmax(vmax, O::sqr(v2));
            bool small = false;
            if constexpr (Acc<A>::kFixed) {
                R wm0, dm0, wm1, dm1;
                axis_bounds<NS>(sx[0], wm0, dm0);
                axis_bounds<NS>(sx[1], wm1, dm1);
                small = fmax(fabs(MV[0]), fabs(MV[1])) * G.qscale[1] * (wm0 * wm1) < kSmallQuanta;
            }
            auto scatter = [&](auto sm) {
                constexpr bool SM = decltype(sm)::value;
#pragma unroll
                for (int ky = 0; ky < NS; ++ky)
#pragma unroll
                    for (int kx = 0; kx < NS; ++kx) {
                        R w, g[3];
                        node_weights<R, 2>(sx, kx, ky, 0, w, g);
                        q[0][ky * NS + kx] += Acc<A>::template from_t<SM>(O::mul(MV[0], w), G.qscale[1]);
                        q[1][ky * NS + kx] += Acc<A>::template from_t<SM>(O::mul(MV[1], w), G.qscale[1]);
                    }
            };
            if (small) scatter(std::true_type{});
            else scatter(std::false_type{});
        }
        const int base = ly * W0 + lx - lxw;
#pragma unroll
        for (int ky = 0; ky < NS; ++ky)
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                A v[NS];
#pragma unroll
                for (int c = 0; c < NS; ++c) v[c] = q[f][ky * NS + c];
                xrow_rmw<NS, A, true>(s2 + f * W + base + ky * W0, v, lxw, tseg);
            }
    }
    vmax = warp_max(vmax);
    if (lane == 0) atomic_max_nonneg(&clk->vmax_bits, (double)vmax);
    if (err) atomicOr(&clk->err, ERR_TILE);
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        int idx[3];
        const int64_t node = slot_node<P>(G, so, i, idx);
        if (node < 0) continue;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const A v = s2[a * W + i];
            if (v != A(0)) Acc<A>::add(gr.mv2[a] + node, v);
        }
    }
}

template <int P, class R, class A>
__global__ void __launch_bounds__(kG2PSpan2dThreads, 4) k_grid_g2p_span2d(Geom G, TileState<R> ts, Grid<A, R> gr,
                                                                          Clock* clk)
{
    const int t = blockIdx.x;
    grid_g2p_span2d_tile<P, R, A>(G, ts.pt, gr, ts.tpar[t] ? ts.cs[1] : ts.cs[0], clk, t);
}

// ----------------------------------------- K2: grid update + G2P + P2G
//
// One warp per velocity component d.  The tile's particles are staged row
// chunk by row chunk (32 spans, at most kCap particles) into shared memory by
// bulk copies, kStages deep.  A lane owns one span of the row and keeps the
// values of f_d/m (after the grid BC) at the span's (p+1)^d support nodes in
// registers; for each of its particles it gathers A_d = G2P(f_d/m), forms
// V'_d = V_d + dt A_d, writes it back into the stage and sums M V'_d phi into
// registers.  A completed row's sums go into the warp's own window of mv2_d
// with plain shared-memory adds.  After each chunk the block copies the
// chunk's V' to global memory (coalesced) and takes the largest |V'|.
template <int D>
struct K2Cfg {
    static constexpr int kThreads = 32 * D;
    static constexpr int kFields = 2 * D + 1;      // x[D], v[D], M
    static constexpr int kCap = 256;               // particles per chunk
    static constexpr int kPitch = kCap + 8;        // staged floats per field (16-byte multiple)
    static constexpr int kStages = 2;
    static constexpr int kStageFloats = kStages * kFields * kPitch;
    static constexpr int kHeadFloats = kStageFloats + 8;   // + the stages' mbarriers (32 bytes)
};

// Tile cell starts kept in shared memory (Tvol + 1 words, rounded to 4).
__host__ __device__ inline int tile_cs_words(const Geom& G) { return (G.Tvol + 1 + 3) & ~3; }

// Chunk [lo, hi) of row r of a tile (which ends at re).
struct RowChunk {
    int r;
    uint32_t lo, hi, re;
    bool valid;
};

__device__ __forceinline__ RowChunk next_chunk(const uint32_t* tcs, int nrows, RowChunk c, int cap)
{
    if (c.valid && c.hi < c.re) {
        c.lo = c.hi;
        c.hi = min(c.re, c.lo + (uint32_t)cap);
        return c;
    }
    for (int r = c.r + 1; r < nrows; ++r) {
        const uint32_t rb = tcs[r << 5], re = tcs[(r << 5) + 32];
        if (rb < re) return RowChunk{r, rb, min(re, rb + (uint32_t)cap), re, true};
    }
    return RowChunk{nrows, 0u, 0u, 0u, false};
}

// Copies of one chunk of fields x[D], v[D], M, widened to 16-byte boundaries
// (particle arrays are allocated in multiples of 256 bytes, so the widened
// end stays inside them).
template <int D>
__device__ __forceinline__ void k2_stage(const RowChunk& c, const Particles<float>& pt, float* stage, uint64_t* bar)
{
    typedef K2Cfg<D> C;
    const uint32_t a = c.lo & ~3u, b = (c.hi + 3u) & ~3u;
    const uint32_t bytes = (b - a) * 4u;
    mbar_arrive_expect_tx(bar, bytes * C::kFields);
#pragma unroll
    for (int f = 0; f < C::kFields; ++f) {
        const float* src = f < D ? pt.x[f] : (f < 2 * D ? pt.v[f - D] : pt.M);
        bulk_g2s(stage + f * C::kPitch, src + a, bytes, bar);
    }
}

// TX, TY, TZ > 0 (3D): the tile edges as compile-time constants.
template <int D, int P, bool PER, int TX = 0, int TY = 0, int TZ = 0>
__device__ __forceinline__ void grid_g2p_span_tile(const Geom& G, const Particles<float>& pt,
                                                   const Grid<float, float>& gr, const FieldPtrs& out,
                                                   const uint32_t* __restrict__ cs, Clock* clk, const int tile)
{
    typedef K2Cfg<D> C;
    constexpr bool ST = TX > 0;
    static_assert(!ST || D == 3, "static tiles: 3D");
    const int Tvol = ST ? TX * TY * TZ : G.Tvol;
    const int64_t kb = tile_cs0(G, tile);
    // compile-time tiles read the run state and the tile's particle range
    // while their window copies fly, and return (uniformly) after those
    const int active = clk->active;
    const uint32_t pb = cs[kb], pe = cs[kb + Tvol];
    if (!ST && (!active || pb == pe)) return;
    extern __shared__ __align__(16) float sm[];
    constexpr int NS = P + 1, NYZ = (D == 3) ? NS * NS : NS;
    const int W = ST ? (TX + P) * (TY + P) * (TZ + P) : G.Wvol;
    const int W0 = ST ? TX + P : G.W[0], W1 = ST ? TY + P : G.W[1];
    const int T0 = ST ? TX : G.T[0], T1 = ST ? TY : G.T[1];
    const int sh0 = ST ? clog2(TX) : G.tsh[0], sh1 = ST ? clog2(TY) : G.tsh[1];
    float* stage = sm;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + C::kStageFloats);
    uint32_t* tcs = reinterpret_cast<uint32_t*>(sm + C::kHeadFloats);
    float* sA = sm + C::kHeadFloats + ((Tvol + 1 + 3) & ~3);  // D x W: f/m after BC
    float* s2 = sA + D * W;                                  // D x W: momentum P2G
    int so[3];
    tile_origin(G, tile, so);
    const float dt = (float)clk->dt_cur;
    const bool bc = window_has_bc(G, gr.mask, so);
    if constexpr (ST) {
        // compile-time tiles: the window's m (into the first field of s2) and
        // f (into sA) and the span starts arrive by asynchronous copies, all
        // of a thread's in flight at once; then each thread applies the BC to
        // its own nodes and forms f/m in place.  The loops stay rolled: the
        // copies overlap without unrolling, and the unrolled prologue cost
        // the kernel instruction-cache misses (256^3 blast: 3.10 against
        // 3.02 ms)
        constexpr int WS = (TX + P) * (TY + P) * (TZ + P), NT = C::kThreads, NI = (WS + NT - 1) / NT;
#pragma unroll 1
        for (int q = 0; q < NI; ++q) {
            const int i = (int)threadIdx.x + q * NT;
            if (i < WS) {
                int idx[3];
                const int64_t node = slot_node<P, TX, TY>(G, so, i, idx);
                if (node >= 0) {
                    cp_async4(s2 + i, gr.m + node);
#pragma unroll
                    for (int a = 0; a < D; ++a) cp_async4(sA + a * W + i, gr.f[a] + node);
                } else {
                    s2[i] = 0.f;
#pragma unroll
                    for (int a = 0; a < D; ++a) sA[a * W + i] = 0.f;
                }
            }
        }
        for (int i = threadIdx.x; i <= Tvol; i += blockDim.x) cp_async4(tcs + i, cs + kb + i);
        cp_async_wait_all();
        if (!active || pb == pe) return;
#pragma unroll 1
        for (int q = 0; q < NI; ++q) {
            const int i = (int)threadIdx.x + q * NT;
            if (i < WS) {
                float f[3] = {0.f, 0.f, 0.f}, m = s2[i];
#pragma unroll
                for (int a = 0; a < D; ++a) f[a] = sA[a * W + i];
                if (bc) {
                    int idx[3];
                    const int64_t node = slot_node<P, TX, TY>(G, so, i, idx);
                    if (node >= 0) node_bc<float, D>(G, gr.mask, gr.nrm, node, idx, m, f, 1);
                }
                const float im = m != 0.f ? __frcp_rn(m) : 0.f;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    sA[a * W + i] = f[a] * im;
                    s2[a * W + i] = 0.f;
                }
            }
        }
    } else {
        for (int i = threadIdx.x; i < W; i += blockDim.x) {
            int idx[3];
            const int64_t node = slot_node<P, TX, TY>(G, so, i, idx);
            float f[3] = {0.f, 0.f, 0.f}, m = 0.f;
            if (node >= 0) {
                m = gr.m[node];
#pragma unroll
                for (int a = 0; a < D; ++a) f[a] = gr.f[a][node];
                if (bc) node_bc<float, D>(G, gr.mask, gr.nrm, node, idx, m, f, 1);
            }
            const float im = m != 0.f ? __frcp_rn(m) : 0.f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                sA[a * W + i] = f[a] * im;
                s2[a * W + i] = 0.f;
            }
        }
        for (int i = threadIdx.x; i <= Tvol; i += blockDim.x) tcs[i] = cs[kb + i];
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < C::kStages; ++q) mbar_init(bar + q, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nrows = Tvol >> 5;
    const bool producer = threadIdx.x == 0;
    const float ih = (float)G.inv_h;
    float lo[3], nper[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = (float)G.lo[a];
        nper[a] = G.per[a] ? (float)G.n[a] : 3.0e38f;
    }
    RowChunk c = next_chunk(tcs, nrows, RowChunk{-1, 0u, 0u, 0u, false}, C::kCap);
    RowChunk pc = c;
    int issued = 0;
    if (producer) {
        for (int q = 0; q < C::kStages && pc.valid; ++q) {
            k2_stage<D>(pc, pt, stage + q * C::kFields * C::kPitch, bar + q);
            pc = next_chunk(tcs, nrows, pc, C::kCap);
            ++issued;
        }
    }
    const float* sAd = sA + warp * W;
    float* s2d = s2 + warp * W;
    // f_d/m and the M V'_d sums of the span's nodes, node rows jj (y, z)
    // paired for packed FMAs: rows 2q and 2q+1 in AwP[q][a] / accP[q][a],
    // the last row of an odd count (quadratic basis) in AwT / accT
    constexpr int NP = NYZ / 2;
    constexpr bool ODD = (NYZ & 1) != 0;
    float2 AwP[NP][NS], accP[NP][NS];
    float AwT[NS], accT[NS];
    uint32_t sb = 0, se = 0;
    int base = 0;
    float cb[3] = {0.f, 0.f, 0.f};
    float vmax = 0.f;
    int fail = 0, i = 0;
    for (; c.valid; ++i) {
        const int st = i % C::kStages;
        if (!mbar_wait(bar + st, (uint32_t)(i / C::kStages) & 1u)) fail = 1;
        float* sg = stage + st * C::kFields * C::kPitch;
        const uint32_t a0 = c.lo & ~3u;
        if (c.lo == tcs[c.r << 5]) {
            // a new row: the lane's span, its f_d/m values, zero sums
            const int s = (c.r << 5) + lane;
            sb = tcs[s];
            se = tcs[s + 1];
            const int lx = s & (T0 - 1);
            const int ly = (s >> sh0) & (T1 - 1);
            const int lz = s >> (sh0 + sh1);
            base = (lz * W1 + ly) * W0 + lx;
            cb[0] = (float)(so[0] + lx - (P == 2 ? 1 : 0));
            cb[1] = (float)(so[1] + ly - (P == 2 ? 1 : 0));
            cb[2] = (float)(so[2] + lz - (P == 2 ? 1 : 0));
#pragma unroll
            for (int jj = 0; jj < NYZ; ++jj) {
                const int row = base + ((D == 3 ? jj / NS : 0) * W1 + (D == 3 ? jj % NS : jj)) * W0;
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    const float v = sAd[row + a];
                    if (ODD && jj == NYZ - 1) { AwT[a] = v; accT[a] = 0.f; }
                    else if (jj & 1) { AwP[jj >> 1][a].y = v; accP[jj >> 1][a].y = 0.f; }
                    else { AwP[jj >> 1][a].x = v; accP[jj >> 1][a].x = 0.f; }
                }
            }
        }
        const uint32_t kb0 = max(sb, c.lo), kb1 = min(se, c.hi);
        const uint32_t cnt = kb1 > kb0 ? kb1 - kb0 : 0u;
        // lanes start at different particles of their spans: with 8 particles
        // a span, the 32 lanes then read 32 different banks
        uint32_t rot = cnt ? (uint32_t)lane >> 2 : 0u;     // (lane / 4) mod cnt
        while (rot >= cnt && cnt) rot -= cnt;
        for (uint32_t ii = 0; ii < cnt; ++ii) {
            const uint32_t kk = ii + rot;
            const uint32_t j = kb0 - a0 + (kk >= cnt ? kk - cnt : kk);
            float w[3][3], dw[3][3];
#pragma unroll
            for (int a = 0; a < D; ++a) axis_known<P, PER>(sg[a * C::kPitch + j], lo[a], ih, cb[a], nper[a], w[a], dw[a]);
            float2 yzP[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const int j0 = 2 * q, j1 = 2 * q + 1;
                yzP[q] = D == 3 ? f2(w[1][j0 % NS] * w[2][j0 / NS], w[1][j1 % NS] * w[2][j1 / NS])
                                : f2(w[1][j0], w[1][j1]);
            }
            const float yzT = !ODD ? 0.f : D == 3 ? w[1][NS - 1] * w[2][NS - 1] : w[1][NYZ - 1];
            // A_d = sum over the support of phi f_d/m, x first
            float2 AP = f2(0.f, 0.f);
            float tT = 0.f;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float2 t = f2(0.f, 0.f);
#pragma unroll
                for (int a = 0; a < NS; ++a) t = __ffma2_rn(f2(w[0][a], w[0][a]), AwP[q][a], t);
                AP = __ffma2_rn(yzP[q], t, AP);
            }
            if (ODD) {
#pragma unroll
                for (int a = 0; a < NS; ++a) tT = fmaf(w[0][a], AwT[a], tT);
            }
            const float A = ODD ? fmaf(yzT, tT, AP.x + AP.y) : AP.x + AP.y;
            float* vp = sg + (D + warp) * C::kPitch + j;
            const float vn = fmaf(dt, A, *vp);
            *vp = vn;
            const float mv = sg[2 * D * C::kPitch + j] * vn;
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                const float cm = mv * w[0][a];
#pragma unroll
                for (int q = 0; q < NP; ++q) accP[q][a] = __ffma2_rn(f2(cm, cm), yzP[q], accP[q][a]);
                if (ODD) accT[a] = fmaf(cm, yzT, accT[a]);
            }
        }
        if (c.hi == c.re) {
            // the row is complete: node (lx + a, ly + bb) of each window layer
            // gets acc of span (lx, ly), in NS x NS phases (a, bb).  A row of
            // 32 spans may cover several y-rows of the tile, and lanes
            // (lx, ly) and (lx, ly + 1) add to the same node in phases (a, 1)
            // and (a, 0): the warp barrier between phases orders them
#pragma unroll
            for (int a = 0; a < NS; ++a) {
#pragma unroll
                for (int bb = 0; bb < (D == 3 ? NS : NYZ); ++bb) {
                    __syncwarp();
#pragma unroll
                    for (int c = 0; c < (D == 3 ? NS : 1); ++c) {
                        const int jj = D == 3 ? c * NS + bb : bb;
                        s2d[base + (c * W1 + bb) * W0 + a] +=
                            (ODD && jj == NYZ - 1) ? accT[a] : ((jj & 1) ? accP[jj >> 1][a].y : accP[jj >> 1][a].x);
                    }
                }
            }
            __syncwarp();
        }
        // V' of the chunk is complete in the stage; order the generic
        // accesses to the stages before later bulk copies into them
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (block_bar_or(fail)) { fail = 1; break; }
        // the previous chunk's stage is free (every thread passed its
        // write-back before this barrier): refill it
        if (producer && i >= 1 && pc.valid) {
            const int q = (i - 1) % C::kStages;
            k2_stage<D>(pc, pt, stage + q * C::kFields * C::kPitch, bar + q);
            pc = next_chunk(tcs, nrows, pc, C::kCap);
            ++issued;
        }
        // write the chunk's V' back, coalesced
        for (uint32_t k = c.lo + threadIdx.x; k < c.hi; k += blockDim.x) {
            const uint32_t j = k - a0;
            float v2 = 0.f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float vn = sg[(D + a) * C::kPitch + j];
                pt.v[a][k] = vn;
                v2 = fmaf(vn, vn, v2);
            }
            vmax = fmaxf(vmax, v2);
        }
        c = next_chunk(tcs, nrows, c, C::kCap);
    }
    if (fail && producer) {
        // drain the copies still in flight before the block's memory is reused
        for (int q = i; q < issued; ++q) mbar_wait(bar + (q % C::kStages), (uint32_t)(q / C::kStages) & 1u);
    }
    vmax = warp_max(vmax);
    if (lane == 0) atomic_max_nonneg(&clk->vmax_bits, (double)sqrtf(vmax));
    if (fail) atomicOr(&clk->err, ERR_TIMEOUT);
    __syncthreads();
    if (fail) return;
    flush_window<D, P, TX, TY, TZ>(G, so, s2, D, out);
}

template <int D, int P, bool PER, int TX = 0, int TY = 0, int TZ = 0>
__global__ void __launch_bounds__(K2Cfg<D>::kThreads, 5) k_grid_g2p_span(Geom G, TileState<float> ts,
                                                                         Grid<float, float> gr, FieldPtrs out,
                                                                         Clock* clk,
                                                                         const uint32_t* __restrict__ tiles)
{
    const int t = tiles ? (int)tiles[blockIdx.x] : (int)blockIdx.x;
    grid_g2p_span_tile<D, P, PER, TX, TY, TZ>(G, ts.pt, gr, out, ts.tpar[t] ? ts.cs[1] : ts.cs[0], clk, t);
}

// ------------------------------- K3: G2PD + particle update + move + key

constexpr int kG2PDThreads = 128;
// resident blocks: in 3D four, 128 registers a thread (five blocks at 96
// registers spill in the particle loop: 3.41 against 3.32 ms on the 256^3
// blast), five for the compile-time tiles, whose constant window offsets fit
// 96 registers (2.97 against 3.10 ms); in 2D five (93 registers, no spills)
template <int D, bool ST = false>
constexpr int g2pd_blocks() { return D == 3 && !ST ? 4 : 5; }

// A: grid accumulator type (float, or int64 fixed point read back as float).
// TX, TY, TZ > 0 (3D): the tile edges as compile-time constants.
// WALLS: every face is a wall (no periodic axis, no outflow, no inflow), so
// the periodic wrap and the outflow / recycling paths drop out.
template <int D, int P, class A, int TX = 0, int TY = 0, int TZ = 0, bool WALLS = false>
__device__ __forceinline__ void g2pd_fast_tile(const Geom& G, const Particles<float>& pt, const Grid<A, float>& gr,
                                               const uint32_t* __restrict__ cs, Clock* clk, const Reorder& ro,
                                               const int tile)
{
    constexpr bool ST = TX > 0;
    static_assert(!ST || D == 3, "static tiles: 3D");
    // compile-time tiles read the run state and the tile's particle range
    // while their window loads fly, and return (uniformly) after those
    const int active = clk->active;
    const uint32_t beg = cs[tile_cs0(G, tile)];
    const uint32_t end = cs[tile_cs0(G, tile) + (ST ? TX * TY * TZ : G.Tvol)];
    if (!ST && (!active || beg == end)) return;
    // per node: 3D {Vb_x, Vb_y, Vb_z, V2_y} + {V2_x, V2_z}; 2D {Vb_x, Vb_y, V2_x, V2_y}
    extern __shared__ __align__(16) float4 sn[];
    constexpr int NS = P + 1;
    const int W = ST ? (TX + P) * (TY + P) * (TZ + P) : G.Wvol;
    const int W0 = ST ? TX + P : G.W[0], W1 = ST ? TY + P : G.W[1];
    const int Ta[3] = {ST ? TX : G.T[0], ST ? TY : G.T[1], ST ? TZ : G.T[2]};
    const int sh0 = ST ? clog2(TX) : G.tsh[0], sh1 = ST ? clog2(TY) : G.tsh[1], sh2 = ST ? clog2(TZ) : G.tsh[2];
    int so[3];
    tile_origin(G, tile, so);
    const float dt = (float)clk->dt_cur;
    const bool bc = window_has_bc(G, gr.mask, so);
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        int idx[3];
        const int64_t node = slot_node<P, TX, TY>(G, so, i, idx);
        float mv[3] = {0.f, 0.f, 0.f}, f[3] = {0.f, 0.f, 0.f}, m2[3] = {0.f, 0.f, 0.f}, m = 0.f;
        if (node >= 0) {
            m = Acc<A>::to_real(gr.m[node], G.dqscale[0]);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                mv[a] = Acc<A>::to_real(gr.mv[a][node], G.dqscale[1]);
                f[a] = Acc<A>::to_real(gr.f[a][node], G.dqscale[2]);
                m2[a] = Acc<A>::to_real(gr.mv2[a][node], G.dqscale[1]);
            }
            if (bc) {
                node_bc<float, D>(G, gr.mask, gr.nrm, node, idx, m, mv, 0);
                node_bc<float, D>(G, gr.mask, gr.nrm, node, idx, m, f, 1);
                node_bc<float, D>(G, gr.mask, gr.nrm, node, idx, m, m2, 0);
            }
        }
        const float im = m != 0.f ? __frcp_rn(m) : 0.f;
        float vb[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) vb[a] = fmaf(dt, f[a], mv[a]) * im;
        if (D == 3) {
            sn[i] = make_float4(vb[0], vb[1], vb[2], m2[1] * im);
            reinterpret_cast<float2*>(sn + W)[i] = make_float2(m2[0] * im, m2[2] * im);
        } else {
            sn[i] = make_float4(vb[0], vb[1], m2[0] * im, m2[1] * im);
        }
    }
    if (ST && (!active || beg == end)) return;
    __syncthreads();
    const float gm1 = (float)(G.gamma - 1.0), gam = (float)G.gamma, ih = (float)G.inv_h, hh = (float)G.h;
    const float c0 = (float)G.c0, c1 = (float)G.c1;
    // squares of the largest speeds; sqrt is monotonic and correctly rounded,
    // so the root of the largest square is the largest root
    float vmax2 = 0.f, cmax2 = 0.f;
    int err = 0;
    // the next particle's state is loaded while this one is processed
    float px[3] = {0.f, 0.f, 0.f}, prho = 0.f, pE = 0.f, pQ = 0.f;
    if (beg + threadIdx.x < end) {
        const uint32_t k0 = beg + threadIdx.x;
#pragma unroll
        for (int a = 0; a < D; ++a) px[a] = pt.x[a][k0];
        prho = pt.rho[k0];
        pE = pt.E[k0];
        pQ = pt.Q[k0];
    }
    for (uint32_t k = beg + threadIdx.x; k < end; k += blockDim.x) {
        float x[3], w[3][3], dw[3][3];
        int l[3] = {0, 0, 0}, csp[3] = {0, 0, 0};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) x[a] = px[a];
        const float rho = prho, E = pE, Q = pQ;
        if (k + blockDim.x < end) {
            const uint32_t kn = k + blockDim.x;
#pragma unroll
            for (int a = 0; a < D; ++a) px[a] = pt.x[a][kn];
            prho = pt.rho[kn];
            pE = pt.E[kn];
            pQ = pt.Q[kn];
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            float xi;
            const int c = span_of<float, P, WALLS>(G, a, x[a], xi);
            csp[a] = c;
            weights1d<P>(__fsub_rn(xi, (float)(c - (P == 2 ? 1 : 0))), w[a], dw[a]);
            l[a] = wrap_span<WALLS>(G, a, c) - so[a];
            ok = ok && l[a] >= 0 && l[a] < Ta[a];
        }
        if (!ok) { err |= ERR_TILE; continue; }
        const int base = (l[2] * W1 + l[1]) * W0 + l[0];
        // the particle's old key (its span in this tile)
        const uint32_t okey = ((uint32_t)tile << (sh0 + sh1 + sh2)) |
                              (uint32_t)((((l[2] << sh1) + l[1]) << sh0) | l[0]);
        // Vbar = G2P(mv'/m); div V = trace of G2PD(mv2/m), summed x first,
        // then y, then z, two sums per packed FMA
        const float2* sn2 = reinterpret_cast<const float2*>(sn + W);
        float2 wx[NS], wxd[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            wx[a] = f2(w[0][a], w[0][a]);
            wxd[a] = f2(dw[0][a], w[0][a]);
        }
        // 3D: V01 = {Vb_x, Vb_y}, V2g = {Vb_z, grad_y}, Gxz = {grad_x, grad_z}
        // 2D: V01 = {Vb_x, Vb_y}, Gxz = {grad_x, grad_y}
        float2 V01 = f2(0.f, 0.f), V2g = f2(0.f, 0.f), Gxz = f2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < (D == 3 ? NS : 1); ++c) {
            float2 p01 = f2(0.f, 0.f), p2g = f2(0.f, 0.f), pxz = f2(0.f, 0.f);
#pragma unroll
            for (int bb = 0; bb < NS; ++bb) {
                const int row = base + (c * W1 + bb) * W0;
                float2 r01 = f2(0.f, 0.f), r2g = f2(0.f, 0.f), gxz = f2(0.f, 0.f);
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    const float4 q = sn[row + a];
                    r01 = __ffma2_rn(wx[a], f2(q.x, q.y), r01);
                    if (D == 3) {
                        const float2 q2 = sn2[row + a];
                        r2g = __ffma2_rn(wx[a], f2(q.z, q.w), r2g);
                        gxz = __ffma2_rn(wxd[a], q2, gxz);
                    } else {
                        gxz = __ffma2_rn(wxd[a], f2(q.z, q.w), gxz);
                    }
                }
                const float wy = w[1][bb], dwy = dw[1][bb];
                p01 = __ffma2_rn(f2(wy, wy), r01, p01);
                if (D == 3) {
                    p2g = __ffma2_rn(f2(wy, dwy), r2g, p2g);
                    pxz = __ffma2_rn(f2(wy, wy), gxz, pxz);
                } else {
                    pxz = __ffma2_rn(f2(wy, dwy), gxz, pxz);
                }
            }
            if (D == 3) {
                const float wz = w[2][c], dwz = dw[2][c];
                V01 = __ffma2_rn(f2(wz, wz), p01, V01);
                V2g = __ffma2_rn(f2(wz, wz), p2g, V2g);
                Gxz = __ffma2_rn(f2(wz, dwz), pxz, Gxz);
            } else {
                V01 = p01;
                Gxz = pxz;
            }
        }
        const float vb[3] = {V01.x, V01.y, D == 3 ? V2g.x : 0.f};
        const float dx = Gxz.x, dy = D == 3 ? V2g.y : Gxz.y, dz = D == 3 ? Gxz.y : 0.f;
        const float dv = (dx + dy + (D == 3 ? dz : 0.f)) * ih;
        // Sec. 3 step viii: energy, density, pressure, artificial viscosity
        const float irho = __frcp_rn(rho);
        const float Pk = gm1 * rho * E;
        const float En = E - dt * (Pk + Q) * irho * dv;
        const float den = 1.0f + dt * dv;
        if (!(den > 0.f)) { err |= ERR_NONFINITE; continue; }
        const float rn = __fdividef(rho, den);
        const float Pn = gm1 * rn * En;
        const float c2 = gam * gm1 * En;       // gamma P / rho with P = (gamma - 1) rho e
        const float c2p = c2 > 0.f ? c2 : 0.f;
        float Qn = 0.f;
        if (dv < 0.f) {
            // eq. muart: von Neumann-Richtmyer and Landshoff terms, both
            // proportional to the density
            const float cs = sqrtf(c2p);
            const float t1 = hh * dv;
            Qn = rn * (c0 * t1 * t1 - c1 * hh * cs * dv);
        }
        (void)Pn;
        // step ix: move with Vbar; step x: wrap / hold / recycle; new key
        float xn[3] = {0.f, 0.f, 0.f}, vb2 = 0.f;
        int cn[3] = {0, 0, 0};
        bool out = false;
        // x - x is 0 for a finite x and NaN otherwise
        float fz = __fadd_rn(__fadd_rn(__fsub_rn(En, En), __fsub_rn(rn, rn)), __fsub_rn(Qn, Qn));
#pragma unroll
        for (int a = 0; a < D; ++a) {
            xn[a] = __fadd_rn(x[a], __fmul_rn(dt, vb[a]));
            vb2 = fmaf(vb[a], vb[a], vb2);
            fz = __fadd_rn(fz, __fsub_rn(xn[a], xn[a]));
            float xi;
            cn[a] = span_of<float, P, WALLS>(G, a, xn[a], xi);
            if ((unsigned)(cn[a] - csp[a] + 1) > 2u) err |= ERR_CFL;    // more than one span
            if (!WALLS && !G.per[a]) {
                if (xn[a] < (float)G.lo[a] && G.bc[2 * a] == 3) out = true;
                if (xn[a] >= (float)G.hi[a] && G.bc[2 * a + 1] == 3) out = true;
            }
        }
        if (!(fz == 0.f)) { err |= ERR_NONFINITE; continue; }
        float En_s = En, rn_s = rn, Qn_s = Qn, cpart2 = c2p;
        int sp[3] = {0, 0, 0};
        if (!WALLS && out && G.inflow_face >= 0) {
            const uint32_t gk = pt.gen[k];
            uint32_t c[4] = {gk, 0u, pt.id[k], 0u};
            philox4x32_10(c, (uint32_t)G.seed, (uint32_t)(G.seed >> 32));
            pt.gen[k] = gk + 1u;
            const int af = G.inflow_face / 2, side = G.inflow_face % 2;
            float vin2 = 0.f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float u = __fmul_rn((float)(c[a] >> 8), 1.0f / 16777216.0f);
                if (a == af)
                    xn[a] = side == 0 ? __fadd_rn((float)G.lo[a], __fmul_rn(u, hh))
                                      : __fadd_rn(__fsub_rn((float)G.hi[a], hh), __fmul_rn(u, hh));
                else
                    xn[a] = __fadd_rn((float)G.lo[a], __fmul_rn(u, __fsub_rn((float)G.hi[a], (float)G.lo[a])));
                const float vi = (float)G.inflow_v[a];
                pt.v[a][k] = vi;
                vin2 = fmaf(vi, vi, vin2);
                float xi;
                sp[a] = wrap_span(G, a, span_of<float, P>(G, a, xn[a], xi));
            }
            En_s = (float)G.inflow_e;
            rn_s = (float)G.inflow_rho;
            Qn_s = 0.f;
            const float ci2 = gam * gm1 * En_s;
            cpart2 = ci2 > 0.f ? ci2 : 0.f;
            vmax2 = fmaxf(vmax2, vin2);
        } else {
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float lo = (float)G.lo[a], hi = (float)G.hi[a];
                if (!WALLS && G.per[a]) {
                    const float L = __fsub_rn(hi, lo);
                    if (xn[a] < lo) xn[a] = __fadd_rn(xn[a], L);
                    else if (xn[a] >= hi) xn[a] = __fsub_rn(xn[a], L);
                    float xi;
                    sp[a] = wrap_span(G, a, span_of<float, P>(G, a, xn[a], xi));
                } else {
                    // holding the particle at a face keeps its (clamped) span
                    xn[a] = fminf(fmaxf(xn[a], lo), hi);
                    sp[a] = cn[a];
                }
            }
        }
#pragma unroll
        for (int a = 0; a < D; ++a) pt.x[a][k] = xn[a];
        pt.key[k] = record_key(G, ro, clk, key_of<float>(G, sp), !WALLS && out && G.inflow_face >= 0, (uint32_t)k,
                               tile, okey, err);
        pt.E[k] = En_s;
        pt.rho[k] = rn_s;
        pt.Q[k] = Qn_s;
        vmax2 = fmaxf(vmax2, vb2);
        cmax2 = fmaxf(cmax2, cpart2);
    }
    const float vmax = sqrtf(warp_max(vmax2));
    const float cmax = sqrtf(warp_max(cmax2));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) err |= __shfl_xor_sync(0xffffffffu, err, o);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&clk->vmax_bits, (double)vmax);
        atomic_max_nonneg(&clk->cmax_bits, (double)cmax);
        if (err) atomicOr(&clk->err, err);
    }
}

template <int D, int P, class A, int TX = 0, int TY = 0, int TZ = 0, bool WALLS = false>
__global__ void __launch_bounds__(kG2PDThreads, g2pd_blocks<D, (TX > 0)>()) k_g2pd_fast(Geom G, TileState<float> ts,
                                                                         Grid<A, float> gr, Clock* clk, Reorder ro)
{
    const int t = blockIdx.x;
    g2pd_fast_tile<D, P, A, TX, TY, TZ, WALLS>(G, ts.pt, gr, ts.tpar[t] ? ts.cs[1] : ts.cs[0], clk, ro, t);
}

// Whether every face of the domain is a wall (the WALLS kernels apply).
__host__ __device__ inline bool all_walls(const Geom& G)
{
    for (int a = 0; a < G.dim; ++a)
        if (G.per[a] || G.bc[2 * a] != 0 || G.bc[2 * a + 1] != 0) return false;
    return G.inflow_face < 0;
}

}  // namespace mpm
