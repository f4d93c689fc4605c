// mpm_obstacle.cu -- mpm_set_obstacle_profile: the obstacle of a 2D problem
// from closed loops of boundary points (the aerofoil case of Sec. 4.1, where
// the profile is read from a point file).
//
// Per stored node, on the GPU in binary64: the signed distance to the union of
// the loops' edges (Eq. sdf; negative inside by the even-odd rule), the
// nearest boundary point, then the obstacle cells (a corner with sd <= 0),
// their corner nodes as the mask, and n = grad sd on the masked nodes (the
// normals of eqs. normali1/normali2).  Every operation is a separately
// rounded IEEE operation, so a node's distance and every inside / obstacle
// decision are those of the plain evaluation of the definition.
//
// Compiled into the same translation unit as mpm_api.cu (included at its end).

namespace mpm {

constexpr int kSdfThreads = 256;

struct ProfileEdges {
    const double* ax;
    const double* ay;
    const double* bx;
    const double* by;
    int64_t n;
};

// Node (i, j) of the stored grid at lo + (index - g) h per axis.
__device__ __forceinline__ double node_coord(const Geom& G, int a, int64_t i)
{
    return __dadd_rn(G.lo[a], __dmul_rn((double)(i - G.g[a]), G.h));
}

__global__ void __launch_bounds__(kSdfThreads) k_profile_sd(Geom G, ProfileEdges E, double* __restrict__ sd,
                                                            double* __restrict__ qx, double* __restrict__ qy)
{
    __shared__ double s_e[4][kSdfThreads];
    const int64_t nn = (int64_t)G.N[0] * G.N[1];
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = node < nn;
    const double X = live ? node_coord(G, 0, node % G.N[0]) : 0.0;
    const double Y = live ? node_coord(G, 1, node / G.N[0]) : 0.0;
    double best = __longlong_as_double(0x7ff0000000000000ll);   // +infinity
    double bx_ = X, by_ = Y;
    int inside = 0;
    for (int64_t base = 0; base < E.n; base += kSdfThreads) {
        __syncthreads();
        const int64_t k = base + threadIdx.x;
        if (k < E.n) {
            s_e[0][threadIdx.x] = E.ax[k];
            s_e[1][threadIdx.x] = E.ay[k];
            s_e[2][threadIdx.x] = E.bx[k];
            s_e[3][threadIdx.x] = E.by[k];
        }
        __syncthreads();
        const int cnt = E.n - base < kSdfThreads ? (int)(E.n - base) : kSdfThreads;
        for (int c = 0; c < cnt; ++c) {
            const double ax = s_e[0][c], ay = s_e[1][c], bx = s_e[2][c], by = s_e[3][c];
            const double ex = __dsub_rn(bx, ax), ey = __dsub_rn(by, ay);
            const double wx = __dsub_rn(X, ax), wy = __dsub_rn(Y, ay);
            // nearest point of the edge: a + t (b - a), t clamped to [0, 1]
            const double L2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
            double t = L2 > 0.0 ? __ddiv_rn(__dadd_rn(__dmul_rn(wx, ex), __dmul_rn(wy, ey)), L2) : 0.0;
            t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
            const double cx = __dadd_rn(ax, __dmul_rn(t, ex)), cy = __dadd_rn(ay, __dmul_rn(t, ey));
            const double dx = __dsub_rn(X, cx), dy = __dsub_rn(Y, cy);
            const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            if (d2 < best) {     // the first edge wins ties
                best = d2;
                bx_ = cx;
                by_ = cy;
            }
            // crossing of the ray y = Y, x > X with this edge
            if ((ay > Y) != (by > Y)) {
                const double xc = __dadd_rn(ax, __ddiv_rn(__dmul_rn(__dsub_rn(Y, ay), ex), ey));
                if (X < xc) inside ^= 1;
            }
        }
    }
    if (!live) return;
    const double d = __dsqrt_rn(best);
    sd[node] = inside ? -d : d;
    qx[node] = bx_;
    qy[node] = by_;
}

// Mask = corner nodes of the cells with a corner at sd <= 0; normals = grad sd
// = (X - Q)/|X - Q| outside, (Q - X)/|X - Q| inside, on masked nodes only.
__global__ void __launch_bounds__(kSdfThreads) k_profile_mask(Geom G, const double* __restrict__ sd,
                                                              const double* __restrict__ qx,
                                                              const double* __restrict__ qy, uint8_t* __restrict__ mask,
                                                              double* __restrict__ nrm)
{
    const int64_t nn = (int64_t)G.N[0] * G.N[1];
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nn) return;
    const int64_t ix = node % G.N[0], iy = node / G.N[0];
    // physical node index along each axis; the cells that have it as a corner
    const int64_t p0 = ix - G.g[0], p1 = iy - G.g[1];
    bool m = false;
    for (int oy = -1; oy <= 0 && !m; ++oy)
        for (int ox = -1; ox <= 0 && !m; ++ox) {
            int64_t cx = p0 + ox, cy = p1 + oy;
            if (G.per[0]) cx = ((cx % G.n[0]) + G.n[0]) % G.n[0];
            else if (cx < 0 || cx >= G.n[0]) continue;
            if (G.per[1]) cy = ((cy % G.n[1]) + G.n[1]) % G.n[1];
            else if (cy < 0 || cy >= G.n[1]) continue;
            for (int c = 0; c < 4; ++c) {
                int64_t jx = cx + (c & 1), jy = cy + (c >> 1);
                jx = G.per[0] ? jx % G.n[0] : jx + G.g[0];
                jy = G.per[1] ? jy % G.n[1] : jy + G.g[1];
                if (sd[jy * G.N[0] + jx] <= 0.0) m = true;
            }
        }
    double nx = 0.0, ny = 0.0;
    const double d = fabs(sd[node]);
    if (m && d > 0.0) {
        const double X = node_coord(G, 0, ix), Y = node_coord(G, 1, iy);
        const double s = sd[node] < 0.0 ? -1.0 : 1.0;
        nx = __dmul_rn(s, __ddiv_rn(__dsub_rn(X, qx[node]), d));
        ny = __dmul_rn(s, __ddiv_rn(__dsub_rn(Y, qy[node]), d));
    }
    mask[node] = m ? 1 : 0;
    nrm[node] = nx;
    nrm[nn + node] = ny;
}

}  // namespace mpm

extern "C" mpm_status mpm_set_obstacle_profile(mpm_sim* s, int64_t nloops, const int64_t* loop_len,
                                               const double* pts, uint8_t* mask_out, double* normals_out,
                                               double* sd_out)
{
    using namespace mpm;
    if (!s) return fail(nullptr, MPM_EINVAL, "sim is NULL");
    if (s->batch) return fail(s, MPM_ESTATE, "the simulation is a member of a batch");
    if (s->poisoned) return fail(s, MPM_ESTATE, "simulation is poisoned: " + s->err);
    if (s->G.dim != 2) return fail(s, MPM_EUNSUPPORTED, "point-profile obstacles are two-dimensional");
    if (nloops < 1 || !loop_len || !pts) return fail(s, MPM_EINVAL, "no loops");
    int64_t np = 0;
    for (int64_t l = 0; l < nloops; ++l) {
        if (loop_len[l] < 3 || loop_len[l] > (int64_t)1 << 24) return fail(s, MPM_EINVAL, "a loop needs 3 to 2^24 points");
        np += loop_len[l];
        if (np > (int64_t)1 << 24) return fail(s, MPM_EINVAL, "more than 2^24 profile points");
    }
    for (int64_t k = 0; k < 2 * np; ++k)
        if (!std::isfinite(pts[k])) return fail(s, MPM_EINVAL, "non-finite profile point");
    // edges in loop order: vertex k to vertex k + 1, the last back to the first
    std::vector<double> e(4 * (size_t)np);
    int64_t base = 0;
    for (int64_t l = 0; l < nloops; ++l) {
        for (int64_t k = 0; k < loop_len[l]; ++k) {
            const int64_t a = base + k, b = base + (k + 1) % loop_len[l];
            e[a] = pts[a];
            e[np + a] = pts[np + a];
            e[2 * np + a] = pts[b];
            e[3 * np + a] = pts[np + b];
        }
        base += loop_len[l];
    }
    const Geom& G = s->G;
    const int64_t nn = G.nnode;
    double* de = (double*)dalloc(s, e.size() * sizeof(double));
    double* dsd = (double*)dalloc(s, (size_t)nn * 3 * sizeof(double));
    double* dn = (double*)dalloc(s, (size_t)nn * 2 * sizeof(double));
    uint8_t* dm = (uint8_t*)dalloc(s, (size_t)nn);
    mpm_status st = MPM_OK;
    std::vector<uint8_t> m((size_t)nn);
    std::vector<double> nv((size_t)nn * 2), sdv((size_t)nn);
    if (!de || !dsd || !dn || !dm) {
        st = fail(s, MPM_ENOMEM, "device allocation failed");
    } else {
        cudaStream_t stq = s->stream;
        const unsigned nb = (unsigned)((nn + kSdfThreads - 1) / kSdfThreads);
        const ProfileEdges E = {de, de + np, de + 2 * np, de + 3 * np, np};
        cudaError_t ce = cudaMemcpyAsync(de, e.data(), e.size() * sizeof(double), cudaMemcpyHostToDevice, stq);
        if (ce == cudaSuccess) {
            k_profile_sd<<<nb, kSdfThreads, 0, stq>>>(G, E, dsd, dsd + nn, dsd + 2 * nn);
            k_profile_mask<<<nb, kSdfThreads, 0, stq>>>(G, dsd, dsd + nn, dsd + 2 * nn, dm, dn);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(m.data(), dm, (size_t)nn, cudaMemcpyDeviceToHost, stq);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(nv.data(), dn, (size_t)nn * 2 * sizeof(double), cudaMemcpyDeviceToHost, stq);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(sdv.data(), dsd, (size_t)nn * sizeof(double), cudaMemcpyDeviceToHost, stq);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stq);
        if (ce != cudaSuccess) st = cuda_fail(s, ce, "obstacle profile");
    }
    dfree(s, de);
    dfree(s, dsd);
    dfree(s, dn);
    dfree(s, dm);
    if (st != MPM_OK) return st;
    st = set_obstacle(s, m.data(), nv.data());
    if (st != MPM_OK) return st;
    if (mask_out) memcpy(mask_out, m.data(), (size_t)nn);
    if (normals_out) memcpy(normals_out, nv.data(), (size_t)nn * 2 * sizeof(double));
    if (sd_out) memcpy(sd_out, sdv.data(), (size_t)nn * sizeof(double));
    return MPM_OK;
}
