// mpm_batch.cu -- batched execution of independent simulations (included by
// mpm_api.cu, which defines mpm_sim and the per-type dispatch).
//
// A batch keeps a list of member simulations.  Before the first step after a
// change of members it builds, in one device buffer: a type-independent
// descriptor per member (clock, grid storage, re-order arrays), a typed
// descriptor per member of each kernel-variant group, and the flattened block
// lists ((member, tile) for the tile stages, (member, chunk) for grid
// clearing and the count scans).  One step of the whole batch -- prepare,
// clear, the three tile stages per group, finalize, scans, recycled
// placement, re-order per group, parity flip -- is recorded as a CUDA graph
// and replayed for every step.

#include <algorithm>

namespace {

struct BatchGroup {
    const Vtbl* vt;
    int per;           // blaunch flags: 1 = a periodic axis, 2 = P2G span columns
    std::vector<int> members;      // indices into mpm_batch::members
    size_t smem[4];
    size_t desc_off, tl_off;
    int ntl;
};

}  // namespace

struct mpm_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    std::vector<mpm_sim*> members;
    bool dirty = true;
    void* dev = nullptr;
    size_t dev_cap = 0;
    cudaGraphExec_t graph = nullptr;
    bool graph_ok = true;
    int64_t recordings = 0;
    std::vector<BatchGroup> groups;
    size_t common_off = 0, zero_off = 0, scan_off = 0;
    int nzero = 0, nscan = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_batch_err;

mpm_status bfail(mpm_batch* b, mpm_status st, const std::string& msg)
{
    if (b) b->err = msg; else g_batch_err = msg;
    return st;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

void batch_drop_graph(mpm_batch* b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

// Queue one step of every member on the batch's stream.
void batch_launch_step(mpm_batch* b)
{
    const cudaStream_t st = b->stream;
    const int n = (int)b->members.size();
    char* dev = static_cast<char*>(b->dev);
    const BatchCommon* common = reinterpret_cast<const BatchCommon*>(dev + b->common_off);
    const unsigned nb = (unsigned)((n + 127) / 128);
    int64_t l = 0;
    kb_prepare<<<nb, 128, 0, st>>>(common, n);
    kb_zero<<<b->nzero, 256, 0, st>>>(common, reinterpret_cast<const TileRef*>(dev + b->zero_off));
    l += 2;
    for (int stage = 0; stage < 3; ++stage)
        for (const BatchGroup& g : b->groups) {
            g.vt->blaunch(stage, dev + g.desc_off, reinterpret_cast<const TileRef*>(dev + g.tl_off), g.ntl,
                          g.smem[stage], g.per, st);
            ++l;
        }
    kb_finalize<<<nb, 128, 0, st>>>(common, n);
    ++l;
    // re-order: changed tiles; the relayout of a member whose tile outgrew
    // its region (the kernels return at once for the other members)
    auto stage = [&](int k) {
        for (const BatchGroup& g : b->groups) {
            g.vt->blaunch(k, dev + g.desc_off, reinterpret_cast<const TileRef*>(dev + g.tl_off), g.ntl, g.smem[3],
                          g.per, st);
            ++l;
        }
    };
    stage(3);
    stage(4);
    kb_relayout_bases<<<n, 1024, 0, st>>>(common);
    ++l;
    stage(5);
    kb_step_end<<<b->nscan, kScanThreads, 0, st>>>(common, reinterpret_cast<const TileRef*>(dev + b->scan_off));
    kb_flip<<<nb, 128, 0, st>>>(common, n);
    b->launches = l + 2;
}

// Descriptors, block lists and the graph of one batched step.
mpm_status batch_build(mpm_batch* b)
{
    batch_drop_graph(b);
    b->groups.clear();
    const int n = (int)b->members.size();
    if (n == 0) {
        b->dirty = false;
        return MPM_OK;
    }
    // groups of members that share the kernel variant
    for (int i = 0; i < n; ++i) {
        const mpm_sim* s = b->members[i];
        const int per = ((s->G.per[0] | s->G.per[1] | s->G.per[2]) ? 1 : 0) | (p2g_columns(s->G) ? 2 : 0);
        BatchGroup* g = nullptr;
        for (auto& h : b->groups)
            if (h.vt == s->vt && h.per == per) g = &h;
        if (!g) {
            b->groups.push_back(BatchGroup{s->vt, per, {}, {0, 0, 0, 0}, 0, 0, 0});
            g = &b->groups.back();
        }
        g->members.push_back(i);
        for (int k = 0; k < 3; ++k) g->smem[k] = std::max(g->smem[k], s->vt->smem(s->G, k));
        g->smem[3] = std::max(g->smem[3], reorder_smem(s->G));
    }
    // host image of the device buffer
    std::vector<BatchCommon> common(n);
    std::vector<TileRef> zl, sl;
    for (int i = 0; i < n; ++i) {
        const mpm_sim* s = b->members[i];
        BatchCommon& c = common[i];
        memset(&c, 0, sizeof c);
        c.clk = s->clk;
        c.grid16 = (uint4*)s->grid;
        c.n16 = (int64_t)(s->grid_bytes / 16);
        c.count = s->count;
        c.nkey = s->G.nkey;
        c.ntiles = s->G.ntiles;
        c.tvol = s->G.Tvol;
        c.mwords = s->mwords;
        c.dirty = s->dirty;
        c.ring = s->ring;
        c.tbase = s->tbase;
        c.tbase_next = s->tbase_next;
        c.tcount = s->tcount;
        c.cfl_h = s->G.cfl * s->G.h;
        for (int64_t k = 0; k * kZeroChunk < c.n16; ++k) zl.push_back(TileRef{i, (int)k});
        // (member, k): span counts and tiles [k, k + 1) * kScanTile (nkey >= ntiles)
        for (int64_t k = 0; k < scan_blocks(c.nkey); ++k) sl.push_back(TileRef{i, (int)k});
    }
    size_t off = 0;
    b->common_off = off;
    off = align256(off + n * sizeof(BatchCommon));
    b->zero_off = off;
    off = align256(off + zl.size() * sizeof(TileRef));
    b->scan_off = off;
    off = align256(off + sl.size() * sizeof(TileRef));
    std::vector<std::vector<char>> gdesc(b->groups.size());
    std::vector<std::vector<TileRef>> gtl(b->groups.size());
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        BatchGroup& g = b->groups[gi];
        const size_t ds = g.vt->bdesc_size;
        gdesc[gi].resize(ds * g.members.size());
        for (size_t li = 0; li < g.members.size(); ++li) {
            const mpm_sim* s = b->members[g.members[li]];
            g.vt->bdesc_fill(s, gdesc[gi].data() + li * ds);
            for (int t = 0; t < s->G.ntiles; ++t) gtl[gi].push_back(TileRef{(int)li, t});
        }
        g.ntl = (int)gtl[gi].size();
        g.desc_off = off;
        off = align256(off + gdesc[gi].size());
        g.tl_off = off;
        off = align256(off + gtl[gi].size() * sizeof(TileRef));
        cudaError_t e = g.vt->bset_smem(g.smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, MPM_ECUDA, std::string("shared memory attribute: ") + cudaGetErrorString(e));
        }
    }
    std::vector<char> img(off, 0);
    memcpy(img.data() + b->common_off, common.data(), n * sizeof(BatchCommon));
    if (!zl.empty()) memcpy(img.data() + b->zero_off, zl.data(), zl.size() * sizeof(TileRef));
    if (!sl.empty()) memcpy(img.data() + b->scan_off, sl.data(), sl.size() * sizeof(TileRef));
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        memcpy(img.data() + b->groups[gi].desc_off, gdesc[gi].data(), gdesc[gi].size());
        memcpy(img.data() + b->groups[gi].tl_off, gtl[gi].data(), gtl[gi].size() * sizeof(TileRef));
    }
    b->nzero = (int)zl.size();
    b->nscan = (int)sl.size();
    // the previous buffer may still be read by queued steps: wait before reuse
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, MPM_ECUDA, "synchronize");
    }
    if (off > b->dev_cap) {
        if (b->dev) cudaFree(b->dev);
        b->dev = nullptr;
        b->dev_cap = 0;
        if (cudaMalloc(&b->dev, off) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, MPM_ENOMEM, "device allocation failed");
        }
        b->dev_cap = off;
    }
    if (cudaMemcpyAsync(b->dev, img.data(), off, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, MPM_ECUDA, "descriptor upload");
    }
    // record one step
    if (b->graph_ok) {
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            batch_launch_step(b);
            ok = cudaStreamEndCapture(b->stream, &g) == cudaSuccess && g;
        }
        if (ok) ok = cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            // replay by plain launches from now on
            cudaGetLastError();
            b->graph = nullptr;
            b->graph_ok = false;
        } else {
            ++b->recordings;
        }
    }
    b->dirty = false;
    return MPM_OK;
}

}  // namespace

mpm_status mpm_batch_create(void* stream, mpm_batch** out)
{
    if (!out) return bfail(nullptr, MPM_EINVAL, "out is NULL");
    *out = nullptr;
    mpm_batch* b = new mpm_batch();
    cudaGetDevice(&b->device);
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return bfail(nullptr, MPM_ECUDA, "stream creation failed");
        }
        b->own_stream = true;
    }
    *out = b;
    return MPM_OK;
}

mpm_status mpm_batch_add(mpm_batch* b, mpm_sim* s, int64_t nsteps, double dt, double t_end)
{
    if (!b) return bfail(nullptr, MPM_EINVAL, "batch is NULL");
    if (!s) return bfail(b, MPM_EINVAL, "sim is NULL");
    if (s->batch) return bfail(b, MPM_ESTATE, "the simulation is already a member of a batch");
    if (s->poisoned) return bfail(b, MPM_ESTATE, "simulation is poisoned: " + s->err);
    if (nsteps <= 0 || !std::isfinite(dt) || !std::isfinite(t_end)) return bfail(b, MPM_EINVAL, "bad step arguments");
    if (s->device != b->device) return bfail(b, MPM_EINVAL, "simulation and batch are on different devices");
    if (s->profiling) return bfail(b, MPM_EUNSUPPORTED, "profiling is per simulation; disable it first");
    if (!s->col_off.empty()) return bfail(b, MPM_EUNSUPPORTED, "a coloured simulation runs its own colour passes");
    mpm_status st = ensure_cfl(s);
    if (st != MPM_OK) return bfail(b, st, s->err);
    s->started = true;
    k_set_params<<<1, 1, 0, s->stream>>>(s->clk, dt > 0.0 ? dt : 0.0, t_end > 0.0 ? t_end : 0.0);
    k_set_batch<<<1, 1, 0, s->stream>>>(s->clk, (long long)nsteps, s->cur);
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, s->stream) != cudaSuccess || cudaStreamWaitEvent(b->stream, ev, 0) != cudaSuccess) {
        if (ev) cudaEventDestroy(ev);
        cudaGetLastError();
        return bfail(b, MPM_ECUDA, "stream ordering");
    }
    cudaEventDestroy(ev);
    s->batch = b;
    s->stepped = true;
    b->members.push_back(s);
    b->dirty = true;
    return MPM_OK;
}

mpm_status mpm_batch_remove(mpm_batch* b, mpm_sim* s)
{
    if (!b || !s) return bfail(b, MPM_EINVAL, "NULL argument");
    auto it = std::find(b->members.begin(), b->members.end(), s);
    if (it == b->members.end() || s->batch != b) return bfail(b, MPM_EINVAL, "not a member of this batch");
    b->members.erase(it);
    b->dirty = true;
    s->batch = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, b->stream) != cudaSuccess || cudaStreamWaitEvent(s->stream, ev, 0) != cudaSuccess) {
        if (ev) cudaEventDestroy(ev);
        cudaGetLastError();
        s->poisoned = true;
        return bfail(b, MPM_ECUDA, "stream ordering");
    }
    cudaEventDestroy(ev);
    // no step budget outside the batch
    k_set_batch<<<1, 1, 0, s->stream>>>(s->clk, 0, s->cur);
    return MPM_OK;
}

mpm_status mpm_batch_step_async(mpm_batch* b, int64_t nsteps)
{
    if (!b) return bfail(nullptr, MPM_EINVAL, "batch is NULL");
    if (nsteps < 0) return bfail(b, MPM_EINVAL, "nsteps < 0");
    if (b->members.empty() || nsteps == 0) return MPM_OK;
    if (b->dirty) {
        mpm_status st = batch_build(b);
        if (st != MPM_OK) return st;
    }
    for (int64_t i = 0; i < nsteps; ++i) {
        if (b->graph) {
            const cudaError_t ge = cudaGraphLaunch(b->graph, b->stream);
            if (ge != cudaSuccess) {
                cudaGetLastError();
                return bfail(b, MPM_ECUDA, std::string("graph launch: ") + cudaGetErrorString(ge));
            }
        } else {
            batch_launch_step(b);
        }
    }
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return bfail(b, MPM_ECUDA, std::string("launch: ") + cudaGetErrorString(le));
    // every step switches each member to its other tile-buffer table
    for (mpm_sim* s : b->members) {
        if (nsteps & 1) s->cur ^= 1;
        s->launches += b->launches * nsteps / (int64_t)b->members.size();
    }
    return MPM_OK;
}

mpm_status mpm_batch_sync(mpm_batch* b)
{
    if (!b) return bfail(nullptr, MPM_EINVAL, "batch is NULL");
    std::vector<Clock> c(b->members.size());
    for (size_t i = 0; i < b->members.size(); ++i)
        if (cudaMemcpyAsync(&c[i], b->members[i]->clk, sizeof(Clock), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess) {
            cudaGetLastError();
            return bfail(b, MPM_ECUDA, "read clock");
        }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        for (mpm_sim* s : b->members) s->poisoned = true;
        return bfail(b, MPM_ECUDA, "synchronize");
    }
    // a failed member's error bits stay in its clock: it idles in the batch,
    // and its own first call after leaving reports the status and poisons it
    mpm_status first = MPM_OK;
    for (size_t i = 0; i < b->members.size(); ++i) {
        const int e = c[i].err;
        if (!e || first != MPM_OK) continue;
        first = (e & ERR_CFL) ? MPM_ECFL : (e & ERR_NONFINITE) ? MPM_ENONFINITE
              : (e & ERR_TIMEOUT) ? MPM_ETIMEOUT : MPM_ESTATE;
        b->err = "member " + std::to_string(i) + " raised an error in a batched step";
    }
    return first;
}

mpm_status mpm_batch_info(const mpm_batch* b, int64_t out[4])
{
    if (!b || !out) return MPM_EINVAL;
    out[0] = (int64_t)b->members.size();
    out[1] = (int64_t)b->groups.size();
    out[2] = b->launches;
    out[3] = b->recordings;
    return MPM_OK;
}

void* mpm_batch_stream(const mpm_batch* b) { return b ? (void*)b->stream : nullptr; }

const char* mpm_batch_last_error(const mpm_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

void mpm_batch_destroy(mpm_batch* b)
{
    if (!b) return;
    while (!b->members.empty()) mpm_batch_remove(b, b->members.back());
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    if (b->dev) cudaFree(b->dev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}
