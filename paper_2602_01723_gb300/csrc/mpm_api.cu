// mpm_api.cu -- host side of libmpm: the C ABI declared in include/mpm.h.
// Owns every device buffer, validates arguments, sequences the kernels of
// mpm_forward.cu / mpm_adjoint.cu on the caller's stream and maps the sticky
// device error word to mpm_status.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mpm.h"
#include "mpm_internal.h"

using namespace mpm;

namespace {

const char *g_create_error = "";
thread_local std::string g_create_msg;

}  // namespace


namespace {

mpm_status fail(mpm_ctx *c, mpm_status s, const std::string &m) {
    if (c) c->msg = m;
    return s;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(ctx, MPM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKLAUNCH()                                                                                \
    do {                                                                                          \
        cudaError_t e_ = cudaGetLastError();                                                      \
        if (e_ != cudaSuccess) return fail(ctx, MPM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
mpm_status dalloc(mpm_ctx *ctx, T **p, size_t count, bool zero) {
    if (*p) { cudaFree(*p); *p = nullptr; }
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(ctx, e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    if (zero) {
        e = cudaMemset(*p, 0, count * sizeof(T));
        if (e != cudaSuccess) return fail(ctx, MPM_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
    }
    return MPM_OK;
}

template <typename T> void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

}  // namespace

bool mpm::is_device_ptr(const void *p) { return on_this_device(p); }

bool mpm::stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusActive;
}

namespace {

mpm_status status_from_err(mpm_ctx *ctx, unsigned err) {
    if (!err) return MPM_OK;
    std::string m = "device error:";
    mpm_status s = MPM_OK;
    if (err & ERRB_DOMAIN) { m += " particle outside the grid stencil range or bad material/instance id;"; s = MPM_ERR_OUT_OF_DOMAIN; }
    if (err & ERRB_NONFINITE) { m += " non-finite state or J <= 0 under Neo-Hookean;"; if (!s) s = MPM_ERR_NONFINITE; }
    if (err & ERRB_CAPACITY) { m += " grid block pool or chunk list exhausted;"; if (!s) s = MPM_ERR_CAPACITY; }
    if (err & ERRB_CFL) { m += " a particle moved more than one cell in a substep;"; if (!s) s = MPM_ERR_CFL; }
    if (err & ERRB_TIMEOUT) { m += " bounded wait expired;"; if (!s) s = MPM_ERR_TIMEOUT; }
    ctx->msg = m;
    ctx->sticky = MPM_ERR_STATE;
    return s;
}

mpm_status check_device_error(mpm_ctx *ctx, cudaStream_t st) {
    CK(cudaStreamSynchronize(st));
    unsigned err = 0;
    CK(cudaMemcpy(&err, ctx->D.err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    return status_from_err(ctx, err);
}

// copy a caller array to a device pointer usable by kernels (staging host data)
mpm_status stage_in(mpm_ctx *ctx, const void *src, size_t bytes, size_t &off, const void **dev, cudaStream_t st) {
    *dev = nullptr;
    if (!src) return MPM_OK;
    if (is_device_ptr(src)) { *dev = src; return MPM_OK; }
    if (stream_capturing(st)) return fail(ctx, MPM_ERR_INVALID_ARG, "inside a stream capture the inputs must be device arrays");
    off = (off + 255) & ~size_t(255);
    if (off + bytes > ctx->stage_bytes) return fail(ctx, MPM_ERR_CUDA, "internal: staging buffer too small");
    void *d = (char *)ctx->stage + off;
    CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st));
    *dev = d;
    off += bytes;
    return MPM_OK;
}

mpm_status ensure_stage(mpm_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->stage_bytes) return MPM_OK;
    dfree(ctx->stage);
    ctx->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->stage, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); ctx->stage = nullptr; return fail(ctx, MPM_ERR_OOM, "staging allocation failed"); }
    ctx->stage_bytes = bytes;
    return MPM_OK;
}

mpm_status ensure_particles(mpm_ctx *ctx, long long n) {
    if (n <= ctx->cap && ctx->D.rec) return MPM_OK;
    long long cap = n;
    if (ctx->opt.max_particles > cap) cap = ctx->opt.max_particles;
    Dev &D = ctx->D;
    mpm_status s;
    if ((s = dalloc(ctx, &D.rec, (size_t)cap * REC_F4, false))) return s;
    if ((s = dalloc(ctx, &D.key, (size_t)cap, false))) return s;
    if ((s = dalloc(ctx, &D.rank, (size_t)cap, false))) return s;
    if ((s = dalloc(ctx, &D.sorted, (size_t)cap, false))) return s;
    ctx->cap = cap;
    // grid pool: at most 27 active blocks per occupied block
    unsigned long long occ_max = (unsigned long long)std::min<long long>(cap, ctx->total_blocks);
    unsigned long long pool = ctx->opt.max_active_blocks > 0 ? (unsigned long long)ctx->opt.max_active_blocks
                                                             : std::min<unsigned long long>(ctx->total_blocks, 27ull * occ_max);
    if (pool > 0xffffffffull / BLK_NODES) pool = 0xffffffffull / BLK_NODES;
    if (pool > ctx->pool_blocks) {
        for (int k = 0; k < 2; ++k) {
            if ((s = dalloc(ctx, &D.gmv[k], (size_t)pool * BLK_NODES, true))) return s;
            if ((s = dalloc(ctx, &D.gv[k], (size_t)pool * BLK_NODES, true))) return s;
            if ((s = dalloc(ctx, &D.active[k], (size_t)pool, false))) return s;
        }
        ctx->pool_blocks = (unsigned)pool;
    }
    D.max_active = ctx->pool_blocks;
    if ((s = ensure_chunks(ctx))) return s;
    ++ctx->generation;
    // staging: inputs are at most 30 floats per particle
    return ensure_stage(ctx, (size_t)cap * 30 * sizeof(float) + 16 * 256);
}

cudaStream_t S(void *stream) { return (cudaStream_t)stream; }

// Lists of the direct binning, sized from the binning of the load that just
// completed: per block max(64, 1.5 x the largest block count) particles (a
// multiple of 32), for up to 8 x the occupied blocks + 256 pool slots (the
// active blocks around the occupied ones number about 3 x); overflow entries
// and work items for every particle.  A later compression beyond these sizes
// costs one-particle work items (counted in mpm_stats), not correctness.
mpm_status ensure_direct(mpm_ctx *ctx, cudaStream_t st) {
    Dev &D = ctx->D;
    unsigned c[CTR_COUNT];
    CK(cudaMemcpyAsync(c, D.ctr, sizeof(c), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const unsigned maxcnt = c[CTR_MAX_COUNT], nocc = c[CTR_N_OCC];
    unsigned cap = std::max(64u, (maxcnt + maxcnt / 2 + 31u) / 32u * 32u);
    cap = std::min(cap, 8192u);
    const unsigned long long blocks = std::min<unsigned long long>(ctx->pool_blocks, 8ull * nocc + 256ull);
    const size_t slist = (size_t)blocks * cap;
    const size_t n = (size_t)ctx->cap;
    const size_t chunks = n / 16 + (size_t)std::min<long long>(ctx->cap, ctx->total_blocks) + 1 + n;
    mpm_status s;
    bool grew = false;
    for (int k = 0; k < 2; ++k) {
        if (slist > ctx->slist_alloc && (s = dalloc(ctx, &D.slist[k], slist, false))) return s;
        if (2 * n > ctx->ovf_alloc && (s = dalloc(ctx, &D.ovf[k], 2 * n, false))) return s;
        if ((size_t)ctx->total_blocks > ctx->occd_alloc && (s = dalloc(ctx, &D.occd[k], (size_t)ctx->total_blocks, false)))
            return s;
        if (chunks > ctx->chunksd_alloc && (s = dalloc(ctx, &D.chunksd[k], chunks, false))) return s;
    }
    if (slist > ctx->slist_alloc) { ctx->slist_alloc = slist; grew = true; }
    if (2 * n > ctx->ovf_alloc) { ctx->ovf_alloc = 2 * n; grew = true; }
    if ((size_t)ctx->total_blocks > ctx->occd_alloc) { ctx->occd_alloc = (size_t)ctx->total_blocks; grew = true; }
    if (chunks > ctx->chunksd_alloc) { ctx->chunksd_alloc = chunks; grew = true; }
    if (D.slist_cap != cap || D.slist_blocks != (unsigned)(ctx->slist_alloc / cap)) grew = true;
    // every list entry a work item can reach is written by the binning that
    // made the item; cleared here all the same, so that any entry is a
    // particle index of this load
    for (int k = 0; k < 2; ++k) CK(cudaMemsetAsync(D.slist[k], 0, ctx->slist_alloc * sizeof(unsigned), st));
    D.slist_cap = cap;
    D.slist_blocks = (unsigned)std::min<size_t>(ctx->slist_alloc / cap, ctx->pool_blocks);
    D.ovf_cap = (unsigned)(ctx->ovf_alloc / 2);
    D.max_chunks_d = (unsigned)std::min<size_t>(ctx->chunksd_alloc, 0xffffffffu);
    if (grew) ++ctx->generation;   // kernel arguments changed: recapture the graphs
    ctx->direct_ready = true;
    return MPM_OK;
}

}  // namespace

// chunk list large enough for the current chunk size and particle capacity
mpm_status mpm::ensure_chunks(mpm_ctx *ctx) {
    Dev &D = ctx->D;
    unsigned long long occ_max = (unsigned long long)std::min<long long>(ctx->cap, ctx->total_blocks);
    unsigned long long chunks = (unsigned long long)(ctx->cap / D.chunk) + occ_max + 1;
    if (chunks > ctx->chunk_cap) {
        mpm_status s = dalloc(ctx, &D.chunks, (size_t)chunks, false);
        if (s) return s;
        ctx->chunk_cap = (unsigned)chunks;
        ++ctx->generation;
    }
    D.max_chunks = ctx->chunk_cap;
    return MPM_OK;
}

// ===========================================================================
// internal sequencing shared with the adjoint translation unit
// ===========================================================================
namespace mpm {

void L_plan(mpm_ctx *ctx, int bump_mask, cudaStream_t st) {
    launch_plan(ctx->D, bump_mask, st);
    ++ctx->launches;
    ctx->bins_pending = false;
}
void L_prepare(mpm_ctx *ctx, int upd_par, int act_par, int do_sort, cudaStream_t st, int keep_momentum) {
    launch_prepare(ctx->D, upd_par, act_par, do_sort, keep_momentum, ctx->grid_small, st);
    ++ctx->launches;
}
void L_bin(mpm_ctx *ctx, cudaStream_t st) {
    launch_bin(ctx->D, st);
    ++ctx->launches;
    ctx->bins_pending = true;
}
void L_between(mpm_ctx *ctx, int upd, int act, cudaStream_t st) {
    launch_between(ctx->D, upd, act, ctx->grid_small, st);
    ++ctx->launches;
    ctx->bins_pending = false;
}
void L_substep(mpm_ctx *ctx, int mode, int gpar, int spar, cudaStream_t st, bool direct, int in_par) {
    cudaEvent_t *ev = nullptr;
    if (ctx->trace_on) {
        std::vector<cudaEvent_t> &pool = ctx->trace_ev[mode];
        size_t u = ctx->trace_used[mode];
        while (pool.size() < u + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); break; }
            pool.push_back(e);
        }
        if (pool.size() >= u + 2) {
            ev = &pool[u];
            ctx->trace_used[mode] = u + 2;
            cudaEventRecord(ev[0], st);
        }
    }
    Dev Dc = ctx->D;
    if (in_par >= 0) {   // the work items and lists of the direct binning into buffer in_par
        Dc.chunks = ctx->D.chunksd[in_par];
        Dc.chunk_ctr = CTR_D_CH + in_par;
        Dc.sorted = ctx->D.slist[in_par];
        Dc.ovf_in = ctx->D.ovf[in_par];
    }
    launch_substep(Dc, mode, gpar, spar, ctx->grid_sub[mode], direct, st);
    ++ctx->launches;
    if (ev) cudaEventRecord(ev[1], st);
}

// one steady-state substep: grid update of buffer par with the activation of
// the other buffer and the sort, fused G2P + P2G, plan of the new grouping
// (which opens a fresh epoch for buffer par, activated in the next substep)
static void middle_substep(mpm_ctx *ctx, int par, cudaStream_t st) {
    L_prepare(ctx, par, par ^ 1, 1, st);
    L_substep(ctx, 1, par, par ^ 1, st);
    L_plan(ctx, 1 << par, st);
}

// one steady-state substep with direct binning: between-substep work for
// buffer par (grid update, work items of the last binning, activation of the
// other buffer), then the fused G2P + P2G binning into the other buffer
static void middle_direct(mpm_ctx *ctx, int par, cudaStream_t st) {
    L_between(ctx, par, par ^ 1, st);
    L_substep(ctx, 1, par, par ^ 1, st, true, par);
}

// CUDA graph of two steady-state substeps (parity 0 then 1; with direct
// binning, which starts at substep 1, parity 1 then 0).  It is captured
// on a library-owned stream (the legacy default stream cannot be captured)
// the first time it is needed for this particle count and these buffers, and
// replayed on the caller's stream.
static cudaGraphExec_t graph_pair(mpm_ctx *ctx, cudaStream_t st, bool direct) {
    const long long key = ((long long)ctx->D.n * 1000003ll + ctx->generation) * 2 + (direct ? 1 : 0);
    if (ctx->graph2 && ctx->graph_key == key) return ctx->graph2;
    if (ctx->graph2) { cudaGraphExecDestroy(ctx->graph2); ctx->graph2 = nullptr; }
    cudaStreamCaptureStatus cs;
    if (st && (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)) {
        cudaGetLastError();
        return nullptr;   // the caller is capturing: launch directly into its capture
    }
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ctx->cap_stream = nullptr;
        return nullptr;
    }
    const long long l0 = ctx->launches;
    cudaGraph_t g = nullptr;
    cudaStream_t cst = ctx->cap_stream;
    if (cudaStreamBeginCapture(cst, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    if (direct) {
        middle_direct(ctx, 1, cst);
        middle_direct(ctx, 0, cst);
    } else {
        middle_substep(ctx, 0, cst);
        middle_substep(ctx, 1, cst);
    }
    if (cudaStreamEndCapture(cst, &g) != cudaSuccess || !g) { cudaGetLastError(); ctx->launches = l0; return nullptr; }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) { cudaGetLastError(); ex = nullptr; }
    cudaGraphDestroy(g);
    ctx->launches = l0;   // capture launched nothing
    ctx->graph2 = ex;
    ctx->graph_key = key;
    return ex;
}

// forward of n substeps from the current state (bins must be valid);
// leaves the state advanced and binned.  With tape != NULL the records after
// substep s (s = 0 .. n_sub-1) are also copied to tape + (s+1) * tape_stride.
bool direct_forward(const mpm_ctx *ctx, int n_sub) {
    return ctx->direct_ready && ctx->D.scatter != 0 && n_sub > 1;
}

mpm_status run_substeps(mpm_ctx *ctx, int n_sub, cudaStream_t st, float4 *tape, size_t tape_stride,
                        const std::vector<StateCopy> *copies) {
    if (n_sub <= 0) return MPM_OK;
    const size_t rec_bytes = (size_t)ctx->D.n * REC_F4 * sizeof(float4);
    auto tape_copy = [&](int s) -> bool {
        return !tape || cudaMemcpyAsync(tape + (size_t)(s + 1) * tape_stride, ctx->D.rec, rec_bytes,
                                        cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    };
    L_plan(ctx, 3, st);               // epochs for buffer 0 (P2G below) and 1 (first fused substep)
    L_prepare(ctx, -1, 0, 1, st);
    L_substep(ctx, 0, 0, 0, st);
    const int middle = n_sub - 1;
    // Direct binning (forward runs without a tape, scatter strategies 1 and
    // 2): the fused substeps place each particle straight into its new
    // block's list, and one k_between launch (no scan, no sort) prepares the
    // next substep.  Substep 0 runs on the plan above.
    // The copies are taken after the fused kernel that completes their state;
    // a graph pair is not replayed across one.
    if (!tape && direct_forward(ctx, n_sub)) {
        size_t ci = 0;
        auto due = [&](int state) { return copies && ci < copies->size() && (*copies)[ci].state == state; };
        auto copy_after = [&](int state) -> bool {
            for (; due(state); ++ci)
                if (cudaMemcpyAsync((*copies)[ci].dst, ctx->D.rec, rec_bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                    return false;
            return true;
        };
        CK(cudaMemsetAsync(ctx->D.ctr + CTR_D_OCC, 0, 6 * sizeof(unsigned), st));
        L_prepare(ctx, 0, 1, 0, st);
        L_substep(ctx, 1, 0, 1, st, true, -1);
        if (!copy_after(1)) return fail(ctx, MPM_ERR_CUDA, "state copy failed");
        cudaGraphExec_t ex = nullptr;
        if (ctx->use_graph && !ctx->trace_on && middle >= 5 && !stream_capturing(st)) ex = graph_pair(ctx, st, true);
        for (int s = 1; s < middle;) {
            if (ex && (s & 1) && s + 1 < middle && !due(s + 1)) {   // substeps s and s + 1
                if (cudaGraphLaunch(ex, st) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ctx, MPM_ERR_CUDA, "graph launch failed");
                }
                ctx->launches += 4;   // two substeps: between + fused substep each
                s += 2;
            } else {
                middle_direct(ctx, s & 1, st);
                s += 1;
            }
            if (!copy_after(s)) return fail(ctx, MPM_ERR_CUDA, "state copy failed");
        }
        L_between(ctx, middle & 1, -1, st);              // work items of the last binning
        L_substep(ctx, 2, middle & 1, 0, st, false, middle & 1);
        ctx->bins_pending = true;     // the last substep binned the new positions (for a sort)
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(ctx, MPM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
        return MPM_OK;
    }
    int s = 0;
    // inside the caller's stream capture the substeps go straight into its graph
    if (ctx->use_graph && !ctx->trace_on && !tape && middle >= 4 && !stream_capturing(st)) {
        cudaGraphExec_t ex = graph_pair(ctx, st, false);
        if (ex) {
            for (; s + 1 < middle; s += 2) {
                if (cudaGraphLaunch(ex, st) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ctx, MPM_ERR_CUDA, "graph launch failed");
                }
                ctx->launches += 6;   // two substeps: prepare, fused substep and plan each
            }
        }
    }
    for (; s < n_sub; ++s) {
        const int par = s & 1;
        if (s < middle) {
            middle_substep(ctx, par, st);
        } else {
            L_prepare(ctx, par, -1, s > 0, st);           // sort for the latest plan
            L_substep(ctx, 2, par, 0, st);
        }
        if (!tape_copy(s)) return fail(ctx, MPM_ERR_CUDA, "tape copy failed");
    }
    ctx->bins_pending = true;     // the last substep binned the new positions
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, MPM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return MPM_OK;
}

void rebin(mpm_ctx *ctx, cudaStream_t st) {
    if (ctx->bins_pending) L_plan(ctx, 0, st);
    L_bin(ctx, st);
}

mpm_status ctx_fail(mpm_ctx *ctx, mpm_status s, const std::string &m) { return fail(ctx, s, m); }
mpm_status ctx_check(mpm_ctx *ctx, cudaStream_t st) { return check_device_error(ctx, st); }

}  // namespace mpm

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

MPM_API mpm_status mpm_default_options(mpm_options *opt) {
    if (!opt) return MPM_ERR_INVALID_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->n_instances = 1;
    opt->bound = 3;
    opt->walls[0] = MPM_WALL_SLIP;
    opt->walls[1] = MPM_WALL_SLIP;
    opt->walls[2] = MPM_WALL_STICKY;
    opt->walls[3] = MPM_WALL_SLIP;
    opt->walls[4] = MPM_WALL_SLIP;
    opt->walls[5] = MPM_WALL_SLIP;
    opt->ckpt_every = 20;
    opt->scatter = 1;
    return MPM_OK;
}

MPM_API mpm_status mpm_create(const int32_t grid_res[3], float dx, float dt, const float gravity[3],
                              const mpm_material *table, int32_t n_materials, const mpm_options *opt,
                              mpm_ctx **out) {
    g_create_error = "";
    if (!out) { g_create_error = "out is NULL"; return MPM_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!grid_res || !gravity || !table || n_materials < 1) { g_create_error = "NULL argument or no materials"; return MPM_ERR_INVALID_ARG; }
    for (int d = 0; d < 3; ++d)
        if (grid_res[d] < 8 || grid_res[d] % 4 != 0 || grid_res[d] > 4096) {
            g_create_error = "grid_res must be multiples of 4 in [8, 4096]";
            return MPM_ERR_INVALID_ARG;
        }
    if (!(dx > 0.f) || !(dt > 0.f) || !std::isfinite(dx) || !std::isfinite(dt)) { g_create_error = "dx and dt must be positive"; return MPM_ERR_INVALID_ARG; }
    mpm_options o;
    mpm_default_options(&o);
    if (opt) o = *opt;
    if (o.n_instances < 1 || o.bound < 0 || o.ckpt_every < 0 || o.scatter < 0 || o.scatter > 2 || o.chunk < 0 ||
        o.tape_grid < 0 || o.tape_grid > 1) {
        g_create_error = "bad options";
        return MPM_ERR_INVALID_ARG;
    }
    if (o.ckpt_every == 0) o.ckpt_every = 20;
    for (int i = 0; i < 6; ++i)
        if (o.walls[i] < 0 || o.walls[i] > 2) { g_create_error = "bad wall type"; return MPM_ERR_INVALID_ARG; }
    for (int m = 0; m < n_materials; ++m) {
        const mpm_material &t = table[m];
        if (t.elastic < 0 || t.elastic > 5 || t.plastic < 0 || t.plastic > 4 || !(t.E > 0.f) || !(t.rho > 0.f) ||
            !(t.nu > -1.f && t.nu < 0.5f)) {
            g_create_error = "bad material table entry";
            return MPM_ERR_INVALID_ARG;
        }
    }
    long long bpi = (long long)(grid_res[0] / 4) * (grid_res[1] / 4) * (grid_res[2] / 4);
    long long total = bpi * o.n_instances;
    if (total > (1ll << 31)) { g_create_error = "too many grid blocks"; return MPM_ERR_INVALID_ARG; }

    mpm_ctx *ctx = new (std::nothrow) mpm_ctx();
    if (!ctx) { g_create_error = "host allocation failed"; return MPM_ERR_OOM; }
    cudaGetDevice(&ctx->device);
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    std::memset(&ctx->D, 0, sizeof(Dev));
    ctx->D.chunk_ctr = CTR_N_CHUNKS;
    Dev &D = ctx->D;
    for (int d = 0; d < 3; ++d) {
        ctx->R[d] = grid_res[d];
        D.R[d] = grid_res[d];
        D.NB[d] = grid_res[d] / 4;
        ctx->g[d] = gravity[d];
        D.g[d] = gravity[d];
    }
    D.bpi = (int)bpi;
    D.n_inst = o.n_instances;
    ctx->dx = dx; ctx->dt = dt;
    D.dx = dx; D.inv_dx = 1.f / dx; D.dt = dt;
    D.qf = position_fraction_bits(std::max(grid_res[0], std::max(grid_res[1], grid_res[2])));
    D.q_cell = std::ldexp(1.f, D.qf);
    D.q_unit = std::ldexp(1.f, -D.qf);
    D.bound = o.bound;
    for (int i = 0; i < 6; ++i) D.wall[i] = o.walls[i];
    ctx->opt = o;
    ctx->table.assign(table, table + n_materials);
    ctx->total_blocks = total;
    D.chunk = o.chunk > 0 ? std::min(o.chunk, substep_chunk_max()) : 128;
    mpm_status s = MPM_OK;
#define CREATE_TRY(x)                              \
    if ((s = (x)) != MPM_OK) {                     \
        g_create_msg = ctx->msg;                   \
        g_create_error = g_create_msg.c_str();     \
        mpm_destroy(ctx);                          \
        return s;                                  \
    }
    std::vector<float> E(n_materials), nu(n_materials), rho(n_materials), ys(n_materials), al(n_materials);
    std::vector<int> el(n_materials), pl(n_materials);
    for (int m = 0; m < n_materials; ++m) {
        E[m] = table[m].E; nu[m] = table[m].nu; rho[m] = table[m].rho; ys[m] = table[m].yield_stress;
        el[m] = table[m].elastic; pl[m] = table[m].plastic;
        // Drucker-Prager alpha of the friction angle (Klar et al. 2016)
        double sphi = std::sin(table[m].friction_angle_deg * M_PI / 180.0);
        al[m] = (float)(std::sqrt(2.0 / 3.0) * 2.0 * sphi / (3.0 - sphi));
    }
    CREATE_TRY(dalloc(ctx, &ctx->mE, n_materials, false));
    CREATE_TRY(dalloc(ctx, &ctx->mnu, n_materials, false));
    CREATE_TRY(dalloc(ctx, &ctx->mrho, n_materials, false));
    CREATE_TRY(dalloc(ctx, &ctx->myield, n_materials, false));
    CREATE_TRY(dalloc(ctx, &ctx->malpha, n_materials, false));
    CREATE_TRY(dalloc(ctx, &ctx->mel, n_materials, false));
    CREATE_TRY(dalloc(ctx, &ctx->mpl, n_materials, false));
    cudaMemcpy(ctx->mE, E.data(), n_materials * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(ctx->mnu, nu.data(), n_materials * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(ctx->mrho, rho.data(), n_materials * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(ctx->myield, ys.data(), n_materials * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(ctx->malpha, al.data(), n_materials * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(ctx->mel, el.data(), n_materials * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(ctx->mpl, pl.data(), n_materials * 4, cudaMemcpyHostToDevice);
    for (int k = 0; k < 2; ++k) {
        CREATE_TRY(dalloc(ctx, &D.page[k], (size_t)total, false));
        CREATE_TRY(dalloc(ctx, &D.page_epoch[k], (size_t)total, true));
    }
    CREATE_TRY(dalloc(ctx, &D.bcount, (size_t)total, true));
    CREATE_TRY(dalloc(ctx, &D.bstart, (size_t)total, false));
    CREATE_TRY(dalloc(ctx, &D.occ, (size_t)total, false));
    CREATE_TRY(dalloc(ctx, &D.plan, (size_t)total, false));
    CREATE_TRY(dalloc(ctx, &D.ctr, CTR_COUNT, true));
    CREATE_TRY(dalloc(ctx, &D.err, 1, true));
    D.scatter = o.scatter;
    D.xm = 0;
    for (int m = 0; m < n_materials; ++m)
        if (el[m] > 1 || pl[m] > 2) D.xm = 1;   // further models: the XM kernel variant
    for (int m = 0; m < 3; ++m) {
        int occ = substep_occupancy(m, D.scatter, D.chunk, D.xm != 0);
        ctx->grid_sub[m] = ctx->sm_count * (occ > 0 ? occ : 1);
    }
    ctx->grid_small = ctx->sm_count * 8;
    ctx->adj_pl = ADJ_ELASTIC;
    ctx->adj_el = ADJ_FCR;
    for (int m = 0; m < n_materials; ++m) {
        if (pl[m] > 2) ctx->adj_pl = ADJ_ALL;
        else if (pl[m] != 0) ctx->adj_pl = std::max(ctx->adj_pl, (int)ADJ_PLASTIC);
        if (el[m] > 1) ctx->adj_el = ADJ_ALL;
        else if (el[m] == 1) ctx->adj_el = std::max(ctx->adj_el, (int)ADJ_FCR_NH);
    }
    ctx->grid_adj = ctx->sm_count * adjoint_occupancy(ctx->adj_pl, ctx->adj_el);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        g_create_msg = std::string("create: ") + cudaGetErrorString(e);
        g_create_error = g_create_msg.c_str();
        mpm_destroy(ctx);
        return MPM_ERR_CUDA;
    }
    *out = ctx;
    return MPM_OK;
#undef CREATE_TRY
}

MPM_API mpm_status mpm_load_particles(mpm_ctx *ctx, int64_t n, const float *x, const float *v, const float *C,
                                      const float *F, const float *vol, const int32_t *material_id,
                                      const int32_t *instance, const float *params, void *stream) {
    TraceRange trace_range("mpm_load_particles");
    if (!ctx) return MPM_ERR_INVALID_ARG;
    if (n <= 0 || n > (1ll << 31) - 1 || !x || !vol || !material_id)
        return fail(ctx, MPM_ERR_INVALID_ARG, "n must be in [1, 2^31) and x, vol, material_id non-NULL");
    if (any_on_other_device({x, v, C, F, vol, material_id, instance, params}))
        return fail(ctx, MPM_ERR_INVALID_ARG, "an array lives on another device than the current one");
    cudaStream_t st = S(stream);
    const bool cap = stream_capturing(st);
    if (cap && (n > ctx->cap || !ctx->D.rec))
        return fail(ctx, MPM_ERR_STATE, "inside a stream capture n must fit the capacity of an earlier load");
    mpm_status s = ensure_particles(ctx, n);
    if (s) return s;
    Dev &D = ctx->D;
    D.n = (int)n;
    size_t off = 0;
    LoadArgs a;
    std::memset(&a, 0, sizeof(a));
    const void *p;
    if ((s = stage_in(ctx, x, n * 12, off, &p, st))) return s; a.x = (const float *)p;
    if ((s = stage_in(ctx, v, n * 12, off, &p, st))) return s; a.v = (const float *)p;
    if ((s = stage_in(ctx, C, n * 36, off, &p, st))) return s; a.C = (const float *)p;
    if ((s = stage_in(ctx, F, n * 36, off, &p, st))) return s; a.F = (const float *)p;
    if ((s = stage_in(ctx, vol, n * 4, off, &p, st))) return s; a.vol = (const float *)p;
    if ((s = stage_in(ctx, material_id, n * 4, off, &p, st))) return s; a.mat = (const int *)p;
    if ((s = stage_in(ctx, instance, n * 4, off, &p, st))) return s; a.inst = (const int *)p;
    if ((s = stage_in(ctx, params, n * 12, off, &p, st))) return s; a.params = (const float *)p;
    a.table = MatTable{(int)ctx->table.size(), ctx->mE, ctx->mnu, ctx->mrho, ctx->myield, ctx->malpha, ctx->mel, ctx->mpl};
    CK(cudaMemsetAsync(D.err, 0, sizeof(unsigned), st));
    CK(cudaMemsetAsync(D.bcount, 0, (size_t)ctx->total_blocks * sizeof(unsigned), st));
    CK(cudaMemsetAsync(D.ctr + CTR_N_OCC, 0, sizeof(unsigned), st));
    CK(cudaMemsetAsync(D.ctr + CTR_D_OVF_TOTAL, 0, 2 * sizeof(unsigned), st));   // and CTR_MAX_COUNT
    launch_load(D, a, st);
    ++ctx->launches;
    L_bin(ctx, st);
    CKLAUNCH();
    ctx->sticky = MPM_OK;
    ctx->loaded = true;
    ctx->recorded = 0;
    ctx->record_broken = false;
    if (cap) return MPM_OK;   // device errors surface at the next synchronising call
    s = check_device_error(ctx, st);
    if (s) {
        ctx->loaded = false;
        return s;
    }
    return ensure_direct(ctx, st);
}

MPM_API mpm_status mpm_step(mpm_ctx *ctx, int32_t n_substeps, int32_t record, void *stream) {
    TraceRange trace_range("mpm_step");
    if (!ctx) return MPM_ERR_INVALID_ARG;
    if (n_substeps < 0) return fail(ctx, MPM_ERR_INVALID_ARG, "n_substeps < 0");
    if (!ctx->loaded || ctx->sticky) return fail(ctx, MPM_ERR_STATE, "no valid particle state (load particles first)");
    if (n_substeps == 0) return MPM_OK;
    cudaStream_t st = S(stream);
    if (!record) {
        if (ctx->recorded > 0) ctx->record_broken = true;
        return run_substeps(ctx, n_substeps, st);
    }
    return record_substeps(ctx, n_substeps, st);
}

MPM_API mpm_status mpm_get_particles(mpm_ctx *ctx, float *x, float *v, float *C, float *F, void *stream) {
    if (!ctx) return MPM_ERR_INVALID_ARG;
    if (!ctx->loaded) return fail(ctx, MPM_ERR_STATE, "no particles loaded");
    if (any_on_other_device({x, v, C, F})) return fail(ctx, MPM_ERR_INVALID_ARG, "an array lives on another device than the current one");
    cudaStream_t st = S(stream);
    Dev &D = ctx->D;
    size_t n = (size_t)D.n;
    float *outs[4] = {x, v, C, F};
    size_t widths[4] = {3, 3, 9, 9};
    float *dptr[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t off = 0;
    for (int i = 0; i < 4; ++i) {
        if (!outs[i]) continue;
        if (is_device_ptr(outs[i])) { dptr[i] = outs[i]; continue; }
        off = (off + 255) & ~size_t(255);
        dptr[i] = (float *)((char *)ctx->stage + off);
        off += n * widths[i] * sizeof(float);
    }
    if (off > ctx->stage_bytes) return fail(ctx, MPM_ERR_CUDA, "internal: staging too small");
    launch_export(D, dptr[0], dptr[1], dptr[2], dptr[3], st);
    ++ctx->launches;
    CKLAUNCH();
    for (int i = 0; i < 4; ++i)
        if (outs[i] && dptr[i] != outs[i])
            CK(cudaMemcpyAsync(outs[i], dptr[i], n * widths[i] * sizeof(float), cudaMemcpyDeviceToHost, st));
    return MPM_OK;
}

MPM_API mpm_status mpm_sync(mpm_ctx *ctx, void *stream) {
    if (!ctx) return MPM_ERR_INVALID_ARG;
    return check_device_error(ctx, S(stream));
}

MPM_API mpm_status mpm_stats(mpm_ctx *ctx, int64_t counters[16], void *stream) {
    if (!ctx || !counters) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = S(stream);
    CK(cudaStreamSynchronize(st));
    unsigned c[CTR_COUNT], err = 0;
    CK(cudaMemcpy(c, ctx->D.ctr, sizeof(c), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&err, ctx->D.err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 16; ++i) counters[i] = 0;
    counters[0] = ctx->D.n;
    counters[1] = c[CTR_N_PLAN];
    counters[2] = std::max(c[CTR_N_ACTIVE], c[CTR_N_ACTIVE + 1]);
    counters[3] = c[CTR_N_CHUNKS];
    counters[4] = c[CTR_FALLBACKS];
    counters[5] = ctx->recorded;
    counters[6] = err;
    counters[7] = ctx->pool_blocks;
    counters[8] = ctx->launches;
    counters[9] = ctx->adj.gt ? ctx->adj.gt_pool : 0;
    counters[10] = ctx->adj.gt_reruns;
    counters[11] = c[CTR_D_OVF_TOTAL];
    counters[12] = ctx->direct_ready ? ctx->D.slist_cap : 0;
    counters[13] = ctx->direct_ready ? ctx->D.slist_blocks : 0;
    return MPM_OK;
}

MPM_API mpm_status mpm_trace(mpm_ctx *ctx, int32_t enable, double ms[3], int64_t count[3]) {
    if (!ctx) return MPM_ERR_INVALID_ARG;
    if (ms && count) {
        for (int m = 0; m < 3; ++m) {
            ms[m] = 0.0;
            count[m] = 0;
            for (size_t u = 0; u + 1 < ctx->trace_used[m]; u += 2) {
                float t = 0.f;
                if (cudaEventSynchronize(ctx->trace_ev[m][u + 1]) != cudaSuccess ||
                    cudaEventElapsedTime(&t, ctx->trace_ev[m][u], ctx->trace_ev[m][u + 1]) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ctx, MPM_ERR_CUDA, "trace: event query failed");
                }
                ms[m] += t;
                count[m] += 1;
            }
        }
    }
    for (int m = 0; m < 3; ++m) ctx->trace_used[m] = 0;
    ctx->trace_on = enable != 0;
    return MPM_OK;
}

MPM_API mpm_status mpm_record_reset(mpm_ctx *ctx) {
    if (!ctx) return MPM_ERR_INVALID_ARG;
    ctx->recorded = 0;
    ctx->record_broken = false;
    return MPM_OK;
}

MPM_API const char *mpm_last_error(const mpm_ctx *ctx) {
    if (!ctx) return g_create_error;
    return ctx->msg.c_str();
}

MPM_API mpm_status mpm_destroy(mpm_ctx *ctx) {
    if (!ctx) return MPM_OK;
    Dev &D = ctx->D;
    dfree(D.rec); dfree(D.key); dfree(D.rank); dfree(D.sorted); dfree(D.bcount); dfree(D.bstart);
    dfree(D.occ); dfree(D.plan); dfree(D.chunks); dfree(D.ctr); dfree(D.err);
    for (int k = 0; k < 2; ++k) {
        dfree(D.page[k]); dfree(D.page_epoch[k]); dfree(D.active[k]); dfree(D.gmv[k]); dfree(D.gv[k]);
        dfree(D.slist[k]); dfree(D.ovf[k]); dfree(D.occd[k]); dfree(D.chunksd[k]);
    }
    dfree(ctx->mE); dfree(ctx->mnu); dfree(ctx->mrho); dfree(ctx->myield); dfree(ctx->malpha);
    dfree(ctx->mel); dfree(ctx->mpl);
    dfree(ctx->stage);
    free_adjoint(ctx->adj);
    for (int k = 0; k < MPM_MAX_SNAPSHOTS; ++k) dfree(ctx->snap[k]);
    dfree(ctx->bgdo_work); dfree(ctx->bgdo_G); dfree(ctx->bgdo_sum); dfree(ctx->cov0);
    for (int m = 0; m < 3; ++m)
        for (cudaEvent_t e : ctx->trace_ev[m]) cudaEventDestroy(e);
    if (ctx->graph2) cudaGraphExecDestroy(ctx->graph2);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
    return MPM_OK;
}

MPM_API mpm_status mpm_reduce_by_material(mpm_ctx *ctx, const float *per_particle, float *per_material, void *stream) {
    if (!ctx || !per_particle || !per_material) return MPM_ERR_INVALID_ARG;
    if (!ctx->loaded) return fail(ctx, MPM_ERR_STATE, "no particles loaded");
    if (!is_device_ptr(per_particle) || !is_device_ptr(per_material))
        return fail(ctx, MPM_ERR_INVALID_ARG, "per_particle and per_material must be device arrays");
    const int nm = (int)ctx->table.size();
    if (3 * nm * sizeof(float) > 48 * 1024) return fail(ctx, MPM_ERR_INVALID_ARG, "too many materials for the reduction");
    cudaStream_t st = S(stream);
    CK(cudaMemsetAsync(per_material, 0, 3 * nm * sizeof(float), st));
    launch_reduce_by_material(ctx->D, nm, per_particle, per_material, st);
    ++ctx->launches;
    CKLAUNCH();
    return MPM_OK;
}

MPM_API mpm_status mpm_set_tuning(mpm_ctx *ctx, int32_t scatter, int32_t chunk, int32_t use_graph) {
    if (!ctx) return MPM_ERR_INVALID_ARG;
    if (scatter < 0 || scatter > 2 || chunk < 16 || chunk > substep_chunk_max() || chunk % 16 != 0)
        return fail(ctx, MPM_ERR_INVALID_ARG, "scatter in {0,1,2}, chunk a multiple of 16 in [16, 128]");
    Dev &D = ctx->D;
    const int old_chunk = D.chunk;
    D.chunk = chunk;
    mpm_status s = ensure_chunks(ctx);
    if (s) { D.chunk = old_chunk; return s; }
    D.scatter = scatter;
    for (int m = 0; m < 3; ++m) {
        int occ = substep_occupancy(m, D.scatter, D.chunk, D.xm != 0);
        ctx->grid_sub[m] = ctx->sm_count * (occ > 0 ? occ : 1);
    }
    ctx->use_graph = use_graph != 0;
    ++ctx->generation;   // kernel arguments changed: recapture
    return MPM_OK;
}

MPM_API mpm_status mpm_autotune(mpm_ctx *ctx, int32_t n_substeps, int32_t out[3], void *stream) {
    TraceRange trace_range("mpm_autotune");
    if (!ctx || n_substeps < 2) return MPM_ERR_INVALID_ARG;
    if (!ctx->loaded || ctx->sticky) return fail(ctx, MPM_ERR_STATE, "no valid particle state");
    cudaStream_t st = S(stream);
    Dev &D = ctx->D;
    const size_t bytes = (size_t)D.n * REC_F4 * sizeof(float4);
    // snapshot of the records; the trials run from it and it is restored after
    float4 *snap = (float4 *)ctx->stage;
    bool own = false;
    if (bytes > ctx->stage_bytes) {
        if (cudaMalloc(&snap, bytes) != cudaSuccess) { cudaGetLastError(); return fail(ctx, MPM_ERR_OOM, "autotune snapshot"); }
        own = true;
    }
    CK(cudaMemcpyAsync(snap, D.rec, bytes, cudaMemcpyDeviceToDevice, st));
    const int scat0 = D.scatter, chunk0 = D.chunk;
    const bool graph0 = ctx->use_graph;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bs = scat0, bc = chunk0;
    // scatter strategies x particles per work chunk (chunks of <= 64 run
    // 64-thread CTAs at twice the CTAs per SM, larger ones 128-thread CTAs)
    const int scats[2] = {1, 2}, chunks[4] = {32, 64, 96, 128};
    mpm_status s = MPM_OK;
    for (int a = 0; a < 2 && !s; ++a)
        for (int b = 0; b < 4 && !s; ++b) {
            if ((s = mpm_set_tuning(ctx, scats[a], chunks[b], graph0))) break;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && !s; ++rep) {   // first pass warms up (and captures the graph)
                CK(cudaMemcpyAsync(D.rec, snap, bytes, cudaMemcpyDeviceToDevice, st));
                L_plan(ctx, 0, st);
                L_bin(ctx, st);
                cudaEventRecord(e0, st);
                s = run_substeps(ctx, n_substeps, st);
                cudaEventRecord(e1, st);
                CK(cudaEventSynchronize(e1));
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (!s && ms < best) { best = ms; bs = scats[a]; bc = chunks[b]; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    mpm_status s2 = mpm_set_tuning(ctx, s ? scat0 : bs, s ? chunk0 : bc, graph0);
    cudaMemcpyAsync(D.rec, snap, bytes, cudaMemcpyDeviceToDevice, st);
    L_plan(ctx, 0, st);
    L_bin(ctx, st);
    mpm_status s3 = check_device_error(ctx, st);
    if (own) cudaFree(snap);
    if (s) return s;
    if (s2) return s2;
    if (s3) return s3;
    if (out) { out[0] = D.scatter; out[1] = D.chunk; out[2] = (int32_t)(best * 1000.f); }
    return MPM_OK;
}

// P2G of the current state into dense caller arrays m (n_inst*R0*R1*R2) and
// mv (x3); the particle state is left unchanged.  Diagnostic entry point used
// by the teacher-forced parity tests.
MPM_API mpm_status mpm_snapshot(mpm_ctx *ctx, int32_t slot, void *stream) {
    if (!ctx) return MPM_ERR_INVALID_ARG;
    if (slot < 0 || slot >= MPM_MAX_SNAPSHOTS) return fail(ctx, MPM_ERR_INVALID_ARG, "snapshot slot out of range");
    if (!ctx->loaded || ctx->sticky) return fail(ctx, MPM_ERR_STATE, "no valid particle state (load particles first)");
    mpm_status s;
    if (!ctx->snap[slot] || ctx->snap_cap[slot] < ctx->cap) {
        if ((s = dalloc(ctx, &ctx->snap[slot], (size_t)ctx->cap * REC_F4, false))) return s;
        ctx->snap_cap[slot] = ctx->cap;
    }
    CK(cudaMemcpyAsync(ctx->snap[slot], ctx->D.rec, (size_t)ctx->D.n * REC_F4 * sizeof(float4),
                       cudaMemcpyDeviceToDevice, S(stream)));
    ctx->snap_n[slot] = ctx->D.n;
    return MPM_OK;
}

MPM_API mpm_status mpm_bgdo_default_options(mpm_bgdo_options *opt) {
    if (!opt) return MPM_ERR_INVALID_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->delta_target = 0.1f;
    opt->w = -1.f;
    return MPM_OK;
}

MPM_API mpm_status mpm_bgdo(mpm_ctx *ctx, int32_t n_keys, const int32_t *slots, const mpm_bgdo_options *opt,
                            float *G, float *log_E, float *g_tau, float *delta, void *stream) {
    TraceRange trace_range("mpm_bgdo");
    if (!ctx) return MPM_ERR_INVALID_ARG;
    if (n_keys < 1 || n_keys > MPM_MAX_SNAPSHOTS || !slots)
        return fail(ctx, MPM_ERR_INVALID_ARG, "n_keys must be in [1, MPM_MAX_SNAPSHOTS] with a slot list");
    if (any_on_other_device({G, log_E, g_tau, delta})) return fail(ctx, MPM_ERR_INVALID_ARG, "an array lives on another device than the current one");
    mpm_bgdo_options o;
    mpm_bgdo_default_options(&o);
    if (opt) o = *opt;
    if (!std::isfinite(o.delta_target) || !(o.w <= 1.f) || (o.per_material & ~1) || (o.delta_pre_step & ~1))
        return fail(ctx, MPM_ERR_INVALID_ARG, "bgdo options: delta_target finite, w <= 1, flags 0 or 1");
    if (o.per_material && 2 * ctx->table.size() * sizeof(double) > 48 * 1024)
        return fail(ctx, MPM_ERR_INVALID_ARG, "too many materials for the per-material average");
    if (!ctx->loaded || ctx->sticky) return fail(ctx, MPM_ERR_STATE, "no valid particle state (load particles first)");
    for (int k = 0; k < n_keys; ++k) {
        const int sl = slots[k];
        if (sl < 0 || sl >= MPM_MAX_SNAPSHOTS) return fail(ctx, MPM_ERR_INVALID_ARG, "snapshot slot out of range");
        if (!ctx->snap[sl] || ctx->snap_n[sl] != ctx->D.n)
            return fail(ctx, MPM_ERR_STATE, "slot " + std::to_string(sl) + " holds no snapshot of this particle count");
    }
    cudaStream_t st = S(stream);
    Dev &D = ctx->D;
    const size_t n = (size_t)D.n;
    const int nm = (int)ctx->table.size();
    mpm_status s;
    if (ctx->bgdo_cap < ctx->cap) {
        if ((s = dalloc(ctx, &ctx->bgdo_work, (size_t)ctx->cap * REC_F4, false))) return s;
        if ((s = dalloc(ctx, &ctx->bgdo_G, (size_t)ctx->cap, false))) return s;
        ctx->bgdo_cap = ctx->cap;
    }
    if (o.per_material && !ctx->bgdo_sum && (s = dalloc(ctx, &ctx->bgdo_sum, 2 * (size_t)nm, false))) return s;
    // outputs: device pointers are written directly, host ones through the staging buffer
    float *outs[4] = {G, log_E, g_tau, delta};
    const size_t widths[4] = {1, 1, (size_t)n_keys, (size_t)n_keys};
    float *dptr[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t offs[4] = {0, 0, 0, 0}, off = 0;
    bool host_out = false;
    for (int i = 0; i < 4; ++i) {
        if (!outs[i]) continue;
        if (is_device_ptr(outs[i])) { dptr[i] = outs[i]; continue; }
        off = (off + 255) & ~size_t(255);
        offs[i] = off;
        off += n * widths[i] * sizeof(float);
        host_out = true;
    }
    if (host_out) {
        // the stream may still use the staging buffer: reallocate only after it drains
        if (off > ctx->stage_bytes) CK(cudaStreamSynchronize(st));
        if ((s = ensure_stage(ctx, off))) return s;
        for (int i = 0; i < 4; ++i)
            if (outs[i] && !dptr[i]) dptr[i] = (float *)((char *)ctx->stage + offs[i]);
    }
    const size_t rec_bytes = n * REC_F4 * sizeof(float4);
    for (int k = 0; k < n_keys; ++k) {
        const float4 *key = ctx->snap[slots[k]];
        const float4 *post = key;
        if (!o.delta_pre_step) {
            // the pseudo substep: the ordinary substep on a copy of the key frame
            CK(cudaMemcpyAsync(ctx->bgdo_work, key, rec_bytes, cudaMemcpyDeviceToDevice, st));
            float4 *saved = D.rec;
            D.rec = ctx->bgdo_work;
            rebin(ctx, st);
            s = run_substeps(ctx, 1, st);
            D.rec = saved;
            if (s) return s;
            post = ctx->bgdo_work;
        }
        launch_bgdo_accum(D, key, post, k == 0, 1.f / (float)n_keys, o.delta_target, o.w, ctx->bgdo_G,
                          dptr[2] ? dptr[2] + (size_t)k * n : nullptr, dptr[3] ? dptr[3] + (size_t)k * n : nullptr, st);
        ++ctx->launches;
        CKLAUNCH();
    }
    if (o.per_material) {
        CK(cudaMemsetAsync(ctx->bgdo_sum, 0, 2 * (size_t)nm * sizeof(double), st));
        launch_bgdo_material_sum(D, nm, ctx->bgdo_G, ctx->bgdo_sum, st);
        ++ctx->launches;
    }
    if (dptr[0] || dptr[1]) {
        launch_bgdo_finish(D, nm, ctx->bgdo_G, o.per_material ? ctx->bgdo_sum : nullptr, dptr[0], dptr[1], st);
        ++ctx->launches;
    }
    CKLAUNCH();
    if (!o.delta_pre_step) rebin(ctx, st);   // bins of the current state again
    CKLAUNCH();
    for (int i = 0; i < 4; ++i)
        if (outs[i] && dptr[i] != outs[i])
            CK(cudaMemcpyAsync(outs[i], dptr[i], n * widths[i] * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (host_out) return check_device_error(ctx, st);
    return MPM_OK;
}

MPM_API mpm_status mpm_load_covariance(mpm_ctx *ctx, const float *cov0, void *stream) {
    if (!ctx || !cov0) return MPM_ERR_INVALID_ARG;
    if (!ctx->loaded) return fail(ctx, MPM_ERR_STATE, "no particles loaded");
    if (any_on_other_device({cov0})) return fail(ctx, MPM_ERR_INVALID_ARG, "an array lives on another device than the current one");
    const size_t n = (size_t)ctx->D.n;
    mpm_status s;
    if (ctx->cov_cap < ctx->cap) {
        if ((s = dalloc(ctx, &ctx->cov0, (size_t)ctx->cap * 6, false))) return s;
        ctx->cov_cap = ctx->cap;
    }
    CK(cudaMemcpyAsync(ctx->cov0, cov0, n * 6 * sizeof(float), cudaMemcpyDefault, S(stream)));
    ctx->cov_n = ctx->D.n;
    return MPM_OK;
}

MPM_API mpm_status mpm_get_covariance(mpm_ctx *ctx, float *cov, void *stream) {
    if (!ctx || !cov) return MPM_ERR_INVALID_ARG;
    if (!ctx->loaded) return fail(ctx, MPM_ERR_STATE, "no particles loaded");
    if (any_on_other_device({cov})) return fail(ctx, MPM_ERR_INVALID_ARG, "an array lives on another device than the current one");
    if (!ctx->cov0 || ctx->cov_n != ctx->D.n)
        return fail(ctx, MPM_ERR_STATE, "no rest covariances loaded for this particle count");
    cudaStream_t st = S(stream);
    const size_t n = (size_t)ctx->D.n;
    float *d = cov;
    // the kernel stores float2: a device pointer off an 8-byte boundary goes through staging
    if (!is_device_ptr(cov) || ((uintptr_t)cov & 7u)) {
        if (n * 6 * sizeof(float) > ctx->stage_bytes) return fail(ctx, MPM_ERR_CUDA, "internal: staging too small");
        d = (float *)ctx->stage;
    }
    launch_covariance(ctx->D, ctx->cov0, d, st);
    ++ctx->launches;
    CKLAUNCH();
    if (d != cov) CK(cudaMemcpyAsync(cov, d, n * 6 * sizeof(float), cudaMemcpyDefault, st));
    return MPM_OK;
}

MPM_API mpm_status mpm_debug_p2g(mpm_ctx *ctx, float *m, float *mv, void *stream) {
    if (!ctx || !m || !mv) return MPM_ERR_INVALID_ARG;
    if (!ctx->loaded || ctx->sticky) return fail(ctx, MPM_ERR_STATE, "no valid particle state");
    if (!is_device_ptr(m) || !is_device_ptr(mv)) return fail(ctx, MPM_ERR_INVALID_ARG, "m, mv must be device arrays");
    cudaStream_t st = S(stream);
    Dev &D = ctx->D;
    size_t nn = (size_t)ctx->total_blocks * BLK_NODES;
    CK(cudaMemsetAsync(m, 0, nn * sizeof(float), st));
    CK(cudaMemsetAsync(mv, 0, 3 * nn * sizeof(float), st));
    L_plan(ctx, 1, st);
    L_prepare(ctx, -1, 0, 1, st);
    L_substep(ctx, 0, 0, 0, st);
    launch_grid_dense(D, 0, 0, m, mv, st);
    ++ctx->launches;
    // clear the momentum buffer again (the update zeroes it); the binning of
    // the current positions was consumed by the plan, so rebuild it
    L_prepare(ctx, 0, -1, 0, st);
    L_bin(ctx, st);
    CKLAUNCH();
    return check_device_error(ctx, st);
}

}  // extern "C"
