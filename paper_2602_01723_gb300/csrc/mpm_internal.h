// mpm_internal.h -- declarations shared by the host side (mpm_api.cu) and the
// kernel translation units of libmpm.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/mpm.h"
#include <nvtx3/nvToolsExt.h>

#include "mpm_dev.cuh"
#include "mpm_ptr.h"

namespace mpm {

// material table as device arrays
struct MatTable {
    int n;
    const float *E, *nu, *rho, *yield, *alpha;
    const int *elastic, *plastic;
};

struct LoadArgs {
    const float *x, *v, *C, *F, *vol, *params;
    const int *mat, *inst;
    MatTable table;
};

// A named range on a profiler's timeline for the lifetime of the object: the
// host-side phases of an entry point (load, forward substeps, reverse pass,
// BGDO, autotuning).  Without an attached tool the calls return at once.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

inline int grid_for(long long n, int threads, int cap = 152 * 16) {
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

void launch_load(const Dev &D, const LoadArgs &a, cudaStream_t st);
void launch_bin(const Dev &D, cudaStream_t st);
void launch_plan(const Dev &D, int bump_mask, cudaStream_t st);
void launch_prepare(const Dev &D, int upd_par, int act_par, int do_sort, int keep_momentum, int grid, cudaStream_t st);
// direct: the fused mode bins straight into the scatter buffer's lists
void launch_substep(const Dev &D, int mode, int gpar, int spar, int grid, bool direct, cudaStream_t st);
// between two direct-binning substeps: grid update of upd, work items of its
// binning, activation of act (see k_between)
void launch_between(const Dev &D, int upd, int act, int grid, cudaStream_t st);
void launch_export(const Dev &D, float *x, float *v, float *C, float *F, cudaStream_t st);
void launch_grid_dense(const Dev &D, int par, int which, float *m, float *mv, cudaStream_t st);
int substep_occupancy(int mode, int scatter, int chunk, bool xm);
int substep_chunk_max();
// model sets of the reverse kernels: plasticity ADJ_ELASTIC (none) or
// ADJ_PLASTIC (von Mises / Drucker-Prager); elasticity ADJ_FCR
// (fixed-corotated) or ADJ_FCR_NH (and Neo-Hookean); ADJ_ALL: any model
enum { ADJ_ELASTIC = 0, ADJ_PLASTIC = 1, ADJ_FCR = 0, ADJ_FCR_NH = 1, ADJ_ALL = 2 };
int adjoint_occupancy(int pl, int el);

// recorded trajectory and reverse-pass buffers
struct AdjointStore {
    std::vector<float4 *> ckpt;     // ckpt[c]: records at recorded substep c * ckpt_every
    float4 *tape = nullptr;         // ckpt_every states of one segment
    size_t tape_states = 0;
    float4 *adj[2] = {nullptr, nullptr};   // adjoint state (x v C F) per particle, 6 float4
    float4 *gpar = nullptr;         // parameter gradients per particle (log E, nu, yield, 0)
    float4 *gbar = nullptr;         // grid adjoint pool
    float4 *final_state = nullptr;  // recorded end state, restored after the reverse pass
    float *frames = nullptr;        // staged dL/dx
    size_t frames_bytes = 0;
    long long cap = 0;              // particle capacity the checkpoints were sized for
    long long cap_adj = 0;          // particle capacity of adj / gpar / final_state
    long long tape_cap = 0;         // particle capacity of the tape
    unsigned pool = 0;              // grid-adjoint pool capacity (blocks)
    // frame injection driven from device memory (so that one captured
    // segment graph serves every segment): per substep the first frame
    // adjoint to add, per frame the next one at the same substep, and the
    // current segment's first substep and dL/dx base
    int *frame_first = nullptr;     // recorded substeps + 1 entries
    int *frame_next = nullptr;      // frames
    long long frame_cap = 0, frame_first_cap = 0;
    void *seg = nullptr;            // device SegParams
    // grid tape: for every state of a segment its records, binning, counters
    // and grid, kept from the segment's recompute so that a reverse substep
    // runs only its adjoint kernels.  Two banks, so that the recompute of the
    // next segment (on `side`) overlaps the reverse of the current one.  One
    // allocation: a 256-byte header (word 0: grid-pool overflow flag), then
    // bank 0's gt_bank_states slots, then bank 1's, gt_slot_bytes each (layout
    // in gt_layout).  gt_pool: grid-pool blocks per slot; gt_shape: particle
    // capacity, chunk capacity, total blocks and gt_pool it was sized for.
    char *gt = nullptr;
    size_t gt_slot_bytes = 0, gt_bank_states = 0;
    unsigned gt_pool = 0;
    unsigned gt_pool_want = 0;      // grid-pool blocks per slot after an overflow
    long long gt_shape[4] = {0, 0, 0, 0};
    long long gt_gen = 0;           // counts grid-tape allocations (part of the graph keys)
    long long gt_reruns = 0;        // reverse passes run again after a grid-tape overflow
    bool strict = false;            // the reverse pass is being captured by the caller: no reruns
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // CUDA graphs of the reverse pass's steps, keyed by their shape (segment
    // lengths, banks, adjoint parity) and buffers; least recently used replaced
    static constexpr int NGRAPH = 6;
    static constexpr int NKEY = 14;
    cudaGraphExec_t seg_graph[NGRAPH] = {};
    long long seg_key[NGRAPH][NKEY] = {};
    long long seg_launches[NGRAPH] = {};
    long long seg_used[NGRAPH] = {};
    long long seg_clock = 0;
};
void free_adjoint(AdjointStore &a);

}  // namespace mpm

struct mpm_ctx {
    int device = 0;
    int sm_count = 0;
    int R[3];
    float dx, dt, g[3];
    mpm_options opt;
    std::vector<mpm_material> table;
    mpm::Dev D;
    float *mE = nullptr, *mnu = nullptr, *mrho = nullptr, *myield = nullptr, *malpha = nullptr;
    int *mel = nullptr, *mpl = nullptr;
    long long cap = 0;            // particle capacity
    long long total_blocks = 0;
    unsigned pool_blocks = 0;     // allocated grid pool capacity (blocks)
    unsigned chunk_cap = 0;
    void *stage = nullptr;        // staging for host inputs / outputs
    size_t stage_bytes = 0;
    bool loaded = false;
    mpm_status sticky = MPM_OK;
    std::string msg;
    int grid_sub[3] = {0, 0, 0};
    int grid_small = 0;
    int grid_adj = 0;             // reverse G2P / P2G kernels: SMs x resident CTAs per SM
    int adj_pl = 2;               // plasticity of the reverse G2P kernel (ADJ_*)
    int adj_el = 2;               // elasticity of the reverse P2G kernel (ADJ_*)
    long long recorded = 0;       // substeps recorded since the last load / reset
    bool record_broken = false;
    mpm::AdjointStore adj;
    // tracing: kernel launch count, and CUDA event pairs around substep kernels
    long long launches = 0;
    bool trace_on = false;
    std::vector<cudaEvent_t> trace_ev[3];   // per substep mode: start, end, start, end, ...
    size_t trace_used[3] = {0, 0, 0};
    // CUDA graph of two steady-state substeps (one per grid-buffer parity)
    bool use_graph = true;
    cudaStream_t cap_stream = nullptr;   // library-owned stream the graph is captured on
    cudaGraphExec_t graph2 = nullptr;
    long long graph_key = -1;     // (n, buffer generation) the graph was captured for
    long long generation = 0;     // bumped whenever a device buffer the kernels use is reallocated
    bool bins_pending = false;    // a binning (counts / occupied list) awaits its plan
    // direct binning of the steady-state forward substeps: its lists are
    // sized at each load (outside a capture) from the load's binning
    bool direct_ready = false;
    size_t slist_alloc = 0, ovf_alloc = 0, chunksd_alloc = 0, occd_alloc = 0;   // elements per buffer
    // BGDO key frames (records of the whole particle set) and stage-2 scratch
    float4 *snap[MPM_MAX_SNAPSHOTS] = {};
    long long snap_n[MPM_MAX_SNAPSHOTS] = {};     // particle count at the snapshot (0: empty)
    long long snap_cap[MPM_MAX_SNAPSHOTS] = {};
    float4 *bgdo_work = nullptr;   // pseudo-substep state
    long long bgdo_cap = 0;
    float *bgdo_G = nullptr;       // per-particle accumulator
    double *bgdo_sum = nullptr;    // per-material sum and count (2 * n_materials)
    // rest covariance of each particle's Gaussian kernel (n x 6)
    float *cov0 = nullptr;
    long long cov_n = 0, cov_cap = 0;
};

namespace mpm {
// kernel launches through these wrappers are counted (and the substep kernel
// timed when tracing is on)
// plan of the current grouping; opens fresh epochs for the buffers in bump_mask
void L_plan(mpm_ctx *ctx, int bump_mask, cudaStream_t st);
// grid update of upd_par, activation of act_par, sorted index (see k_prepare)
void L_prepare(mpm_ctx *ctx, int upd_par, int act_par, int do_sort, cudaStream_t st, int keep_momentum = 0);
// direct: bin straight into the scatter buffer's lists (fused mode); in_par
// >= 0: read the work items of the direct binning into buffer in_par
void L_substep(mpm_ctx *ctx, int mode, int gpar, int spar, cudaStream_t st, bool direct = false, int in_par = -1);
void L_between(mpm_ctx *ctx, int upd, int act, cudaStream_t st);
void L_bin(mpm_ctx *ctx, cudaStream_t st);
void launch_bgdo_accum(const Dev &D, const float4 *key, const float4 *post, int first, float inv_k,
                       float delta_target, float w, float *G, float *g_tau, float *delta, cudaStream_t st);
void launch_bgdo_material_sum(const Dev &D, int n_mat, const float *G, double *sum, cudaStream_t st);
void launch_bgdo_finish(const Dev &D, int n_mat, const float *G, const double *sum, float *Gout, float *logE,
                        cudaStream_t st);
void launch_covariance(const Dev &D, const float *cov0, float *out, cudaStream_t st);
void launch_reduce_by_material(const Dev &D, int n_mat, const float *per_particle, float *out, cudaStream_t st);
mpm_status ensure_chunks(mpm_ctx *ctx);
// re-bins the records D.rec points at (after the bins of another state)
void rebin(mpm_ctx *ctx, cudaStream_t st);
// a copy of the particle records taken once `state` substeps of a run are done
// (1 <= state < n_sub), in increasing order of state
struct StateCopy {
    int state;
    float4 *dst;
};
mpm_status run_substeps(mpm_ctx *ctx, int n_sub, cudaStream_t st, float4 *tape = nullptr, size_t tape_stride = 0,
                        const std::vector<StateCopy> *copies = nullptr);
// whether run_substeps bins directly for a run of n_sub substeps without a tape
bool direct_forward(const mpm_ctx *ctx, int n_sub);
mpm_status record_substeps(mpm_ctx *ctx, int n_sub, cudaStream_t st);
mpm_status ctx_fail(mpm_ctx *ctx, mpm_status s, const std::string &m);
mpm_status ctx_check(mpm_ctx *ctx, cudaStream_t st);
bool is_device_ptr(const void *p);
// the stream is being captured into a CUDA graph (by the caller)
bool stream_capturing(cudaStream_t st);
}  // namespace mpm
