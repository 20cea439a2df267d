// mpm_forward.cu -- forward kernels of the MLS-MPM substep.
//
// Pipeline of one call advancing S substeps (grid buffers alternate by
// parity; particles are grouped by their 4x4x4 grid block at the start):
//   plan -> activate/sort -> P2G(x_0)
//   repeat: grid update(s) -> [activate(s+1) -> G2P(s) fused with P2G(s+1)
//           -> plan -> sort]            ... last substep: G2P(S-1) only
// The fused kernel reads each particle once per substep: it gathers the
// grid velocity at x_s, updates x, v, C, F (and applies the return map),
// evaluates the stress of the new F and scatters mass and momentum at x_{s+1}
// into a shared-memory tile, then bins the particle for the next substep.
// Without a tape the forward bins directly from substep 1 on: the fused
// kernel writes each particle's index into the list of its new block (at
// the block's pool slot), and k_between (grid update, chunks from the list
// counts, activation of the next buffer) replaces plan and sort:
//   ... -> [k_between(s) -> G2P(s) fused with P2G(s+1) + list write] -> ...
#include "mpm_dev.cuh"
#include "mpm_internal.h"
#include "mpm_math.cuh"

namespace mpm {

// ---------------------------------------------------------------------------
// particle load: caller arrays -> records
// ---------------------------------------------------------------------------
__global__ void k_load(Dev D, const float *__restrict__ x, const float *__restrict__ v, const float *__restrict__ C,
                       const float *__restrict__ F, const float *__restrict__ vol, const int *__restrict__ mat,
                       const int *__restrict__ inst, const float *__restrict__ params, MatTable T) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < D.n; p += gridDim.x * blockDim.x) {
        int m = mat[p];
        int in = inst ? inst[p] : 0;
        if (m < 0 || m >= T.n || in < 0 || in >= D.n_inst) {
            set_err(D, ERRB_DOMAIN);
            m = m < 0 ? 0 : (m >= T.n ? T.n - 1 : m);
            in = in < 0 ? 0 : (in >= D.n_inst ? D.n_inst - 1 : in);
        }
        float E = T.E[m], nu = T.nu[m], ys = T.yield[m];
        if (params) {
            E = expf(params[3 * p]);
            nu = params[3 * p + 1];
            ys = params[3 * p + 2];
        }
        // Lame parameters (App. B.1)
        float mu = E / (2.f * (1.f + nu));
        float lam = E * nu / ((1.f + nu) * (1.f - 2.f * nu));
        float vp = vol[p];
        float c[9], f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            c[i] = C ? C[9 * p + i] : 0.f;
            f[i] = F ? F[9 * p + i] : ((i % 4 == 0) ? 1.f : 0.f);
        }
        // every input the substep reads must be finite: a NaN would otherwise be
        // dropped silently by the fixed-point scatter instead of reported
        bool fin = isfinite(x[3 * p]) && isfinite(x[3 * p + 1]) && isfinite(x[3 * p + 2]) && isfinite(vp) &&
                   isfinite(mu) && isfinite(lam) && isfinite(ys);
        // fixed-point position: cells = x / dx, rounded to 2^-qf of a cell
        // (exact for FP32 inputs away from the origin); beyond +-2^30 units it
        // saturates, and the binning reports the particle as out of the domain
        int q[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double u = (double)x[3 * p + d] / (double)D.dx * (double)D.q_cell;
            u = isfinite(u) ? fmin(fmax(u, -1073741824.0), 1073741824.0) : 0.0;
            q[d] = (int)llrint(u);
        }
        if (v) fin = fin && isfinite(v[3 * p]) && isfinite(v[3 * p + 1]) && isfinite(v[3 * p + 2]);
#pragma unroll
        for (int i = 0; i < 9; ++i) fin = fin && isfinite(c[i]) && isfinite(f[i]);
        if (!fin) set_err(D, ERRB_NONFINITE);
        int info = T.elastic[m] | (T.plastic[m] << 4) | (m << 8);
        float4 *r = D.rec + (size_t)p * REC_F4;
        r[0] = make_float4(__int_as_float(q[0]), __int_as_float(q[1]), __int_as_float(q[2]), T.rho[m] * vp);
        r[1] = v ? make_float4(v[3 * p], v[3 * p + 1], v[3 * p + 2], vp) : make_float4(0.f, 0.f, 0.f, vp);
        r[2] = make_float4(c[0], c[1], c[2], c[3]);
        r[3] = make_float4(c[4], c[5], c[6], c[7]);
        r[4] = make_float4(c[8], f[0], f[1], f[2]);
        r[5] = make_float4(f[3], f[4], f[5], f[6]);
        r[6] = make_float4(f[7], f[8], mu, lam);
        r[7] = make_float4(ys, __int_as_float(info), __int_as_float(in), T.alpha[m]);
    }
}

// ---------------------------------------------------------------------------
// binning helpers
// ---------------------------------------------------------------------------

// Particle block key from its fixed-point position; false when the stencil
// leaves the grid.
__device__ __forceinline__ bool particle_key(const Dev &D, int q0, int q1, int q2, int inst, unsigned &key) {
    float f;
    int b0 = base_cell_q(q0, D, f), b1 = base_cell_q(q1, D, f), b2 = base_cell_q(q2, D, f);
    bool ok = b0 >= 0 && b1 >= 0 && b2 >= 0 && b0 <= D.R[0] - 3 && b1 <= D.R[1] - 3 && b2 <= D.R[2] - 3;
    if (!ok) {   // keep the index in range; the error bit makes the result void
        b0 = min(max(b0, 0), D.R[0] - 3);
        b1 = min(max(b1, 0), D.R[1] - 3);
        b2 = min(max(b2, 0), D.R[2] - 3);
    }
    key = block_key(D, inst, b0 >> 2, b1 >> 2, b2 >> 2);
    return ok;
}

// Warp-aggregated counting: lanes with equal keys share one atomic; the first
// particle of a block appends the block to the occupied list.  All lanes in
// `mask` must call both halves together.  bin_begin issues the atomic;
// bin_end consumes its result, so work placed between them hides its latency.
struct BinTicket {
    unsigned peers, base, key;
};
__device__ __forceinline__ BinTicket bin_begin(const Dev &D, unsigned mask, unsigned key) {
    BinTicket t;
    t.key = key;
    t.peers = __match_any_sync(mask, key);
    t.base = 0;
    if ((int)(threadIdx.x & 31) == __ffs(t.peers) - 1) t.base = atomicAdd(&D.bcount[key], (unsigned)__popc(t.peers));
    return t;
}
__device__ __forceinline__ void bin_end(const Dev &D, const BinTicket &t, unsigned p) {
    const int leader = __ffs(t.peers) - 1;
    if ((int)(threadIdx.x & 31) == leader && t.base == 0) {
        unsigned slot = atomicAdd(&D.ctr[CTR_N_OCC], 1u);
        D.occ[slot] = t.key;
    }
    const unsigned base = __shfl_sync(t.peers, t.base, leader);
    D.key[p] = t.key;
    D.rank[p] = base + __popc(t.peers & lanemask_lt());
}
__device__ __forceinline__ void bin_particle(const Dev &D, unsigned mask, unsigned p, unsigned key) {
    BinTicket t = bin_begin(D, mask, key);
    bin_end(D, t, p);
    // the largest block count (sizes the per-block lists of the direct binning)
    if ((int)(threadIdx.x & 31) == __ffs(t.peers) - 1) atomicMax(&D.ctr[CTR_MAX_COUNT], t.base + __popc(t.peers));
}

// Direct binning into the lists of grid buffer par: the particle of rank r in
// a block with pool slot sl goes to slist[par][sl * slist_cap + r]; one whose
// list is full (r >= slist_cap) or whose slot lies beyond the lists (or is not
// active, a broken grouping already reported) goes to an overflow entry.
__device__ __forceinline__ void bin_end_direct(const Dev &D, const BinTicket &t, unsigned p, int slot, int par) {
    const int leader = __ffs(t.peers) - 1;
    if ((int)(threadIdx.x & 31) == leader && t.base == 0) {
        const unsigned i = atomicAdd(&D.ctr[CTR_D_OCC + par], 1u);
        D.occd[par][i] = t.key;
    }
    const unsigned rank = __shfl_sync(t.peers, t.base, leader) + __popc(t.peers & lanemask_lt());
    if (slot >= 0 && (unsigned)slot < D.slist_blocks && rank < D.slist_cap) {
        D.slist[par][(size_t)slot * D.slist_cap + rank] = p;
    } else {
        const unsigned o = atomicAdd(&D.ctr[CTR_D_OVF + par], 1u);
        atomicAdd(&D.ctr[CTR_D_OVF_TOTAL], 1u);
        if (o < D.ovf_cap) {
            D.ovf[par][2 * (size_t)o] = p;
            D.ovf[par][2 * (size_t)o + 1] = t.key;
        } else {
            set_err(D, ERRB_CAPACITY);
        }
    }
}

__global__ void k_bin(Dev D) {
    int stride = gridDim.x * blockDim.x;
    for (int p0 = blockIdx.x * blockDim.x; p0 < D.n; p0 += stride) {
        int p = p0 + threadIdx.x;
        bool valid = p < D.n;
        unsigned mask = __ballot_sync(0xffffffffu, valid);
        if (!valid) continue;
        float4 r0 = D.rec[(size_t)p * REC_F4];
        int inst = __float_as_int(D.rec[(size_t)p * REC_F4 + 7].z);
        unsigned key;
        if (!particle_key(D, rec_q(r0.x), rec_q(r0.y), rec_q(r0.z), inst, key)) set_err(D, ERRB_DOMAIN);
        bin_particle(D, mask, (unsigned)p, key);
    }
}

// ---------------------------------------------------------------------------
// plan: one CTA scans the occupied blocks -> block starts and work chunks
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_scan2(unsigned a, unsigned b, unsigned &ea, unsigned &eb, unsigned &ta,
                                            unsigned &tb, unsigned *sh) {
    // exclusive scan of (a, b) over a 1024-thread CTA; sh: 64 unsigned
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned ya = __shfl_up_sync(0xffffffffu, ia, o), yb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += ya; ib += yb; }
    }
    if (lane == 31) { sh[w] = ia; sh[32 + w] = ib; }
    __syncthreads();
    if (w == 0) {
        unsigned sa = sh[lane], sb = sh[32 + lane];
        unsigned xa = sa, xb = sb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
            if (lane >= o) { xa += ya; xb += yb; }
        }
        sh[lane] = xa - sa;
        sh[32 + lane] = xb - sb;
        if (lane == 31) { sh[64] = xa; sh[65] = xb; }
    }
    __syncthreads();
    ea = sh[w] + ia - a;
    eb = sh[32 + w] + ib - b;
    ta = sh[64];
    tb = sh[65];
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_plan(Dev D, int bump_mask) {
    __shared__ unsigned sh[66];
    const unsigned n = D.ctr[CTR_N_OCC];
    const unsigned CH = (unsigned)D.chunk;
    unsigned total = 0, tchunks = 0;
    for (unsigned b0 = 0; b0 < n; b0 += blockDim.x) {
        unsigned i = b0 + threadIdx.x;
        unsigned key = 0, cnt = 0;
        if (i < n) {
            key = D.occ[i];
            cnt = D.bcount[key];
        }
        unsigned nch = (cnt + CH - 1) / CH;
        unsigned ec, ek, tc, tk;
        block_scan2(cnt, nch, ec, ek, tc, tk, sh);
        if (i < n) {
            unsigned start = total + ec;
            D.bstart[key] = start;
            D.plan[i] = key;
            D.bcount[key] = 0;
            for (unsigned j = 0; j < nch; ++j) {
                unsigned ci = tchunks + ek + j;
                if (ci < D.max_chunks) D.chunks[ci] = make_int4((int)key, (int)(start + j * CH), (int)min(CH, cnt - j * CH), 0);
                else set_err(D, ERRB_CAPACITY);
            }
        }
        total += tc;
        tchunks += tk;
    }
    if (threadIdx.x == 0) {
        D.ctr[CTR_N_PLAN] = n;
        D.ctr[CTR_N_CHUNKS] = min(tchunks, D.max_chunks);
        D.ctr[CTR_N_OCC] = 0;
        // open a fresh activation epoch for each grid buffer in bump_mask
        for (int par = 0; par < 2; ++par)
            if (bump_mask & (1 << par)) {
                const unsigned e = D.ctr[CTR_EPOCH] + 1;
                D.ctr[CTR_EPOCH] = e;
                D.ctr[CTR_EPOCH_OF + par] = e;
                D.ctr[CTR_N_ACTIVE + par] = 0;
            }
    }
}

// Activation of buffer par around the listed blocks under epoch ep, item i
// of items = 27 x blocks: the neighbour i % 27 of block i / 27, if inside the
// grid, takes the epoch and, the first time, a pool slot.  All lanes of a
// warp call it together (the slot counter is claimed once per warp).
__device__ __forceinline__ void activate_item(const Dev &D, const unsigned *blocks, unsigned i, unsigned items,
                                              int par, unsigned ep) {
    unsigned nk = 0;
    bool fresh = false;
    if (i < items) {
        const unsigned b = i / 27u, o = i - b * 27u;
        int inst, bx, by, bz;
        key_coords(D, blocks[b], inst, bx, by, bz);
        const int nx = bx + (int)(o / 9u) - 1, ny = by + (int)((o / 3u) % 3u) - 1, nz = bz + (int)(o % 3u) - 1;
        if (nx >= 0 && ny >= 0 && nz >= 0 && nx < D.NB[0] && ny < D.NB[1] && nz < D.NB[2]) {
            nk = block_key(D, inst, nx, ny, nz);
            fresh = atomicMax(&D.page_epoch[par][nk], ep) != ep;
        }
    }
    const unsigned slot = warp_claim(&D.ctr[CTR_N_ACTIVE + par], fresh ? 1u : 0u);
    if (fresh) {
        if (slot < D.max_active) {
            D.page[par][nk] = (int)slot;
            D.active[par][slot] = nk;
        } else {
            D.page[par][nk] = -1;
            set_err(D, ERRB_CAPACITY);
        }
    }
}

// ---------------------------------------------------------------------------
// one launch between two substep kernels, three independent parts:
//   * the grid update (App. A) of buffer upd_par: v = mv/m + dt g for m > 0,
//     then the walls; clears the momentum unless keep_momentum;
//   * activation in buffer act_par of the 3x3x3 block neighbourhood of every
//     occupied block of the current grouping (its epoch was opened by k_plan);
//   * the sorted particle index of the current grouping.
// upd_par / act_par < 0 skip a part.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void apply_walls(const Dev &D, int I, int J, int K, float &u0, float &u1, float &u2) {
    int idx[3] = {I, J, K};
    bool sticky = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (idx[d] < D.bound && D.wall[2 * d] == 2) sticky = true;
        if (idx[d] >= D.R[d] - D.bound && D.wall[2 * d + 1] == 2) sticky = true;
    }
    if (sticky) { u0 = u1 = u2 = 0.f; return; }
    float *u[3] = {&u0, &u1, &u2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (idx[d] < D.bound && D.wall[2 * d] == 1 && *u[d] < 0.f) *u[d] = 0.f;
        if (idx[d] >= D.R[d] - D.bound && D.wall[2 * d + 1] == 1 && *u[d] > 0.f) *u[d] = 0.f;
    }
}

__global__ void k_prepare(Dev D, int upd_par, int act_par, int do_sort, int keep_momentum) {
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    // each warp takes one kind of item (a grid node, an activation neighbour,
    // a particle to sort), ranges rounded up to whole warps: no thread chains
    // the dependent loads of several parts
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lim = upd_par >= 0 ? min(D.ctr[CTR_N_ACTIVE + upd_par], D.max_active) * BLK_NODES : 0u;
    const unsigned n_act = act_par >= 0 ? D.ctr[CTR_N_PLAN] * 27u : 0u;
    const unsigned n_sort = do_sort ? (unsigned)D.n : 0u;
    const unsigned e0 = (lim + 31u) & ~31u, e1 = e0 + ((n_act + 31u) & ~31u), e2 = e1 + ((n_sort + 31u) & ~31u);
    const unsigned ep_act = act_par >= 0 ? D.ctr[CTR_EPOCH_OF + act_par] : 0u;
    for (unsigned w0 = tid - lane; w0 < e2; w0 += stride) {
        if (w0 < e0) {   // grid update of upd_par
            const unsigned i = w0 + lane;
            if (i >= lim) continue;
            const unsigned slot = i >> 6, l = i & 63u;
            int inst, bx, by, bz;
            key_coords(D, D.active[upd_par][slot], inst, bx, by, bz);
            const int I = bx * BLK + (int)(l >> 4), J = by * BLK + (int)((l >> 2) & 3u), K = bz * BLK + (int)(l & 3u);
            const float4 a = D.gmv[upd_par][i];
            float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
            if (a.w > 0.f) {
                const float im = 1.f / a.w;
                float u0 = a.x * im + D.dt * D.g[0], u1 = a.y * im + D.dt * D.g[1], u2 = a.z * im + D.dt * D.g[2];
                apply_walls(D, I, J, K, u0, u1, u2);
                out = make_float4(u0, u1, u2, a.w);
            }
            D.gv[upd_par][i] = out;
            if (!keep_momentum) D.gmv[upd_par][i] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (w0 < e1) {   // activation of act_par: one neighbour of a planned block
            activate_item(D, D.plan, w0 - e0 + lane, n_act, act_par, ep_act);
        } else {   // the sorted index
            const unsigned p = w0 - e1 + lane;
            if (p < n_sort) D.sorted[D.bstart[D.key[p]] + D.rank[p]] = p;
        }
    }
}

// ---------------------------------------------------------------------------
// between two substeps of direct binning (one launch, no scan and no sort):
//   * the grid update of buffer upd, which the last substep's scatter filled
//     (App. A: v = mv/m + dt g, walls), clearing its momentum;
//   * the work items of the binning that substep made: each occupied block's
//     list (at its pool slot in upd) in items of <= chunk particles, and one
//     item per overflow entry;
//   * the activation of buffer act (< 0: none) around the occupied blocks, for
//     the next scatter, under a fresh epoch: EPOCH_OF[upd] + 1, above every
//     epoch either buffer holds (upd's is the latest opened).
// The counters it reads are not written in this launch; thread 0 of CTA 0
// resets the ones the next substep's binning starts from.
// ---------------------------------------------------------------------------
__global__ void k_between(Dev D, int upd, int act) {
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    const unsigned nocc = D.ctr[CTR_D_OCC + upd];
    const unsigned novf = min(D.ctr[CTR_D_OVF + upd], D.ovf_cap);
    const unsigned ep_upd = D.ctr[CTR_EPOCH_OF + upd];
    const unsigned ep_new = ep_upd + 1u;
    const unsigned CH = (unsigned)D.chunk;
    if (tid == 0) {
        D.ctr[CTR_N_PLAN] = nocc;
        if (act >= 0) {
            D.ctr[CTR_EPOCH] = ep_new;
            D.ctr[CTR_EPOCH_OF + act] = ep_new;
            D.ctr[CTR_D_OCC + act] = 0;
            D.ctr[CTR_D_OVF + act] = 0;
        }
    }
    // Each warp takes one kind of item, so that no thread chains the
    // dependent loads of several: the grid update of upd (one node), the
    // lists of the occupied blocks (one block), the overflow entries (one
    // entry) and the activation of act around the occupied blocks (one
    // neighbour).  The ranges are rounded up to whole warps, and the
    // counters are claimed once per warp.
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lim = min(D.ctr[CTR_N_ACTIVE + upd], D.max_active) * BLK_NODES;
    const unsigned e0 = (lim + 31u) & ~31u, e1 = e0 + ((nocc + 31u) & ~31u), e2 = e1 + ((novf + 31u) & ~31u);
    const unsigned e3 = e2 + (act >= 0 ? (nocc * 27u + 31u) & ~31u : 0u);
    for (unsigned w0 = tid - lane; w0 < e3; w0 += stride) {
        if (w0 < e0) {   // grid update of upd
            const unsigned i = w0 + lane;
            if (i >= lim) continue;
            const unsigned slot = i >> 6, l = i & 63u;
            int inst, bx, by, bz;
            key_coords(D, D.active[upd][slot], inst, bx, by, bz);
            const int I = bx * BLK + (int)(l >> 4), J = by * BLK + (int)((l >> 2) & 3u), K = bz * BLK + (int)(l & 3u);
            const float4 a = D.gmv[upd][i];
            float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
            if (a.w > 0.f) {
                const float im = 1.f / a.w;
                float u0 = a.x * im + D.dt * D.g[0], u1 = a.y * im + D.dt * D.g[1], u2 = a.z * im + D.dt * D.g[2];
                apply_walls(D, I, J, K, u0, u1, u2);
                out = make_float4(u0, u1, u2, a.w);
            }
            D.gv[upd][i] = out;
            D.gmv[upd][i] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (w0 < e1) {   // work items: the list of an occupied block
            const unsigned i = w0 - e0 + lane;
            unsigned key = 0, main = 0;
            int sl = -1;
            if (i < nocc) {
                key = D.occd[upd][i];
                const unsigned cnt = D.bcount[key];
                D.bcount[key] = 0;
                sl = D.page_epoch[upd][key] == ep_upd ? D.page[upd][key] : -1;
                main = (sl >= 0 && (unsigned)sl < D.slist_blocks) ? min(cnt, D.slist_cap) : 0u;
            }
            const unsigned nch = (main + CH - 1) / CH;
            const unsigned c0 = warp_claim(&D.ctr[CTR_D_CH + upd], nch);
            for (unsigned j = 0; j < nch; ++j) {
                if (c0 + j < D.max_chunks_d)
                    D.chunksd[upd][c0 + j] = make_int4((int)key, (int)((unsigned)sl * D.slist_cap + j * CH),
                                                       (int)min(CH, main - j * CH), 0);
                else
                    set_err(D, ERRB_CAPACITY);
            }
        } else if (w0 < e2) {   // one work item per overflow entry (list 1)
            const unsigned o = w0 - e1 + lane;
            const unsigned c = warp_claim(&D.ctr[CTR_D_CH + upd], o < novf ? 1u : 0u);
            if (o >= novf) continue;
            if (c < D.max_chunks_d) D.chunksd[upd][c] = make_int4((int)D.ovf[upd][2 * o + 1], (int)(2 * o), 1, 1);
            else set_err(D, ERRB_CAPACITY);
        } else {   // activation of act: one neighbour of an occupied block
            activate_item(D, D.occd[upd], w0 - e2 + lane, nocc * 27u, act, ep_new);
        }
    }
}

// ---------------------------------------------------------------------------
// the substep kernel
//   MODE_P2G: scatter at the current positions (first substep of a call)
//   MODE_FUSED: G2P(s) + update + return map + stress + P2G(s+1) + binning
//   MODE_G2P: G2P(s) + update + return map + binning (last substep)
//
// One CTA works on one chunk (<= TPB particles of one 4^3-node block) at a
// time, one particle per thread, and software-pipelines the chunks it owns
// (c, c + G, c + 2G, ... for grid size G):
//   0. staging arrives ahead of use through cp.async copies into shared
//      memory.  While chunk c is processed, the descriptor of chunk c + 2G,
//      and the sorted indices and page-table words of chunk c + G are copied
//      (issued before phase A); the records of chunk c + G (warp-coalesced:
//      each copy instruction moves four whole 128-byte records) and the grid
//      velocities of its 6^3-node gather tile (issued after phase A, when
//      those buffers are free) arrive during phases B and flush.  No thread
//      waits on a dependent global load at the start of a chunk;
//   A. per particle: gather v and C (App. A G2P), x += dt v, F <- (I + dt C) F,
//      one SVD serving the return map and the next stress, Kirchhoff stress,
//      affine momentum A = m C - 4 dt V tau / dx^2 (§4.2); the new record goes
//      to global memory and a 16-float scatter packet replaces the staged
//      record; the particle is binned for the next substep;
//   B. packets are scattered into the 8^3-node tile (nodes 4B-1 .. 4B+6) and
//      the tile is flushed with one vector reduction per touched node.  With
//      the fixed-point tile the warps take the packets ordered by (rank
//      within bank, bank of the base node): one loop iteration moves every
//      lane by the same node offset, so lanes with distinct base banks hit
//      distinct banks in all 108 atomics, and the first warps of a chunk see
//      at most two-way conflicts.
// SCAT selects the scatter of phase B: 0 = float shared-memory atomics;
// 1 = int32 fixed-point shared-memory atomics with a per-chunk scale (native
// integer atomics; the scale keeps the rounding below 2^-30 of the chunk's
// total per quantity); 2 = vector reductions straight into the global grid.
// ---------------------------------------------------------------------------
enum { MODE_P2G = 0, MODE_FUSED = 1, MODE_G2P = 2 };

constexpr int GT = 6;    // gather tile edge (nodes 4B .. 4B+5)
constexpr int GT3 = GT * GT * GT;
constexpr int ST = 8;    // scatter tile edge (nodes 4B-1 .. 4B+6)
constexpr int ST3 = ST * ST * ST;
constexpr int STP = ST + 1;            // padded row of the fixed-point tile (breaks bank aliasing)
constexpr int ST3P = ST * ST * STP;
constexpr int CH_MAX = 128;            // particles per chunk (one per thread)
__device__ __forceinline__ int tidx(int i, int j, int k) { return (i * ST + j) * STP + k; }

__device__ __forceinline__ int page_slot(const Dev &D, int par, unsigned ep, int inst, int bx, int by, int bz) {
    if (bx < 0 || by < 0 || bz < 0 || bx >= D.NB[0] || by >= D.NB[1] || bz >= D.NB[2]) return -1;
    unsigned k = block_key(D, inst, bx, by, bz);
    // both words are loaded before either is tested: one round trip
    const unsigned e = D.page_epoch[par][k];
    const int sl = D.page[par][k];
    return e == ep ? sl : -1;
}

__device__ __forceinline__ int node_local(int I, int J, int K) { return ((I & 3) * 4 + (J & 3)) * 4 + (K & 3); }

constexpr int PK_F4 = 5;          // scatter packet: X(3) m | P(3) - | Ad(9) (+3 spare)
constexpr int RS_F4 = REC_F4 + 1; // staged record stride: 144 B keeps per-thread float4 reads conflict-free
template <int TPB> struct SubstepSmem {
    float4 rec[TPB * RS_F4];         // the chunk's records, staged ahead of use
    float4 pk[TPB * PK_F4];          // scatter packets of the chunk's particles
    float4 g[GT3];                   // gather tile: (v, m) per node
    union {
        float f[4 * ST3P];           // scatter tile, component-major [m0 | m1 | m2 | m], padded rows
        int i[4 * ST3P];
    } t;
    int4 cd[3];                      // chunk descriptors, ring of (c, c + G, c + 2G)
    unsigned pidx[TPB];              // sorted particle indices of the next chunk
    unsigned pe[35];                 // page-table words of the next chunk: epoch ...
    int ps[35];                      // ... and pool slot; 0..26 scatter blocks, 27..34 gather blocks
    int slot_s[2][27];               // pool slot of blocks (B-1 .. B+1)^3 in the scatter grid, per chunk parity
    float red[2 * (TPB / 32)];
    float scale[2];
    int ccount[32];                  // packets per bank of their base node (scatter order)
    int ptab[TPB];                   // packets of rank < r
    unsigned mtab[TPB];              // banks holding a packet of rank r
    int prank[TPB], pcol[TPB];       // each packet's bank and rank within it
    int perm[TPB];                   // scatter order: packets by (rank, bank)
};

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- staging steps (every thread of the CTA calls them) ---------------------
// level 2: sorted indices of chunk ch and its page-table lookups: 27
// scatter-grid blocks (B-1 .. B+1)^3 and 8 gather-grid blocks (B .. B+1)^3,
// one per thread of the last two warps; a block outside the grid gets an
// epoch that never matches
template <int TPB, bool GATHER, bool SCATTER>
__device__ __forceinline__ void stage_level2(const Dev &D, SubstepSmem<TPB> &S, int4 ch, int gpar, int spar,
                                             unsigned ep_g, unsigned ep_s) {
    const int tid = threadIdx.x;
    if (tid < ch.z) cp_async4(&S.pidx[tid], (ch.w ? D.ovf_in : D.sorted) + ch.y + tid);
    int inst, bx, by, bz;
    key_coords(D, (unsigned)ch.x, inst, bx, by, bz);
    const int t = tid - (TPB - 64 > 0 ? 64 : 0);    // the lookups go to the last warps of the CTA
    if (t >= 0 && t < 35 && (t < 27 ? SCATTER : GATHER)) {
        int qx, qy, qz, par;
        unsigned ep;
        if (t < 27) { qx = bx + t / 9 - 1; qy = by + (t / 3) % 3 - 1; qz = bz + t % 3 - 1; par = spar; ep = ep_s; }
        else { const int u = t - 27; qx = bx + (u >> 2); qy = by + ((u >> 1) & 1); qz = bz + (u & 1); par = gpar; ep = ep_g; }
        if (qx < 0 || qy < 0 || qz < 0 || qx >= D.NB[0] || qy >= D.NB[1] || qz >= D.NB[2]) {
            S.pe[t] = ep + 1u;
            S.ps[t] = -1;
        } else {
            const unsigned k = block_key(D, inst, qx, qy, qz);
            cp_async4(&S.pe[t], D.page_epoch[par] + k);
            cp_async4(&S.ps[t], D.page[par] + k);
        }
    }
}

// level 3: the chunk's records (warp-coalesced: instruction w of a warp moves
// float4 l % 8 of records 4 w + l / 8 of the warp's 32) and its gather tile.
// Needs the level-2 words of the chunk in shared memory.
template <int TPB, bool GATHER>
__device__ __forceinline__ void stage_level3(const Dev &D, SubstepSmem<TPB> &S, int4 ch, int gpar, unsigned ep_g) {
    const int tid = threadIdx.x, lane = tid & 31, wbase = tid & ~31;
    const int piece = lane & 7;
    if (!GATHER || (piece != 2 && piece != 3)) {   // G2P does not read the old C
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int j = wbase + 4 * w + (lane >> 3);
            if (j < ch.z) cp_async16(&S.rec[j * RS_F4 + piece], D.rec + (size_t)S.pidx[j] * REC_F4 + piece);
        }
    }
    if (GATHER) {
        int inst, bx, by, bz;
        key_coords(D, (unsigned)ch.x, inst, bx, by, bz);
        for (int t = tid; t < GT3; t += TPB) {
            const int i = t / (GT * GT), j = (t / GT) % GT, k = t % GT;
            const int b = 27 + (((i >> 2) << 2) | ((j >> 2) << 1) | (k >> 2));
            const int sl = S.pe[b] == ep_g ? S.ps[b] : -1;
            if (sl >= 0) cp_async16(&S.g[t], D.gv[gpar] + (size_t)sl * BLK_NODES + node_local(i, j, k));
            else S.g[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// pool slots of the scatter blocks from the level-2 words (threads 27 of the last warps)
template <int TPB>
__device__ __forceinline__ void stage_slots(SubstepSmem<TPB> &S, int buf, unsigned ep_s) {
    const int t = threadIdx.x - (TPB - 64 > 0 ? 64 : 0);
    if (t >= 0 && t < 27) S.slot_s[buf][t] = S.pe[t] == ep_s ? S.ps[t] : -1;
}

// TPB: threads per CTA = largest chunk (one particle per thread); 64 or 128.
// Both variants cap registers at 128 (16 warps per SM); the 64-thread one
// runs twice as many independent CTAs, which overlap each other's staging.
// DB (fused mode): the new binning goes straight into the scatter buffer's
// per-block lists (bin_end_direct) instead of keys and ranks for a sort.
// XM: the further constitutive models (StVK, Hencky, fluid, volume; fluid and
// Sigma plasticity).  Without it the kernel handles fixed-corotated and
// Neo-Hookean with von Mises / Drucker-Prager only, and its register
// allocation is not shared with the rarer models.
template <int MODE, int SCAT, int TPB, bool XM, bool DB>
__global__ void __launch_bounds__(TPB, 512 / TPB) k_substep(Dev D, int gpar, int spar) {
    extern __shared__ float4 smem_raw[];
    SubstepSmem<TPB> &S = *reinterpret_cast<SubstepSmem<TPB> *>(smem_raw);
    constexpr bool GATHER = MODE != MODE_P2G;
    constexpr bool SCATTER = MODE != MODE_G2P;
    if (DB && blockIdx.x == 0 && threadIdx.x == 0) {
        // counters this kernel does not read and the next launch starts from:
        // the activation count of the gather buffer (activated again next)
        // and the work items of the binning made now
        D.ctr[CTR_N_ACTIVE + gpar] = 0;
        D.ctr[CTR_D_CH + spar] = 0;
    }
    // the first two descriptors are read alongside the counters: any index
    // within the array's capacity is readable, and one beyond the count is
    // dropped below
    const unsigned cap_ch = D.chunk_ctr == CTR_N_CHUNKS ? D.max_chunks : D.max_chunks_d;
    int4 cd0 = make_int4(0, 0, 0, 0), cd1 = cd0;
    if (threadIdx.x == 0) {
        if (blockIdx.x < cap_ch) cd0 = D.chunks[blockIdx.x];
        if (blockIdx.x + gridDim.x < cap_ch) cd1 = D.chunks[blockIdx.x + gridDim.x];
    }
    const unsigned n_chunks = min(D.ctr[D.chunk_ctr], cap_ch);
    const unsigned ep_g = GATHER ? D.ctr[CTR_EPOCH_OF + gpar] : 0u;
    const unsigned ep_s = SCATTER ? D.ctr[CTR_EPOCH_OF + spar] : 0u;
    const float dx = D.dx, inv_dx = D.inv_dx, dt = D.dt;
    const int tid = threadIdx.x, T = TPB;
    unsigned c = blockIdx.x;
    if (c >= n_chunks) return;

    // prologue: descriptors of chunks c and c + G; levels 2 and 3 of chunk c
    if (tid == 0) {
        S.cd[0] = cd0;
        if (c + gridDim.x < n_chunks) S.cd[1] = cd1;
    }
    if (SCATTER && SCAT != 2)
        for (int t = tid; t < 4 * ST3P; t += T) S.t.i[t] = 0;
    if (tid < 32) S.ccount[tid] = 0;
    __syncthreads();
    stage_level2<TPB, GATHER, SCATTER>(D, S, S.cd[0], gpar, spar, ep_g, ep_s);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (SCATTER) stage_slots<TPB>(S, 0, ep_s);
    stage_level3<TPB, GATHER>(D, S, S.cd[0], gpar, ep_g);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    for (int kc = 0;; ++kc) {
        const int4 ch = S.cd[kc % 3];
        const int cnt = min(ch.z, TPB);
        const unsigned cn = c + gridDim.x;
        const bool has_next = cn < n_chunks;
        const unsigned p_cur = tid < cnt ? S.pidx[tid] : 0u;   // read before level 2 of c + G overwrites it
        // level 1 of chunk c + 2G and level 2 of chunk c + G, in flight during phase A
        if (tid == 0 && cn + gridDim.x < n_chunks) cp_async16(&S.cd[(kc + 2) % 3], D.chunks + cn + gridDim.x);
        if (has_next) stage_level2<TPB, GATHER, SCATTER>(D, S, S.cd[(kc + 1) % 3], gpar, spar, ep_g, ep_s);
        cp_async_commit();
        int inst, bx, by, bz;
        key_coords(D, (unsigned)ch.x, inst, bx, by, bz);
        const int ox = bx * BLK, oy = by * BLK, oz = bz * BLK;   // gather tile origin (node)
        const int rounds = 1;

        // ---- A. per-particle update -----------------------------------------
        float bnd_m = 0.f, bnd_v = 0.f;
        {
            const int j = tid;
            const bool valid = j < cnt;
            const unsigned lane_mask = __ballot_sync(0xffffffffu, valid);
            if (valid) {
            const unsigned p = p_cur;
            const float4 *nr = S.rec + j * RS_F4;
            float4 *sr = S.pk + j * PK_F4;
            const float4 r0 = nr[0], r1 = nr[1], r6 = nr[6], r7 = nr[7];
            int q[3] = {rec_q(r0.x), rec_q(r0.y), rec_q(r0.z)};
            const float mass = r0.w, vol = r1.w;
            float v[3] = {r1.x, r1.y, r1.z};
            const float mu = r6.z, lam = r6.w, yield = r7.x;
            const int info = __float_as_int(r7.y);
            const int elastic = info & 15, plastic = (info >> 4) & 15;
            float F[9], Cm[9], U[9], s3[3], e3[3];
            {
                const float4 r4 = nr[4], r5 = nr[5];
                F[0] = r4.y; F[1] = r4.z; F[2] = r4.w; F[3] = r5.x; F[4] = r5.y; F[5] = r5.z; F[6] = r5.w;
                F[7] = r6.x; F[8] = r6.y;
                Cm[8] = r4.x;
            }
            float4 *rp = D.rec + (size_t)p * REC_F4;
            unsigned key = 0;
            bool in_dom = true;
            BinTicket ticket;
            if (GATHER) {
                float f0, f1, f2;
                int b0 = base_cell_q(q[0], D, f0) - ox, b1 = base_cell_q(q[1], D, f1) - oy,
                    b2 = base_cell_q(q[2], D, f2) - oz;
                if ((unsigned)b0 > 3u || (unsigned)b1 > 3u || (unsigned)b2 > 3u) {   // grouping invariant broken
                    set_err(D, ERRB_CFL);
                    b0 = min(max(b0, 0), 3); b1 = min(max(b1, 0), 3); b2 = min(max(b2, 0), 3);
                }
                float w0[3], w1[3], w2[3];
                bspline_w(f0, w0);
                bspline_w(f1, w1);
                bspline_w(f2, w2);
                // separable sums over the 3x3x3 stencil: for each (i, j) the k-sums
                // S = sum_k w2 g and T = sum_k w2 (k - f2) g, then the j-sums, then
                // v = sum w g and Bm = sum w g (o - f)^T
                float vn[3] = {0.f, 0.f, 0.f};
                float Bm[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                const float wz1[3] = {w2[0] * (0.f - f2), w2[1] * (1.f - f2), w2[2] * (2.f - f2)};
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float Ui[3] = {0.f, 0.f, 0.f}, Vi[3] = {0.f, 0.f, 0.f}, Wi[3] = {0.f, 0.f, 0.f};
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) {
                        float Sij[3] = {0.f, 0.f, 0.f}, Tij[3] = {0.f, 0.f, 0.f};
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float4 g = S.g[((b0 + i) * GT + (b1 + jj)) * GT + (b2 + k)];
                            Sij[0] += w2[k] * g.x; Sij[1] += w2[k] * g.y; Sij[2] += w2[k] * g.z;
                            Tij[0] += wz1[k] * g.x; Tij[1] += wz1[k] * g.y; Tij[2] += wz1[k] * g.z;
                        }
                        const float wj = w1[jj], wjd = w1[jj] * ((float)jj - f1);
#pragma unroll
                        for (int r = 0; r < 3; ++r) { Ui[r] += wj * Sij[r]; Vi[r] += wjd * Sij[r]; Wi[r] += wj * Tij[r]; }
                    }
                    const float wi = w0[i], wid = w0[i] * ((float)i - f0);
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        vn[r] += wi * Ui[r];
                        Bm[3 * r] += wid * Ui[r];
                        Bm[3 * r + 1] += wi * Vi[r];
                        Bm[3 * r + 2] += wi * Wi[r];
                    }
                }
                // C = 4/dx^2 sum w v (x_i - x_p)^T with (x_i - x_p) = (o - f) dx
                const float cs = 4.f * inv_dx;
#pragma unroll
                for (int t = 0; t < 9; ++t) Cm[t] = cs * Bm[t];
#pragma unroll
                for (int d = 0; d < 3; ++d) { v[d] = vn[d]; q[d] = advance_q(q[d], vn[d], D); }
                if (!(isfinite(vn[0]) && isfinite(vn[1]) && isfinite(vn[2]))) set_err(D, ERRB_NONFINITE);
                in_dom = particle_key(D, q[0], q[1], q[2], inst, key);
                ticket = bin_begin(D, lane_mask, key);      // result consumed after the SVD
                rp[1] = make_float4(v[0], v[1], v[2], vol);
                rp[2] = make_float4(Cm[0], Cm[1], Cm[2], Cm[3]);
                rp[3] = make_float4(Cm[4], Cm[5], Cm[6], Cm[7]);
                // F <- (I + dt C) F
                float G[9];
#pragma unroll
                for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc)
                        G[3 * rr + cc] = F[3 * rr + cc] + dt * (Cm[3 * rr] * F[cc] + Cm[3 * rr + 1] * F[3 + cc] +
                                                                Cm[3 * rr + 2] * F[6 + cc]);
                if (XM && plastic >= PLASTIC_FLUID) {
                    // volume-only plasticity: F = c I, whose SVD is U = V = I, s = c
                    const float cm1 = volume_plastic(plastic, G);
#pragma unroll
                    for (int t = 0; t < 9; ++t) U[t] = (t % 4 == 0) ? 1.f : 0.f;
#pragma unroll
                    for (int t = 0; t < 3; ++t) { s3[t] = 1.f + cm1; e3[t] = cm1; }
                } else if (plastic != PLASTIC_NONE || (SCATTER && (XM ? elastic_needs_svd(elastic) : elastic == 0))) {
                    // one SVD of the updated F serves the return map and the next stress
                    float Vv[9], d3[3];
                    const int fb = svd3_robust(G, U, Vv, s3, e3, d3);
                    if (fb) {
                        atomicAdd(&D.ctr[CTR_FALLBACKS], 1u);
                        if (fb == 2) set_err(D, ERRB_NONFINITE);
                    }
                    if (plastic != PLASTIC_NONE) {
                        const float alpha = r7.w;
                        float z[3], ze[3];
                        const int rm = return_map(plastic, s3, e3, d3, mu, lam, yield, alpha, z, ze);
                        if (rm != RM_ELASTIC) {
                            usvt(G, U, z, Vv);
#pragma unroll
                            for (int t = 0; t < 3; ++t) { s3[t] = z[t]; e3[t] = ze[t]; }
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < 9; ++t) F[t] = G[t];
                rp[0] = make_float4(__int_as_float(q[0]), __int_as_float(q[1]), __int_as_float(q[2]), mass);
                rp[4] = make_float4(Cm[8], F[0], F[1], F[2]);
                rp[5] = make_float4(F[3], F[4], F[5], F[6]);
                rp[6] = make_float4(F[7], F[8], mu, lam);
            } else {
                const float4 r2 = nr[2], r3 = nr[3];
                Cm[0] = r2.x; Cm[1] = r2.y; Cm[2] = r2.z; Cm[3] = r2.w;
                Cm[4] = r3.x; Cm[5] = r3.y; Cm[6] = r3.z; Cm[7] = r3.w;
                if (XM ? elastic_needs_svd(elastic) : elastic == 0) {
                    float Vv[9], d3[3];
                    const int fb = svd3_robust(F, U, Vv, s3, e3, d3);
                    if (fb) {
                        atomicAdd(&D.ctr[CTR_FALLBACKS], 1u);
                        if (fb == 2) set_err(D, ERRB_NONFINITE);
                    }
                }
            }

            if (!GATHER) in_dom = particle_key(D, q[0], q[1], q[2], inst, key);
            if (!in_dom) set_err(D, ERRB_DOMAIN);

            if (SCATTER) {
                // Kirchhoff stress of F (App. B.1 / App. A) and the affine momentum
                // A = m C - 4 dt V / dx^2 tau of the §4.2 equation, as Ad = A dx
                Sym tau;
                bool tau_ok = true;
                if (XM) tau_ok = kirchhoff(elastic, F, U, s3, e3, mu, lam, tau);
                else if (elastic == ELASTIC_FCR) tau = tau_fcr(U, s3, e3, mu, lam);
                else tau_ok = tau_nh(F, mu, lam, tau);
                if (!tau_ok) {
                    set_err(D, ERRB_NONFINITE);
                    tau = Sym{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                }
                const float kf = 4.f * dt * vol * inv_dx * inv_dx;
                float Ad[9];
                Ad[0] = (mass * Cm[0] - kf * tau.xx) * dx; Ad[1] = (mass * Cm[1] - kf * tau.xy) * dx;
                Ad[2] = (mass * Cm[2] - kf * tau.xz) * dx; Ad[3] = (mass * Cm[3] - kf * tau.xy) * dx;
                Ad[4] = (mass * Cm[4] - kf * tau.yy) * dx; Ad[5] = (mass * Cm[5] - kf * tau.yz) * dx;
                Ad[6] = (mass * Cm[6] - kf * tau.xz) * dx; Ad[7] = (mass * Cm[7] - kf * tau.yz) * dx;
                Ad[8] = (mass * Cm[8] - kf * tau.zz) * dx;
                const float P0 = mass * v[0], P1 = mass * v[1], P2 = mass * v[2];
                // tile-local continuous node coordinate of the new position (the
                // integer offset is taken off in fixed point; one rounding)
                const float X0 = (float)(q[0] - ((ox - 1) << D.qf)) * D.q_unit,
                            X1 = (float)(q[1] - ((oy - 1) << D.qf)) * D.q_unit,
                            X2 = (float)(q[2] - ((oz - 1) << D.qf)) * D.q_unit;
                // base cell floor(X - 0.5) in [0, ST-3] keeps the 3^3 stencil in the tile
                const bool in_tile = in_dom && X0 >= 0.5f && X1 >= 0.5f && X2 >= 0.5f && X0 < (float)ST - 1.5f &&
                                     X1 < (float)ST - 1.5f && X2 < (float)ST - 1.5f;
                float pm = mass;
                if (in_dom && !in_tile) {
                    // moved out of the tile: straight to the global grid
                    pm = 0.f;
                    float f0, f1, f2;
                    const int g0 = base_cell_q(q[0], D, f0), g1 = base_cell_q(q[1], D, f1),
                              g2 = base_cell_q(q[2], D, f2);
                    float w0[3], w1[3], w2[3];
                    bspline_w(f0, w0);
                    bspline_w(f1, w1);
                    bspline_w(f2, w2);
                    for (int i = 0; i < 3; ++i)
                        for (int jj = 0; jj < 3; ++jj)
                            for (int k = 0; k < 3; ++k) {
                                const float d0 = (float)i - f0, d1 = (float)jj - f1, d2 = (float)k - f2;
                                const float wt = w0[i] * w1[jj] * w2[k];
                                const int I = g0 + i, J = g1 + jj, K = g2 + k;
                                const int sl = page_slot(D, spar, ep_s, inst, I >> 2, J >> 2, K >> 2);
                                if (sl >= 0)
                                    red_add_v4(D.gmv[spar] + (size_t)sl * BLK_NODES + node_local(I, J, K),
                                               wt * (P0 + Ad[0] * d0 + Ad[1] * d1 + Ad[2] * d2),
                                               wt * (P1 + Ad[3] * d0 + Ad[4] * d1 + Ad[5] * d2),
                                               wt * (P2 + Ad[6] * d0 + Ad[7] * d1 + Ad[8] * d2), wt * mass);
                                else
                                    set_err(D, ERRB_CFL);
                            }
                } else if (!in_dom) {
                    pm = 0.f;
                }
                if (SCAT == 1) {
                    bnd_m += pm;
                    float am = fmaxf(fabsf(Ad[0]), fmaxf(fabsf(Ad[1]), fabsf(Ad[2])));
                    am = fmaxf(am, fmaxf(fabsf(Ad[3]), fmaxf(fabsf(Ad[4]), fabsf(Ad[5]))));
                    am = fmaxf(am, fmaxf(fabsf(Ad[6]), fmaxf(fabsf(Ad[7]), fabsf(Ad[8]))));
                    const float ap = fmaxf(fabsf(P0), fmaxf(fabsf(P1), fabsf(P2)));
                    bnd_v += pm > 0.f ? ap + 4.5f * am : 0.f;
                }
                sr[0] = make_float4(X0, X1, X2, pm);
                sr[1] = make_float4(P0, P1, P2, 0.f);
                sr[2] = make_float4(Ad[0], Ad[1], Ad[2], Ad[3]);
                sr[3] = make_float4(Ad[4], Ad[5], Ad[6], Ad[7]);
                sr[4] = make_float4(Ad[8], 0.f, 0.f, 0.f);
            }
            if (DB) {
                // pool slot of the new block in the scatter buffer: one of the
                // chunk block's 27 neighbours (a particle moves at most a cell)
                float fq;
                const int d0 = (base_cell_q(q[0], D, fq) >> 2) - bx + 1, d1 = (base_cell_q(q[1], D, fq) >> 2) - by + 1,
                          d2 = (base_cell_q(q[2], D, fq) >> 2) - bz + 1;
                const bool near = (unsigned)d0 < 3u && (unsigned)d1 < 3u && (unsigned)d2 < 3u;
                // beyond the neighbourhood (a broken grouping, already reported)
                // the page table is read, as k_between reads it for the block
                const int slot = near ? S.slot_s[kc & 1][(d0 * 3 + d1) * 3 + d2]
                                      : (D.page_epoch[spar][key] == ep_s ? D.page[spar][key] : -1);
                bin_end_direct(D, ticket, p, slot, spar);
            } else if (MODE != MODE_P2G) {
                bin_end(D, ticket, p);
            }
            }
        }

        if (SCATTER && SCAT == 1 && tid < cnt) {
            // bank of the packet's base node: every node of its stencil is the
            // base plus an offset common to all packets in one loop iteration,
            // and the tile's component stride is a multiple of 32 banks
            const float4 q = S.pk[tid * PK_F4];
            int col = 0;
            if (q.w > 0.f)
                col = tidx((int)floorf(q.x - 0.5f), (int)floorf(q.y - 0.5f), (int)floorf(q.z - 0.5f)) & 31;
            S.pcol[tid] = col;
            S.prank[tid] = atomicAdd(&S.ccount[col], 1);
        }
        if (SCATTER && SCAT == 1) {
            // per-chunk fixed-point scales from the sums of the per-particle bounds
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                bnd_m += __shfl_xor_sync(0xffffffffu, bnd_m, o);
                bnd_v += __shfl_xor_sync(0xffffffffu, bnd_v, o);
            }
            if ((tid & 31) == 0) { S.red[tid >> 5] = bnd_m; S.red[(TPB / 32) + (tid >> 5)] = bnd_v; }
        }
        // level 2 of chunk c + G has landed; phase A is done with the record and
        // gather-tile buffers, so level 3 of chunk c + G goes in flight now
        cp_async_wait_all();
        __syncthreads();
        if (SCATTER && SCAT == 1) {
            // per rank level r: the packets of lower rank, and the banks with a packet of rank r
            const int lane = tid & 31, w = tid >> 5;
            const int cc = S.ccount[lane];
            int mx = cc;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            for (int rr = w; rr < mx; rr += T / 32) {
                const unsigned m = __ballot_sync(0xffffffffu, cc > rr);
                int sm = min(cc, rr);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
                if (lane == 0) { S.mtab[rr] = m; S.ptab[rr] = sm; }
            }
        }
        if (has_next) {
            if (SCATTER) stage_slots<TPB>(S, (kc + 1) & 1, ep_s);
            stage_level3<TPB, GATHER>(D, S, S.cd[(kc + 1) % 3], gpar, ep_g);
        }
        cp_async_commit();

        if (SCATTER) {
            if (SCAT == 1 && tid == 0) {
                float bm = 0.f, bv = 0.f;
                for (int w = 0; w < T / 32; ++w) { bm += S.red[w]; bv += S.red[(TPB / 32) + w]; }
                S.scale[0] = bm > 0.f ? 1073741824.f / bm : 1.f;     // 2^30 / bound
                S.scale[1] = bv > 0.f ? 1073741824.f / bv : 1.f;
            }
            if (SCAT == 1) {
                __syncthreads();
                if (tid < cnt) {
                    const int r = S.prank[tid], k = S.pcol[tid];
                    S.perm[S.ptab[r] + __popc(S.mtab[r] & ((1u << k) - 1u))] = tid;
                }
                if (tid < 32) S.ccount[tid] = 0;
                __syncthreads();
            }
            const float sc_m = SCAT == 1 ? S.scale[0] : 1.f, sc_v = SCAT == 1 ? S.scale[1] : 1.f;

            // ---- B. scatter packets -------------------------------------------
            // lane-transposed mapping: the warp's lanes take packets S/32 apart
            // (sorted neighbours share a cell and would hit the same nodes)
            const int span = rounds * (T >> 5);
            for (int r = 0; r < rounds; ++r) {
                const int u = r * T + tid;
                int j;
                if (SCAT == 1) {
                    if (u >= cnt) continue;
                    j = S.perm[u];   // warps take packets by (rank, bank): few bank conflicts
                } else {
                    j = (u & 31) * span + (u >> 5);
                    if (j >= cnt) continue;
                }
                const float4 q0 = S.pk[j * PK_F4];
                if (!(q0.w > 0.f)) continue;
                const float4 q1r = S.pk[j * PK_F4 + 1], q2 = S.pk[j * PK_F4 + 2], q3 = S.pk[j * PK_F4 + 3],
                             q4 = S.pk[j * PK_F4 + 4];
                // the fixed-point scale is folded into the packet (1 for SCAT != 1)
                const float4 q1 = make_float4(q1r.x * sc_v, q1r.y * sc_v, q1r.z * sc_v, 0.f);
                const float qm = q0.w * sc_m;
                const float Ad[9] = {q2.x * sc_v, q2.y * sc_v, q2.z * sc_v, q2.w * sc_v, q3.x * sc_v,
                                     q3.y * sc_v, q3.z * sc_v, q3.w * sc_v, q4.x * sc_v};
                const float b0f = floorf(q0.x - 0.5f), b1f = floorf(q0.y - 0.5f), b2f = floorf(q0.z - 0.5f);
                const float f0 = q0.x - b0f, f1 = q0.y - b1f, f2 = q0.z - b2f;
                const int t0 = (int)b0f, t1 = (int)b1f, t2 = (int)b2f;
                float w0[3], w1[3], w2[3];
                bspline_w(f0, w0);
                bspline_w(f1, w1);
                bspline_w(f2, w2);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float d0 = (float)i - f0;
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) {
                        const float d1 = (float)jj - f1;
                        const float wij = w0[i] * w1[jj];
                        const float a0 = q1.x + Ad[0] * d0 + Ad[1] * d1, a1 = q1.y + Ad[3] * d0 + Ad[4] * d1,
                                    a2 = q1.z + Ad[6] * d0 + Ad[7] * d1;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float d2 = (float)k - f2;
                            const float wt = wij * w2[k];
                            const float m0 = wt * (a0 + Ad[2] * d2), m1 = wt * (a1 + Ad[5] * d2),
                                        m2 = wt * (a2 + Ad[8] * d2), mm = wt * qm;
                            const int node = tidx(t0 + i, t1 + jj, t2 + k);
                            if (SCAT == 0) {
                                atomicAdd(&S.t.f[node], m0);
                                atomicAdd(&S.t.f[ST3P + node], m1);
                                atomicAdd(&S.t.f[2 * ST3P + node], m2);
                                atomicAdd(&S.t.f[3 * ST3P + node], mm);
                            } else if (SCAT == 1) {
                                atomicAdd(&S.t.i[node], __float2int_rn(m0));
                                atomicAdd(&S.t.i[ST3P + node], __float2int_rn(m1));
                                atomicAdd(&S.t.i[2 * ST3P + node], __float2int_rn(m2));
                                atomicAdd(&S.t.i[3 * ST3P + node], __float2int_rn(mm));
                            } else {
                                const int I = ox - 1 + t0 + i, J = oy - 1 + t1 + jj, K = oz - 1 + t2 + k;
                                const int sl = S.slot_s[kc & 1][(((I >> 2) - bx + 1) * 3 + ((J >> 2) - by + 1)) * 3 +
                                                                ((K >> 2) - bz + 1)];
                                if (sl >= 0)
                                    red_add_v4(D.gmv[spar] + (size_t)sl * BLK_NODES + node_local(I, J, K), m0, m1,
                                               m2, mm);
                                else
                                    set_err(D, ERRB_CAPACITY);
                            }
                        }
                    }
                }
            }
            if (SCAT != 2) {
                __syncthreads();
                // flush: one vector reduction per node that received mass
                const float iv = 1.f / sc_v, im = 1.f / sc_m;
                for (int t = tid; t < ST3; t += T) {
                    const int i = t / (ST * ST), j = (t / ST) % ST, k = t % ST;
                    const int q = tidx(i, j, k);
                    float mm, a0, a1, a2;
                    if (SCAT == 0) {
                        mm = S.t.f[3 * ST3P + q]; a0 = S.t.f[q]; a1 = S.t.f[ST3P + q]; a2 = S.t.f[2 * ST3P + q];
                    } else {
                        const int mi = S.t.i[3 * ST3P + q];
                        mm = (float)mi * im;
                        if (mi == 0) mm = 0.f;
                        a0 = (float)S.t.i[q] * iv; a1 = (float)S.t.i[ST3P + q] * iv; a2 = (float)S.t.i[2 * ST3P + q] * iv;
                    }
                    // cleared for the next chunk as it is read
                    S.t.i[q] = 0; S.t.i[ST3P + q] = 0; S.t.i[2 * ST3P + q] = 0; S.t.i[3 * ST3P + q] = 0;
                    if (mm != 0.f) {
                        const int I = ox - 1 + i, J = oy - 1 + j, K = oz - 1 + k;
                        const int sl = S.slot_s[kc & 1][(((I >> 2) - bx + 1) * 3 + ((J >> 2) - by + 1)) * 3 +
                                                        ((K >> 2) - bz + 1)];
                        if (sl >= 0) red_add_v4(D.gmv[spar] + (size_t)sl * BLK_NODES + node_local(I, J, K), a0, a1, a2, mm);
                        else set_err(D, ERRB_CAPACITY);
                    }
                }
            }
        }
        // level 3 of chunk c + G has landed
        cp_async_wait_all();
        __syncthreads();
        if (!has_next) break;
        c = cn;
    }
}

// ---------------------------------------------------------------------------
// export: records -> caller layout
// ---------------------------------------------------------------------------
__global__ void k_export(Dev D, float *x, float *v, float *C, float *F) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < D.n; p += gridDim.x * blockDim.x) {
        const float4 *r = D.rec + (size_t)p * REC_F4;
        float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4], r5 = r[5], r6 = r[6];
        if (x) {
            // fixed point -> world units, rounded once to FP32
            const double u = (double)D.q_unit * (double)D.dx;
            x[3 * p] = (float)(rec_q(r0.x) * u);
            x[3 * p + 1] = (float)(rec_q(r0.y) * u);
            x[3 * p + 2] = (float)(rec_q(r0.z) * u);
        }
        if (v) { v[3 * p] = r1.x; v[3 * p + 1] = r1.y; v[3 * p + 2] = r1.z; }
        if (C) {
            float c[9] = {r2.x, r2.y, r2.z, r2.w, r3.x, r3.y, r3.z, r3.w, r4.x};
            for (int i = 0; i < 9; ++i) C[9 * p + i] = c[i];
        }
        if (F) {
            float f[9] = {r4.y, r4.z, r4.w, r5.x, r5.y, r5.z, r5.w, r6.x, r6.y};
            for (int i = 0; i < 9; ++i) F[9 * p + i] = f[i];
        }
    }
}

// dense copy of one grid buffer (debug / parity): m and mv per node of every
// active block, written into caller arrays of R0*R1*R2 (*3) per instance
__global__ void k_grid_dense(Dev D, int par, int which, float *m_out, float *mv_out) {
    const unsigned total = min(D.ctr[CTR_N_ACTIVE + par], D.max_active) * BLK_NODES;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        unsigned slot = i >> 6, l = i & 63u;
        int inst, bx, by, bz;
        key_coords(D, D.active[par][slot], inst, bx, by, bz);
        int I = bx * BLK + (int)(l >> 4), J = by * BLK + (int)((l >> 2) & 3u), K = bz * BLK + (int)(l & 3u);
        size_t nd = (size_t)inst * D.R[0] * D.R[1] * D.R[2] + ((size_t)I * D.R[1] + J) * D.R[2] + K;
        float4 a = which ? D.gv[par][i] : D.gmv[par][i];
        m_out[nd] = a.w;
        mv_out[3 * nd] = a.x;
        mv_out[3 * nd + 1] = a.y;
        mv_out[3 * nd + 2] = a.z;
    }
}

// ---------------------------------------------------------------------------
// per-material sums of per-particle values (n x 3): shared-memory partial
// sums per CTA, then one global atomic per material and component
// ---------------------------------------------------------------------------
__global__ void k_reduce_by_material(Dev D, int n_mat, const float *__restrict__ vals, float *out) {
    extern __shared__ float acc[];   // 3 * n_mat
    for (int t = threadIdx.x; t < 3 * n_mat; t += blockDim.x) acc[t] = 0.f;
    __syncthreads();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < D.n; p += gridDim.x * blockDim.x) {
        const int m = __float_as_int(D.rec[(size_t)p * REC_F4 + 7].y) >> 8;
        if (m >= 0 && m < n_mat) {
            atomicAdd(&acc[3 * m], vals[3 * p]);
            atomicAdd(&acc[3 * m + 1], vals[3 * p + 1]);
            atomicAdd(&acc[3 * m + 2], vals[3 * p + 2]);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * n_mat; t += blockDim.x)
        if (acc[t] != 0.f) atomicAdd(&out[t], acc[t]);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
void launch_load(const Dev &D, const LoadArgs &a, cudaStream_t st) {
    k_load<<<grid_for(D.n, 256), 256, 0, st>>>(D, a.x, a.v, a.C, a.F, a.vol, a.mat, a.inst, a.params, a.table);
}
void launch_bin(const Dev &D, cudaStream_t st) { k_bin<<<grid_for(D.n, 256), 256, 0, st>>>(D); }
void launch_plan(const Dev &D, int bump_mask, cudaStream_t st) { k_plan<<<1, 1024, 0, st>>>(D, bump_mask); }
void launch_prepare(const Dev &D, int upd_par, int act_par, int do_sort, int keep_momentum, int grid, cudaStream_t st) {
    k_prepare<<<grid, 256, 0, st>>>(D, upd_par, act_par, do_sort, keep_momentum);
}
template <int MODE, int SCAT, int TPB, bool XM, bool DB = false>
static void launch_sub(const Dev &D, int gpar, int spar, int grid, cudaStream_t st) {
    k_substep<MODE, SCAT, TPB, XM, DB><<<grid, TPB, sizeof(SubstepSmem<TPB>), st>>>(D, gpar, spar);
}
template <int TPB>
static void launch_tpb(const Dev &D, int mode, int gpar, int spar, int grid, bool direct, cudaStream_t st) {
    if (direct && mode == MODE_FUSED) {   // direct binning: scatter strategies 1 and 2
        if (D.xm) launch_sub<MODE_FUSED, 1, TPB, true, true>(D, gpar, spar, grid, st);
        else if (D.scatter == 2) launch_sub<MODE_FUSED, 2, TPB, false, true>(D, gpar, spar, grid, st);
        else launch_sub<MODE_FUSED, 1, TPB, false, true>(D, gpar, spar, grid, st);
        return;
    }
    if (D.xm) {   // further models: the shared-memory fixed-point scatter only
        if (mode == MODE_G2P) launch_sub<MODE_G2P, 2, TPB, true>(D, gpar, spar, grid, st);
        else if (mode == MODE_P2G) launch_sub<MODE_P2G, 1, TPB, true>(D, gpar, spar, grid, st);
        else launch_sub<MODE_FUSED, 1, TPB, true>(D, gpar, spar, grid, st);
        return;
    }
    if (mode == MODE_G2P) { launch_sub<MODE_G2P, 2, TPB, false>(D, gpar, spar, grid, st); return; }
    if (mode == MODE_P2G) {
        if (D.scatter == 0) launch_sub<MODE_P2G, 0, TPB, false>(D, gpar, spar, grid, st);
        else if (D.scatter == 1) launch_sub<MODE_P2G, 1, TPB, false>(D, gpar, spar, grid, st);
        else launch_sub<MODE_P2G, 2, TPB, false>(D, gpar, spar, grid, st);
        return;
    }
    if (D.scatter == 0) launch_sub<MODE_FUSED, 0, TPB, false>(D, gpar, spar, grid, st);
    else if (D.scatter == 1) launch_sub<MODE_FUSED, 1, TPB, false>(D, gpar, spar, grid, st);
    else launch_sub<MODE_FUSED, 2, TPB, false>(D, gpar, spar, grid, st);
}
// the chunk size selects the CTA size: chunks of <= 64 particles run 64-thread CTAs
void launch_substep(const Dev &D, int mode, int gpar, int spar, int grid, bool direct, cudaStream_t st) {
    if (D.chunk <= 64) launch_tpb<64>(D, mode, gpar, spar, grid, direct, st);
    else launch_tpb<128>(D, mode, gpar, spar, grid, direct, st);
}
void launch_between(const Dev &D, int upd, int act, int grid, cudaStream_t st) {
    k_between<<<grid, 256, 0, st>>>(D, upd, act);
}
void launch_export(const Dev &D, float *x, float *v, float *C, float *F, cudaStream_t st) {
    k_export<<<grid_for(D.n, 256), 256, 0, st>>>(D, x, v, C, F);
}
void launch_grid_dense(const Dev &D, int par, int which, float *m, float *mv, cudaStream_t st) {
    k_grid_dense<<<1024, 256, 0, st>>>(D, par, which, m, mv);
}
template <int MODE, int SCAT, int TPB, bool XM> static int occ_of() {
    int nb = 0;
    cudaFuncSetAttribute(k_substep<MODE, SCAT, TPB, XM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(SubstepSmem<TPB>));
    if constexpr (MODE == MODE_FUSED && SCAT != 0)   // its direct-binning variant
        cudaFuncSetAttribute(k_substep<MODE, SCAT, TPB, XM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SubstepSmem<TPB>));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_substep<MODE, SCAT, TPB, XM, false>, TPB,
                                                  sizeof(SubstepSmem<TPB>));
    return nb;
}
template <int TPB> static int occ_tpb(int mode, int scatter, bool xm) {
    if (xm)
        return mode == MODE_G2P ? occ_of<MODE_G2P, 2, TPB, true>()
                                : mode == MODE_P2G ? occ_of<MODE_P2G, 1, TPB, true>() : occ_of<MODE_FUSED, 1, TPB, true>();
    if (mode == MODE_G2P) return occ_of<MODE_G2P, 2, TPB, false>();
    if (mode == MODE_P2G)
        return scatter == 0 ? occ_of<MODE_P2G, 0, TPB, false>()
                            : scatter == 1 ? occ_of<MODE_P2G, 1, TPB, false>() : occ_of<MODE_P2G, 2, TPB, false>();
    return scatter == 0 ? occ_of<MODE_FUSED, 0, TPB, false>()
                        : scatter == 1 ? occ_of<MODE_FUSED, 1, TPB, false>() : occ_of<MODE_FUSED, 2, TPB, false>();
}
// resident CTAs per SM of the substep kernel for a mode, scatter strategy, chunk size and model set
int substep_occupancy(int mode, int scatter, int chunk, bool xm) {
    return chunk <= 64 ? occ_tpb<64>(mode, scatter, xm) : occ_tpb<128>(mode, scatter, xm);
}
int substep_chunk_max() { return CH_MAX; }

void launch_reduce_by_material(const Dev &D, int n_mat, const float *vals, float *out, cudaStream_t st) {
    k_reduce_by_material<<<grid_for(D.n, 256, 152 * 4), 256, 3 * n_mat * sizeof(float), st>>>(D, n_mat, vals, out);
}

}  // namespace mpm
