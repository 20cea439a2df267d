// mpm_dev.cuh -- device-side context, particle record layout and the small
// helpers every kernel of libmpm shares.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mpm {

// One particle = one 128-byte record (8 x float4), stored in the caller's
// order and never permuted; kernels reach particles through the sorted index.
//   f4[0] = q0 q1 q2 mass        f4[1] = v0 v1 v2 vol
//   f4[2] = C0 C1 C2 C3          f4[3] = C4 C5 C6 C7
//   f4[4] = C8 F0 F1 F2          f4[5] = F3 F4 F5 F6
//   f4[6] = F7 F8 mu lambda      f4[7] = yield info instance alpha
// (alpha: Drucker-Prager coefficient of the friction angle; nu = lambda / (2 (lambda + mu)))
// info bits: elastic model [0,4), plastic model [4,8), material id [8,32).
//
// Positions q0 q1 q2 are int32 bit patterns: signed fixed point in grid-cell
// units, x_d = q_d 2^-qf dx, with qf fraction bits per context (Dev::qf).
// Every cell then has the same resolution, 2^-qf of a cell, where an FP32
// world coordinate loses precision away from the origin: at 256 nodes per
// axis (qf = 22) a position resolves 2.4e-7 of a cell everywhere, against
// 1.5e-5 of a cell for an FP32 coordinate near the middle of the domain.  That
// FP32 rounding, taken once per substep by x += dt v, would otherwise bound
// the trajectory's agreement with an exact integrator.  The base node and the
// spline fraction of a position follow exactly from integer arithmetic
// (base_cell_q).
constexpr int REC_F4 = 8;

// fraction bits of the fixed-point position for a grid of at most r_max
// nodes per axis: the largest |q| (twice the grid, leaving room for particles
// that leave it) fits in int32, and qf <= 23 keeps the spline fraction's
// numerator below 2^24, so that it converts to float exactly
inline int position_fraction_bits(int r_max) {
    int lg = 0;
    while ((1 << lg) < 2 * r_max) ++lg;
    const int qf = 31 - lg;
    return qf < 23 ? qf : 23;
}

// The grid is block-sparse: 4x4x4-node blocks, a dense page table per grid
// buffer (block key -> pool slot), an epoch tag per entry telling whether the
// entry belongs to the current substep, and a pool of active blocks.  Two
// grid buffers alternate between consecutive substeps (parity).
constexpr int BLK = 4;
constexpr int BLK_NODES = 64;

// sticky device error bits
enum : unsigned {
    ERRB_DOMAIN = 1u << 0,
    ERRB_NONFINITE = 1u << 1,
    ERRB_CAPACITY = 1u << 2,
    ERRB_CFL = 1u << 3,
    ERRB_TIMEOUT = 1u << 4,
};

struct Dev {
    // geometry
    int R[3];              // nodes per axis of one instance grid
    int NB[3];             // blocks per axis
    int bpi;               // blocks per instance
    int n_inst;
    float dx, inv_dx, dt;
    int qf;                // fraction bits of the fixed-point positions
    float q_cell;          // 2^qf: fixed-point units per cell
    float q_unit;          // 2^-qf: cells per fixed-point unit
    float g[3];
    int bound;
    int wall[6];
    // particles
    int n;
    float4 *rec;           // n * REC_F4
    // binning (current positions)
    unsigned *key;         // n
    unsigned *rank;        // n
    unsigned *sorted;      // n: particle index by (block, rank)
    unsigned *bcount;      // total blocks: particles per block (zero outside a binning window)
    unsigned *bstart;      // total blocks: first sorted slot of each occupied block
    unsigned *occ;         // occupied blocks being collected by the binning kernel
    unsigned *plan;        // occupied blocks of the grouping in use
    int4 *chunks;          // work items the substep kernel reads: (block key, first index, count, list)
    unsigned *ctr;         // device counters, see CTR_*
    int chunk_ctr;         // index in ctr of the number of work items (CTR_N_CHUNKS unless direct)
    // list 0 of a work item: `sorted` (the counting sort, or a direct binning's
    // per-block lists); list 1: the overflow entries (particle, block key) of a
    // direct binning, one particle per work item
    const unsigned *ovf_in;
    // direct binning (the steady-state substeps of a forward run): the fused
    // kernel places each particle straight into the list of its new block,
    // at the block's pool slot in the scatter buffer; per grid buffer:
    unsigned *slist[2];    // slist_blocks lists of slist_cap particle indices
    unsigned *ovf[2];      // (particle, block key) of particles whose list was full or beyond slist_blocks
    unsigned *occd[2];     // occupied blocks of the binning
    int4 *chunksd[2];      // work items of the binning
    unsigned slist_cap, slist_blocks, ovf_cap, max_chunks_d;
    // grid buffers (index = parity)
    int *page[2];
    unsigned *page_epoch[2];
    unsigned *active[2];
    float4 *gmv[2];        // (mv.x, mv.y, mv.z, m) per node, zero outside a substep
    float4 *gv[2];         // (v.x, v.y, v.z, m) per node after the grid update
    unsigned max_active;
    unsigned max_chunks;
    int chunk;             // particles per chunk
    int scatter;           // scatter strategy of the substep kernel (0 shared tile, 2 direct)
    int xm;                // the material table uses models beyond FCR / NH / VM / DP
    unsigned *err;         // sticky error bits
};

// device counters (Dev::ctr)
enum {
    CTR_N_OCC = 0,         // blocks collected in occ
    CTR_N_PLAN = 1,        // blocks in plan
    CTR_N_CHUNKS = 2,
    CTR_EPOCH = 3,         // monotonically increasing activation epoch
    CTR_EPOCH_OF = 4,      // [4], [5]: epoch of grid buffer 0 / 1
    CTR_N_ACTIVE = 6,      // [6], [7]: active blocks of grid buffer 0 / 1
    CTR_FALLBACKS = 8,     // FP64 SVD branch count
    CTR_D_OCC = 16,        // [16], [17]: occupied blocks of the direct binning into buffer 0 / 1
    CTR_D_OVF = 18,        // [18], [19]: its overflow entries
    CTR_D_CH = 20,         // [20], [21]: its work items
    CTR_D_OVF_TOTAL = 22,  // particles placed in overflow entries since the last load
    CTR_MAX_COUNT = 23,    // largest block count of the last full binning (k_bin)
    CTR_COUNT = 32
};

__device__ __forceinline__ unsigned block_key(const Dev &D, int inst, int bx, int by, int bz) {
    return (unsigned)inst * (unsigned)D.bpi + (unsigned)((bx * D.NB[1] + by) * D.NB[2] + bz);
}

__device__ __forceinline__ void key_coords(const Dev &D, unsigned key, int &inst, int &bx, int &by, int &bz) {
    inst = (int)(key / (unsigned)D.bpi);
    int r = (int)(key - (unsigned)inst * (unsigned)D.bpi);
    bz = r % D.NB[2];
    r /= D.NB[2];
    by = r % D.NB[1];
    bx = r / D.NB[1];
}

// base cell of a position along one axis; identical arithmetic everywhere a
// particle is binned or transferred
__device__ __forceinline__ int base_cell(float x, float inv_dx, float &fx) {
    float X = x * inv_dx;
    float b = floorf(X - 0.5f);
    fx = X - b;
    return (int)b;
}

// the same for a fixed-point position q (cells = q 2^-qf): b = floor(X - 1/2)
// by an arithmetic shift, fx = X - b in [0.5, 1.5) exactly (the numerator
// q - b 2^qf stays below 1.5 2^qf <= 1.5 2^23)
__device__ __forceinline__ int base_cell_q(int q, const Dev &D, float &fx) {
    const int b = (q - (1 << (D.qf - 1))) >> D.qf;
    fx = (float)(q - (b << D.qf)) * D.q_unit;
    return b;
}

// fixed-point position after a displacement of dt v: the displacement in
// cells is rounded once to the fixed-point grid; the sum saturates in int32
// (a particle that far out is reported as out of the domain)
__device__ __forceinline__ int advance_q(int q, float v, const Dev &D) {
    float dq = D.dt * v * D.inv_dx * D.q_cell;
    dq = fminf(fmaxf(dq, -1.0e9f), 1.0e9f);          // NaN becomes a bound too
    const long long s = (long long)q + (long long)__float2ll_rn(dq);
    return (int)(s < -2147483647ll ? -2147483647ll : (s > 2147483647ll ? 2147483647ll : s));
}

__device__ __forceinline__ int rec_q(float f) { return __float_as_int(f); }

__device__ __forceinline__ void set_err(const Dev &D, unsigned bit) { atomicOr(D.err, bit); }

__device__ __forceinline__ void red_add_v4(float4 *addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Claims n consecutive indices of *ctr for each lane (n = 0: none) with one
// atomic per warp; returns the lane's first index.  Every lane of the warp
// must call it together (a warp-uniform loop).
__device__ __forceinline__ unsigned warp_claim(unsigned *ctr, unsigned n) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += u;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned base = 0;
    if (lane == 31 && total) base = atomicAdd(ctr, total);
    return __shfl_sync(0xffffffffu, base, 31) + incl - n;
}

}  // namespace mpm
