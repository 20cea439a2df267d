// mpm_dev.cuh -- device-side context, particle record layout and the small
// helpers every kernel of libmpm shares.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mpm {

// One particle = one 128-byte record (8 x float4), stored in the caller's
// order and never permuted; kernels reach particles through the sorted index.
//   f4[0] = x0 x1 x2 mass        f4[1] = v0 v1 v2 vol
//   f4[2] = C0 C1 C2 C3          f4[3] = C4 C5 C6 C7
//   f4[4] = C8 F0 F1 F2          f4[5] = F3 F4 F5 F6
//   f4[6] = F7 F8 mu lambda      f4[7] = yield info instance alpha
// (alpha: Drucker-Prager coefficient of the friction angle; nu = lambda / (2 (lambda + mu)))
// info bits: elastic model [0,4), plastic model [4,8), material id [8,32).
constexpr int REC_F4 = 8;

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
    int4 *chunks;          // work items: (block key, first sorted slot, count, 0)
    unsigned *ctr;         // device counters, see CTR_*
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
    CTR_COUNT = 16
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

}  // namespace mpm
