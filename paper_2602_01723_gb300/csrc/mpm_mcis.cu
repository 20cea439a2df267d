// mpm_mcis.cu -- Monte Carlo Importance Sampling of interior fill points
// (§4.1 "Monte Carlo Importance Sampling", steps 1-4) for objects given as
// contiguous ranges of surface points (the cluster C_k) and candidates Q_k:
//   d_j = min_{c in C_k} |q_j - c|;  w_j = max(exp(-d_j^2 / 2 sigma^2), eps);
//   p_j = w_j / sum w;  n_k i.i.d. draws with P(s = q_j) = p_j.
//
// GPU layout:
//   * surface points are binned per object into a uniform grid over the unit
//     cube (App. C.1 normalises every scene to it; coordinates outside are
//     clamped into the border cells, which keeps every pair within the
//     cut-off in neighbouring cells) with a counting sort;
//   * every candidate searches rings of cells in order of distance and stops
//     once the best distance is below the ring's lower bound.  Beyond
//     d_cut = sigma sqrt(2 ln(1/eps)) the weight is eps whatever the
//     distance, so the search radius is d_cut.  Distances are screened in
//     FP32 and confirmed in FP64, so the minimum is the exact FP64 one;
//   * weights are summed as integers round(w 2^40), which makes the
//     cumulative sums independent of the summation order, and each draw
//     binary-searches its object's cumulative sums for floor(u W_k).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mpm.h"
#include "mpm_ptr.h"
#include "mpm_scan.cuh"

namespace {

thread_local std::string g_mcis_msg;

constexpr double WSCALE = 1099511627776.0;   // 2^40
constexpr int RINGS = 6;                      // cell edge >= d_cut / 6: rings 0..6 cover d_cut

__device__ __forceinline__ int find_range(const int64_t *off, int n, int64_t i) {
    int lo = 0, hi = n;   // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int cell_of(float x, float inv_h, int G) {
    int c = (int)floorf(x * inv_h);
    return c < 0 ? 0 : (c >= G ? G - 1 : c);
}

struct Grid {
    int G;            // cells per axis
    float inv_h;
    long long cells;  // per object
};

__global__ void k_mc_count(int n_obj, const int64_t *soff, const float *surf, Grid g, unsigned *cnt,
                           unsigned *rank) {
    const int64_t n = soff[n_obj];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_range(soff, n_obj, s);
        const int cx = cell_of(surf[3 * s], g.inv_h, g.G), cy = cell_of(surf[3 * s + 1], g.inv_h, g.G),
                  cz = cell_of(surf[3 * s + 2], g.inv_h, g.G);
        const long long key = (long long)k * g.cells + ((long long)cx * g.G + cy) * g.G + cz;
        rank[s] = atomicAdd(&cnt[key], 1u);
    }
}

__global__ void k_mc_scatter(int n_obj, const int64_t *soff, const float *surf, Grid g, const unsigned *start,
                             const unsigned *rank, float4 *sorted) {
    const int64_t n = soff[n_obj];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_range(soff, n_obj, s);
        const float x = surf[3 * s], y = surf[3 * s + 1], z = surf[3 * s + 2];
        const long long key =
            (long long)k * g.cells +
            ((long long)cell_of(x, g.inv_h, g.G) * g.G + cell_of(y, g.inv_h, g.G)) * g.G + cell_of(z, g.inv_h, g.G);
        sorted[start[key] + rank[s]] = make_float4(x, y, z, 0.f);
    }
}

// inclusive scan of int64 weights: per-block scans, block totals, offsets
__global__ void __launch_bounds__(1024) k_mc_scan_i64_block(const long long *in, long long *out, long long n,
                                                             long long *totals) {
    __shared__ long long sh[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long x = i < n ? in[i] : 0;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        long long t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    if (i < n) out[i] = x + (w > 0 ? sh[w - 1] : 0);
    if (threadIdx.x == 0) totals[blockIdx.x] = sh[(blockDim.x >> 5) - 1];
}

__global__ void __launch_bounds__(1024) k_mc_scan_i64_totals(long long *totals, long long nb) {
    // exclusive scan of the block totals, in place, one CTA
    __shared__ long long sh[32];
    long long carry = 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (long long b = 0; b < nb; b += blockDim.x) {
        const long long i = b + threadIdx.x;
        const long long v = i < nb ? totals[i] : 0;
        long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sh[w] = x;
        __syncthreads();
        if (w == 0) {
            long long t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            sh[lane] = t;
        }
        __syncthreads();
        if (i < nb) totals[i] = carry + (w > 0 ? sh[w - 1] : 0) + x - v;
        const long long total = sh[(blockDim.x >> 5) - 1];
        __syncthreads();
        carry += total;
    }
}

__global__ void k_mc_scan_i64_add(long long *out, long long n, const long long *totals) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] += totals[blockIdx.x];
}

// candidates in (object, cell) order, so that the threads of a warp search
// the same cells
__global__ void k_mc_cand_count(int n_obj, const int64_t *coff, const float *cand, Grid g, unsigned *cnt,
                                unsigned *rank) {
    const int64_t n = coff[n_obj];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_range(coff, n_obj, j);
        const long long key = (long long)k * g.cells +
                              ((long long)cell_of(cand[3 * j], g.inv_h, g.G) * g.G + cell_of(cand[3 * j + 1], g.inv_h, g.G)) *
                                  g.G + cell_of(cand[3 * j + 2], g.inv_h, g.G);
        rank[j] = atomicAdd(&cnt[key], 1u);
    }
}
__global__ void k_mc_cand_scatter(int n_obj, const int64_t *coff, const float *cand, Grid g, const unsigned *start,
                                  const unsigned *rank, unsigned *order) {
    const int64_t n = coff[n_obj];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_range(coff, n_obj, j);
        const long long key = (long long)k * g.cells +
                              ((long long)cell_of(cand[3 * j], g.inv_h, g.G) * g.G + cell_of(cand[3 * j + 1], g.inv_h, g.G)) *
                                  g.G + cell_of(cand[3 * j + 2], g.inv_h, g.G);
        order[start[key] + rank[j]] = (unsigned)j;
    }
}


// squared distance along one axis from q to cell c of edge h, in FP32
__device__ __forceinline__ float box_d2f(float q, int c, float h) {
    const float lo = (float)c * h, hi = lo + h;
    const float e = q < lo ? lo - q : (q > hi ? q - hi : 0.f);
    return e * e;
}

// steps 1 and 2 per candidate: exact nearest-surface distance within d_cut, weight
__global__ void k_mc_nn(int n_obj, const int64_t *coff, const float *cand, const unsigned *order, Grid g,
                        const unsigned *start, const unsigned *cnt, const float4 *sorted, double sigma, double eps,
                        double *d, double *w, long long *wq) {
    const int64_t n = coff[n_obj];
    const double h = 1.0 / (double)g.inv_h;
    const float hf = 1.f / g.inv_h;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = order[t];
        const int k = find_range(coff, n_obj, j);
        const float qx = cand[3 * j], qy = cand[3 * j + 1], qz = cand[3 * j + 2];
        const int cx = cell_of(qx, g.inv_h, g.G), cy = cell_of(qy, g.inv_h, g.G), cz = cell_of(qz, g.inv_h, g.G);
        const long long base = (long long)k * g.cells;
        double best = INFINITY;
        float screen = INFINITY;   // best * (1 + 1e-6), rounded up to FP32
        for (int r = 0; r <= RINGS; ++r) {
            // cells of ring r lie at least (r - 1) h away: stop once the best is closer
            const double lb = (double)(r - 1) * h;
            if (r > 1 && best <= lb * lb) break;
            // pruning threshold in FP32: the FP32 box distance of a cell within d_cut is
            // within 1.3e-7 of the exact one (cell edges and differences rounded), so this
            // margin never skips a cell that could hold a closer point
            const float prune = (float)best * 1.00001f + 2e-7f;
            for (int ix = -r; ix <= r; ++ix) {
                const int x = cx + ix;
                if (x < 0 || x >= g.G) continue;
                for (int iy = -r; iy <= r; ++iy) {
                    const int y = cy + iy;
                    if (y < 0 || y >= g.G) continue;
                    // ring r only: the whole row on its x or y faces, else its two z ends
                    const bool face = ix == -r || ix == r || iy == -r || iy == r;
                    const int zstep = (face || r == 0) ? 1 : 2 * r;
                    for (int iz = -r; iz <= r; iz += zstep) {
                        const int z = cz + iz;
                        if (z < 0 || z >= g.G) continue;
                        // a cell wholly farther than the best point holds nothing closer
                        // (cells are clamped at the cube's faces, so only interior cells are skipped)
                        if (x > 0 && y > 0 && z > 0 && x < g.G - 1 && y < g.G - 1 && z < g.G - 1 &&
                            box_d2f(qx, x, hf) + box_d2f(qy, y, hf) + box_d2f(qz, z, hf) > prune)
                            continue;
                        const long long key = base + ((long long)x * g.G + y) * g.G + z;
                        const unsigned s0 = start[key], s1 = s0 + cnt[key];
                        for (unsigned s = s0; s < s1; ++s) {
                            const float4 c = sorted[s];
                            const float ex = qx - c.x, ey = qy - c.y, ez = qz - c.z;
                            const float d2f = ex * ex + ey * ey + ez * ez;
                            // the FP32 value is within 1e-6 relative of the exact one, so a
                            // point closer than best passes this FP32 screen
                            if (d2f <= screen) {
                                const double fx = (double)qx - (double)c.x, fy = (double)qy - (double)c.y,
                                             fz = (double)qz - (double)c.z;
                                const double d2 = fx * fx + fy * fy + fz * fz;
                                if (d2 < best) {
                                    best = d2;
                                    screen = __double2float_ru(best * (1.0 + 1e-6));
                                }
                            }
                        }
                    }
                }
            }
        }
        // nothing within the searched rings: the distance is at least d_cut, so the weight is eps
        const double wt = isinf(best) ? eps : fmax(exp(-best / (2.0 * sigma * sigma)), eps);
        if (d) d[j] = sqrt(best);
        if (w) w[j] = wt;
        wq[j] = (long long)floor(wt * WSCALE + 0.5);
    }
}

// step 4: draw i of object k picks the first candidate whose cumulative weight
// (within the object) exceeds floor(u_i W_k)
__global__ void k_mc_draw(int n_obj, const int64_t *coff, const int64_t *doff, const double *u, const long long *cum,
                          int64_t *picked) {
    const int64_t n = doff[n_obj];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_range(doff, n_obj, i);
        const int64_t c0 = coff[k], c1 = coff[k + 1];
        if (c1 == c0) { picked[i] = -1; continue; }
        const long long base = c0 > 0 ? cum[c0 - 1] : 0;
        const long long total = cum[c1 - 1] - base;
        const long long t = (long long)floor(u[i] * (double)total);
        int64_t lo = c0, hi = c1 - 1;   // first j with cum[j] - base > t; the last candidate if none
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cum[mid] - base > t) hi = mid; else lo = mid + 1;
        }
        picked[i] = lo;
    }
}

bool is_dev(const void *p) { return mpm::on_this_device(p); }

int blocks_for(long long n, int t) {
    long long b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

extern "C" MPM_API mpm_status mpm_mcis(int32_t n_obj, const int64_t *surf_off, const float *surf,
                                       const int64_t *cand_off, const float *cand, const int64_t *draw_off,
                                       const double *u, double sigma, double eps, double *d, double *w,
                                       int64_t *picked, void *stream) {
    g_mcis_msg.clear();
    if (n_obj < 1 || !surf_off || !cand_off || !draw_off || !(sigma > 0.0) || !(eps > 0.0) || !(eps < 1.0)) {
        g_mcis_msg = "mcis: n_obj >= 1, offsets non-NULL, sigma > 0, 0 < eps < 1";
        return MPM_ERR_INVALID_ARG;
    }
    for (int k = 0; k < n_obj; ++k)
        if (surf_off[k + 1] < surf_off[k] || cand_off[k + 1] < cand_off[k] || draw_off[k + 1] < draw_off[k]) {
            g_mcis_msg = "mcis: offsets must be non-decreasing";
            return MPM_ERR_INVALID_ARG;
        }
    if (surf_off[0] != 0 || cand_off[0] != 0 || draw_off[0] != 0) {
        g_mcis_msg = "mcis: offsets must start at 0";
        return MPM_ERR_INVALID_ARG;
    }
    if (mpm::any_on_other_device({surf, cand, u, d, w, picked})) {
        g_mcis_msg = "mcis: an array lives on another device than the current one";
        return MPM_ERR_INVALID_ARG;
    }
    const long long ns = surf_off[n_obj], nc = cand_off[n_obj], nd = draw_off[n_obj];
    if ((ns > 0 && !surf) || (nc > 0 && !cand) || (nd > 0 && (!u || !picked)) || ns >= (1ll << 32)) {
        g_mcis_msg = "mcis: missing arrays or too many surface points";
        return MPM_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const double cut = sigma * std::sqrt(2.0 * std::log(1.0 / eps));
    Grid g;
    // cell edge 1/G >= d_cut / RINGS, so rings 0..RINGS hold every point within d_cut
    g.G = (int)std::floor(RINGS / cut);
    if (g.G < 1) g.G = 1;
    if (g.G > 256) g.G = 256;
    g.inv_h = (float)g.G;
    g.cells = (long long)g.G * g.G * g.G;
    const long long keys = g.cells * n_obj;
    if (keys >= (1ll << 31)) { g_mcis_msg = "mcis: grid too large"; return MPM_ERR_INVALID_ARG; }

    // scratch: one stream-ordered allocation carved into pieces
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const long long nb = (nc + 1023) / 1024;
    size_t off = 0;
    const size_t o_soff = off; off += al((n_obj + 1) * 8);
    const size_t o_coff = off; off += al((n_obj + 1) * 8);
    const size_t o_doff = off; off += al((n_obj + 1) * 8);
    const size_t o_surf = off; off += al(ns * 12);
    const size_t o_cand = off; off += al(nc * 12);
    const size_t o_u = off; off += al(nd * 8);
    const size_t o_cnt = off; off += al(keys * 4);
    const size_t o_start = off; off += al(keys * 4);
    const size_t o_rank = off; off += al(ns * 4);
    const size_t o_cnt2 = off; off += al(keys * 4);
    const size_t o_start2 = off; off += al(keys * 4);
    const size_t o_crank = off; off += al(nc * 4);
    const size_t o_order = off; off += al(nc * 4);
    const size_t o_sorted = off; off += al(ns * 16);
    const size_t o_wq = off; off += al(nc * 8);
    const size_t o_cum = off; off += al(nc * 8);
    const size_t o_tot = off; off += al((nb + 1) * 8);
    const size_t o_kb = off; off += al(((keys + SC_T - 1) / SC_T + 1) * 8);   // cell-count scan block sums
    const size_t o_kt = off; off += al(8);
    const size_t o_d = off; off += al(nc * 8);
    const size_t o_w = off; off += al(nc * 8);
    const size_t o_pick = off; off += al(nd * 8);
    char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, off ? off : 256, st) != cudaSuccess) {
        cudaGetLastError();
        g_mcis_msg = "mcis: device allocation failed";
        return MPM_ERR_OOM;
    }
    auto P = [&](size_t o) { return (void *)(buf + o); };
    mpm_status status = MPM_OK;
#define MC_CK(call)                                                                  \
    do {                                                                             \
        if ((call) != cudaSuccess) {                                                 \
            g_mcis_msg = std::string("mcis: ") + cudaGetErrorString(cudaGetLastError()); \
            status = MPM_ERR_CUDA;                                                   \
            goto done;                                                               \
        }                                                                            \
    } while (0)
    {
        int64_t *dsoff = (int64_t *)P(o_soff), *dcoff = (int64_t *)P(o_coff), *ddoff = (int64_t *)P(o_doff);
        MC_CK(cudaMemcpyAsync(dsoff, surf_off, (n_obj + 1) * 8, cudaMemcpyHostToDevice, st));
        MC_CK(cudaMemcpyAsync(dcoff, cand_off, (n_obj + 1) * 8, cudaMemcpyHostToDevice, st));
        MC_CK(cudaMemcpyAsync(ddoff, draw_off, (n_obj + 1) * 8, cudaMemcpyHostToDevice, st));
        const float *dsurf = surf, *dcand = cand;
        const double *du = u;
        if (ns > 0 && !is_dev(surf)) { MC_CK(cudaMemcpyAsync(P(o_surf), surf, ns * 12, cudaMemcpyHostToDevice, st)); dsurf = (const float *)P(o_surf); }
        if (nc > 0 && !is_dev(cand)) { MC_CK(cudaMemcpyAsync(P(o_cand), cand, nc * 12, cudaMemcpyHostToDevice, st)); dcand = (const float *)P(o_cand); }
        if (nd > 0 && !is_dev(u)) { MC_CK(cudaMemcpyAsync(P(o_u), u, nd * 8, cudaMemcpyHostToDevice, st)); du = (const double *)P(o_u); }
        unsigned *cnt = (unsigned *)P(o_cnt), *start = (unsigned *)P(o_start), *rank = (unsigned *)P(o_rank);
        unsigned *cnt2 = (unsigned *)P(o_cnt2), *start2 = (unsigned *)P(o_start2);
        float4 *sorted = (float4 *)P(o_sorted);
        long long *wq = (long long *)P(o_wq), *cum = (long long *)P(o_cum), *tot = (long long *)P(o_tot);
        MC_CK(cudaMemsetAsync(cnt, 0, keys * 4, st));
        if (ns > 0) {
            k_mc_count<<<blocks_for(ns, 256), 256, 0, st>>>(n_obj, dsoff, dsurf, g, cnt, rank);
            MC_CK(cudaGetLastError());
        }
        scan_counts(cnt, start, keys, (unsigned long long *)P(o_kb), (unsigned long long *)P(o_kt), st);
        MC_CK(cudaGetLastError());
        if (ns > 0) {
            k_mc_scatter<<<blocks_for(ns, 256), 256, 0, st>>>(n_obj, dsoff, dsurf, g, start, rank, sorted);
            MC_CK(cudaGetLastError());
        }
        double *dd = d && is_dev(d) ? d : (double *)P(o_d);
        double *dw = w && is_dev(w) ? w : (double *)P(o_w);
        int64_t *dp = picked && is_dev(picked) ? picked : (int64_t *)P(o_pick);
        if (nc > 0) {
            unsigned *crank = (unsigned *)P(o_crank), *order = (unsigned *)P(o_order);
            MC_CK(cudaMemsetAsync(cnt2, 0, keys * 4, st));
            k_mc_cand_count<<<blocks_for(nc, 256), 256, 0, st>>>(n_obj, dcoff, dcand, g, cnt2, crank);
            scan_counts(cnt2, start2, keys, (unsigned long long *)P(o_kb), (unsigned long long *)P(o_kt), st);
            k_mc_cand_scatter<<<blocks_for(nc, 256), 256, 0, st>>>(n_obj, dcoff, dcand, g, start2, crank, order);
            MC_CK(cudaGetLastError());
            k_mc_nn<<<blocks_for(nc, 128), 128, 0, st>>>(n_obj, dcoff, dcand, order, g, start, cnt, sorted, sigma, eps,
                                                           dd, dw, wq);
            MC_CK(cudaGetLastError());
            k_mc_scan_i64_block<<<(unsigned)nb, 1024, 0, st>>>(wq, cum, nc, tot);
            k_mc_scan_i64_totals<<<1, 1024, 0, st>>>(tot, nb);
            k_mc_scan_i64_add<<<(unsigned)nb, 1024, 0, st>>>(cum, nc, tot);
            MC_CK(cudaGetLastError());
        }
        if (nd > 0) {
            k_mc_draw<<<blocks_for(nd, 256), 256, 0, st>>>(n_obj, dcoff, ddoff, du, cum, dp);
            MC_CK(cudaGetLastError());
        }
        if (d && dd != d) MC_CK(cudaMemcpyAsync(d, dd, nc * 8, cudaMemcpyDeviceToHost, st));
        if (w && dw != w) MC_CK(cudaMemcpyAsync(w, dw, nc * 8, cudaMemcpyDeviceToHost, st));
        if (nd > 0 && dp != picked) MC_CK(cudaMemcpyAsync(picked, dp, nd * 8, cudaMemcpyDeviceToHost, st));
    }
done:
    cudaFreeAsync(buf, st);
    if (status == MPM_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        g_mcis_msg = std::string("mcis: ") + cudaGetErrorString(cudaGetLastError());
        status = MPM_ERR_CUDA;
    }
#undef MC_CK
    return status;
}

extern "C" MPM_API const char *mpm_mcis_last_error(void) { return g_mcis_msg.c_str(); }
