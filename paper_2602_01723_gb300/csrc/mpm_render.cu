// mpm_render.cu -- splatting of the (deformed) Gaussian kernels into a
// headless image (§3.1): Sigma' = J W Sigma W^T J^T and front-to-back
// compositing Col = sum_i col_i alpha_i prod_{j<i} (1 - alpha_j).
//
// Pipeline (one stream, scratch from the stream-ordered allocator):
//   1. per Gaussian: camera position, projected covariance dilated by 0.3,
//      its inverse (conic), the 3-sigma square and the 16x16 tiles it
//      touches;
//   2. one (tile, depth) key per touched tile, sorted by a stable LSD radix
//      sort (8-bit digits over the tile and depth bits) -- the depth is a
//      positive float, whose bit pattern orders like its value;
//   3. per tile the range of its sorted keys;
//   4. one CTA per tile, one thread per pixel: the tile's Gaussians are
//      staged in shared memory in batches and composited front to back; a
//      pixel stops once its transmittance would drop below 1e-4, the CTA once
//      all its pixels have.
// Conventions where the paper defers to 3DGS: Gaussians nearer than 0.2 are
// not drawn; alpha = min(0.99, o exp(power)), skipped below 1/255 or for
// power > 0; the background is added with the remaining transmittance.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/mpm.h"
#include "mpm_ptr.h"
#include "mpm_scan.cuh"

namespace {

thread_local std::string g_render_msg;
constexpr int TS = 16;            // tile edge in pixels
constexpr int RS_THREADS = 256;   // radix sort: threads per CTA
constexpr int RS_ITEMS = 8;       // keys per thread per CTA tile
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

struct Cam {
    float R[9], T[3];
    float fx, fy, cx, cy;
    int W, H, gx, gy;
};

// 1. projection per Gaussian
__global__ void k_rd_pre(long long n, const float *mean, const float *cov, const float *opac, Cam c, float4 *g0,
                         float4 *g1, int4 *rect, unsigned *cnt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        cnt[i] = 0;
        const float px = mean[3 * i], py = mean[3 * i + 1], pz = mean[3 * i + 2];
        const float tx = c.R[0] * px + c.R[1] * py + c.R[2] * pz + c.T[0];
        const float ty = c.R[3] * px + c.R[4] * py + c.R[5] * pz + c.T[1];
        // the depth orders the compositing: rounded operation by operation in a
        // fixed order (no contraction), so that its value does not depend on
        // the compiler
        const float tz = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[6], px), __fmul_rn(c.R[7], py)),
                                             __fmul_rn(c.R[8], pz)), c.T[2]);
        if (!(tz > 0.2f)) continue;
        const float *s = cov + 6 * i;
        const float S[9] = {s[0], s[1], s[2], s[1], s[3], s[4], s[2], s[4], s[5]};
        float WS[9], Sc[9];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q)
                WS[3 * r + q] = c.R[3 * r] * S[q] + c.R[3 * r + 1] * S[3 + q] + c.R[3 * r + 2] * S[6 + q];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q)
                Sc[3 * r + q] = WS[3 * r] * c.R[3 * q] + WS[3 * r + 1] * c.R[3 * q + 1] + WS[3 * r + 2] * c.R[3 * q + 2];
        const float iz = 1.f / tz;
        const float J[6] = {c.fx * iz, 0.f, -c.fx * tx * iz * iz, 0.f, c.fy * iz, -c.fy * ty * iz * iz};
        float JS[6];
        for (int r = 0; r < 2; ++r)
            for (int q = 0; q < 3; ++q) JS[3 * r + q] = J[3 * r] * Sc[q] + J[3 * r + 1] * Sc[3 + q] + J[3 * r + 2] * Sc[6 + q];
        const float a = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2] + 0.3f;
        const float b = JS[0] * J[3] + JS[1] * J[4] + JS[2] * J[5];
        const float d = JS[3] * J[3] + JS[4] * J[4] + JS[5] * J[5] + 0.3f;
        const float det = a * d - b * b;
        if (!(det > 0.f)) continue;
        const float mid = 0.5f * (a + d), disc = sqrtf(fmaxf(0.1f, mid * mid - det));
        const float rad = ceilf(3.f * sqrtf(fmaxf(mid + disc, mid - disc)));
        const float u = c.fx * tx * iz + c.cx, v = c.fy * ty * iz + c.cy;
        const int x0 = (int)fminf((float)c.gx, fmaxf(0.f, floorf((u - rad) / TS)));
        const int x1 = (int)fminf((float)c.gx, fmaxf(0.f, floorf((u + rad + TS - 1) / TS)));
        const int y0 = (int)fminf((float)c.gy, fmaxf(0.f, floorf((v - rad) / TS)));
        const int y1 = (int)fminf((float)c.gy, fmaxf(0.f, floorf((v + rad + TS - 1) / TS)));
        if (x1 <= x0 || y1 <= y0) continue;
        const float idet = 1.f / det;
        g0[i] = make_float4(u, v, d * idet, -b * idet);
        g1[i] = make_float4(a * idet, opac[i], tz, 0.f);
        rect[i] = make_int4(x0, x1, y0, y1);
        cnt[i] = (unsigned)((x1 - x0) * (y1 - y0));
    }
}


// 2. one key per touched tile
__global__ void k_rd_dup(long long n, const float4 *g1, const int4 *rect, const unsigned *cnt, const unsigned *off,
                         int gx, unsigned long long *keys, unsigned *vals) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (cnt[i] == 0) continue;
        const int4 r = rect[i];
        const unsigned long long db = __float_as_uint(g1[i].z);
        unsigned o = off[i];
        for (int y = r.z; y < r.w; ++y)
            for (int x = r.x; x < r.y; ++x) {
                keys[o] = ((unsigned long long)(y * gx + x) << 32) | db;
                vals[o] = (unsigned)i;
                ++o;
            }
    }
}

// radix sort, pass histogram: hist[digit * nblocks + block]
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const unsigned long long *keys, long long n, int shift,
                                                          unsigned *hist, int nblocks) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_ITEMS; ++j) {
        const long long i = base + j * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// radix sort, stable scatter: element order within a CTA tile is (item round, thread)
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const unsigned long long *keys, const unsigned *vals,
                                                             long long n, int shift, const unsigned *hoff,
                                                             int nblocks, unsigned long long *okeys, unsigned *ovals) {
    __shared__ unsigned run[256];
    __shared__ unsigned wc[RS_THREADS / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    run[tid] = hoff[(long long)tid * nblocks + blockIdx.x];
    const long long base = (long long)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_ITEMS; ++j) {
        for (int q = 0; q < RS_THREADS / 32; ++q) wc[q][tid] = 0;
        __syncthreads();
        const long long i = base + j * RS_THREADS + tid;
        const bool ok = i < n;
        const unsigned long long k = ok ? keys[i] : 0ull;
        const unsigned d = ok ? ((unsigned)(k >> shift) & 255u) : 256u;   // 256: no element
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned lt = peers & ((1u << lane) - 1u);
        if (ok && lt == 0) wc[w][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            unsigned pos = run[d] + __popc(lt);
            for (int q = 0; q < w; ++q) pos += wc[q][d];
            okeys[pos] = k;
            ovals[pos] = vals[i];
        }
        __syncthreads();
        unsigned add = 0;
        for (int q = 0; q < RS_THREADS / 32; ++q) add += wc[q][tid];
        run[tid] += add;
        __syncthreads();
    }
}

// 3. per tile the range [start, end) of its sorted keys
__global__ void k_rd_ranges(const unsigned long long *keys, long long n, uint2 *ranges) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const unsigned t = (unsigned)(keys[s] >> 32);
        if (s == 0 || (unsigned)(keys[s - 1] >> 32) != t) ranges[t].x = (unsigned)s;
        if (s == n - 1 || (unsigned)(keys[s + 1] >> 32) != t) ranges[t].y = (unsigned)(s + 1);
    }
}

// 4. compositing, one CTA per tile
__global__ void __launch_bounds__(TS * TS) k_rd_blend(Cam c, const uint2 *ranges, const unsigned *vals,
                                                      const float4 *g0, const float4 *g1, const float *col,
                                                      float bg0, float bg1, float bg2, float *img, float *trans) {
    __shared__ float4 s0[TS * TS], s1[TS * TS];
    __shared__ float sc[TS * TS * 3];
    const int tile = blockIdx.x, tx = tile % c.gx, ty = tile / c.gx;
    const int px = tx * TS + (threadIdx.x % TS), py = ty * TS + (threadIdx.x / TS);
    const bool inside = px < c.W && py < c.H;
    const uint2 r = ranges[tile];
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    bool done = !inside;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    for (unsigned b = r.x; b < r.y; b += TS * TS) {
        if (__syncthreads_count(done) == TS * TS) break;
        const unsigned s = b + threadIdx.x;
        if (s < r.y) {
            const unsigned i = vals[s];
            s0[threadIdx.x] = g0[i];
            s1[threadIdx.x] = g1[i];
            sc[3 * threadIdx.x] = col[3 * i];
            sc[3 * threadIdx.x + 1] = col[3 * i + 1];
            sc[3 * threadIdx.x + 2] = col[3 * i + 2];
        }
        __syncthreads();
        const int m = (int)min((unsigned)(TS * TS), r.y - b);
        for (int q = 0; q < m && !done; ++q) {
            const float4 a = s0[q], e = s1[q];
            const float dx = fx - a.x, dy = fy - a.y;
            const float power = -0.5f * (a.z * dx * dx + e.x * dy * dy) - a.w * dx * dy;
            if (power > 0.f) continue;
            const float alpha = fminf(0.99f, e.y * expf(power));
            if (alpha < 1.f / 255.f) continue;
            const float tt = T * (1.f - alpha);
            if (tt < 1e-4f) { done = true; continue; }
            C0 += sc[3 * q] * alpha * T;
            C1 += sc[3 * q + 1] * alpha * T;
            C2 += sc[3 * q + 2] * alpha * T;
            T = tt;
        }
    }
    if (inside) {
        float *o = img + 3 * ((size_t)py * c.W + px);
        o[0] = C0 + T * bg0;
        o[1] = C1 + T * bg1;
        o[2] = C2 + T * bg2;
        if (trans) trans[(size_t)py * c.W + px] = T;
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

extern "C" MPM_API mpm_status mpm_render(int64_t n, const float *mean, const float *cov, const float *color,
                                         const float *opacity, const float view[12], float fx, float fy, float cx,
                                         float cy, int32_t width, int32_t height, const float bg[3], float *image,
                                         float *trans, void *stream) {
    g_render_msg.clear();
    if (n < 0 || (n > 0 && (!mean || !cov || !color || !opacity)) || !view || !bg || !image || width < 1 ||
        height < 1 || width > 16384 || height > 16384 || n >= (1ll << 31)) {
        g_render_msg = "render: bad arguments";
        return MPM_ERR_INVALID_ARG;
    }
    if (mpm::any_on_other_device({mean, cov, color, opacity, image, trans})) {
        g_render_msg = "render: an array lives on another device than the current one";
        return MPM_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Cam c;
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) c.R[3 * r + q] = view[4 * r + q];
        c.T[r] = view[4 * r + 3];
    }
    c.fx = fx; c.fy = fy; c.cx = cx; c.cy = cy;
    c.W = width; c.H = height;
    c.gx = (width + TS - 1) / TS;
    c.gy = (height + TS - 1) / TS;
    const long long tiles = (long long)c.gx * c.gy;
    int tile_bits = 0;
    while ((1ll << tile_bits) < tiles) ++tile_bits;
    const long long npix = (long long)width * height;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    mpm_status status = MPM_OK;
    char *buf = nullptr, *kbuf = nullptr;
    unsigned long long total = 0;
#define RD_CK(call)                                                                   \
    do {                                                                              \
        if ((call) != cudaSuccess) {                                                  \
            g_render_msg = std::string("render: ") + cudaGetErrorString(cudaGetLastError()); \
            status = MPM_ERR_CUDA;                                                    \
            goto done;                                                                \
        }                                                                             \
    } while (0)
    {
        size_t off = 0;
        const size_t o_mean = off; off += al(n * 12);
        const size_t o_cov = off; off += al(n * 24);
        const size_t o_col = off; off += al(n * 12);
        const size_t o_op = off; off += al(n * 4);
        const size_t o_g0 = off; off += al(n * 16);
        const size_t o_g1 = off; off += al(n * 16);
        const size_t o_rect = off; off += al(n * 16);
        const size_t o_cnt = off; off += al(n * 4);
        const size_t o_off = off; off += al(n * 4);
        const size_t o_tot = off; off += al(8);
        const size_t o_bt = off; off += al(((n + SC_T - 1) / SC_T + 1) * 8);
        const size_t o_rng = off; off += al(tiles * 8);
        const size_t o_img = off; off += al(npix * 12);
        const size_t o_tr = off; off += al(npix * 4);
        if (cudaMallocAsync((void **)&buf, off, st) != cudaSuccess) {
            cudaGetLastError();
            buf = nullptr;
            g_render_msg = "render: device allocation failed";
            return MPM_ERR_OOM;
        }
        auto P = [&](size_t o) { return (void *)(buf + o); };
        const float *dmean = mean, *dcov = cov, *dcol = color, *dop = opacity;
        if (n > 0 && !is_dev(mean)) { RD_CK(cudaMemcpyAsync(P(o_mean), mean, n * 12, cudaMemcpyHostToDevice, st)); dmean = (const float *)P(o_mean); }
        if (n > 0 && !is_dev(cov)) { RD_CK(cudaMemcpyAsync(P(o_cov), cov, n * 24, cudaMemcpyHostToDevice, st)); dcov = (const float *)P(o_cov); }
        if (n > 0 && !is_dev(color)) { RD_CK(cudaMemcpyAsync(P(o_col), color, n * 12, cudaMemcpyHostToDevice, st)); dcol = (const float *)P(o_col); }
        if (n > 0 && !is_dev(opacity)) { RD_CK(cudaMemcpyAsync(P(o_op), opacity, n * 4, cudaMemcpyHostToDevice, st)); dop = (const float *)P(o_op); }
        float4 *g0 = (float4 *)P(o_g0), *g1 = (float4 *)P(o_g1);
        int4 *rect = (int4 *)P(o_rect);
        unsigned *cnt = (unsigned *)P(o_cnt), *offs = (unsigned *)P(o_off);
        unsigned long long *dtot = (unsigned long long *)P(o_tot);
        uint2 *ranges = (uint2 *)P(o_rng);
        RD_CK(cudaMemsetAsync(ranges, 0, tiles * 8, st));
        RD_CK(cudaMemsetAsync(dtot, 0, 8, st));
        if (n > 0) {
            k_rd_pre<<<blocks_for(n, 256), 256, 0, st>>>(n, dmean, dcov, dop, c, g0, g1, rect, cnt);
            scan_counts(cnt, offs, n, (unsigned long long *)P(o_bt), dtot, st);
            RD_CK(cudaGetLastError());
            RD_CK(cudaMemcpyAsync(&total, dtot, 8, cudaMemcpyDeviceToHost, st));
            RD_CK(cudaStreamSynchronize(st));
        }
        if (total >= (1ull << 32)) { g_render_msg = "render: too many tile overlaps"; status = MPM_ERR_CAPACITY; goto done; }
        if (total > 0) {
            const long long nk = (long long)total;
            const int nb = (int)((nk + RS_TILE - 1) / RS_TILE);
            size_t ko = 0;
            const size_t o_k0 = ko; ko += al(nk * 8);
            const size_t o_k1 = ko; ko += al(nk * 8);
            const size_t o_v0 = ko; ko += al(nk * 4);
            const size_t o_v1 = ko; ko += al(nk * 4);
            const size_t o_h = ko; ko += al((size_t)256 * nb * 4);
            const size_t o_ho = ko; ko += al((size_t)256 * nb * 4);
            const size_t o_ht = ko; ko += al(8);
            const size_t o_hb = ko; ko += al(((256ll * nb + SC_T - 1) / SC_T + 1) * 8);
            if (cudaMallocAsync((void **)&kbuf, ko, st) != cudaSuccess) {
                cudaGetLastError();
                kbuf = nullptr;
                g_render_msg = "render: device allocation failed";
                status = MPM_ERR_OOM;
                goto done;
            }
            unsigned long long *k0 = (unsigned long long *)(kbuf + o_k0), *k1 = (unsigned long long *)(kbuf + o_k1);
            unsigned *v0 = (unsigned *)(kbuf + o_v0), *v1 = (unsigned *)(kbuf + o_v1);
            unsigned *hist = (unsigned *)(kbuf + o_h), *hoff = (unsigned *)(kbuf + o_ho);
            unsigned long long *htot = (unsigned long long *)(kbuf + o_ht);
            k_rd_dup<<<blocks_for(n, 256), 256, 0, st>>>(n, g1, rect, cnt, offs, c.gx, k0, v0);
            RD_CK(cudaGetLastError());
            // keys: depth bits 0..31, tile above; 8-bit digits up to the tile's top bit
            const int bits = 32 + tile_bits;
            for (int shift = 0; shift < bits; shift += 8) {
                k_rs_hist<<<nb, RS_THREADS, 0, st>>>(k0, nk, shift, hist, nb);
                scan_counts(hist, hoff, (long long)256 * nb, (unsigned long long *)(kbuf + o_hb), htot, st);
                k_rs_scatter<<<nb, RS_THREADS, 0, st>>>(k0, v0, nk, shift, hoff, nb, k1, v1);
                RD_CK(cudaGetLastError());
                unsigned long long *tk = k0; k0 = k1; k1 = tk;
                unsigned *tv = v0; v0 = v1; v1 = tv;
            }
            k_rd_ranges<<<blocks_for(nk, 256), 256, 0, st>>>(k0, nk, ranges);
            RD_CK(cudaGetLastError());
            float *dimg = is_dev(image) ? image : (float *)P(o_img);
            float *dtr = trans ? (is_dev(trans) ? trans : (float *)P(o_tr)) : nullptr;
            k_rd_blend<<<(unsigned)tiles, TS * TS, 0, st>>>(c, ranges, v0, g0, g1, dcol, bg[0], bg[1], bg[2], dimg, dtr);
            RD_CK(cudaGetLastError());
            if (dimg != image) RD_CK(cudaMemcpyAsync(image, dimg, npix * 12, cudaMemcpyDeviceToHost, st));
            if (trans && dtr != trans) RD_CK(cudaMemcpyAsync(trans, dtr, npix * 4, cudaMemcpyDeviceToHost, st));
        } else {
            // nothing visible: the background everywhere
            float *dimg = is_dev(image) ? image : (float *)P(o_img);
            float *dtr = trans ? (is_dev(trans) ? trans : (float *)P(o_tr)) : nullptr;
            k_rd_blend<<<(unsigned)tiles, TS * TS, 0, st>>>(c, ranges, nullptr, g0, g1, dcol, bg[0], bg[1], bg[2], dimg, dtr);
            RD_CK(cudaGetLastError());
            if (dimg != image) RD_CK(cudaMemcpyAsync(image, dimg, npix * 12, cudaMemcpyDeviceToHost, st));
            if (trans && dtr != trans) RD_CK(cudaMemcpyAsync(trans, dtr, npix * 4, cudaMemcpyDeviceToHost, st));
        }
    }
done:
    if (kbuf) cudaFreeAsync(kbuf, st);
    if (buf) cudaFreeAsync(buf, st);
    if (status == MPM_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        g_render_msg = std::string("render: ") + cudaGetErrorString(cudaGetLastError());
        status = MPM_ERR_CUDA;
    }
#undef RD_CK
    return status;
}

extern "C" MPM_API const char *mpm_render_last_error(void) { return g_render_msg.c_str(); }
