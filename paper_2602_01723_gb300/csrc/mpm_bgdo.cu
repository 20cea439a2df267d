// mpm_bgdo.cu -- kernels of BGDO stage 2 (§4.3 "Optimization Algorithm";
// Algorithm 1, Stage 2; App. F): per-particle signals of one pseudo substep
// from a key frame, their average over key frames, the optional per-material
// mean and the log-E update.  The pseudo substep itself is the ordinary
// substep of mpm_forward.cu run on a copy of the key frame.
#include <cuda_runtime.h>

#include "mpm_internal.h"
#include "mpm_math.cuh"

namespace mpm {

// Young's modulus from the Lame pair (inverse of App. B.1 at fixed nu)
__device__ __forceinline__ float young_of(float mu, float lam) { return mu * (3.f * lam + 2.f * mu) / (lam + mu); }

// Adds one key frame's contribution to G.  key: the key-frame records; post:
// the records after the pseudo substep (== key when delta is taken before it).
//   g_tau = |tau(F_key)|_F: d|tau|/d log E equals |tau| because tau is linear
//           in (mu, lambda) and both are proportional to E at fixed nu
//   delta = |F_post - I|_F
//   G    += (eta log(1 + g_tau) - (1 - eta)(delta - delta_target)) / K
__global__ void k_bgdo_accum(Dev D, const float4 *__restrict__ key, const float4 *__restrict__ post, int first,
                             float inv_k, float delta_target, float w, float *__restrict__ G,
                             float *__restrict__ g_tau, float *__restrict__ delta) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < D.n; p += gridDim.x * blockDim.x) {
        const float4 *r = key + (size_t)p * REC_F4;
        const float4 r4 = r[4], r5 = r[5], r6 = r[6], r7 = r[7];
        const float F[9] = {r4.y, r4.z, r4.w, r5.x, r5.y, r5.z, r5.w, r6.x, r6.y};
        const float mu = r6.z, lam = r6.w;
        const int elastic = __float_as_int(r7.y) & 15;
        Sym t;
        float U[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f}, s[3] = {1.f, 1.f, 1.f}, e[3] = {0.f, 0.f, 0.f};
        if (elastic_needs_svd(elastic)) {
            float V[9], d[3];
            if (svd3_robust(F, U, V, s, e, d) == 2) set_err(D, ERRB_NONFINITE);
        }
        if (!kirchhoff(elastic, F, U, s, e, mu, lam, t)) {
            set_err(D, ERRB_NONFINITE);
            t = Sym{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        }
        const float g = sqrtf(t.xx * t.xx + t.yy * t.yy + t.zz * t.zz +
                              2.f * (t.xy * t.xy + t.xz * t.xz + t.yz * t.yz));
        float Fn[9];
        if (post == key) {
#pragma unroll
            for (int i = 0; i < 9; ++i) Fn[i] = F[i];
        } else {
            const float4 *q = post + (size_t)p * REC_F4;
            const float4 q4 = q[4], q5 = q[5], q6 = q[6];
            Fn[0] = q4.y; Fn[1] = q4.z; Fn[2] = q4.w; Fn[3] = q5.x; Fn[4] = q5.y;
            Fn[5] = q5.z; Fn[6] = q5.w; Fn[7] = q6.x; Fn[8] = q6.y;
        }
        Fn[0] -= 1.f; Fn[4] -= 1.f; Fn[8] -= 1.f;
        float d2 = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) d2 += Fn[i] * Fn[i];
        const float dl = sqrtf(d2);
        const float eta = w >= 0.f ? w : fminf(1.f, 0.1f * log1pf(young_of(mu, lam)));
        const float c = eta * log1pf(g) - (1.f - eta) * (dl - delta_target);
        G[p] = (first ? 0.f : G[p]) + c * inv_k;
        if (g_tau) g_tau[p] = g;
        if (delta) delta[p] = dl;
    }
}

// per-material sums of G and counts (sum[2m], sum[2m+1]) in FP64; lanes of a
// warp that share a material id combine before the atomic
__global__ void k_bgdo_material_sum(Dev D, int n_mat, const float *__restrict__ G, double *sum) {
    extern __shared__ double acc[];   // 2 * n_mat
    for (int t = threadIdx.x; t < 2 * n_mat; t += blockDim.x) acc[t] = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < D.n; base += gridDim.x * blockDim.x) {
        const int p = base + threadIdx.x;
        int m = -1;
        double g = 0.0;
        if (p < D.n) {
            m = __float_as_int(D.rec[(size_t)p * REC_F4 + 7].y) >> 8;
            g = (double)G[p];
            if (m < 0 || m >= n_mat) m = -1;
        }
        const unsigned same = __match_any_sync(0xffffffffu, m);
        // sum over the lanes in `same`
        double gs = 0.0, cs = 0.0;
        const double vc = m >= 0 ? 1.0 : 0.0;
#pragma unroll
        for (int o = 0; o < 32; ++o) {
            const double og = __shfl_sync(0xffffffffu, g, o), oc = __shfl_sync(0xffffffffu, vc, o);
            if ((same >> o) & 1u) { gs += og; cs += oc; }
        }
        const int leader = __ffs(same) - 1;
        if (m >= 0 && lane == leader) {
            atomicAdd(&acc[2 * m], gs);
            atomicAdd(&acc[2 * m + 1], cs);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * n_mat; t += blockDim.x)
        if (acc[t] != 0.0) atomicAdd(&sum[t], acc[t]);
}

// G_p <- mean of its material (when sum != NULL); log_E_p = log E_p - G_p
__global__ void k_bgdo_finish(Dev D, int n_mat, const float *__restrict__ Gin, const double *__restrict__ sum,
                              float *__restrict__ Gout, float *__restrict__ logE) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < D.n; p += gridDim.x * blockDim.x) {
        float g = Gin[p];
        if (sum) {
            const int m = __float_as_int(D.rec[(size_t)p * REC_F4 + 7].y) >> 8;
            g = (m >= 0 && m < n_mat && sum[2 * m + 1] > 0.0) ? (float)(sum[2 * m] / sum[2 * m + 1]) : __int_as_float(0x7fc00000);
        }
        if (Gout) Gout[p] = g;
        if (logE) {
            const float4 r6 = D.rec[(size_t)p * REC_F4 + 6];
            logE[p] = logf(young_of(r6.z, r6.w)) - g;
        }
    }
}

void launch_bgdo_accum(const Dev &D, const float4 *key, const float4 *post, int first, float inv_k,
                       float delta_target, float w, float *G, float *g_tau, float *delta, cudaStream_t st) {
    k_bgdo_accum<<<grid_for(D.n, 128), 128, 0, st>>>(D, key, post, first, inv_k, delta_target, w, G, g_tau, delta);
}
void launch_bgdo_material_sum(const Dev &D, int n_mat, const float *G, double *sum, cudaStream_t st) {
    k_bgdo_material_sum<<<grid_for(D.n, 256, 152 * 4), 256, 2 * n_mat * sizeof(double), st>>>(D, n_mat, G, sum);
}
void launch_bgdo_finish(const Dev &D, int n_mat, const float *G, const double *sum, float *Gout, float *logE,
                        cudaStream_t st) {
    k_bgdo_finish<<<grid_for(D.n, 256), 256, 0, st>>>(D, n_mat, G, sum, Gout, logE);
}

}  // namespace mpm
