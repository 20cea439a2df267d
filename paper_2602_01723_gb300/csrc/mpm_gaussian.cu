// mpm_gaussian.cu -- the Gaussian kernel each particle carries (§3.1) follows
// the deformation: Sigma(t) = F(t) Sigma F(t)^T (§3.2).  The covariance is a
// function of the current F and the rest covariance only, so it is evaluated
// when it is read, not carried through every substep.
#include <cuda_runtime.h>

#include "mpm_internal.h"

namespace mpm {

// cov0, out: n x 6 (xx xy xz yy yz zz); F read from the particle records
__global__ void k_covariance(Dev D, const float *__restrict__ cov0, float *__restrict__ out) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < D.n; p += gridDim.x * blockDim.x) {
        const float4 *r = D.rec + (size_t)p * REC_F4;
        const float4 r4 = r[4], r5 = r[5], r6 = r[6];
        const float F[9] = {r4.y, r4.z, r4.w, r5.x, r5.y, r5.z, r5.w, r6.x, r6.y};
        const float2 *c2 = reinterpret_cast<const float2 *>(cov0 + (size_t)6 * p);
        const float2 a = c2[0], b = c2[1], c = c2[2];
        const float S[9] = {a.x, a.y, b.x, a.y, b.y, c.x, b.x, c.x, c.y};
        float M[9];   // F Sigma
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                M[3 * i + j] = F[3 * i] * S[j] + F[3 * i + 1] * S[3 + j] + F[3 * i + 2] * S[6 + j];
        float T[6];   // (F Sigma) F^T, upper triangle
        T[0] = M[0] * F[0] + M[1] * F[1] + M[2] * F[2];
        T[1] = M[0] * F[3] + M[1] * F[4] + M[2] * F[5];
        T[2] = M[0] * F[6] + M[1] * F[7] + M[2] * F[8];
        T[3] = M[3] * F[3] + M[4] * F[4] + M[5] * F[5];
        T[4] = M[3] * F[6] + M[4] * F[7] + M[5] * F[8];
        T[5] = M[6] * F[6] + M[7] * F[7] + M[8] * F[8];
        float2 *o2 = reinterpret_cast<float2 *>(out + (size_t)6 * p);
        o2[0] = make_float2(T[0], T[1]);
        o2[1] = make_float2(T[2], T[3]);
        o2[2] = make_float2(T[4], T[5]);
    }
}

void launch_covariance(const Dev &D, const float *cov0, float *out, cudaStream_t st) {
    k_covariance<<<grid_for(D.n, 256), 256, 0, st>>>(D, cov0, out);
}

}  // namespace mpm
