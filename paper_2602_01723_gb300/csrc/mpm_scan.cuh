// mpm_scan.cuh -- exclusive scan of unsigned counts over many CTAs, shared
// by the splatting and MCIS translation units (internal linkage in each).
#pragma once
#include <cuda_runtime.h>

namespace {

// exclusive scan of n unsigned counts over many CTAs, three phases:
//   1. each CTA scans its 1024 counts and stores their sum in btot[block];
//   2. one CTA scans the block sums (exclusive, in place) and writes the
//      grand total to *total;
//   3. each CTA adds its block's offset.
constexpr int SC_T = 1024;
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long &tot) {
    __shared__ unsigned long long sh[SC_T / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    const unsigned long long ex = (w > 0 ? sh[w - 1] : 0ull) + x - v;
    tot = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return ex;
}
__global__ void __launch_bounds__(SC_T) k_sc_block(const unsigned *in, unsigned *out, long long n,
                                                   unsigned long long *btot) {
    const long long i = blockIdx.x * (long long)SC_T + threadIdx.x;
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan(i < n ? in[i] : 0u, tot);
    if (i < n) out[i] = (unsigned)ex;
    if (threadIdx.x == 0) btot[blockIdx.x] = tot;
}
__global__ void __launch_bounds__(SC_T) k_sc_totals(unsigned long long *btot, long long nb, unsigned long long *total) {
    unsigned long long carry = 0;
    for (long long b0 = 0; b0 < nb; b0 += SC_T) {
        const long long i = b0 + threadIdx.x;
        unsigned long long tot;
        const unsigned long long ex = block_exclusive_scan(i < nb ? btot[i] : 0ull, tot);
        if (i < nb) btot[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}
__global__ void __launch_bounds__(SC_T) k_sc_add(unsigned *out, long long n, const unsigned long long *btot) {
    const long long i = blockIdx.x * (long long)SC_T + threadIdx.x;
    if (i < n) out[i] += (unsigned)btot[blockIdx.x];
}

// exclusive scan of n counts into out (sums below 2^32), grand total to *total;
// btot: ceil(n / SC_T) scratch words
inline void scan_counts(const unsigned *in, unsigned *out, long long n, unsigned long long *btot, unsigned long long *total,
                 cudaStream_t st) {
    const long long nb = (n + SC_T - 1) / SC_T;
    if (nb > 0) k_sc_block<<<(unsigned)nb, SC_T, 0, st>>>(in, out, n, btot);
    k_sc_totals<<<1, SC_T, 0, st>>>(btot, nb, total);
    if (nb > 0) k_sc_add<<<(unsigned)nb, SC_T, 0, st>>>(out, n, btot);
}

}  // namespace
