// mpm_adjoint.cu -- recorded forward pass (checkpoints every ckpt_every
// substeps) and the reverse pass of the MLS-MPM substep.
//
// Reverse of one substep (state S_s -> S_{s+1}), given the adjoint of S_{s+1}:
//   S_s's binning and grid (mv, m and the updated v): kept in the grid tape
//               by the segment's recompute, or rebuilt (bin S_s, P2G, grid
//               update keeping (mv, m)) when the tape is off
//   k_adj_g2p : reverse of the return map, the F update, advection and the
//               G2P gathers; scatters the grid-velocity adjoint and writes the
//               partial adjoint of x and F
//   k_adj_grid: reverse of v = mask (mv/m + dt g) per node
//   k_adj_p2g : reverse of the P2G scatter and of the stress; completes the
//               adjoint of x, v, C, F and adds the parameter gradients
// The derivatives are taken by hand from the forward in mpm_forward.cu; the
// SVD-based pieces use closed forms in the singular basis (see the comments
// at plastic_adjoint and fcr_adjoint).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>
#include <string>

#include "mpm_internal.h"
#include "mpm_math.cuh"

namespace mpm {

// adjoint state of one particle: 6 float4 = x(3) v(3) C(9) F(9)
constexpr int ADJ_F4 = 6;

// ---------------------------------------------------------------------------
// device math of the reverse pass
// ---------------------------------------------------------------------------

// M = U Z V^T
__device__ __forceinline__ void u_z_vt(float M[9], const float U[9], const float Z[9], const float V[9]) {
    float T[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) T[3 * r + c] = U[3 * r] * Z[c] + U[3 * r + 1] * Z[3 + c] + U[3 * r + 2] * Z[6 + c];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[3 * r + c] = T[3 * r] * V[3 * c] + T[3 * r + 1] * V[3 * c + 1] + T[3 * r + 2] * V[3 * c + 2];
}
// K = U^T M V
__device__ __forceinline__ void ut_m_v(float K[9], const float U[9], const float M[9], const float V[9]) {
    float T[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) T[3 * r + c] = U[r] * M[c] + U[3 + r] * M[3 + c] + U[6 + r] * M[6 + c];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) K[3 * r + c] = T[3 * r] * V[c] + T[3 * r + 1] * V[3 + c] + T[3 * r + 2] * V[6 + c];
}

// Reverse of F_new = U diag(z(s)) V^T (the return map).  With K = U^T Fbar V:
//   diagonal:     sbar_k = sum_i K_ii dz_i/ds_k   (plus the parameter terms)
//   off-diagonal: Y_ij = K_ij (A+B)/2 + K_ji (A-B)/2,
//                 A = (z_i - z_j)/(s_i - s_j), B = (z_i + z_j)/(s_i + s_j)
//   Gbar = U (diag(sbar) + Y) V^T.
// In the projected case z_i = exp(h_i) with h_i - h_j = c (eps_i - eps_j),
// c = 1 - dgamma/|eps_hat|, so A = (z_j/s_j) expm1(c D)/expm1(D) with
// D = eps_i - eps_j, whose limit as D -> 0 is the isotropic c z_j / s_j.
__device__ void plastic_adjoint(int plastic, int rm, const float U[9], const float V[9], const float s[3],
                                const float d[3], const float z[3], float mu, float lam, float yield, float alpha,
                                const float Fbar[9], float Gbar[9], float &mubar, float &lambar, float &ybar) {
    float K[9];
    ut_m_v(K, U, Fbar, V);
    float Y[9];
    if (rm == RM_TIP) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Y[3 * i + j] = i == j ? 0.f : (K[3 * i + j] - K[3 * j + i]) / (s[i] + s[j]);
        u_z_vt(Gbar, U, Y, V);
        return;
    }
    // projected case
    float eps[3], deps[3], tr = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool clamped = !(s[i] > MPM_SIGMA_FLOOR);
        eps[i] = log_sigma(s[i], d[i]);
        deps[i] = clamped ? 0.f : 1.f / s[i];
        tr += eps[i];
    }
    const float m3 = tr * (1.f / 3.f);
    const float e[3] = {eps[0] - m3, eps[1] - m3, eps[2] - m3};
    const float nrm = sqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    float dg, ddg[3], ddg_mu, ddg_lam, ddg_y;
    if (plastic == PLASTIC_VM) {
        dg = nrm - yield / (2.f * mu);
#pragma unroll
        for (int k = 0; k < 3; ++k) ddg[k] = e[k] / nrm;
        ddg_mu = yield / (2.f * mu * mu);
        ddg_lam = 0.f;
        ddg_y = -1.f / (2.f * mu);
    } else {
        const float kap = (3.f * lam + 2.f * mu) / (2.f * mu) * alpha;
        dg = nrm + kap * tr;
#pragma unroll
        for (int k = 0; k < 3; ++k) ddg[k] = e[k] / nrm + kap;
        ddg_mu = tr * (-3.f * lam * alpha / (2.f * mu * mu));
        ddg_lam = tr * (3.f * alpha / (2.f * mu));
        ddg_y = 0.f;
    }
    const float inv_n = 1.f / nrm;
    float Jz[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float Pik = (i == k ? 1.f : 0.f) - (1.f / 3.f);
            const float dunit = (Pik - e[i] * e[k] * inv_n * inv_n) * inv_n;
            const float dh = (i == k ? 1.f : 0.f) - ddg[k] * e[i] * inv_n - dg * dunit;
            Jz[3 * i + k] = z[i] * dh * deps[k];
        }
    float sb[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k) sb[k] = K[0] * Jz[k] + K[4] * Jz[3 + k] + K[8] * Jz[6 + k];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float f = -z[i] * e[i] * inv_n * K[4 * i];
        mubar += f * ddg_mu;
        lambar += f * ddg_lam;
        ybar += f * ddg_y;
    }
    const float c = 1.f - dg * inv_n;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (i == j) { Y[4 * i] = sb[i]; continue; }
            float A;
            if (s[i] > MPM_SIGMA_FLOOR && s[j] > MPM_SIGMA_FLOOR) {
                const float D = eps[i] - eps[j];
                const float phi = fabsf(D) < 1e-3f ? c * (1.f + 0.5f * (c - 1.f) * D) : expm1f(c * D) / expm1f(D);
                A = z[j] / s[j] * phi;
            } else {
                A = (z[i] - z[j]) / (s[i] - s[j]);
            }
            const float B = (z[i] + z[j]) / (s[i] + s[j]);
            Y[3 * i + j] = K[3 * i + j] * 0.5f * (A + B) + K[3 * j + i] * 0.5f * (A - B);
        }
    u_z_vt(Gbar, U, Y, V);
}

// Reverse of the fixed-corotated Kirchhoff stress tau = 2 mu (F - R) F^T +
// lam J (J - 1) I for a symmetric adjoint T, in the singular basis of F:
// with W = U^T T U,
//   Z_ii = 2 mu W_ii (s_i + e_i) + Jbar prod_{k != i} s_k,  Jbar = lam tr(T) (2J - 1)
//   Z_ij = 2 mu W_ij [(s_j + e_j) - (s_j - s_i)/(s_i + s_j)]  (i != j)
//   Fbar += U Z V^T,  mubar += 2 sum_i e_i s_i W_ii,  lambar += tr(T) J (J - 1).
// (The (s_j - s_i)/(s_i + s_j) term is the reverse of the polar rotation.)
__device__ void fcr_adjoint(const float U[9], const float V[9], const float s[3], const float e[3], float mu,
                            float lam, const float T[9], float Fbar[9], float &mubar, float &lambar) {
    float W[9];
    ut_m_v(W, U, T, U);
    const float jm1 = e[0] + e[1] + e[2] + e[0] * e[1] + e[0] * e[2] + e[1] * e[2] + e[0] * e[1] * e[2];
    const float J = 1.f + jm1;
    const float trT = T[0] + T[4] + T[8];
    const float Jbar = lam * trT * (2.f * J - 1.f);
    float Z[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (i == j) {
                const float po = s[(i + 1) % 3] * s[(i + 2) % 3];
                Z[4 * i] = 2.f * mu * W[4 * i] * (s[i] + e[i]) + Jbar * po;
            } else {
                Z[3 * i + j] = 2.f * mu * W[3 * i + j] * ((s[j] + e[j]) - (s[j] - s[i]) / (s[i] + s[j]));
            }
        }
    float D[9];
    u_z_vt(D, U, Z, V);
#pragma unroll
    for (int t = 0; t < 9; ++t) Fbar[t] += D[t];
    mubar += 2.f * (e[0] * s[0] * W[0] + e[1] * s[1] * W[4] + e[2] * s[2] * W[8]);
    lambar += trT * J * jm1;
}

// Reverse of the Neo-Hookean Kirchhoff stress tau = mu (F F^T - I) + lam log J I:
//   Fbar += 2 mu T F + lam tr(T) F^{-T};  mubar += <T, F F^T - I>;  lambar += tr(T) log J
__device__ void nh_adjoint(const float F[9], float mu, float lam, const float T[9], float Fbar[9], float &mubar,
                           float &lambar) {
    const float cof[9] = {F[4] * F[8] - F[5] * F[7], F[5] * F[6] - F[3] * F[8], F[3] * F[7] - F[4] * F[6],
                          F[2] * F[7] - F[1] * F[8], F[0] * F[8] - F[2] * F[6], F[1] * F[6] - F[0] * F[7],
                          F[1] * F[5] - F[2] * F[4], F[2] * F[3] - F[0] * F[5], F[0] * F[4] - F[1] * F[3]};
    const float jm1 = det_minus_one(F);
    const float J = 1.f + jm1;
    const float trT = T[0] + T[4] + T[8];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Fbar[3 * r + c] += 2.f * mu * (T[3 * r] * F[c] + T[3 * r + 1] * F[3 + c] + T[3 * r + 2] * F[6 + c]) +
                               lam * trT * cof[3 * r + c] / J;
    // <T, F F^T - I> with F F^T - I = H + H^T + H H^T, H = F - I
    float h[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) h[t] = F[t];
    h[0] -= 1.f; h[4] -= 1.f; h[8] -= 1.f;
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float ffi = h[3 * i + j] + h[3 * j + i] + h[3 * i] * h[3 * j] + h[3 * i + 1] * h[3 * j + 1] +
                              h[3 * i + 2] * h[3 * j + 2];
            acc += T[3 * i + j] * ffi;
        }
    mubar += acc;
    lambar += trT * log1pf(jm1);
}

// Reverse of the further elastic models (out of line, like their forward):
//   StVK:   Fbar += 2 mu (2 T F E + F B) + lam tr(T)(2J - 1) cof F,  B = F^T T F,
//           mubar += 2 <T, F E F^T>, lambar += tr(T) J (J - 1)
//   Hencky: in the singular basis, with K = U^T T U and eps = log s:
//           Z_kk = (2 mu K_kk + lam tr K) / s_k,
//           Z_ij = 4 mu K_ij s_j (eps_i - eps_j) / (s_i^2 - s_j^2)   (i != j),
//           Fbar += U Z V^T, mubar += 2 sum K_ii eps_i, lambar += tr K tr eps
//           (floored singular values carry no derivative)
//   fluid:  Fbar += lam tr(T)(2J - 1) cof F, lambar += tr(T) J (J - 1)
//   volume: kappabar = tr(T)(J - 1/J): mubar += 2/3 kappabar, lambar += kappabar,
//           Fbar += kappa tr(T)(1 + 1/J^2) cof F
static __device__ __noinline__ void more_adjoint(int elastic, const float *F, const float *U, const float *V, const float *s,
                                          const float *e, float mu, float lam, const float *T, float *Fbar,
                                          float *mubar, float *lambar) {
    const float trT = T[0] + T[4] + T[8];
    const float jm1 = det_minus_one(F);
    const float J = 1.f + jm1;
    const float cof[9] = {F[4] * F[8] - F[5] * F[7], F[5] * F[6] - F[3] * F[8], F[3] * F[7] - F[4] * F[6],
                          F[2] * F[7] - F[1] * F[8], F[0] * F[8] - F[2] * F[6], F[1] * F[6] - F[0] * F[7],
                          F[1] * F[5] - F[2] * F[4], F[2] * F[3] - F[0] * F[5], F[0] * F[4] - F[1] * F[3]};
    if (elastic == ELASTIC_STVK) {
        float h[9];
        for (int i = 0; i < 9; ++i) h[i] = F[i];
        h[0] -= 1.f; h[4] -= 1.f; h[8] -= 1.f;
        float E[9], FE[9], TF[9], B[9], A[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                E[3 * i + j] = 0.5f * (h[3 * i + j] + h[3 * j + i] + h[i] * h[j] + h[3 + i] * h[3 + j] +
                                       h[6 + i] * h[6 + j]);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                FE[3 * i + j] = F[3 * i] * E[j] + F[3 * i + 1] * E[3 + j] + F[3 * i + 2] * E[6 + j];
                TF[3 * i + j] = T[3 * i] * F[j] + T[3 * i + 1] * F[3 + j] + T[3 * i + 2] * F[6 + j];
            }
        float acc = 0.f;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                // B = F^T (T F), A = F E F^T
                B[3 * i + j] = F[i] * TF[j] + F[3 + i] * TF[3 + j] + F[6 + i] * TF[6 + j];
                A[3 * i + j] = FE[3 * i] * F[3 * j] + FE[3 * i + 1] * F[3 * j + 1] + FE[3 * i + 2] * F[3 * j + 2];
                acc += T[3 * i + j] * A[3 * i + j];
            }
        const float Jbar = lam * trT * (2.f * J - 1.f);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                const float tfe = T[3 * i] * FE[j] + T[3 * i + 1] * FE[3 + j] + T[3 * i + 2] * FE[6 + j];
                const float fb = F[3 * i] * B[j] + F[3 * i + 1] * B[3 + j] + F[3 * i + 2] * B[6 + j];
                Fbar[3 * i + j] += 2.f * mu * (2.f * tfe + fb) + Jbar * cof[3 * i + j];
            }
        *mubar += 2.f * acc;
        *lambar += trT * J * jm1;
    } else if (elastic == ELASTIC_HENCKY) {
        float K[9];
        ut_m_v(K, U, T, U);
        float eps[3];
        bool live[3];
        for (int i = 0; i < 3; ++i) {
            live[i] = s[i] > MPM_SIGMA_FLOOR;
            eps[i] = live[i] ? log1pf(e[i]) : -9.210340371976184f;
        }
        const float trK = K[0] + K[4] + K[8], tre = eps[0] + eps[1] + eps[2];
        float Z[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                if (i == j) {
                    Z[4 * i] = live[i] ? (2.f * mu * K[4 * i] + lam * trK) / s[i] : 0.f;
                    continue;
                }
                float q;   // (eps_i - eps_j) / (s_i - s_j)
                const float ds = s[i] - s[j];
                if (live[i] && live[j]) {
                    const float r = ds / s[j];
                    q = fabsf(r) < 1e-3f ? (1.f - 0.5f * r + r * r * (1.f / 3.f)) / s[j] : log1pf(r) / ds;
                } else {
                    q = ds != 0.f ? (eps[i] - eps[j]) / ds : 0.f;
                }
                const float ss = s[i] + s[j];
                Z[3 * i + j] = ss != 0.f ? 4.f * mu * K[3 * i + j] * s[j] * q / ss : 0.f;
            }
        float D[9];
        u_z_vt(D, U, Z, V);
        for (int t = 0; t < 9; ++t) Fbar[t] += D[t];
        *mubar += 2.f * (K[0] * eps[0] + K[4] * eps[1] + K[8] * eps[2]);
        *lambar += trK * tre;
    } else if (elastic == ELASTIC_FLUID) {
        const float Jbar = lam * trT * (2.f * J - 1.f);
        for (int t = 0; t < 9; ++t) Fbar[t] += Jbar * cof[t];
        *lambar += trT * J * jm1;
    } else if (elastic == ELASTIC_VOLUME) {
        const float kappa = 2.f * mu / 3.f + lam, kb = trT * jm1 * (2.f + jm1) / J;
        *mubar += (2.f / 3.f) * kb;
        *lambar += kb;
        const float Jbar = kappa * trT * (1.f + 1.f / (J * J));
        for (int t = 0; t < 9; ++t) Fbar[t] += Jbar * cof[t];
    }
}

// Reverse of the volume-only plasticity F = c I, c = J^{1/3} (J clamped for
// Sigma, where a clamp stops the derivative): Gbar = tr(Fbar) c / (3 J) cof G
static __device__ __noinline__ void volume_plastic_adjoint(int plastic, const float *G, const float *Fbar, float *Gbar) {
    float jm1 = det_minus_one(G);
    const bool clamped = plastic == PLASTIC_SIGMA && (jm1 < 0.05f - 1.f || jm1 > 1.2f - 1.f);
    const float J = 1.f + jm1;
    const float c = J > 0.f ? expf(log1pf(jm1) * (1.f / 3.f)) : cbrtf(J);
    const float k = clamped ? 0.f : (Fbar[0] + Fbar[4] + Fbar[8]) * c / (3.f * J);
    Gbar[0] = k * (G[4] * G[8] - G[5] * G[7]); Gbar[1] = k * (G[5] * G[6] - G[3] * G[8]);
    Gbar[2] = k * (G[3] * G[7] - G[4] * G[6]); Gbar[3] = k * (G[2] * G[7] - G[1] * G[8]);
    Gbar[4] = k * (G[0] * G[8] - G[2] * G[6]); Gbar[5] = k * (G[1] * G[6] - G[0] * G[7]);
    Gbar[6] = k * (G[1] * G[5] - G[2] * G[4]); Gbar[7] = k * (G[2] * G[3] - G[0] * G[5]);
    Gbar[8] = k * (G[0] * G[4] - G[1] * G[3]);
}

// (mubar, lambar) -> (d/d log E, d/d nu), with E and nu recovered from mu, lambda
__device__ __forceinline__ void lame_chain(float mu, float lam, float mubar, float lambar, float &gE, float &gnu) {
    const float nu = lam / (2.f * (lam + mu));
    gE = mubar * mu + lambar * lam;
    const float q = 1.f - 2.f * nu;
    gnu = mubar * (-mu / (1.f + nu)) + lambar * (2.f * mu * (1.f + 2.f * nu * nu) / ((1.f + nu) * q * q));
}

// ---------------------------------------------------------------------------
// reverse kernels (chunked like the forward: particles of one 4^3 block)
// ---------------------------------------------------------------------------
constexpr int GT = 6, GT3 = 216;
constexpr int ADJ_THREADS = 128;

// The reverse G2P and P2G kernels are specialised for the models a material
// table uses, so that the common tables do not carry the registers, stack and
// instruction footprint of the rarer models.  The reverse G2P (which reverses
// the return map) by plasticity:
//   ADJ_ELASTIC  none
//   ADJ_PLASTIC  von Mises / Drucker-Prager
//   ADJ_ALL      also fluid / Sigma plasticity
// and the reverse P2G (which reverses the stress) by elasticity:
//   ADJ_FCR      fixed-corotated only
//   ADJ_FCR_NH   fixed-corotated and Neo-Hookean
//   ADJ_ALL      also StVK, Hencky, fluid and volume elasticity

__device__ __forceinline__ int page_slot_a(const Dev &D, int par, unsigned ep, int inst, int bx, int by, int bz) {
    if (bx < 0 || by < 0 || bz < 0 || bx >= D.NB[0] || by >= D.NB[1] || bz >= D.NB[2]) return -1;
    const unsigned k = block_key(D, inst, bx, by, bz);
    return D.page_epoch[par][k] == ep ? D.page[par][k] : -1;
}
__device__ __forceinline__ int node_loc(int I, int J, int K) { return ((I & 3) * 4 + (J & 3)) * 4 + (K & 3); }

// loads the 6^3-node tile (blocks B .. B+1) of pool `src` into shared memory
__device__ void load_tile(const Dev &D, const float4 *src, unsigned ep, int inst, int bx, int by, int bz,
                          float4 *tile, int *slots) {
    if (threadIdx.x < 8) {
        const int o = threadIdx.x;
        slots[o] = page_slot_a(D, 0, ep, inst, bx + (o >> 2), by + ((o >> 1) & 1), bz + (o & 1));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < GT3; t += blockDim.x) {
        const int i = t / (GT * GT), j = (t / GT) % GT, k = t % GT;
        const int sl = slots[((i >> 2) << 2) | ((j >> 2) << 1) | (k >> 2)];
        tile[t] = sl >= 0 ? src[(size_t)sl * BLK_NODES + node_loc(i, j, k)] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
}

struct ParticleIn {
    int q[3];                      // fixed-point position (cells = q 2^-qf)
    float v[3], C[9], F[9];
    float mass, vol, mu, lam, yield, alpha;
    int elastic, plastic;
};
__device__ __forceinline__ void unpack_particle(const float4 r[REC_F4], ParticleIn &P) {
    P.q[0] = rec_q(r[0].x); P.q[1] = rec_q(r[0].y); P.q[2] = rec_q(r[0].z); P.mass = r[0].w;
    P.v[0] = r[1].x; P.v[1] = r[1].y; P.v[2] = r[1].z; P.vol = r[1].w;
    P.C[0] = r[2].x; P.C[1] = r[2].y; P.C[2] = r[2].z; P.C[3] = r[2].w;
    P.C[4] = r[3].x; P.C[5] = r[3].y; P.C[6] = r[3].z; P.C[7] = r[3].w; P.C[8] = r[4].x;
    P.F[0] = r[4].y; P.F[1] = r[4].z; P.F[2] = r[4].w; P.F[3] = r[5].x; P.F[4] = r[5].y; P.F[5] = r[5].z;
    P.F[6] = r[5].w; P.F[7] = r[6].x; P.F[8] = r[6].y;
    P.mu = r[6].z; P.lam = r[6].w; P.yield = r[7].x;
    const int info = __float_as_int(r[7].y);
    P.elastic = info & 15;
    P.plastic = (info >> 4) & 15;
    P.alpha = r[7].w;
}

// shared memory of the reverse G2P kernel
constexpr int GTP = GT + 1;                  // padded row of the fixed-point tile
constexpr int GT3P = GT * GT * GTP;
__device__ __forceinline__ int gidx(int i, int j, int k) { return (i * GT + j) * GTP + k; }
constexpr int AS_F4 = 13;                   // staged stride: record words 0,1,4..7 (6) + adjoint (6), odd
struct AdjG2PSmem {
    float4 st[ADJ_THREADS * AS_F4];          // staged record and adjoint of the chunk's particles
    float4 g[GT3];                           // grid velocity tile (v, m)
    int t[3 * GT3P];                         // fixed-point grid-velocity adjoint, component-major
    float4 pk[ADJ_THREADS * 4];              // packets: f(3) - | vt(3) - | Ct(9) ...
    int4 cd[3];                              // chunk descriptors, ring of (c, c + G, c + 2G)
    unsigned pidx[ADJ_THREADS];              // sorted indices of the next chunk
    unsigned pe[8];                          // page words of the next chunk's 8 tile blocks
    int ps[8];
    int slot[2][8];                          // pool slots of the tile blocks, per chunk parity
    float red[ADJ_THREADS / 32];
    float scale;
};

__device__ __forceinline__ unsigned a_smem(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void a_cp16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(a_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void a_cp4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void a_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void a_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// the descriptors of this CTA's first two chunks (thread 0), read alongside
// the chunk count: any index within the array's capacity is readable, and
// one beyond the count is not used
__device__ __forceinline__ void first_descriptors(const Dev &D, int4 &cd0, int4 &cd1) {
    cd0 = cd1 = make_int4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        if (blockIdx.x < D.max_chunks) cd0 = D.chunks[blockIdx.x];
        if (blockIdx.x + gridDim.x < D.max_chunks) cd1 = D.chunks[blockIdx.x + gridDim.x];
    }
}

// level 2 of a chunk: sorted indices and the page words of its 8 tile blocks
template <typename SM>
__device__ __forceinline__ void adj_stage2(const Dev &D, SM &S, int4 ch, unsigned ep) {
    const int tid = threadIdx.x;
    if (tid < ch.z) a_cp4(&S.pidx[tid], D.sorted + ch.y + tid);
    const int t = tid - 64;   // lookups on the third warp
    if (t >= 0 && t < 8) {
        int inst, bx, by, bz;
        key_coords(D, (unsigned)ch.x, inst, bx, by, bz);
        const int qx = bx + (t >> 2), qy = by + ((t >> 1) & 1), qz = bz + (t & 1);
        if (qx >= D.NB[0] || qy >= D.NB[1] || qz >= D.NB[2]) {
            S.pe[t] = ep + 1u;
            S.ps[t] = -1;
        } else {
            const unsigned k = block_key(D, inst, qx, qy, qz);
            a_cp4(&S.pe[t], D.page_epoch[0] + k);
            a_cp4(&S.ps[t], D.page[0] + k);
        }
    }
}
// level 3: records and adjoints (instruction w of a warp: float4 l % 8 of particles 4 w + l / 8)
// and the gather tile; needs the level-2 words in shared memory
__device__ __forceinline__ void adj_stage3(const Dev &D, AdjG2PSmem &S, int4 ch, const float4 *ain, int buf,
                                           unsigned ep) {
    const int tid = threadIdx.x, lane = tid & 31, wbase = tid & ~31, piece = lane & 7;
    if (tid < 8) S.slot[buf][tid] = S.pe[tid] == ep ? S.ps[tid] : -1;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const int j = wbase + 4 * w + (lane >> 3);
        if (j < ch.z) {
            const size_t p = S.pidx[j];
            if (piece != 2 && piece != 3)
                a_cp16(&S.st[j * AS_F4 + (piece < 2 ? piece : piece - 2)], D.rec + p * REC_F4 + piece);
            if (piece < ADJ_F4) a_cp16(&S.st[j * AS_F4 + 6 + piece], ain + p * ADJ_F4 + piece);
        }
    }
    for (int t = tid; t < GT3; t += ADJ_THREADS) {
        const int i = t / (GT * GT), j = (t / GT) % GT, k = t % GT;
        const int b = ((i >> 2) << 2) | ((j >> 2) << 1) | (k >> 2);
        const int sl = S.pe[b] == ep ? S.ps[b] : -1;
        if (sl >= 0) a_cp16(&S.g[t], D.gv[0] + (size_t)sl * BLK_NODES + node_loc(i, j, k));
        else S.g[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Reverse of G2P, advection, F update and return map for the particles of
// one chunk per iteration, software-pipelined over the chunks a CTA owns:
// the next chunk's indices and page words (level 2, in flight during phase
// A) and its records, adjoints and grid-velocity tile (level 3, in flight
// during phase B and the flush) arrive by cp.async.  Phase A (one particle
// per thread): recompute v', C', G = (I + dt C') F; reverse the return map,
// the F update and advection; accumulate the position adjoint of the
// gathers; leave a packet (position in the tile, vbar_tot, Cbar_tot).  Phase
// B: scatter the grid-velocity adjoint wt (vbar_tot + 4/dx^2 Cbar_tot
// (x_i - x_p)) into an int32 fixed-point tile (per-chunk scale 2^30 / sum of
// per-particle bounds) and flush it with one vector reduction per touched
// node.
template <int MS>
__global__ void __launch_bounds__(ADJ_THREADS, 3) k_adj_g2p(Dev D, const float4 *__restrict__ ain, float4 *aout,
                                                         float4 *gpar, float4 *gbar) {
    __shared__ AdjG2PSmem S;
    int4 cd0, cd1;
    first_descriptors(D, cd0, cd1);
    const unsigned n_chunks = min(D.ctr[CTR_N_CHUNKS], D.max_chunks);
    const unsigned ep = D.ctr[CTR_EPOCH_OF + 0];
    const float dx = D.dx, inv_dx = D.inv_dx, dt = D.dt;
    const float c4 = 4.f * inv_dx * inv_dx;
    const int tid = threadIdx.x;
    unsigned c = blockIdx.x;
    if (c >= n_chunks) return;
    // prologue: descriptors of c and c + G, levels 2 and 3 of chunk c
    if (tid == 0) {
        S.cd[0] = cd0;
        if (c + gridDim.x < n_chunks) S.cd[1] = cd1;
    }
    for (int t = tid; t < 3 * GT3P; t += ADJ_THREADS) S.t[t] = 0;
    __syncthreads();
    adj_stage2(D, S, S.cd[0], ep);
    a_commit();
    a_wait();
    __syncthreads();
    adj_stage3(D, S, S.cd[0], ain, 0, ep);
    a_commit();
    a_wait();
    __syncthreads();
    for (int kc = 0;; ++kc) {
        const int4 ch = S.cd[kc % 3];
        const int cnt = min(ch.z, ADJ_THREADS);
        const unsigned cn = c + gridDim.x;
        const bool has_next = cn < n_chunks;
        const bool valid = tid < cnt;
        const unsigned p = valid ? S.pidx[tid] : 0u;   // read before level 2 of c + G overwrites it
        if (tid == 0 && cn + gridDim.x < n_chunks) a_cp16(&S.cd[(kc + 2) % 3], D.chunks + cn + gridDim.x);
        if (has_next) adj_stage2(D, S, S.cd[(kc + 1) % 3], ep);
        a_commit();
        int inst, bx, by, bz;
        key_coords(D, (unsigned)ch.x, inst, bx, by, bz);
        float4 rr[REC_F4], aa[ADJ_F4];
        if (valid) {
            const float4 *q = S.st + tid * AS_F4;
            rr[0] = q[0]; rr[1] = q[1]; rr[4] = q[2]; rr[5] = q[3]; rr[6] = q[4]; rr[7] = q[5];
#pragma unroll
            for (int w = 0; w < ADJ_F4; ++w) aa[w] = q[6 + w];
        }
        float bnd = 0.f;
        if (valid) {
            rr[2] = rr[3] = make_float4(0.f, 0.f, 0.f, 0.f);
            ParticleIn P;
            unpack_particle(rr, P);
            float f[3];
            int b[3];
            b[0] = base_cell_q(P.q[0], D, f[0]) - bx * BLK;
            b[1] = base_cell_q(P.q[1], D, f[1]) - by * BLK;
            b[2] = base_cell_q(P.q[2], D, f[2]) - bz * BLK;
            const bool ok = (unsigned)b[0] <= 3u && (unsigned)b[1] <= 3u && (unsigned)b[2] <= 3u;
            if (!ok) { set_err(D, ERRB_CFL); b[0] = min(max(b[0], 0), 3); b[1] = min(max(b[1], 0), 3); b[2] = min(max(b[2], 0), 3); }
            float w[3][3], dw[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a) { bspline_w(f[a], w[a]); bspline_dw(f[a], dw[a]); }
            // adjoint of the new state
            const float xb[3] = {aa[0].x, aa[0].y, aa[0].z};
            const float vb[3] = {aa[0].w, aa[1].x, aa[1].y};
            const float Cb[9] = {aa[1].z, aa[1].w, aa[2].x, aa[2].y, aa[2].z, aa[2].w, aa[3].x, aa[3].y, aa[3].z};
            const float Fb[9] = {aa[3].w, aa[4].x, aa[4].y, aa[4].z, aa[4].w, aa[5].x, aa[5].y, aa[5].z, aa[5].w};
            // x' = x + dt v': the velocity's total adjoint
            float xa[3] = {xb[0], xb[1], xb[2]};
            const float vt[3] = {vb[0] + dt * xb[0], vb[1] + dt * xb[1], vb[2] + dt * xb[2]};
            // The reverse of the gathers v' = sum w v_i and C' = c4 sum w v_i (x_i - x_p)^T
            // gives the position adjoint sum_i wbar_i grad w_i - c4 Ct^T sum_i w_i v_i,
            // with wbar_i = vt . v_i + c4 v_i^T Ct (x_i - x_p) and Ct the total adjoint
            // of C'.  The second term is c4 Ct^T v' (v' = sum w v_i), taken once after
            // the node loop.  Without plasticity Ct = Cb + dt Fb F^T does not depend
            // on C', so one pass over the 27 nodes recomputes v', C' and accumulates
            // the first term; with plasticity Ct needs the return map of C', and a
            // second pass follows.
            float Ct[9];
            float vn[3] = {0.f, 0.f, 0.f}, Bm[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (MS == ADJ_ELASTIC) {
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc)
                        Ct[3 * r + cc] = Cb[3 * r + cc] + dt * (Fb[3 * r] * P.F[3 * cc] + Fb[3 * r + 1] * P.F[3 * cc + 1] +
                                                                 Fb[3 * r + 2] * P.F[3 * cc + 2]);
            }
            const float cdx = c4 * dx;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int jj = 0; jj < 3; ++jj)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float wij = w[0][i] * w[1][jj];
                        const float wt = wij * w[2][k];
                        const float4 g = S.g[((b[0] + i) * GT + (b[1] + jj)) * GT + (b[2] + k)];
                        const float dd[3] = {(float)i - f[0], (float)jj - f[1], (float)k - f[2]};
                        const float a3[3] = {wt * g.x, wt * g.y, wt * g.z};
#pragma unroll
                        for (int r = 0; r < 3; ++r) {
                            vn[r] += a3[r];
#pragma unroll
                            for (int cc = 0; cc < 3; ++cc) Bm[3 * r + cc] += a3[r] * dd[cc];
                        }
                        if (MS == ADJ_ELASTIC) {
                            const float vi[3] = {g.x, g.y, g.z};
                            float wbar = 0.f;
#pragma unroll
                            for (int r = 0; r < 3; ++r)
                                wbar += vi[r] * (vt[r] + cdx * (Ct[3 * r] * dd[0] + Ct[3 * r + 1] * dd[1] + Ct[3 * r + 2] * dd[2]));
                            const float gw[3] = {dw[0][i] * w[1][jj] * w[2][k], w[0][i] * dw[1][jj] * w[2][k],
                                                 wij * dw[2][k]};
#pragma unroll
                            for (int cc = 0; cc < 3; ++cc) xa[cc] += wbar * inv_dx * gw[cc];
                        }
                    }
            float Cn[9], G[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) Cn[t] = 4.f * inv_dx * Bm[t];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    G[3 * r + cc] = P.F[3 * r + cc] + dt * (Cn[3 * r] * P.F[cc] + Cn[3 * r + 1] * P.F[3 + cc] +
                                                            Cn[3 * r + 2] * P.F[6 + cc]);
            // reverse of the return map
            float Gb[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) Gb[t] = Fb[t];
            float mubar = 0.f, lambar = 0.f, ybar = 0.f;
            if (MS == ADJ_ALL && P.plastic >= PLASTIC_FLUID) {
                volume_plastic_adjoint(P.plastic, G, Fb, Gb);
            } else if (MS != ADJ_ELASTIC && P.plastic != PLASTIC_NONE) {
                float U[9], V[9], s3[3], e3[3], d3[3], z[3], ze[3];
                svd3_robust(G, U, V, s3, e3, d3);
                const int rm = return_map(P.plastic, s3, e3, d3, P.mu, P.lam, P.yield, P.alpha, z, ze);
                if (rm != RM_ELASTIC)
                    plastic_adjoint(P.plastic, rm, U, V, s3, d3, z, P.mu, P.lam, P.yield, P.alpha, Fb, Gb, mubar,
                                    lambar, ybar);
            }
            // G = (I + dt C') F
            float Fp[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    if (MS != ADJ_ELASTIC)
                        Ct[3 * r + cc] = Cb[3 * r + cc] + dt * (Gb[3 * r] * P.F[3 * cc] + Gb[3 * r + 1] * P.F[3 * cc + 1] +
                                                                 Gb[3 * r + 2] * P.F[3 * cc + 2]);
                    Fp[3 * r + cc] = Gb[3 * r + cc] + dt * (Cn[r] * Gb[cc] + Cn[3 + r] * Gb[3 + cc] + Cn[6 + r] * Gb[6 + cc]);
                }
            if (MS != ADJ_ELASTIC) {
                // second pass: the weights' term with the Ct of the return map's
                // reverse (the outer loop stays rolled; its weights are selected,
                // not indexed, so that they stay in registers)
#pragma unroll 1
                for (int i = 0; i < 3; ++i) {
                    const float wi = i == 0 ? w[0][0] : (i == 1 ? w[0][1] : w[0][2]);
                    const float dwi = i == 0 ? dw[0][0] : (i == 1 ? dw[0][1] : dw[0][2]);
                    const float di = (float)i - f[0];
                    const float4 *gi = S.g + (b[0] + i) * GT * GT;
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj)
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float4 g = gi[(b[1] + jj) * GT + (b[2] + k)];
                            const float dd[3] = {di, (float)jj - f[1], (float)k - f[2]};
                            const float vi[3] = {g.x, g.y, g.z};
                            float wbar = 0.f;
#pragma unroll
                            for (int r = 0; r < 3; ++r)
                                wbar += vi[r] * (vt[r] + cdx * (Ct[3 * r] * dd[0] + Ct[3 * r + 1] * dd[1] + Ct[3 * r + 2] * dd[2]));
                            const float gw[3] = {dwi * w[1][jj] * w[2][k], wi * dw[1][jj] * w[2][k],
                                                 wi * w[1][jj] * dw[2][k]};
#pragma unroll
                            for (int cc = 0; cc < 3; ++cc) xa[cc] += wbar * inv_dx * gw[cc];
                        }
                }
            }
            // - c4 Ct^T v'
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) xa[cc] -= c4 * (Ct[cc] * vn[0] + Ct[3 + cc] * vn[1] + Ct[6 + cc] * vn[2]);
            float4 *op = aout + (size_t)p * ADJ_F4;
            op[0] = make_float4(xa[0], xa[1], xa[2], 0.f);
            op[1] = make_float4(0.f, 0.f, 0.f, 0.f);
            op[2] = make_float4(0.f, 0.f, 0.f, 0.f);
            op[3] = make_float4(0.f, 0.f, 0.f, Fp[0]);
            op[4] = make_float4(Fp[1], Fp[2], Fp[3], Fp[4]);
            op[5] = make_float4(Fp[5], Fp[6], Fp[7], Fp[8]);
            float gE, gnu;
            lame_chain(P.mu, P.lam, mubar, lambar, gE, gnu);
            float4 g4 = gpar[p];
            g4.x += gE; g4.y += gnu; g4.z += ybar;
            gpar[p] = g4;
            // packet for the scatter of the grid-velocity adjoint
            // base cell (0..3 per axis) exactly in .w as 1 + b0 + 4 b1 + 16 b2 (> 0 marks a valid packet)
            S.pk[tid * 4 + 0] = make_float4(f[0], f[1], f[2], (float)(1 + b[0] + 4 * b[1] + 16 * b[2]));
            S.pk[tid * 4 + 1] = make_float4(vt[0], vt[1], vt[2], Ct[0]);
            S.pk[tid * 4 + 2] = make_float4(Ct[1], Ct[2], Ct[3], Ct[4]);
            S.pk[tid * 4 + 3] = make_float4(Ct[5], Ct[6], Ct[7], Ct[8]);
            float cm = 0.f;
#pragma unroll
            for (int t = 0; t < 9; ++t) cm = fmaxf(cm, fabsf(Ct[t]));
            bnd = fmaxf(fabsf(vt[0]), fmaxf(fabsf(vt[1]), fabsf(vt[2]))) + 4.5f * c4 * dx * cm;
        } else {
            S.pk[tid * 4] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // per-chunk fixed-point scale
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bnd += __shfl_xor_sync(0xffffffffu, bnd, o);
        if ((tid & 31) == 0) S.red[tid >> 5] = bnd;
        // level 2 of chunk c + G has landed and phase A is done with the staged
        // buffers: level 3 of chunk c + G goes in flight
        a_wait();
        __syncthreads();
        if (has_next) adj_stage3(D, S, S.cd[(kc + 1) % 3], ain, (kc + 1) & 1, ep);
        a_commit();
        if (tid == 0) {
            float bs = 0.f;
            for (int wq = 0; wq < ADJ_THREADS / 32; ++wq) bs += S.red[wq];
            S.scale = bs > 0.f ? 1073741824.f / bs : 1.f;
        }
        __syncthreads();
        const float sc = S.scale;
        // phase B: lane-transposed mapping spreads a warp over the chunk's cells
        {
            const int j = (tid & 31) * (ADJ_THREADS / 32) + (tid >> 5);
            const float4 q0 = S.pk[j * 4];
            if (j < cnt && q0.w > 0.f) {
                const float4 q1 = S.pk[j * 4 + 1], q2 = S.pk[j * 4 + 2], q3 = S.pk[j * 4 + 3];
                const float vt[3] = {q1.x * sc, q1.y * sc, q1.z * sc};
                const float Cs[9] = {q1.w * sc * c4 * dx, q2.x * sc * c4 * dx, q2.y * sc * c4 * dx,
                                     q2.z * sc * c4 * dx, q2.w * sc * c4 * dx, q3.x * sc * c4 * dx,
                                     q3.y * sc * c4 * dx, q3.z * sc * c4 * dx, q3.w * sc * c4 * dx};
                const int code = (int)q0.w - 1;
                const int b[3] = {code & 3, (code >> 2) & 3, (code >> 4) & 3};
                const float f[3] = {q0.x, q0.y, q0.z};
                float w[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a) bspline_w(f[a], w[a]);
#pragma unroll 1
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj)
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float wt = w[0][i] * w[1][jj] * w[2][k];
                            const float d[3] = {(float)i - f[0], (float)jj - f[1], (float)k - f[2]};
                            const int node = gidx(b[0] + i, b[1] + jj, b[2] + k);
#pragma unroll
                            for (int r = 0; r < 3; ++r)
                                atomicAdd(&S.t[r * GT3P + node],
                                          __float2int_rn(wt * (vt[r] + Cs[3 * r] * d[0] + Cs[3 * r + 1] * d[1] + Cs[3 * r + 2] * d[2])));
                        }
            }
        }
        __syncthreads();
        const float isc = 1.f / sc;
        for (int t = tid; t < GT3; t += ADJ_THREADS) {
            const int i = t / (GT * GT), j = (t / GT) % GT, k = t % GT;
            const int q = gidx(i, j, k);
            const int a0 = S.t[q], a1 = S.t[GT3P + q], a2 = S.t[2 * GT3P + q];
            S.t[q] = 0; S.t[GT3P + q] = 0; S.t[2 * GT3P + q] = 0;   // cleared for the next chunk
            if (a0 | a1 | a2) {
                const int sl = S.slot[kc & 1][((i >> 2) << 2) | ((j >> 2) << 1) | (k >> 2)];
                if (sl >= 0)
                    red_add_v4(gbar + (size_t)sl * BLK_NODES + node_loc(i, j, k), (float)a0 * isc, (float)a1 * isc,
                               (float)a2 * isc, 0.f);
                else
                    set_err(D, ERRB_CAPACITY);
            }
        }
        // level 3 of chunk c + G has landed
        a_wait();
        __syncthreads();
        if (!has_next) break;
        c = cn;
    }
}

// reverse of the grid update, per active node: ubar = mask * vbar,
// Pbar = ubar / m, mbar = -(ubar . P) / m^2; also clears the momentum pool
__global__ void k_adj_grid(Dev D, float4 *gbar) {
    const unsigned total = min(D.ctr[CTR_N_ACTIVE + 0], D.max_active) * BLK_NODES;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const float4 a = D.gmv[0][i];
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a.w > 0.f) {
            const unsigned slot = i >> 6, l = i & 63u;
            int inst, bx, by, bz;
            key_coords(D, D.active[0][slot], inst, bx, by, bz);
            const int idx[3] = {bx * BLK + (int)(l >> 4), by * BLK + (int)((l >> 2) & 3u), bz * BLK + (int)(l & 3u)};
            const float im = 1.f / a.w;
            const float u[3] = {a.x * im + D.dt * D.g[0], a.y * im + D.dt * D.g[1], a.z * im + D.dt * D.g[2]};
            float mask[3] = {1.f, 1.f, 1.f};
            bool sticky = false;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (idx[d] < D.bound && D.wall[2 * d] == 2) sticky = true;
                if (idx[d] >= D.R[d] - D.bound && D.wall[2 * d + 1] == 2) sticky = true;
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (sticky) mask[d] = 0.f;
                if (idx[d] < D.bound && D.wall[2 * d] == 1 && u[d] < 0.f) mask[d] = 0.f;
                if (idx[d] >= D.R[d] - D.bound && D.wall[2 * d + 1] == 1 && u[d] > 0.f) mask[d] = 0.f;
            }
            const float4 vb = gbar[i];
            const float ub[3] = {mask[0] * vb.x, mask[1] * vb.y, mask[2] * vb.z};
            out = make_float4(ub[0] * im, ub[1] * im, ub[2] * im, -(ub[0] * a.x + ub[1] * a.y + ub[2] * a.z) * im * im);
        }
        gbar[i] = out;
        D.gmv[0][i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

constexpr int PS_F4 = 13;                   // staged stride: record (8), adjoint words 0,3,4,5 (4), gpar (1)
struct AdjP2GSmem {
    float4 st[ADJ_THREADS * PS_F4];
    float4 g[GT3];                           // grid adjoint tile (Pbar, mbar)
    int4 cd[3];
    unsigned pidx[ADJ_THREADS];
    unsigned pe[8];
    int ps[8];
};

// level 3 of the reverse P2G: records, the adjoint words it updates, the
// parameter gradients and the grid-adjoint tile
__device__ __forceinline__ void adj_p2g_stage3(const Dev &D, AdjP2GSmem &S, int4 ch, const float4 *aout,
                                               const float4 *gpar, const float4 *gbar, unsigned ep) {
    const int tid = threadIdx.x, lane = tid & 31, wbase = tid & ~31, piece = lane & 7;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const int j = wbase + 4 * w + (lane >> 3);
        if (j < ch.z) {
            const size_t p = S.pidx[j];
            a_cp16(&S.st[j * PS_F4 + piece], D.rec + p * REC_F4 + piece);
            if (piece < 4) a_cp16(&S.st[j * PS_F4 + 8 + piece], aout + p * ADJ_F4 + (piece == 0 ? 0 : piece + 2));
            else if (piece == 4) a_cp16(&S.st[j * PS_F4 + 12], gpar + p);
        }
    }
    for (int t = tid; t < GT3; t += ADJ_THREADS) {
        const int i = t / (GT * GT), j = (t / GT) % GT, k = t % GT;
        const int b = ((i >> 2) << 2) | ((j >> 2) << 1) | (k >> 2);
        const int sl = S.pe[b] == ep ? S.ps[b] : -1;
        if (sl >= 0) a_cp16(&S.g[t], gbar + (size_t)sl * BLK_NODES + node_loc(i, j, k));
        else S.g[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// three CTAs per SM (168 registers, a few bytes of spill) measured faster than two at 216
template <int EL>
__global__ void __launch_bounds__(ADJ_THREADS, 3) k_adj_p2g(Dev D, float4 *aout, float4 *gpar, const float4 *gbar) {
    __shared__ AdjP2GSmem S;
    int4 cd0, cd1;
    first_descriptors(D, cd0, cd1);
    const unsigned n_chunks = min(D.ctr[CTR_N_CHUNKS], D.max_chunks);
    const unsigned ep = D.ctr[CTR_EPOCH_OF + 0];
    const float dx = D.dx, inv_dx = D.inv_dx, dt = D.dt;
    const int tid = threadIdx.x;
    unsigned c = blockIdx.x;
    if (c >= n_chunks) return;
    if (tid == 0) {
        S.cd[0] = cd0;
        if (c + gridDim.x < n_chunks) S.cd[1] = cd1;
    }
    __syncthreads();
    adj_stage2(D, S, S.cd[0], ep);
    a_commit();
    a_wait();
    __syncthreads();
    adj_p2g_stage3(D, S, S.cd[0], aout, gpar, gbar, ep);
    a_commit();
    a_wait();
    __syncthreads();
    for (int kc = 0;; ++kc) {
        const int4 ch = S.cd[kc % 3];
        const int cnt = min(ch.z, ADJ_THREADS);
        const unsigned cn = c + gridDim.x;
        const bool has_next = cn < n_chunks;
        const unsigned p = tid < cnt ? S.pidx[tid] : 0u;   // read before level 2 of c + G overwrites it
        if (tid == 0 && cn + gridDim.x < n_chunks) a_cp16(&S.cd[(kc + 2) % 3], D.chunks + cn + gridDim.x);
        if (has_next) adj_stage2(D, S, S.cd[(kc + 1) % 3], ep);
        a_commit();
        int inst, bx, by, bz;
        key_coords(D, (unsigned)ch.x, inst, bx, by, bz);
        bool ok = tid < cnt;
        float4 o0, o3, o4, o5, g4;
        float xa[3], va[3], Ab[9], Fb[9], mubar = 0.f, lambar = 0.f;
        ParticleIn P;
        if (ok) {
            const float4 *q = S.st + tid * PS_F4;
            float4 rr[REC_F4];
#pragma unroll
            for (int w = 0; w < REC_F4; ++w) rr[w] = q[w];
            o0 = q[8]; o3 = q[9]; o4 = q[10]; o5 = q[11]; g4 = q[12];
            unpack_particle(rr, P);
            float f[3];
            int b[3];
            b[0] = base_cell_q(P.q[0], D, f[0]) - bx * BLK;
            b[1] = base_cell_q(P.q[1], D, f[1]) - by * BLK;
            b[2] = base_cell_q(P.q[2], D, f[2]) - bz * BLK;
            if ((unsigned)b[0] > 3u || (unsigned)b[1] > 3u || (unsigned)b[2] > 3u) { set_err(D, ERRB_CFL); ok = false; }
        }
        if (ok) {
            float f[3];
            int b[3];
            b[0] = base_cell_q(P.q[0], D, f[0]) - bx * BLK;
            b[1] = base_cell_q(P.q[1], D, f[1]) - by * BLK;
            b[2] = base_cell_q(P.q[2], D, f[2]) - bz * BLK;
            float w[3][3], dw[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a) { bspline_w(f[a], w[a]); bspline_dw(f[a], dw[a]); }
            // recompute the stress and the affine momentum A = m C - k tau
            float U[9], V[9], s3[3], e3[3], d3[3];
            Sym tau;
            if (EL == ADJ_ALL) {
                if (elastic_needs_svd(P.elastic)) svd3_robust_cold(P.F, U, V, s3, e3, d3);
                if (!kirchhoff(P.elastic, P.F, U, s3, e3, P.mu, P.lam, tau)) tau = Sym{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            } else if (EL == ADJ_FCR || P.elastic == ELASTIC_FCR) {
                svd3_robust_cold(P.F, U, V, s3, e3, d3);
                tau = tau_fcr(U, s3, e3, P.mu, P.lam);
            } else if (!tau_nh(P.F, P.mu, P.lam, tau)) {
                tau = Sym{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            }
            const float kf = 4.f * dt * P.vol * inv_dx * inv_dx;
            const float A[9] = {P.mass * P.C[0] - kf * tau.xx, P.mass * P.C[1] - kf * tau.xy,
                                P.mass * P.C[2] - kf * tau.xz, P.mass * P.C[3] - kf * tau.xy,
                                P.mass * P.C[4] - kf * tau.yy, P.mass * P.C[5] - kf * tau.yz,
                                P.mass * P.C[6] - kf * tau.xz, P.mass * P.C[7] - kf * tau.yz,
                                P.mass * P.C[8] - kf * tau.zz};
#pragma unroll
            for (int t = 0; t < 3; ++t) xa[t] = va[t] = 0.f;
#pragma unroll
            for (int t = 0; t < 9; ++t) Ab[t] = 0.f;
            // The P2G node contribution is w_i (m v + A (x_i - x_p)) and w_i m: its
            // reverse gives the position adjoint sum_i wbar_i grad w_i -
            // A^T sum_i w_i Pbar_i, with wbar_i = Pbar_i . (m v + A (x_i - x_p)) +
            // m mbar_i.  The second term is A^T va / m (va = m sum_i w_i Pbar_i),
            // taken once after the node loop.  The outer loop stays rolled; its
            // weights are selected, not indexed, so that they stay in registers.
            const float Pm[3] = {P.mass * P.v[0], P.mass * P.v[1], P.mass * P.v[2]};
            float sPb[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
            for (int i = 0; i < 3; ++i) {
                const float wi = i == 0 ? w[0][0] : (i == 1 ? w[0][1] : w[0][2]);
                const float dwi = i == 0 ? dw[0][0] : (i == 1 ? dw[0][1] : dw[0][2]);
                const float di = ((float)i - f[0]) * dx;
                const float4 *gi = S.g + (b[0] + i) * GT * GT;
#pragma unroll
                for (int jj = 0; jj < 3; ++jj)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float wjk = w[1][jj] * w[2][k];
                        const float wt = wi * wjk;
                        const float gw[3] = {dwi * wjk, wi * dw[1][jj] * w[2][k], wi * w[1][jj] * dw[2][k]};
                        const float dp[3] = {di, ((float)jj - f[1]) * dx, ((float)k - f[2]) * dx};
                        const float4 g = gi[(b[1] + jj) * GT + (b[2] + k)];
                        const float Pb[3] = {g.x, g.y, g.z};
                        float wbar = g.w * P.mass;
#pragma unroll
                        for (int r = 0; r < 3; ++r) {
                            const float Adr = A[3 * r] * dp[0] + A[3 * r + 1] * dp[1] + A[3 * r + 2] * dp[2];
                            wbar += Pb[r] * (Pm[r] + Adr);
                            const float wp = wt * Pb[r];
                            sPb[r] += wp;
#pragma unroll
                            for (int cc = 0; cc < 3; ++cc) Ab[3 * r + cc] += wp * dp[cc];
                        }
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) xa[cc] += wbar * inv_dx * gw[cc];
                    }
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) va[r] = P.mass * sPb[r];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) xa[cc] -= A[cc] * sPb[0] + A[3 + cc] * sPb[1] + A[6 + cc] * sPb[2];
            // C enters A as m C; tau as -k tau (tau symmetric: use the symmetric part)
            float T[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) T[3 * r + cc] = -0.5f * kf * (Ab[3 * r + cc] + Ab[3 * cc + r]);
#pragma unroll
            for (int t = 0; t < 9; ++t) Fb[t] = 0.f;
            if (EL == ADJ_FCR || P.elastic == ELASTIC_FCR) fcr_adjoint(U, V, s3, e3, P.mu, P.lam, T, Fb, mubar, lambar);
            else if (EL != ADJ_ALL || P.elastic == ELASTIC_NH) nh_adjoint(P.F, P.mu, P.lam, T, Fb, mubar, lambar);
            else more_adjoint(P.elastic, P.F, U, V, s3, e3, P.mu, P.lam, T, Fb, &mubar, &lambar);
        }
        // level 2 of chunk c + G has landed; the staged buffers are free
        a_wait();
        __syncthreads();
        if (has_next) adj_p2g_stage3(D, S, S.cd[(kc + 1) % 3], aout, gpar, gbar, ep);
        a_commit();
        if (ok) {
            float4 *op = aout + (size_t)p * ADJ_F4;
            op[0] = make_float4(o0.x + xa[0], o0.y + xa[1], o0.z + xa[2], va[0]);
            op[1] = make_float4(va[1], va[2], P.mass * Ab[0], P.mass * Ab[1]);
            op[2] = make_float4(P.mass * Ab[2], P.mass * Ab[3], P.mass * Ab[4], P.mass * Ab[5]);
            op[3] = make_float4(P.mass * Ab[6], P.mass * Ab[7], P.mass * Ab[8], o3.w + Fb[0]);
            op[4] = make_float4(o4.x + Fb[1], o4.y + Fb[2], o4.z + Fb[3], o4.w + Fb[4]);
            op[5] = make_float4(o5.x + Fb[5], o5.y + Fb[6], o5.z + Fb[7], o5.w + Fb[8]);
            float gE, gnu;
            lame_chain(P.mu, P.lam, mubar, lambar, gE, gnu);
            g4.x += gE; g4.y += gnu;
            gpar[p] = g4;
        }
        a_wait();
        __syncthreads();
        if (!has_next) break;
        c = cn;
    }
}

// clears the grid-adjoint pool of the active blocks
__global__ void k_adj_clear(Dev D, float4 *gbar) {
    const unsigned total = min(D.ctr[CTR_N_ACTIVE + 0], D.max_active) * BLK_NODES;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        gbar[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// adjoint of positions += dL/dx of one frame
// the current segment of the reverse pass, read by k_inject_tab
struct SegParams {
    const float *dldx;     // n_frames x n x 3
    long long s0;          // first substep of the segment
};
__global__ void k_set_seg(SegParams *sp, const float *dldx, long long s0) {
    sp->dldx = dldx;
    sp->s0 = s0;
}
// adds the loss gradient of every frame taken after substep s0 + j + 1
__global__ void k_inject_tab(int n, float4 *adj, const int *frame_first, const int *frame_next, const SegParams *sp,
                             int j) {
    const long long sub = sp->s0 + j + 1;
    int f = frame_first[sub];
    if (f < 0) return;
    const float *base = sp->dldx;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        float4 a = adj[(size_t)p * ADJ_F4];
        for (int g = f, guard = 0; g >= 0 && guard < 1 << 20; g = frame_next[g], ++guard) {
            const float *dl = base + (size_t)g * n * 3;
            a.x += dl[3 * p];
            a.y += dl[3 * p + 1];
            a.z += dl[3 * p + 2];
        }
        adj[(size_t)p * ADJ_F4] = a;
    }
}

// between two reverse substeps from the grid tape: clears the grid adjoint
// of the substep just reversed (the active blocks counted in prev_ctr; NULL:
// nothing to clear) and adds the loss gradient of every frame taken after
// substep s0 + j + 1
__global__ void k_adj_between(int n, float4 *adj, const int *frame_first, const int *frame_next, const SegParams *sp,
                              int j, const unsigned *prev_ctr, unsigned max_active, float4 *gbar) {
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    if (prev_ctr) {
        const unsigned total = min(prev_ctr[CTR_N_ACTIVE], max_active) * BLK_NODES;
        for (unsigned i = tid; i < total; i += stride) gbar[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const long long sub = sp->s0 + j + 1;
    const int f = frame_first[sub];
    if (f < 0) return;
    const float *base = sp->dldx;
    for (int p = (int)tid; p < n; p += (int)stride) {
        float4 a = adj[(size_t)p * ADJ_F4];
        for (int g = f, guard = 0; g >= 0 && guard < 1 << 20; g = frame_next[g], ++guard) {
            const float *dl = base + (size_t)g * n * 3;
            a.x += dl[3 * p];
            a.y += dl[3 * p + 1];
            a.z += dl[3 * p + 2];
        }
        adj[(size_t)p * ADJ_F4] = a;
    }
}

// the frame table from a by-value list (no host copy, so that it can be
// captured in a graph): per substep s <= S the first frame taken after s,
// per frame the next one taken there; one CTA
constexpr int FRAMES_BY_VALUE = 64;
struct FrameList {
    int n;
    int sub[FRAMES_BY_VALUE];
};
__global__ void k_frame_table(FrameList fl, int *first, int *next, long long S) {
    for (long long i = threadIdx.x; i <= S; i += blockDim.x) first[i] = -1;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int f = fl.n - 1; f >= 0; --f) {
            next[f] = first[fl.sub[f]];
            first[fl.sub[f]] = f;
        }
}

__global__ void k_export_grads(int n, const float4 *gpar, const float4 *adj, float *dparams, float *dstate0) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 g = gpar[p];
        dparams[3 * p] = g.x;
        dparams[3 * p + 1] = g.y;
        dparams[3 * p + 2] = g.z;
        if (dstate0) {
            const float *a = reinterpret_cast<const float *>(adj + (size_t)p * ADJ_F4);
            for (int t = 0; t < 24; ++t) dstate0[24 * p + t] = a[t];
        }
    }
}

// one state of a checkpoint segment as the reverse kernels read it: records,
// binning, counters (with grid buffer `par` renamed to buffer 0) and grid
struct TapeSlot {
    float4 *rec;
    unsigned *sorted;
    int4 *chunks;
    unsigned *ctr;
    unsigned *active;
    int *page;
    unsigned *page_epoch;
    float4 *gmv, *gv;
};

// Copies the current state, its binning and its grid (buffer par, after the
// grid update) into a tape slot, and clears the momentum of buffer par as the
// grid update would have.  The slot's page table receives only the entries
// of the active blocks, tagged with this activation's epoch; entries left
// from earlier uses carry older epochs, which the lookups reject.  A grid of
// more than gcap active blocks does not fit the slot: the kernel raises
// *over and records an empty slot (no chunks, no blocks), whose reverse
// kernels then do nothing; the host re-runs the reverse pass with larger
// slots.
__global__ void k_tape_save(Dev D, int par, TapeSlot T, unsigned gcap, unsigned *over, int strict) {
    const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    const size_t n = (size_t)D.n;
    const unsigned n_all = min(D.ctr[CTR_N_ACTIVE + par], D.max_active);
    const bool fits = n_all <= gcap;
    const unsigned n_act = fits ? n_all : 0u;
    const unsigned n_ch = fits ? min(D.ctr[CTR_N_CHUNKS], D.max_chunks) : 0u;
    const unsigned ep = D.ctr[CTR_EPOCH_OF + par];
    if (tid == 0 && !fits) {
        atomicOr(over, 1u);
        if (strict) set_err(D, ERRB_CAPACITY);   // no rerun possible: reported as an error
    }
    if (tid < CTR_COUNT) {
        unsigned v = D.ctr[tid];
        if (tid == CTR_N_ACTIVE) v = n_act;
        else if (tid == CTR_EPOCH_OF) v = ep;
        else if (tid == CTR_N_CHUNKS) v = n_ch;
        T.ctr[tid] = v;
    }
    for (size_t i = tid; i < n * REC_F4; i += stride) T.rec[i] = D.rec[i];
    for (size_t i = tid; i < n; i += stride) T.sorted[i] = D.sorted[i];
    for (size_t i = tid; i < n_ch; i += stride) T.chunks[i] = D.chunks[i];
    for (size_t a = tid; a < n_act; a += stride) {
        const unsigned k = D.active[par][a];
        T.active[a] = k;
        T.page[k] = (int)a;
        T.page_epoch[k] = ep;
    }
    const size_t kept = (size_t)n_act * BLK_NODES, nodes = (size_t)n_all * BLK_NODES;
    for (size_t i = tid; i < nodes; i += stride) {
        if (i < kept) {
            T.gmv[i] = D.gmv[par][i];
            T.gv[i] = D.gv[par][i];
        }
        D.gmv[par][i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// resident CTAs per SM of the reverse G2P (plasticity pl) and P2G
// (elasticity el) kernels: the smaller of the two
template <typename K> static int occupancy_of(K kernel) {
    int a = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, kernel, ADJ_THREADS, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return a;
}
int adjoint_occupancy(int pl, int el) {
    const int a = pl == ADJ_ELASTIC ? occupancy_of(k_adj_g2p<ADJ_ELASTIC>)
                                    : (pl == ADJ_PLASTIC ? occupancy_of(k_adj_g2p<ADJ_PLASTIC>) : occupancy_of(k_adj_g2p<ADJ_ALL>));
    const int b = el == ADJ_FCR ? occupancy_of(k_adj_p2g<ADJ_FCR>)
                                : (el == ADJ_FCR_NH ? occupancy_of(k_adj_p2g<ADJ_FCR_NH>) : occupancy_of(k_adj_p2g<ADJ_ALL>));
    return std::max(1, std::min(a, b));
}

// the reverse G2P / P2G pair of the context's model set
static void launch_adj_g2p(const mpm_ctx *ctx, const Dev &D, const float4 *ain, float4 *aout, cudaStream_t st) {
    const AdjointStore &A = ctx->adj;
    const int grid = ctx->grid_adj;
    if (ctx->adj_pl == ADJ_ELASTIC) k_adj_g2p<ADJ_ELASTIC><<<grid, ADJ_THREADS, 0, st>>>(D, ain, aout, A.gpar, A.gbar);
    else if (ctx->adj_pl == ADJ_PLASTIC) k_adj_g2p<ADJ_PLASTIC><<<grid, ADJ_THREADS, 0, st>>>(D, ain, aout, A.gpar, A.gbar);
    else k_adj_g2p<ADJ_ALL><<<grid, ADJ_THREADS, 0, st>>>(D, ain, aout, A.gpar, A.gbar);
}
static void launch_adj_p2g(const mpm_ctx *ctx, const Dev &D, float4 *aout, cudaStream_t st) {
    const AdjointStore &A = ctx->adj;
    const int grid = ctx->grid_adj;
    if (ctx->adj_el == ADJ_FCR) k_adj_p2g<ADJ_FCR><<<grid, ADJ_THREADS, 0, st>>>(D, aout, A.gpar, A.gbar);
    else if (ctx->adj_el == ADJ_FCR_NH) k_adj_p2g<ADJ_FCR_NH><<<grid, ADJ_THREADS, 0, st>>>(D, aout, A.gpar, A.gbar);
    else k_adj_p2g<ADJ_ALL><<<grid, ADJ_THREADS, 0, st>>>(D, aout, A.gpar, A.gbar);
}

void free_adjoint(AdjointStore &a) {
    for (float4 *p : a.ckpt)
        if (p) cudaFree(p);
    a.ckpt.clear();
    if (a.tape) cudaFree(a.tape);
    if (a.adj[0]) cudaFree(a.adj[0]);
    if (a.adj[1]) cudaFree(a.adj[1]);
    if (a.gpar) cudaFree(a.gpar);
    if (a.gbar) cudaFree(a.gbar);
    if (a.frames) cudaFree(a.frames);
    if (a.final_state) cudaFree(a.final_state);
    if (a.frame_first) cudaFree(a.frame_first);
    if (a.frame_next) cudaFree(a.frame_next);
    if (a.seg) cudaFree(a.seg);
    if (a.gt) cudaFree(a.gt);
    if (a.side) cudaStreamDestroy(a.side);
    if (a.ev_fork) cudaEventDestroy(a.ev_fork);
    if (a.ev_join) cudaEventDestroy(a.ev_join);
    for (int e = 0; e < AdjointStore::NGRAPH; ++e)
        if (a.seg_graph[e]) cudaGraphExecDestroy(a.seg_graph[e]);
    a = AdjointStore();
}

// checkpoint slot c, allocated if needed (not inside a stream capture)
static mpm_status checkpoint_slot(mpm_ctx *ctx, size_t c, cudaStream_t st) {
    AdjointStore &A = ctx->adj;
    const size_t bytes = (size_t)ctx->cap * REC_F4 * sizeof(float4);
    if (A.ckpt.size() <= c) A.ckpt.resize(c + 1, nullptr);
    if (!A.ckpt[c] || A.cap != ctx->cap) {
        if (stream_capturing(st))
            return ctx_fail(ctx, MPM_ERR_STATE, "inside a stream capture the checkpoints must exist from an earlier "
                                                "recorded run at least as long");
        if (A.ckpt[c]) cudaFree(A.ckpt[c]);
        A.ckpt[c] = nullptr;
        cudaError_t e = cudaMalloc(&A.ckpt[c], bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            A.ckpt[c] = nullptr;
            return ctx_fail(ctx, MPM_ERR_OOM, "checkpoint allocation failed");
        }
    }
    return MPM_OK;
}

static mpm_status save_checkpoint(mpm_ctx *ctx, size_t c, cudaStream_t st) {
    mpm_status s = checkpoint_slot(ctx, c, st);
    if (s) return s;
    cudaError_t e = cudaMemcpyAsync(ctx->adj.ckpt[c], ctx->D.rec, (size_t)ctx->D.n * REC_F4 * sizeof(float4),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return ctx_fail(ctx, MPM_ERR_CUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
    return MPM_OK;
}

// forward with checkpoints at every ckpt_every-th recorded substep
mpm_status record_substeps(mpm_ctx *ctx, int n_sub, cudaStream_t st) {
    if (ctx->record_broken)
        return ctx_fail(ctx, MPM_ERR_STATE, "recording interrupted by an unrecorded step; call mpm_record_reset");
    if (ctx->adj.cap != ctx->cap && !ctx->adj.ckpt.empty()) {
        for (float4 *p : ctx->adj.ckpt)
            if (p) cudaFree(p);
        ctx->adj.ckpt.clear();
    }
    const long long k = ctx->opt.ckpt_every;
    if (direct_forward(ctx, n_sub)) {
        // one run; the checkpoints of the states it reaches are copied after
        // the substeps that complete them
        if (ctx->recorded % k == 0) {
            mpm_status s = save_checkpoint(ctx, (size_t)(ctx->recorded / k), st);
            if (s) return s;
        }
        std::vector<StateCopy> copies;
        for (long long j = k - ctx->recorded % k; j < n_sub; j += k) {
            const size_t c = (size_t)((ctx->recorded + j) / k);
            mpm_status s = checkpoint_slot(ctx, c, st);
            if (s) return s;
            copies.push_back(StateCopy{(int)j, ctx->adj.ckpt[c]});
        }
        ctx->adj.cap = ctx->cap;
        mpm_status s = run_substeps(ctx, n_sub, st, nullptr, 0, &copies);
        if (s) return s;
        ctx->recorded += n_sub;
        return MPM_OK;
    }
    int remaining = n_sub;
    while (remaining > 0) {
        if (ctx->recorded % k == 0) {
            mpm_status s = save_checkpoint(ctx, (size_t)(ctx->recorded / k), st);
            if (s) return s;
            ctx->adj.cap = ctx->cap;
        }
        const int seg = (int)std::min<long long>(remaining, k - ctx->recorded % k);
        mpm_status s = run_substeps(ctx, seg, st);
        if (s) return s;
        ctx->recorded += seg;
        remaining -= seg;
    }
    return MPM_OK;
}

template <typename T>
static mpm_status dev_alloc(mpm_ctx *ctx, T **p, size_t count) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return ctx_fail(ctx, MPM_ERR_OOM, "reverse-pass allocation failed");
    }
    return MPM_OK;
}

// consume any pending binning, then bin the current records

// reverse of one substep whose input state is `state`
static void adjoint_substep(mpm_ctx *ctx, float4 *state, float4 *ain, float4 *aout, cudaStream_t st) {
    Dev &D = ctx->D;
    AdjointStore &A = ctx->adj;
    float4 *saved = D.rec;
    D.rec = state;
    rebin(ctx, st);
    L_plan(ctx, 1, st);
    L_prepare(ctx, -1, 0, 1, st);
    L_substep(ctx, 0, 0, 0, st);                       // P2G of the recorded state
    L_prepare(ctx, 0, -1, 0, st, 1);                   // v = mask(mv/m + dt g), keeping (mv, m)
    launch_adj_g2p(ctx, D, ain, aout, st);
    k_adj_grid<<<ctx->grid_small, 256, 0, st>>>(D, A.gbar);
    launch_adj_p2g(ctx, D, aout, st);
    k_adj_clear<<<ctx->grid_small, 256, 0, st>>>(D, A.gbar);
    ctx->launches += 4;
    D.rec = saved;
}

constexpr size_t GT_HEADER = 256;   // grid-tape header: word 0 = overflow flag

// byte offsets of the parts of one grid-tape slot (records, sorted index,
// chunks, counters, active list, page table, page epochs, momentum, velocity)
// for a grid pool of `pool` blocks; returns the slot size
static size_t gt_layout(const mpm_ctx *ctx, unsigned pool, size_t off[9]) {
    const size_t cap = (size_t)ctx->cap, nb = (size_t)ctx->total_blocks, gp = pool;
    const size_t bytes[9] = {cap * REC_F4 * sizeof(float4), cap * sizeof(unsigned), (size_t)ctx->chunk_cap * sizeof(int4),
                             CTR_COUNT * sizeof(unsigned), gp * sizeof(unsigned), nb * sizeof(int), nb * sizeof(unsigned),
                             gp * BLK_NODES * sizeof(float4), gp * BLK_NODES * sizeof(float4)};
    size_t o = 0;
    for (int i = 0; i < 9; ++i) {
        off[i] = o;
        o += (bytes[i] + 255) & ~size_t(255);
    }
    return o;
}

static TapeSlot tape_slot(mpm_ctx *ctx, int bank, int j) {
    AdjointStore &A = ctx->adj;
    size_t off[9];
    gt_layout(ctx, A.gt_pool, off);
    char *b = A.gt + GT_HEADER + ((size_t)bank * A.gt_bank_states + (size_t)j) * A.gt_slot_bytes;
    TapeSlot T;
    T.rec = reinterpret_cast<float4 *>(b + off[0]);
    T.sorted = reinterpret_cast<unsigned *>(b + off[1]);
    T.chunks = reinterpret_cast<int4 *>(b + off[2]);
    T.ctr = reinterpret_cast<unsigned *>(b + off[3]);
    T.active = reinterpret_cast<unsigned *>(b + off[4]);
    T.page = reinterpret_cast<int *>(b + off[5]);
    T.page_epoch = reinterpret_cast<unsigned *>(b + off[6]);
    T.gmv = reinterpret_cast<float4 *>(b + off[7]);
    T.gv = reinterpret_cast<float4 *>(b + off[8]);
    return T;
}

static unsigned *gt_over(mpm_ctx *ctx) { return reinterpret_cast<unsigned *>(ctx->adj.gt); }

// grid-pool blocks per slot: the whole pool after an overflow, else twice
// the larger activation of the two working grids plus slack (the recorded
// end state's; read synchronously, once per allocation)
static unsigned gt_pool_for(mpm_ctx *ctx, cudaStream_t st) {
    AdjointStore &A = ctx->adj;
    if (A.gt_pool_want) return std::min(A.gt_pool_want, ctx->pool_blocks);
    unsigned c[CTR_COUNT];
    if (cudaMemcpyAsync(c, ctx->D.ctr, sizeof(c), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return ctx->pool_blocks;
    }
    const unsigned long long want = 2ull * std::max(c[CTR_N_ACTIVE], c[CTR_N_ACTIVE + 1]) + 256ull;
    return (unsigned)std::min<unsigned long long>(want, ctx->pool_blocks);
}

// the side stream and fork / join events of the overlapped reverse pass
static bool ensure_side(mpm_ctx *ctx) {
    AdjointStore &A = ctx->adj;
    if (!A.side && cudaStreamCreateWithFlags(&A.side, cudaStreamNonBlocking) != cudaSuccess) A.side = nullptr;
    if (!A.ev_fork && cudaEventCreateWithFlags(&A.ev_fork, cudaEventDisableTiming) != cudaSuccess) A.ev_fork = nullptr;
    if (!A.ev_join && cudaEventCreateWithFlags(&A.ev_join, cudaEventDisableTiming) != cudaSuccess) A.ev_join = nullptr;
    if (A.side && A.ev_fork && A.ev_join) return true;
    cudaGetLastError();
    return false;
}

// grid tape of two banks of `states` slots for the current capacities,
// zeroed (epoch 0 never belongs to an activation, and the overflow flag
// starts clear); false when it cannot be allocated
static bool ensure_grid_tape(mpm_ctx *ctx, size_t states, cudaStream_t st) {
    AdjointStore &A = ctx->adj;
    const long long shape[3] = {ctx->cap, (long long)ctx->chunk_cap, ctx->total_blocks};
    if (A.gt && A.gt_bank_states >= states && std::equal(shape, shape + 3, A.gt_shape) &&
        (!A.gt_pool_want || A.gt_pool >= std::min(A.gt_pool_want, ctx->pool_blocks)))
        return true;
    if (A.gt) cudaFree(A.gt);
    A.gt = nullptr;
    A.gt_bank_states = 0;
    if (!ensure_side(ctx)) return false;
    const unsigned pool = gt_pool_for(ctx, st);
    size_t off[9];
    const size_t slot = gt_layout(ctx, pool, off), bytes = GT_HEADER + 2 * states * slot;
    if (cudaMalloc(&A.gt, bytes) != cudaSuccess) {
        cudaGetLastError();
        A.gt = nullptr;
        return false;
    }
    if (cudaMemsetAsync(A.gt, 0, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(A.gt);
        A.gt = nullptr;
        return false;
    }
    A.gt_slot_bytes = slot;
    A.gt_bank_states = states;
    A.gt_pool = pool;
    std::copy(shape, shape + 3, A.gt_shape);
    A.gt_shape[3] = pool;
    ++A.gt_gen;
    return true;
}

// The segment's forward from its checkpoint (in D.rec, binned by the
// caller), keeping every state s = 0 .. len-1 with its binning and grid in
// slot s of grid-tape bank `bank`.  The last state is scattered and its grid
// updated as well, since its reverse substep reads them.  The grid update
// keeps the momentum for the save, which clears it.  Leaves the last state
// in D.rec with no binning pending.
static void tape_segment(mpm_ctx *ctx, int len, int bank, cudaStream_t st) {
    AdjointStore &A = ctx->adj;
    L_plan(ctx, 3, st);               // epochs for buffer 0 (P2G below) and 1 (first fused substep)
    L_prepare(ctx, -1, 0, 1, st);
    L_substep(ctx, 0, 0, 0, st);
    for (int s = 0; s < len; ++s) {
        const int par = s & 1;
        const bool more = s + 1 < len;
        L_prepare(ctx, par, more ? par ^ 1 : -1, s > 0, st, 1);
        k_tape_save<<<ctx->grid_small, 256, 0, st>>>(ctx->D, par, tape_slot(ctx, bank, s), A.gt_pool, gt_over(ctx),
                                                     A.strict ? 1 : 0);
        ++ctx->launches;
        if (more) {
            L_substep(ctx, 1, par, par ^ 1, st);
            L_plan(ctx, 1 << par, st);
        }
    }
}

// the device context of a grid-tape slot: its records, binning, counters
// and grid in place of the working ones (as grid buffer 0)
static Dev slot_dev(mpm_ctx *ctx, const TapeSlot &T) {
    Dev Dj = ctx->D;
    Dj.rec = T.rec;
    Dj.sorted = T.sorted;
    Dj.chunks = T.chunks;
    Dj.ctr = T.ctr;
    Dj.active[0] = T.active;
    Dj.page[0] = T.page;
    Dj.page_epoch[0] = T.page_epoch;
    Dj.gmv[0] = T.gmv;
    Dj.gv[0] = T.gv;
    return Dj;
}

// reverse of one substep from a grid-tape slot: the adjoint kernels only
// (the grid adjoint it leaves is cleared by the next k_adj_between, or by
// the segment's final clear)
static void adjoint_taped(mpm_ctx *ctx, const TapeSlot &T, float4 *ain, float4 *aout, cudaStream_t st) {
    AdjointStore &A = ctx->adj;
    const Dev Dj = slot_dev(ctx, T);
    launch_adj_g2p(ctx, Dj, ain, aout, st);
    k_adj_grid<<<ctx->grid_small, 256, 0, st>>>(Dj, A.gbar);
    launch_adj_p2g(ctx, Dj, aout, st);
    ctx->launches += 3;
}

// reverse substeps len-1 .. 0 of a segment from grid-tape bank `bank`;
// before each, one launch clears the previous substep's grid adjoint and
// injects the frame gradients from the device table.  Leaves the grid
// adjoint zero.
static void reverse_segment(mpm_ctx *ctx, int len, int bank, int cur, int pg, cudaStream_t st) {
    AdjointStore &A = ctx->adj;
    const int n = ctx->D.n;
    for (int j = len - 1; j >= 0; --j) {
        const unsigned *prev = j + 1 < len ? tape_slot(ctx, bank, j + 1).ctr : nullptr;
        k_adj_between<<<pg, 256, 0, st>>>(n, A.adj[cur], A.frame_first, A.frame_next, (const SegParams *)A.seg, j,
                                          prev, ctx->D.max_active, A.gbar);
        ++ctx->launches;
        adjoint_taped(ctx, tape_slot(ctx, bank, j), A.adj[cur], A.adj[cur ^ 1], st);
        cur ^= 1;
    }
    k_adj_clear<<<ctx->grid_small, 256, 0, st>>>(slot_dev(ctx, tape_slot(ctx, bank, 0)), A.gbar);
    ++ctx->launches;
}

// One segment of the reverse pass without the grid tape, on the checkpoint
// already in D.rec: tape the segment's states by one forward pass, then
// reverse its substeps from the last, each rebuilding its state's binning
// and grid.  Leaves the adjoint in adj[cur ^ (len & 1)].
static mpm_status segment_body(mpm_ctx *ctx, int len, int cur, int pg, cudaStream_t st) {
    Dev &D = ctx->D;
    AdjointStore &A = ctx->adj;
    const size_t n = (size_t)D.n;
    rebin(ctx, st);
    if (cudaMemcpyAsync(A.tape, D.rec, n * REC_F4 * sizeof(float4), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return ctx_fail(ctx, MPM_ERR_CUDA, "tape copy");
    mpm_status s;
    if (len > 1 && (s = run_substeps(ctx, len - 1, st, A.tape, (size_t)ctx->cap * REC_F4))) return s;
    for (int j = len - 1; j >= 0; --j) {
        k_inject_tab<<<pg, 256, 0, st>>>((int)n, A.adj[cur], A.frame_first, A.frame_next, (const SegParams *)A.seg, j);
        ++ctx->launches;
        adjoint_substep(ctx, A.tape + (size_t)j * ctx->cap * REC_F4, A.adj[cur], A.adj[cur ^ 1], st);
        cur ^= 1;
    }
    return MPM_OK;
}

// One step of the reverse pass.  kind 0: a whole segment without the grid
// tape (lenR substeps, adjoint parity cur).  kind 1: the reverse of a
// segment of lenR substeps (0: none) from grid-tape bank bankR and, at the
// same time on the side stream, the recompute of the segment before it
// (lenP substeps, 0: none) into bank bankP, from the checkpoint the caller
// has put in D.rec.  The two touch disjoint memory: the recompute the
// working state, grids and binning, the reverse only its bank's slots and
// the adjoint buffers.
struct RevJob {
    int kind, lenR, bankR, cur, lenP, bankP;
};

static mpm_status run_job(mpm_ctx *ctx, const RevJob &J, int pg, cudaStream_t st) {
    if (J.kind == 0) return segment_body(ctx, J.lenR, J.cur, pg, st);
    AdjointStore &A = ctx->adj;
    const bool fork = J.lenP > 0 && J.lenR > 0;
    cudaStream_t sp = st;
    if (fork) {
        if (cudaEventRecord(A.ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(A.side, A.ev_fork, 0) != cudaSuccess)
            return ctx_fail(ctx, MPM_ERR_CUDA, "reverse pass: stream fork");
        sp = A.side;
    }
    if (J.lenP > 0) {
        rebin(ctx, sp);
        tape_segment(ctx, J.lenP, J.bankP, sp);
    }
    if (J.lenR > 0) reverse_segment(ctx, J.lenR, J.bankR, J.cur, pg, st);
    if (fork && (cudaEventRecord(A.ev_join, A.side) != cudaSuccess || cudaStreamWaitEvent(st, A.ev_join, 0) != cudaSuccess))
        return ctx_fail(ctx, MPM_ERR_CUDA, "reverse pass: stream join");
    return MPM_OK;
}

// the step as a CUDA graph, captured on the library's own stream (the side
// stream joins the capture through the fork event) the first time a step of
// this shape runs with these buffers
static cudaGraphExec_t job_graph(mpm_ctx *ctx, const RevJob &J, int pg, long long &launches) {
    AdjointStore &A = ctx->adj;
    constexpr int NK = AdjointStore::NKEY, NG = AdjointStore::NGRAPH;
    auto u = [](const void *p) { return (long long)(uintptr_t)p; };
    const long long key[NK] = {J.kind, J.lenR, J.bankR * 2 + J.cur, J.lenP * 2 + J.bankP,
                               (long long)ctx->D.n * 1000003ll + ctx->generation, u(A.gbar), u(A.adj[0]), u(A.adj[1]),
                               u(A.gpar), u(A.frame_first), u(A.frame_next), u(A.seg), u(A.tape), A.gt_gen};
    ++A.seg_clock;
    for (int e = 0; e < NG; ++e)
        if (A.seg_graph[e] && std::equal(key, key + NK, A.seg_key[e])) {
            A.seg_used[e] = A.seg_clock;
            launches = A.seg_launches[e];
            return A.seg_graph[e];
        }
    int e = 0;   // least recently used entry
    for (int i = 1; i < NG; ++i)
        if (A.seg_used[i] < A.seg_used[e]) e = i;
    if (A.seg_graph[e]) { cudaGraphExecDestroy(A.seg_graph[e]); A.seg_graph[e] = nullptr; }
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ctx->cap_stream = nullptr;
        return nullptr;
    }
    const long long l0 = ctx->launches;
    const bool pend = ctx->bins_pending;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const mpm_status s = run_job(ctx, J, pg, ctx->cap_stream);
    if (cudaStreamEndCapture(ctx->cap_stream, &g) != cudaSuccess || !g || s) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        ctx->launches = l0;
        ctx->bins_pending = pend;
        return nullptr;
    }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) { cudaGetLastError(); ex = nullptr; }
    cudaGraphDestroy(g);
    launches = ctx->launches - l0;        // kernels one replay launches
    ctx->launches = l0;                   // capture launched nothing
    ctx->bins_pending = pend;             // replays start from this state
    if (ex) {
        A.seg_graph[e] = ex;
        A.seg_launches[e] = launches;
        A.seg_used[e] = A.seg_clock;
        std::copy(key, key + NK, A.seg_key[e]);
    }
    return ex;
}

// runs one step: its graph where graphs are in use, else directly
static mpm_status run_step(mpm_ctx *ctx, const RevJob &J, int pg, cudaStream_t st) {
    long long per = 0;
    // inside the caller's capture the step's kernels go straight into its graph
    cudaGraphExec_t ex = (ctx->use_graph && !ctx->trace_on && !ctx->adj.strict) ? job_graph(ctx, J, pg, per) : nullptr;
    if (!ex) return run_job(ctx, J, pg, st);
    if (cudaGraphLaunch(ex, st) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, MPM_ERR_CUDA, "reverse-pass graph launch failed");
    }
    ctx->launches += per;
    ctx->bins_pending = false;    // every step ends with its binning consumed
    return MPM_OK;
}

}  // namespace mpm

using namespace mpm;

extern "C" MPM_API mpm_status mpm_backward(mpm_ctx *ctx, int32_t n_frames, const int32_t *frame_substep,
                                           const float *dL_dx, float *dL_dparams, float *dL_dstate0, void *stream) {
    TraceRange trace_range("mpm_backward");
    if (!ctx) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!ctx->loaded || ctx->sticky) return ctx_fail(ctx, MPM_ERR_STATE, "no valid particle state");
    if (ctx->record_broken) return ctx_fail(ctx, MPM_ERR_STATE, "the recording was interrupted by an unrecorded step");
    const long long S = ctx->recorded;
    if (S <= 0) return ctx_fail(ctx, MPM_ERR_STATE, "nothing recorded: call mpm_step with record != 0 first");
    if (n_frames < 0 || (n_frames > 0 && (!frame_substep || !dL_dx)) || !dL_dparams)
        return ctx_fail(ctx, MPM_ERR_INVALID_ARG, "bad frames / gradient arguments");
    if (any_on_other_device({dL_dx, dL_dparams, dL_dstate0}))
        return ctx_fail(ctx, MPM_ERR_INVALID_ARG, "an array lives on another device than the current one");
    for (int f = 0; f < n_frames; ++f)
        if (frame_substep[f] < 0 || frame_substep[f] > S)
            return ctx_fail(ctx, MPM_ERR_INVALID_ARG, "frame_substep outside [0, recorded substeps]");
    Dev &D = ctx->D;
    AdjointStore &A = ctx->adj;
    const size_t n = (size_t)D.n;
    const long long k = ctx->opt.ckpt_every;
    mpm_status s;
    // Inside the caller's stream capture nothing may allocate or synchronise:
    // the buffers come from an earlier call outside the capture, inputs and
    // outputs are device arrays, and a grid-tape overflow (which cannot be
    // rerun inside a graph) is reported as a device capacity error.
    const bool cap = stream_capturing(st);
    A.strict = cap;
    const char *warm = "inside a stream capture, call mpm_backward once outside it first with the same sizes "
                       "(it allocates its buffers then)";
    if (cap && (!is_device_ptr(dL_dparams) || (dL_dstate0 && !is_device_ptr(dL_dstate0)) ||
                (n_frames > 0 && !is_device_ptr(dL_dx)) || n_frames > FRAMES_BY_VALUE))
        return ctx_fail(ctx, MPM_ERR_INVALID_ARG, "inside a stream capture dL_dx and the outputs must be device "
                                                  "arrays, and there may be at most 64 frames");
    if (cap && (A.cap_adj != ctx->cap || A.pool != ctx->pool_blocks || A.frame_first_cap < S + 1 ||
                A.frame_cap < std::max(n_frames, 1) || !A.seg))
        return ctx_fail(ctx, MPM_ERR_STATE, warm);
    if (A.cap_adj != ctx->cap) {
        if ((s = dev_alloc(ctx, &A.adj[0], (size_t)ctx->cap * ADJ_F4)) || (s = dev_alloc(ctx, &A.adj[1], (size_t)ctx->cap * ADJ_F4)) ||
            (s = dev_alloc(ctx, &A.gpar, (size_t)ctx->cap)) || (s = dev_alloc(ctx, &A.final_state, (size_t)ctx->cap * REC_F4))) {
            A.cap_adj = 0;
            return s;
        }
        A.cap_adj = ctx->cap;
    }
    if (A.pool != ctx->pool_blocks) {
        if ((s = dev_alloc(ctx, &A.gbar, (size_t)ctx->pool_blocks * BLK_NODES))) { A.pool = 0; return s; }
        A.pool = ctx->pool_blocks;
        if (cudaMemsetAsync(A.gbar, 0, (size_t)A.pool * BLK_NODES * sizeof(float4), st) != cudaSuccess)
            return ctx_fail(ctx, MPM_ERR_CUDA, "memset");
    }
    const size_t tape_states = (size_t)std::min<long long>(k, S);
    if (cap) {
        // use what an earlier call left: no allocation here
        const long long shape[3] = {ctx->cap, (long long)ctx->chunk_cap, ctx->total_blocks};
        const bool gt_ok = ctx->opt.tape_grid == 0 && A.gt && A.gt_bank_states >= tape_states &&
                           std::equal(shape, shape + 3, A.gt_shape);
        const bool tape_ok = A.tape && A.tape_states >= tape_states && A.tape_cap == ctx->cap;
        if (!gt_ok && !tape_ok) return ctx_fail(ctx, MPM_ERR_STATE, warm);
    }
    bool use_gt = ctx->opt.tape_grid == 0 && (cap ? (A.gt && A.gt_bank_states >= tape_states)
                                                   : ensure_grid_tape(ctx, tape_states, st));
    if (ctx->opt.tape_grid != 0 && A.gt) {
        cudaFree(A.gt);
        A.gt = nullptr;
        A.gt_bank_states = 0;
    }
    auto ensure_record_tape = [&]() -> mpm_status {
        if (A.tape_states >= tape_states && A.tape_cap == ctx->cap) return MPM_OK;
        mpm_status r = dev_alloc(ctx, &A.tape, tape_states * (size_t)ctx->cap * REC_F4);
        if (r) { A.tape_states = 0; return r; }
        A.tape_states = tape_states;
        A.tape_cap = ctx->cap;
        return MPM_OK;
    };
    if (use_gt) {
        if (A.tape && !cap) {
            cudaFree(A.tape);   // the grid tape holds the records too
            A.tape = nullptr;
            A.tape_states = 0;
        }
    } else if ((s = ensure_record_tape())) {
        return s;
    }
    // stage dL/dx
    const size_t fbytes = (size_t)n_frames * n * 3 * sizeof(float);
    const float *dldx = dL_dx;
    if (n_frames > 0 && !is_device_ptr(dL_dx)) {
        if (A.frames_bytes < fbytes) {
            if ((s = dev_alloc(ctx, &A.frames, fbytes / sizeof(float)))) { A.frames_bytes = 0; return s; }
            A.frames_bytes = fbytes;
        }
        if (cudaMemcpyAsync(A.frames, dL_dx, fbytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return ctx_fail(ctx, MPM_ERR_CUDA, "dL_dx copy");
        dldx = A.frames;
    }
    if (cudaMemcpyAsync(A.final_state, D.rec, n * REC_F4 * sizeof(float4), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return ctx_fail(ctx, MPM_ERR_CUDA, "backward set-up copies");
    // frame table: per substep the first frame taken after it, per frame the next one there
    if (A.frame_first_cap < S + 1) {
        if ((s = dev_alloc(ctx, &A.frame_first, (size_t)S + 1))) { A.frame_first_cap = 0; return s; }
        A.frame_first_cap = S + 1;
    }
    if (A.frame_cap < std::max(n_frames, 1)) {
        if ((s = dev_alloc(ctx, &A.frame_next, (size_t)std::max(n_frames, 1)))) { A.frame_cap = 0; return s; }
        A.frame_cap = std::max(n_frames, 1);
    }
    if (!A.seg) {
        if (cudaMalloc(&A.seg, sizeof(SegParams)) != cudaSuccess) {
            cudaGetLastError();
            A.seg = nullptr;
            return ctx_fail(ctx, MPM_ERR_OOM, "reverse-pass allocation failed");
        }
    }
    if (n_frames <= FRAMES_BY_VALUE) {
        FrameList fl;
        fl.n = n_frames;
        for (int f = 0; f < n_frames; ++f) fl.sub[f] = frame_substep[f];
        k_frame_table<<<1, 256, 0, st>>>(fl, A.frame_first, A.frame_next, S);
        ++ctx->launches;
    } else {
        std::vector<int> first((size_t)S + 1, -1), next((size_t)std::max(n_frames, 1), -1);
        for (int f = n_frames - 1; f >= 0; --f) {
            next[f] = first[frame_substep[f]];
            first[frame_substep[f]] = f;
        }
        // pageable host memory: the copies complete before cudaMemcpyAsync returns
        if (cudaMemcpyAsync(A.frame_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(A.frame_next, next.data(), next.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return ctx_fail(ctx, MPM_ERR_CUDA, "frame table copy");
    }
    const int pg = grid_for((long long)n, 256);
    const long long nseg = (S + k - 1) / k;
    auto seg_len = [&](long long c) { return (int)std::min<long long>(k, S - c * k); };
    auto restore = [&](long long c) -> bool {
        return cudaMemcpyAsync(D.rec, A.ckpt[(size_t)c], n * REC_F4 * sizeof(float4), cudaMemcpyDeviceToDevice, st) ==
               cudaSuccess;
    };
    for (int attempt = 0;; ++attempt) {
    // the slot-overflow flag of this attempt (a rerun may keep the tape)
    if (use_gt && cudaMemsetAsync(gt_over(ctx), 0, sizeof(unsigned), st) != cudaSuccess)
        return ctx_fail(ctx, MPM_ERR_CUDA, "backward set-up copies");
    if (cudaMemsetAsync(A.adj[0], 0, n * ADJ_F4 * sizeof(float4), st) != cudaSuccess ||
        cudaMemsetAsync(A.gpar, 0, n * sizeof(float4), st) != cudaSuccess)
        return ctx_fail(ctx, MPM_ERR_CUDA, "backward set-up copies");
    int cur = 0;
    if (use_gt) {
        // the last segment's recompute, then per segment c its reverse
        // alongside the recompute of segment c-1 (banks alternate by parity)
        if (!restore(nseg - 1)) return ctx_fail(ctx, MPM_ERR_CUDA, "checkpoint restore");
        if (ctx->bins_pending) L_plan(ctx, 0, st);
        if ((s = run_step(ctx, RevJob{1, 0, 0, 0, seg_len(nseg - 1), (int)((nseg - 1) & 1)}, pg, st))) return s;
        for (long long c = nseg - 1; c >= 0; --c) {
            if (c > 0 && !restore(c - 1)) return ctx_fail(ctx, MPM_ERR_CUDA, "checkpoint restore");
            k_set_seg<<<1, 1, 0, st>>>((SegParams *)A.seg, dldx, c * k);
            ++ctx->launches;
            const RevJob J{1, seg_len(c), (int)(c & 1), cur, c > 0 ? seg_len(c - 1) : 0,
                           c > 0 ? (int)((c - 1) & 1) : 0};
            if ((s = run_step(ctx, J, pg, st))) return s;
            cur ^= (seg_len(c) & 1);
        }
    } else {
        for (long long c = nseg - 1; c >= 0; --c) {
            // the segment's input state, its pending binning consumed here so
            // that every segment starts from the same host-side state
            if (!restore(c)) return ctx_fail(ctx, MPM_ERR_CUDA, "checkpoint restore");
            if (ctx->bins_pending) L_plan(ctx, 0, st);
            k_set_seg<<<1, 1, 0, st>>>((SegParams *)A.seg, dldx, c * k);
            ++ctx->launches;
            if ((s = run_step(ctx, RevJob{0, seg_len(c), 0, cur, 0, 0}, pg, st))) return s;
            cur ^= (seg_len(c) & 1);
        }
    }
    // frames taken at substep 0
    k_set_seg<<<1, 1, 0, st>>>((SegParams *)A.seg, dldx, -1);
    k_inject_tab<<<pg, 256, 0, st>>>((int)n, A.adj[cur], A.frame_first, A.frame_next, (const SegParams *)A.seg, 0);
    ctx->launches += 2;
    // outputs
    float *dp = dL_dparams, *ds = dL_dstate0;
    const bool dp_dev = is_device_ptr(dL_dparams), ds_dev = !dL_dstate0 || is_device_ptr(dL_dstate0);
    if (!dp_dev || !ds_dev) {
        // host outputs go through the context's staging buffer (>= 30 floats per particle)
        float *tmp = reinterpret_cast<float *>(ctx->stage);
        if (!dp_dev) dp = tmp;
        if (!ds_dev) ds = tmp + ((n * 3 + 63) & ~size_t(63));
    }
    k_export_grads<<<pg, 256, 0, st>>>((int)n, A.gpar, A.adj[cur], dp, ds);
    ++ctx->launches;
    if (!dp_dev && cudaMemcpyAsync(dL_dparams, dp, n * 3 * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ctx_fail(ctx, MPM_ERR_CUDA, "gradient copy");
    if (dL_dstate0 && !ds_dev &&
        cudaMemcpyAsync(dL_dstate0, ds, n * 24 * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ctx_fail(ctx, MPM_ERR_CUDA, "state adjoint copy");

    // restore the recorded end state and its binning
    if (cudaMemcpyAsync(D.rec, A.final_state, n * REC_F4 * sizeof(float4), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return ctx_fail(ctx, MPM_ERR_CUDA, "state restore");
    rebin(ctx, st);
    if (cudaGetLastError() != cudaSuccess) return ctx_fail(ctx, MPM_ERR_CUDA, "reverse-pass launch failed");
    if (cap) return MPM_OK;   // errors surface at the next synchronising call (mpm_sync)
    if ((s = ctx_check(ctx, st))) return s;
    if (!use_gt) return MPM_OK;
    unsigned over = 0;
    if (cudaMemcpy(&over, gt_over(ctx), sizeof(over), cudaMemcpyDeviceToHost) != cudaSuccess)
        return ctx_fail(ctx, MPM_ERR_CUDA, "grid-tape flag read");
    if (!over) return MPM_OK;
    if (attempt > 0) return ctx_fail(ctx, MPM_ERR_CAPACITY, "grid tape overflow with the whole pool per slot");
    // a state's grid did not fit its slot: slots of the whole pool (or, if
    // those do not fit, no grid tape), and the reverse pass again
    A.gt_pool_want = ctx->pool_blocks;
    ++A.gt_reruns;
    use_gt = ensure_grid_tape(ctx, tape_states, st);
    if (!use_gt && (s = ensure_record_tape())) return s;
    }
}
