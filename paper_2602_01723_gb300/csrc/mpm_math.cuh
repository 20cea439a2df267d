// mpm_math.cuh -- per-particle device math of the MLS-MPM substep:
// quadratic B-spline weights, closed-form 3x3 SVD, Kirchhoff stresses
// (fixed-corotated, Neo-Hookean) and the von Mises / Drucker-Prager return
// maps, in the form the fused kernels need.
//
// Matrices are 3x3 row-major arrays.  The SVD convention is the rotation
// variant one: det U = det V = +1, sigma_0 >= sigma_1 >= |sigma_2|, and the
// last singular value carries the sign of det F.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace mpm {

// ---------------------------------------------------------------------------
// scalar helpers that dispatch on float / double
// ---------------------------------------------------------------------------
__device__ __forceinline__ float t_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double t_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float t_acos(float x) { return acosf(x); }
__device__ __forceinline__ double t_acos(double x) { return acos(x); }
__device__ __forceinline__ float t_cos(float x) { return cosf(x); }
__device__ __forceinline__ double t_cos(double x) { return cos(x); }
__device__ __forceinline__ float t_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double t_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float t_log(float x) { return logf(x); }
__device__ __forceinline__ double t_log(double x) { return log(x); }
__device__ __forceinline__ float t_exp(float x) { return expf(x); }
__device__ __forceinline__ double t_exp(double x) { return exp(x); }
__device__ __forceinline__ float t_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double t_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float t_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double t_abs(double x) { return fabs(x); }

// reciprocal and reciprocal square root: the MUFU approximations in FP32
// (relative error of a few ulp, enough wherever a quantity is normalised or
// only its relative precision matters), exact IEEE operations in FP64
__device__ __forceinline__ float t_rcp(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double t_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float t_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double t_rsqrt(double x) { return 1.0 / sqrt(x); }

template <typename T> struct Tol;
template <> struct Tol<float> {
    static constexpr float rank = 1e-3f;     // sigma_2/sigma_0 below this goes to the FP64 branch
    static constexpr float tiny = 1e-30f;
};
template <> struct Tol<double> {
    static constexpr double rank = 0.0;
    static constexpr double tiny = 1e-300;
};

template <typename T>
__device__ __forceinline__ void cross3(T c[3], const T a[3], const T b[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename T>
__device__ __forceinline__ T dot3(const T a[3], const T b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// ---------------------------------------------------------------------------
// quadratic B-spline, fx = x/dx - base in [0.5, 1.5)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bspline_w(float fx, float w[3]) {
    float a = 1.5f - fx, b = fx - 1.0f, c = fx - 0.5f;
    w[0] = 0.5f * a * a;
    w[1] = 0.75f - b * b;
    w[2] = 0.5f * c * c;
}
__device__ __forceinline__ void bspline_dw(float fx, float dw[3]) {   // d w / d fx
    dw[0] = fx - 1.5f;
    dw[1] = -2.0f * (fx - 1.0f);
    dw[2] = fx - 0.5f;
}

// ---------------------------------------------------------------------------
// Closed-form SVD of a 3x3 matrix.
//
// Eigen-decomposition of D = F^T F - I, formed from H = F - I as
// H + H^T + H^T H so that small strains keep their relative precision:
//  * the deviatoric part scaled to the depressed characteristic cubic
//    y^3 - 3y = 2r (Smith 1961), whose most isolated root is found by Newton
//    iteration from an analytic start;
//  * its eigenvector as the largest cross product of two rows of the shifted
//    matrix (Kopp 2008);
//  * the remaining pair by one exact 2x2 Jacobi rotation in the orthogonal
//    complement, which stays well defined when the pair is degenerate.
// U follows from F V by Gram-Schmidt; U = [u0 u1 u0 x u1] gives det U = +1,
// and the last singular value is u2 . F v2 (signed).
//
// Outputs: U, V, s (signed singular values), e = s - 1 (computed as
// d/(1 + s) for positive s), and d = s^2 - 1 (the eigenvalues of D).
// Returns false when F is rank deficient or not finite: the FP32 caller then
// repeats the decomposition in FP64.
// ---------------------------------------------------------------------------
template <typename T>
__device__ bool svd3(const T F[9], T U[9], T V[9], T s[3], T e[3], T d[3]) {
    T h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = F[i];
    h[0] -= T(1); h[4] -= T(1); h[8] -= T(1);
    // D = H + H^T + H^T H  (symmetric)
    T D[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            T v = h[3 * i + j] + h[3 * j + i] + h[i] * h[j] + h[3 + i] * h[3 + j] + h[6 + i] * h[6 + j];
            D[3 * i + j] = v;
            D[3 * j + i] = v;
        }
    T q = (D[0] + D[4] + D[8]) * T(1.0 / 3.0);
    T b00 = D[0] - q, b11 = D[4] - q, b22 = D[8] - q, b01 = D[1], b02 = D[2], b12 = D[5];
    T p2 = (b00 * b00 + b11 * b11 + b22 * b22 + T(2) * (b01 * b01 + b02 * b02 + b12 * b12)) * T(1.0 / 6.0);
    T y[3];
    T vv[3][3];   // eigenvectors (as rows here; transposed into V below)
    if (!(p2 > T(0))) {
        if (!(p2 == T(0))) return false;     // NaN
        y[0] = y[1] = y[2] = T(0);
        vv[0][0] = T(1); vv[0][1] = T(0); vv[0][2] = T(0);
        vv[1][0] = T(0); vv[1][1] = T(1); vv[1][2] = T(0);
        vv[2][0] = T(0); vv[2][1] = T(0); vv[2][2] = T(1);
        p2 = T(0);
    } else {
        T p = t_sqrt(p2), ip = t_rcp(p);
        T c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = b01 * ip, c02 = b02 * ip, c12 = b12 * ip;
        T r = T(0.5) * (c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02));
        r = r > T(1) ? T(1) : (r < T(-1) ? T(-1) : r);
        // The roots of y^3 - 3y - 2r = 0 lie in [-2, 2].  For r >= 0 the
        // largest one (in [sqrt3, 2]) is the most isolated, for r < 0 the
        // smallest.  Newton from +-2, whose first step is taken analytically;
        // f' = 3y^2 - 3 >= 6 on that interval, and the error squares each step
        // (4e-2, 2e-3, 3e-6, 1e-11 for the worst case r = 0).
        const T sg = r >= T(0) ? T(1) : T(-1);
        T yi = sg * (T(2) - (T(2) - T(2) * sg * r) * T(1.0 / 9.0));
#pragma unroll
        for (int it = 0; it < 3; ++it) {
            const T y2 = yi * yi;
            yi -= (y2 * yi - T(3) * yi - T(2) * r) * t_rcp(T(3) * y2 - T(3));
        }
        // eigenvector of the isolated root: null vector of C - yi I
        T m0[3] = {c00 - yi, c01, c02}, m1[3] = {c01, c11 - yi, c12}, m2[3] = {c02, c12, c22 - yi};
        T x01[3], x02[3], x12[3];
        cross3(x01, m0, m1);
        cross3(x02, m0, m2);
        cross3(x12, m1, m2);
        T n01 = dot3(x01, x01), n02 = dot3(x02, x02), n12 = dot3(x12, x12);
        T vi[3];
        T nbest = n01;
        vi[0] = x01[0]; vi[1] = x01[1]; vi[2] = x01[2];
        if (n02 > nbest) { nbest = n02; vi[0] = x02[0]; vi[1] = x02[1]; vi[2] = x02[2]; }
        if (n12 > nbest) { nbest = n12; vi[0] = x12[0]; vi[1] = x12[1]; vi[2] = x12[2]; }
        if (!(nbest > Tol<T>::tiny)) return false;
        T inv = t_rsqrt(nbest);
        vi[0] *= inv; vi[1] *= inv; vi[2] *= inv;
        // orthonormal basis (e1, e2) of the complement
        T ax[3] = {T(0), T(0), T(0)};
        T a0 = t_abs(vi[0]), a1 = t_abs(vi[1]), a2 = t_abs(vi[2]);
        if (a0 <= a1 && a0 <= a2) ax[0] = T(1);
        else if (a1 <= a2) ax[1] = T(1);
        else ax[2] = T(1);
        T e1[3], e2[3];
        cross3(e1, vi, ax);
        T ne = t_rsqrt(dot3(e1, e1));
        e1[0] *= ne; e1[1] *= ne; e1[2] *= ne;
        cross3(e2, vi, e1);
        // 2x2 block of C in that basis
        T Ce1[3] = {c00 * e1[0] + c01 * e1[1] + c02 * e1[2], c01 * e1[0] + c11 * e1[1] + c12 * e1[2],
                    c02 * e1[0] + c12 * e1[1] + c22 * e1[2]};
        T Ce2[3] = {c00 * e2[0] + c01 * e2[1] + c02 * e2[2], c01 * e2[0] + c11 * e2[1] + c12 * e2[2],
                    c02 * e2[0] + c12 * e2[1] + c22 * e2[2]};
        T aa = dot3(e1, Ce1), bb = dot3(e1, Ce2), cc = dot3(e2, Ce2);
        T cs = T(1), sn = T(0), tj = T(0);
        if (bb != T(0)) {
            T th = (cc - aa) * t_rcp(T(2) * bb);
            tj = (th >= T(0) ? T(1) : T(-1)) * t_rcp(t_abs(th) + t_sqrt(th * th + T(1)));
            cs = t_rsqrt(tj * tj + T(1));
            sn = tj * cs;
        }
        T ya = aa - tj * bb, yb = cc + tj * bb;
        T wa[3], wb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) { wa[k] = cs * e1[k] - sn * e2[k]; wb[k] = sn * e1[k] + cs * e2[k]; }
        // gather the three eigenpairs and sort by eigenvalue, descending
        y[0] = yi; y[1] = ya; y[2] = yb;
#pragma unroll
        for (int k = 0; k < 3; ++k) { vv[0][k] = vi[k]; vv[1][k] = wa[k]; vv[2][k] = wb[k]; }
#define MPM_SWAP_PAIR(i, j)                                                   \
        if (y[i] < y[j]) {                                                    \
            T t_ = y[i]; y[i] = y[j]; y[j] = t_;                              \
            for (int k = 0; k < 3; ++k) { T u_ = vv[i][k]; vv[i][k] = vv[j][k]; vv[j][k] = u_; } \
        }
        MPM_SWAP_PAIR(0, 1)
        MPM_SWAP_PAIR(1, 2)
        MPM_SWAP_PAIR(0, 1)
#undef MPM_SWAP_PAIR
        p2 = p;   // reuse as the scale
    }
    // eigenvalues of D and the right singular vectors (det V = +1)
    T pscale = p2;   // p, or 0 for the isotropic case
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = q + pscale * y[k];
    cross3(vv[2], vv[0], vv[1]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) V[3 * r + c] = vv[c][r];
    // U from F V
    T f0[3], f1[3], f2[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        f0[r] = F[3 * r] * vv[0][0] + F[3 * r + 1] * vv[0][1] + F[3 * r + 2] * vv[0][2];
        f1[r] = F[3 * r] * vv[1][0] + F[3 * r + 1] * vv[1][1] + F[3 * r + 2] * vv[1][2];
        f2[r] = F[3 * r] * vv[2][0] + F[3 * r + 1] * vv[2][1] + F[3 * r + 2] * vv[2][2];
    }
    T n0 = dot3(f0, f0);
    if (!(n0 > Tol<T>::tiny)) return false;
    T in0 = t_rsqrt(n0);
    T u0[3] = {f0[0] * in0, f0[1] * in0, f0[2] * in0};
    T pr = dot3(u0, f1);
    T g1[3] = {f1[0] - pr * u0[0], f1[1] - pr * u0[1], f1[2] - pr * u0[2]};
    T n1 = dot3(g1, g1);
    T u1[3];
    if (!(n1 > Tol<T>::rank * Tol<T>::rank * n0) || !(n1 > Tol<T>::tiny)) {
        if (Tol<T>::rank > T(0) || !(n1 == n1)) return false;
        // FP64 branch, rank <= 1: any unit vector orthogonal to u0
        T ax[3] = {T(0), T(0), T(0)};
        T a0 = t_abs(u0[0]), a1 = t_abs(u0[1]), a2 = t_abs(u0[2]);
        if (a0 <= a1 && a0 <= a2) ax[0] = T(1);
        else if (a1 <= a2) ax[1] = T(1);
        else ax[2] = T(1);
        cross3(u1, u0, ax);
        T nn = t_rsqrt(dot3(u1, u1));
        u1[0] *= nn; u1[1] *= nn; u1[2] *= nn;
    } else {
        T in1 = t_rsqrt(n1);
        u1[0] = g1[0] * in1; u1[1] = g1[1] * in1; u1[2] = g1[2] * in1;
    }
    T u2[3];
    cross3(u2, u0, u1);
#pragma unroll
    for (int r = 0; r < 3; ++r) { U[3 * r] = u0[r]; U[3 * r + 1] = u1[r]; U[3 * r + 2] = u2[r]; }
    T s2sign = dot3(u2, f2);
    // singular values from the eigenvalues of D; s - 1 = d / (1 + s)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        T sq = T(1) + d[k];
        if (!(sq > T(0))) return false;
        s[k] = t_sqrt(sq);
        e[k] = d[k] * t_rcp(T(1) + s[k]);
    }
    {
        T sq = T(1) + d[2];
        sq = sq > T(0) ? sq : T(0);
        T m = t_sqrt(sq);
        if (Tol<T>::rank > T(0) && !(m > Tol<T>::rank * s[0])) return false;
        if (s2sign >= T(0)) { s[2] = m; e[2] = d[2] * t_rcp(T(1) + m); }
        else { s[2] = -m; e[2] = -m - T(1); }
    }
    return true;
}

// FP32 SVD with the FP64 branch for rank-deficient or non-finite input.
// Returns 0 on the FP32 path, 1 when the FP64 branch ran, 2 when both failed.
// The FP64 branch out of line, for kernels whose instruction footprint
// matters more than a call on the rare slow path.  Arguments and results
// pass by value, so that the caller's arrays stay in registers on the fast
// path; status 1 FP64 ok, 2 FP64 failed.
struct Svd3Out {
    float U[9], V[9], s[3], e[3], d[3];
    int status;
};
struct Mat3f {
    float a[9];
};
static __device__ __noinline__ Svd3Out svd3_fp64_out(Mat3f F) {
    double Fd[9], Ud[9], Vd[9], sd[3], ed[3], dd[3];
#pragma unroll
    for (int i = 0; i < 9; ++i) Fd[i] = (double)F.a[i];
    const bool ok = svd3<double>(Fd, Ud, Vd, sd, ed, dd);
    Svd3Out o;
#pragma unroll
    for (int i = 0; i < 9; ++i) { o.U[i] = (float)Ud[i]; o.V[i] = (float)Vd[i]; }
#pragma unroll
    for (int i = 0; i < 3; ++i) { o.s[i] = (float)sd[i]; o.e[i] = (float)ed[i]; o.d[i] = (float)dd[i]; }
    o.status = ok ? 1 : 2;
    return o;
}
__device__ __forceinline__ int svd3_robust_cold(const float F[9], float U[9], float V[9], float s[3], float e[3],
                                                float d[3]) {
    if (svd3<float>(F, U, V, s, e, d)) return 0;
    Mat3f Fm;
#pragma unroll
    for (int i = 0; i < 9; ++i) Fm.a[i] = F[i];
    const Svd3Out o = svd3_fp64_out(Fm);
#pragma unroll
    for (int i = 0; i < 9; ++i) { U[i] = o.U[i]; V[i] = o.V[i]; }
#pragma unroll
    for (int i = 0; i < 3; ++i) { s[i] = o.s[i]; e[i] = o.e[i]; d[i] = o.d[i]; }
    return o.status;
}

__device__ __forceinline__ int svd3_robust(const float F[9], float U[9], float V[9], float s[3], float e[3],
                                           float d[3]) {
    if (svd3<float>(F, U, V, s, e, d)) return 0;
    double Fd[9], Ud[9], Vd[9], sd[3], ed[3], dd[3];
#pragma unroll
    for (int i = 0; i < 9; ++i) Fd[i] = (double)F[i];
    bool ok = svd3<double>(Fd, Ud, Vd, sd, ed, dd);
#pragma unroll
    for (int i = 0; i < 9; ++i) { U[i] = (float)Ud[i]; V[i] = (float)Vd[i]; }
#pragma unroll
    for (int i = 0; i < 3; ++i) { s[i] = (float)sd[i]; e[i] = (float)ed[i]; d[i] = (float)dd[i]; }
    return ok ? 1 : 2;
}

// ---------------------------------------------------------------------------
// Kirchhoff stress tau = P F^T (symmetric; stored as xx yy zz xy xz yz)
// fixed-corotated: tau = 2 mu (F - R) F^T + lambda J (J - 1) I
//                      = U diag(2 mu (s_i - 1) s_i) U^T + lambda J (J - 1) I
// Neo-Hookean:     tau = mu (F F^T - I) + lambda log J I,
//                  F F^T - I = H + H^T + H H^T with H = F - I.
// ---------------------------------------------------------------------------
struct Sym { float xx, yy, zz, xy, xz, yz; };

__device__ __forceinline__ Sym tau_fcr(const float U[9], const float s[3], const float e[3], float mu, float lam) {
    float k0 = 2.f * mu * e[0] * s[0], k1 = 2.f * mu * e[1] * s[1], k2 = 2.f * mu * e[2] * s[2];
    // J - 1 = prod(1 + e) - 1 without cancellation
    float jm1 = e[0] + e[1] + e[2] + e[0] * e[1] + e[0] * e[2] + e[1] * e[2] + e[0] * e[1] * e[2];
    float vol = lam * (1.f + jm1) * jm1;
    Sym t;
    t.xx = k0 * U[0] * U[0] + k1 * U[1] * U[1] + k2 * U[2] * U[2] + vol;
    t.yy = k0 * U[3] * U[3] + k1 * U[4] * U[4] + k2 * U[5] * U[5] + vol;
    t.zz = k0 * U[6] * U[6] + k1 * U[7] * U[7] + k2 * U[8] * U[8] + vol;
    t.xy = k0 * U[0] * U[3] + k1 * U[1] * U[4] + k2 * U[2] * U[5];
    t.xz = k0 * U[0] * U[6] + k1 * U[1] * U[7] + k2 * U[2] * U[8];
    t.yz = k0 * U[3] * U[6] + k1 * U[4] * U[7] + k2 * U[5] * U[8];
    return t;
}

// J - 1 = det(I + H) - 1 = tr H + (sum of principal 2x2 minors of H) + det H
__device__ __forceinline__ float det_minus_one(const float F[9]) {
    float h0 = F[0] - 1.f, h4 = F[4] - 1.f, h8 = F[8] - 1.f;
    float m2 = h0 * h4 - F[1] * F[3] + h0 * h8 - F[2] * F[6] + h4 * h8 - F[5] * F[7];
    float dh = h0 * (h4 * h8 - F[5] * F[7]) - F[1] * (F[3] * h8 - F[5] * F[6]) + F[2] * (F[3] * F[7] - h4 * F[6]);
    return (h0 + h4 + h8) + m2 + dh;
}

// returns false when J <= 0 (log J undefined)
__device__ __forceinline__ bool tau_nh(const float F[9], float mu, float lam, Sym &t) {
    float jm1 = det_minus_one(F);
    if (!(jm1 > -1.f)) return false;
    float vol = lam * log1pf(jm1);
    float h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = F[i];
    h[0] -= 1.f; h[4] -= 1.f; h[8] -= 1.f;
    // (H + H^T + H H^T)_ij = h_ij + h_ji + sum_k h_ik h_jk
    t.xx = mu * (2.f * h[0] + h[0] * h[0] + h[1] * h[1] + h[2] * h[2]) + vol;
    t.yy = mu * (2.f * h[4] + h[3] * h[3] + h[4] * h[4] + h[5] * h[5]) + vol;
    t.zz = mu * (2.f * h[8] + h[6] * h[6] + h[7] * h[7] + h[8] * h[8]) + vol;
    t.xy = mu * (h[1] + h[3] + h[0] * h[3] + h[1] * h[4] + h[2] * h[5]);
    t.xz = mu * (h[2] + h[6] + h[0] * h[6] + h[1] * h[7] + h[2] * h[8]);
    t.yz = mu * (h[5] + h[7] + h[3] * h[6] + h[4] * h[7] + h[5] * h[8]);
    return true;
}

// ---------------------------------------------------------------------------
// Further elastic models of App. B.1 (kept out of line: the substep kernel's
// register allocation stays that of the fixed-corotated / Neo-Hookean path)
//   2 StVK, Green strain E = (F^T F - I)/2:
//       tau = 2 mu F E F^T + lambda J (J - 1) I
//   3 Hencky (SigmaElasticity; also App. A's StVK, whose P F^T is this):
//       tau = U diag(2 mu eps + lambda tr eps) U^T, eps = log max(s, 1e-4)
//   4 fluid:  tau = lambda J (J - 1) I
//   5 volume: tau = kappa (J - 1/J) I, kappa = 2 mu / 3 + lambda (gamma = 2)
// Returns false when the state is outside the model's domain (J <= 0 for 5).
// ---------------------------------------------------------------------------
enum { ELASTIC_FCR = 0, ELASTIC_NH = 1, ELASTIC_STVK = 2, ELASTIC_HENCKY = 3, ELASTIC_FLUID = 4,
       ELASTIC_VOLUME = 5 };
#define MPM_SIGMA_FLOOR 1e-4f

__device__ __forceinline__ bool elastic_needs_svd(int elastic) {
    return elastic == ELASTIC_FCR || elastic == ELASTIC_HENCKY;
}

static __device__ __noinline__ bool tau_more(int elastic, const float *F, const float *U, const float *s, const float *e,
                                      float mu, float lam, Sym *out) {
    Sym t{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float jm1 = det_minus_one(F);
    bool ok = true;
    if (elastic == ELASTIC_STVK) {
        float h[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = F[i];
        h[0] -= 1.f; h[4] -= 1.f; h[8] -= 1.f;
        float E[9];   // (H + H^T + H^T H) / 2
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                E[3 * i + j] = 0.5f * (h[3 * i + j] + h[3 * j + i] + h[i] * h[j] + h[3 + i] * h[3 + j] +
                                       h[6 + i] * h[6 + j]);
        float A[9];   // F E
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                A[3 * i + j] = F[3 * i] * E[j] + F[3 * i + 1] * E[3 + j] + F[3 * i + 2] * E[6 + j];
        const float k = 2.f * mu, vol = lam * (1.f + jm1) * jm1;
        t.xx = k * (A[0] * F[0] + A[1] * F[1] + A[2] * F[2]) + vol;
        t.yy = k * (A[3] * F[3] + A[4] * F[4] + A[5] * F[5]) + vol;
        t.zz = k * (A[6] * F[6] + A[7] * F[7] + A[8] * F[8]) + vol;
        t.xy = k * (A[0] * F[3] + A[1] * F[4] + A[2] * F[5]);
        t.xz = k * (A[0] * F[6] + A[1] * F[7] + A[2] * F[8]);
        t.yz = k * (A[3] * F[6] + A[4] * F[7] + A[5] * F[8]);
    } else if (elastic == ELASTIC_HENCKY) {
        float eps[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) eps[i] = s[i] > MPM_SIGMA_FLOOR ? log1pf(e[i]) : -9.210340371976184f;
        const float tr = lam * (eps[0] + eps[1] + eps[2]);
        const float d0 = 2.f * mu * eps[0] + tr, d1 = 2.f * mu * eps[1] + tr, d2 = 2.f * mu * eps[2] + tr;
        t.xx = d0 * U[0] * U[0] + d1 * U[1] * U[1] + d2 * U[2] * U[2];
        t.yy = d0 * U[3] * U[3] + d1 * U[4] * U[4] + d2 * U[5] * U[5];
        t.zz = d0 * U[6] * U[6] + d1 * U[7] * U[7] + d2 * U[8] * U[8];
        t.xy = d0 * U[0] * U[3] + d1 * U[1] * U[4] + d2 * U[2] * U[5];
        t.xz = d0 * U[0] * U[6] + d1 * U[1] * U[7] + d2 * U[2] * U[8];
        t.yz = d0 * U[3] * U[6] + d1 * U[4] * U[7] + d2 * U[5] * U[8];
    } else if (elastic == ELASTIC_FLUID) {
        t.xx = t.yy = t.zz = lam * (1.f + jm1) * jm1;
    } else if (elastic == ELASTIC_VOLUME) {
        if (jm1 > -1.f) {
            // J - 1/J = (J - 1)(J + 1) / J
            t.xx = t.yy = t.zz = (2.f * mu / 3.f + lam) * jm1 * (2.f + jm1) / (1.f + jm1);
        } else {
            ok = false;
        }
    } else {
        ok = false;
    }
    *out = t;
    return ok;
}

// Kirchhoff stress of any elastic model; U, s, e must hold the SVD of F when
// elastic_needs_svd(elastic)
__device__ __forceinline__ bool kirchhoff(int elastic, const float F[9], const float U[9], const float s[3],
                                          const float e[3], float mu, float lam, Sym &t) {
    if (elastic == ELASTIC_FCR) { t = tau_fcr(U, s, e, mu, lam); return true; }
    if (elastic == ELASTIC_NH) return tau_nh(F, mu, lam, t);
    return tau_more(elastic, F, U, s, e, mu, lam, &t);
}

// Volume-only plasticity: 3 fluid (App. A): F <- J^{1/3} I; 4 Sigma
// (App. B.2): J clamped to [0.05, 1.2], F <- J^{1/3} I.  Writes c I into G
// and returns c - 1 (cbrt keeps the sign of an inverted J under 3).
static __device__ __noinline__ float volume_plastic(int plastic, float *G) {
    float jm1 = det_minus_one(G);
    if (plastic == 4) jm1 = fminf(fmaxf(jm1, 0.05f - 1.f), 1.2f - 1.f);
    const float cm1 = jm1 > -1.f ? expm1f(log1pf(jm1) * (1.f / 3.f)) : cbrtf(1.f + jm1) - 1.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) G[i] = 0.f;
    G[0] = G[4] = G[8] = 1.f + cm1;
    return cm1;
}

// ---------------------------------------------------------------------------
// Return maps on the singular values (von Mises, Drucker-Prager with zero
// cohesion).  eps = log(max(s, 1e-4)); eps_hat its deviatoric part.
//   VM: dgamma = |eps_hat| - yield/(2 mu)
//   DP: tr(eps) > 0 -> cone tip (all s = 1);
//       dgamma = |eps_hat| + (3 lam + 2 mu)/(2 mu) tr(eps) alpha
//   dgamma > 0: eps <- eps - dgamma eps_hat / |eps_hat|
// On return z = new singular values and ze = z - 1.  Returns 0 elastic,
// 1 projected, 2 cone tip.
// ---------------------------------------------------------------------------
enum { PLASTIC_NONE = 0, PLASTIC_VM = 1, PLASTIC_DP = 2, PLASTIC_FLUID = 3, PLASTIC_SIGMA = 4 };
enum { RM_ELASTIC = 0, RM_PROJECT = 1, RM_TIP = 2 };

__device__ __forceinline__ float log_sigma(float s, float d) {
    // log(s) = 0.5 log1p(s^2 - 1) keeps precision near s = 1
    return s > MPM_SIGMA_FLOOR ? 0.5f * log1pf(d) : -9.210340371976184f;   // log(1e-4)
}

__device__ __forceinline__ int return_map(int plastic, const float s[3], const float e[3], const float d[3], float mu,
                                          float lam, float yield, float alpha, float z[3], float ze[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) { z[i] = s[i]; ze[i] = e[i]; }
    if (plastic == PLASTIC_NONE) return RM_ELASTIC;
    float eps[3] = {log_sigma(s[0], d[0]), log_sigma(s[1], d[1]), log_sigma(s[2], d[2])};
    float tr = eps[0] + eps[1] + eps[2];
    float m = tr * (1.f / 3.f);
    float h0 = eps[0] - m, h1 = eps[1] - m, h2 = eps[2] - m;
    float nrm = sqrtf(h0 * h0 + h1 * h1 + h2 * h2);
    float dg;
    if (plastic == PLASTIC_VM) {
        dg = nrm - yield / (2.f * mu);
        if (!(dg > 0.f)) return RM_ELASTIC;
    } else {
        if (tr > 0.f) {
            z[0] = z[1] = z[2] = 1.f;
            ze[0] = ze[1] = ze[2] = 0.f;
            return RM_TIP;
        }
        dg = nrm + (3.f * lam + 2.f * mu) / (2.f * mu) * tr * alpha;
        if (!(dg > 0.f)) return RM_ELASTIC;
    }
    float c = dg / nrm;
    float n0 = eps[0] - c * h0, n1 = eps[1] - c * h1, n2 = eps[2] - c * h2;
    ze[0] = expm1f(n0); ze[1] = expm1f(n1); ze[2] = expm1f(n2);
    z[0] = 1.f + ze[0]; z[1] = 1.f + ze[1]; z[2] = 1.f + ze[2];
    return RM_PROJECT;
}

// M = U diag(z) V^T
__device__ __forceinline__ void usvt(float M[9], const float U[9], const float z[3], const float V[9]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            M[3 * r + c] = U[3 * r] * z[0] * V[3 * c] + U[3 * r + 1] * z[1] * V[3 * c + 1] +
                           U[3 * r + 2] * z[2] * V[3 * c + 2];
}

}  // namespace mpm
