/*
 * mpm_oracle.c -- plain, slow FP64 CPU oracle of the MLS-MPM substep and of its
 * reverse-mode adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load this file or
 * the library built from it: it is used by tests/, by the smoke check and by the
 * timed CPU baseline of bench.py.  It shares no code, header or table with the
 * CUDA library; both only consume the same seeded inputs.
 *
 * What it follows (FastPhysGS, arXiv 2602.01723):
 *   - substep order: stress from F, P2G, grid update, G2P, plasticity
 *     (Algorithm 1, Stage 1; §3.2 "Material Point Method");
 *   - P2G with the MLS stress term inside the affine momentum
 *     (§4.2, momentum-exchange equation; App. A "Particle to Grid Transfer");
 *   - grid update v = mv/m + dt*g, then walls (App. A "Grid Update");
 *   - G2P: v_p, C_p = 4/dx^2 sum w v (x_i - x_p)^T, x += dt v (App. A
 *     "Grid to Particle Transfer"); F <- (I + dt C) F (MLS-MPM form);
 *   - fixed-corotated Kirchhoff stress (App. B.1, CorotatedElasticity) and
 *     Neo-Hookean (App. A, eq. neo_hookean, times F^T);
 *   - Lame parameters from (E, nu) (App. B.1);
 *   - von Mises and Drucker-Prager return maps on log singular values
 *     (App. A, eq. von_mises and eq. drucker_prager; App. B.2);
 *   - the further models of App. B.1 (StVK with Green strain, Hencky /
 *     SigmaElasticity, FluidElasticity, VolumeElasticity) and the
 *     volume-only plasticity of App. A (fluid) and App. B.2 (Sigma);
 *   - BGDO stage 2: key-frame pseudo step, stress-norm gradient in log E,
 *     log compression and Frobenius deformation guidance (§4.3, Algorithm 1,
 *     App. F);
 *   - the Gaussian kernel's covariance after deformation, F Sigma F^T
 *     (§3.2, with Sigma = R S S^T R^T of §3.1);
 *   - MCIS fill sampling (§4.1) and the splatting of the Gaussians into an
 *     image (§3.1).
 * Where the paper is silent this code reads it as follows: the interpolation
 * kernel is the quadratic B-spline; walls are a 3-node band per face (sticky
 * floor, slip elsewhere); the SVD has det U = det V = +1 with the sign of
 * det F on the smallest singular value; the Drucker-Prager delta-gamma is
 * that of Klar et al. 2016; singular values are floored at 1e-4 before log.
 *
 * Matrices are 3x3 row-major doubles.  Grids are dense, node (I,J,K) at
 * ((I*res1)+J)*res2+K, positions I*dx.
 *
 * The SVD here is cyclic Jacobi on F^T F; the CUDA path uses a different,
 * closed-form method.  Results are compared only on invariant quantities.
 *
 * Parity unpinned: the free-running trajectory over many substeps (orc_run).
 * The paper prints no trajectory to check it against.  Its pins are those
 * of each step (conservation of mass and momentum, free fall, a rigid
 * rotation carried exactly, the stress and return-map identities) and the
 * central differences of its own adjoint.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Configuration and per-particle material description                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    int res[3];          /* grid nodes per axis */
    double dx, dt;
    double gravity[3];
    int bound;           /* wall band thickness in nodes */
    int wall[6];         /* faces x-, x+, y-, y+, z-, z+ : 0 open, 1 slip, 2 sticky */
} orc_cfg;

typedef struct {
    const double *mass;      /* m_p = rho V_p */
    const double *vol;       /* V_p */
    const double *logE;      /* log Young's modulus */
    const double *nu;        /* Poisson ratio */
    const double *yield;     /* von Mises yield stress sigma_y */
    const double *phi_deg;   /* Drucker-Prager friction angle, degrees */
    const int *elastic;      /* 0 fixed-corotated, 1 Neo-Hookean, 2 StVK, 3 Hencky, 4 fluid, 5 volume */
    const int *plastic;      /* 0 identity, 1 von Mises, 2 Drucker-Prager, 3 fluid, 4 Sigma */
} orc_material;

enum { ORC_OK = 0, ORC_OUT_OF_DOMAIN = 1, ORC_NONFINITE = 2 };

#define SIGMA_FLOOR 1e-4     /* floor on singular values before the log */

/* ------------------------------------------------------------------------ */
/* Small dense 3x3 helpers                                                   */
/* ------------------------------------------------------------------------ */

static void m_zero(double A[9]) { memset(A, 0, 9 * sizeof(double)); }
static void m_eye(double A[9]) { m_zero(A); A[0] = A[4] = A[8] = 1.0; }
static void m_copy(double D[9], const double A[9]) { memcpy(D, A, 9 * sizeof(double)); }

static void m_mul(double D[9], const double A[9], const double B[9]) {      /* D = A B */
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    m_copy(D, T);
}
static void m_mul_tn(double D[9], const double A[9], const double B[9]) {   /* D = A^T B */
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * k + i] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    m_copy(D, T);
}
static void m_mul_nt(double D[9], const double A[9], const double B[9]) {   /* D = A B^T */
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * j + k];
            T[3 * i + j] = s;
        }
    m_copy(D, T);
}
static void m_transpose(double D[9], const double A[9]) {
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[3 * i + j] = A[3 * j + i];
    m_copy(D, T);
}
static double m_det(const double A[9]) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6])
         + A[2] * (A[3] * A[7] - A[4] * A[6]);
}
/* cofactor matrix: cof(A) = det(A) A^{-T} */
static void m_cofactor(double D[9], const double A[9]) {
    D[0] = A[4] * A[8] - A[5] * A[7];
    D[1] = A[5] * A[6] - A[3] * A[8];
    D[2] = A[3] * A[7] - A[4] * A[6];
    D[3] = A[2] * A[7] - A[1] * A[8];
    D[4] = A[0] * A[8] - A[2] * A[6];
    D[5] = A[1] * A[6] - A[0] * A[7];
    D[6] = A[1] * A[5] - A[2] * A[4];
    D[7] = A[2] * A[3] - A[0] * A[5];
    D[8] = A[0] * A[4] - A[1] * A[3];
}
static double m_dot(const double A[9], const double B[9]) {
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += A[i] * B[i];
    return s;
}
static double m_trace(const double A[9]) { return A[0] + A[4] + A[8]; }

static void v_cross(double c[3], const double a[3], const double b[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double v_dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------------ */
/* Quadratic B-spline weights (the interpolation kernel N(x_i - x_p) of the  */
/* §4.2 momentum equation; the paper names no kernel, the quadratic B-spline  */
/* is the reading taken).  fx = x/dx - base, base = floor(x/dx - 0.5).        */
/* ------------------------------------------------------------------------ */

void orc_bspline(double fx, double w[3], double dw[3]) {
    w[0] = 0.5 * (1.5 - fx) * (1.5 - fx);
    w[1] = 0.75 - (fx - 1.0) * (fx - 1.0);
    w[2] = 0.5 * (fx - 0.5) * (fx - 0.5);
    dw[0] = fx - 1.5;             /* d w / d fx */
    dw[1] = -2.0 * (fx - 1.0);
    dw[2] = fx - 0.5;
}

/* base cell and fractional offset of a particle; returns 0 when the 3x3x3
 * stencil lies inside the grid, nonzero otherwise. */
static int locate(const orc_cfg *cfg, const double x[3], int base[3], double fx[3]) {
    for (int d = 0; d < 3; ++d) {
        double X = x[d] / cfg->dx;
        if (!(X == X)) return ORC_NONFINITE;
        double b = floor(X - 0.5);
        if (b < 0.0 || b > (double)(cfg->res[d] - 3)) return ORC_OUT_OF_DOMAIN;
        base[d] = (int)b;
        fx[d] = X - b;
    }
    return ORC_OK;
}

static long node_index(const orc_cfg *cfg, int I, int J, int K) {
    return ((long)I * cfg->res[1] + J) * cfg->res[2] + K;
}

/* ------------------------------------------------------------------------ */
/* Lame parameters from (E, nu), App. B.1                                    */
/* ------------------------------------------------------------------------ */

void orc_lame(double E, double nu, double *mu, double *lam) {
    *mu = E / (2.0 * (1.0 + nu));
    *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

/* d(mu, lambda) / d(log E, nu) */
static void lame_grad(double logE, double nu, double d[4] /* dmu/dlogE, dmu/dnu, dlam/dlogE, dlam/dnu */) {
    double E = exp(logE), mu, lam;
    orc_lame(E, nu, &mu, &lam);
    double q = (1.0 + nu) * (1.0 - 2.0 * nu);
    d[0] = mu;
    d[1] = -E / (2.0 * (1.0 + nu) * (1.0 + nu));
    d[2] = lam;
    d[3] = E * (1.0 + 2.0 * nu * nu) / (q * q);
}

/* ------------------------------------------------------------------------ */
/* 3x3 SVD by cyclic Jacobi on F^T F.                                        */
/* Convention (reading of the paper, which states none): det U = det V = +1,  */
/* singular values sorted s0 >= s1 >= |s2|, the last one carries sign(det F). */
/* ------------------------------------------------------------------------ */

static void sym_eig_jacobi(const double Ain[9], double V[9], double lam[3]) {
    double A[9];
    m_copy(A, Ain);
    m_eye(V);
    static const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off == 0.0 || off <= 1e-40 * dia) break;
        for (int r = 0; r < 3; ++r) {
            int p = P[r], q = Q[r];
            double apq = A[3 * p + q];
            if (apq == 0.0) continue;
            double app = A[3 * p + p], aqq = A[3 * q + q];
            double theta = (aqq - app) / (2.0 * apq);
            double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            /* A <- J^T A J with J the rotation in the (p,q) plane */
            for (int k = 0; k < 3; ++k) {       /* columns p, q */
                double akp = A[3 * k + p], akq = A[3 * k + q];
                A[3 * k + p] = c * akp - s * akq;
                A[3 * k + q] = s * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {       /* rows p, q */
                double apk = A[3 * p + k], aqk = A[3 * q + k];
                A[3 * p + k] = c * apk - s * aqk;
                A[3 * q + k] = s * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {       /* V <- V J */
                double vkp = V[3 * k + p], vkq = V[3 * k + q];
                V[3 * k + p] = c * vkp - s * vkq;
                V[3 * k + q] = s * vkp + c * vkq;
            }
        }
    }
    lam[0] = A[0]; lam[1] = A[4]; lam[2] = A[8];
}

static void any_orthogonal_unit(const double a[3], double out[3]) {
    /* unit vector orthogonal to unit vector a */
    double e[3] = {0, 0, 0};
    int k = (fabs(a[0]) <= fabs(a[1]) && fabs(a[0]) <= fabs(a[2])) ? 0 : (fabs(a[1]) <= fabs(a[2]) ? 1 : 2);
    e[k] = 1.0;
    double c[3];
    v_cross(c, a, e);
    double n = sqrt(v_dot(c, c));
    out[0] = c[0] / n; out[1] = c[1] / n; out[2] = c[2] / n;
}

void orc_svd(const double F[9], double U[9], double S[3], double V[9]) {
    double A[9], lam[3], W[9];
    m_mul_tn(A, F, F);
    sym_eig_jacobi(A, W, lam);
    /* sort eigenpairs descending */
    int idx[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (lam[idx[j]] > lam[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) V[3 * r + c] = W[3 * r + idx[c]];
    if (m_det(V) < 0.0)
        for (int r = 0; r < 3; ++r) V[3 * r + 2] = -V[3 * r + 2];
    /* U columns from F V with Gram-Schmidt; u2 = u0 x u1 makes det U = +1 */
    double FV[9];
    m_mul(FV, F, V);
    double f0[3] = {FV[0], FV[3], FV[6]}, f1[3] = {FV[1], FV[4], FV[7]}, f2[3] = {FV[2], FV[5], FV[8]};
    double u0[3], u1[3], u2[3];
    double n0 = sqrt(v_dot(f0, f0));
    if (n0 > 0.0) { u0[0] = f0[0] / n0; u0[1] = f0[1] / n0; u0[2] = f0[2] / n0; }
    else { u0[0] = V[0]; u0[1] = V[3]; u0[2] = V[6]; }
    double p = v_dot(u0, f1);
    double r1[3] = {f1[0] - p * u0[0], f1[1] - p * u0[1], f1[2] - p * u0[2]};
    double n1 = sqrt(v_dot(r1, r1));
    if (n1 > 1e-300) { u1[0] = r1[0] / n1; u1[1] = r1[1] / n1; u1[2] = r1[2] / n1; }
    else any_orthogonal_unit(u0, u1);
    v_cross(u2, u0, u1);
    for (int r = 0; r < 3; ++r) { U[3 * r + 0] = u0[r]; U[3 * r + 1] = u1[r]; U[3 * r + 2] = u2[r]; }
    S[0] = v_dot(u0, f0);
    S[1] = v_dot(u1, f1);
    S[2] = v_dot(u2, f2);
}

static void usvt(double D[9], const double U[9], const double s[3], const double V[9]) {
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[3 * i + j] = U[3 * i + j] * s[j];
    m_mul_nt(D, T, V);
}

/* polar rotation R = U V^T of F = R S */
void orc_polar(const double F[9], double R[9]) {
    double U[9], S[3], V[9];
    orc_svd(F, U, S, V);
    m_mul_nt(R, U, V);
}

/* ------------------------------------------------------------------------ */
/* Elasticity: Kirchhoff stress tau = P F^T                                  */
/*   fixed-corotated: tau = 2 mu (F - R) F^T + lambda J (J - 1) I  (App. B.1)  */
/*   Neo-Hookean: P = mu (F - F^{-T}) + lambda log J F^{-T} (App. A), so      */
/*                tau = mu (F F^T - I) + lambda log J I                        */
/* ------------------------------------------------------------------------ */

/* Further elastic models of App. B.1 (model codes 2..5):
 *   2 StVK, Green strain E = (F^T F - I)/2: the App. B.1 expression read as a
 *     first Piola-Kirchhoff stress P = 2 mu F E + lambda J (J - 1) F^{-T}, so
 *     tau = P F^T = 2 mu F E F^T + lambda J (J - 1) I;
 *   3 Hencky / SigmaElasticity, eps = log Sigma:
 *     tau = U diag(2 mu eps + lambda tr(eps)) U^T (the same tau as App. A's
 *     StVK, whose P = U (2 mu Sigma^{-1} log Sigma + lambda tr(log Sigma)
 *     Sigma^{-1}) V^T gives P F^T = this); singular values are floored at
 *     1e-4 before the log, as in the return maps;
 *   4 FluidElasticity: tau = lambda J (J - 1) I;
 *   5 VolumeElasticity: tau = kappa (J - J^{1 - gamma}) I, kappa =
 *     2 mu / 3 + lambda, gamma = 2 (J <= 0 is non-finite).                  */
int orc_kirchhoff(int model, const double F[9], double mu, double lam, double tau[9]) {
    double J = m_det(F);
    if (model == 2) {
        double E[9], FE[9];
        m_mul_tn(E, F, F);
        for (int i = 0; i < 9; ++i) E[i] *= 0.5;
        E[0] -= 0.5; E[4] -= 0.5; E[8] -= 0.5;
        m_mul(FE, F, E);
        m_mul_nt(tau, FE, F);
        for (int i = 0; i < 9; ++i) tau[i] *= 2.0 * mu;
        double vol = lam * J * (J - 1.0);
        tau[0] += vol; tau[4] += vol; tau[8] += vol;
        return ORC_OK;
    }
    if (model == 3) {
        double U[9], S[3], V[9], eps[3], d[3];
        orc_svd(F, U, S, V);
        double tr = 0.0;
        for (int i = 0; i < 3; ++i) { eps[i] = log(S[i] > SIGMA_FLOOR ? S[i] : SIGMA_FLOOR); tr += eps[i]; }
        for (int i = 0; i < 3; ++i) d[i] = 2.0 * mu * eps[i] + lam * tr;
        usvt(tau, U, d, U);
        return ORC_OK;
    }
    if (model == 4) {
        memset(tau, 0, 9 * sizeof(double));
        tau[0] = tau[4] = tau[8] = lam * J * (J - 1.0);
        return ORC_OK;
    }
    if (model == 5) {
        if (!(J > 0.0)) return ORC_NONFINITE;
        double kappa = 2.0 * mu / 3.0 + lam;
        memset(tau, 0, 9 * sizeof(double));
        tau[0] = tau[4] = tau[8] = kappa * (J - 1.0 / J);
        return ORC_OK;
    }
    if (model == 0) {
        double R[9], M[9];
        orc_polar(F, R);
        for (int i = 0; i < 9; ++i) M[i] = F[i] - R[i];
        m_mul_nt(tau, M, F);
        for (int i = 0; i < 9; ++i) tau[i] *= 2.0 * mu;
        double vol = lam * J * (J - 1.0);
        tau[0] += vol; tau[4] += vol; tau[8] += vol;
        return ORC_OK;
    }
    if (!(J > 0.0)) return ORC_NONFINITE;       /* log J undefined (reading 13) */
    m_mul_nt(tau, F, F);
    tau[0] -= 1.0; tau[4] -= 1.0; tau[8] -= 1.0;
    for (int i = 0; i < 9; ++i) tau[i] *= mu;
    double vol = lam * log(J);
    tau[0] += vol; tau[4] += vol; tau[8] += vol;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Plasticity (App. A eq. von_mises / eq. drucker_prager, App. B.2).          */
/* psi(F) = U Z(Sigma) V^T with eps = log(max(Sigma, floor)).                 */
/* Drucker-Prager delta-gamma: the strain-space return map of Klar et al.     */
/* 2016 (cited by the paper), zero cohesion:                                  */
/*   alpha = sqrt(2/3) 2 sin(phi) / (3 - sin(phi)),                           */
/*   dgamma = |eps_hat| + (3 lambda + 2 mu)/(2 mu) tr(eps) alpha.             */
/* The map is written as z_i = exp(h_i) and reports which case applied.       */
/* ------------------------------------------------------------------------ */

enum { PM_ELASTIC = 0, PM_PROJECT = 1, PM_TIP = 2 };

double orc_dp_alpha(double phi_deg) {
    double s = sin(phi_deg * M_PI / 180.0);
    return sqrt(2.0 / 3.0) * 2.0 * s / (3.0 - s);
}

/* returns the case; z = new singular values */
static int return_map_sigma(int model, const double s[3], double mu, double lam, double yield,
                            double phi_deg, double z[3]) {
    z[0] = s[0]; z[1] = s[1]; z[2] = s[2];
    if (model == 0) return PM_ELASTIC;
    double eps[3], tr = 0.0;
    for (int i = 0; i < 3; ++i) { eps[i] = log(s[i] > SIGMA_FLOOR ? s[i] : SIGMA_FLOOR); tr += eps[i]; }
    double e[3], nrm = 0.0;
    for (int i = 0; i < 3; ++i) { e[i] = eps[i] - tr / 3.0; nrm += e[i] * e[i]; }
    nrm = sqrt(nrm);
    double dgamma;
    if (model == 1) {
        dgamma = nrm - yield / (2.0 * mu);
        if (dgamma <= 0.0) return PM_ELASTIC;
    } else {
        if (tr > 0.0) { z[0] = z[1] = z[2] = 1.0; return PM_TIP; }
        double alpha = orc_dp_alpha(phi_deg);
        dgamma = nrm + (3.0 * lam + 2.0 * mu) / (2.0 * mu) * tr * alpha;
        if (dgamma <= 0.0) return PM_ELASTIC;
    }
    for (int i = 0; i < 3; ++i) z[i] = exp(eps[i] - dgamma * e[i] / nrm);
    return PM_PROJECT;
}

/* Volume-only plasticity (model codes 3, 4):
 *   3 fluid (App. A eq. fluid_plasticity): F <- J^{1/3} I;
 *   4 SigmaPlasticity (App. B.2): J clamped to [0.05, 1.2], F <- J^{1/3} I.
 * cbrt keeps the sign of J, so an inverted F stays inverted under (3).      */
int orc_return_map(int model, const double F[9], double mu, double lam, double yield, double phi_deg,
                   double Fout[9]) {
    if (model == 0) { m_copy(Fout, F); return PM_ELASTIC; }
    if (model == 3 || model == 4) {
        double J = m_det(F);
        if (model == 4) J = J < 0.05 ? 0.05 : (J > 1.2 ? 1.2 : J);
        double c = cbrt(J);
        memset(Fout, 0, 9 * sizeof(double));
        Fout[0] = Fout[4] = Fout[8] = c;
        return PM_PROJECT;
    }
    double U[9], S[3], V[9], z[3];
    orc_svd(F, U, S, V);
    int c = return_map_sigma(model, S, mu, lam, yield, phi_deg, z);
    if (c == PM_ELASTIC) { m_copy(Fout, F); return c; }
    usvt(Fout, U, z, V);
    return c;
}

/* ------------------------------------------------------------------------ */
/* Forward substep pieces                                                    */
/* ------------------------------------------------------------------------ */

static void particle_lame(const orc_material *mat, long p, double *mu, double *lam) {
    orc_lame(exp(mat->logE[p]), mat->nu[p], mu, lam);
}

/* P2G (§4.2 momentum equation; App. A): grid_m[node], grid_mv[3*node] are
 * zeroed and accumulated. */
int orc_p2g(const orc_cfg *cfg, long n, const double *x, const double *v, const double *C, const double *F,
            const orc_material *mat, double *grid_m, double *grid_mv) {
    long nn = (long)cfg->res[0] * cfg->res[1] * cfg->res[2];
    memset(grid_m, 0, nn * sizeof(double));
    memset(grid_mv, 0, 3 * nn * sizeof(double));
    double dx = cfg->dx, dt = cfg->dt;
    for (long p = 0; p < n; ++p) {
        int base[3]; double fx[3];
        int st = locate(cfg, x + 3 * p, base, fx);
        if (st) return st;
        double mu, lam, tau[9];
        particle_lame(mat, p, &mu, &lam);
        st = orc_kirchhoff(mat->elastic[p], F + 9 * p, mu, lam, tau);
        if (st) return st;
        double mp = mat->mass[p], Vp = mat->vol[p];
        double k = 4.0 * dt * Vp / (dx * dx);
        double A[9];
        for (int i = 0; i < 9; ++i) A[i] = mp * C[9 * p + i] - k * tau[i];
        double w[3][3], dw[3][3];
        for (int d = 0; d < 3; ++d) orc_bspline(fx[d], w[d], dw[d]);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l) {
                    double wt = w[0][i] * w[1][j] * w[2][l];
                    double dpos[3] = {(i - fx[0]) * dx, (j - fx[1]) * dx, (l - fx[2]) * dx};
                    long nd = node_index(cfg, base[0] + i, base[1] + j, base[2] + l);
                    grid_m[nd] += wt * mp;
                    for (int r = 0; r < 3; ++r) {
                        double Ad = A[3 * r] * dpos[0] + A[3 * r + 1] * dpos[1] + A[3 * r + 2] * dpos[2];
                        grid_mv[3 * nd + r] += wt * (mp * v[3 * p + r] + Ad);
                    }
                }
    }
    return ORC_OK;
}

/* Wall rule (reading; the paper states none): band of cfg->bound nodes on each
 * face.  A sticky face zeroes the whole velocity; a slip face zeroes the
 * normal component when it points out of the domain.  Returns per-component
 * pass-through mask (1 keeps the component, 0 zeroes it). */
static void wall_mask(const orc_cfg *cfg, const int I[3], const double u[3], double mask[3]) {
    mask[0] = mask[1] = mask[2] = 1.0;
    int sticky = 0;
    for (int d = 0; d < 3; ++d) {
        if (I[d] < cfg->bound && cfg->wall[2 * d] == 2) sticky = 1;
        if (I[d] >= cfg->res[d] - cfg->bound && cfg->wall[2 * d + 1] == 2) sticky = 1;
    }
    if (sticky) { mask[0] = mask[1] = mask[2] = 0.0; return; }
    for (int d = 0; d < 3; ++d) {
        if (I[d] < cfg->bound && cfg->wall[2 * d] == 1 && u[d] < 0.0) mask[d] = 0.0;
        if (I[d] >= cfg->res[d] - cfg->bound && cfg->wall[2 * d + 1] == 1 && u[d] > 0.0) mask[d] = 0.0;
    }
}

/* Grid update (App. A): v = mv/m + dt g for m > 0, then walls; v = 0 where m = 0. */
void orc_grid_update(const orc_cfg *cfg, const double *grid_m, const double *grid_mv, double *grid_v) {
    for (int I = 0; I < cfg->res[0]; ++I)
        for (int J = 0; J < cfg->res[1]; ++J)
            for (int K = 0; K < cfg->res[2]; ++K) {
                long nd = node_index(cfg, I, J, K);
                double *vv = grid_v + 3 * nd;
                if (!(grid_m[nd] > 0.0)) { vv[0] = vv[1] = vv[2] = 0.0; continue; }
                double u[3], mask[3];
                for (int d = 0; d < 3; ++d) u[d] = grid_mv[3 * nd + d] / grid_m[nd] + cfg->dt * cfg->gravity[d];
                int idx[3] = {I, J, K};
                wall_mask(cfg, idx, u, mask);
                for (int d = 0; d < 3; ++d) vv[d] = mask[d] * u[d];
            }
}

/* G2P + advection + F update + plasticity (App. A; Algorithm 1 Stage 1).
 * Reads x, F (old); writes x, v, C, F (new) in place. */
int orc_g2p(const orc_cfg *cfg, long n, double *x, double *v, double *C, double *F,
            const orc_material *mat, const double *grid_v) {
    double dx = cfg->dx, dt = cfg->dt;
    for (long p = 0; p < n; ++p) {
        int base[3]; double fx[3];
        int st = locate(cfg, x + 3 * p, base, fx);
        if (st) return st;
        double w[3][3], dw[3][3];
        for (int d = 0; d < 3; ++d) orc_bspline(fx[d], w[d], dw[d]);
        double vp[3] = {0, 0, 0}, Bp[9];
        m_zero(Bp);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l) {
                    double wt = w[0][i] * w[1][j] * w[2][l];
                    double dpos[3] = {(i - fx[0]) * dx, (j - fx[1]) * dx, (l - fx[2]) * dx};
                    const double *vi = grid_v + 3 * node_index(cfg, base[0] + i, base[1] + j, base[2] + l);
                    for (int r = 0; r < 3; ++r) {
                        vp[r] += wt * vi[r];
                        for (int c = 0; c < 3; ++c) Bp[3 * r + c] += wt * vi[r] * dpos[c];
                    }
                }
        double Cn[9], G[9], Fn[9];
        for (int i = 0; i < 9; ++i) Cn[i] = 4.0 / (dx * dx) * Bp[i];
        double IC[9];
        for (int i = 0; i < 9; ++i) IC[i] = dt * Cn[i];
        IC[0] += 1.0; IC[4] += 1.0; IC[8] += 1.0;
        m_mul(G, IC, F + 9 * p);
        double mu, lam;
        particle_lame(mat, p, &mu, &lam);
        orc_return_map(mat->plastic[p], G, mu, lam, mat->yield[p], mat->phi_deg[p], Fn);
        for (int r = 0; r < 3; ++r) { v[3 * p + r] = vp[r]; x[3 * p + r] += dt * vp[r]; }
        m_copy(C + 9 * p, Cn);
        m_copy(F + 9 * p, Fn);
    }
    return ORC_OK;
}

static long n_nodes(const orc_cfg *cfg) { return (long)cfg->res[0] * cfg->res[1] * cfg->res[2]; }

/* one full substep in place */
int orc_substep(const orc_cfg *cfg, long n, double *x, double *v, double *C, double *F, const orc_material *mat) {
    long nn = n_nodes(cfg);
    double *gm = (double *)malloc(nn * sizeof(double));
    double *gmv = (double *)malloc(3 * nn * sizeof(double));
    double *gv = (double *)malloc(3 * nn * sizeof(double));
    int st = orc_p2g(cfg, n, x, v, C, F, mat, gm, gmv);
    if (!st) {
        orc_grid_update(cfg, gm, gmv, gv);
        st = orc_g2p(cfg, n, x, v, C, F, mat, gv);
    }
    free(gm); free(gmv); free(gv);
    return st;
}

/* Runs n_sub substeps.  When tape != NULL it receives (n_sub+1) snapshots of
 * the state, each n x 24 doubles laid out [x(3) v(3) C(9) F(9)] per particle. */
static void pack_state(double *dst, long n, const double *x, const double *v, const double *C, const double *F) {
    for (long p = 0; p < n; ++p) {
        double *r = dst + 24 * p;
        memcpy(r, x + 3 * p, 3 * sizeof(double));
        memcpy(r + 3, v + 3 * p, 3 * sizeof(double));
        memcpy(r + 6, C + 9 * p, 9 * sizeof(double));
        memcpy(r + 15, F + 9 * p, 9 * sizeof(double));
    }
}
static void unpack_state(const double *src, long n, double *x, double *v, double *C, double *F) {
    for (long p = 0; p < n; ++p) {
        const double *r = src + 24 * p;
        memcpy(x + 3 * p, r, 3 * sizeof(double));
        memcpy(v + 3 * p, r + 3, 3 * sizeof(double));
        memcpy(C + 9 * p, r + 6, 9 * sizeof(double));
        memcpy(F + 9 * p, r + 15, 9 * sizeof(double));
    }
}

int orc_run(const orc_cfg *cfg, long n, double *x, double *v, double *C, double *F, const orc_material *mat,
            int n_sub, double *tape) {
    if (tape) pack_state(tape, n, x, v, C, F);
    for (int s = 0; s < n_sub; ++s) {
        int st = orc_substep(cfg, n, x, v, C, F, mat);
        if (st) return st;
        if (tape) pack_state(tape + (long)(s + 1) * n * 24, n, x, v, C, F);
    }
    return ORC_OK;
}

/* ======================================================================== */
/* Adjoint (reverse mode) of one substep, derived by hand from the forward   */
/* above.  Given the state at the start of the substep and the adjoint of     */
/* the state at its end, it returns the adjoint of the start state and adds   */
/* the parameter gradients (d/d logE, d/d nu, d/d yield) into g_param.        */
/* ======================================================================== */

/* adjoint of the polar rotation R = U V^T:  Fbar += U Y V^T with
 * K = U^T Rbar V, Y_ij = (K_ij - K_ji) / (s_i + s_j), Y_ii = 0. */
static void polar_adjoint(const double U[9], const double S[3], const double V[9], const double Rbar[9],
                          double Fbar[9]) {
    double K[9], T[9], Y[9];
    m_mul_tn(T, U, Rbar);
    m_mul(K, T, V);
    m_zero(Y);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (i != j) Y[3 * i + j] = (K[3 * i + j] - K[3 * j + i]) / (S[i] + S[j]);
    double D[9];
    m_mul(T, U, Y);
    m_mul_nt(D, T, V);
    for (int i = 0; i < 9; ++i) Fbar[i] += D[i];
}

/* (log a - log b) / (a - b) for a, b > 0; 1/a at a = b */
static double log_divdiff(double a, double b) {
    double d = a - b;
    if (fabs(d) <= 1e-6 * (a + b)) return 2.0 / (a + b);
    return (log(a) - log(b)) / d;
}

/* adjoint of the Kirchhoff stress; adds to Fbar, mubar, lambar */
static void kirchhoff_adjoint(int model, const double F[9], double mu, double lam, const double taubar[9],
                              double Fbar[9], double *mubar, double *lambar) {
    double J = m_det(F), cof[9];
    m_cofactor(cof, F);                  /* dJ/dF */
    double trb = m_trace(taubar);
    if (model == 2) {
        /* tau = 2 mu F E F^T + lam J (J-1) I, E = (F^T F - I)/2:
         * d<tb, F E F^T> = <tb F E + tb^T F E + F (B + B^T)/2, dF>, B = F^T tb F */
        double E[9], FE[9], A[9], B[9], T[9], X[9];
        m_mul_tn(E, F, F);
        for (int i = 0; i < 9; ++i) E[i] *= 0.5;
        E[0] -= 0.5; E[4] -= 0.5; E[8] -= 0.5;
        m_mul(FE, F, E);
        m_mul_nt(A, FE, F);
        *mubar += 2.0 * m_dot(taubar, A);
        *lambar += trb * J * (J - 1.0);
        m_mul_tn(T, F, taubar);
        m_mul(B, T, F);
        double Bs[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Bs[3 * i + j] = 0.5 * (B[3 * i + j] + B[3 * j + i]);
        double tbs[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) tbs[3 * i + j] = taubar[3 * i + j] + taubar[3 * j + i];
        m_mul(X, tbs, FE);
        m_mul(T, F, Bs);
        for (int i = 0; i < 9; ++i) X[i] += T[i];
        double Jbar = lam * trb * (2.0 * J - 1.0);
        for (int i = 0; i < 9; ++i) Fbar[i] += 2.0 * mu * X[i] + Jbar * cof[i];
        return;
    }
    if (model == 3) {
        /* tau = h(b), b = F F^T = U diag(beta) U^T, h_i = 2 mu eps_i + lam tr eps,
         * eps_i = log(max(sigma_i, floor)).  With K = U^T sym(taubar) U:
         * bbar~_kk = sum_i K_ii dh_i/dbeta_k, bbar~_ij = K_ij (h_i - h_j)/(beta_i - beta_j),
         * Fbar += (bbar + bbar^T) F. */
        double U[9], S[3], V[9], eps[3], live[3], beta[3], tr = 0.0;
        orc_svd(F, U, S, V);
        for (int i = 0; i < 3; ++i) {
            live[i] = S[i] > SIGMA_FLOOR ? 1.0 : 0.0;
            eps[i] = log(live[i] > 0.0 ? S[i] : SIGMA_FLOOR);
            beta[i] = S[i] * S[i];
            tr += eps[i];
        }
        double tbs[9], T[9], K[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) tbs[3 * i + j] = 0.5 * (taubar[3 * i + j] + taubar[3 * j + i]);
        m_mul_tn(T, U, tbs);
        m_mul(K, T, U);
        double trK = K[0] + K[4] + K[8];
        for (int i = 0; i < 3; ++i) *mubar += 2.0 * K[4 * i] * eps[i];
        *lambar += trK * tr;
        double Bt[9];
        m_zero(Bt);
        for (int k = 0; k < 3; ++k)   /* d eps_k / d beta_k = 1 / (2 beta_k) */
            Bt[4 * k] = live[k] * (2.0 * mu * K[4 * k] + lam * trK) / (2.0 * beta[k]);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                if (i == j) continue;
                double dd = (live[i] > 0.0 && live[j] > 0.0) ? mu * log_divdiff(beta[i], beta[j]) : 0.0;
                Bt[3 * i + j] = K[3 * i + j] * dd;      /* 2 mu (eps_i - eps_j)/(beta_i - beta_j) */
            }
        double Bb[9], D[9];
        m_mul(T, U, Bt);
        m_mul_nt(Bb, T, U);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) D[3 * i + j] = Bb[3 * i + j] + Bb[3 * j + i];
        m_mul(T, D, F);
        for (int i = 0; i < 9; ++i) Fbar[i] += T[i];
        return;
    }
    if (model == 4) {
        *lambar += trb * J * (J - 1.0);
        double Jbar = lam * trb * (2.0 * J - 1.0);
        for (int i = 0; i < 9; ++i) Fbar[i] += Jbar * cof[i];
        return;
    }
    if (model == 5) {
        double kappa = 2.0 * mu / 3.0 + lam, kbar = trb * (J - 1.0 / J);
        *mubar += 2.0 / 3.0 * kbar;
        *lambar += kbar;
        double Jbar = kappa * trb * (1.0 + 1.0 / (J * J));
        for (int i = 0; i < 9; ++i) Fbar[i] += Jbar * cof[i];
        return;
    }
    if (model == 0) {
        double U[9], S[3], V[9], R[9], M[9], T[9];
        orc_svd(F, U, S, V);
        m_mul_nt(R, U, V);
        for (int i = 0; i < 9; ++i) M[i] = F[i] - R[i];
        /* tau = 2 mu M F^T + lam J (J-1) I */
        m_mul_nt(T, M, F);
        *mubar += 2.0 * m_dot(taubar, T);
        *lambar += trb * J * (J - 1.0);
        double Mbar[9], TbF[9];
        m_mul(Mbar, taubar, F);                 /* d/dM of <taubar, M F^T> */
        for (int i = 0; i < 9; ++i) Mbar[i] *= 2.0 * mu;
        m_mul_tn(TbF, taubar, M);               /* d/dF of <taubar, M F^T> via F^T: taubar^T M */
        for (int i = 0; i < 9; ++i) Fbar[i] += Mbar[i] + 2.0 * mu * TbF[i];
        double Rbar[9];
        for (int i = 0; i < 9; ++i) Rbar[i] = -Mbar[i];
        polar_adjoint(U, S, V, Rbar, Fbar);
        double Jbar = lam * trb * (2.0 * J - 1.0);
        for (int i = 0; i < 9; ++i) Fbar[i] += Jbar * cof[i];
    } else {
        /* tau = mu (F F^T - I) + lam log J I */
        double FFt[9], T[9];
        m_mul_nt(FFt, F, F);
        FFt[0] -= 1.0; FFt[4] -= 1.0; FFt[8] -= 1.0;
        *mubar += m_dot(taubar, FFt);
        *lambar += trb * log(J);
        double S2[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) S2[3 * i + j] = taubar[3 * i + j] + taubar[3 * j + i];
        m_mul(T, S2, F);
        for (int i = 0; i < 9; ++i) Fbar[i] += mu * T[i] + lam * trb / J * cof[i];
    }
}

/* z(sigma) of the return map and its derivatives:
 *   Jz[i][k] = d z_i / d sigma_k, dz_dmu[i], dz_dlam[i], dz_dy[i]. */
static int return_map_jacobian(int model, const double s[3], double mu, double lam, double yield, double phi_deg,
                               double z[3], double Jz[9], double dz_dmu[3], double dz_dlam[3], double dz_dy[3]) {
    int c = return_map_sigma(model, s, mu, lam, yield, phi_deg, z);
    for (int i = 0; i < 3; ++i) { dz_dmu[i] = dz_dlam[i] = dz_dy[i] = 0.0; }
    m_zero(Jz);
    if (c == PM_ELASTIC) { Jz[0] = Jz[4] = Jz[8] = 1.0; return c; }
    if (c == PM_TIP) return c;
    double eps[3], tr = 0.0, deps[3];
    for (int i = 0; i < 3; ++i) {
        int clamped = !(s[i] > SIGMA_FLOOR);
        eps[i] = log(clamped ? SIGMA_FLOOR : s[i]);
        deps[i] = clamped ? 0.0 : 1.0 / s[i];
        tr += eps[i];
    }
    double e[3], nrm = 0.0;
    for (int i = 0; i < 3; ++i) { e[i] = eps[i] - tr / 3.0; nrm += e[i] * e[i]; }
    nrm = sqrt(nrm);
    double dgamma, ddg_deps[3], ddg_dmu, ddg_dlam, ddg_dy;
    if (model == 1) {
        dgamma = nrm - yield / (2.0 * mu);
        for (int k = 0; k < 3; ++k) ddg_deps[k] = e[k] / nrm;
        ddg_dmu = yield / (2.0 * mu * mu);
        ddg_dlam = 0.0;
        ddg_dy = -1.0 / (2.0 * mu);
    } else {
        double alpha = orc_dp_alpha(phi_deg);
        double kap = (3.0 * lam + 2.0 * mu) / (2.0 * mu) * alpha;
        dgamma = nrm + kap * tr;
        for (int k = 0; k < 3; ++k) ddg_deps[k] = e[k] / nrm + kap;
        ddg_dmu = tr * (-3.0 * lam * alpha / (2.0 * mu * mu));
        ddg_dlam = tr * (3.0 * alpha / (2.0 * mu));
        ddg_dy = 0.0;
    }
    /* h_i = eps_i - dgamma e_i / nrm ; z_i = exp(h_i) */
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) {
            double Pik = (i == k ? 1.0 : 0.0) - 1.0 / 3.0;
            double dunit = (Pik - e[i] * e[k] / (nrm * nrm)) / nrm;   /* d(e_i/nrm)/d eps_k */
            double dh = (i == k ? 1.0 : 0.0) - ddg_deps[k] * e[i] / nrm - dgamma * dunit;
            Jz[3 * i + k] = z[i] * dh * deps[k];
        }
        dz_dmu[i] = -z[i] * ddg_dmu * e[i] / nrm;
        dz_dlam[i] = -z[i] * ddg_dlam * e[i] / nrm;
        dz_dy[i] = -z[i] * ddg_dy * e[i] / nrm;
    }
    return c;
}

/* adjoint of psi(G) = U diag(z(sigma)) V^T.  K = U^T Fbar_out V;
 *   sigma_bar_k = sum_i K_ii dz_i/dsigma_k;
 *   off-diagonal: Y_ij = K_ij (A+B)/2 + K_ji (A-B)/2, with
 *   A = (z_i - z_j)/(s_i - s_j) (divided difference; at s_i = s_j its limit
 *   dz_i/ds_i - dz_i/ds_j for an isotropic map) and B = (z_i + z_j)/(s_i + s_j). */
static void plastic_adjoint(int model, const double G[9], double mu, double lam, double yield, double phi_deg,
                            const double Fbar_out[9], double Gbar[9], double *mubar, double *lambar, double *ybar) {
    if (model == 0) { m_copy(Gbar, Fbar_out); return; }
    if (model == 3 || model == 4) {
        /* F = c I, c = J^{1/3} (clamped J for model 4, where a clamp stops the
         * derivative): dc = (c / 3J) dJ, dJ = <cof G, dG> */
        double J = m_det(G), cof[9];
        m_cofactor(cof, G);
        int clamped = model == 4 && (J < 0.05 || J > 1.2);
        double c = cbrt(J), k = clamped ? 0.0 : m_trace(Fbar_out) * c / (3.0 * J);
        for (int i = 0; i < 9; ++i) Gbar[i] = k * cof[i];
        return;
    }
    double U[9], S[3], V[9], z[3], Jz[9], dmu[3], dlam[3], dy[3];
    orc_svd(G, U, S, V);
    int c = return_map_jacobian(model, S, mu, lam, yield, phi_deg, z, Jz, dmu, dlam, dy);
    if (c == PM_ELASTIC) { m_copy(Gbar, Fbar_out); return; }
    double K[9], T[9], Y[9];
    m_mul_tn(T, U, Fbar_out);
    m_mul(K, T, V);
    m_zero(Y);
    for (int k = 0; k < 3; ++k) {
        double sb = 0.0;
        for (int i = 0; i < 3; ++i) sb += K[4 * i] * Jz[3 * i + k];
        Y[4 * k] = sb;
    }
    for (int i = 0; i < 3; ++i) {
        *mubar += K[4 * i] * dmu[i];
        *lambar += K[4 * i] * dlam[i];
        *ybar += K[4 * i] * dy[i];
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (i == j) continue;
            double A, B;
            double ds = S[i] - S[j], scale = fabs(S[i]) + fabs(S[j]);
            if (fabs(ds) > 1e-6 * scale) A = (z[i] - z[j]) / ds;
            else A = Jz[3 * i + i] - Jz[3 * i + j];
            B = (z[i] + z[j]) / (S[i] + S[j]);
            Y[3 * i + j] = K[3 * i + j] * 0.5 * (A + B) + K[3 * j + i] * 0.5 * (A - B);
        }
    m_mul(T, U, Y);
    m_mul_nt(Gbar, T, V);
}

/* adj layout per particle: [x(3) v(3) C(9) F(9)].  adj_out is the adjoint of
 * the end state; adj_in receives the adjoint of the start state.  g_param is
 * n x 3 (logE, nu, yield), accumulated. */
int orc_substep_adjoint(const orc_cfg *cfg, long n, const double *state, const orc_material *mat,
                        const double *adj_out, double *adj_in, double *g_param) {
    long nn = n_nodes(cfg);
    double dx = cfg->dx, dt = cfg->dt, inv_dx2 = 1.0 / (dx * dx);
    double *x = (double *)malloc(3 * n * sizeof(double)), *v = (double *)malloc(3 * n * sizeof(double));
    double *C = (double *)malloc(9 * n * sizeof(double)), *F = (double *)malloc(9 * n * sizeof(double));
    unpack_state(state, n, x, v, C, F);
    double *gm = (double *)calloc(nn, sizeof(double)), *gP = (double *)calloc(3 * nn, sizeof(double));
    double *gv = (double *)calloc(3 * nn, sizeof(double)), *gmask = (double *)calloc(3 * nn, sizeof(double));
    double *gvbar = (double *)calloc(3 * nn, sizeof(double));
    double *gmbar = (double *)calloc(nn, sizeof(double)), *gPbar = (double *)calloc(3 * nn, sizeof(double));
    int st = orc_p2g(cfg, n, x, v, C, F, mat, gm, gP);
    if (st) goto done;
    /* grid update, keeping the wall masks */
    for (int I = 0; I < cfg->res[0]; ++I)
        for (int J = 0; J < cfg->res[1]; ++J)
            for (int K = 0; K < cfg->res[2]; ++K) {
                long nd = node_index(cfg, I, J, K);
                if (!(gm[nd] > 0.0)) continue;
                double u[3], mask[3];
                for (int d = 0; d < 3; ++d) u[d] = gP[3 * nd + d] / gm[nd] + dt * cfg->gravity[d];
                int idx[3] = {I, J, K};
                wall_mask(cfg, idx, u, mask);
                for (int d = 0; d < 3; ++d) { gv[3 * nd + d] = mask[d] * u[d]; gmask[3 * nd + d] = mask[d]; }
            }
    /* G2P reverse: scatter onto grid velocity adjoints, partial particle adjoints */
    for (long p = 0; p < n; ++p) {
        const double *ao = adj_out + 24 * p;
        double *ai = adj_in + 24 * p;
        memset(ai, 0, 24 * sizeof(double));
        int base[3]; double fx[3];
        locate(cfg, x + 3 * p, base, fx);
        double w[3][3], dw[3][3];
        for (int d = 0; d < 3; ++d) orc_bspline(fx[d], w[d], dw[d]);
        /* recompute v', C' */
        double vp[3] = {0, 0, 0}, Cn[9];
        m_zero(Cn);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l) {
                    double wt = w[0][i] * w[1][j] * w[2][l];
                    double dpos[3] = {(i - fx[0]) * dx, (j - fx[1]) * dx, (l - fx[2]) * dx};
                    const double *vi = gv + 3 * node_index(cfg, base[0] + i, base[1] + j, base[2] + l);
                    for (int r = 0; r < 3; ++r) {
                        vp[r] += wt * vi[r];
                        for (int c = 0; c < 3; ++c) Cn[3 * r + c] += 4.0 * inv_dx2 * wt * vi[r] * dpos[c];
                    }
                }
        double IC[9], G[9];
        for (int i = 0; i < 9; ++i) IC[i] = dt * Cn[i];
        IC[0] += 1.0; IC[4] += 1.0; IC[8] += 1.0;
        m_mul(G, IC, F + 9 * p);
        double mu, lam, mubar = 0.0, lambar = 0.0, ybar = 0.0, Gbar[9];
        particle_lame(mat, p, &mu, &lam);
        plastic_adjoint(mat->plastic[p], G, mu, lam, mat->yield[p], mat->phi_deg[p], ao + 15, Gbar,
                        &mubar, &lambar, &ybar);
        /* G = (I + dt C') F */
        double Cbar[9], T[9];
        m_mul_nt(T, Gbar, F + 9 * p);
        for (int i = 0; i < 9; ++i) Cbar[i] = ao[6 + i] + dt * T[i];
        m_mul_tn(T, IC, Gbar);
        for (int i = 0; i < 9; ++i) ai[15 + i] += T[i];
        /* x' = x + dt v' */
        double vbar[3];
        for (int r = 0; r < 3; ++r) { ai[r] += ao[r]; vbar[r] = ao[3 + r] + dt * ao[r]; }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l) {
                    int o[3] = {i, j, l};
                    double wt = w[0][i] * w[1][j] * w[2][l];
                    double gw[3] = {dw[0][i] * w[1][j] * w[2][l] / dx, w[0][i] * dw[1][j] * w[2][l] / dx,
                                    w[0][i] * w[1][j] * dw[2][l] / dx};
                    double dpos[3] = {(i - fx[0]) * dx, (j - fx[1]) * dx, (l - fx[2]) * dx};
                    long nd = node_index(cfg, base[0] + o[0], base[1] + o[1], base[2] + o[2]);
                    const double *vi = gv + 3 * nd;
                    double wbar = 0.0, dposbar[3] = {0, 0, 0};
                    for (int r = 0; r < 3; ++r) {
                        double cd = Cbar[3 * r] * dpos[0] + Cbar[3 * r + 1] * dpos[1] + Cbar[3 * r + 2] * dpos[2];
                        gvbar[3 * nd + r] += wt * vbar[r] + 4.0 * inv_dx2 * wt * cd;
                        wbar += vbar[r] * vi[r] + 4.0 * inv_dx2 * vi[r] * cd;
                    }
                    for (int c = 0; c < 3; ++c) {
                        double s = 0.0;
                        for (int r = 0; r < 3; ++r) s += Cbar[3 * r + c] * vi[r];
                        dposbar[c] = 4.0 * inv_dx2 * wt * s;
                    }
                    for (int d = 0; d < 3; ++d) ai[d] += wbar * gw[d] - dposbar[d];
                }
        double dl[4];
        lame_grad(mat->logE[p], mat->nu[p], dl);
        g_param[3 * p + 0] += mubar * dl[0] + lambar * dl[2];
        g_param[3 * p + 1] += mubar * dl[1] + lambar * dl[3];
        g_param[3 * p + 2] += ybar;
    }
    /* grid update reverse */
    for (long nd = 0; nd < nn; ++nd) {
        if (!(gm[nd] > 0.0)) continue;
        double m = gm[nd], s = 0.0;
        for (int d = 0; d < 3; ++d) {
            double ub = gmask[3 * nd + d] * gvbar[3 * nd + d];
            gPbar[3 * nd + d] = ub / m;
            s += ub * gP[3 * nd + d];
        }
        gmbar[nd] = -s / (m * m);
    }
    /* P2G reverse: gather grid adjoints */
    for (long p = 0; p < n; ++p) {
        double *ai = adj_in + 24 * p;
        int base[3]; double fx[3];
        locate(cfg, x + 3 * p, base, fx);
        double w[3][3], dw[3][3];
        for (int d = 0; d < 3; ++d) orc_bspline(fx[d], w[d], dw[d]);
        double mu, lam, tau[9];
        particle_lame(mat, p, &mu, &lam);
        orc_kirchhoff(mat->elastic[p], F + 9 * p, mu, lam, tau);
        double mp = mat->mass[p], kf = 4.0 * dt * mat->vol[p] * inv_dx2;
        double A[9], Abar[9];
        for (int i = 0; i < 9; ++i) A[i] = mp * C[9 * p + i] - kf * tau[i];
        m_zero(Abar);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l) {
                    double wt = w[0][i] * w[1][j] * w[2][l];
                    double gw[3] = {dw[0][i] * w[1][j] * w[2][l] / dx, w[0][i] * dw[1][j] * w[2][l] / dx,
                                    w[0][i] * w[1][j] * dw[2][l] / dx};
                    double dpos[3] = {(i - fx[0]) * dx, (j - fx[1]) * dx, (l - fx[2]) * dx};
                    long nd = node_index(cfg, base[0] + i, base[1] + j, base[2] + l);
                    const double *Pb = gPbar + 3 * nd;
                    double wbar = gmbar[nd] * mp;
                    double dposbar[3] = {0, 0, 0};
                    for (int r = 0; r < 3; ++r) {
                        double Ad = A[3 * r] * dpos[0] + A[3 * r + 1] * dpos[1] + A[3 * r + 2] * dpos[2];
                        wbar += Pb[r] * (mp * v[3 * p + r] + Ad);
                        ai[3 + r] += wt * mp * Pb[r];
                        for (int c = 0; c < 3; ++c) {
                            Abar[3 * r + c] += wt * Pb[r] * dpos[c];
                            dposbar[c] += wt * A[3 * r + c] * Pb[r];
                        }
                    }
                    for (int d = 0; d < 3; ++d) ai[d] += wbar * gw[d] - dposbar[d];
                }
        double taubar[9], mubar = 0.0, lambar = 0.0;
        for (int i = 0; i < 9; ++i) { ai[6 + i] += mp * Abar[i]; taubar[i] = -kf * Abar[i]; }
        kirchhoff_adjoint(mat->elastic[p], F + 9 * p, mu, lam, taubar, ai + 15, &mubar, &lambar);
        double dl[4];
        lame_grad(mat->logE[p], mat->nu[p], dl);
        g_param[3 * p + 0] += mubar * dl[0] + lambar * dl[2];
        g_param[3 * p + 1] += mubar * dl[1] + lambar * dl[3];
    }
done:
    free(x); free(v); free(C); free(F);
    free(gm); free(gP); free(gv); free(gmask); free(gvbar); free(gmbar); free(gPbar);
    return st;
}

/* Trajectory adjoint.  tape holds (n_sub+1) states from orc_run.  Frame f is
 * the state after frame_sub[f] substeps; dLdx[f] (n x 3) is the loss gradient
 * with respect to the positions of that frame.  Writes the adjoint of the
 * initial state (n x 24) and the parameter gradients (n x 3, overwritten). */
int orc_backward(const orc_cfg *cfg, long n, const orc_material *mat, int n_sub, const double *tape,
                 int n_frames, const int *frame_sub, const double *dLdx, double *adj0, double *g_param) {
    double *a = (double *)calloc(24 * n, sizeof(double)), *b = (double *)calloc(24 * n, sizeof(double));
    memset(g_param, 0, 3 * n * sizeof(double));
    int st = ORC_OK;
    for (int s = n_sub; s >= 0; --s) {
        for (int f = 0; f < n_frames; ++f)
            if (frame_sub[f] == s)
                for (long p = 0; p < n; ++p)
                    for (int d = 0; d < 3; ++d) a[24 * p + d] += dLdx[((long)f * n + p) * 3 + d];
        if (s == 0) break;
        st = orc_substep_adjoint(cfg, n, tape + (long)(s - 1) * n * 24, mat, a, b, g_param);
        if (st) break;
        double *t = a; a = b; b = t;
    }
    memcpy(adj0, a, 24 * n * sizeof(double));
    free(a); free(b);
    return st;
}

/* ------------------------------------------------------------------------ */
/* BGDO stage 2: the gradient-based backward optimisation of log E from      */
/* stored key frames (§4.3 "Optimization Algorithm", Algorithm 1, App. F).   */
/*                                                                          */
/* For every key frame k with state (x, v, C, F)_k and every particle p:     */
/*   s_p      = |tau_p(F_p, log E_p)|_F, tau the Kirchhoff stress of the     */
/*              particle's elastic model;                                    */
/*   g_tau,p  = d s_p / d log E_p (the derivative is taken through the Lame   */
/*              parameters, d mu / d log E = mu, d lambda / d log E = lambda  */
/*              at fixed nu, App. B.1);                                      */
/*   gt_p     = log(1 + |g_tau,p|)                       (App. F.3);         */
/*   F'_p     = the F of one pseudo substep from the key frame, after the     */
/*              return map (Algorithm 1, Stage 2);                           */
/*   delta_p  = |F'_p - I|_F                             (App. F.2);         */
/*   eta_p    = min(1, 0.1 log(1 + E_p)) (§4.3 eq. eq_target), or the fixed   */
/*              weight w of Algorithm 1 when w >= 0;                          */
/*   G_p     += (eta_p gt_p - (1 - eta_p)(delta_p - delta_target)) / K.      */
/* Then log E_p <- log E_p - G_p (done by the caller).  Readings: the norms   */
/* are per particle (App. F.2 defines delta on one 3x3 F'); compression      */
/* is applied per key frame before the average (Algorithm 1); with           */
/* per_material the G of all particles carrying the same label is replaced   */
/* by its mean (the spatial average App. F.3 mentions).  delta_pre_step      */
/* takes delta from the key frame's own F, the d_F of the §4.3 equation.     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double delta_target;
    double w;
    int per_material;
    int delta_pre_step;
} orc_bgdo_opt;

/* d tau / d log E at fixed nu: tau is linear in (mu, lambda) for every model
 * here, so it is mu tau(F; 1, 0) + lambda tau(F; 0, 1). */
static int kirchhoff_dlogE(int model, const double F[9], double mu, double lam, double dtau[9]) {
    double a[9], b[9];
    int st = orc_kirchhoff(model, F, 1.0, 0.0, a);
    if (st) return st;
    st = orc_kirchhoff(model, F, 0.0, 1.0, b);
    if (st) return st;
    for (int i = 0; i < 9; ++i) dtau[i] = mu * a[i] + lam * b[i];
    return ORC_OK;
}

/* keys: n_keys packed states (n x 24 each).  label/n_labels are used only with
 * per_material.  g_tau and delta (n_keys x n, nullable) receive the per-key
 * signals.  G (n) receives the update. */
int orc_bgdo(const orc_cfg *cfg, long n, int n_keys, const double *keys, const orc_material *mat,
             const int *label, int n_labels, const orc_bgdo_opt *opt, double *G, double *g_tau,
             double *delta) {
    double *x = (double *)malloc(3 * n * sizeof(double)), *v = (double *)malloc(3 * n * sizeof(double));
    double *C = (double *)malloc(9 * n * sizeof(double)), *F = (double *)malloc(9 * n * sizeof(double));
    double *F0 = (double *)malloc(9 * n * sizeof(double));
    int st = ORC_OK;
    for (long p = 0; p < n; ++p) G[p] = 0.0;
    for (int k = 0; k < n_keys && !st; ++k) {
        unpack_state(keys + (size_t)k * n * 24, n, x, v, C, F);
        memcpy(F0, F, 9 * n * sizeof(double));
        if (!opt->delta_pre_step) st = orc_substep(cfg, n, x, v, C, F, mat);   /* pseudo step */
        for (long p = 0; p < n && !st; ++p) {
            double mu, lam, tau[9], dtau[9];
            particle_lame(mat, p, &mu, &lam);
            st = orc_kirchhoff(mat->elastic[p], F0 + 9 * p, mu, lam, tau);
            if (!st) st = kirchhoff_dlogE(mat->elastic[p], F0 + 9 * p, mu, lam, dtau);
            if (st) break;
            double s = sqrt(m_dot(tau, tau));
            double g = s > 0.0 ? m_dot(tau, dtau) / s : 0.0;
            double gt = log(1.0 + fabs(g));
            const double *Fn = opt->delta_pre_step ? F0 + 9 * p : F + 9 * p;
            double d2 = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double t = Fn[3 * i + j] - (i == j ? 1.0 : 0.0);
                    d2 += t * t;
                }
            double dl = sqrt(d2);
            double E = exp(mat->logE[p]);
            double eta = opt->w >= 0.0 ? opt->w : fmin(1.0, 0.1 * log(1.0 + E));
            G[p] += (eta * gt - (1.0 - eta) * (dl - opt->delta_target)) / n_keys;
            if (g_tau) g_tau[(size_t)k * n + p] = g;
            if (delta) delta[(size_t)k * n + p] = dl;
        }
    }
    if (!st && opt->per_material) {
        double *sum = (double *)calloc(n_labels, sizeof(double));
        long *cnt = (long *)calloc(n_labels, sizeof(long));
        for (long p = 0; p < n; ++p) { sum[label[p]] += G[p]; cnt[label[p]] += 1; }
        for (long p = 0; p < n; ++p) G[p] = sum[label[p]] / cnt[label[p]];
        free(sum); free(cnt);
    }
    free(x); free(v); free(C); free(F); free(F0);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Gaussian-kernel covariance carried by a particle (§3.1, §3.2): the        */
/* kernel deforms with the particle, Sigma(t) = F(t) Sigma F(t)^T.           */
/* cov0 and out hold the symmetric 3x3 as xx xy xz yy yz zz per particle.    */
/* ------------------------------------------------------------------------ */

static void sym_unpack(const double *c, double S[9]) {
    S[0] = c[0]; S[1] = c[1]; S[2] = c[2];
    S[3] = c[1]; S[4] = c[3]; S[5] = c[4];
    S[6] = c[2]; S[7] = c[4]; S[8] = c[5];
}

void orc_covariance(long n, const double *F, const double *cov0, double *out) {
    for (long p = 0; p < n; ++p) {
        double S[9], FS[9], T[9];
        sym_unpack(cov0 + 6 * p, S);
        m_mul(FS, F + 9 * p, S);
        m_mul_nt(T, FS, F + 9 * p);
        double *o = out + 6 * p;
        o[0] = T[0]; o[1] = T[1]; o[2] = T[2]; o[3] = T[4]; o[4] = T[5]; o[5] = T[8];
    }
}

/* ------------------------------------------------------------------------ */
/* MCIS, Monte Carlo Importance Sampling of interior fill points (§4.1,     */
/* steps 1-4).  Per object k (cluster C_k with candidates Q_k, given as      */
/* contiguous ranges surf_off[k]..surf_off[k+1], cand_off[k]..cand_off[k+1]):*/
/*   d_j = min_{c in C_k} |q_j - c|                     (step 1)             */
/*   w_j = max(exp(-d_j^2 / (2 sigma^2)), eps)          (step 2)             */
/*   p_j = w_j / sum_j' w_j'                            (step 3)             */
/*   n_k i.i.d. draws with P(s = q_j) = p_j             (step 4)             */
/* Readings: the draws are with replacement (each draw has the stated law); */
/* draw i of object k takes the uniform u_i in [0, 1) given as input and     */
/* returns the first candidate whose cumulative weight exceeds               */
/* floor(u_i W_k), with the weights summed as integers w_j 2^40 rounded to   */
/* nearest, so that the cumulative sums do not depend on summation order.   */
/* Distances are exact: brute force over C_k in double precision.           */
/* ------------------------------------------------------------------------ */

#define MCIS_WSCALE 1099511627776.0   /* 2^40 */

void orc_mcis(int n_obj, const long *surf_off, const double *surf, const long *cand_off, const double *cand,
              const long *draw_off, const double *u, double sigma, double eps, double *d_out, double *w_out,
              long long *cum_out, long *picked) {
    for (int k = 0; k < n_obj; ++k) {
        const long c0 = cand_off[k], nc = cand_off[k + 1] - cand_off[k];
        long long *cum = (long long *)malloc((nc > 0 ? nc : 1) * sizeof(long long));
        long long total = 0;
        for (long j = 0; j < nc; ++j) {
            const double *q = cand + 3 * (c0 + j);
            double best = INFINITY;
            for (long c = surf_off[k]; c < surf_off[k + 1]; ++c) {
                double e0 = q[0] - surf[3 * c], e1 = q[1] - surf[3 * c + 1], e2 = q[2] - surf[3 * c + 2];
                double d2 = e0 * e0 + e1 * e1 + e2 * e2;
                if (d2 < best) best = d2;
            }
            double w = exp(-best / (2.0 * sigma * sigma));
            if (w < eps) w = eps;
            total += (long long)floor(w * MCIS_WSCALE + 0.5);   /* round half up: exact for w <= 1 */
            cum[j] = total;
            if (d_out) d_out[c0 + j] = sqrt(best);
            if (w_out) w_out[c0 + j] = w;
            if (cum_out) cum_out[c0 + j] = total;
        }
        for (long i = draw_off[k]; i < draw_off[k + 1]; ++i) {
            if (nc == 0) { picked[i] = -1; continue; }
            const long long t = (long long)floor(u[i] * (double)total);
            long j = 0;
            while (j < nc - 1 && cum[j] <= t) ++j;     /* first cumulative weight above t */
            picked[i] = c0 + j;
        }
        free(cum);
    }
}

/* ------------------------------------------------------------------------ */
/* Splatting of the deformed Gaussian kernels (§3.1): a Gaussian with mean   */
/* mu and covariance Sigma projects to Sigma' = J W Sigma W^T J^T, with W    */
/* the rotation of the view transform and J the Jacobian of the perspective  */
/* projection at the mean; a pixel's colour blends the Gaussians front to    */
/* back, Col = sum_i col_i alpha_i prod_{j<i} (1 - alpha_j), with           */
/* alpha_i = o_i exp(-1/2 d^T Sigma'^{-1} d), d = pixel centre - projected   */
/* mean.  Readings where the paper defers to 3DGS (its cited renderer):      */
/*   - view: camera coordinates t = R mu + T (row-major 3x4 [R | T]);        */
/*     u = fx t_x / t_z + cx, v = fy t_y / t_z + cy; Gaussians with           */
/*     t_z <= 0.2 are not drawn;                                             */
/*   - Sigma' is dilated by 0.3 I (pixel low-pass);                          */
/*   - a Gaussian touches the 16x16-pixel tiles its square of half-width     */
/*     ceil(3 sqrt(lambda_max(Sigma'))) around (u, v) overlaps, and only     */
/*     pixels of those tiles;                                                */
/*   - alpha = min(0.99, o exp(power)); skipped when power > 0 or alpha <     */
/*     1/255; a pixel stops when its transmittance would drop below 1e-4;   */
/*   - the background is added with the remaining transmittance;            */
/*   - order: by t_z, ties by index.                                         */
/* Brute force per pixel over all Gaussians, in double precision.            */
/*                                                                          */
/* Order ambiguity (optional output amb, per pixel).  An implementation that */
/* computes t_z in lower precision may order two Gaussians whose depths lie  */
/* within its rounding the other way, and may draw or drop a Gaussian whose  */
/* t_z lies within its rounding of 0.2.  Gaussian i's depth is given the     */
/* error bound delta_i = tie_eps (|R_20 mu_0| + |R_21 mu_1| + |R_22 mu_2| +  */
/* |T_2|).  Swapping two layers that follow each other at a pixel, with      */
/* transmittance T in front of them, changes the colour by                   */
/*     T alpha_1 alpha_2 (col_1 - col_2)                                     */
/* and leaves the transmittance behind them unchanged (both orders leave     */
/* T (1 - alpha_1)(1 - alpha_2)).  amb adds, per pixel, T alpha_1 alpha_2    */
/* max_k |col_1k - col_2k| for every pair of consecutive contributing layers */
/* whose depths differ by at most delta_1 + delta_2, and T alpha for every   */
/* Gaussian within its delta of the near plane (drawn or not): a bound on    */
/* how far any such reordering can move the pixel.                          */
/* ------------------------------------------------------------------------ */

typedef struct { double u, v, ca, cb, cc, depth, delta; int rx0, rx1, ry0, ry1, ok, maybe; } orc_splat;

static int splat_cmp_depth(const void *a, const void *b) {
    const double *x = (const double *)a, *y = (const double *)b;
    if (x[0] < y[0]) return -1;
    if (x[0] > y[0]) return 1;
    return x[1] < y[1] ? -1 : (x[1] > y[1]);
}

void orc_render(long n, const double *mean, const double *cov, const double *col, const double *opac,
                const double *view, double fx, double fy, double cx, double cy, int W, int H, const double *bg,
                double *img, double *T_out, double tie_eps, double *amb) {
    const int TS = 16;
    const int gx = (W + TS - 1) / TS, gy = (H + TS - 1) / TS;
    orc_splat *sp = (orc_splat *)malloc((n > 0 ? n : 1) * sizeof(orc_splat));
    double *order = (double *)malloc((n > 0 ? n : 1) * 2 * sizeof(double));
    long m = 0;
    for (long i = 0; i < n; ++i) {
        const double *R = view, *p = mean + 3 * i;
        double t[3];
        for (int r = 0; r < 3; ++r) t[r] = R[4 * r] * p[0] + R[4 * r + 1] * p[1] + R[4 * r + 2] * p[2] + R[4 * r + 3];
        const double delta = tie_eps * (fabs(R[8] * p[0]) + fabs(R[9] * p[1]) + fabs(R[10] * p[2]) + fabs(R[11]));
        sp[i].ok = 0;
        /* drawn when t_z > 0.2; within delta of it, amb counts it either way */
        const int maybe = amb && fabs(t[2] - 0.2) <= delta;
        if (!(t[2] > 0.2) && !maybe) continue;
        const double *c = cov + 6 * i;
        double S[9] = {c[0], c[1], c[2], c[1], c[3], c[4], c[2], c[4], c[5]}, Wr[9], WS[9], Sc[9];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) Wr[3 * r + q] = R[4 * r + q];
        m_mul(WS, Wr, S);
        m_mul_nt(Sc, WS, Wr);                      /* W Sigma W^T, camera frame */
        const double iz = 1.0 / t[2];
        const double J[6] = {fx * iz, 0.0, -fx * t[0] * iz * iz, 0.0, fy * iz, -fy * t[1] * iz * iz};
        double JS[6];
        for (int r = 0; r < 2; ++r)
            for (int q = 0; q < 3; ++q)
                JS[3 * r + q] = J[3 * r] * Sc[q] + J[3 * r + 1] * Sc[3 + q] + J[3 * r + 2] * Sc[6 + q];
        double a = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2] + 0.3;
        double b = JS[0] * J[3] + JS[1] * J[4] + JS[2] * J[5];
        double d = JS[3] * J[3] + JS[4] * J[4] + JS[5] * J[5] + 0.3;
        const double det = a * d - b * b;
        if (!(det > 0.0)) continue;
        const double mid = 0.5 * (a + d), disc = sqrt(fmax(0.1, mid * mid - det));
        const double lmax = fmax(mid + disc, mid - disc);
        const double rad = ceil(3.0 * sqrt(lmax));
        const double u = fx * t[0] * iz + cx, v = fy * t[1] * iz + cy;
        int x0 = (int)fmin(gx, fmax(0.0, floor((u - rad) / TS))), x1 = (int)fmin(gx, fmax(0.0, floor((u + rad + TS - 1) / TS)));
        int y0 = (int)fmin(gy, fmax(0.0, floor((v - rad) / TS))), y1 = (int)fmin(gy, fmax(0.0, floor((v + rad + TS - 1) / TS)));
        if (x1 <= x0 || y1 <= y0) continue;
        sp[i].u = u; sp[i].v = v; sp[i].depth = t[2]; sp[i].delta = delta;
        sp[i].ca = d / det; sp[i].cb = -b / det; sp[i].cc = a / det;
        sp[i].rx0 = x0; sp[i].rx1 = x1; sp[i].ry0 = y0; sp[i].ry1 = y1; sp[i].ok = 1;
        sp[i].maybe = maybe;
        order[2 * m] = t[2];
        order[2 * m + 1] = (double)i;
        ++m;
    }
    qsort(order, m, 2 * sizeof(double), splat_cmp_depth);
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            const int tx = px / TS, ty = py / TS;
            double T = 1.0, C[3] = {0.0, 0.0, 0.0}, A = 0.0;
            long prev = -1;                    /* previous contributing layer */
            double prev_alpha = 0.0, prev_T = 1.0;
            for (long q = 0; q < m; ++q) {
                const long i = (long)order[2 * q + 1];
                const orc_splat *g = &sp[i];
                if (tx < g->rx0 || tx >= g->rx1 || ty < g->ry0 || ty >= g->ry1) continue;
                const double dx = (px + 0.5) - g->u, dy = (py + 0.5) - g->v;
                const double power = -0.5 * (g->ca * dx * dx + g->cc * dy * dy) - g->cb * dx * dy;
                if (power > 0.0) continue;
                double alpha = fmin(0.99, opac[i] * exp(power));
                if (alpha < 1.0 / 255.0) continue;
                if (g->maybe) {
                    A += T * alpha;
                    if (!(g->depth > 0.2)) continue;       /* not drawn here */
                }
                const double tt = T * (1.0 - alpha);
                if (tt < 1e-4) break;
                if (amb && prev >= 0 && fabs(g->depth - sp[prev].depth) <= g->delta + sp[prev].delta) {
                    double dc = 0.0;
                    for (int k = 0; k < 3; ++k) dc = fmax(dc, fabs(col[3 * i + k] - col[3 * prev + k]));
                    A += prev_T * prev_alpha * alpha * dc;
                }
                for (int k = 0; k < 3; ++k) C[k] += col[3 * i + k] * alpha * T;
                prev = i; prev_alpha = alpha; prev_T = T;
                T = tt;
            }
            double *o = img + 3 * ((size_t)py * W + px);
            for (int k = 0; k < 3; ++k) o[k] = C[k] + T * bg[k];
            if (T_out) T_out[(size_t)py * W + px] = T;
            if (amb) amb[(size_t)py * W + px] = A;
        }
    free(sp);
    free(order);
}
