// mpm_noalloc.cu -- mpm_substep_noalloc: one MLS-MPM substep that allocates
// no device memory.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// budgeted once at start-up and must not grow, code that runs while another
// allocator owns the device's memory, or a latency-critical path that cannot
// accept the implicit device-wide synchronisation cudaMalloc / cudaFree may
// cause.  For them this entry point keeps its only scratch -- a dense grid of
// at most MPM_NOALLOC_MAX_NODES nodes (16 bytes each, 4 MiB) and one error
// word -- in file-scope __device__ arrays.  Every GPU that loads libmpm holds
// that memory until the process exits.
//
// Scratch rules: every call reuses the same arrays and finds there whatever
// the previous call left, so each call zeroes the grid nodes and the error
// word it uses before it runs.  Calls whose GPU work overlaps (on different
// streams, or from different host threads to the same device) race on the
// scratch and give wrong results; callers must serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/mpm.h"
#include "mpm_dev.cuh"
#include "mpm_math.cuh"
#include "mpm_ptr.h"

namespace {

using namespace mpm;

constexpr int MAX_NODES = MPM_NOALLOC_MAX_NODES;
constexpr int MAX_MATERIALS = MPM_NOALLOC_MAX_MATERIALS;

static __device__ __align__(256) float4 g_noalloc_grid[MAX_NODES];
static __device__ __align__(256) unsigned g_noalloc_err[64];

// device addresses of the scratch arrays, looked up once per device
struct Scratch {
    float4 *grid = nullptr;
    unsigned *err = nullptr;
};
constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
Scratch g_scratch[MAX_DEVICES];
bool g_ready[MAX_DEVICES] = {};

struct Params {
    int R[3];
    float dx, inv_dx, dt;
    float g[3];
    int bound;
    int wall[6];
    int n;
    int n_mat;
    float E[MAX_MATERIALS], nu[MAX_MATERIALS], rho[MAX_MATERIALS], yield[MAX_MATERIALS], alpha[MAX_MATERIALS];
    int elastic[MAX_MATERIALS], plastic[MAX_MATERIALS];
};

__device__ __forceinline__ bool locate(const Params &P, const float *x, int b[3], float f[3]) {
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float X = x[d] * P.inv_dx;
        float bb = floorf(X - 0.5f);
        f[d] = X - bb;
        b[d] = (int)bb;
        ok = ok && b[d] >= 0 && b[d] <= P.R[d] - 3;
    }
    return ok;
}

__global__ void k_na_clear(float4 *grid, unsigned *err, int nodes) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) err[0] = 0u;
    for (; i < nodes; i += gridDim.x * blockDim.x) grid[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// P2G with the stress of F (the momentum equation of §4.2), straight into the
// dense scratch grid with vector reductions
__global__ void k_na_p2g(Params P, float4 *grid, unsigned *err, const float *__restrict__ x,
                         const float *__restrict__ v, const float *__restrict__ C, const float *__restrict__ F,
                         const float *__restrict__ vol, const int *__restrict__ mat) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n) return;
    int m = mat[p];
    if (m < 0 || m >= P.n_mat) { atomicOr(err, ERRB_DOMAIN); return; }
    float xp[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
    int b[3];
    float f[3];
    if (!locate(P, xp, b, f)) { atomicOr(err, ERRB_DOMAIN); return; }
    float Fm[9], Cm[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) { Fm[i] = F[9 * p + i]; Cm[i] = C[9 * p + i]; }
    const float E = P.E[m], nu = P.nu[m];
    const float mu = E / (2.f * (1.f + nu)), lam = E * nu / ((1.f + nu) * (1.f - 2.f * nu));
    const float mass = P.rho[m] * vol[p];
    Sym tau;
    if (P.elastic[m] == 0) {
        float U[9], V[9], s[3], e[3], d[3];
        if (svd3_robust(Fm, U, V, s, e, d) == 2) atomicOr(err, ERRB_NONFINITE);
        tau = tau_fcr(U, s, e, mu, lam);
    } else if (!tau_nh(Fm, mu, lam, tau)) {
        atomicOr(err, ERRB_NONFINITE);
        tau = Sym{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    }
    const float kf = 4.f * P.dt * vol[p] * P.inv_dx * P.inv_dx;
    const float Ad[9] = {(mass * Cm[0] - kf * tau.xx) * P.dx, (mass * Cm[1] - kf * tau.xy) * P.dx,
                         (mass * Cm[2] - kf * tau.xz) * P.dx, (mass * Cm[3] - kf * tau.xy) * P.dx,
                         (mass * Cm[4] - kf * tau.yy) * P.dx, (mass * Cm[5] - kf * tau.yz) * P.dx,
                         (mass * Cm[6] - kf * tau.xz) * P.dx, (mass * Cm[7] - kf * tau.yz) * P.dx,
                         (mass * Cm[8] - kf * tau.zz) * P.dx};
    const float Pm[3] = {mass * v[3 * p], mass * v[3 * p + 1], mass * v[3 * p + 2]};
    float w0[3], w1[3], w2[3];
    bspline_w(f[0], w0);
    bspline_w(f[1], w1);
    bspline_w(f[2], w2);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                const float wt = w0[i] * w1[j] * w2[k];
                const float d0 = (float)i - f[0], d1 = (float)j - f[1], d2 = (float)k - f[2];
                const int node = ((b[0] + i) * P.R[1] + (b[1] + j)) * P.R[2] + (b[2] + k);
                red_add_v4(grid + node, wt * (Pm[0] + Ad[0] * d0 + Ad[1] * d1 + Ad[2] * d2),
                           wt * (Pm[1] + Ad[3] * d0 + Ad[4] * d1 + Ad[5] * d2),
                           wt * (Pm[2] + Ad[6] * d0 + Ad[7] * d1 + Ad[8] * d2), wt * mass);
            }
}

// grid update (App. A): v = mv/m + dt g, then the walls, in place
__global__ void k_na_update(Params P, float4 *grid, int nodes) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += gridDim.x * blockDim.x) {
        float4 a = grid[i];
        if (!(a.w > 0.f)) { grid[i] = make_float4(0.f, 0.f, 0.f, 0.f); continue; }
        const int K = i % P.R[2], J = (i / P.R[2]) % P.R[1], I = i / (P.R[1] * P.R[2]);
        const int idx[3] = {I, J, K};
        float u[3] = {a.x / a.w + P.dt * P.g[0], a.y / a.w + P.dt * P.g[1], a.z / a.w + P.dt * P.g[2]};
        bool sticky = false;
        for (int d = 0; d < 3; ++d) {
            if (idx[d] < P.bound && P.wall[2 * d] == 2) sticky = true;
            if (idx[d] >= P.R[d] - P.bound && P.wall[2 * d + 1] == 2) sticky = true;
        }
        for (int d = 0; d < 3; ++d) {
            if (sticky) u[d] = 0.f;
            if (idx[d] < P.bound && P.wall[2 * d] == 1 && u[d] < 0.f) u[d] = 0.f;
            if (idx[d] >= P.R[d] - P.bound && P.wall[2 * d + 1] == 1 && u[d] > 0.f) u[d] = 0.f;
        }
        grid[i] = make_float4(u[0], u[1], u[2], a.w);
    }
}

// G2P, advection, F update and return map (App. A; Algorithm 1, Stage 1)
__global__ void k_na_g2p(Params P, const float4 *grid, unsigned *err, const float *x, const float *F,
                         const int *__restrict__ mat, float *x_out, float *v_out, float *C_out, float *F_out) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n) return;
    int m = mat[p];
    if (m < 0 || m >= P.n_mat) return;
    float xp[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
    int b[3];
    float f[3];
    if (!locate(P, xp, b, f)) return;
    float Fm[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Fm[i] = F[9 * p + i];
    float w0[3], w1[3], w2[3];
    bspline_w(f[0], w0);
    bspline_w(f[1], w1);
    bspline_w(f[2], w2);
    float vn[3] = {0.f, 0.f, 0.f}, Bm[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                const float wt = w0[i] * w1[j] * w2[k];
                const float d[3] = {(float)i - f[0], (float)j - f[1], (float)k - f[2]};
                const float4 g = grid[((b[0] + i) * P.R[1] + (b[1] + j)) * P.R[2] + (b[2] + k)];
                const float a[3] = {wt * g.x, wt * g.y, wt * g.z};
                for (int r = 0; r < 3; ++r) {
                    vn[r] += a[r];
                    for (int c = 0; c < 3; ++c) Bm[3 * r + c] += a[r] * d[c];
                }
            }
    float Cn[9], G[9];
    for (int t = 0; t < 9; ++t) Cn[t] = 4.f * P.inv_dx * Bm[t];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            G[3 * r + c] = Fm[3 * r + c] + P.dt * (Cn[3 * r] * Fm[c] + Cn[3 * r + 1] * Fm[3 + c] + Cn[3 * r + 2] * Fm[6 + c]);
    const int plastic = P.plastic[m];
    if (plastic != PLASTIC_NONE) {
        const float E = P.E[m], nu = P.nu[m];
        const float mu = E / (2.f * (1.f + nu)), lam = E * nu / ((1.f + nu) * (1.f - 2.f * nu));
        float U[9], V[9], s[3], e[3], d[3], z[3], ze[3];
        if (svd3_robust(G, U, V, s, e, d) == 2) atomicOr(err, ERRB_NONFINITE);
        if (return_map(plastic, s, e, d, mu, lam, P.yield[m], P.alpha[m], z, ze) != RM_ELASTIC) usvt(G, U, z, V);
    }
    for (int r = 0; r < 3; ++r) {
        const float xn = xp[r] + P.dt * vn[r];
        if (!isfinite(xn)) atomicOr(err, ERRB_NONFINITE);
        x_out[3 * p + r] = xn;
        v_out[3 * p + r] = vn[r];
    }
    for (int t = 0; t < 9; ++t) { C_out[9 * p + t] = Cn[t]; F_out[9 * p + t] = G[t]; }
}

}  // namespace

extern "C" MPM_API mpm_status mpm_substep_noalloc(const int32_t grid_res[3], float dx, float dt, const float gravity[3],
                                                  const mpm_material *table, int32_t n_materials,
                                                  const mpm_options *opt, int64_t n, const float *x, const float *v,
                                                  const float *C, const float *F, const float *vol,
                                                  const int32_t *material_id, float *x_out, float *v_out,
                                                  float *C_out, float *F_out, void *stream) {
    if (!grid_res || !gravity || !table || !x || !v || !C || !F || !vol || !material_id || !x_out || !v_out ||
        !C_out || !F_out)
        return MPM_ERR_INVALID_ARG;
    if (n < 1 || n > (1ll << 31) - 1 || !(dx > 0.f) || !(dt > 0.f) || !std::isfinite(dx) || !std::isfinite(dt) ||
        n_materials < 1 || n_materials > MAX_MATERIALS)
        return MPM_ERR_INVALID_ARG;
    // the checks mpm_create makes on the same arguments, then the scratch
    // capacity, then the arrays: all before any GPU work
    mpm_options o;
    mpm_default_options(&o);
    if (opt) o = *opt;
    if (o.bound < 0) return MPM_ERR_INVALID_ARG;
    for (int i = 0; i < 6; ++i)
        if (o.walls[i] < MPM_WALL_OPEN || o.walls[i] > MPM_WALL_STICKY) return MPM_ERR_INVALID_ARG;
    for (int m = 0; m < n_materials; ++m) {
        const mpm_material &t = table[m];
        if (t.elastic < 0 || t.elastic > 1 || t.plastic < 0 || t.plastic > 2 || !(t.E > 0.f) || !(t.rho > 0.f) ||
            !(t.nu > -1.f && t.nu < 0.5f) || !std::isfinite(t.E) || !std::isfinite(t.rho) ||
            !std::isfinite(t.yield_stress) || !std::isfinite(t.friction_angle_deg))
            return MPM_ERR_INVALID_ARG;
    }
    long long nodes = 1;
    for (int d = 0; d < 3; ++d) {
        if (grid_res[d] < 4) return MPM_ERR_INVALID_ARG;
        nodes *= grid_res[d];
    }
    if (nodes > MAX_NODES) return MPM_ERR_CAPACITY;   // the scratch grid holds at most MAX_NODES nodes
    const void *arrays[] = {x, v, C, F, vol, material_id, x_out, v_out, C_out, F_out};
    for (const void *a : arrays)
        if (!on_this_device(a)) return MPM_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) { cudaGetLastError(); return MPM_ERR_CUDA; }
    {
        // once per device, with that device current: the device addresses of
        // the scratch arrays (host code cannot use the symbols themselves)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_ready[dev]) {
            Scratch s;
            if (cudaGetSymbolAddress((void **)&s.grid, g_noalloc_grid) != cudaSuccess ||
                cudaGetSymbolAddress((void **)&s.err, g_noalloc_err) != cudaSuccess) {
                cudaGetLastError();
                return MPM_ERR_CUDA;
            }
            g_scratch[dev] = s;
            g_ready[dev] = true;
        }
    }
    const Scratch sc = g_scratch[dev];

    Params P;
    for (int d = 0; d < 3; ++d) { P.R[d] = grid_res[d]; P.g[d] = gravity[d]; }
    P.dx = dx; P.inv_dx = 1.f / dx; P.dt = dt;
    P.bound = o.bound;
    for (int i = 0; i < 6; ++i) P.wall[i] = o.walls[i];
    P.n = (int)n;
    P.n_mat = n_materials;
    for (int m = 0; m < n_materials; ++m) {
        const mpm_material &t = table[m];
        P.E[m] = t.E; P.nu[m] = t.nu; P.rho[m] = t.rho; P.yield[m] = t.yield_stress;
        P.elastic[m] = t.elastic; P.plastic[m] = t.plastic;
        const double sphi = std::sin(t.friction_angle_deg * M_PI / 180.0);
        P.alpha[m] = (float)(std::sqrt(2.0 / 3.0) * 2.0 * sphi / (3.0 - sphi));
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nn = (int)nodes;
    const int pgrid = (int)((n + 255) / 256);
    const int ggrid = (nn + 255) / 256 < 4096 ? (nn + 255) / 256 : 4096;
    k_na_clear<<<ggrid, 256, 0, st>>>(sc.grid, sc.err, nn);
    k_na_p2g<<<pgrid, 256, 0, st>>>(P, sc.grid, sc.err, x, v, C, F, vol, material_id);
    k_na_update<<<ggrid, 256, 0, st>>>(P, sc.grid, nn);
    k_na_g2p<<<pgrid, 256, 0, st>>>(P, sc.grid, sc.err, x, F, material_id, x_out, v_out, C_out, F_out);
    if (cudaGetLastError() != cudaSuccess) return MPM_ERR_CUDA;
    unsigned err = 0;
    if (cudaMemcpyAsync(&err, sc.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return MPM_ERR_CUDA;
    }
    if (err & ERRB_DOMAIN) return MPM_ERR_OUT_OF_DOMAIN;
    if (err & ERRB_NONFINITE) return MPM_ERR_NONFINITE;
    return MPM_OK;
}
