/*
 * mpm.h -- C ABI of libmpm: the MLS-MPM substep (APIC transfers, quadratic
 * B-spline) of FastPhysGS (arXiv 2602.01723), its adjoint, and its batched
 * form, on one GPU (sm_103a).
 *
 * The method (what every entry point computes) is the substep of the paper's
 * Algorithm 1, Stage 1:
 *     tau <- Elasticity(F, E);  (x, v, C, F) <- MPMStep(x, v, C, F, tau);
 *     F <- Plasticity(F, E)
 * with MPMStep = P2G (the momentum-exchange equation of §4.2 with the MLS
 * stress term; App. A "Particle to Grid Transfer"), the grid update (App. A
 * "Grid Update": v = mv/m + dt g, then walls), and G2P (App. A "Grid to
 * Particle Transfer", with F <- (I + dt C) F).  Elasticity is fixed-corotated
 * (App. B.1) or Neo-Hookean (App. A, eq. neo_hookean); plasticity is none,
 * von Mises (App. A, eq. von_mises) or Drucker-Prager (App. A, eq.
 * drucker_prager); Lame parameters follow App. B.1.
 *
 * Conventions
 *  - Positions are in world units; grid node (I,J,K) sits at (I,J,K)*dx.  A
 *    particle must keep its 3x3x3 stencil on the grid: 0.5 dx <= x_d <
 *    (grid_res_d - 1.5) dx, otherwise MPM_ERR_OUT_OF_DOMAIN is raised.
 *  - Arrays are contiguous, row-major float32 / int32: x, v are n x 3; C, F
 *    are n x 9 (3x3 row-major).  Array pointers may be device pointers or
 *    host pointers (pinned or pageable): the library copies with
 *    cudaMemcpyDefault on the given stream.  The caller owns every array it
 *    passes; the library never keeps a caller pointer after a call returns.
 *  - Particle order is the caller's order in every input and output.
 *  - stream: a cudaStream_t, or NULL for the legacy default stream.  Calls
 *    enqueue work on it; they do not synchronise unless stated.
 *
 * Errors
 *  - Every entry point returns mpm_status; no C++ exception crosses the ABI.
 *  - Argument checks are synchronous.  Conditions found on the device
 *    (particle leaving the domain, non-finite state, J <= 0 under
 *    Neo-Hookean, grid pool exhausted, a particle moving more than one cell in
 *    a substep) set a sticky device error word; mpm_sync and every call that
 *    synchronises report it, after which the context stays in MPM_ERR_STATE
 *    until mpm_load_particles succeeds.
 *  - mpm_last_error gives a human-readable message for the last failure.
 */
#ifndef MPM_H
#define MPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MPM_API __attribute__((visibility("default")))
#else
#define MPM_API
#endif

typedef struct mpm_ctx mpm_ctx;   /* opaque, owned by the library */

typedef enum {
    MPM_OK = 0,
    MPM_ERR_INVALID_ARG = 1,
    MPM_ERR_OOM = 2,
    MPM_ERR_CUDA = 3,
    MPM_ERR_OUT_OF_DOMAIN = 4,
    MPM_ERR_NONFINITE = 5,
    MPM_ERR_TIMEOUT = 6,
    MPM_ERR_STATE = 7,
    MPM_ERR_CAPACITY = 8,   /* grid block pool or checkpoint budget exhausted */
    MPM_ERR_CFL = 9         /* a particle moved more than one grid cell in one substep */
} mpm_status;

enum { MPM_ELASTIC_FIXED_COROTATED = 0, MPM_ELASTIC_NEO_HOOKEAN = 1 };
enum { MPM_PLASTIC_NONE = 0, MPM_PLASTIC_VON_MISES = 1, MPM_PLASTIC_DRUCKER_PRAGER = 2 };
enum { MPM_WALL_OPEN = 0, MPM_WALL_SLIP = 1, MPM_WALL_STICKY = 2 };

/* One entry of the material table (§4.2: each object instance l_k carries
 * {rho, nu, Phi, E}).  E, nu give the Lame parameters (App. B.1);
 * yield_stress is the von Mises sigma_y; friction_angle_deg the
 * Drucker-Prager friction angle (alpha = sqrt(2/3) 2 sin phi / (3 - sin phi),
 * zero cohesion). */
typedef struct {
    int32_t elastic;            /* MPM_ELASTIC_* */
    int32_t plastic;            /* MPM_PLASTIC_* */
    float E, nu, rho, yield_stress, friction_angle_deg;
} mpm_material;

/* Options.  Fill with mpm_default_options, then override. */
typedef struct {
    int32_t n_instances;        /* independent problems, each on its own grid of grid_res (default 1) */
    int32_t bound;              /* wall band thickness in nodes (default 3) */
    int32_t walls[6];           /* faces x-, x+, y-, y+, z-, z+ (default: y- sticky, others slip) */
    int64_t max_particles;      /* particle capacity (default 0: set by the first load) */
    int64_t max_active_blocks;  /* capacity of the 4x4x4-node block pool per grid buffer (0: automatic) */
    int32_t ckpt_every;         /* checkpoint interval k of the recorded forward pass (default 20) */
    int32_t chunk;              /* particles per work item of the substep kernel, <= 128 (0: 128);
                                   chunks of <= 64 run 64-thread CTAs, larger ones 128-thread CTAs */
    int32_t scatter;            /* P2G scatter: 0 shared-memory float atomics, 1 int32 fixed-point
                                   shared-memory atomics (default), 2 direct global reductions */
    int32_t tape_grid;          /* reverse pass: 0 (default) keeps, for every state of a checkpoint
                                   segment, the records, binning and grid that the segment's
                                   recompute built, so that a reverse substep runs only its adjoint
                                   kernels; two banks of ckpt_every states, so that the recompute
                                   of the next segment overlaps the reverse of this one.  Device
                                   memory per state: 132 B per particle, 8 B per grid block, and
                                   2 KB per block of a grid pool sized at twice the active blocks
                                   (grown to the whole pool, and the pass rerun, if a state
                                   outgrows it).  1 keeps one bank of records only and rebuilds
                                   binning and grid in every reverse substep.  0 falls back to 1
                                   when its memory cannot be allocated. */
    int32_t reserved[7];        /* zero */
} mpm_options;

MPM_API mpm_status mpm_default_options(mpm_options *opt);

/* Creates a context on the current CUDA device.  grid_res: nodes per axis,
 * each a multiple of 4 and >= 8.  dx > 0, dt > 0.  gravity: 3 floats (host).
 * table: n_materials >= 1 entries (host), copied.  opt may be NULL. */
MPM_API mpm_status mpm_create(const int32_t grid_res[3], float dx, float dt, const float gravity[3],
                              const mpm_material *table, int32_t n_materials, const mpm_options *opt,
                              mpm_ctx **out);

/* Replaces the particle set.  x, vol, material_id are required; v (NULL: 0),
 * C (NULL: 0), F (NULL: I) optional; instance (n int32, NULL: all 0) selects
 * the grid of each particle; params (n x 3 float: log E, nu, yield stress;
 * NULL: from the material table) overrides the table per particle.  Particle
 * mass is rho * vol.  Also clears the recorded trajectory.  Synchronises the
 * stream and reports out-of-range inputs, except inside a stream capture (see
 * mpm_backward), where the arrays must be device arrays, n must fit the
 * capacity of an earlier load, and device errors surface at the next
 * synchronising call. */
MPM_API mpm_status mpm_load_particles(mpm_ctx *ctx, int64_t n, const float *x, const float *v, const float *C,
                                      const float *F, const float *vol, const int32_t *material_id,
                                      const int32_t *instance, const float *params, void *stream);

/* Advances n_substeps >= 0 substeps.  With record != 0 the state at every
 * ckpt_every-th substep counted from the last load (or mpm_record_reset) is
 * kept for mpm_backward; the recording must be contiguous (record on every
 * call since the last reset).  Does not synchronise.  Inside a stream capture
 * the substeps are launched into the caller's graph; a recorded run needs
 * the checkpoints of an earlier recorded run at least as long. */
MPM_API mpm_status mpm_step(mpm_ctx *ctx, int32_t n_substeps, int32_t record, void *stream);

/* Copies the current state out, in the caller's particle order; any pointer
 * may be NULL.  Enqueued on the stream; does not synchronise. */
MPM_API mpm_status mpm_get_particles(mpm_ctx *ctx, float *x, float *v, float *C, float *F, void *stream);

/* Reverse pass over the recorded substeps [0, S), S = substeps recorded.
 * frame_substep (host, n_frames ints in 1..S, any order) names the substep
 * after which frame f's positions were taken; dL_dx (n_frames x n x 3) is the
 * loss gradient with respect to those positions.  Writes dL_dparams (n x 3:
 * d/d log E, d/d nu, d/d yield stress, per particle; required) and, when not
 * NULL, dL_dstate0 (n x 24: the adjoint of the initial [x v C F]).  Recomputes
 * each checkpoint segment forward; the recorded state is left unchanged.
 * Synchronises the stream.
 *
 * Stream capture: a whole fwd+bwd (mpm_load_particles, mpm_step with record,
 * mpm_get_particles, mpm_backward, mpm_reduce_by_material) may be captured
 * into one CUDA graph by the caller.  Inside the capture nothing allocates
 * or synchronises: call the same sequence once outside it first (it sizes
 * the checkpoints, tapes and adjoint buffers); dL_dx and the outputs must be
 * device arrays and n_frames <= 64.  A recorded state whose grid outgrows
 * its tape slot, which outside a capture is rerun with larger slots, is then
 * reported as MPM_ERR_CAPACITY by the next mpm_sync.  Replays reuse the
 * host-side state of the capture: call nothing else on the context between
 * replays that changes it. */
MPM_API mpm_status mpm_backward(mpm_ctx *ctx, int32_t n_frames, const int32_t *frame_substep, const float *dL_dx,
                                float *dL_dparams, float *dL_dstate0, void *stream);

/* Drops the recorded trajectory; the next recorded substep is index 0. */
MPM_API mpm_status mpm_record_reset(mpm_ctx *ctx);

/* Waits for the context's work on the stream and reports the sticky device
 * error word. */
MPM_API mpm_status mpm_sync(mpm_ctx *ctx, void *stream);

/* Diagnostics copied to host (synchronises): counters[0] particles,
 * [1] occupied blocks, [2] active blocks of the last grid, [3] work chunks,
 * [4] FP64 SVD fallbacks so far, [5] substeps recorded, [6] device error
 * word, [7] grid pool capacity (blocks), [8] kernels launched by this
 * context so far, [9] grid-tape pool blocks per recorded state (0: no grid
 * tape), [10] reverse passes run again because a state's grid did not fit
 * its grid-tape slot, [11] particles the forward's direct binning placed in
 * one-particle work items since the last load (their block's list was full
 * or beyond the lists), [12] particles per block list and [13] block lists
 * of that binning (sized at each load); [14..15] zero. */
MPM_API mpm_status mpm_stats(mpm_ctx *ctx, int64_t counters[16], void *stream);

/* Tracing of the substep kernel.  When ms and count are not NULL, first
 * returns the summed device time (CUDA events recorded on the launching
 * stream around each launch) and the number of traced launches since the last
 * call, for the three variants: [0] first-substep scatter, [1] fused
 * gather + update + scatter, [2] last-substep gather; this waits for the
 * recorded events.  Then switches tracing on (enable != 0) or off and clears
 * the record. */
MPM_API mpm_status mpm_trace(mpm_ctx *ctx, int32_t enable, double ms[3], int64_t count[3]);

/* Segmented sum of a per-particle n x 3 device array (for example the
 * dL_dparams of mpm_backward) by material id into per_material
 * (n_materials x 3, device, overwritten): per-object or per-instance
 * gradients when each object or instance has its own table entry (§4.2: one
 * parameter set per instance label).  Enqueued on the stream. */
MPM_API mpm_status mpm_reduce_by_material(mpm_ctx *ctx, const float *per_particle, float *per_material,
                                          void *stream);

/* Sets the substep kernel's tuning: scatter strategy (0, 1, 2 as in
 * mpm_options), particles per work chunk (a multiple of 16 in [16, 128]) and
 * whether steady-state substeps replay a CUDA graph (two substeps per graph
 * launch; tracing disables the graph). */
MPM_API mpm_status mpm_set_tuning(mpm_ctx *ctx, int32_t scatter, int32_t chunk, int32_t use_graph);

/* Autotuner: times n_substeps >= 2 substeps from the current state for each
 * scatter strategy in {1, 2} and chunk size in {32, 64, 96, 128} (each
 * trial after a warm-up run), keeps the fastest, and restores the state.  The
 * grid tile (4x4x4-node blocks) is fixed by the data layout.  out
 * (nullable, host): chosen scatter, chosen chunk, best time in microseconds.
 * Synchronises the stream. */
MPM_API mpm_status mpm_autotune(mpm_ctx *ctx, int32_t n_substeps, int32_t out[3], void *stream);

/* ---------------------------------------------------------------------------
 * BGDO (§4.3 "Optimization Algorithm"; Algorithm 1, Stage 2; App. F)
 *
 * Stage 1 is the ordinary forward (mpm_step) with key-frame snapshots taken
 * by mpm_snapshot.  Stage 2 (mpm_bgdo) runs, from every key frame k, one
 * pseudo substep with the current parameters and accumulates per particle p
 *     g_tau = d |tau_p|_F / d log E_p   (= |tau_p|_F: tau is linear in the
 *                                         Lame parameters, App. B.1)
 *     delta = |F'_p - I|_F              (F' after the pseudo substep and the
 *                                         return map, App. F.2)
 *     eta   = min(1, 0.1 log(1 + E_p))  (§4.3, eq. eq_target) or a fixed w
 *     G_p  += (eta log(1 + |g_tau|) - (1 - eta)(delta - delta_target)) / K
 * and the update log E_p <- log E_p - G_p (App. F.3).
 * ------------------------------------------------------------------------ */
#define MPM_MAX_SNAPSHOTS 8

/* Copies the current state of every particle, with its mass, volume and
 * material parameters, into key-frame slot 0 <= slot < MPM_MAX_SNAPSHOTS
 * (library-owned device memory, 128 bytes per particle, allocated on first
 * use of the slot).  A slot can be used by mpm_bgdo while the particle count
 * equals the count at the snapshot; the pseudo substep then uses the
 * parameters stored with the snapshot.  Enqueued on the stream. */
MPM_API mpm_status mpm_snapshot(mpm_ctx *ctx, int32_t slot, void *stream);

typedef struct {
    float delta_target;      /* deformation target (App. F.2); default 0.1 */
    float w;                 /* < 0: eta = min(1, 0.1 log(1 + E)) per particle (default -1);
                                in [0, 1]: the fixed balancing weight w of Algorithm 1 */
    int32_t per_material;    /* 1: G averaged over the particles of each material id */
    int32_t delta_pre_step;  /* 1: delta from the key frame's own F (the d_F of §4.3)
                                instead of the post-step F' (no pseudo substep runs) */
    int32_t reserved[4];     /* zero */
} mpm_bgdo_options;

MPM_API mpm_status mpm_bgdo_default_options(mpm_bgdo_options *opt);

/* BGDO stage 2 over n_keys (1..MPM_MAX_SNAPSHOTS) key-frame slots (host
 * array).  opt may be NULL (defaults).  Outputs, each nullable, in the
 * caller's particle order, host or device: G (n), log_E (n: log E_p - G_p
 * with E_p the current particle's modulus, the updated parameter to load for
 * the next iteration), g_tau and delta (n_keys x n, the per-key signals).
 * The current state and the recorded trajectory are left unchanged.
 * Synchronises the stream when an output is a host pointer.  MPM_ERR_STATE
 * when a slot is empty or was taken with another particle count. */
MPM_API mpm_status mpm_bgdo(mpm_ctx *ctx, int32_t n_keys, const int32_t *slots, const mpm_bgdo_options *opt,
                            float *G, float *log_E, float *g_tau, float *delta, void *stream);

/* ---------------------------------------------------------------------------
 * Gaussian kernels (§3.1: each splat is a Gaussian with covariance
 * Sigma = R S S^T R^T; §3.2: it deforms with its particle,
 * Sigma(t) = F(t) Sigma F(t)^T).  Covariances are symmetric 3x3 stored as
 * n x 6 floats: xx xy xz yy yz zz, in the caller's particle order.
 * ------------------------------------------------------------------------ */

/* Sets the rest covariance Sigma of every currently loaded particle (n x 6,
 * host or device; copied).  Valid while the particle count is unchanged.
 * Enqueued on the stream. */
MPM_API mpm_status mpm_load_covariance(mpm_ctx *ctx, const float *cov0, void *stream);

/* Writes F Sigma F^T of every particle's current F into cov (n x 6, host or
 * device).  MPM_ERR_STATE when no rest covariances match the particle count.
 * Enqueued on the stream; does not synchronise. */
MPM_API mpm_status mpm_get_covariance(mpm_ctx *ctx, float *cov, void *stream);

/* ---------------------------------------------------------------------------
 * MCIS interior fill sampling (§4.1 "Monte Carlo Importance Sampling",
 * steps 1-4).  Independent of any context.  Object k owns surface points
 * surf[surf_off[k] .. surf_off[k+1]) (its cluster C_k), candidate points
 * cand[cand_off[k] .. cand_off[k+1]) (Q_k, already inside the object) and
 * draws draw_off[k] .. draw_off[k+1]:
 *     d_j = min_{c in C_k} |q_j - c|                       (step 1)
 *     w_j = max(exp(-d_j^2 / (2 sigma^2)), eps)            (step 2; the paper
 *                                                            uses sigma 0.02, eps 1e-6)
 *     p_j = w_j / sum w                                    (step 3)
 *     draw i: P(candidate j) = p_j, independent draws       (step 4)
 * Draw i takes the uniform u[i] in [0, 1) and returns the global index of
 * the first candidate of its object whose cumulative weight exceeds
 * floor(u_i W_k), the weights summed as integers floor(w 2^40 + 1/2).
 * Distances are exact (FP64) up to d_cut = sigma sqrt(2 ln(1/eps)); beyond
 * it the weight is eps and d may be larger than the true distance (INFINITY
 * when nothing lies within d_cut).  Coordinates are expected in the unit
 * cube (App. C.1).  Offsets are host arrays of n_obj + 1 int64 starting at
 * 0; surf, cand (n x 3 float), u (double) and the outputs d, w (n_cand
 * double, nullable) and picked (n_draw int64; -1 for an object without
 * candidates) may be host or device.  Synchronises the stream.  The message
 * of a failure is mpm_mcis_last_error().
 * ------------------------------------------------------------------------ */
MPM_API mpm_status mpm_mcis(int32_t n_obj, const int64_t *surf_off, const float *surf, const int64_t *cand_off,
                            const float *cand, const int64_t *draw_off, const double *u, double sigma, double eps,
                            double *d, double *w, int64_t *picked, void *stream);
MPM_API const char *mpm_mcis_last_error(void);

/* Splatting of Gaussian kernels into a headless image (§3.1): Gaussian i
 * has mean mean[i] (n x 3), covariance cov[i] (n x 6: xx xy xz yy yz zz,
 * e.g. from mpm_get_covariance), colour color[i] (n x 3) and opacity
 * opacity[i]; it projects to Sigma' = J W Sigma W^T J^T, dilated by 0.3
 * (pixel low-pass), and pixels composite front to back,
 *     Col = sum_i col_i alpha_i prod_{j<i} (1 - alpha_j) + T bg,
 *     alpha_i = min(0.99, o_i exp(-1/2 d^T Sigma'^{-1} d)).
 * Conventions of the 3DGS renderer the paper cites: Gaussians nearer than
 * 0.2 are not drawn; each touches the 16x16 tiles of its 3-sigma square;
 * alpha below 1/255 is skipped; a pixel stops once its transmittance would
 * fall below 1e-4; equal depths keep the input order.  view (host, 12
 * floats) is the row-major 3x4 world-to-camera transform [R | T]; pixel
 * (x, y) has centre (x + 1/2, y + 1/2) and sees u = fx t_x / t_z + cx,
 * v = fy t_y / t_z + cy.  bg: 3 floats (host).  image (height x width x 3)
 * and trans (height x width, nullable: final transmittance) may be host or
 * device; the inputs too.  Synchronises the stream; the message of a failure
 * is mpm_render_last_error(). */
MPM_API mpm_status mpm_render(int64_t n, const float *mean, const float *cov, const float *color,
                              const float *opacity, const float view[12], float fx, float fy, float cx, float cy,
                              int32_t width, int32_t height, const float bg[3], float *image, float *trans,
                              void *stream);
MPM_API const char *mpm_render_last_error(void);

/* Diagnostic: P2G of the current state into dense device arrays m
 * (n_instances * R0 * R1 * R2 floats, node (b, I, J, K) at
 * ((b * R0 + I) * R1 + J) * R2 + K) and mv (3 floats per node); the particle
 * state is left unchanged.  Synchronises the stream. */
MPM_API mpm_status mpm_debug_p2g(mpm_ctx *ctx, float *m, float *mv, void *stream);

/* ---------------------------------------------------------------------------
 * mpm_substep_noalloc -- one substep without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc.  Examples are an application whose device memory
 * is fixed at start-up, code running while another allocator owns the
 * device's memory, and latency-critical paths that cannot take the implicit
 * device synchronisation of cudaMalloc / cudaFree.  It advances n particles by
 * one substep (the same P2G with stress, grid update with walls, and G2P with
 * the return map as mpm_step) on a dense grid of grid_res nodes, without a
 * context.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Scratch: the grid lives in a file-scope device array of
 * MPM_NOALLOC_MAX_NODES nodes (16 bytes each, 4 MiB), plus one error word;
 * every GPU that loads libmpm holds this memory until the process exits.
 * grid_res[0] * grid_res[1] * grid_res[2] above MPM_NOALLOC_MAX_NODES returns
 * MPM_ERR_CAPACITY before any GPU work; more than MPM_NOALLOC_MAX_MATERIALS
 * table entries return MPM_ERR_INVALID_ARG.
 *
 * Every call shares that scratch and finds the previous call's contents in
 * it; each call clears the nodes and the error word it uses.  Calls whose GPU
 * work overlaps (different streams, or different host threads on one device)
 * race on the scratch: serialise them.
 *
 * Set-up: the first call on a device, with that device current, looks up
 * the scratch's device address for that device (host code cannot use the
 * array's symbol directly) and keeps it for the life of the process; make
 * that first call before any stream capture begins.  The kept address is not
 * looked up again, so do not call this entry point after cudaDeviceReset.
 *
 * Arguments: grid_res, dx, dt, gravity, table, n_materials as in mpm_create
 * (table on the host), checked as mpm_create checks them (nu in (-1, 0.5),
 * E, rho > 0) but with elastic models 0..1 and plastic models 0..2 only;
 * opt (nullable) supplies bound (>= 0) and walls (MPM_WALL_*).  x, v (n x 3),
 * C, F (n x 9), vol (n), material_id (n) are arrays on the current device;
 * the outputs x_out, v_out (n x 3), C_out, F_out (n x 9) are arrays on the
 * current device and may alias the inputs.  Per-particle parameters come from
 * the table only.  Every argument is checked before any GPU work:
 * MPM_ERR_INVALID_ARG for a bad argument, a NULL or host pointer or one on
 * another device, MPM_ERR_CAPACITY for a grid beyond the scratch.  Each call
 * synchronises the stream before it returns, to read the error word: then
 * MPM_ERR_OUT_OF_DOMAIN when a particle's stencil leaves the grid or a
 * material id is out of range, MPM_ERR_NONFINITE on a non-finite result.
 * ------------------------------------------------------------------------- */
#define MPM_NOALLOC_MAX_NODES 262144      /* 64^3 */
#define MPM_NOALLOC_MAX_MATERIALS 16
MPM_API mpm_status mpm_substep_noalloc(const int32_t grid_res[3], float dx, float dt, const float gravity[3],
                                       const mpm_material *table, int32_t n_materials, const mpm_options *opt,
                                       int64_t n, const float *x, const float *v, const float *C, const float *F,
                                       const float *vol, const int32_t *material_id, float *x_out, float *v_out,
                                       float *C_out, float *F_out, void *stream);

/* Last error message of this context (or of the last failed mpm_create when
 * ctx is NULL).  Static storage owned by the library. */
MPM_API const char *mpm_last_error(const mpm_ctx *ctx);

/* Frees every device buffer of the context; NULL-safe. */
MPM_API mpm_status mpm_destroy(mpm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MPM_H */
