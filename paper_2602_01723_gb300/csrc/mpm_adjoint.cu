// mpm_adjoint.cu -- recorded forward pass (checkpoints every ckpt_every
// substeps) and the reverse pass of the MLS-MPM substep.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "mpm_internal.h"

namespace mpm {

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
    a = AdjointStore();
}

static mpm_status save_checkpoint(mpm_ctx *ctx, size_t c, cudaStream_t st) {
    AdjointStore &A = ctx->adj;
    size_t bytes = (size_t)ctx->cap * REC_F4 * sizeof(float4);
    if (A.ckpt.size() <= c) A.ckpt.resize(c + 1, nullptr);
    if (!A.ckpt[c] || A.cap != ctx->cap) {
        if (A.ckpt[c]) cudaFree(A.ckpt[c]);
        cudaError_t e = cudaMalloc(&A.ckpt[c], bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            A.ckpt[c] = nullptr;
            return ctx_fail(ctx, MPM_ERR_OOM, "checkpoint allocation failed");
        }
    }
    cudaError_t e = cudaMemcpyAsync(A.ckpt[c], ctx->D.rec, (size_t)ctx->D.n * REC_F4 * sizeof(float4),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return ctx_fail(ctx, MPM_ERR_CUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
    return MPM_OK;
}

// forward with checkpoints at every ckpt_every-th recorded substep
mpm_status record_substeps(mpm_ctx *ctx, int n_sub, cudaStream_t st) {
    if (ctx->record_broken)
        return ctx_fail(ctx, MPM_ERR_STATE, "recording interrupted by an unrecorded step; call mpm_record_reset");
    const long long k = ctx->opt.ckpt_every;
    int remaining = n_sub;
    while (remaining > 0) {
        if (ctx->recorded % k == 0) {
            mpm_status s = save_checkpoint(ctx, (size_t)(ctx->recorded / k), st);
            if (s) return s;
        }
        int seg = (int)std::min<long long>(remaining, k - ctx->recorded % k);
        mpm_status s = run_substeps(ctx, seg, st);
        if (s) return s;
        ctx->recorded += seg;
        remaining -= seg;
    }
    ctx->adj.cap = ctx->cap;
    return MPM_OK;
}

}  // namespace mpm

extern "C" MPM_API mpm_status mpm_backward(mpm_ctx *ctx, int32_t n_frames, const int32_t *frame_substep,
                                           const float *dL_dx, float *dL_dparams, float *dL_dstate0, void *stream) {
    (void)n_frames; (void)frame_substep; (void)dL_dx; (void)dL_dparams; (void)dL_dstate0; (void)stream;
    if (!ctx) return MPM_ERR_INVALID_ARG;
    return mpm::ctx_fail(ctx, MPM_ERR_STATE, "reverse pass not built yet");
}
