// Host-buffer form of the whole evaluation: f_obj, its adjoint gradient and
// the marginal variances (diagonal of Sigma_c, Section III latent marginals)
// for callers whose thetas and results live in host memory.  The copies run
// on the context's stream around the device-pointer entry points; the call
// returns when the results are in host memory.

#include <algorithm>

#include "common.cuh"

namespace {

int stage_alloc(double** p, size_t elems) {
    if (*p) return BTA_OK;
    cudaError_t e = cudaMalloc((void**)p, elems * sizeof(double));
    if (e != cudaSuccess) {
        *p = nullptr;
        return bta_cuda_fail(e);
    }
    return BTA_OK;
}

}  // namespace

extern "C" int bta_fobj_grad_host(bta_ctx_t ctx, bta_model_t m, const double* thetas, int n_theta, double* f_out,
                                  double* grad_out, double* var_out) {
    if (!ctx || !m || !thetas || !f_out || !grad_out || n_theta < 1) return BTA_ERR_ARG;
    if (m->n != ctx->n || m->b != ctx->b || m->a != ctx->a || m->dim_theta < 1) return BTA_ERR_ARG;
    const int B = ctx->batch, dim = m->dim_theta;
    const long long N = ctx->N;
    if (ctx->hs_dim != 0 && ctx->hs_dim != dim) {
        // staging sized for another model: start over
        for (double** p : {&ctx->hs_theta, &ctx->hs_grad}) {
            cudaFree(*p);
            *p = nullptr;
        }
    }
    BTA_TRY(stage_alloc(&ctx->hs_theta, (size_t)B * dim));
    BTA_TRY(stage_alloc(&ctx->hs_f, (size_t)B));
    BTA_TRY(stage_alloc(&ctx->hs_grad, (size_t)B * dim));
    if (var_out) BTA_TRY(stage_alloc(&ctx->hs_var, (size_t)B * N));
    ctx->hs_dim = dim;
    cudaStream_t s = ctx->stream;
    for (int r0 = 0; r0 < n_theta; r0 += B) {
        const int cnt = std::min(B, n_theta - r0);
        BTA_CUDA_TRY(cudaMemcpyAsync(ctx->hs_theta, thetas + (long long)r0 * dim, (size_t)cnt * dim * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
        BTA_TRY(bta_fobj_grad(ctx, m, ctx->hs_theta, cnt, ctx->hs_f, ctx->hs_grad));
        if (var_out)
            for (int j = 0; j < cnt; ++j) BTA_TRY(bta_selinv_diag(ctx, 2 * j + BTA_QC, ctx->hs_var + j * N));
        BTA_CUDA_TRY(cudaMemcpyAsync(f_out + r0, ctx->hs_f, (size_t)cnt * sizeof(double), cudaMemcpyDeviceToHost, s));
        BTA_CUDA_TRY(cudaMemcpyAsync(grad_out + (long long)r0 * dim, ctx->hs_grad, (size_t)cnt * dim * sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
        if (var_out)
            BTA_CUDA_TRY(cudaMemcpyAsync(var_out + (long long)r0 * N, ctx->hs_var, (size_t)cnt * N * sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
    }
    return bta_sync(ctx);
}
