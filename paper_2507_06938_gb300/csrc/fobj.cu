// The INLA objective f_obj(theta) of Eq. 8 for a Gaussian likelihood,
// evaluated at the conditional mean x = mu (Section III, approximation of the
// joint posterior; Section IV-D.2 for the two independent factorisations).
//
// Per theta: params = map(theta); Q_p is assembled, factored and its
// log-determinant taken on the auxiliary stream while Q_c is assembled and
// factored on the main stream; then mu = Q_c^{-1} b, b = A^T D y, and
//   f = log p(theta) + 1/2 log|Q_p| - 1/2 log|Q_c| - 1/2 (y^T D y - b^T mu)
//       + 1/2 sum_v m_v log tau_eps_v - (m/2) log 2 pi
// with y^T D y - b^T mu = (y - A mu)^T D (y - A mu) + mu^T Q_p mu.

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace {

// b[i] = tau_eps(variable of i) * (A^T y)[i]
__global__ void fobj_rhs_kernel(const double* aty, const double* params, long long nb, int b, int ns, int nr,
                                long long N, double* rhs) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = i < nb ? (int)((i % b) / ns) : (int)((i - nb) / nr);
        rhs[i] = params[5 * v + 4] * aty[i];
    }
}

__global__ void fobj_final_kernel(const double* theta, const double* theta0, int dim, const double* params,
                                  const double* var_stats, int nv, double m_total, const double* scal,
                                  double* f_out) {
    const double LOG_2PI = 1.8378770664093453;
    double lp = 0.0;
    for (int i = 0; i < dim; ++i) {
        const double d = theta[i] - theta0[i];
        lp += -0.5 * d * d;
    }
    lp -= 0.5 * dim * LOG_2PI;
    double yDy = 0.0, logd = 0.0;
    for (int v = 0; v < nv; ++v) {
        const double te = params[5 * v + 4];
        yDy += te * var_stats[v];
        logd += var_stats[nv + v] * log(te);
    }
    const double ld_p = scal[SCAL_LOGDET_P], ld_c = scal[SCAL_LOGDET_C], btmu = scal[SCAL_DOT];
    *f_out = lp + 0.5 * ld_p - 0.5 * ld_c - 0.5 * (yDy - btmu) + 0.5 * logd - 0.5 * m_total * LOG_2PI;
}

}  // namespace

extern "C" int fobj_eval(bta_ctx_t ctx, bta_model_t m, const double* thetas_dev, int n_theta, double* f_out_dev,
                         double* mu_out_dev) {
    if (!ctx || !m || !thetas_dev || !f_out_dev || n_theta < 1) return BTA_ERR_ARG;
    if (m->n != ctx->n || m->b != ctx->b || m->a != ctx->a) return BTA_ERR_ARG;
    cudaStream_t s = ctx->stream, aux = ctx->aux;
    const long long N = ctx->N, nb = (long long)ctx->n * ctx->b;
    double* rhs = ctx->vec + 7 * N;
    double* mu = ctx->vec + 8 * N;
    for (int j = 0; j < n_theta; ++j) {
        const double* theta = thetas_dev + (long long)j * m->dim_theta;
        BTA_TRY(theta_to_params_impl(m, theta, ctx->params, s));
        // fork: Q_p on the auxiliary stream
        BTA_CUDA_TRY(cudaEventRecord(ctx->ev_fork, s));
        BTA_CUDA_TRY(cudaStreamWaitEvent(aux, ctx->ev_fork, 0));
        BTA_TRY(assemble_impl(ctx, m, ctx->params, BTA_QP, aux));
        BTA_TRY(factor_impl(ctx, BTA_QP, aux));
        BTA_TRY(logdet_impl(ctx, BTA_QP, ctx->scal + SCAL_LOGDET_P, aux));
        // Q_c, its log-determinant and the conditional mean on the main stream
        BTA_TRY(assemble_impl(ctx, m, ctx->params, BTA_QC, s));
        BTA_TRY(factor_impl(ctx, BTA_QC, s));
        BTA_TRY(logdet_impl(ctx, BTA_QC, ctx->scal + SCAL_LOGDET_C, s));
        {
            int blocks = (int)std::min<long long>((N + 255) / 256, 152 * 8);
            fobj_rhs_kernel<<<blocks, 256, 0, s>>>(m->aty, ctx->params, nb, ctx->b, m->ns, m->nr > 0 ? m->nr : 1,
                                                  N, rhs);
            BTA_LAUNCH_CHECK();
        }
        BTA_TRY(solve_impl(ctx, BTA_QC, rhs, mu, s));
        // iterative refinement with an FP64 residual on the assembled blocks
        for (int it = 0; it < ctx->refine; ++it) {
            double* res = ctx->vec + N;
            double* corr = ctx->vec + 2 * N;
            BTA_TRY(matvec_impl(ctx, BTA_QC, mu, res, s));
            BTA_TRY(axpby64(s, N, 1.0, rhs, -1.0, res, res));
            BTA_TRY(solve_impl(ctx, BTA_QC, res, corr, s));
            BTA_TRY(axpby64(s, N, 1.0, mu, 1.0, corr, mu));
        }
        BTA_TRY(dot64(s, rhs, mu, N, ctx->red + ctx->red_len / 2, ctx->red_len / 2, ctx->scal + SCAL_DOT));
        // join
        BTA_CUDA_TRY(cudaEventRecord(ctx->ev_join, aux));
        BTA_CUDA_TRY(cudaStreamWaitEvent(s, ctx->ev_join, 0));
        fobj_final_kernel<<<1, 1, 0, s>>>(theta, m->theta0, m->dim_theta, ctx->params, m->var_stats, m->nv,
                                          (double)m->m, ctx->scal, f_out_dev + j);
        BTA_LAUNCH_CHECK();
    }
    if (mu_out_dev)
        BTA_CUDA_TRY(cudaMemcpyAsync(mu_out_dev, mu, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return BTA_OK;
}
