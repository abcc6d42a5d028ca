// The INLA objective f_obj(theta) of Eq. 8 for a Gaussian likelihood,
// evaluated at the conditional mean x = mu (Section III, approximation of the
// joint posterior), for a batch of hyperparameter vectors at once: the
// 2 dim(theta) + 1 points of the central-difference gradient (Eq. 10) are
// independent (Section IV-D.1), and so are Q_p and Q_c of each point
// (Section IV-D.2).  All 2 x batch BTA matrices go through the same kernel
// launches (one matrix per grid slice).
//
// Per theta: params = map(theta); Q_p and Q_c are assembled, factored and
// their log-determinants taken; then mu = Q_c^{-1} b, b = A^T D y (with FP64
// iterative refinement in mixed precision), and
//   f = log p(theta) + 1/2 log|Q_p| - 1/2 log|Q_c| - 1/2 (y^T D y - b^T mu)
//       + 1/2 sum_v m_v log tau_eps_v - (m/2) log 2 pi
// with y^T D y - b^T mu = (y - A mu)^T D (y - A mu) + mu^T Q_p mu.

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace {

// b_j[i] = tau_eps(variable of i) * (A^T y)[i], blockIdx.y = slot j
__global__ void fobj_rhs_kernel(const double* aty, const double* params, long long nb, int b, int ns, int nr,
                                long long N, double* rhs) {
    params += (long long)blockIdx.y * BTA_PSTRIDE;
    rhs += blockIdx.y * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = i < nb ? (int)((i % b) / ns) : (int)((i - nb) / nr);
        rhs[i] = params[5 * v + 4] * aty[i];
    }
}

// blockIdx.x = slot j
__global__ void fobj_final_kernel(const double* theta, const double* theta0, int dim, const double* params,
                                  const double* var_stats, int nv, double m_total, const double* ld_p,
                                  const double* ld_c, const double* dots, double* f_out) {
    const int j = blockIdx.x;
    theta += (long long)j * dim;
    params += (long long)j * BTA_PSTRIDE;
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
    const double btmu = dots[3 * j];
    f_out[j] = lp + 0.5 * ld_p[j] - 0.5 * ld_c[j] - 0.5 * (yDy - btmu) + 0.5 * logd - 0.5 * m_total * LOG_2PI;
}

}  // namespace

// One group of cnt thetas (at `theta`, cnt x dim) -> f (cnt values); mu of
// the group stays in the VEC_MU rows of the Q_c matrices.
static int fobj_group(bta_ctx_t ctx, bta_model_t m, const double* theta, int cnt, double* f, cudaStream_t s) {
    const int B = ctx->batch;
    const long long N = ctx->N, nb = (long long)ctx->n * ctx->b;
    BTA_TRY(prof_phase(ctx, 0, s));
    BTA_TRY(theta_to_params_impl(m, theta, cnt, ctx->params, s));
    if (cnt == B) {
        // all Q_p and Q_c of the batch in one pass
        BTA_TRY(assemble_impl(ctx, m, ctx->params, 0, 2 * B, s));
        BTA_TRY(prof_phase(ctx, 1, s));
        BTA_TRY(factor_impl(ctx, 0, 2 * B, s));
        BTA_TRY(logdet_impl(ctx, 0, 2 * B, ctx->ld, s));
    } else {
        for (int kind = 0; kind < 2; ++kind) BTA_TRY(assemble_impl(ctx, m, ctx->params, kind * B, cnt, s));
        BTA_TRY(prof_phase(ctx, 1, s));
        for (int kind = 0; kind < 2; ++kind) {
            BTA_TRY(factor_impl(ctx, kind * B, cnt, s));
            BTA_TRY(logdet_impl(ctx, kind * B, cnt, ctx->ld + kind * B, s));
        }
    }
    BTA_TRY(prof_phase(ctx, 2, s));
    double* rhs = vec_row(ctx, VEC_RHS, B);
    double* mu = vec_row(ctx, VEC_MU, B);
    {
        int blocks = (int)std::min<long long>((N + 255) / 256, 152 * 8 / cnt + 1);
        fobj_rhs_kernel<<<dim3(blocks, cnt), 256, 0, s>>>(m->aty, ctx->params, nb, ctx->b, m->ns,
                                                          m->nr > 0 ? m->nr : 1, N, rhs);
        BTA_LAUNCH_CHECK();
    }
    BTA_TRY(solve_impl(ctx, B, cnt, rhs, mu, s));
    // iterative refinement with an FP64 residual on the assembled blocks
    for (int it = 0; it < ctx->refine; ++it) {
        double* res = vec_row(ctx, VEC_RES, B);
        double* corr = vec_row(ctx, VEC_CORR, B);
        BTA_TRY(matvec_impl(ctx, B, cnt, mu, res, s));
        BTA_TRY(axpby64(s, cnt * N, 1.0, rhs, -1.0, res, res));
        BTA_TRY(solve_impl(ctx, B, cnt, res, corr, s));
        BTA_TRY(axpby64(s, cnt * N, 1.0, mu, 1.0, corr, mu));
    }
    BTA_TRY(dot_batch64(s, rhs, mu, N, cnt, ctx->red + (long long)B * ctx->red_chunks, ctx->red_chunks,
                        ctx->dots + 3 * B, 3));
    fobj_final_kernel<<<cnt, 1, 0, s>>>(theta, m->theta0, m->dim_theta, ctx->params, m->var_stats, m->nv,
                                        (double)m->m, ctx->ld, ctx->ld + B, ctx->dots + 3 * B, f);
    BTA_LAUNCH_CHECK();
    BTA_TRY(prof_phase(ctx, 3, s));
    return BTA_OK;
}

// Full groups replay a CUDA graph of fobj_group (captured on the second full
// group, so that every one-time set-up has happened outside the capture).  The
// graph is captured and launched on the context's private non-blocking stream,
// ordered after and before the caller's stream by events (the caller's stream
// may be the legacy default stream, which cannot be captured).
static int fobj_full_group_graph(bta_ctx_t ctx, bta_model_t m, cudaStream_t user) {
    cudaStream_t s = ctx->aux;
    BTA_CUDA_TRY(cudaEventRecord(ctx->ev_fork, user));
    BTA_CUDA_TRY(cudaStreamWaitEvent(s, ctx->ev_fork, 0));
    if (ctx->fobj_graph && ctx->graph_model != (const void*)m) {
        cudaGraphExecDestroy(ctx->fobj_graph);
        ctx->fobj_graph = nullptr;
    }
    if (!ctx->fobj_graph) {
        cudaGraph_t g = nullptr;
        // timing events (if profiling) then describe this graph's launches only
        ctx->prof_used = 0;
        ctx->prof_flops = 0.0;
        const long long l0 = bta_launch_count();
        BTA_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const int rc = fobj_group(ctx, m, ctx->theta_buf, ctx->batch, ctx->f_buf, s);
        const cudaError_t ce = cudaStreamEndCapture(s, &g);
        // captured launches run when the graph does, not now
        ctx->graph_kernels = bta_launch_count() - l0;
        bta_note_launches(-ctx->graph_kernels);
        if (rc != BTA_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        BTA_CUDA_TRY(ce);
        const cudaError_t ie = cudaGraphInstantiate(&ctx->fobj_graph, g, 0);
        cudaGraphDestroy(g);
        BTA_CUDA_TRY(ie);
        ctx->graph_model = m;
    }
    BTA_CUDA_TRY(cudaGraphLaunch(ctx->fobj_graph, s));
    bta_note_launches(ctx->graph_kernels);
    BTA_CUDA_TRY(cudaEventRecord(ctx->ev_join, s));
    BTA_CUDA_TRY(cudaStreamWaitEvent(user, ctx->ev_join, 0));
    return BTA_OK;
}

extern "C" int fobj_eval(bta_ctx_t ctx, bta_model_t m, const double* thetas_dev, int n_theta, double* f_out_dev,
                         double* mu_out_dev) {
    if (!ctx || !m || !thetas_dev || !f_out_dev || n_theta < 1) return BTA_ERR_ARG;
    if (m->n != ctx->n || m->b != ctx->b || m->a != ctx->a || m->nv > BTA_MAX_NV ||
        m->dim_theta > BTA_PSTRIDE)
        return BTA_ERR_ARG;
    cudaStream_t s = ctx->stream;
    const int B = ctx->batch;
    const long long N = ctx->N;
    for (int r0 = 0; r0 < n_theta; r0 += B) {
        const int cnt = std::min(B, n_theta - r0);
        const double* theta = thetas_dev + (long long)r0 * m->dim_theta;
        if (cnt == B && ctx->use_graph && ctx->graph_calls++ > 0) {
            BTA_CUDA_TRY(cudaMemcpyAsync(ctx->theta_buf, theta, (size_t)B * m->dim_theta * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s));
            BTA_TRY(fobj_full_group_graph(ctx, m, s));
            BTA_CUDA_TRY(cudaMemcpyAsync(f_out_dev + r0, ctx->f_buf, (size_t)B * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s));
            for (int mm = 0; mm < 2 * B; ++mm) ctx->factored[mm] = 1;
        } else {
            BTA_TRY(fobj_group(ctx, m, theta, cnt, f_out_dev + r0, s));
        }
        for (int j = 0; j < cnt; ++j) ctx->mu_valid[j] = 1;
        if (mu_out_dev)
            BTA_CUDA_TRY(cudaMemcpyAsync(mu_out_dev + (long long)r0 * N, vec_row(ctx, VEC_MU, B),
                                         cnt * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    return BTA_OK;
}

// Independent problems of any shapes: each on its own context's stream, all
// joined onto `join` by events (the evaluations of Section IV-D.1 need no
// common model; concurrency comes from the contexts' distinct streams).
extern "C" int bta_fobj_eval_multi(int count, const bta_ctx_t* ctxs, const bta_model_t* models,
                                   const double* const* thetas_dev, const int* n_theta, double* const* f_out_dev,
                                   double* const* mu_out_dev, double* const* grad_out_dev, void* join_stream) {
    if (count < 1 || !ctxs || !models || !thetas_dev || !n_theta || !f_out_dev) return BTA_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        const bta_ctx_t c = ctxs[i];
        const bta_model_t m = models[i];
        if (!c || !m || !thetas_dev[i] || !f_out_dev[i] || n_theta[i] < 1) return BTA_ERR_ARG;
        if (m->n != c->n || m->b != c->b || m->a != c->a) return BTA_ERR_ARG;
        if (grad_out_dev && grad_out_dev[i] && mu_out_dev && mu_out_dev[i]) return BTA_ERR_ARG;
    }
    cudaStream_t join = (cudaStream_t)join_stream;
    // inputs (thetas) and outputs may have been written or zeroed on `join`
    // just before the call: every distinct problem stream waits for that work
    {
        cudaEvent_t ev = nullptr;
        BTA_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, join);
        for (int i = 0; i < count && e == cudaSuccess; ++i) {
            bool seen = false;
            for (int k = 0; k < i; ++k) seen = seen || ctxs[k]->stream == ctxs[i]->stream;
            if (!seen) e = cudaStreamWaitEvent(ctxs[i]->stream, ev, 0);
        }
        cudaEventDestroy(ev);
        BTA_CUDA_TRY(e);
    }
    int rc = BTA_OK;
    int launched = 0;
    for (int i = 0; i < count && rc == BTA_OK; ++i) {
        double* g = grad_out_dev ? grad_out_dev[i] : nullptr;
        double* mu = mu_out_dev ? mu_out_dev[i] : nullptr;
        rc = g ? bta_fobj_grad(ctxs[i], models[i], thetas_dev[i], n_theta[i], f_out_dev[i], g)
               : fobj_eval(ctxs[i], models[i], thetas_dev[i], n_theta[i], f_out_dev[i], mu);
        launched = i + 1;   // a failed call may still have queued work
    }
    for (int i = 0; i < launched; ++i) {
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            e = cudaEventRecord(ev, ctxs[i]->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(join, ev, 0);
            cudaEventDestroy(ev);   // released once the recorded work has completed
        }
        if (e != cudaSuccess && rc == BTA_OK) rc = bta_cuda_fail(e);
    }
    return rc;
}
