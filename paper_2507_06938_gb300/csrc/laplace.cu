// The INLA objective for non-Gaussian likelihoods: the Laplace approximation
// at the mode x* of the latent field (Section II-A.3 and Eqs. 4, 7, 8).
//
// p_G is built from the GMRF prior and a second-order Taylor expansion of the
// log-likelihood ell around x: Q_c(x) = Q_p + A^T D(x) A with D the negative
// Hessian of ell with respect to the linear predictor eta = A x (Eq. 4).  The
// mode comes from Newton's method: with g = d ell / d eta and D at
// eta_k = A x_k, the next iterate is the mean of that Gaussian,
//   Q_c(x_k) x_{k+1} = A^T (g + D eta_k),
// so every Newton step is one assembly of Q_c with per-observation weights,
// one BTA factorisation and one solve -- the hot path of the Gaussian case
// run newton_iters times.  At x* the quadratic form of p_G vanishes and the
// -N/2 log 2 pi terms of Eqs. 1 and 3 cancel:
//   f = log p(theta) + ell(y | x*) + 1/2 log|Q_p| - 1/2 x*^T Q_p x* - 1/2 log|Q_c(x*)|.
// Likelihoods (independent observations):
//   BTA_LIK_POISSON  (log link): ell = y eta - exp(eta) - log y!, g = y - exp(eta), D = exp(eta)
//   BTA_LIK_GAUSSIAN (noise precision d_v of the observation's variable):
//                    ell = 1/2 log d - 1/2 log 2 pi - 1/2 d (y - eta)^2, g = d (y - eta), D = d
// (for the Gaussian the Taylor expansion is exact and one step reaches mu).

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace {

constexpr int LAP_THREADS = 256;

struct LapObs {
    int m, nv, ns, nr, b;
    long long N, nb;
    const int* tv;
    const int* s;
    const double* w;
    const int* gpos;
    const double* X;
    const double* y;
};

// Per (observation k, slot blockIdx.y): eta_k = (A x)_k, then the curvature
// d_k = D_kk, the Newton right-hand-side term c_k = g_k + d_k eta_k and the
// log-likelihood term ell_k.
__global__ void lap_eta_lik_kernel(LapObs o, int lik, const double* x, long long xs, const double* params,
                                   double* dvec, double* cvec, double* ell, long long os) {
    const int j = blockIdx.y;
    x += j * xs;
    params += (long long)j * BTA_PSTRIDE;
    dvec += j * os;
    cvec += j * os;
    ell += j * os;
    const double LOG_2PI = 1.8378770664093453;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < o.m; k += gridDim.x * blockDim.x) {
        const int tv = o.tv[k], t = tv / o.nv, v = tv % o.nv;
        const long long base = (long long)t * o.b + (long long)v * o.ns;
        double eta = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q) eta += o.w[3 * k + q] * x[base + o.s[3 * k + q]];
        for (int r = 0; r < o.nr; ++r) eta += o.X[(long long)k * o.nr + r] * x[o.nb + v * o.nr + r];
        const double y = o.y[k];
        double d, g, l;
        if (lik == BTA_LIK_POISSON) {
            const double e = exp(eta);
            d = e;
            g = y - e;
            l = y * eta - e - lgamma(y + 1.0);
        } else {
            const double tau = params[5 * v + 4];
            const double r = y - eta;
            d = tau;
            g = tau * r;
            l = 0.5 * log(tau) - 0.5 * LOG_2PI - 0.5 * tau * r * r;
        }
        dvec[k] = d;
        cvec[k] = g + d * eta;
        ell[k] = l;
    }
}

// Scatter of the weighted observation terms of Q_c (Gram, arrow and tip parts
// in the model's layouts) and of the Newton right-hand side A^T c.  The tip
// and fixed-effect entries, shared by all observations, are summed in shared
// memory first (one global atomic per entry and CTA).
__global__ void lap_scatter_kernel(LapObs o, const double* dvec, const double* cvec, long long os, double* gram,
                                   long long gstride, double* arrow, long long astride, double* tip,
                                   long long tstride, double* rhs, long long rs) {
    extern __shared__ double sh[];   // nv nr nr tip entries, then nv nr fixed-effect rhs entries
    const int j = blockIdx.y;
    dvec += j * os;
    cvec += j * os;
    gram += j * gstride;
    arrow += j * astride;
    tip += j * tstride;
    rhs += j * rs;
    const int ntip = o.nv * o.nr * o.nr, nfe = o.nv * o.nr;
    for (int e = threadIdx.x; e < ntip + nfe; e += blockDim.x) sh[e] = 0.0;
    __syncthreads();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < o.m; k += gridDim.x * blockDim.x) {
        const double d = dvec[k], c = cvec[k];
        const int tv = o.tv[k], t = tv / o.nv, v = tv % o.nv;
        const long long base = (long long)t * o.b + (long long)v * o.ns;
        double w[3];
        int s[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            w[q] = o.w[3 * k + q];
            s[q] = o.s[3 * k + q];
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
#pragma unroll
            for (int r = 0; r < 3; ++r) atomicAdd(&gram[o.gpos[9 * k + 3 * q + r]], d * w[q] * w[r]);
            atomicAdd(&rhs[base + s[q]], c * w[q]);
        }
        for (int r = 0; r < o.nr; ++r) {
            const double xr = o.X[(long long)k * o.nr + r];
            for (int q = 0; q < 3; ++q)
                atomicAdd(&arrow[((long long)tv * o.nr + r) * o.ns + s[q]], d * xr * w[q]);
            for (int r2 = 0; r2 < o.nr; ++r2)
                atomicAdd(&sh[(v * o.nr + r) * o.nr + r2], d * xr * o.X[(long long)k * o.nr + r2]);
            atomicAdd(&sh[ntip + v * o.nr + r], c * xr);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ntip; e += blockDim.x)
        if (sh[e] != 0.0) atomicAdd(&tip[e], sh[e]);
    for (int e = threadIdx.x; e < nfe; e += blockDim.x)
        if (sh[ntip + e] != 0.0) atomicAdd(&rhs[o.nb + e], sh[ntip + e]);
}

// Parameter slots for the weighted assembly: the observation weights carry
// D, so the noise-precision entries become 1.
__global__ void lap_params_kernel(const double* params, int nv, double* out) {
    const double* p = params + (long long)blockIdx.x * BTA_PSTRIDE;
    double* q = out + (long long)blockIdx.x * BTA_PSTRIDE;
    for (int i = threadIdx.x; i < BTA_PSTRIDE; i += blockDim.x) q[i] = (i < 5 * nv && i % 5 == 4) ? 1.0 : p[i];
}

// step[j] = max_i |xn_j[i] - x_j[i]|, then x_j = xn_j (one CTA per slot)
__global__ void lap_step_kernel(const double* xn, double* x, long long N, double* step) {
    __shared__ double red[LAP_THREADS];
    const int j = blockIdx.x;
    xn += j * N;
    x += j * N;
    double mx = 0.0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        mx = fmax(mx, fabs(xn[i] - x[i]));
        x[i] = xn[i];
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) step[j] = red[0];
}

__global__ void fill_kernel(double* x, long long n, double v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

// f_j = log p(theta_j) + ell_j + 1/2 log|Q_p| - 1/2 x*^T Q_p x* - 1/2 log|Q_c(x*)|
__global__ void lap_final_kernel(const double* theta, const double* theta0, int dim, const double* ell,
                                 const double* quad, const double* ld_p, const double* ld_c, double* f) {
    const int j = blockIdx.x;
    theta += (long long)j * dim;
    double lp = 0.0;
    for (int i = 0; i < dim; ++i) {
        const double d = theta[i] - theta0[i];
        lp += -0.5 * d * d;
    }
    lp -= 0.5 * dim * 1.8378770664093453;
    f[j] = lp + ell[3 * j] + 0.5 * ld_p[j] - 0.5 * quad[3 * j] - 0.5 * ld_c[j];
}

}  // namespace

extern "C" int bta_fobj_laplace(bta_ctx_t ctx, bta_model_t m, const double* thetas_dev, int n_theta, int likelihood,
                                int newton_iters, double* f_out_dev, double* x_out_dev, double* step_out_dev) {
    if (!ctx || !m || !thetas_dev || !f_out_dev || n_theta < 1 || newton_iters < 1 || newton_iters > 1000)
        return BTA_ERR_ARG;
    if (likelihood != BTA_LIK_GAUSSIAN && likelihood != BTA_LIK_POISSON) return BTA_ERR_ARG;
    if (m->n != ctx->n || m->b != ctx->b || m->a != ctx->a || m->nv > BTA_MAX_NV || m->dim_theta > BTA_PSTRIDE)
        return BTA_ERR_ARG;
    const int ntip = m->nv * m->nr * m->nr, nfe = m->nv * m->nr;
    const size_t scatter_smem = (size_t)(ntip + nfe) * sizeof(double);
    if (scatter_smem > 48 * 1024) return BTA_ERR_ARG;
    cudaStream_t s = ctx->stream;
    const int B = ctx->batch;
    const long long N = ctx->N, nb = (long long)ctx->n * ctx->b;
    const long long gsz = (long long)m->nt * m->nv * m->nnz, asz = (long long)m->nt * m->nv * m->nr * m->ns;
    const long long msz = std::max(1, m->m);
    // per slot: gram | arrow | tip | d | c | ell; then x_new (B x N), tmp (B x N),
    // params (B x PSTRIDE), ones (m), scalars (3 B), step (B)
    const long long per = gsz + asz + ntip + 3 * msz;
    const size_t tail = 2 * (size_t)B * N + (size_t)B * BTA_PSTRIDE;
    if (!ctx->lap || ctx->lap_model != (const void*)m) {
        if (ctx->lap) cudaFree(ctx->lap);
        ctx->lap = nullptr;
        const size_t total = (size_t)B * per + tail + msz + 4 * (size_t)B;
        cudaError_t e = cudaMalloc((void**)&ctx->lap, total * sizeof(double));
        if (e != cudaSuccess) {
            ctx->lap = nullptr;
            return bta_cuda_fail(e);
        }
        ctx->lap_slot = per;
        ctx->lap_model = m;
        double* ones = ctx->lap + (size_t)B * per + tail;
        fill_kernel<<<(int)std::min<long long>((msz + 255) / 256, 1216), 256, 0, s>>>(ones, msz, 1.0);
        BTA_LAUNCH_CHECK();
    }
    double* W = ctx->lap;
    double* gram = W;
    double* arrow = W + gsz;
    double* tip = arrow + asz;
    double* dvec = tip + ntip;
    double* cvec = dvec + msz;
    double* ell = cvec + msz;
    double* xnew = W + (size_t)B * per;   // B x N
    double* tmp = xnew + (size_t)B * N;   // B x N
    double* prm = tmp + (size_t)B * N;    // B x PSTRIDE
    double* ones = prm + (size_t)B * BTA_PSTRIDE;
    double* scal = ones + msz;            // per slot: [0] ell sum, [1] x^T Q_p x, [2] unused (3 apart)
    double* step = scal + 3 * (size_t)B;  // B values
    LapObs o{m->m, m->nv, m->ns, m->nr, ctx->b, N, nb, m->obs_tv, m->obs_s, m->obs_w, m->obs_gpos, m->obs_X, m->obs_y};
    ObsWeights wts{gram, arrow, tip, per, per, per};
    const int obs_blocks = (int)std::max(1, std::min((m->m + LAP_THREADS - 1) / LAP_THREADS, 1216));
    for (int r0 = 0; r0 < n_theta; r0 += B) {
        const int cnt = std::min(B, n_theta - r0);
        const double* theta = thetas_dev + (long long)r0 * m->dim_theta;
        double* x = vec_row(ctx, VEC_MU, B);
        double* rhs = vec_row(ctx, VEC_RHS, B);
        BTA_TRY(theta_to_params_impl(m, theta, cnt, ctx->params, s));
        lap_params_kernel<<<cnt, 64, 0, s>>>(ctx->params, m->nv, prm);
        BTA_LAUNCH_CHECK();
        // the prior does not depend on x: Q_p once
        BTA_TRY(assemble_impl(ctx, m, ctx->params, 0, cnt, s));
        BTA_TRY(factor_impl(ctx, 0, cnt, s));
        BTA_TRY(logdet_impl(ctx, 0, cnt, ctx->ld, s));
        BTA_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)cnt * N * sizeof(double), s));
        for (int it = 0;; ++it) {
            // curvature and right-hand side at x_k, Q_c(x_k)
            lap_eta_lik_kernel<<<dim3(obs_blocks, cnt), LAP_THREADS, 0, s>>>(o, likelihood, x, N, ctx->params, dvec,
                                                                             cvec, ell, per);
            BTA_LAUNCH_CHECK();
            for (int j = 0; j < cnt; ++j)
                BTA_CUDA_TRY(cudaMemsetAsync(gram + j * per, 0, (size_t)(gsz + asz + ntip) * sizeof(double), s));
            BTA_CUDA_TRY(cudaMemsetAsync(rhs, 0, (size_t)cnt * N * sizeof(double), s));
            lap_scatter_kernel<<<dim3(obs_blocks, cnt), LAP_THREADS, scatter_smem, s>>>(
                o, dvec, cvec, per, gram, per, arrow, per, tip, per, rhs, N);
            BTA_LAUNCH_CHECK();
            BTA_TRY(assemble_weighted_impl(ctx, m, prm, B, cnt, s, wts));
            BTA_TRY(factor_impl(ctx, B, cnt, s));
            if (it == newton_iters) break;
            // x_{k+1} = Q_c(x_k)^{-1} A^T (g + D eta), refined with an FP64 residual in mixed precision
            BTA_TRY(solve_impl(ctx, B, cnt, rhs, xnew, s));
            for (int rit = 0; rit < ctx->refine; ++rit) {
                double* res = vec_row(ctx, VEC_RES, B);
                double* corr = vec_row(ctx, VEC_CORR, B);
                BTA_TRY(matvec_impl(ctx, B, cnt, xnew, res, s));
                BTA_TRY(axpby64(s, cnt * N, 1.0, rhs, -1.0, res, res));
                BTA_TRY(solve_impl(ctx, B, cnt, res, corr, s));
                BTA_TRY(axpby64(s, cnt * N, 1.0, xnew, 1.0, corr, xnew));
            }
            lap_step_kernel<<<cnt, LAP_THREADS, 0, s>>>(xnew, x, N, step);
            BTA_LAUNCH_CHECK();
        }
        BTA_TRY(logdet_impl(ctx, B, cnt, ctx->ld + B, s));
        // sum of the log-likelihood terms at x* and x*^T Q_p x*
        for (int j = 0; j < cnt; ++j)
            BTA_TRY(dot_batch64(s, ell + j * per, ones, m->m, 1, ctx->red + (long long)j * ctx->red_chunks,
                                ctx->red_chunks, scal + 3 * j, 3));
        BTA_TRY(matvec_impl(ctx, 0, cnt, x, tmp, s));
        BTA_TRY(dot_batch64(s, x, tmp, N, cnt, ctx->red, ctx->red_chunks, scal + 1, 3));
        lap_final_kernel<<<cnt, 1, 0, s>>>(theta, m->theta0, m->dim_theta, scal, scal + 1, ctx->ld, ctx->ld + B,
                                           f_out_dev + r0);
        BTA_LAUNCH_CHECK();
        if (x_out_dev)
            BTA_CUDA_TRY(cudaMemcpyAsync(x_out_dev + (long long)r0 * N, x, (size_t)cnt * N * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s));
        if (step_out_dev)
            BTA_CUDA_TRY(cudaMemcpyAsync(step_out_dev + r0, step, (size_t)cnt * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s));
    }
    return BTA_OK;
}
