// Forward/backward block substitution with BTA Cholesky factors, the BTA
// matrix-vector product and iterative refinement (Section III-A, triangular
// solve; Section IV-E), batched over a range of matrices (vectors N apart).
// The diagonal solves use the stored inverses L_ii^{-1}, so every step is a
// GEMV bound by the HBM read of the factor.
//
//   forward:  z_i = L_ii^{-1} (r_i - L_{i,i-1} z_{i-1}),  z_t = L_tt^{-1} (r_t - sum_i L_{t,i} z_i)
//   backward: x_t = L_tt^{-T} z_t,  x_i = L_ii^{-T} (z_i - L_{i+1,i}^T x_{i+1} - L_{t,i}^T x_t)
// The arrow blocks L_{t,i} of all i form one a x (n b) column-major matrix.

#include <algorithm>

#include "common.cuh"

namespace {

__global__ void axpby_kernel(long long len, double alpha, const double* x, double beta, const double* y,
                             double* out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = alpha * x[e] + (beta != 0.0 ? beta * y[e] : 0.0);
}

__global__ void ratio_sqrt_kernel(const double* num, const double* den, double* out) {
    *out = sqrt(*num) / sqrt(*den);
}

// out[j] = sqrt(d[3j + 1] / d[3j + 2]) for j < count (one thread each)
__global__ void ratio_sqrt_batch_kernel(const double* d, int count, double* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) out[j] = sqrt(d[3 * j + 1]) / sqrt(d[3 * j + 2]);
}

}  // namespace

int axpby64(cudaStream_t s, long long len, double alpha, const double* x, double beta, const double* y,
            double* out) {
    if (len <= 0) return BTA_OK;
    int blocks = (int)std::min<long long>((len + 255) / 256, 152 * 8);
    axpby_kernel<<<blocks, 256, 0, s>>>(len, alpha, x, beta, y, out);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

// r, x: cnt vectors N apart; scratch rows VEC_Z / VEC_TMP of the same matrices.
int solve_impl(bta_ctx_t ctx, int m0, int cnt, const double* r, double* x, cudaStream_t s) {
    if (ctx->tparts > 1) return psolve_impl(ctx, m0, cnt, r, x, s);
    const int n = ctx->n, b = ctx->b, a = ctx->a;
    const long long N = ctx->N, nb = (long long)n * b, bb = (long long)b * b;
    const BtaStore& L = ctx->L;
    const double* LB = L.B + m0 * L.sB;
    const double* LR = L.R + m0 * L.sR;
    const double* Linv = ctx->Linv + m0 * ctx->sLinv;
    const long long sX = ctx->sLinv;
    double* z = vec_row(ctx, VEC_Z, m0);
    double* tmp = vec_row(ctx, VEC_TMP, m0);
    // forward
    for (int i = 0; i < n; ++i) {
        const double* ri = r + (long long)i * b;
        if (i > 0) {
            BTA_TRY(gemv64(s, b, b, LB + (i - 1) * bb, b, 0, 0, z + (long long)(i - 1) * b, -1.0, ri, 1.0, tmp, cnt,
                           L.sB, N, N));
            ri = tmp;
        }
        BTA_TRY(gemv64(s, b, b, Linv + i * bb, b, 0, 1, ri, 1.0, nullptr, 0.0, z + (long long)i * b, cnt, sX, N, N));
    }
    if (a > 0) {
        BTA_TRY(gemv64(s, a, (int)nb, LR, a, 0, 0, z, -1.0, r + nb, 1.0, tmp, cnt, L.sR, N, N));
        BTA_TRY(gemv64(s, a, a, Linv + n * bb, a, 0, 1, tmp, 1.0, nullptr, 0.0, z + nb, cnt, sX, N, N));
        // backward tip: x_t = L_tt^{-T} z_t ; z_i -= L_{t,i}^T x_t
        BTA_TRY(gemv64(s, a, a, Linv + n * bb, a, 1, 2, z + nb, 1.0, nullptr, 0.0, x + nb, cnt, sX, N, N));
        BTA_TRY(gemv64(s, (int)nb, a, LR, a, 1, 0, x + nb, -1.0, z, 1.0, z, cnt, L.sR, N, N));
    }
    for (int i = n - 1; i >= 0; --i) {
        const double* zi = z + (long long)i * b;
        if (i < n - 1) {
            BTA_TRY(gemv64(s, b, b, LB + i * bb, b, 1, 0, x + (long long)(i + 1) * b, -1.0, zi, 1.0, tmp, cnt,
                           L.sB, N, N));
            zi = tmp;
        }
        BTA_TRY(gemv64(s, b, b, Linv + i * bb, b, 1, 2, zi, 1.0, nullptr, 0.0, x + (long long)i * b, cnt, sX, N, N));
    }
    return BTA_OK;
}

// y_j = Q_{m0+j} x_j with the assembled blocks (vectors N apart).
int matvec_impl(bta_ctx_t ctx, int m0, int cnt, const double* x, double* y, cudaStream_t s) {
    const int n = ctx->n, b = ctx->b, a = ctx->a;
    const long long N = ctx->N, nb = (long long)n * b, bb = (long long)b * b;
    const BtaStore& Q = ctx->Q;
    for (int j = 0; j < cnt; ++j) {
        const int m = m0 + j;
        const double* xj = x + j * N;
        double* yj = y + j * N;
        // y_i = D_i x_i
        BTA_TRY(gemv64(s, b, b, Q.D + m * Q.sD, b, 0, 0, xj, 1.0, nullptr, 0.0, yj, n, bb, b, b));
        if (n > 1) {
            // y_{i+1} += B_i x_i ;  y_i += B_i^T x_{i+1}
            BTA_TRY(gemv64(s, b, b, Q.B + m * Q.sB, b, 0, 0, xj, 1.0, yj + b, 1.0, yj + b, n - 1, bb, b, b));
            BTA_TRY(gemv64(s, b, b, Q.B + m * Q.sB, b, 1, 0, xj + b, 1.0, yj, 1.0, yj, n - 1, bb, b, b));
        }
    }
    if (a > 0) {
        const double* QR = Q.R + m0 * Q.sR;
        BTA_TRY(gemv64(s, (int)nb, a, QR, a, 1, 0, x + nb, 1.0, y, 1.0, y, cnt, Q.sR, N, N));
        BTA_TRY(gemv64(s, a, (int)nb, QR, a, 0, 0, x, 1.0, nullptr, 0.0, y + nb, cnt, Q.sR, N, N));
        BTA_TRY(gemv64(s, a, a, Q.T + m0 * Q.sT, a, 0, 0, x + nb, 1.0, y + nb, 1.0, y + nb, cnt, Q.sT, N, N));
    }
    return BTA_OK;
}

extern "C" int bta_matvec(bta_ctx_t ctx, int which, const double* x_dev, double* y_dev) {
    if (!ctx || !x_dev || !y_dev) return BTA_ERR_ARG;
    const int m = storage_index(ctx, which);
    if (m < 0) return BTA_ERR_ARG;
    return matvec_impl(ctx, m, 1, x_dev, y_dev, ctx->stream);
}

extern "C" int bta_solve(bta_ctx_t ctx, int which, const double* rhs_dev, double* x_dev, int refine_iters,
                         double* resid_dev) {
    if (!ctx || !rhs_dev || !x_dev || refine_iters < 0) return BTA_ERR_ARG;
    const int m = storage_index(ctx, which);
    if (m < 0) return BTA_ERR_ARG;
    if (!ctx->factored[m]) return BTA_ERR_STATE;
    cudaStream_t s = ctx->stream;
    const long long N = ctx->N;
    double* rcopy = vec_row(ctx, VEC_RCOPY, m);   // private copy: rhs may alias x
    double* res = vec_row(ctx, VEC_RES, m);
    double* corr = vec_row(ctx, VEC_CORR, m);
    BTA_CUDA_TRY(cudaMemcpyAsync(rcopy, rhs_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    BTA_TRY(solve_impl(ctx, m, 1, rcopy, x_dev, s));
    for (int it = 0; it < refine_iters; ++it) {
        BTA_TRY(matvec_impl(ctx, m, 1, x_dev, res, s));
        BTA_TRY(axpby64(s, N, 1.0, rcopy, -1.0, res, res));       // res = r - Q x
        BTA_TRY(solve_impl(ctx, m, 1, res, corr, s));
        BTA_TRY(axpby64(s, N, 1.0, x_dev, 1.0, corr, x_dev));
    }
    if (resid_dev) {
        double* d = ctx->dots + 3 * m;
        BTA_TRY(matvec_impl(ctx, m, 1, x_dev, res, s));
        BTA_TRY(axpby64(s, N, 1.0, rcopy, -1.0, res, res));
        double* part = ctx->red + (long long)m * ctx->red_chunks;
        BTA_TRY(dot_batch64(s, res, res, N, 1, part, ctx->red_chunks, d + 1, 1));
        BTA_TRY(dot_batch64(s, rcopy, rcopy, N, 1, part, ctx->red_chunks, d + 2, 1));
        ratio_sqrt_kernel<<<1, 1, 0, s>>>(d + 1, d + 2, resid_dev);
        BTA_LAUNCH_CHECK();
    }
    return BTA_OK;
}

// ||b - Q_c mu||_2 / ||b||_2 of every slot's conditional mean from the last
// f_obj group, with the assembled FP64 blocks of Q_c.
extern "C" int bta_fobj_residual(bta_ctx_t ctx, double* out_dev) {
    if (!ctx || !out_dev) return BTA_ERR_ARG;
    const int B = ctx->batch;
    for (int j = 0; j < B; ++j)
        if (!ctx->mu_valid[j]) return BTA_ERR_STATE;
    cudaStream_t s = ctx->stream;
    const long long N = ctx->N;
    double* rhs = vec_row(ctx, VEC_RHS, B);
    double* mu = vec_row(ctx, VEC_MU, B);
    double* res = vec_row(ctx, VEC_RES, B);
    BTA_TRY(matvec_impl(ctx, B, B, mu, res, s));
    BTA_TRY(axpby64(s, B * N, 1.0, rhs, -1.0, res, res));
    double* d = ctx->dots + 3 * B;
    double* part = ctx->red + (long long)B * ctx->red_chunks;
    BTA_TRY(dot_batch64(s, res, res, N, B, part, ctx->red_chunks, d + 1, 3));
    BTA_TRY(dot_batch64(s, rhs, rhs, N, B, part, ctx->red_chunks, d + 2, 3));
    ratio_sqrt_batch_kernel<<<(B + 127) / 128, 128, 0, s>>>(d, B, out_dev);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}
