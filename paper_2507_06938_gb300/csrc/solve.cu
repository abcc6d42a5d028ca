// Forward/backward block substitution with a BTA Cholesky factor, the BTA
// matrix-vector product and iterative refinement (Section III-A, triangular
// solve; Section IV-E).  The diagonal solves use the stored inverses
// L_ii^{-1}, so every step is a GEMV bound by the HBM read of the factor.
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

}  // namespace

int axpby64(cudaStream_t s, long long len, double alpha, const double* x, double beta, const double* y,
            double* out) {
    if (len <= 0) return BTA_OK;
    int blocks = (int)std::min<long long>((len + 255) / 256, 152 * 8);
    axpby_kernel<<<blocks, 256, 0, s>>>(len, alpha, x, beta, y, out);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

// Scratch vectors (rows of ctx->vec, length N each): 0 rhs copy, 1 residual,
// 2 correction, 3/4 z/tmp of Q_p, 5/6 z/tmp of Q_c, 7 f_obj right-hand side,
// 8 f_obj conditional mean.
int solve_impl(bta_ctx_t ctx, int which, const double* r, double* x, cudaStream_t s) {
    const int n = ctx->n, b = ctx->b, a = ctx->a;
    const long long N = ctx->N, nb = (long long)n * b, bb = (long long)b * b;
    const BtaMat& L = ctx->L[which];
    const double* Linv = ctx->Linv[which];
    double* z = ctx->vec + N * (3 + 2 * which);
    double* tmp = ctx->vec + N * (4 + 2 * which);
    // forward
    for (int i = 0; i < n; ++i) {
        const double* ri = r + (long long)i * b;
        if (i > 0) {
            BTA_TRY(gemv64(s, b, b, L.B + (i - 1) * bb, b, 0, 0, z + (long long)(i - 1) * b, -1.0, ri, 1.0, tmp));
            ri = tmp;
        }
        BTA_TRY(gemv64(s, b, b, Linv + i * bb, b, 0, 1, ri, 1.0, nullptr, 0.0, z + (long long)i * b));
    }
    if (a > 0) {
        BTA_TRY(gemv64(s, a, (int)nb, L.R, a, 0, 0, z, -1.0, r + nb, 1.0, tmp));
        BTA_TRY(gemv64(s, a, a, Linv + n * bb, a, 0, 1, tmp, 1.0, nullptr, 0.0, z + nb));
        // backward tip: x_t = L_tt^{-T} z_t ; u = L_R^T x_t
        BTA_TRY(gemv64(s, a, a, Linv + n * bb, a, 1, 2, z + nb, 1.0, nullptr, 0.0, x + nb));
        BTA_TRY(gemv64(s, (int)nb, a, L.R, a, 1, 0, x + nb, -1.0, z, 1.0, z));   // z_i -= L_{t,i}^T x_t
    }
    for (int i = n - 1; i >= 0; --i) {
        const double* zi = z + (long long)i * b;
        if (i < n - 1) {
            BTA_TRY(gemv64(s, b, b, L.B + i * bb, b, 1, 0, x + (long long)(i + 1) * b, -1.0, zi, 1.0, tmp));
            zi = tmp;
        }
        BTA_TRY(gemv64(s, b, b, Linv + i * bb, b, 1, 2, zi, 1.0, nullptr, 0.0, x + (long long)i * b));
    }
    return BTA_OK;
}

int matvec_impl(bta_ctx_t ctx, int which, const double* x, double* y, cudaStream_t s) {
    const int n = ctx->n, b = ctx->b, a = ctx->a;
    const long long nb = (long long)n * b, bb = (long long)b * b;
    const BtaMat& Q = ctx->Q[which];
    // y_i = D_i x_i
    BTA_TRY(gemv64(s, b, b, Q.D, b, 0, 0, x, 1.0, nullptr, 0.0, y, n, bb, b, b));
    if (n > 1) {
        // y_{i+1} += B_i x_i ;  y_i += B_i^T x_{i+1}
        BTA_TRY(gemv64(s, b, b, Q.B, b, 0, 0, x, 1.0, y + b, 1.0, y + b, n - 1, bb, b, b));
        BTA_TRY(gemv64(s, b, b, Q.B, b, 1, 0, x + b, 1.0, y, 1.0, y, n - 1, bb, b, b));
    }
    if (a > 0) {
        BTA_TRY(gemv64(s, (int)nb, a, Q.R, a, 1, 0, x + nb, 1.0, y, 1.0, y));
        BTA_TRY(gemv64(s, a, (int)nb, Q.R, a, 0, 0, x, 1.0, nullptr, 0.0, y + nb));
        BTA_TRY(gemv64(s, a, a, Q.T, a, 0, 0, x + nb, 1.0, y + nb, 1.0, y + nb));
    }
    return BTA_OK;
}

extern "C" int bta_matvec(bta_ctx_t ctx, int which, const double* x_dev, double* y_dev) {
    if (!ctx || !x_dev || !y_dev || (which != BTA_QP && which != BTA_QC)) return BTA_ERR_ARG;
    return matvec_impl(ctx, which, x_dev, y_dev, ctx->stream);
}

extern "C" int bta_solve(bta_ctx_t ctx, int which, const double* rhs_dev, double* x_dev, int refine_iters,
                         double* resid_dev) {
    if (!ctx || !rhs_dev || !x_dev || refine_iters < 0 || (which != BTA_QP && which != BTA_QC))
        return BTA_ERR_ARG;
    if (!ctx->factored[which]) return BTA_ERR_STATE;
    cudaStream_t s = ctx->stream;
    const long long N = ctx->N;
    double* rcopy = ctx->vec;   // row 0: private copy of the right-hand side (rhs may alias x)
    BTA_CUDA_TRY(cudaMemcpyAsync(rcopy, rhs_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    BTA_TRY(solve_impl(ctx, which, rcopy, x_dev, s));
    double* res = ctx->vec + N * 1;
    double* corr = ctx->vec + N * 2;
    for (int it = 0; it < refine_iters; ++it) {
        BTA_TRY(matvec_impl(ctx, which, x_dev, res, s));
        BTA_TRY(axpby64(s, N, 1.0, rcopy, -1.0, res, res));       // res = r - Q x
        BTA_TRY(solve_impl(ctx, which, res, corr, s));
        BTA_TRY(axpby64(s, N, 1.0, x_dev, 1.0, corr, x_dev));
    }
    if (resid_dev) {
        BTA_TRY(matvec_impl(ctx, which, x_dev, res, s));
        BTA_TRY(axpby64(s, N, 1.0, rcopy, -1.0, res, res));
        BTA_TRY(dot64(s, res, res, N, ctx->red, ctx->red_len / 2, ctx->scal + SCAL_NRM_R));
        BTA_TRY(dot64(s, rcopy, rcopy, N, ctx->red, ctx->red_len / 2, ctx->scal + SCAL_NRM_B));
        ratio_sqrt_kernel<<<1, 1, 0, s>>>(ctx->scal + SCAL_NRM_R, ctx->scal + SCAL_NRM_B, resid_dev);
        BTA_LAUNCH_CHECK();
    }
    return BTA_OK;
}
