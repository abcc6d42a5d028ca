// Block Cholesky of a BTA matrix and its log-determinant (Section III-A,
// cost O(n (b^3 + a^3)) of Section IV-D.2).
//
//   for i = 0..n-1:
//     (L_ii, L_ii^{-1}) = chol_inv(D_i)                 recursive, FP64 leaves
//     L_{i+1,i} = B_i L_ii^{-T}                          GEMM, triangular operand
//     D_{i+1}  <- Q.D_{i+1} - L_{i+1,i} L_{i+1,i}^T      lower-output GEMM (SYRK)
//     L_{t,i}   = Racc_i L_ii^{-T}                       Racc_0 = R_0
//     Racc_{i+1} = R_{i+1} - L_{t,i} L_{i+1,i}^T
//     T        <- T - L_{t,i} L_{t,i}^T
//   (L_tt, L_tt^{-1}) = chol_inv(T)
// The assembled blocks Q are only read, so they stay available for residuals.

#include <algorithm>

#include "common.cuh"

namespace {

size_t bsq(const bta_ctx_t c) { return (size_t)c->b * c->b; }

}  // namespace

int factor_impl(bta_ctx_t ctx, int which, cudaStream_t s) {
    const int n = ctx->n, b = ctx->b, a = ctx->a;
    const BtaMat& Q = ctx->Q[which];
    const BtaMat& L = ctx->L[which];
    double* Linv = ctx->Linv[which];
    double* W = ctx->work[which];                 // chol_inv scratch (b*b/2 + b)
    double* Racc = W + bsq(ctx) / 2 + b;          // a*b
    long long* status = ctx->status;
    const int leaf = ctx->leaf;

    BTA_TRY(copy_mat64(s, Q.D, b, L.D, b, b, b, 1));
    if (a > 0) {
        BTA_TRY(copy_mat64(s, Q.T, a, L.T, a, a, a, 1));
        BTA_TRY(copy_mat64(s, Q.R, a, Racc, a, a, b, 0));
    }
    for (int i = 0; i < n; ++i) {
        double* Di = L.D + i * bsq(ctx);
        double* Xi = Linv + i * bsq(ctx);
        BTA_TRY(chol_inv64(s, Di, b, Xi, b, b, (long long)i * b, status, W, leaf, &ctx->exec[which]));
        Gemm64 g{};
        if (i < n - 1) {
            // L_{i+1,i} = B_i X_i^T
            g = Gemm64{};
            g.M = b; g.N = b; g.K = b;
            g.A = Q.B + i * bsq(ctx); g.lda = b;
            g.B = Xi; g.ldb = b; g.tb = 1; g.shB = 2;
            g.C = L.B + i * bsq(ctx); g.ldc = b; g.alpha = 1.0;
            cudaEvent_t stop;
            BTA_TRY(prof_begin(ctx, s, (double)b * b * b, &stop));
            BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
            if (stop) BTA_CUDA_TRY(cudaEventRecord(stop, s));
            // D_{i+1} = Q.D_{i+1} - L_{i+1,i} L_{i+1,i}^T   (lower)
            g = Gemm64{};
            g.M = b; g.N = b; g.K = b;
            g.A = L.B + i * bsq(ctx); g.lda = b;
            g.B = L.B + i * bsq(ctx); g.ldb = b; g.tb = 1;
            g.Cin = Q.D + (i + 1) * bsq(ctx); g.ldci = b; g.beta = 1.0;
            g.C = L.D + (i + 1) * bsq(ctx); g.ldc = b; g.alpha = -1.0; g.lowerC = 1;
            BTA_TRY(prof_begin(ctx, s, (double)b * b * b, &stop));
            BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
            if (stop) BTA_CUDA_TRY(cudaEventRecord(stop, s));
        }
        if (a > 0) {
            double* Lri = L.R + (size_t)i * a * b;
            // L_{t,i} = Racc X_i^T
            g = Gemm64{};
            g.M = a; g.N = b; g.K = b;
            g.A = Racc; g.lda = a;
            g.B = Xi; g.ldb = b; g.tb = 1; g.shB = 2;
            g.C = Lri; g.ldc = a; g.alpha = 1.0;
            BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
            if (i < n - 1) {
                // Racc = R_{i+1} - L_{t,i} L_{i+1,i}^T
                g = Gemm64{};
                g.M = a; g.N = b; g.K = b;
                g.A = Lri; g.lda = a;
                g.B = L.B + i * bsq(ctx); g.ldb = b; g.tb = 1;
                g.Cin = Q.R + (size_t)(i + 1) * a * b; g.ldci = a; g.beta = 1.0;
                g.C = Racc; g.ldc = a; g.alpha = -1.0;
                BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
            }
            // T -= L_{t,i} L_{t,i}^T   (lower)
            g = Gemm64{};
            g.M = a; g.N = a; g.K = b;
            g.A = Lri; g.lda = a;
            g.B = Lri; g.ldb = a; g.tb = 1;
            g.Cin = L.T; g.ldci = a; g.beta = 1.0;
            g.C = L.T; g.ldc = a; g.alpha = -1.0; g.lowerC = 1;
            BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
        }
    }
    if (a > 0)
        BTA_TRY(chol_inv64(s, L.T, a, Linv + (size_t)n * bsq(ctx), a, a, (long long)n * b, status, W, leaf));
    ctx->factored[which] = 1;
    return BTA_OK;
}

int logdet_impl(bta_ctx_t ctx, int which, double* out, cudaStream_t s) {
    const int n = ctx->n, b = ctx->b, a = ctx->a;
    const BtaMat& L = ctx->L[which];
    // 2 sum log diag over the n diagonal blocks, then the tip
    double* part = ctx->red + (which ? ctx->red_len / 2 : 0);
    const int plen = ctx->red_len / 2;
    BTA_TRY(logdiag_sum64(s, L.D, b, b, n, bsq(ctx), part, plen, out, 2.0, 0));
    if (a > 0) BTA_TRY(logdiag_sum64(s, L.T, a, a, 1, 0, part, plen, out, 2.0, 1));
    return BTA_OK;
}

extern "C" int bta_factor(bta_ctx_t ctx, int which) {
    if (!ctx || (which != BTA_QP && which != BTA_QC)) return BTA_ERR_ARG;
    return factor_impl(ctx, which, ctx->stream);
}

extern "C" int bta_logdet(bta_ctx_t ctx, int which, double* out_dev) {
    if (!ctx || !out_dev || (which != BTA_QP && which != BTA_QC)) return BTA_ERR_ARG;
    if (!ctx->factored[which]) return BTA_ERR_STATE;
    return logdet_impl(ctx, which, out_dev, ctx->stream);
}

extern "C" double bta_flops_factor(int n, int b, int a) {
    const double B = b, A = a, Nn = n;
    return Nn * B * B * B / 3.0 + (Nn - 1) * 2.0 * B * B * B + Nn * (A * B * B + A * A * B) +
           (Nn - 1) * 2.0 * A * B * B + A * A * A / 3.0;
}

extern "C" double bta_flops_selinv(int n, int b, int a) {
    const double B = b, A = a, Nn = n;
    return Nn * 2.0 * B * B * B / 3.0 + (Nn - 1) * 5.0 * B * B * B + 6.0 * Nn * A * B * B;
}
