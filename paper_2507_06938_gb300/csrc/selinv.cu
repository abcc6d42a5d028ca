// Selected inversion of a factored BTA matrix (Section III-A, selected
// inversion; the entries of Sigma = Q^{-1} on the BTA pattern give the
// marginal variances of Section III, latent marginals).
//
// From Sigma L = L^{-T} restricted to block rows j >= i of block column i,
// with G_i = L_{i+1,i} L_ii^{-1} and F_i = L_{t,i} L_ii^{-1}:
//   Sigma_tt      = L_tt^{-T} L_tt^{-1}
//   Sigma_{i+1,i} = -Sigma_{i+1,i+1} G_i - Sigma_{t,i+1}^T F_i
//   Sigma_{t,i}   = -Sigma_{t,i+1} G_i - Sigma_tt F_i
//   Sigma_ii      = L_ii^{-T} L_ii^{-1} - Sigma_{i+1,i}^T G_i - Sigma_{t,i}^T F_i
// for i = n-1 down to 0 (terms with index n are absent).  Every step is a
// GEMM on the FP64 pipe; Sigma_ii is computed on its lower triangle and then
// mirrored.

#include <algorithm>

#include "common.cuh"

int selinv_impl(bta_ctx_t ctx, int which, cudaStream_t s) {
    const int n = ctx->n, b = ctx->b, a = ctx->a;
    const long long bb = (long long)b * b, ab = (long long)a * b;
    const BtaMat& L = ctx->L[which];
    const BtaMat& S = ctx->S[which];
    const double* Linv = ctx->Linv[which];
    double* G = ctx->work[which];         // b x b
    double* F = G + bb;                   // a x b
    const double* XT = Linv + n * bb;     // L_tt^{-1}
    Gemm64 g{};
    if (a > 0) {
        g = Gemm64{};
        g.M = a; g.N = a; g.K = a;
        g.A = XT; g.lda = a; g.ta = 1; g.shA = 2;
        g.B = XT; g.ldb = a; g.shB = 1;
        g.C = S.T; g.ldc = a; g.alpha = 1.0;
        BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
    }
    for (int i = n - 1; i >= 0; --i) {
        const double* Xi = Linv + i * bb;
        double* SDi = S.D + i * bb;
        double* SRi = S.R + i * ab;
        if (a > 0) {
            // F = L_{t,i} X_i
            g = Gemm64{};
            g.M = a; g.N = b; g.K = b;
            g.A = L.R + i * ab; g.lda = a;
            g.B = Xi; g.ldb = b; g.shB = 1;
            g.C = F; g.ldc = a; g.alpha = 1.0;
            BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
        }
        if (i < n - 1) {
            double* SBi = S.B + i * bb;
            // G = L_{i+1,i} X_i
            g = Gemm64{};
            g.M = b; g.N = b; g.K = b;
            g.A = L.B + i * bb; g.lda = b;
            g.B = Xi; g.ldb = b; g.shB = 1;
            g.C = G; g.ldc = b; g.alpha = 1.0;
            BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
            // Sigma_{i+1,i} = -Sigma_{i+1,i+1} G  (- Sigma_{t,i+1}^T F)
            g = Gemm64{};
            g.M = b; g.N = b; g.K = b;
            g.A = S.D + (i + 1) * bb; g.lda = b;
            g.B = G; g.ldb = b;
            g.C = SBi; g.ldc = b; g.alpha = -1.0;
            BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
            if (a > 0) {
                g = Gemm64{};
                g.M = b; g.N = b; g.K = a;
                g.A = S.R + (i + 1) * ab; g.lda = a; g.ta = 1;
                g.B = F; g.ldb = a;
                g.Cin = SBi; g.ldci = b; g.beta = 1.0;
                g.C = SBi; g.ldc = b; g.alpha = -1.0;
                BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
                // Sigma_{t,i} = -Sigma_{t,i+1} G - Sigma_tt F
                g = Gemm64{};
                g.M = a; g.N = b; g.K = b;
                g.A = S.R + (i + 1) * ab; g.lda = a;
                g.B = G; g.ldb = b;
                g.C = SRi; g.ldc = a; g.alpha = -1.0;
                BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
                g = Gemm64{};
                g.M = a; g.N = b; g.K = a;
                g.A = S.T; g.lda = a;
                g.B = F; g.ldb = a;
                g.Cin = SRi; g.ldci = a; g.beta = 1.0;
                g.C = SRi; g.ldc = a; g.alpha = -1.0;
                BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
            }
        } else if (a > 0) {
            // Sigma_{t,n-1} = -Sigma_tt F
            g = Gemm64{};
            g.M = a; g.N = b; g.K = a;
            g.A = S.T; g.lda = a;
            g.B = F; g.ldb = a;
            g.C = SRi; g.ldc = a; g.alpha = -1.0;
            BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
        }
        // Sigma_ii = X_i^T X_i - Sigma_{i+1,i}^T G - Sigma_{t,i}^T F   (lower, then mirrored)
        g = Gemm64{};
        g.M = b; g.N = b; g.K = b;
        g.A = Xi; g.lda = b; g.ta = 1; g.shA = 2;
        g.B = Xi; g.ldb = b; g.shB = 1;
        g.C = SDi; g.ldc = b; g.alpha = 1.0; g.lowerC = 1;
        BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
        if (i < n - 1) {
            g = Gemm64{};
            g.M = b; g.N = b; g.K = b;
            g.A = S.B + i * bb; g.lda = b; g.ta = 1;
            g.B = G; g.ldb = b;
            g.Cin = SDi; g.ldci = b; g.beta = 1.0;
            g.C = SDi; g.ldc = b; g.alpha = -1.0; g.lowerC = 1;
            BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
        }
        if (a > 0) {
            g = Gemm64{};
            g.M = b; g.N = b; g.K = a;
            g.A = SRi; g.lda = a; g.ta = 1;
            g.B = F; g.ldb = a;
            g.Cin = SDi; g.ldci = b; g.beta = 1.0;
            g.C = SDi; g.ldc = b; g.alpha = -1.0; g.lowerC = 1;
            BTA_TRY(gemm_exec(&ctx->exec[which], s, g));
        }
        BTA_TRY(symmetrize_lower64(s, SDi, b, b));
    }
    return BTA_OK;
}

namespace {

__global__ void selinv_diag_kernel(const double* SD, const double* ST, int n, int b, int a, double* out) {
    const long long nb = (long long)n * b, N = nb + a;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < nb) {
            const long long i = e / b, k = e - i * b;
            out[e] = SD[i * b * (long long)b + k * (b + 1)];
        } else {
            const long long k = e - nb;
            out[e] = ST[k * (a + 1)];
        }
    }
}

}  // namespace

extern "C" int bta_selinv_diag(bta_ctx_t ctx, int which, double* out_dev) {
    if (!ctx || !out_dev || (which != BTA_QP && which != BTA_QC)) return BTA_ERR_ARG;
    if (!ctx->S[which].D) return BTA_ERR_STATE;
    const long long N = ctx->N;
    int blocks = (int)std::min<long long>((N + 255) / 256, 152 * 8);
    selinv_diag_kernel<<<blocks, 256, 0, ctx->stream>>>(ctx->S[which].D, ctx->S[which].T, ctx->n, ctx->b,
                                                        ctx->a, out_dev);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

extern "C" int bta_selinv(bta_ctx_t ctx, int which) {
    if (!ctx || (which != BTA_QP && which != BTA_QC)) return BTA_ERR_ARG;
    if (!ctx->factored[which]) return BTA_ERR_STATE;
    BTA_TRY(ensure_sigma(ctx, which));
    return selinv_impl(ctx, which, ctx->stream);
}
