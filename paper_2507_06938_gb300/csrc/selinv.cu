// Selected inversion of factored BTA matrices (Section III-A, selected
// inversion; the entries of Sigma = Q^{-1} on the BTA pattern give the
// marginal variances of Section III, latent marginals), batched over a range
// of matrices.
//
// From Sigma L = L^{-T} restricted to block rows j >= i of block column i,
// with G_i = L_{i+1,i} L_ii^{-1} and F_i = L_{t,i} L_ii^{-1}:
//   Sigma_tt      = L_tt^{-T} L_tt^{-1}
//   Sigma_{i+1,i} = -Sigma_{i+1,i+1} G_i - Sigma_{t,i+1}^T F_i
//   Sigma_{t,i}   = -Sigma_{t,i+1} G_i - Sigma_tt F_i
//   Sigma_ii      = L_ii^{-T} L_ii^{-1} - Sigma_{i+1,i}^T G_i - Sigma_{t,i}^T F_i
// for i = n-1 down to 0 (terms with index n are absent).  The products with a
// b x b output go through the context's GEMM executor (tensor cores in mixed
// precision); the arrow and tip products stay FP64 and run on a third stream
// (F_i one step ahead, Sigma_{t,i} beside the b x b product of its step).  Sigma_ii is computed on its lower
// triangle and then mirrored.

#include <algorithm>

#include "common.cuh"

int selinv_impl(bta_ctx_t ctx, int m0, int cnt, cudaStream_t s) {
    if (ctx->tparts > 1) return pselinv_impl(ctx, m0, cnt, s);
    const int n = ctx->n, b = ctx->b, a = ctx->a;
    const long long bb = (long long)b * b, ab = (long long)a * b;
    const BtaStore& L = ctx->L;
    const BtaStore& S = ctx->S;
    const double* LB = L.B + m0 * L.sB;
    const double* LR = L.R + m0 * L.sR;
    double* SD = S.D + m0 * S.sD;
    double* SB = S.B + m0 * S.sB;
    double* SR = S.R + m0 * S.sR;
    double* ST = S.T + m0 * S.sT;
    const double* Linv = ctx->Linv + m0 * ctx->sLinv;
    const long long sX = ctx->sLinv, sW = ctx->sWork;
    double* G = ctx->work + m0 * ctx->sWork;   // b x b
    double* Fb[2] = {G + bb, G + bb + ab};     // a x b, F_i in Fb[i & 1]
    const double* XT = Linv + n * bb;          // L_tt^{-1}
    const GemmExec* ex = &ctx->exec;
    // the arrow products (F_i and Sigma_{t,i}) run on the third stream, one
    // step ahead for F, beside the b x b products of the main stream
    const bool side = a > 0 && ctx->fork && ctx->fork->s3;
    cudaStream_t as = side ? ctx->fork->s3 : s;
    auto fork = [&]() -> int {
        if (!side) return BTA_OK;
        BTA_CUDA_TRY(cudaEventRecord(ctx->fork->ev3_fork, s));
        BTA_CUDA_TRY(cudaStreamWaitEvent(as, ctx->fork->ev3_fork, 0));
        return BTA_OK;
    };
    auto join = [&]() -> int {
        if (!side) return BTA_OK;
        BTA_CUDA_TRY(cudaEventRecord(ctx->fork->ev3_join, as));
        BTA_CUDA_TRY(cudaStreamWaitEvent(s, ctx->fork->ev3_join, 0));
        return BTA_OK;
    };
    // F_i = L_{t,i} X_i
    auto arrow_F = [&](int i, cudaStream_t st) -> int {
        Gemm64 g{};
        g.M = a; g.N = b; g.K = b;
        g.A = LR + i * ab; g.lda = a;
        g.B = Linv + i * bb; g.ldb = b; g.shB = 1;
        g.C = Fb[i & 1]; g.ldc = a; g.alpha = 1.0;
        g.batch = cnt; g.sA = L.sR; g.sB = sX; g.sC = sW;
        return gemm64(st, g);
    };
    Gemm64 g{};
    if (a > 0) {
        // Sigma_tt = X_T^T X_T
        g = Gemm64{};
        g.M = a; g.N = a; g.K = a;
        g.A = XT; g.lda = a; g.ta = 1; g.shA = 2;
        g.B = XT; g.ldb = a; g.shB = 1;
        g.C = ST; g.ldc = a; g.alpha = 1.0;
        g.batch = cnt; g.sA = sX; g.sB = sX; g.sC = S.sT;
        BTA_TRY(gemm64(s, g));
        BTA_TRY(fork());
        BTA_TRY(arrow_F(n - 1, as));
    }
    for (int i = n - 1; i >= 0; --i) {
        const double* Xi = Linv + i * bb;
        double* SDi = SD + i * bb;
        double* SRi = SR + i * ab;
        double* F = Fb[i & 1];
        if (i < n - 1) {
            double* SBi = SB + i * bb;
            // G = L_{i+1,i} X_i
            g = Gemm64{};
            g.M = b; g.N = b; g.K = b;
            g.A = LB + i * bb; g.lda = b;
            g.B = Xi; g.ldb = b; g.shB = 1;
            g.C = G; g.ldc = b; g.alpha = 1.0;
            g.batch = cnt; g.sA = L.sB; g.sB = sX; g.sC = sW;
            BTA_TRY(gemm_exec(ex, s, g));
            if (a > 0) {
                BTA_TRY(fork());
                // Sigma_{t,i} = -Sigma_{t,i+1} G - Sigma_tt F      (third stream)
                g = Gemm64{};
                g.M = a; g.N = b; g.K = b;
                g.A = SR + (i + 1) * ab; g.lda = a;
                g.B = G; g.ldb = b;
                g.C = SRi; g.ldc = a; g.alpha = -1.0;
                g.batch = cnt; g.sA = S.sR; g.sB = sW; g.sC = S.sR;
                BTA_TRY(gemm64(as, g));
                g = Gemm64{};
                g.M = a; g.N = b; g.K = a;
                g.A = ST; g.lda = a;
                g.B = F; g.ldb = a;
                g.Cin = SRi; g.ldci = a; g.beta = 1.0;
                g.C = SRi; g.ldc = a; g.alpha = -1.0;
                g.batch = cnt; g.sA = S.sT; g.sB = sW; g.sCi = S.sR; g.sC = S.sR;
                BTA_TRY(gemm64(as, g));
                if (i > 0) BTA_TRY(arrow_F(i - 1, as));
            }
            // Sigma_{i+1,i} = -Sigma_{i+1,i+1} G  (- Sigma_{t,i+1}^T F)
            g = Gemm64{};
            g.M = b; g.N = b; g.K = b;
            g.A = SD + (i + 1) * bb; g.lda = b;
            g.B = G; g.ldb = b;
            g.C = SBi; g.ldc = b; g.alpha = -1.0;
            g.batch = cnt; g.sA = S.sD; g.sB = sW; g.sC = S.sB;
            BTA_TRY(gemm_exec(ex, s, g));
            if (a > 0) {
                // Sigma_{t,i+1} and F_i were made final by the previous step's join
                g = Gemm64{};
                g.M = b; g.N = b; g.K = a;
                g.A = SR + (i + 1) * ab; g.lda = a; g.ta = 1;
                g.B = F; g.ldb = a;
                g.Cin = SBi; g.ldci = b; g.beta = 1.0;
                g.C = SBi; g.ldc = b; g.alpha = -1.0;
                g.batch = cnt; g.sA = S.sR; g.sB = sW; g.sCi = S.sB; g.sC = S.sB;
                BTA_TRY(gemm_exec(ex, s, g));
            }
        } else if (a > 0) {
            // Sigma_{t,n-1} = -Sigma_tt F      (third stream, after F_{n-1})
            g = Gemm64{};
            g.M = a; g.N = b; g.K = a;
            g.A = ST; g.lda = a;
            g.B = F; g.ldb = a;
            g.C = SRi; g.ldc = a; g.alpha = -1.0;
            g.batch = cnt; g.sA = S.sT; g.sB = sW; g.sC = S.sR;
            BTA_TRY(gemm64(as, g));
            if (i > 0) BTA_TRY(arrow_F(i - 1, as));
        }
        // Sigma_ii = X_i^T X_i - Sigma_{i+1,i}^T G - Sigma_{t,i}^T F   (lower, then mirrored)
        const double* Xs = Xi;
        long long sXs = sX;
        if (ctx->lowmem) {
            // Sigma_ii takes X_i's slot: the product reads a copy.  F_{n-1}
            // (third stream, issued before the loop) reads that slot too; the
            // later F_i were joined at the end of step i + 1
            if (i == n - 1) BTA_TRY(join());
            double* Xw = ctx->xtmp + m0 * bb;
            BTA_TRY(copy_mat64(s, Xi, b, Xw, b, b, b, 0, cnt, sX, bb));
            Xs = Xw;
            sXs = bb;
        }
        g = Gemm64{};
        g.M = b; g.N = b; g.K = b;
        g.A = Xs; g.lda = b; g.ta = 1; g.shA = 2;
        g.B = Xs; g.ldb = b; g.shB = 1;
        g.C = SDi; g.ldc = b; g.alpha = 1.0; g.lowerC = 1;
        g.batch = cnt; g.sA = sXs; g.sB = sXs; g.sC = S.sD;
        BTA_TRY(gemm_exec(ex, s, g));
        if (i < n - 1) {
            g = Gemm64{};
            g.M = b; g.N = b; g.K = b;
            g.A = SB + i * bb; g.lda = b; g.ta = 1;
            g.B = G; g.ldb = b;
            g.Cin = SDi; g.ldci = b; g.beta = 1.0;
            g.C = SDi; g.ldc = b; g.alpha = -1.0; g.lowerC = 1;
            g.batch = cnt; g.sA = S.sB; g.sB = sW; g.sCi = S.sD; g.sC = S.sD;
            BTA_TRY(gemm_exec(ex, s, g));
        }
        if (a > 0) {
            // Sigma_{t,i} (and F_{i-1}) from the third stream
            BTA_TRY(join());
            g = Gemm64{};
            g.M = b; g.N = b; g.K = a;
            g.A = SRi; g.lda = a; g.ta = 1;
            g.B = F; g.ldb = a;
            g.Cin = SDi; g.ldci = b; g.beta = 1.0;
            g.C = SDi; g.ldc = b; g.alpha = -1.0; g.lowerC = 1;
            g.batch = cnt; g.sA = S.sR; g.sB = sW; g.sCi = S.sD; g.sC = S.sD;
            BTA_TRY(gemm_exec(ex, s, g));
        }
        BTA_TRY(symmetrize_lower64(s, SDi, b, b, cnt, S.sD));
    }
    // the low-memory layout has overwritten the factor
    if (ctx->lowmem)
        for (int m = m0; m < m0 + cnt; ++m) ctx->factored[m] = 0;
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
    if (!ctx || !out_dev) return BTA_ERR_ARG;
    const int m = storage_index(ctx, which);
    if (m < 0) return BTA_ERR_ARG;
    if (!ctx->S.D) return BTA_ERR_STATE;
    const long long N = ctx->N;
    int blocks = (int)std::min<long long>((N + 255) / 256, 152 * 8);
    selinv_diag_kernel<<<blocks, 256, 0, ctx->stream>>>(ctx->S.D + m * ctx->S.sD, ctx->S.T + m * ctx->S.sT, ctx->n,
                                                        ctx->b, ctx->a, out_dev);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

extern "C" int bta_selinv(bta_ctx_t ctx, int which) {
    if (!ctx) return BTA_ERR_ARG;
    const int m = storage_index(ctx, which);
    if (m < 0) return BTA_ERR_ARG;
    if (!ctx->factored[m]) return BTA_ERR_STATE;
    BTA_TRY(ensure_sigma(ctx));
    return selinv_impl(ctx, m, 1, ctx->stream);
}

extern "C" int bta_selinv_batch(bta_ctx_t ctx, int kind) {
    if (!ctx || (kind != BTA_QP && kind != BTA_QC)) return BTA_ERR_ARG;
    const int m0 = kind * ctx->batch;
    for (int m = m0; m < m0 + ctx->batch; ++m)
        if (!ctx->factored[m]) return BTA_ERR_STATE;
    BTA_TRY(ensure_sigma(ctx));
    return selinv_impl(ctx, m0, ctx->batch, ctx->stream);
}
