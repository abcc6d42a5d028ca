// Block Cholesky of BTA matrices and their log-determinants (Section III-A,
// cost O(n (b^3 + a^3)) of Section IV-D.2), for a range of matrices of one
// shape at once: every launch below carries all matrices of the range.
//
//   for i = 0..n-1:
//     (L_ii, L_ii^{-1}) = chol_inv(D_i)                 recursive, FP64 leaves
//     L_{i+1,i} = B_i L_ii^{-T}                          GEMM, triangular operand
//     D_{i+1}  <- Q.D_{i+1} - L_{i+1,i} L_{i+1,i}^T      lower-output GEMM (SYRK)
//     L_{t,i}   = Racc_i L_ii^{-T}                       Racc_0 = R_0
//     Racc_{i+1} = R_{i+1} - L_{t,i} L_{i+1,i}^T
//     T        <- T - L_{t,i} L_{t,i}^T
//   (L_tt, L_tt^{-1}) = chol_inv(T)                      FP64
// The assembled blocks Q are only read, so they stay available for residuals.

#include <algorithm>

#include "common.cuh"

namespace {

// acc[m] (= or +=) 2 sum_k log D_m[k, k] of one diagonal factor block per
// matrix (blockIdx.x = matrix): the log-determinant of the low-memory layout,
// taken before X_i replaces L_ii
__global__ void logdiag_acc_kernel(const double* D, int b, long long sD, double* acc, int first) {
    __shared__ double red[32];
    D += blockIdx.x * sD;
    double v = 0.0;
    for (int k = threadIdx.x; k < b; k += blockDim.x) v += log(D[k * (long long)(b + 1)]);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        acc[blockIdx.x] = (first ? 0.0 : acc[blockIdx.x]) + 2.0 * s;
    }
}

// out[j] = acc[j] + 2 sum_k log T_j[k, k] (blockIdx.x = matrix)
__global__ void logdet_tip_kernel(const double* acc, const double* T, int a, long long sT, double* out) {
    __shared__ double red[32];
    T += blockIdx.x * sT;
    double v = 0.0;
    for (int k = threadIdx.x; k < a; k += blockDim.x) v += log(T[k * (long long)(a + 1)]);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        out[blockIdx.x] = acc[blockIdx.x] + 2.0 * s;
    }
}

}  // namespace

int factor_impl(bta_ctx_t ctx, int m0, int cnt, cudaStream_t s) {
    if (ctx->tparts > 1) return pfactor_impl(ctx, m0, cnt, s);
    const int n = ctx->n, b = ctx->b, a = ctx->a;
    const long long bb = (long long)b * b, ab = (long long)a * b;
    const BtaStore& Q = ctx->Q;
    const BtaStore& L = ctx->L;
    double* QD = Q.D + m0 * Q.sD;
    double* QB = Q.B + m0 * Q.sB;
    double* QR = Q.R + m0 * Q.sR;
    double* QT = Q.T + m0 * Q.sT;
    double* LD = L.D + m0 * L.sD;
    double* LB = L.B + m0 * L.sB;
    double* LR = L.R + m0 * L.sR;
    double* LT = L.T + m0 * L.sT;
    double* Linv = ctx->Linv + m0 * ctx->sLinv;
    double* W = ctx->work + m0 * ctx->sWork;          // chol_inv scratch (b*b/2 + 2b)
    double* Racc = W + bb / 2 + 2 * b;               // a*b
    const long long sW = ctx->sWork, sX = ctx->sLinv;
    long long* status = ctx->status;
    const int leaf = ctx->leaf;
    const GemmExec* ex = &ctx->exec;

    BTA_TRY(copy_mat64(s, QD, b, LD, b, b, b, 1, cnt, Q.sD, L.sD));
    if (a > 0) {
        BTA_TRY(copy_mat64(s, QT, a, LT, a, a, a, 1, cnt, Q.sT, L.sT));
        BTA_TRY(copy_mat64(s, QR, a, Racc, a, a, b, 0, cnt, Q.sR, sW));
    }
    for (int i = 0; i < n; ++i) {
        double* Di = LD + i * bb;
        double* Xi = Linv + i * bb;
        long long sXi = sX;
        if (ctx->lowmem) {
            // L_ii and X_i side by side in the D slot and the X buffer; the
            // slot keeps X_i once the diagonal of L_ii is summed
            double* Xw = ctx->xtmp + m0 * bb;
            BTA_TRY(chol_inv64(s, Di, b, Xw, b, b, (long long)i * b, status, W, leaf, ex, cnt, L.sD, bb, sW, m0,
                               ctx->batch, ctx->fork));
            logdiag_acc_kernel<<<cnt, 256, 0, s>>>(Di, b, L.sD, ctx->ldacc + m0, i == 0 ? 1 : 0);
            BTA_LAUNCH_CHECK();
            BTA_TRY(copy_mat64(s, Xw, b, Di, b, b, b, 0, cnt, bb, L.sD));
            sXi = L.sD;
        } else {
            BTA_TRY(chol_inv64(s, Di, b, Xi, b, b, (long long)i * b, status, W, leaf, ex, cnt, L.sD, sX, sW, m0,
                               ctx->batch, ctx->fork));
        }
        Gemm64 g{};
        if (i < n - 1) {
            // L_{i+1,i} = B_i X_i^T
            g = Gemm64{};
            g.M = b; g.N = b; g.K = b;
            g.A = QB + i * bb; g.lda = b;
            g.B = Xi; g.ldb = b; g.tb = 1; g.shB = 2;
            g.C = LB + i * bb; g.ldc = b; g.alpha = 1.0;
            g.batch = cnt; g.sA = Q.sB; g.sB = sXi; g.sC = L.sB;
            cudaEvent_t stop;
            BTA_TRY(prof_begin(ctx, s, (double)cnt * b * b * b, &stop));
            BTA_TRY(gemm_exec(ex, s, g));
            if (stop) BTA_TRY(prof_record(stop, s));
            // D_{i+1} = Q.D_{i+1} - L_{i+1,i} L_{i+1,i}^T   (lower)
            g = Gemm64{};
            g.M = b; g.N = b; g.K = b;
            g.A = LB + i * bb; g.lda = b;
            g.B = LB + i * bb; g.ldb = b; g.tb = 1;
            g.Cin = QD + (i + 1) * bb; g.ldci = b; g.beta = 1.0;
            g.C = LD + (i + 1) * bb; g.ldc = b; g.alpha = -1.0; g.lowerC = 1;
            g.batch = cnt; g.sA = L.sB; g.sB = L.sB; g.sCi = Q.sD; g.sC = L.sD;
            BTA_TRY(prof_begin(ctx, s, (double)cnt * b * b * b, &stop));
            BTA_TRY(gemm_exec(ex, s, g));
            if (stop) BTA_TRY(prof_record(stop, s));
        }
        if (a > 0) {
            // the arrow products need X_i and L_{i+1,i} only, and nothing on the
            // diagonal chain needs them: they run on the third stream
            cudaStream_t as = s;
            if (ctx->fork && ctx->fork->s3) {
                as = ctx->fork->s3;
                BTA_CUDA_TRY(cudaEventRecord(ctx->fork->ev3_fork, s));
                BTA_CUDA_TRY(cudaStreamWaitEvent(as, ctx->fork->ev3_fork, 0));
            }
            double* Lri = LR + i * ab;
            // L_{t,i} = Racc X_i^T
            g = Gemm64{};
            g.M = a; g.N = b; g.K = b;
            g.A = Racc; g.lda = a;
            g.B = Xi; g.ldb = b; g.tb = 1; g.shB = 2;
            g.C = Lri; g.ldc = a; g.alpha = 1.0;
            g.batch = cnt; g.sA = sW; g.sB = sXi; g.sC = L.sR;
            BTA_TRY(gemm64(as, g));
            if (i < n - 1) {
                // Racc = R_{i+1} - L_{t,i} L_{i+1,i}^T
                g = Gemm64{};
                g.M = a; g.N = b; g.K = b;
                g.A = Lri; g.lda = a;
                g.B = LB + i * bb; g.ldb = b; g.tb = 1;
                g.Cin = QR + (i + 1) * ab; g.ldci = a; g.beta = 1.0;
                g.C = Racc; g.ldc = a; g.alpha = -1.0;
                g.batch = cnt; g.sA = L.sR; g.sB = L.sB; g.sCi = Q.sR; g.sC = sW;
                BTA_TRY(gemm64(as, g));
            }
            // T -= L_{t,i} L_{t,i}^T   (lower, FP64)
            g = Gemm64{};
            g.M = a; g.N = a; g.K = b;
            g.A = Lri; g.lda = a;
            g.B = Lri; g.ldb = a; g.tb = 1;
            g.Cin = LT; g.ldci = a; g.beta = 1.0;
            g.C = LT; g.ldc = a; g.alpha = -1.0; g.lowerC = 1;
            g.batch = cnt; g.sA = L.sR; g.sB = L.sR; g.sCi = L.sT; g.sC = L.sT;
            BTA_TRY(gemm64(as, g));
        }
    }
    if (a > 0 && ctx->fork && ctx->fork->s3) {
        // join the arrow stream before the tip is factored
        BTA_CUDA_TRY(cudaEventRecord(ctx->fork->ev3_join, ctx->fork->s3));
        BTA_CUDA_TRY(cudaStreamWaitEvent(s, ctx->fork->ev3_join, 0));
    }
    if (a > 0)
        BTA_TRY(chol_inv64(s, LT, a, Linv + (long long)n * bb, a, a, (long long)n * b, status, W, leaf, nullptr, cnt,
                           L.sT, sX, sW, m0, ctx->batch));
    for (int m = m0; m < m0 + cnt; ++m) ctx->factored[m] = 1;
    return BTA_OK;
}

int logdet_impl(bta_ctx_t ctx, int m0, int cnt, double* out, cudaStream_t s) {
    const int n = ctx->n, b = ctx->b, a = ctx->a;
    const BtaStore& L = ctx->L;
    if (ctx->lowmem) {
        // the diagonal blocks were summed while they were factored
        logdet_tip_kernel<<<cnt, 32, 0, s>>>(ctx->ldacc + m0, L.T + m0 * L.sT, a, L.sT, out);
        BTA_LAUNCH_CHECK();
        return BTA_OK;
    }
    // 2 sum log diag over the n diagonal blocks and the tip of every matrix
    double* part = ctx->red + (long long)m0 * ctx->red_chunks;
    return logdet_batch64(s, L.D + m0 * L.sD, b, b, n, (long long)b * b, L.sD, L.T + m0 * L.sT, a, L.sT, cnt, part,
                          ctx->red_chunks, out, 2.0);
}

extern "C" int bta_factor(bta_ctx_t ctx, int which) {
    if (!ctx) return BTA_ERR_ARG;
    const int m = storage_index(ctx, which);
    if (m < 0) return BTA_ERR_ARG;
    return factor_impl(ctx, m, 1, ctx->stream);
}

extern "C" int bta_factor_batch(bta_ctx_t ctx, int kind) {
    if (!ctx || (kind != BTA_QP && kind != BTA_QC)) return BTA_ERR_ARG;
    return factor_impl(ctx, kind * ctx->batch, ctx->batch, ctx->stream);
}

extern "C" int bta_logdet(bta_ctx_t ctx, int which, double* out_dev) {
    if (!ctx || !out_dev) return BTA_ERR_ARG;
    const int m = storage_index(ctx, which);
    if (m < 0) return BTA_ERR_ARG;
    if (!ctx->factored[m]) return BTA_ERR_STATE;
    return logdet_impl(ctx, m, 1, out_dev, ctx->stream);
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
