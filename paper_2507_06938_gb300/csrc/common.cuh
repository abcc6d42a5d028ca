// Internal declarations shared by the CUDA sources of libbta.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "bta.h"

#define BTA_MAX_NV 8

// ---------------------------------------------------------------- error plumbing
#define BTA_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return bta_cuda_fail(e_);     \
    } while (0)

#define BTA_TRY(expr)                                        \
    do {                                                     \
        int r_ = (expr);                                     \
        if (r_ != BTA_OK) return r_;                         \
    } while (0)

int bta_cuda_fail(cudaError_t e);

// Every kernel launch of the library is followed by BTA_LAUNCH_CHECK(): it
// counts the launch (bta_launch_count) and turns a launch error into a code.
void bta_note_launch();
#define BTA_LAUNCH_CHECK()                                   \
    do {                                                     \
        bta_note_launch();                                   \
        BTA_CUDA_TRY(cudaGetLastError());                    \
    } while (0)

// ---------------------------------------------------------------- model (device copies)
struct bta_model_s {
    int nv, ns, nt, nr, m, dim_theta;
    int n, b, a;
    long long N;
    int nnz;                 // union sparsity pattern of C, G and G C^-1 G
    int* rowptr;             // ns + 1
    int* col;                // nnz
    double* cval;            // lumped mass on the pattern (diagonal only)
    double* gval;            // stiffness
    double* kval;            // G C^{-1} G
    double* gram;            // nt * nv * nnz: sum over observations of w_j w_l
    double* arrow;           // nt * nv * nr * ns: sum of X_r w_j
    double* tipgram;         // nv * nr * nr: sum of X_r X_r'
    double* aty;             // N: A^T y (per variable, unscaled by tau_eps)
    double* theta0;          // dim_theta
    double* var_stats;       // 2 nv: ||y_v||^2, m_v
    double beta_prec;
};

// ---------------------------------------------------------------- dense GEMM descriptor
struct Gemm64 {
    int M, N, K;
    const double* A; long long lda; int ta; int shA;   // shA: shape of op(A): 0 general, 1 lower, 2 upper
    const double* B; long long ldb; int tb; int shB;   // shB: shape of op(B)
    const double* Cin; long long ldci; double beta;    // Cin read only if beta != 0
    double* C; long long ldc; double alpha;
    int lowerC;                                        // compute/write only entries m >= n
    int batch = 1;
    long long sA = 0, sB = 0, sCi = 0, sC = 0;         // batch strides (elements)
};

// A GEMM executor: how the factorisation and selected inversion run their
// dense products (FP64 DFMA, or the digit-split tensor-core path for the
// large ones in mixed precision).
struct GemmExec {
    int (*fn)(const GemmExec* ex, cudaStream_t s, const Gemm64& g);
    void* ws;          // digit workspace (mixed path)
    size_t ws_bytes;
    int* err;          // device error flag of the tensor-core kernel
    int min_dim;       // smallest M, N (and K) sent to the tensor-core path
};

// ---------------------------------------------------------------- BTA storage
struct BtaMat {
    double* D = nullptr;     // n * b * b
    double* B = nullptr;     // (n-1) * b * b
    double* R = nullptr;     // n * a * b
    double* T = nullptr;     // a * a
};

struct bta_ctx_s {
    int n, b, a, precision;
    long long N;
    cudaStream_t stream;
    cudaStream_t aux;        // second stream: Q_p runs beside Q_c inside fobj_eval
    cudaEvent_t ev_fork, ev_join;
    BtaMat Q[2], L[2], S[2];
    double* Linv[2] = {nullptr, nullptr};   // n * b * b, then a * a (tip)
    double* work[2] = {nullptr, nullptr};   // per-matrix scratch for the factor / selinv
    size_t work_elems;
    double* vec;             // vectors: 4 * N
    double* red;             // reduction partials
    int red_len;
    double* scal;            // device scalars (see SCAL_* below)
    long long* status;       // [0] error code, [1] info
    double* params;          // model parameters of the last fobj_eval
    GemmExec exec[2];        // per matrix (Q_p and Q_c run on different streams)
    int* oz_err = nullptr;   // device flag of the tensor-core GEMM (time-out)
    int refine = 0;          // refinement steps of the f_obj solve
    int factored[2] = {0, 0};
    int leaf;                // leaf size of the recursive diagonal factorisation
    long long last_info = -1;
    // optional event timing of the b x b x b Schur-update GEMM launches
    int prof = 0;
    std::vector<cudaEvent_t> prof_ev;   // pairs (start, stop)
    size_t prof_used = 0;
    double prof_flops = 0.0;
};

// Record an event pair around the next launch on stream s when profiling.
int prof_begin(bta_ctx_t ctx, cudaStream_t s, double flops, cudaEvent_t* stop_out);

enum {
    SCAL_LOGDET_P = 0,
    SCAL_LOGDET_C = 1,
    SCAL_DOT = 2,
    SCAL_NRM_R = 3,
    SCAL_NRM_B = 4,
    SCAL_COUNT = 16
};

// ---------------------------------------------------------------- FP64 dense kernels (dense64.cu)


int gemm64(cudaStream_t s, const Gemm64& g);


int gemm_exec(const GemmExec* ex, cudaStream_t s, const Gemm64& g);

int chol_inv64(cudaStream_t s, double* A, long long lda, double* X, long long ldx, int n,
               long long row0, long long* status, double* W, int leaf, const GemmExec* ex = nullptr);
int copy_mat64(cudaStream_t s, const double* src, long long lds, double* dst, long long ldd,
               int rows, int cols, int lower_only);
// C = beta Cin (C = 0 if beta == 0); only entries m >= n when lower
int scale_into64(cudaStream_t s, int M, int N, const double* Cin, long long ldci, double beta, double* C,
                 long long ldc, int lower);
// Digit-split tensor-core GEMM (ozaki.cu): same contract as gemm64 (batch 1).
size_t ozaki_workspace_bytes(int M, int N, int K);
int ozaki_gemm(cudaStream_t s, const Gemm64& g, void* ws, int* err);
int gemm_mixed_fn(const GemmExec* ex, cudaStream_t s, const Gemm64& g);
int symmetrize_lower64(cudaStream_t s, double* A, long long lda, int n);
// y = alpha * op(A) x + beta * yin   (op(A) shape: 0 general, 1 lower, 2 upper)
int gemv64(cudaStream_t s, int M, int N, const double* A, long long lda, int ta, int sh,
           const double* x, double alpha, const double* yin, double beta, double* y, int batch = 1,
           long long sA = 0, long long sx = 0, long long sy = 0);
// out[0] = sum_i log(A[i*(lda+1)]) for the diagonals of `count` blocks spaced by `stride`
int logdiag_sum64(cudaStream_t s, const double* A, long long lda, int dim, int count,
                  long long stride, double* partial, int partial_len, double* out, double scale,
                  int accumulate);
// out = sum x_i y_i (two-pass, deterministic)
int dot64(cudaStream_t s, const double* x, const double* y, long long len, double* partial,
          int partial_len, double* out);

// ---------------------------------------------------------------- internal drivers
int factor_impl(bta_ctx_t ctx, int which, cudaStream_t s);
int logdet_impl(bta_ctx_t ctx, int which, double* out, cudaStream_t s);
int solve_impl(bta_ctx_t ctx, int which, const double* rhs, double* x, cudaStream_t s);
int matvec_impl(bta_ctx_t ctx, int which, const double* x, double* y, cudaStream_t s);
int assemble_impl(bta_ctx_t ctx, bta_model_t m, const double* params, int which, cudaStream_t s);
int theta_to_params_impl(bta_model_t m, const double* theta, double* params, cudaStream_t s);
int ensure_sigma(bta_ctx_t ctx, int which);
int selinv_impl(bta_ctx_t ctx, int which, cudaStream_t s);
int axpby64(cudaStream_t s, long long len, double alpha, const double* x, double beta, const double* y,
            double* out);
