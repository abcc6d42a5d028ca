// Internal declarations shared by the CUDA sources of libbta.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "bta.h"

#define BTA_MAX_NV 8
// doubles per parameter slot: [kappa, tau, rho, sigma, tau_eps] x nv + lambda
#define BTA_PSTRIDE (5 * BTA_MAX_NV + BTA_MAX_NV * BTA_MAX_NV)

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

// Raise kernel `fn`'s dynamic shared-memory limit to at least `bytes` on the
// current device.  The attribute is per device and context, so the setting is
// remembered per (kernel, device); thread safe.
int ensure_dyn_smem(const void* fn, int bytes);

// Every kernel launch of the library is followed by BTA_LAUNCH_CHECK(): it
// counts the launch (bta_launch_count) and turns a launch error into a code.
void bta_note_launch();
void bta_note_launches(long long delta);   // graph replays and captures
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
    // per observation k (non-Gaussian likelihoods): tv = t nv + v, the three
    // triangle nodes and barycentric weights, the positions of the nine
    // products w_q w_r in the Gram pattern of (t, v), covariates and y
    int* obs_tv;             // m
    int* obs_s;              // 3 m
    double* obs_w;           // 3 m
    int* obs_gpos;           // 9 m
    double* obs_X;           // m nr
    double* obs_y;           // m
};

// ---------------------------------------------------------------- dense GEMM descriptor
// C = alpha op(A) op(B) + beta Cin for `batch` independent products whose
// operands are `sA`, `sB`, `sCi`, `sC` elements apart.
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
    void* ws;          // digit workspace (mixed path), for all matrices of a batch
    size_t ws_bytes;
    int* err;          // device error flag of the tensor-core kernel
    int min_dim;       // smallest M, N (and K) sent to the tensor-core path
    int df_leaf = 0;   // > 0: diagonal leaves of this order in double-float (leaf_df32.cu)
    int slices = 5;    // digit slices of the split products: 5 (35 bits) or 7 (49 bits)
    long long epi_wait = 0;   // wait limit of the tensor kernel's epilogue hand-off (0: default)
    int tile = 0;      // tile configuration of the split product (autotuned)
    int occupancy = 1; // waves of the persistent split-product grid before a K split (autotuned)
    int fp64_ctas = 2; // CTAs per SM the FP64 GEMM aims for through its K split (autotuned)
    // row tiles per band of the split product's tile order, for products with a
    // triangular operand, for general ones and for lower-triangle outputs
    // (autotuned; 1 = row by row)
    int band_tri = 1;
    int band_gen = 8;
    int band_low = 1;
};

// Side stream, events and executor for the products of the recursive
// diagonal-block factorisation that lie off its critical path.
constexpr int CHOL_FORK_DEPTH = 8;
struct CholFork {
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev[2 * CHOL_FORK_DEPTH] = {};
    GemmExec ex2{};   // the context's executor with a digit workspace of its own
    // third stream for the FP64 arrow products of the block recurrences,
    // which are off the critical path of the diagonal chain
    cudaStream_t s3 = nullptr;
    cudaEvent_t ev3_fork = nullptr, ev3_join = nullptr;
};

// ---------------------------------------------------------------- BTA storage
// `nmat` BTA matrices of one shape, matrix after matrix: the blocks of matrix
// m start at D + m sD, B + m sB, R + m sR, T + m sT.
struct BtaStore {
    double* D = nullptr;     // n * b * b per matrix
    double* B = nullptr;     // (n-1) * b * b
    double* R = nullptr;     // n * a * b
    double* T = nullptr;     // a * a
    long long sD = 0, sB = 0, sR = 0, sT = 0;
    // elements between the allocation and D, B, R (a leading padding block of
    // the time-partitioned layout; 0 otherwise)
    long long oD = 0, oB = 0, oR = 0;
};

// Scratch vectors: row r of matrix m is vec + (r * nmat + m) * N.
enum { VEC_RCOPY = 0, VEC_RES, VEC_CORR, VEC_Z, VEC_TMP, VEC_RHS, VEC_MU, VEC_ROWS };

struct bta_ctx_s {
    int n, b, a, precision;
    // block slots per matrix in the D, B, R and L^{-1} arrays: n (n - 1 for B)
    // normally, P h (with one leading padding slot) when time-partitioned
    int blk = 0;
    long long tip_off = 0;   // elements from a matrix's L^{-1} blocks to its L_tt^{-1}
    int batch;               // parameter slots; matrix storage index m = kind * batch + slot
    int nmat;                // 2 * batch
    long long N;
    cudaStream_t stream;
    cudaStream_t aux;        // second stream for a partial batch (Q_p beside Q_c)
    CholFork* fork = nullptr;  // side stream of the diagonal-block recursion
    cudaEvent_t ev_fork, ev_join;
    BtaStore Q, L, S;
    double* Linv = nullptr;  // per matrix: n b^2, then a^2 (tip)
    long long sLinv = 0;
    double* work = nullptr;  // per-matrix scratch of the factor / selinv
    long long sWork = 0;
    double* vec = nullptr;   // VEC_ROWS x nmat x N
    double* red = nullptr;   // reduction partials
    int red_chunks = 0;      // partial sums per matrix
    double* ld = nullptr;    // log-determinant of every matrix (nmat)
    double* dots = nullptr;  // per-matrix scalars: [0] b^T mu, [1] |r|^2, [2] |b|^2 (3 x nmat)
    long long* status;       // [0] error code, [1] row, [2] matrix (public index)
    double* params;          // parameter slots (batch x BTA_PSTRIDE)
    GemmExec exec;
    int* oz_err = nullptr;   // device flag of the tensor-core GEMM (time-out)
    int refine = 0;          // refinement steps of the f_obj solve
    std::vector<int> factored;   // per storage index
    std::vector<int> mu_valid;   // per slot: an f_obj evaluation has left mu (and b) there
    int leaf;                // leaf size of the recursive diagonal factorisation
    long long last_info = -1;
    int last_matrix = -1;
    // CUDA graph of one full f_obj group (batch thetas), replayed with the
    // thetas staged in theta_buf and the values written to f_buf
    cudaGraphExec_t fobj_graph = nullptr;
    const void* graph_model = nullptr;
    int graph_calls = 0;     // full groups evaluated so far (the first runs uncaptured)
    long long graph_kernels = 0;   // kernel nodes of the captured graph
    int use_graph = 1;
    double* theta_buf = nullptr;   // batch x dim_theta (dim <= BTA_PSTRIDE)
    double* f_buf = nullptr;       // batch
    double* adj = nullptr;         // adjoint trace records (3 x batch)
    // device staging of the host-buffer entry point (allocated on first use)
    double* hs_theta = nullptr;    // batch x dim_theta
    double* hs_f = nullptr;        // batch
    double* hs_grad = nullptr;     // batch x dim_theta
    double* hs_var = nullptr;      // batch x N
    int hs_dim = 0;
    // low-memory layout (bta_set_low_memory): the factor's D array has a spare
    // slot per matrix, the inverse blocks X_i replace L_ii in it (Linv aliases
    // L.D) and the selected inverse overwrites the factor (S aliases L)
    int lowmem = 0;
    double* xtmp = nullptr;   // nmat b^2: X of the block being factored, X_i copy of the selected inversion
    double* ldacc = nullptr;  // nmat: 2 sum log diag(L_ii), accumulated while the blocks are factored
    // parallel-in-time path (bta_set_time_partitions): P > 1 time partitions
    int tparts = 1;
    struct PTimeStore* pts = nullptr;
    // workspace of the Laplace evaluation (allocated on first use)
    double* lap = nullptr;         // per slot: obs weights, obs rhs terms, log-likelihood terms, x_new, params
    long long lap_slot = 0;        // doubles per slot
    const void* lap_model = nullptr;
    // optional event timing of the b x b x b Schur-update GEMM launches
    int prof = 0;
    std::vector<cudaEvent_t> prof_ev;   // pairs (start, stop)
    size_t prof_used = 0;
    double prof_flops = 0.0;
    // phase boundaries of the last full-group gradient evaluation (profiling on):
    // [0] start, [1] assembled, [2] factored + log-det, [3] f (solve, refinement),
    // [4] selected inversions, [5] adjoint traces and gradient
    cudaEvent_t phase_ev[BTA_PHASES + 1] = {};
    int phase_seen = 0;      // bit k: boundary k recorded since profiling was enabled
};

// boundary k of the phase timing, when profiling is on (fobj.cu, adjoint.cu)
int prof_phase(bta_ctx_t ctx, int k, cudaStream_t s);

// public matrix index (2 slot + kind) <-> storage index (kind batch + slot)
inline int storage_index(const bta_ctx_s* c, int which) {
    if (which < 0 || which >= 2 * c->batch) return -1;
    return (which % 2) * c->batch + which / 2;
}
inline int public_index(const bta_ctx_s* c, int m) { return 2 * (m % c->batch) + m / c->batch; }

// Record an event pair around the next launch on stream s when profiling.
int prof_begin(bta_ctx_t ctx, cudaStream_t s, double flops, cudaEvent_t* stop_out);
int prof_record(cudaEvent_t e, cudaStream_t s);

// ---------------------------------------------------------------- FP64 dense kernels (dense64.cu)
int gemm64(cudaStream_t s, const Gemm64& g, int ctas_per_sm = 2);
int gemm_exec(const GemmExec* ex, cudaStream_t s, const Gemm64& g);

// Recursive Cholesky + inverse of `batch` lower n x n matrices (strides sA, sX;
// scratch W with stride sW).  status receives the first non-positive pivot:
// row row0 + k of the matrix with storage index m_first + instance, reported
// by its public index for a context of `nbatch` parameter slots.
// With `fork`, the product L21 X11 of every recursion node (independent of
// the factorisation of A22) runs on fork->s2 with its own digit workspace,
// joined back before X21 is formed; the subtrees then need about n^2/3 of
// scratch per matrix instead of n^2/4.
struct CholFork;
int chol_inv64(cudaStream_t s, double* A, long long lda, double* X, long long ldx, int n,
               long long row0, long long* status, double* W, int leaf, const GemmExec* ex = nullptr,
               int batch = 1, long long sA = 0, long long sX = 0, long long sW = 0, int m_first = 0,
               int nbatch = 1, const CholFork* fork = nullptr, int depth = 0, int per = 1);
// Double-float Cholesky + inverse of `batch` blocks of order n <= 128 (leaf_df32.cu).
int chol_inv_df32_launch(cudaStream_t s, double* A, long long lda, long long sA, double* X, long long ldx,
                         long long sX, int n, long long row0, long long* status, int batch, int m_first,
                         int nbatch, int per = 1);
// C = beta Cin + alpha op(A) op(B) in double-float on the FP32 pipe (leaf_df32.cu)
int gemm_df32(cudaStream_t s, const Gemm64& g);
int copy_mat64(cudaStream_t s, const double* src, long long lds, double* dst, long long ldd,
               int rows, int cols, int lower_only, int batch = 1, long long ss = 0, long long sd = 0);
// C = beta Cin (C = 0 if beta == 0); only entries m >= n when lower
int scale_into64(cudaStream_t s, int M, int N, const double* Cin, long long ldci, double beta, double* C,
                 long long ldc, int lower, int batch = 1, long long sCi = 0, long long sC = 0);
int symmetrize_lower64(cudaStream_t s, double* A, long long lda, int n, int batch = 1, long long sA = 0);
// y = alpha * op(A) x + beta * yin   (op(A) shape: 0 general, 1 lower, 2 upper)
int gemv64(cudaStream_t s, int M, int N, const double* A, long long lda, int ta, int sh,
           const double* x, double alpha, const double* yin, double beta, double* y, int batch = 1,
           long long sA = 0, long long sx = 0, long long sy = 0);
// out[m] = scale * (sum_k log A_m[k (lda+1)] over `nblk` diagonal blocks of
// dimension dim spaced by `stride`, + sum_k log T_m[k (a+1)] over the tip)
int logdet_batch64(cudaStream_t s, const double* A, long long lda, int dim, int nblk, long long stride,
                   long long sA, const double* T, int a, long long sT, int count, double* partial,
                   int chunks, double* out, double scale);
// out[m * ostride] = sum_i x_m[i] y_m[i] for `count` vector pairs of length len
int dot_batch64(cudaStream_t s, const double* x, const double* y, long long len, int count, double* partial,
                int chunks, double* out, long long ostride);

// ---------------------------------------------------------------- tensor cores (ozaki.cu)
size_t ozaki_workspace_bytes(int M, int N, int K, int slices);
// same contract as gemm64 (any batch); ws holds batch x ozaki_workspace_bytes;
// slices = 5 (35-bit digits) or 7 (49-bit digits)
// tile: 0 (128 x 96, 2 stages) or 1 (128 x 64, 3 stages) for 5 slices; 7 slices
// use 128 x 64, 2 stages.  occupancy: waves of the persistent grid below
// which the K dimension is split.
int ozaki_gemm(cudaStream_t s, const Gemm64& g, void* ws, int* err, int slices, long long epi_wait = 0,
               int tile = 0, int occupancy = 1, int band = 1);
int ozaki_tiles_for(int slices, int* out, int cap);
int gemm_mixed_fn(const GemmExec* ex, cudaStream_t s, const Gemm64& g);
// true when gemm_exec sends g to the split-precision path, whose operands are
// read completely (digit split) before C is written: C may then alias A or B
bool gemm_mixed_takes(const GemmExec* ex, const Gemm64& g);

// ---------------------------------------------------------------- entry points on matrices m0 .. m0+count-1
int factor_impl(bta_ctx_t ctx, int m0, int count, cudaStream_t s);
int logdet_impl(bta_ctx_t ctx, int m0, int count, double* out, cudaStream_t s);
// x_j = Q_{m0+j}^{-1} r_j, vectors N apart
int solve_impl(bta_ctx_t ctx, int m0, int count, const double* r, double* x, cudaStream_t s);
int matvec_impl(bta_ctx_t ctx, int m0, int count, const double* x, double* y, cudaStream_t s);
int selinv_impl(bta_ctx_t ctx, int m0, int count, cudaStream_t s);
// the same over P > 1 time partitions (ptime.cu), used when ctx->tparts > 1
int pfactor_impl(bta_ctx_t ctx, int m0, int count, cudaStream_t s);
int psolve_impl(bta_ctx_t ctx, int m0, int count, const double* r, double* x, cudaStream_t s);
int pselinv_impl(bta_ctx_t ctx, int m0, int count, cudaStream_t s);
void ptime_free(bta_ctx_t ctx);
// assemble matrices m0.. (kind = m / batch, parameters of slot m % batch at
// params + slot * BTA_PSTRIDE)
int assemble_impl(bta_ctx_t ctx, bta_model_t m, const double* params, int m0, int count, cudaStream_t s);
// The observation terms A^T D A of Q_c with a weight per observation and slot
// (layouts of bta_model_s::gram / arrow / tipgram, one copy per slot).
struct ObsWeights {
    const double* gram;  const double* arrow;  const double* tip;
    long long gram_stride, arrow_stride, tip_stride;
};
int assemble_weighted_impl(bta_ctx_t ctx, bta_model_t m, const double* params, int m0, int count, cudaStream_t s,
                           const ObsWeights& w);
// theta (count x dim_theta) -> parameter slots (count x BTA_PSTRIDE)
int theta_to_params_impl(bta_model_t m, const double* theta, int count, double* params, cudaStream_t s);
int ensure_sigma(bta_ctx_t ctx);
// (re)allocation of a block store with `blk` slots per matrix and `lead`
// leading padding slots (api.cu); store_release frees it
int store_alloc(BtaStore& M, int nmat, int n, int b, int a, int blk, int lead);
void store_release(BtaStore& M);
int axpby64(cudaStream_t s, long long len, double alpha, const double* x, double beta, const double* y,
            double* out);
inline double* vec_row(bta_ctx_t c, int row, int m) { return c->vec + ((long long)row * c->nmat + m) * c->N; }
