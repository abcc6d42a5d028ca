// FP64 dense building blocks of the BTA factorisation, solve and selected
// inversion: a tiled DFMA GEMM with triangular-operand and lower-output
// variants, the recursive diagonal-block Cholesky + inverse, matrix copies,
// GEMV and deterministic reductions, all batched over independent matrices
// (blockIdx.z / blockIdx.y = matrix).  On GB300 the FP64 pipe (measured
// 1.2 TFLOP/s for DFMA, 1.05 for DMMA) bounds the GEMM and the Cholesky;
// the GEMV and copies are bound by HBM.

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace {

// ---------------------------------------------------------------- GEMM
// Tile (16 MI) x (16 NJ) x 16 per CTA of 256 threads; thread (tx, ty),
// tx = tid % 16 along m, ty = tid / 16 along n, owns rows m0 + tx + 16 i and
// columns n0 + ty + 16 j.  Column-major output: lanes write consecutive rows.
// blockIdx.z = matrix * ksplit + split; with ksplit > 1 every split atomically
// adds alpha * partial into a C that already holds beta Cin.
constexpr int BK = 16, GT = 256;

__device__ __forceinline__ double load_opA(const Gemm64& p, const double* A, int m, int k, int kend) {
    if (m >= p.M || k >= kend) return 0.0;
    if (p.shA == 1 && k > m) return 0.0;
    if (p.shA == 2 && k < m) return 0.0;
    return p.ta ? A[k + (long long)m * p.lda] : A[m + (long long)k * p.lda];
}

__device__ __forceinline__ double load_opB(const Gemm64& p, const double* B, int k, int nn, int kend) {
    if (nn >= p.N || k >= kend) return 0.0;
    if (p.shB == 1 && nn > k) return 0.0;
    if (p.shB == 2 && nn < k) return 0.0;
    return p.tb ? B[nn + (long long)k * p.ldb] : B[k + (long long)nn * p.ldb];
}

template <int MI, int NJ, int BKT = BK>
__global__ void __launch_bounds__(GT) gemm64_kernel(Gemm64 p, int ksplit) {
    constexpr int TBM = 16 * MI, TBN = 16 * NJ;
    __shared__ double As[BKT][TBM + 1];
    __shared__ double Bs[BKT][TBN + 1];
    const int m0 = blockIdx.x * TBM, n0 = blockIdx.y * TBN;
    if (p.lowerC && m0 + TBM - 1 < n0) return;
    const int z = blockIdx.z / ksplit, split = blockIdx.z % ksplit;
    const double* A = p.A + z * p.sA;
    const double* B = p.B + z * p.sB;
    const double* Cin = p.Cin ? p.Cin + z * p.sCi : nullptr;
    double* C = p.C + z * p.sC;
    int kb = 0, ke = p.K;
    if (p.shA == 1) ke = min(ke, m0 + TBM);
    if (p.shA == 2) kb = max(kb, m0);
    if (p.shB == 1) kb = max(kb, n0);
    if (p.shB == 2) ke = min(ke, n0 + TBN);
    kb = (kb / BKT) * BKT;
    if (ksplit > 1) {
        // split [kb, ke) into ksplit chunks of whole BKT tiles
        const int tiles = (ke - kb + BKT - 1) / BKT;
        const int per = (tiles + ksplit - 1) / ksplit;
        const int s0 = kb + split * per * BKT;
        const int s1 = min(ke, s0 + per * BKT);
        kb = s0;
        ke = s1;
        if (kb >= ke) return;
    }
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    double acc[MI][NJ];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[i][j] = 0.0;

    for (int k0 = kb; k0 < ke; k0 += BKT) {
        // op(A) tile TBM x BKT: lanes along the contiguous stored dimension
        for (int e = tid; e < TBM * BKT; e += GT) {
            int mm, kk;
            if (!p.ta) { mm = e % TBM; kk = e / TBM; } else { kk = e % BKT; mm = e / BKT; }
            As[kk][mm] = load_opA(p, A, m0 + mm, k0 + kk, ke);
        }
        for (int e = tid; e < TBN * BKT; e += GT) {
            int nn, kk;
            if (!p.tb) { kk = e % BKT; nn = e / BKT; } else { nn = e % TBN; kk = e / TBN; }
            Bs[kk][nn] = load_opB(p, B, k0 + kk, n0 + nn, ke);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BKT; ++kk) {
            double a[MI], b[NJ];
#pragma unroll
            for (int i = 0; i < MI; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < NJ; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int nn = n0 + ty + 16 * j;
        if (nn >= p.N) continue;
#pragma unroll
        for (int i = 0; i < MI; ++i) {
            const int mm = m0 + tx + 16 * i;
            if (mm >= p.M) continue;
            if (p.lowerC && mm < nn) continue;
            double* c = C + mm + (long long)nn * p.ldc;
            if (ksplit > 1) {
                atomicAdd(c, p.alpha * acc[i][j]);
            } else {
                double v = p.alpha * acc[i][j];
                if (p.beta != 0.0) v += p.beta * Cin[mm + (long long)nn * p.ldci];
                *c = v;
            }
        }
    }
}

// Thin GEMM for op(A) with at most 16 rows (the arrow products
// L_{t,i} = R X^T, R -= L_t L_B^T, F = L_t X, Sigma_t G of a BTA matrix with a
// narrow arrowhead).  A 16-row tile of the kernel above would spend 3/4 of
// its DFMAs on padding rows when M = 4.  Here a CTA owns 64 columns; warp w
// works on columns n0 + 32 (w & 1) + lane and rows R g .. R g + R - 1 of row
// group g = w / 2, so a row group beyond M is a whole idle warp and every
// DFMA issued is a useful one.  The op(A) chunk is read from shared memory as
// a broadcast, the op(B) chunk is staged coalesced for either stride order.
constexpr int TH_TN = 64, TH_BK = 32;

template <int R>
__global__ void __launch_bounds__(GT) gemm64_thin_kernel(Gemm64 p, int ksplit) {
    constexpr int TM = 4 * R;
    __shared__ double As[TH_BK][TM];
    __shared__ double Bs[TH_BK][TH_TN + 1];
    const int n0 = blockIdx.x * TH_TN;
    const int z = blockIdx.y / ksplit, split = blockIdx.y % ksplit;
    const double* A = p.A + z * p.sA;
    const double* B = p.B + z * p.sB;
    const double* Cin = p.Cin ? p.Cin + z * p.sCi : nullptr;
    double* C = p.C + z * p.sC;
    int kb = 0, ke = p.K;
    if (p.shA == 1) ke = min(ke, p.M);
    if (p.shB == 1) kb = max(kb, n0);
    if (p.shB == 2) ke = min(ke, n0 + TH_TN);
    kb = (kb / TH_BK) * TH_BK;
    if (ksplit > 1) {
        const int tiles = (ke - kb + TH_BK - 1) / TH_BK;
        const int per = (tiles + ksplit - 1) / ksplit;
        const int s0 = kb + split * per * TH_BK;
        const int s1 = min(ke, s0 + per * TH_BK);
        kb = s0;
        ke = s1;
        if (kb >= ke) return;
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = warp >> 1, col = (warp & 1) * 32 + lane;
    const bool active = grp * R < p.M;        // warp-uniform
    double acc[R];
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = 0.0;
    for (int k0 = kb; k0 < ke; k0 += TH_BK) {
        for (int e = tid; e < TM * TH_BK; e += GT) {
            int mm, kk;
            if (!p.ta) { mm = e % TM; kk = e / TM; } else { kk = e % TH_BK; mm = e / TH_BK; }
            As[kk][mm] = load_opA(p, A, mm, k0 + kk, ke);
        }
        for (int e = tid; e < TH_TN * TH_BK; e += GT) {
            int nn, kk;
            if (!p.tb) { kk = e % TH_BK; nn = e / TH_BK; } else { nn = e % TH_TN; kk = e / TH_TN; }
            Bs[kk][nn] = load_opB(p, B, k0 + kk, n0 + nn, ke);
        }
        __syncthreads();
        if (active) {
#pragma unroll 8
            for (int kk = 0; kk < TH_BK; ++kk) {
                const double bv = Bs[kk][col];
#pragma unroll
                for (int i = 0; i < R; ++i) acc[i] = fma(As[kk][grp * R + i], bv, acc[i]);
            }
        }
        __syncthreads();
    }
    const int nn = n0 + col;
    if (!active || nn >= p.N) return;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int mm = grp * R + i;
        if (mm >= p.M) continue;
        if (p.lowerC && mm < nn) continue;
        double* c = C + mm + (long long)nn * p.ldc;
        if (ksplit > 1) {
            atomicAdd(c, p.alpha * acc[i]);
        } else {
            double v = p.alpha * acc[i];
            if (p.beta != 0.0) v += p.beta * Cin[mm + (long long)nn * p.ldci];
            *c = v;
        }
    }
}

// C = beta Cin (entries m >= n only when lower), the start of a split-K GEMM.
// blockIdx.y = matrix.
__global__ void scale_into_kernel(int M, int N, const double* Cin, long long ldci, double beta, double* C,
                                  long long ldc, int lower, long long sCi, long long sC) {
    const long long total = (long long)M * N;
    C += blockIdx.y * sC;
    if (Cin) Cin += blockIdx.y * sCi;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % M), j = (int)(e / M);
        if (lower && i < j) continue;
        C[i + j * ldc] = (beta != 0.0 && Cin) ? beta * Cin[i + j * ldci] : 0.0;
    }
}

// ---------------------------------------------------------------- leaf Cholesky + inverse
// One CTA per matrix factors an n x n (n <= 64) lower block A = L L^T in
// shared memory and forms X = L^{-1} by right-looking forward elimination of
// L X = I.  Iteration k updates the trailing matrix with column k of L and
// eliminates with column k-1, so each iteration needs one barrier.  The
// reciprocal square root of pivot k+1 is computed by the thread that finishes
// that pivot in iteration k (Newton-Raphson for 1/sqrt, seeded in FP32), so
// no FP64 division or square root sits on the critical path: FP64 latency,
// not throughput, bounds this kernel on GB300.  Output: L and X (lower; the
// strict upper parts of both tiles are written as zeros).
constexpr int LEAF_MAX = 64;
constexpr int LDS = LEAF_MAX + 1;

// 1/sqrt(d) by two Newton-Raphson steps y <- y (3 - d y^2) / 2 from an FP32
// estimate, after scaling d by an even power of two into [1, 4); NaN unless
// d > 0.
__device__ __forceinline__ double newton_rsqrt(double d) {
    if (!(d > 0.0) || isinf(d)) return nan("");
    const int e = ilogb(d) & ~1;
    const double m = ldexp(d, -e);
    double y = (double)rsqrtf((float)m);
    y = y * (1.5 - 0.5 * m * y * y);
    y = y * (1.5 - 0.5 * m * y * y);
    return ldexp(y, -e / 2);
}

__global__ void __launch_bounds__(256) chol_inv_leaf_kernel(double* A, long long lda, long long sA, double* X,
                                                            long long ldx, long long sX, int n, long long row0,
                                                            long long* status, int m_first, int nbatch,
                                                            int per) {
    extern __shared__ double sm[];
    double* S = sm;                 // working matrix, column-major, ld LDS
    double* L = sm + LDS * LEAF_MAX;
    double* W = sm + 2 * LDS * LEAF_MAX;
    double* ys = sm + 3 * LDS * LEAF_MAX;   // 1/L_kk
    A += blockIdx.x * sA;
    X += blockIdx.x * sX;
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    for (int e = tid; e < n * n; e += nthr) {
        int i = e % n, j = e / n;
        S[j * LDS + i] = (i >= j) ? A[i + (long long)j * lda] : 0.0;
        W[j * LDS + i] = (i == j) ? 1.0 : 0.0;
        L[j * LDS + i] = 0.0;
    }
    __syncthreads();
    if (tid == 0) ys[0] = newton_rsqrt(S[0]);
    const int rows_per = n <= 32 ? 32 : LEAF_MAX;
    const int row = tid % rows_per;      // row handled by this thread
    const int lane_q = tid / rows_per;   // column phase
    const int nq = nthr / rows_per;
    for (int k = 0; k <= n; ++k) {
        __syncthreads();
        if (k < n) {
            const double y = ys[k];
            if (tid == 0 && !(y > 0.0) && status) {
                if (atomicCAS((unsigned long long*)status, 0ull, (unsigned long long)BTA_ERR_NOT_PD) == 0ull) {
                    status[1] = row0 + k;
                    const int mm = m_first + (int)blockIdx.x / per;   // storage index -> public index
                    status[2] = 2 * (mm % nbatch) + mm / nbatch;
                }
            }
            if (row >= k && row < n && lane_q == 0) L[k * LDS + row] = S[k * LDS + row] * y;
            if (row > k && row < n) {
                const double sik = S[k * LDS + row] * (y * y);
                for (int j = k + 1 + lane_q; j <= row; j += nq) {
                    const double v = S[j * LDS + row] - sik * S[k * LDS + j];
                    S[j * LDS + row] = v;
                    if (j == k + 1 && row == k + 1) ys[k + 1] = newton_rsqrt(v);   // next pivot is final
                }
            }
        }
        if (k > 0) {
            const int c = k - 1;   // eliminate with column c of L (complete since iteration c)
            const double yc = ys[c];
            if (row > c && row < n) {
                const double f = L[c * LDS + row] * yc;
                for (int j = lane_q; j <= c; j += nq) W[j * LDS + row] -= f * W[j * LDS + c];
            }
            // row c of X is final: W[c][:] / L[c][c]
            if (tid <= c) X[c + (long long)tid * ldx] = W[tid * LDS + c] * yc;
        }
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nthr) {
        int i = e % n, j = e / n;
        A[i + (long long)j * lda] = (i >= j) ? L[j * LDS + i] : 0.0;
        if (i < j) X[i + (long long)j * ldx] = 0.0;
    }
}

// ---------------------------------------------------------------- copies (blockIdx.y = matrix)
__global__ void copy_mat_kernel(const double* src, long long lds, double* dst, long long ldd, int rows,
                                int cols, int lower_only, long long ss, long long sd) {
    src += blockIdx.y * ss;
    dst += blockIdx.y * sd;
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % rows), j = (int)(e / rows);
        if (lower_only && i < j) continue;
        dst[i + j * ldd] = src[i + j * lds];
    }
}

__global__ void symmetrize_kernel(double* A, long long lda, int n, long long sA) {
    A += blockIdx.y * sA;
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        if (i < j) A[i + j * lda] = A[j + i * lda];
    }
}

// ---------------------------------------------------------------- GEMV (blockIdx.y = matrix)
// y[m] = alpha sum_n op(A)[m][n] x[n] + beta yin[m].  These are HBM-bound
// (each element of A is read once), so what matters is enough loads in flight:
//   non-transposed: a CTA of 32 warps owns 32 rows; lanes read consecutive rows
//     (256-byte segments), warps split the columns, and each thread keeps four
//     columns in flight with independent accumulators;
//   transposed: a warp owns one output and its lanes stride down the stored
//     column (coalesced), four loads in flight, shuffle reduction;
//   short rows (non-transposed, M <= 16, the arrow rows R of a BTA matrix
//     against a vector of length n b): one CTA of 1024 threads per matrix,
//     each thread taking whole columns of M contiguous values;
//   short columns (transposed, N <= 16, R^T x_t): one thread per output.
constexpr int GV_WARPS = 32;
constexpr int GV_SHORT = 16;

__global__ void __launch_bounds__(32 * GV_WARPS) gemv_n_kernel(int M, int N, const double* A, long long lda,
                                                              int sh, const double* x, double alpha,
                                                              const double* yin, double beta, double* y,
                                                              long long sA, long long sx, long long sy) {
    __shared__ double part[GV_WARPS][33];
    A += blockIdx.y * sA;
    x += blockIdx.y * sx;
    y += blockIdx.y * sy;
    if (yin) yin += blockIdx.y * sy;
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    const int m = blockIdx.x * 32 + lane;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (m < M) {
        int nb = 0, ne = N;
        if (sh == 1) ne = min(N, m + 1);
        if (sh == 2) nb = m;
        const double* Am = A + m;
        int n = nb + w;
        for (; n + 3 * GV_WARPS < ne; n += 4 * GV_WARPS) {
            a0 = fma(Am[(long long)n * lda], x[n], a0);
            a1 = fma(Am[(long long)(n + GV_WARPS) * lda], x[n + GV_WARPS], a1);
            a2 = fma(Am[(long long)(n + 2 * GV_WARPS) * lda], x[n + 2 * GV_WARPS], a2);
            a3 = fma(Am[(long long)(n + 3 * GV_WARPS) * lda], x[n + 3 * GV_WARPS], a3);
        }
        for (; n < ne; n += GV_WARPS) a0 = fma(Am[(long long)n * lda], x[n], a0);
    }
    part[w][lane] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    if (w == 0 && m < M) {
        double s = 0.0;
        for (int q = 0; q < GV_WARPS; ++q) s += part[q][lane];
        double v = alpha * s;
        if (beta != 0.0) v += beta * yin[m];
        y[m] = v;
    }
}

__global__ void __launch_bounds__(256) gemv_t_kernel(int M, int N, const double* A, long long lda, int sh,
                                                     const double* x, double alpha, const double* yin,
                                                     double beta, double* y, long long sA, long long sx,
                                                     long long sy) {
    // op(A) = A^T: op(A)[m][n] = A[n + m*lda], op(A) is M x N, A stored N x M.
    A += blockIdx.y * sA;
    x += blockIdx.y * sx;
    y += blockIdx.y * sy;
    if (yin) yin += blockIdx.y * sy;
    const int lane = threadIdx.x % 32;
    const int m = blockIdx.x * 8 + threadIdx.x / 32;
    if (m >= M) return;
    int nb = 0, ne = N;
    if (sh == 1) ne = min(N, m + 1);
    if (sh == 2) nb = m;
    const double* col = A + (long long)m * lda;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int n = nb + lane;
    for (; n + 96 < ne; n += 128) {
        a0 = fma(col[n], x[n], a0);
        a1 = fma(col[n + 32], x[n + 32], a1);
        a2 = fma(col[n + 64], x[n + 64], a2);
        a3 = fma(col[n + 96], x[n + 96], a3);
    }
    for (; n < ne; n += 32) a0 = fma(col[n], x[n], a0);
    double acc = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        double v = alpha * acc;
        if (beta != 0.0) v += beta * yin[m];
        y[m] = v;
    }
}

// M <= GV_SHORT rows, general op(A) shape only
__global__ void __launch_bounds__(1024) gemv_short_n_kernel(int M, int N, const double* A, long long lda,
                                                            const double* x, double alpha, const double* yin,
                                                            double beta, double* y, long long sA, long long sx,
                                                            long long sy) {
    __shared__ double red[GV_SHORT][33];
    A += blockIdx.y * sA;
    x += blockIdx.y * sx;
    y += blockIdx.y * sy;
    if (yin) yin += blockIdx.y * sy;
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    double acc[GV_SHORT];
#pragma unroll
    for (int i = 0; i < GV_SHORT; ++i) acc[i] = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const double xn = x[n];
        const double* c = A + (long long)n * lda;
#pragma unroll
        for (int i = 0; i < GV_SHORT; ++i)
            if (i < M) acc[i] = fma(c[i], xn, acc[i]);
    }
#pragma unroll
    for (int i = 0; i < GV_SHORT; ++i) {
        if (i >= M) break;
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[i][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < M) {
        const int i = threadIdx.x;
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x / 32); ++q) s += red[i][q];
        double v = alpha * s;
        if (beta != 0.0) v += beta * yin[i];
        y[i] = v;
    }
}

// N <= GV_SHORT columns of op(A) = A^T, general shape only
__global__ void __launch_bounds__(256) gemv_short_t_kernel(int M, int N, const double* A, long long lda,
                                                           const double* x, double alpha, const double* yin,
                                                           double beta, double* y, long long sA, long long sx,
                                                           long long sy) {
    A += blockIdx.y * sA;
    x += blockIdx.y * sx;
    y += blockIdx.y * sy;
    if (yin) yin += blockIdx.y * sy;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double* r = A + (long long)m * lda;
    double s = 0.0;
    for (int n = 0; n < N; ++n) s = fma(r[n], x[n], s);
    double v = alpha * s;
    if (beta != 0.0) v += beta * yin[m];
    y[m] = v;
}

// ---------------------------------------------------------------- reductions (blockIdx.y = matrix)
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        s = (lane < (int)(blockDim.x / 32)) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

__global__ void logdiag_partial_kernel(const double* A, long long lda, int dim, int nblk, long long stride,
                                       long long sA, double* partial) {
    A += blockIdx.y * sA;
    const long long total = (long long)dim * nblk;
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int blk = (int)(e / dim), k = (int)(e % dim);
        acc += log(A[blk * stride + k * (lda + 1)]);
    }
    double s = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

__global__ void logdet_finish_kernel(const double* partial, int chunks, const double* T, int a, long long sT,
                                     double* out, double scale) {
    const int m = blockIdx.x;
    double acc = 0.0;
    for (int e = threadIdx.x; e < chunks; e += blockDim.x) acc += partial[m * chunks + e];
    if (T)
        for (int k = threadIdx.x; k < a; k += blockDim.x) acc += log(T[m * sT + k * (a + 1)]);
    double s = block_sum(acc);
    if (threadIdx.x == 0) out[m] = scale * s;
}

__global__ void dot_partial_kernel(const double* x, const double* y, long long len, double* partial) {
    x += blockIdx.y * len;
    y += blockIdx.y * len;
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
         e += (long long)gridDim.x * blockDim.x)
        acc = fma(x[e], y[e], acc);
    double s = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

__global__ void dot_finish_kernel(const double* partial, int chunks, double* out, long long ostride) {
    const int m = blockIdx.x;
    double acc = 0.0;
    for (int e = threadIdx.x; e < chunks; e += blockDim.x) acc += partial[m * chunks + e];
    double s = block_sum(acc);
    if (threadIdx.x == 0) out[m * ostride] = s;
}

}  // namespace

// ==================================================================== host launchers
static int gemm64_thin(cudaStream_t s, const Gemm64& g) {
    const int gn = (g.N + TH_TN - 1) / TH_TN;
    const long long ctas = (long long)gn * g.batch;
    const int kchunks = std::max(1, (g.K + TH_BK - 1) / TH_BK);
    // about four CTAs per SM; each split keeps at least two K chunks
    const long long want = 4LL * 152;
    int ksplit = (int)std::min<long long>(std::max(1, kchunks / 2), std::max<long long>(1, (want + ctas - 1) / ctas));
    if ((long long)g.batch * ksplit > 65535) ksplit = std::max(1, 65535 / g.batch);
    if (ksplit > 1) {
        const bool inplace = (g.Cin == g.C && g.ldci == g.ldc && g.beta == 1.0 && g.sCi == g.sC);
        if (!inplace) BTA_TRY(scale_into64(s, g.M, g.N, g.Cin, g.ldci, g.beta, g.C, g.ldc, g.lowerC, g.batch, g.sCi, g.sC));
    }
    dim3 grid(gn, g.batch * ksplit);
    const int R = (g.M + 3) / 4;
    if (R == 1) gemm64_thin_kernel<1><<<grid, GT, 0, s>>>(g, ksplit);
    else if (R == 2) gemm64_thin_kernel<2><<<grid, GT, 0, s>>>(g, ksplit);
    else if (R == 3) gemm64_thin_kernel<3><<<grid, GT, 0, s>>>(g, ksplit);
    else gemm64_thin_kernel<4><<<grid, GT, 0, s>>>(g, ksplit);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

int gemm64(cudaStream_t s, const Gemm64& g, int ctas_per_sm) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return BTA_OK;
    if (g.M <= 16 && g.N >= TH_TN) return gemm64_thin(s, g);
    if (g.K <= 8 && g.M > 32 && g.N > 32) {
        // rank-a updates of b x b blocks (Sigma -= Sigma_t^T F): one K tile of
        // the 64 x 64 kernel sized to K, no padding DFMAs, no split
        const int gm = (g.M + 63) / 64, gn = (g.N + 63) / 64;
        dim3 grid(gm, gn, g.batch);
        if (g.K <= 4) gemm64_kernel<4, 4, 4><<<grid, GT, 0, s>>>(g, 1);
        else gemm64_kernel<4, 4, 8><<<grid, GT, 0, s>>>(g, 1);
        BTA_LAUNCH_CHECK();
        return BTA_OK;
    }
    // The FP64 pipe of one SM is slow (2 DFMA per clock), so every product is
    // spread over about `ctas_per_sm` (default two, autotuned) CTAs per SM:
    // pick the largest micro-tile that still reaches that with a K split of
    // whole 16-wide slices, else the smallest tile with the largest split.
    const long long want = (long long)std::max(1, ctas_per_sm) * 152;
    int MI = 1, NJ = 1, ksplit = 1;
    const int kslices = std::max(1, (g.K + BK - 1) / BK);
    for (int sz = 4; sz >= 1; sz /= 2) {
        const int mi = std::min(sz, g.M <= 16 ? 1 : (g.M <= 32 ? 2 : 4));
        const int nj = std::min(sz, g.N <= 16 ? 1 : (g.N <= 32 ? 2 : 4));
        const int gm = (g.M + 16 * mi - 1) / (16 * mi), gn = (g.N + 16 * nj - 1) / (16 * nj);
        long long tiles = (long long)gm * gn;
        if (g.lowerC) tiles = (tiles + gm) / 2;
        tiles *= g.batch;
        const int maxsplit = std::min(64, std::max(1, kslices / (sz == 4 ? 4 : 2)));
        if (tiles * maxsplit >= want || sz == 1) {
            MI = mi;
            NJ = nj;
            ksplit = (int)std::min<long long>(maxsplit, std::max<long long>(1, (want + tiles - 1) / tiles));
            break;
        }
    }
    if ((long long)g.batch * ksplit > 65535) ksplit = std::max(1, 65535 / g.batch);
    const int TBM = 16 * MI, TBN = 16 * NJ;
    const int gm = (g.M + TBM - 1) / TBM, gn = (g.N + TBN - 1) / TBN;
    if (ksplit > 1) {
        const bool inplace = (g.Cin == g.C && g.ldci == g.ldc && g.beta == 1.0 && g.sCi == g.sC);
        if (!inplace) BTA_TRY(scale_into64(s, g.M, g.N, g.Cin, g.ldci, g.beta, g.C, g.ldc, g.lowerC, g.batch, g.sCi, g.sC));
    }
    dim3 grid(gm, gn, g.batch * ksplit);
#define BTA_GEMM_CASE(mi, nj) \
    if (MI == mi && NJ == nj) gemm64_kernel<mi, nj><<<grid, GT, 0, s>>>(g, ksplit);
    BTA_GEMM_CASE(1, 1) BTA_GEMM_CASE(1, 2) BTA_GEMM_CASE(1, 4)
    BTA_GEMM_CASE(2, 1) BTA_GEMM_CASE(2, 2) BTA_GEMM_CASE(2, 4)
    BTA_GEMM_CASE(4, 1) BTA_GEMM_CASE(4, 2) BTA_GEMM_CASE(4, 4)
#undef BTA_GEMM_CASE
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

int gemm_exec(const GemmExec* ex, cudaStream_t s, const Gemm64& g) {
    if (!ex) return gemm64(s, g);
    if (!ex->fn) return gemm64(s, g, ex->fp64_ctas);
    return ex->fn(ex, s, g);
}

static int leaf_launch(cudaStream_t s, double* A, long long lda, long long sA, double* X, long long ldx,
                       long long sX, int n, long long row0, long long* status, int batch, int m_first, int nbatch,
                       int per) {
    const size_t smem = (3 * LDS * LEAF_MAX + LEAF_MAX + 1) * sizeof(double);
    BTA_TRY(ensure_dyn_smem((const void*)chol_inv_leaf_kernel, (int)smem));
    const int threads = 256;
    chol_inv_leaf_kernel<<<batch, threads, smem, s>>>(A, lda, sA, X, ldx, sX, n, row0, status, m_first, nbatch, per);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

// Recursive Cholesky + inverse of the lower n x n matrix at A (in place) into
// X (lower), for `batch` matrices at once.  W: scratch of at least
// ceil(n/2)^2 + n doubles per matrix.
//   [A11      ]   L11 = chol(A11), X11 = L11^{-1}
//   [A21  A22 ]   L21 = A21 X11^T, A22 -= L21 L21^T, L22 = chol(A22), X22 = L22^{-1}
//                 X21 = -X22 (L21 X11)
int chol_inv64(cudaStream_t s, double* A, long long lda, double* X, long long ldx, int n, long long row0,
               long long* status, double* W, int leaf, const GemmExec* ex, int batch, long long sA,
               long long sX, long long sW, int m_first, int nbatch, const CholFork* fork, int depth, int per) {
    if (n <= 0 || batch <= 0) return BTA_OK;
    if (ex && ex->df_leaf > 0) {
        // mixed precision: double-float leaves on the FP32 pipe
        leaf = std::min(ex->df_leaf, 128);
        if (n <= leaf)
            return chol_inv_df32_launch(s, A, lda, sA, X, ldx, sX, n, row0, status, batch, m_first, nbatch, per);
    } else {
        leaf = std::max(8, std::min(leaf, LEAF_MAX));
        if (n <= leaf)
            return leaf_launch(s, A, lda, sA, X, ldx, sX, n, row0, status, batch, m_first, nbatch, per);
    }
    const int half = (n + 1) / 2;
    int n1 = ((half + leaf - 1) / leaf) * leaf;
    if (n1 >= n) n1 = leaf;
    const int n2 = n - n1;
    double* A11 = A;
    double* A21 = A + n1;
    double* A22 = A + n1 + n1 * lda;
    double* X11 = X;
    double* X21 = X + n1;
    double* X22 = X + n1 + n1 * ldx;
    // W (n2 x n1) belongs to this node while L21 X11 runs beside the subtree
    // of A22; the subtrees then use the scratch after it
    const bool forked = fork && fork->s2 && depth < CHOL_FORK_DEPTH;
    double* Wc = forked ? W + (long long)n2 * n1 : W;
    BTA_TRY(chol_inv64(s, A11, lda, X11, ldx, n1, row0, status, Wc, leaf, ex, batch, sA, sX, sW, m_first, nbatch,
                       fork, depth + 1, per));
    Gemm64 g{};
    // W (n2 x n1) = A21 * X11^T      (op(B) upper)
    g = Gemm64{};
    g.M = n2; g.N = n1; g.K = n1;
    g.A = A21; g.lda = lda; g.ta = 0; g.shA = 0;
    g.B = X11; g.ldb = ldx; g.tb = 1; g.shB = 2;
    g.C = W; g.ldc = n2; g.alpha = 1.0; g.beta = 0.0;
    g.batch = batch; g.sA = sA; g.sB = sX; g.sC = sW;
    if (gemm_mixed_takes(ex, g)) {
        // the split-precision product reads A21 completely before writing: in place
        g.C = A21; g.ldc = lda; g.sC = sA;
        BTA_TRY(gemm_exec(ex, s, g));
    } else {
        BTA_TRY(gemm_exec(ex, s, g));
        BTA_TRY(copy_mat64(s, W, n2, A21, lda, n2, n1, 0, batch, sW, sA));
    }
    // A22 -= L21 L21^T  (lower)
    g = Gemm64{};
    g.M = n2; g.N = n2; g.K = n1;
    g.A = A21; g.lda = lda; g.ta = 0;
    g.B = A21; g.ldb = lda; g.tb = 1;
    g.Cin = A22; g.ldci = lda; g.beta = 1.0;
    g.C = A22; g.ldc = lda; g.alpha = -1.0; g.lowerC = 1;
    g.batch = batch; g.sA = sA; g.sB = sA; g.sCi = sA; g.sC = sA;
    BTA_TRY(gemm_exec(ex, s, g));
    // W = L21 * X11   (op(B) lower); independent of the factorisation of A22
    g = Gemm64{};
    g.M = n2; g.N = n1; g.K = n1;
    g.A = A21; g.lda = lda;
    g.B = X11; g.ldb = ldx; g.tb = 0; g.shB = 1;
    g.C = W; g.ldc = n2; g.alpha = 1.0; g.beta = 0.0;
    g.batch = batch; g.sA = sA; g.sB = sX; g.sC = sW;
    if (forked) {
        cudaEvent_t ev_fork = fork->ev[2 * depth], ev_join = fork->ev[2 * depth + 1];
        BTA_CUDA_TRY(cudaEventRecord(ev_fork, s));
        BTA_CUDA_TRY(cudaStreamWaitEvent(fork->s2, ev_fork, 0));
        BTA_TRY(gemm_exec(ex && ex->fn ? &fork->ex2 : ex, fork->s2, g));
        BTA_CUDA_TRY(cudaEventRecord(ev_join, fork->s2));
        BTA_TRY(chol_inv64(s, A22, lda, X22, ldx, n2, row0 + n1, status, Wc, leaf, ex, batch, sA, sX, sW, m_first,
                           nbatch, fork, depth + 1, per));
        BTA_CUDA_TRY(cudaStreamWaitEvent(s, ev_join, 0));
    } else {
        BTA_TRY(chol_inv64(s, A22, lda, X22, ldx, n2, row0 + n1, status, Wc, leaf, ex, batch, sA, sX, sW, m_first,
                           nbatch, nullptr, 0, per));
        BTA_TRY(gemm_exec(ex, s, g));
    }
    // X21 = -X22 * W   (op(A) lower)
    g = Gemm64{};
    g.M = n2; g.N = n1; g.K = n2;
    g.A = X22; g.lda = ldx; g.ta = 0; g.shA = 1;
    g.B = W; g.ldb = n2; g.tb = 0;
    g.C = X21; g.ldc = ldx; g.alpha = -1.0; g.beta = 0.0;
    g.batch = batch; g.sA = sX; g.sB = sW; g.sC = sX;
    BTA_TRY(gemm_exec(ex, s, g));
    return BTA_OK;
}

static int grid_for(long long total) {
    return (int)std::min<long long>(std::max<long long>(1, (total + 255) / 256), 152 * 8);
}

int scale_into64(cudaStream_t s, int M, int N, const double* Cin, long long ldci, double beta, double* C,
                 long long ldc, int lower, int batch, long long sCi, long long sC) {
    long long total = (long long)M * N;
    if (total <= 0 || batch <= 0) return BTA_OK;
    dim3 grid(std::max(1, grid_for(total) / batch), batch);
    scale_into_kernel<<<grid, 256, 0, s>>>(M, N, Cin, ldci, beta, C, ldc, lower, sCi, sC);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

int copy_mat64(cudaStream_t s, const double* src, long long lds, double* dst, long long ldd, int rows, int cols,
               int lower_only, int batch, long long ss, long long sd) {
    long long total = (long long)rows * cols;
    if (total <= 0 || batch <= 0) return BTA_OK;
    dim3 grid(std::max(1, grid_for(total) / batch), batch);
    copy_mat_kernel<<<grid, 256, 0, s>>>(src, lds, dst, ldd, rows, cols, lower_only, ss, sd);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

int symmetrize_lower64(cudaStream_t s, double* A, long long lda, int n, int batch, long long sA) {
    long long total = (long long)n * n;
    if (total <= 0 || batch <= 0) return BTA_OK;
    dim3 grid(std::max(1, grid_for(total) / batch), batch);
    symmetrize_kernel<<<grid, 256, 0, s>>>(A, lda, n, sA);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

int gemv64(cudaStream_t s, int M, int N, const double* A, long long lda, int ta, int sh, const double* x,
           double alpha, const double* yin, double beta, double* y, int batch, long long sA, long long sx,
           long long sy) {
    if (M <= 0 || batch <= 0) return BTA_OK;
    if (batch > 65535) return BTA_ERR_ARG;
    if (!ta && sh == 0 && M <= GV_SHORT && N >= 4096) {
        gemv_short_n_kernel<<<dim3(1, batch), 1024, 0, s>>>(M, N, A, lda, x, alpha, yin, beta, y, sA, sx, sy);
    } else if (ta && sh == 0 && N <= GV_SHORT && M >= 4096) {
        dim3 grid((M + 255) / 256, batch);
        gemv_short_t_kernel<<<grid, 256, 0, s>>>(M, N, A, lda, x, alpha, yin, beta, y, sA, sx, sy);
    } else if (!ta) {
        dim3 grid((M + 31) / 32, batch);
        gemv_n_kernel<<<grid, 32 * GV_WARPS, 0, s>>>(M, N, A, lda, sh, x, alpha, yin, beta, y, sA, sx, sy);
    } else {
        dim3 grid((M + 7) / 8, batch);
        gemv_t_kernel<<<grid, 256, 0, s>>>(M, N, A, lda, sh, x, alpha, yin, beta, y, sA, sx, sy);
    }
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

int logdet_batch64(cudaStream_t s, const double* A, long long lda, int dim, int nblk, long long stride,
                   long long sA, const double* T, int a, long long sT, int count, double* partial, int chunks,
                   double* out, double scale) {
    if (count <= 0) return BTA_OK;
    dim3 grid(chunks, count);
    logdiag_partial_kernel<<<grid, 256, 0, s>>>(A, lda, dim, nblk, stride, sA, partial);
    BTA_LAUNCH_CHECK();
    logdet_finish_kernel<<<count, 256, 0, s>>>(partial, chunks, a > 0 ? T : nullptr, a, sT, out, scale);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

int dot_batch64(cudaStream_t s, const double* x, const double* y, long long len, int count, double* partial,
                int chunks, double* out, long long ostride) {
    if (count <= 0) return BTA_OK;
    dim3 grid(chunks, count);
    dot_partial_kernel<<<grid, 256, 0, s>>>(x, y, len, partial);
    BTA_LAUNCH_CHECK();
    dot_finish_kernel<<<count, 256, 0, s>>>(partial, chunks, out, ostride);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}
