// Diagonal-block Cholesky + inverse in double-float arithmetic for the
// mixed-precision path.
//
// On GB300 an FP64 instruction is both low-throughput (2 lanes per clock per
// SM) and long-latency, which makes the small, sequential pivot steps of the
// diagonal blocks the critical path of the factorisation.  Here one CTA per
// matrix factors an n x n block (n <= 128) entirely in shared memory with
// values held as unevaluated sums hi + lo of two FP32 numbers (about 48
// significand bits, well above the 36 bits of the tensor-core products of
// the mixed path), using only the FP32 pipe:
//   error-free sum (Knuth's TwoSum) and product (FMA-based TwoProduct),
//   1/sqrt by one Newton-Raphson step in double-float from an FP32 seed.
// Phase 1: right-looking Cholesky, one barrier per pivot; column k is scaled
//   to L in place one iteration later (nothing reads it then).  L is written
//   to global memory (FP64).
// Phase 2: in-place inversion X = L^{-1} column by column from the right:
//   X(i, j) = -(1/L_jj) sum_{k=j+1..i} X(i, k) L(k, j),  X(j, j) = 1/L_jj.
// A non-positive pivot records BTA_ERR_NOT_PD (global row, matrix) in the
// status word and poisons the results with NaN.

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int DF_MAX = 128;
constexpr int DF_LD = DF_MAX + 1;
constexpr int DF_THREADS = 1024;

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_double(df a) { return (double)a.hi + (double)a.lo; }

// a + b, both double-float
__device__ __forceinline__ df df_add(df a, df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// a * b, both double-float
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}

// 1/sqrt(x) for x > 0: FP32 estimate y0, then y = y0 + y0 (1 - x y0^2) / 2
// with the residual 1 - x y0^2 formed in double-float; NaN unless x > 0.
__device__ __forceinline__ df df_rsqrt(df x) {
    if (!(x.hi > 0.f) || isinf(x.hi)) return {__int_as_float(0x7fc00000), 0.f};
    const float y0 = rsqrtf(x.hi);
    df t = df_mul(x, df{y0, 0.f});
    t = df_mul(t, df{y0, 0.f});
    const df r = df_add(df{1.f, 0.f}, df_neg(t));
    const float corr = __fmul_rn(__fmul_rn(0.5f, y0), r.hi);
    const float h = __fadd_rn(y0, corr);
    return {h, __fsub_rn(corr, __fsub_rn(h, y0))};
}

__global__ void __launch_bounds__(DF_THREADS) chol_inv_df32_kernel(double* A, long long lda, long long sA, double* X,
                                                                   long long ldx, long long sX, int n,
                                                                   long long row0, long long* status, int m_first,
                                                                   int nbatch) {
    extern __shared__ float smf[];
    float* Sh = smf;                      // column-major, ld DF_LD
    float* Sl = smf + DF_LD * DF_MAX;
    float* yh = smf + 2 * DF_LD * DF_MAX; // 1/L_kk (double-float)
    float* yl = yh + DF_MAX + 1;
    float* ph = yl + DF_MAX + 1;          // phase-2 partial sums (nq x rows_per)
    float* pl = ph + DF_THREADS;
    A += blockIdx.x * sA;
    X += blockIdx.x * sX;
    const int tid = threadIdx.x;
    for (int e = tid; e < n * n; e += DF_THREADS) {
        const int i = e % n, j = e / n;
        const df v = (i >= j) ? df_make(A[i + (long long)j * lda]) : df{0.f, 0.f};
        Sh[j * DF_LD + i] = v.hi;
        Sl[j * DF_LD + i] = v.lo;
    }
    __syncthreads();
    if (tid == 0) {
        const df y = df_rsqrt(df{Sh[0], Sl[0]});
        yh[0] = y.hi;
        yl[0] = y.lo;
    }
    const int rows_per = n <= 32 ? 32 : (n <= 64 ? 64 : DF_MAX);
    const int row = tid % rows_per;
    const int q = tid / rows_per;
    const int nq = DF_THREADS / rows_per;
    // ---------------------------------------------------------------- phase 1
    for (int k = 0; k <= n; ++k) {
        __syncthreads();
        if (k < n) {
            const df y = df{yh[k], yl[k]};
            if (tid == 0 && !(y.hi > 0.f) && status) {
                if (atomicCAS((unsigned long long*)status, 0ull, (unsigned long long)BTA_ERR_NOT_PD) == 0ull) {
                    status[1] = row0 + k;
                    const int mm = m_first + (int)blockIdx.x;
                    status[2] = 2 * (mm % nbatch) + mm / nbatch;
                }
            }
            if (row > k && row < n) {
                const df y2 = df_mul(y, y);
                const df sik = df_mul(df{Sh[k * DF_LD + row], Sl[k * DF_LD + row]}, y2);
                for (int j = k + 1 + q; j <= row; j += nq) {
                    const df skj = df{Sh[k * DF_LD + j], Sl[k * DF_LD + j]};
                    const df v = df_add(df{Sh[j * DF_LD + row], Sl[j * DF_LD + row]}, df_neg(df_mul(sik, skj)));
                    Sh[j * DF_LD + row] = v.hi;
                    Sl[j * DF_LD + row] = v.lo;
                    if (j == k + 1 && row == k + 1) {   // the next pivot is final
                        const df yn = df_rsqrt(v);
                        yh[k + 1] = yn.hi;
                        yl[k + 1] = yn.lo;
                    }
                }
            }
        }
        if (k > 0 && q == 0 && row >= k - 1 && row < n) {
            // column k-1 is complete: scale it to L (nobody reads it in this iteration)
            const int c = k - 1;
            const df v = df_mul(df{Sh[c * DF_LD + row], Sl[c * DF_LD + row]}, df{yh[c], yl[c]});
            Sh[c * DF_LD + row] = v.hi;
            Sl[c * DF_LD + row] = v.lo;
        }
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += DF_THREADS) {
        const int i = e % n, j = e / n;
        A[i + (long long)j * lda] = (i >= j) ? df_double(df{Sh[j * DF_LD + i], Sl[j * DF_LD + i]}) : 0.0;
    }
    // ---------------------------------------------------------------- phase 2
    // Column j: every row i > j is a dot product over k in (j, i] of X(i, k)
    // (columns > j, already inverted) and L(k, j) (column j, still L), split
    // over the nq threads of the row; partial sums meet in shared memory.
    for (int j = n - 1; j >= 0; --j) {
        __syncthreads();
        if (row > j && row < n) {
            df acc{0.f, 0.f};
            for (int k = j + 1 + q; k <= row; k += nq)
                acc = df_add(acc, df_mul(df{Sh[k * DF_LD + row], Sl[k * DF_LD + row]},
                                         df{Sh[j * DF_LD + k], Sl[j * DF_LD + k]}));
            ph[q * rows_per + row] = acc.hi;
            pl[q * rows_per + row] = acc.lo;
        }
        __syncthreads();
        if (q == 0 && row >= j && row < n) {
            if (row == j) {
                Sh[j * DF_LD + j] = yh[j];
                Sl[j * DF_LD + j] = yl[j];
            } else {
                df sum{ph[row], pl[row]};
                for (int qq = 1; qq < nq; ++qq) sum = df_add(sum, df{ph[qq * rows_per + row], pl[qq * rows_per + row]});
                const df xij = df_neg(df_mul(sum, df{yh[j], yl[j]}));
                Sh[j * DF_LD + row] = xij.hi;
                Sl[j * DF_LD + row] = xij.lo;
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += DF_THREADS) {
        const int i = e % n, j = e / n;
        X[i + (long long)j * ldx] = (i >= j) ? df_double(df{Sh[j * DF_LD + i], Sl[j * DF_LD + i]}) : 0.0;
    }
}

}  // namespace

size_t chol_inv_df32_smem_bytes() {
    // S (hi, lo), y (hi, lo), partial sums (hi, lo)
    return (2 * (size_t)DF_LD * DF_MAX + 2 * (DF_MAX + 1) + 2 * (size_t)DF_THREADS) * sizeof(float);
}

int chol_inv_df32_launch(cudaStream_t s, double* A, long long lda, long long sA, double* X, long long ldx,
                         long long sX, int n, long long row0, long long* status, int batch, int m_first,
                         int nbatch) {
    if (n > DF_MAX || n < 1 || batch < 1) return BTA_ERR_ARG;
    static bool attr_set = false;
    const size_t smem = chol_inv_df32_smem_bytes();
    if (!attr_set) {
        BTA_CUDA_TRY(cudaFuncSetAttribute(chol_inv_df32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        attr_set = true;
    }
    chol_inv_df32_kernel<<<batch, DF_THREADS, smem, s>>>(A, lda, sA, X, ldx, sX, n, row0, status, m_first, nbatch);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}
