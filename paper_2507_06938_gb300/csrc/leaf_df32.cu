// Diagonal-block Cholesky + inverse in double-float arithmetic for the
// mixed-precision path.
//
// On GB300 an FP64 instruction is both low-throughput (2 lanes per clock per
// SM) and long-latency, which makes the small, sequential pivot steps of the
// diagonal blocks the critical path of the factorisation.  Here one CTA per
// matrix factors an n x n block (n <= 128) entirely in shared memory with
// values held as unevaluated sums hi + lo of two FP32 numbers (about 48
// significand bits, well above the 36 bits of the tensor-core products of
// the mixed path), using only the FP32 and integer pipes:
//   error-free sum (Knuth's TwoSum) and product (FMA-based TwoProduct),
//   1/sqrt by one Newton-Raphson step in double-float from an FP32 seed,
//   FP64 <-> double-float conversion on the bit patterns (one FP64 addition
//   per stored element).
// Two right-looking recurrences share one loop with one barrier per step,
// and the updates of a step are dealt to consecutive threads densely (an
// index table of the lower triangle for the Cholesky, a rectangle for the
// inverse), so that warps issue only useful work:
// Cholesky.  Step k subtracts (a_ik / a_kk) a_jk from a_ij for k < j <= i;
//   the thread that finishes a_{k+1,k+1} computes the next 1/sqrt pivot at
//   once; column k is scaled to L one step later (nobody reads it then).
// Inverse: X = L^{-1} by forward substitution on the identity.  Step i makes
//   row i + 1 of X final and subtracts L(r, i) X(i, j) from B(r, j) for
//   r > i, j <= i.  It needs only column i of L and row i of X, so it runs
//   two steps behind the Cholesky, in the same barrier interval.  The strict
//   lower triangle of B / X lives transposed in the strict upper triangle of
//   the shared-memory matrix, whose lower triangle holds L: the two
//   recurrences never touch the same entry.
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

// x as hi + lo: hi keeps the top 24 significand bits (truncated), lo the
// rest rounded to 24 bits (relative error below 2^-47 of x).  Integer work
// except one conversion of the low bits; FP32-range exponents only (others
// take the library conversion).
__device__ __forceinline__ df df_from_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const int E = e - 1023;
    if (e == 0) return {0.f, 0.f};
    if (E < -74 || E > 127) {   // the low word's scale 2^(E-52) must be a normal FP32 (or x not finite)
        const float h = __double2float_rn(x);
        return {h, __double2float_rn(x - (double)h)};
    }
    const unsigned int sgn = (unsigned int)(b >> 63) << 31;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    const float hi = __uint_as_float(sgn | ((unsigned int)(E + 127) << 23) | (unsigned int)(m >> 29));
    const unsigned int rest = (unsigned int)(m & ((1u << 29) - 1));
    float lo = 0.f;
    if (rest) {
        // rest * 2^(E - 52): the low 29 bits, rounded to FP32
        lo = __uint2float_rn(rest) * __uint_as_float((unsigned int)(E - 52 + 127) << 23);
        lo = __uint_as_float(__float_as_uint(lo) | sgn);
    }
    return {hi, lo};
}

// FP32 value as a double from its bit pattern (zero or normal).
__device__ __forceinline__ double f_to_double(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int ef = (u >> 23) & 0xFF;
    if (ef == 0) return 0.0;
    if (ef == 0xFF) return (double)f;
    const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                                    ((unsigned long long)(ef - 127 + 1023) << 52) |
                                    ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double df_to_double(df a) { return f_to_double(a.hi) + f_to_double(a.lo); }

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

// c - a * b, all double-float
__device__ __forceinline__ df df_fnms(df c, df a, df b) { return df_add(c, df_neg(df_mul(a, b))); }

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
                                                                   int nbatch, int per) {
    extern __shared__ float smf[];
    // M[r][c] at (c * DF_LD + r): lower triangle = A, then L; strict upper = B / X transposed
    float* Sh = smf;
    float* Sl = smf + DF_LD * DF_MAX;
    float* yh = smf + 2 * DF_LD * DF_MAX;   // 1/L_kk (double-float)
    float* yl = yh + DF_MAX + 1;
    // lower-triangle entries (i, j), i >= j, column by column: the entries with
    // j > k (the trailing matrix of pivot k) are the suffix from colstart(k+1)
    unsigned short* tri = reinterpret_cast<unsigned short*>(yl + DF_MAX + 1);
    A += blockIdx.x * sA;
    X += blockIdx.x * sX;
    const int tid = threadIdx.x;
    auto colstart = [n](int j) { return j * n - j * (j - 1) / 2; };
    for (int j = tid; j < n; j += DF_THREADS)
        for (int i = j; i < n; ++i) tri[colstart(j) + i - j] = (unsigned short)((i << 8) | j);
    for (int e = tid; e < n * n; e += DF_THREADS) {
        const int i = e % n, j = e / n;
        const df v = (i >= j) ? df_from_double(A[i + (long long)j * lda]) : df{0.f, 0.f};
        Sh[j * DF_LD + i] = v.hi;
        Sl[j * DF_LD + i] = v.lo;
    }
    __syncthreads();
    if (tid == 0) {
        const df y = df_rsqrt(df{Sh[0], Sl[0]});
        yh[0] = y.hi;
        yl[0] = y.lo;
    }
    // Cholesky (right-looking, on the lower triangle) and the inverse X = L^-1
    // (right-looking forward substitution, on the strict upper triangle, which
    // holds B(r, j) (r > j) at M[j][r]; zero from the load) run in one loop of
    // n + 1 barrier intervals.  Interval k does Cholesky step k and inverse
    // step i = k - 2, which needs column i of L (scaled in interval i + 1),
    // row i of X (final after inverse step i - 1) and y_{i+1} (computed in
    // interval i): the two steps touch disjoint entries.
    //   Cholesky step k: M[i][j] -= M[i][k] y_k^2 M[j][k] for i >= j > k (the
    //   columns stay unscaled until complete; column k-1 is scaled by y_{k-1}
    //   in the same interval, nobody reads it then).
    //   Inverse step i: B(r, j) -= L(r, i) X(i, j) for r > i, j <= i, with
    //   X(i, i) = y_i; row i + 1 is final after this step, X(i+1, j) =
    //   B(i+1, j) y_{i+1}.
    for (int k = 0; k <= n; ++k) {
        __syncthreads();
        const int count1 = k < n ? (n - k - 1) * (n - k) / 2 : 0;
        const int i2 = k - 2;
        const int R2 = n - 1 - i2;
        const int count2 = (i2 >= 0 && i2 <= n - 2) ? R2 * (i2 + 1) : 0;
        df y2 = {0.f, 0.f};
        if (k < n) {
            const df y = df{yh[k], yl[k]};
            if (tid == 0 && !(y.hi > 0.f) && status) {
                if (atomicCAS((unsigned long long*)status, 0ull, (unsigned long long)BTA_ERR_NOT_PD) == 0ull) {
                    status[1] = row0 + k;
                    const int mm = m_first + (int)blockIdx.x / per;
                    status[2] = 2 * (mm % nbatch) + mm / nbatch;
                }
            }
            y2 = df_mul(y, y);
        }
        const int base = k < n ? colstart(k + 1) : 0;
        // the first Cholesky entry is the next pivot (k+1, k+1): thread 0
        // updates it first and computes its 1/sqrt at once
        for (int t = tid; t < count1 + count2; t += DF_THREADS) {
            if (t < count1) {
                const int ij = tri[base + t];
                const int i = ij >> 8, j = ij & 255;
                const df aik = df{Sh[k * DF_LD + i], Sl[k * DF_LD + i]};
                const df ajk = df{Sh[k * DF_LD + j], Sl[k * DF_LD + j]};
                const df v = df_fnms(df{Sh[j * DF_LD + i], Sl[j * DF_LD + i]}, df_mul(aik, y2), ajk);
                Sh[j * DF_LD + i] = v.hi;
                Sl[j * DF_LD + i] = v.lo;
                if (t == 0) {
                    const df yn = df_rsqrt(v);
                    yh[k + 1] = yn.hi;
                    yl[k + 1] = yn.lo;
                }
            } else {
                const int u = t - count1;
                const int j = u / R2;
                const int r = i2 + 1 + (u - j * R2);
                const df lri = df{Sh[i2 * DF_LD + r], Sl[i2 * DF_LD + r]};
                const df xij = (j == i2) ? df{yh[i2], yl[i2]} : df{Sh[i2 * DF_LD + j], Sl[i2 * DF_LD + j]};
                df bv = df_fnms(df{Sh[r * DF_LD + j], Sl[r * DF_LD + j]}, lri, xij);
                if (r == i2 + 1) bv = df_mul(bv, df{yh[r], yl[r]});
                Sh[r * DF_LD + j] = bv.hi;
                Sl[r * DF_LD + j] = bv.lo;
            }
        }
        if (k > 0) {
            // column k-1 is complete: scale it to L
            const int c = k - 1;
            const int rowc = c + (DF_THREADS - 1 - tid);   // the last threads, least loaded above
            if (rowc < n && tid >= DF_THREADS - (n - c)) {
                const df v = df_mul(df{Sh[c * DF_LD + rowc], Sl[c * DF_LD + rowc]}, df{yh[c], yl[c]});
                Sh[c * DF_LD + rowc] = v.hi;
                Sl[c * DF_LD + rowc] = v.lo;
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += DF_THREADS) {
        const int i = e % n, j = e / n;
        A[i + (long long)j * lda] = (i >= j) ? df_to_double(df{Sh[j * DF_LD + i], Sl[j * DF_LD + i]}) : 0.0;
    }
    for (int e = tid; e < n * n; e += DF_THREADS) {
        const int i = e % n, j = e / n;
        double v = 0.0;
        if (i > j) v = df_to_double(df{Sh[i * DF_LD + j], Sl[i * DF_LD + j]});
        else if (i == j) v = df_to_double(df{yh[i], yl[i]});
        X[i + (long long)j * ldx] = v;
    }
}

// ------------------------------------------------------------------ GEMM
// C = beta Cin + alpha op(A) op(B) in double-float on the FP32 pipe, for the
// small products of the recursive diagonal-block factorisation in the mixed
// path (orders below the tensor-core threshold): no digit split, about 48
// significand bits.  Tile (16 TI) x (16 TI) per CTA of 256 threads, TI x TI
// outputs per thread; K tiles of 16 staged in shared memory as hi/lo pairs.
// Triangular operand shapes, lower output and batching as in the FP64 GEMM.
constexpr int DG_BK = 16, DG_T = 256;

__device__ __forceinline__ double dg_loadA(const Gemm64& p, const double* A, int m, int k, int kend) {
    if (m >= p.M || k >= kend) return 0.0;
    if (p.shA == 1 && k > m) return 0.0;
    if (p.shA == 2 && k < m) return 0.0;
    return p.ta ? A[k + (long long)m * p.lda] : A[m + (long long)k * p.lda];
}

__device__ __forceinline__ double dg_loadB(const Gemm64& p, const double* B, int k, int nn, int kend) {
    if (nn >= p.N || k >= kend) return 0.0;
    if (p.shB == 1 && nn > k) return 0.0;
    if (p.shB == 2 && nn < k) return 0.0;
    return p.tb ? B[nn + (long long)k * p.ldb] : B[k + (long long)nn * p.ldb];
}

// acc + a b with a, b double-float (error-free product of the high words,
// first-order cross terms, TwoSum into the accumulator)
__device__ __forceinline__ df df_fma(df acc, df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    float t = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    t = __fadd_rn(t, __fadd_rn(acc.lo, e));
    const float h = __fadd_rn(s, t);
    return {h, __fsub_rn(t, __fsub_rn(h, s))};
}

template <int TI>
__global__ void __launch_bounds__(DG_T) gemm_df32_kernel(Gemm64 p) {
    constexpr int TB = 16 * TI;
    __shared__ float Ah[DG_BK][TB + 1], Al[DG_BK][TB + 1], Bh[DG_BK][TB + 1], Bl[DG_BK][TB + 1];
    const int m0 = blockIdx.x * TB, n0 = blockIdx.y * TB, z = blockIdx.z;
    if (p.lowerC && m0 + TB - 1 < n0) return;
    const double* A = p.A + z * p.sA;
    const double* B = p.B + z * p.sB;
    const double* Cin = p.Cin ? p.Cin + z * p.sCi : nullptr;
    double* C = p.C + z * p.sC;
    int kb = 0, ke = p.K;
    if (p.shA == 1) ke = min(ke, m0 + TB);
    if (p.shA == 2) kb = max(kb, m0);
    if (p.shB == 1) kb = max(kb, n0);
    if (p.shB == 2) ke = min(ke, n0 + TB);
    kb = (kb / DG_BK) * DG_BK;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    df acc[TI][TI];
#pragma unroll
    for (int i = 0; i < TI; ++i)
#pragma unroll
        for (int j = 0; j < TI; ++j) acc[i][j] = df{0.f, 0.f};
    for (int k0 = kb; k0 < ke; k0 += DG_BK) {
        for (int e = tid; e < TB * DG_BK; e += DG_T) {
            int mm, kk;
            if (!p.ta) { mm = e % TB; kk = e / TB; } else { kk = e % DG_BK; mm = e / DG_BK; }
            const df v = df_from_double(dg_loadA(p, A, m0 + mm, k0 + kk, ke));
            Ah[kk][mm] = v.hi;
            Al[kk][mm] = v.lo;
        }
        for (int e = tid; e < TB * DG_BK; e += DG_T) {
            int nn, kk;
            if (!p.tb) { kk = e % DG_BK; nn = e / DG_BK; } else { nn = e % TB; kk = e / TB; }
            const df v = df_from_double(dg_loadB(p, B, k0 + kk, n0 + nn, ke));
            Bh[kk][nn] = v.hi;
            Bl[kk][nn] = v.lo;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < DG_BK; ++kk) {
            df a[TI], b[TI];
#pragma unroll
            for (int i = 0; i < TI; ++i) a[i] = df{Ah[kk][tx + 16 * i], Al[kk][tx + 16 * i]};
#pragma unroll
            for (int j = 0; j < TI; ++j) b[j] = df{Bh[kk][ty + 16 * j], Bl[kk][ty + 16 * j]};
#pragma unroll
            for (int i = 0; i < TI; ++i)
#pragma unroll
                for (int j = 0; j < TI; ++j) acc[i][j] = df_fma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < TI; ++j) {
        const int nn = n0 + ty + 16 * j;
        if (nn >= p.N) continue;
#pragma unroll
        for (int i = 0; i < TI; ++i) {
            const int mm = m0 + tx + 16 * i;
            if (mm >= p.M || (p.lowerC && mm < nn)) continue;
            double v = p.alpha * df_to_double(acc[i][j]);
            if (p.beta != 0.0) v += p.beta * Cin[mm + (long long)nn * p.ldci];
            C[mm + (long long)nn * p.ldc] = v;
        }
    }
}

}  // namespace

size_t chol_inv_df32_smem_bytes() {
    // M (hi, lo), y (hi, lo), lower-triangle index table
    return (2 * (size_t)DF_LD * DF_MAX + 2 * (DF_MAX + 1)) * sizeof(float) +
           (size_t)DF_MAX * (DF_MAX + 1) / 2 * sizeof(unsigned short);
}

int chol_inv_df32_launch(cudaStream_t s, double* A, long long lda, long long sA, double* X, long long ldx,
                         long long sX, int n, long long row0, long long* status, int batch, int m_first,
                         int nbatch, int per) {
    if (n > DF_MAX || n < 1 || batch < 1) return BTA_ERR_ARG;
    const size_t smem = chol_inv_df32_smem_bytes();
    BTA_TRY(ensure_dyn_smem((const void*)chol_inv_df32_kernel, (int)smem));
    chol_inv_df32_kernel<<<batch, DF_THREADS, smem, s>>>(A, lda, sA, X, ldx, sX, n, row0, status, m_first, nbatch,
                                                         per);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

// Double-float GEMM (same contract as gemm64, any batch <= 65535).
int gemm_df32(cudaStream_t s, const Gemm64& g) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return BTA_OK;
    if (g.batch > 65535) return BTA_ERR_ARG;
    // small outputs: 16 x 16 tiles (more CTAs); otherwise 32 x 32
    const bool small = (long long)((g.M + 31) / 32) * ((g.N + 31) / 32) * g.batch < 2 * 152;
    if (small) {
        dim3 grid((g.M + 15) / 16, (g.N + 15) / 16, g.batch);
        gemm_df32_kernel<1><<<grid, DG_T, 0, s>>>(g);
    } else {
        dim3 grid((g.M + 31) / 32, (g.N + 31) / 32, g.batch);
        gemm_df32_kernel<2><<<grid, DG_T, 0, s>>>(g);
    }
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}
