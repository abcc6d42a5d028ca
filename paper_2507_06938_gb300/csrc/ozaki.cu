// Split-precision FP64 GEMM on the tcgen05 tensor cores (mixed path of the
// BTA Schur updates and selected inversion).
//
// C += alpha * op(A) op(B) with FP64 A, B, C.  Every row i of op(A) is written
// as 2^{e_i} sum_{p<S} d_p 2^{-7(p+1)} with integer digits (S slices, 7S bits
// below the row's largest binary exponent, rounded; |d_0| <= 128, |d_p| <= 64
// for p >= 1), every column j of op(B) the same way with exponent f_j.  A
// digit is exact in bf16.  Grouping the digit products by level s = p + q,
//   (op(A) op(B))_ij ~ 2^{e_i + f_j - 14} sum_{s<S} 2^{-7s} L_s(i,j),
//   L_s = sum_k sum_{p+q=s} d_p(i,k) d_q(k,j)
// (levels s >= S fall below the digits' own precision).  Per k the level
// sums are integers bounded by 2^14 (s = 0, 1), 20480 (s = 2), 24576 (s = 3),
// 28672 (s = 4), 32768 (s = 5) and 36864 (s = 6).  Each level has its own
// FP32 accumulator in tensor memory (tcgen05.mma kind::f16).  Two variants:
//
//   S = 5 (35-bit digits, 128 x 96 tiles): levels 0 and 1 stay below 2^24,
//   hence exact, over 1024 values of k; level 2 is exact over 512 and is
//   drained that often; levels 3 and 4 run over 1024 values of k past 2^24,
//   where each of at most 320 accumulation steps rounds by at most 2 units:
//   2^-37 and 2^-44 of the output scale |A_i||B_j|K, below the 2^-35
//   truncation of the digits.  A drain scales a level by 2^{-7s} and adds it
//   into a double-float sum (two FP32 words, error-free TwoSum).
//
//   S = 7 (49-bit digits, 128 x 64 tiles, for ill-conditioned matrices):
//   levels 0 and 1 are drained every 1024 values of k, levels 2..6 every
//   512, so levels 0..5 are exact integers when drained (level 6 may round
//   by one unit in 2^{-56} of the output scale).  A drain converts each
//   level to an integer and adds it into a 64-bit fixed-point sum in units
//   of level 5 (level 6 rounded to that unit), so the sum over chunks is
//   exact: a double-float sum would round by 2^-48 at every drain, above the
//   2^-49 truncation of the digits.  A work unit spans at most 16 chunks
//   (K <= 8192 per unit, a K split beyond), which bounds the sum by 2^63.
//
// The result goes into C with one FP64 addition per element; the
// power-of-two scaling and the widening to FP64 are done on bit patterns or
// integers, because the FP64 pipe of GB300 (~1.2 TFLOP/s) is the scarce unit
// and the bf16 tensor pipe (~1.9 PFLOP/s) the plentiful one.
//
// Kernel (persistent, one CTA of 576 threads per SM, 128 x TN output tiles):
//   warp 0      TMA producer: for every 32-wide K block all S digit slices
//               of the A tile (128 x 32) and of the B tile (TN x 32), 64-byte
//               swizzle, into a 2-stage shared-memory ring (70 KB a stage for
//               S = 5, 84 KB for S = 7), so that each digit is read from L2
//               once per tile
//   warp 1      allocates 512 TMEM columns (S accumulators of TN columns) and,
//               from one thread, issues the S(S+1)/2 digit pairs of each
//               16-wide K step as tcgen05.mma (M = 128, K = 16) over stacked B
//               slices (N = TN, 2 TN, ..., up to 256; see Cfg::piece)
//   warps 2..17 drain the level group B after every 512-long K chunk and
//               group A after every second chunk, then update C while the
//               next tile's products run
// Work units are (matrix, tile, K part); a K split (atomic adds into C) only
// appears when the tiles alone cannot fill the GPU, or, for S = 7, when K
// exceeds 8192.  The units go out in waves of one per CTA, every second wave
// in reverse CTA order; inside a matrix the tiles are numbered in bands of a
// tuned number of row tiles, column by column within a band (unit_of,
// decode_unit).  Every wait on an mbarrier is bounded in time; on expiry the
// kernel records an error, stops issuing, drains what it issued and frees its
// tensor memory.

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "common.cuh"

namespace oz {

constexpr int TM = 128, TK = 32;          // output tile rows; K block (64-byte rows)
constexpr int ROW_BYTES = TK * 2;         // one digit row of a K block; the swizzle span
static_assert(ROW_BYTES == 32 || ROW_BYTES == 64 || ROW_BYTES == 128, "K block of 16, 32 or 64");
constexpr int KB_PER_CHUNK = 512 / TK;    // exactness bound of the levels drained every chunk
constexpr int EPI_WARPS = 16;             // 4 per TMEM lane quarter
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t A_SLICE_BYTES = TM * TK * 2;   // 8 KB
constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;   // about 2 s
constexpr int PAD_K = 64;                 // digit array K padding (split tile)
constexpr int MAX_MT = 128;               // row tiles per matrix (M <= 16384)
constexpr int INT_MAX_CHUNKS = 16;        // S = 7: chunks per work unit (64-bit sum bound)

// One tcgen05.mma of a K step: A slice p times the B slices q0 .. q0+n-1
// stacked (N = n TN), adding the pairs (p, q0 + j) into the level
// accumulators p + q0 + j.  kind: 0 accumulate, 1 first write of the group-A
// levels it covers (on the chunk that resets group A), 2 first write of
// group-B levels (every chunk).  The p = 0 pieces come first, so every level
// is first written by them at the start of a chunk.
struct Piece { int p, q0, n, kind; };

template <int S, int TN> struct Cfg;

// 35-bit digits, 128 x 96 tiles: 5 levels x 96 columns = 480 of the 512 TMEM
// columns.  Group A = levels 0, 1, 3, 4 (every second chunk), group B = level 2.
template <> struct Cfg<5, 96> {
    static constexpr unsigned GROUP_A = 0x1Bu, GROUP_B = 0x04u;
    static constexpr int PIECES = 9;
    static constexpr int CBUF_BUFS = 2;    // 8-column staging buffers of the bulk reduce-add, per warp
    static constexpr bool INT_ACC = false;
    __host__ __device__ static constexpr Piece piece(int i) {
        constexpr Piece t[PIECES] = {{0, 0, 2, 1}, {0, 2, 1, 2}, {0, 3, 2, 1}, {1, 0, 2, 0}, {1, 2, 2, 0},
                                     {2, 0, 2, 0}, {2, 2, 1, 0}, {3, 0, 2, 0}, {4, 0, 1, 0}};
        return t[i];
    }
};

// 35-bit digits, 128 x 64 tiles (room for a third TMA stage): 320 TMEM
// columns, the same level groups, 15 pairs as 7 MMAs of N <= 256.
template <> struct Cfg<5, 64> {
    static constexpr unsigned GROUP_A = 0x1Bu, GROUP_B = 0x04u;
    static constexpr int PIECES = 7;
    static constexpr int CBUF_BUFS = 1;
    static constexpr bool INT_ACC = false;
    __host__ __device__ static constexpr Piece piece(int i) {
        constexpr Piece t[PIECES] = {{0, 0, 2, 1}, {0, 2, 1, 2}, {0, 3, 2, 1}, {1, 0, 4, 0},
                                     {2, 0, 3, 0}, {3, 0, 2, 0}, {4, 0, 1, 0}};
        return t[i];
    }
};

// 49-bit digits, 128 x 64 tiles: 7 levels x 64 columns = 448 TMEM columns.
// Group A = levels 0, 1 (every second chunk), group B = levels 2..6 (every
// chunk); 28 pairs as 11 MMAs of N <= 256.
template <> struct Cfg<7, 64> {
    static constexpr unsigned GROUP_A = 0x03u, GROUP_B = 0x7Cu;
    static constexpr int PIECES = 11;
    static constexpr int CBUF_BUFS = 1;
    static constexpr bool INT_ACC = true;
    __host__ __device__ static constexpr Piece piece(int i) {
        constexpr Piece t[PIECES] = {{0, 0, 2, 1}, {0, 2, 4, 2}, {0, 6, 1, 2}, {1, 0, 4, 0},
                                     {1, 4, 2, 0}, {2, 0, 4, 0}, {2, 4, 1, 0}, {3, 0, 4, 0},
                                     {4, 0, 3, 0}, {5, 0, 2, 0}, {6, 0, 1, 0}};
        return t[i];
    }
};

template <int S, int TN_, int STG> struct Geo {
    static constexpr int TN = TN_;
    static constexpr int STAGES = STG;
    static constexpr int EPI_COLS = TN / (EPI_WARPS / 4);   // columns per epilogue thread
    static constexpr uint32_t B_SLICE_BYTES = TN * TK * 2;
    static constexpr uint32_t STAGE_BYTES = S * (A_SLICE_BYTES + B_SLICE_BYTES);
    // per epilogue warp, 32-row x 8-column FP64 buffers for the bulk reduce-add of C
    static constexpr uint32_t CBUF_BYTES = Cfg<S, TN>::CBUF_BUFS * 8 * 32 * 8;
    static constexpr size_t SMEM_BYTES =
        1024 /*alignment slack*/ + STAGES * STAGE_BYTES + EPI_WARPS * CBUF_BYTES + 256;
    static_assert(SMEM_BYTES <= 232448, "shared memory of one CTA");
    static_assert(S * TN <= (int)TMEM_COLS, "level accumulators must fit in tensor memory");
    static_assert(EPI_COLS % 8 == 0, "epilogue columns in groups of 8");
    static_assert(TM % TN == 0 || TN == 96, "row padding of aliased operands");
};

// The launch configurations of the split product: (slices, tile width,
// TMA stages).  tile 0 is the default of each slice count; the autotuner may
// pick another one of the same slice count.
struct TileCfg { int S, TN, STG; };
constexpr TileCfg kTiles[] = {{5, 96, 2}, {5, 64, 3}, {7, 64, 2}};
constexpr int NUM_TILES = 3;

struct Args {
    int M, N;            // output extent
    long long sC;        // matrix stride of C
    int Mp, Np;          // padded rows per digit slice
    int kblocks;         // padded K / TK
    int gm, gn;          // row and column tiles per matrix
    int tiles;           // tiles per matrix (lower-output tiles only when lowerC)
    int ksplit;          // K parts per tile (atomic adds into C when > 1)
    int units;           // matrices * tiles * ksplit
    const int* expA;     // Mp exponents of the rows of op(A), per matrix
    const int* expB;     // Np exponents of the columns of op(B), per matrix
    double* C;
    long long ldc;
    double alpha;
    int lowerC;          // only entries m >= n (tiles strictly above skipped)
    int shA, shB;        // triangular shapes of op(A), op(B): K blocks outside them are zero, skipped
    int* err;            // set to 1 on a wait time-out
    const double* Cin;   // C = beta Cin + alpha op(A) op(B) when ksplit == 1 and Cin != C
    long long ldci, sCi;
    double beta;
    int inplace;         // Cin is C with beta = 1 (or the K split pre-initialised C)
    int bulk;            // in-place accumulation through bulk reduce-add (C, ldc, sC 16-byte aligned)
    long long epi_wait;  // wait limit (cycles) of the epilogue's accumulator hand-off
    int band;            // row tiles per band of the tile order of a general output (1: row by row)
    int mcum[MAX_MT + 1];// lowerC: tiles of row tiles 0..m-1
};

struct Unit {
    int inst, m0, n0;
    int kbl;             // first K block of the tile
    int c0, c1;          // chunk range [c0, c1) of this unit (chunks of KB_PER_CHUNK blocks from kbl)
    int kbh;             // end of the tile's K blocks
};

// Decode work unit u; returns false when the unit has no K blocks.
// The i-th unit of CTA `cta` in a grid of g CTAs: the units go out in waves
// of g, every second wave in reverse CTA order, so that a CTA that drew a
// cheap unit (a short K extent under a triangular operand) draws a dear one
// next and the CTAs' totals stay even.  Every role of a CTA walks the same
// sequence.
__device__ __forceinline__ int unit_of(int i, int cta, int g) { return i * g + ((i & 1) ? g - 1 - cta : cta); }

template <int TN>
__device__ __forceinline__ bool decode_unit(const Args& a, int u, Unit& w) {
    const int kpart = u % a.ksplit;
    u /= a.ksplit;
    const int tile = u % a.tiles;
    w.inst = u / a.tiles;
    int mt, nt;
    if (a.lowerC) {
        // lower-triangle tiles: row tile mt holds column tiles nt with
        // nt TN <= (mt + 1) TM - 1, so column nt starts at row tile
        // floor(nt TN / TM) and the rows of a band that hold it are a suffix of
        // the band.  The band (a.band row tiles) is found from the row-major
        // counts, then walked column by column: first the columns every row of
        // the band holds, then the partial ones near the diagonal.
        int m = 0;
        while (m + 1 < a.gm && a.mcum[m + 1] <= tile) ++m;
        const int r0 = (m / a.band) * a.band, r1 = min(a.gm, r0 + a.band), rows = r1 - r0;
        int idx = tile - a.mcum[r0];
        const int nfull = a.mcum[r0 + 1] - a.mcum[r0];
        if (idx < nfull * rows) {
            mt = r0 + idx % rows;
            nt = idx / rows;
        } else {
            idx -= nfull * rows;
            nt = nfull;
            mt = r1 - 1;
            for (; nt < a.gn; ++nt) {
                const int f = max(r0, (nt * TN) / TM);
                const int here = f < r1 ? r1 - f : 0;
                if (idx < here) {
                    mt = f + idx;
                    break;
                }
                idx -= here;
            }
        }
    } else {
        // bands of a.band row tiles, column by column inside a band (a.band = 1:
        // row by row).  With bands of 8 the units in flight at one time (one per
        // SM) cover about 8 x 19 tiles and share their A and B digit panels in
        // L2; row by row they cover one or two row tiles against every column
        // panel.  Which is faster depends on the shape (a triangular operand
        // makes the tiles' K extents uneven): the autotuner chooses.
        const int band = tile / (a.band * a.gn);
        const int in = tile - band * a.band * a.gn;
        const int rows = min(a.band, a.gm - band * a.band);
        mt = band * a.band + in % rows;
        nt = in / rows;
    }
    w.m0 = mt * TM;
    w.n0 = nt * TN;
    int kbl = 0, kbh = a.kblocks;
    if (a.shA == 1) kbh = min(kbh, (w.m0 + TM + TK - 1) / TK);   // op(A) lower: k <= m
    if (a.shA == 2) kbl = max(kbl, w.m0 / TK);                    // op(A) upper: k >= m
    if (a.shB == 1) kbl = max(kbl, w.n0 / TK);                    // op(B) lower: k >= n
    if (a.shB == 2) kbh = min(kbh, (w.n0 + TN + TK - 1) / TK);    // op(B) upper: k <= n
    w.kbl = kbl;
    w.kbh = kbh;
    const int nch = max(0, (kbh - kbl + KB_PER_CHUNK - 1) / KB_PER_CHUNK);
    const int per = (nch + a.ksplit - 1) / a.ksplit;
    w.c0 = min(nch, kpart * per);
    w.c1 = min(nch, w.c0 + per);
    return w.c1 > w.c0;
}

// Prefetch the C (or Cin) tile of unit w into L2 ahead of the epilogue's
// read-modify-write: one bulk prefetch per column of the tile.
template <int TN>
__device__ __forceinline__ void prefetch_c_tile(const double* base, long long ld, const Unit& w, int M, int N) {
    const int rows = min(TM, M - w.m0);
    const int ncols = min(TN, N - w.n0);
    for (int j = 0; j < ncols; ++j) {
        const double* col = base + w.m0 + (long long)(w.n0 + j) * ld;
        uintptr_t lo = reinterpret_cast<uintptr_t>(col);
        const uintptr_t hi = reinterpret_cast<uintptr_t>(col + rows);
        lo = (lo + 15) & ~uintptr_t(15);
        const uintptr_t bytes = (hi - lo) & ~uintptr_t(15);
        if (hi > lo && bytes >= 16)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((uint32_t)bytes) : "memory");
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `parity` to complete.  Returns false (and
// raises the CTA abort flag and the global error flag) after `limit` cycles
// (about 2 s by default), or at once if another thread has already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* err,
                                          long long limit = WAIT_LIMIT_CYCLES) {
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > limit) {
            *abort = 1;
            atomicExch(err, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major tile whose rows are ROW_BYTES
// long, 8-row groups 8 ROW_BYTES apart, swizzled over ROW_BYTES (the layout a
// TMA copy with the matching CU_TENSOR_MAP_SWIZZLE_* mode writes).  Layout
// codes of the descriptor: 6 = 32-byte, 4 = 64-byte, 2 = 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t addr) {
    constexpr uint64_t layout = ROW_BYTES == 32 ? 6 : (ROW_BYTES == 64 ? 4 : 2);
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(16 >> 4) << 16;                // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((8 * ROW_BYTES) >> 4) << 32;   // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                        // descriptor version
    d |= layout << 61;
    return d;
}

// Instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_for_n(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld_8cols(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void reg_fence8(uint32_t* r) {
    asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// error-free sum: hi + lo <- hi + x exactly (Knuth's TwoSum), lo accumulates
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// f 2^e as a double, built from the bit pattern of the FP32 value f (zero or
// normal; the accumulated values here never reach the subnormal range).
__device__ __forceinline__ double f2d_scaled(float f, int e) {
    const uint32_t u = __float_as_uint(f);
    const int ef = (int)((u >> 23) & 0xFF);
    if (ef == 0) return 0.0;
    const int ed = ef - 127 + 1023 + e;
    if (ed <= 0 || ed >= 2047) return ldexp((double)f, e);   // outside the normal range: exact slow path
    const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)ed << 52) |
                                    ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

// v 2^e for a 64-bit integer v: the conversion rounds to the nearest double,
// the scaling adds e to the exponent field (exact in the normal range).
__device__ __forceinline__ double ll2d_scaled(long long v, int e) {
    if (v == 0) return 0.0;
    const double d = __ll2double_rn(v);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    const int ed = (int)((bits >> 52) & 0x7FF) + e;
    if (ed <= 0 || ed >= 2047) return ldexp(d, e);
    return __longlong_as_double((long long)((bits & ~(0x7FFull << 52)) | ((unsigned long long)ed << 52)));
}

// Drain of one level (tensor memory address taddr: lane quarter, level,
// column group) into this thread's EPI_COLS sums.  Double-float variant:
// hi + lo += 2^{-7 lv} L.
template <int EPI_COLS>
__device__ __forceinline__ void drain_level_df(uint32_t taddr, int lv, float* hi, float* lo) {
    const float scale = __uint_as_float((uint32_t)(127 - 7 * lv) << 23);   // 2^{-7 lv}
#pragma unroll
    for (int h = 0; h < EPI_COLS / 8; ++h) {
        uint32_t r[8];
        tmem_ld_8cols(taddr + h * 8, r);
        tmem_wait_ld();
        reg_fence8(r);
#pragma unroll
        for (int j = 0; j < 8; ++j) df_add(hi[h * 8 + j], lo[h * 8 + j], __uint_as_float(r[j]) * scale);
    }
}

// Fixed-point variant: acc += L 2^{7 (5 - lv)} for lv <= 5 (L is an integer
// held exactly in FP32), acc += round(L / 2^7) for lv = 6.
template <int EPI_COLS>
__device__ __forceinline__ void drain_level_int(uint32_t taddr, int lv, long long* acc) {
#pragma unroll
    for (int h = 0; h < EPI_COLS / 8; ++h) {
        uint32_t r[8];
        tmem_ld_8cols(taddr + h * 8, r);
        tmem_wait_ld();
        reg_fence8(r);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const long long v = (long long)__float2int_rn(__uint_as_float(r[j]));   // |L| < 2^25: exact
            if (lv <= 5) acc[h * 8 + j] += v << (7 * (5 - lv));
            else acc[h * 8 + j] += (v + 64) >> 7;
        }
    }
}

template <int S, int TN, int STAGES>
__global__ void __launch_bounds__(THREADS, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ Args a) {
    using CF = Cfg<S, TN>;
    using G = Geo<S, TN, STAGES>;
    constexpr int EPI_COLS = G::EPI_COLS;
    constexpr uint32_t STAGE_BYTES = G::STAGE_BYTES;
    constexpr uint32_t B_SLICE_BYTES = G::B_SLICE_BYTES;
    constexpr uint32_t CBUF_BYTES = G::CBUF_BYTES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    double* cbuf = reinterpret_cast<double*>(smem + STAGES * STAGE_BYTES);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + EPI_WARPS * CBUF_BYTES);
    uint64_t* empty = full + STAGES;
    // accumulator hand-off: group A (drained every second chunk) and group B
    // (drained every chunk), see Cfg
    uint64_t* fullA = empty + STAGES;
    uint64_t* emptyA = fullA + 1;
    uint64_t* fullB = emptyA + 1;
    uint64_t* emptyB = fullB + 1;
    uint64_t* drain = emptyB + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(fullA, 1);
        mbar_init(emptyA, EPI_WARPS);
        mbar_init(fullB, 1);
        mbar_init(emptyB, EPI_WARPS);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------------ TMA producer
            int it = 0;
            for (int wv = 0; wv * (int)gridDim.x < a.units && !*abort_flag; ++wv) {
                const int u = unit_of(wv, blockIdx.x, gridDim.x);
                Unit w;
                if (u >= a.units || !decode_unit<TN>(a, u, w)) continue;
                const int kb0 = w.kbl + w.c0 * KB_PER_CHUNK;
                const int kb1 = min(w.kbh, w.kbl + w.c1 * KB_PER_CHUNK);
                const int kb_last = w.kbl + (w.c1 - 1) * KB_PER_CHUNK;
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int st = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&empty[st], ph ^ 1, abort_flag, a.err)) break;
                    if (kb == kb_last && a.ksplit == 1) {
                        if (a.inplace)
                            prefetch_c_tile<TN>(a.C + w.inst * a.sC, a.ldc, w, a.M, a.N);
                        else if (a.Cin != nullptr && a.beta != 0.0)
                            prefetch_c_tile<TN>(a.Cin + w.inst * a.sCi, a.ldci, w, a.M, a.N);
                    }
                    uint8_t* sA = smem + st * STAGE_BYTES;
                    uint8_t* sB = sA + S * A_SLICE_BYTES;
                    mbar_expect_tx(&full[st], STAGE_BYTES);
#pragma unroll
                    for (int p = 0; p < S; ++p) {
                        tma_load_2d(smem_u32(sA + p * A_SLICE_BYTES), &tmA, &full[st], kb * TK,
                                    (w.inst * S + p) * a.Mp + w.m0);
                        tma_load_2d(smem_u32(sB + p * B_SLICE_BYTES), &tmB, &full[st], kb * TK,
                                    (w.inst * S + p) * a.Np + w.n0);
                    }
                }
            }
            if (*abort_flag) {
                // let the copies already issued land before the CTA exits
                const int first = max(0, it - STAGES);
                for (int j = first; j < it; ++j) {
                    const int st = j % STAGES;
                    const long long t0 = clock64();
                    while (!mbar_try_wait(&full[st], (j / STAGES) & 1) && clock64() - t0 < WAIT_LIMIT_CYCLES) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------------------ MMA issuer
            int it = 0, nA = 0, nB = 0;
            bool ok = true;
            for (int wv = 0; ok && wv * (int)gridDim.x < a.units && !*abort_flag; ++wv) {
                const int u = unit_of(wv, blockIdx.x, gridDim.x);
                Unit w;
                if (u >= a.units || !decode_unit<TN>(a, u, w)) continue;
                for (int c = w.c0; ok && c < w.c1; ++c) {
                    const int kb0 = w.kbl + c * KB_PER_CHUNK, kb1 = min(w.kbh, kb0 + KB_PER_CHUNK);
                    const bool resetA = ((c - w.c0) & 1) == 0;
                    const bool drainA = ((c - w.c0) & 1) == 1 || c == w.c1 - 1;
                    if (resetA) {
                        if (!mbar_wait(emptyA, (nA & 1) ^ 1, abort_flag, a.err)) {
                            ok = false;
                            break;
                        }
                        fence_after_sync();
                    }
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int st = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1;
                        if (!mbar_wait(&full[st], ph, abort_flag, a.err)) {
                            ok = false;
                            break;
                        }
                        fence_after_sync();
                        const uint32_t sA = smem_u32(smem + st * STAGE_BYTES);
                        const uint32_t sB = sA + S * A_SLICE_BYTES;
                        const uint64_t dA = smem_desc_sw(sA), dB = smem_desc_sw(sB);
#pragma unroll
                        for (int k = 0; k < TK / 16; ++k) {
                            bool waitedB = false;
#pragma unroll
                            for (int i = 0; i < CF::PIECES; ++i) {
                                const Piece pc = CF::piece(i);
                                if (pc.kind == 2 && kb == kb0 && k == 0 && !waitedB) {
                                    // group B restarts every chunk: its previous sums must be drained
                                    if (!mbar_wait(emptyB, (nB & 1) ^ 1, abort_flag, a.err)) {
                                        ok = false;
                                        break;
                                    }
                                    fence_after_sync();
                                    waitedB = true;
                                }
                                // descriptor start addresses are in 16-byte units
                                const uint64_t offA = (uint64_t)((pc.p * A_SLICE_BYTES + k * 32) >> 4);
                                const uint64_t offB = (uint64_t)((pc.q0 * B_SLICE_BYTES + k * 32) >> 4);
                                const bool first = kb == kb0 && k == 0 && (pc.kind == 2 || (pc.kind == 1 && resetA));
                                umma_bf16(tmem_base + (pc.p + pc.q0) * TN, dA + offA, dB + offB,
                                          idesc_for_n(pc.n * TN), first ? 0u : 1u);
                            }
                            if (!ok) break;
                        }
                        if (!ok) break;
                        umma_commit(&empty[st]);
                    }
                    if (!ok) break;
                    umma_commit(fullB);
                    ++nB;
                    if (drainA) {
                        umma_commit(fullA);
                        ++nA;
                    }
                }
            }
            // all MMAs issued by this thread have completed once `drain` fires
            umma_commit(drain);
            const long long t0 = clock64();
            while (!mbar_try_wait(drain, 0) && clock64() - t0 < WAIT_LIMIT_CYCLES) {
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int quarter = warp % 4;          // TMEM lanes 32*quarter .. +31
        const int colbase = ((warp - 2) / 4) * EPI_COLS;
        const int row = quarter * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        // S = 5: double-float sums; S = 7: 64-bit fixed point in units of level 5
        float hi[CF::INT_ACC ? 1 : EPI_COLS], lo[CF::INT_ACC ? 1 : EPI_COLS];
        long long acc[CF::INT_ACC ? EPI_COLS : 1];
        int nA = 0, nB = 0;
        bool ok = true;
        for (int wv = 0; ok && wv * (int)gridDim.x < a.units; ++wv) {
            const int u = unit_of(wv, blockIdx.x, gridDim.x);
            if (u >= a.units) continue;
            Unit w;
            // a unit without K blocks still writes beta Cin when there is no K split
            if (!decode_unit<TN>(a, u, w) && (a.ksplit > 1 || a.inplace)) continue;
#pragma unroll
            for (int j = 0; j < EPI_COLS; ++j) {
                if constexpr (CF::INT_ACC) {
                    acc[j] = 0;
                } else {
                    hi[j] = 0.f;
                    lo[j] = 0.f;
                }
            }
            for (int c = w.c0; c < w.c1; ++c) {
                const bool drainA = ((c - w.c0) & 1) == 1 || c == w.c1 - 1;
                if (!mbar_wait(fullB, nB & 1, abort_flag, a.err, a.epi_wait)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
#pragma unroll
                for (int lv = 0; lv < S; ++lv) {
                    if (!(CF::GROUP_B & (1u << lv))) continue;
                    if constexpr (CF::INT_ACC)
                        drain_level_int<EPI_COLS>(tmem_base + lane_addr + lv * TN + colbase, lv, acc);
                    else
                        drain_level_df<EPI_COLS>(tmem_base + lane_addr + lv * TN + colbase, lv, hi, lo);
                }
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(emptyB);
                ++nB;
                if (drainA) {
                    if (!mbar_wait(fullA, nA & 1, abort_flag, a.err, a.epi_wait)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
#pragma unroll
                    for (int lv = 0; lv < S; ++lv) {
                        if (!(CF::GROUP_A & (1u << lv))) continue;
                        if constexpr (CF::INT_ACC)
                            drain_level_int<EPI_COLS>(tmem_base + lane_addr + lv * TN + colbase, lv, acc);
                        else
                            drain_level_df<EPI_COLS>(tmem_base + lane_addr + lv * TN + colbase, lv, hi, lo);
                    }
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(emptyA);
                    ++nA;
                }
            }
            if (!ok) break;
            // value of column jj of this thread's row, times 2^e
            auto value = [&](int jj, int e) -> double {
                if constexpr (CF::INT_ACC) return ll2d_scaled(acc[jj], e - 35);
                else return f2d_scaled(hi[jj], e) + f2d_scaled(lo[jj], e);
            };
            // C update from registers (tensor memory is already free for the next unit)
            const int i = w.m0 + row;
            const int rows_here = a.M - (w.m0 + quarter * 32);   // rows of this warp inside C
            if (a.bulk && rows_here > 0 && (rows_here >= 32 || (rows_here & 1) == 0)) {
                // C += v through the L2: v staged per 8 columns in shared memory,
                // one bulk reduce-add (FP64) per column of 32 (or fewer, even) rows
                const int ea = (i < a.M) ? a.expA[(long long)w.inst * a.Mp + i] - 14 : 0;
                const int* expB = a.expB + (long long)w.inst * a.Np;
                double* Cw = a.C + w.inst * a.sC + (w.m0 + quarter * 32);
                const uint32_t bytes = (uint32_t)min(rows_here, 32) * 8u;
                const bool neg = a.alpha == -1.0, unit_alpha = neg || a.alpha == 1.0;
                double* wbuf = cbuf + (warp - 2) * (CBUF_BYTES / 8);
#pragma unroll
                for (int g = 0; g < EPI_COLS / 8; ++g) {
                    double* bufg = wbuf + (g % CF::CBUF_BUFS) * 256;
                    if (g >= CF::CBUF_BUFS) {
                        // the bulk reads of the group that used this buffer must be done
                        if (lane == 0) {
                            if constexpr (CF::CBUF_BUFS == 2)
                                asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                            else
                                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                        }
                        __syncwarp();
                    }
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const int nn = w.n0 + colbase + g * 8 + jj;
                        double v = 0.0;
                        if (i < a.M && nn < a.N && !(a.lowerC && i < nn)) {
                            v = value(g * 8 + jj, ea + expB[nn]);
                            if (!unit_alpha) v *= a.alpha;
                            else if (neg) v = -v;
                        }
                        bufg[jj * 32 + lane] = v;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const int nn = w.n0 + colbase + g * 8 + jj;
                            if (nn < a.N)
                                asm volatile(
                                    "cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(
                                        Cw + (long long)nn * a.ldc),
                                    "r"(smem_u32(bufg + jj * 32)), "r"(bytes)
                                    : "memory");
                        }
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                }
                if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                __syncwarp();
            } else if (i < a.M) {
                const int ea = a.expA[(long long)w.inst * a.Mp + i] - 14;
                const int* expB = a.expB + (long long)w.inst * a.Np;
                double* Cm = a.C + w.inst * a.sC;
                const double* Ci = a.inplace ? Cm : a.Cin + w.inst * a.sCi;
                const long long ldi = a.inplace ? a.ldc : a.ldci;
                const double beta = a.inplace ? 1.0 : a.beta;
                const bool atomic = a.ksplit > 1;
                const bool neg = a.alpha == -1.0, unit_alpha = neg || a.alpha == 1.0;
#pragma unroll
                for (int j0 = 0; j0 < EPI_COLS; j0 += 8) {
                    double cv[8];
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const int nn = w.n0 + colbase + j0 + jj;
                        const bool valid = nn < a.N && !(a.lowerC && i < nn);
                        cv[jj] = (valid && !atomic && beta != 0.0) ? Ci[i + (long long)nn * ldi] : 0.0;
                    }
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const int nn = w.n0 + colbase + j0 + jj;
                        if (nn >= a.N || (a.lowerC && i < nn)) continue;
                        double v = value(j0 + jj, ea + expB[nn]);
                        if (!unit_alpha) v *= a.alpha;
                        else if (neg) v = -v;
                        double* c = Cm + i + (long long)nn * a.ldc;
                        if (atomic) {
                            atomicAdd(c, v);
                        } else if (beta == 0.0) {
                            *c = v;
                        } else {
                            *c = (beta == 1.0 ? cv[jj] : beta * cv[jj]) + v;
                        }
                    }
                }
            }
        }
        // every bulk reduce-add of this warp has landed before the CTA exits
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------------ digit split
// Rows r < R of X (R x K, X[r][k] = P[r*sr + k*sk]) with an optional
// triangular mask (shape 1: X[r][k] = 0 for k > r; shape 2: for k < r).
// e_r = exponent of the row maximum (|X[r][k]| < 2^{e_r}).  Each entry is
// turned into the 7S-bit fixed-point integer V = round(X[r][k] 2^{7S - e_r})
// (|V| <= 2^{7S}, ties rounded away from zero) and |V| into balanced
// base-128 digits u_0..u_{S-1}, |V| = sum_s u_s 128^{S-1-s}, |u_s| <= 64 for
// s >= 1 and |u_0| <= 128; the digits of V are d_s = sign(X) u_s, so that
// X[r][k] 2^{-e_r} = sum_s d_s 2^{-7(s+1)} up to 2^{-7S-1}.  Only integer and
// FP32 operations are used (the FP64 pipe of GB300 is the slow one).
// Output: dig[s][r][k] (bf16, rows padded to Rp, K padded to Kp with zeros)
// and exp[r] (0 for padding rows).
constexpr int SPLIT_THREADS = 256;
constexpr int SPLIT_SMEM_TARGET = 73728;   // rows x Kp staged per CTA: 3 CTAs per SM

struct SplitJob {
    const double* P;
    long long sr, sk, sP;   // strides of X[r][k] and between matrices
    int R, K, shape, Rp, Kp;
    int* expo;              // Rp per matrix
    __nv_bfloat16* dig;     // S * Rp * Kp per matrix
};

// Signed digit d as an FP32 bit pattern whose upper half is the bf16
// pattern: 0x4B400000 + d is 1.5 2^23 + d (exact for |d| < 2^22), so
// subtracting 1.5 2^23 leaves d exactly; d ^ s - s (s = 0 or -1, folded into
// the base) negates it.
__device__ __forceinline__ uint32_t digit_bits(uint32_t base, uint32_t d, uint32_t sg) {
    return __float_as_uint(__uint_as_float(base + (d ^ sg)) - 12582912.0f);
}

// The S digits of x for a row with exponent e, as FP32 bit patterns whose
// upper halves are the bf16 patterns (c = 1075 - 7S + e).  V comes from the
// 53-bit significand m of |x| = m 2^{ef - 1075}: V = round(m 2^{-(c - ef)}),
// with c - ef >= 53 - 7S + 1 whenever |x| < 2^e (a shift of 63 or more
// gives 0, which also covers e = 4096 for rows holding a NaN or an
// infinity).  Each digit is peeled off as ((t + 64) mod 128) - 64 with the
// carry (t + 64) >> 7, four digits from the low 28 bits of V and the rest
// from the high bits.
template <int S>
__device__ __forceinline__ void digits_of(double x, int c, uint32_t (&f)[S]) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const uint32_t h = (uint32_t)(bits >> 32);
    const int ef = (int)((h >> 20) & 0x7FF);
    // zero and subnormals (far below the resolution of any row) give 0
    const unsigned long long m = ef ? ((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : 0ull;
    const int sft = max(0, min(c - ef - 1, 63));
    const unsigned long long V = ((m >> sft) + 1) >> 1;   // round half away from zero on |x|
    uint32_t lo = (uint32_t)V & 0xFFFFFFFu;
    uint32_t top = (uint32_t)(V >> 28);
    const uint32_t sg = (uint32_t)((int32_t)h >> 31);
    const uint32_t base = 0x4B400000u - sg;
#pragma unroll
    for (int sl = S - 1; sl >= S - 4; --sl) {
        const uint32_t t = lo + 64u;
        const uint32_t d = (t & 127u) - 64u;
        lo = t >> 7;
        f[sl] = digit_bits(base, d, sg);
    }
    top += lo;   // carry out of the low 28 bits
#pragma unroll
    for (int sl = S - 5; sl >= 1; --sl) {
        const uint32_t t = top + 64u;
        const uint32_t d = (t & 127u) - 64u;
        top = t >> 7;
        f[sl] = digit_bits(base, d, sg);
    }
    f[0] = digit_bits(base, top, sg);
}

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Rows per CTA for a K extent: the largest of 8, 4, 2, 1 whose staged rows
// fit SPLIT_SMEM_TARGET (1 row up to the 227 KB of one CTA).
inline int split_rows(int Kp) {
    for (int rs = 8; rs >= 1; rs >>= 1)
        if ((size_t)rs * (Kp + 4) * 8 <= (size_t)SPLIT_SMEM_TARGET) return rs;
    return 1;
}
inline size_t split_smem(int rs, int Kp) { return (size_t)rs * (Kp + 4) * 8; }

// One CTA per (RS-row block, matrix) of one or two operands (blockIdx.x runs
// over the row blocks of job 0, then of job 1; blockIdx.y = matrix).  The RS
// rows are read once from global memory into shared memory (cp.async, lanes
// along the contiguous stored dimension; row stride Kp + 4 keeps the
// column-order fills free of bank conflicts), then the row exponents and the
// digits are computed from there; each thread writes four consecutive k of
// every digit slice with one 8-byte store.
template <int RS, int S>
__global__ void __launch_bounds__(SPLIT_THREADS) split_kernel(SplitJob j0, SplitJob j1) {
    extern __shared__ double stile[];   // RS x (Kp + 4)
    __shared__ int row_e[RS];
    __shared__ unsigned int row_m[RS];
    static_assert(RS >= 1 && RS <= SPLIT_THREADS / 32 && (SPLIT_THREADS / 32) % RS == 0, "rows per CTA");
    int rb = blockIdx.x;
    const int nrb0 = j0.Rp / RS;
    const bool second = rb >= nrb0;
    const SplitJob& J = second ? j1 : j0;
    if (second) rb -= nrb0;
    const int z = blockIdx.y;
    const double* P = J.P + z * J.sP;
    int* expo = J.expo + (long long)z * J.Rp;
    __nv_bfloat16* dig = J.dig + (long long)z * S * J.Rp * J.Kp;
    const int r0 = rb * RS;
    const int ld = J.Kp + 4;
    for (int e = threadIdx.x; e < RS * J.Kp; e += SPLIT_THREADS) {
        int rr, kk;
        if (J.sr == 1) { rr = e % RS; kk = e / RS; } else { kk = e % J.Kp; rr = e / J.Kp; }
        const int r = r0 + rr;
        double* dst = stile + rr * ld + kk;
        if (r < J.R && kk < J.K && !(J.shape == 1 && kk > r) && !(J.shape == 2 && kk < r))
            cp_async8(dst, P + r * J.sr + kk * J.sk);
        else
            *dst = 0.0;
    }
    if (threadIdx.x < RS) row_m[threadIdx.x] = 0u;
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    {
        // largest exponent field of each row: WPR warps per row, each over an
        // interleaved share of the row, combined in shared memory
        constexpr int WPR = (SPLIT_THREADS / 32) / RS;
        const int rr = warp / WPR, q = warp % WPR;
        unsigned int m = 0;
        const double* row = stile + rr * ld;
        for (int k = q * 32 + lane; k < J.Kp; k += 32 * WPR)
            m = max(m, (unsigned int)((__double2hiint(row[k]) >> 20) & 0x7FF));
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) atomicMax(&row_m[rr], m);
    }
    __syncthreads();
    if (threadIdx.x < RS) {
        const unsigned int m = row_m[threadIdx.x];
        // |x| < 2^(ef - 1023 + 1) for a normal number with exponent field ef;
        // a NaN or Inf in the row gives a huge exponent, so the product
        // overflows to a non-finite value instead of passing silently
        const int e = m == 0 ? 0 : (m == 0x7FF ? 4096 : (int)m - 1023 + 1);
        row_e[threadIdx.x] = e;
        expo[r0 + threadIdx.x] = e;
    }
    __syncthreads();
    const int per = J.Kp / 4;   // Kp is a multiple of 64
    for (int e = threadIdx.x; e < RS * per; e += SPLIT_THREADS) {
        const int kk = 4 * (e % per), rr = e / per;
        const double* row = stile + rr * ld + kk;
        const int c = 1075 - 7 * S + row_e[rr];
        uint32_t f0[S], f1[S], f2[S], f3[S];
        digits_of<S>(row[0], c, f0);
        digits_of<S>(row[1], c, f1);
        digits_of<S>(row[2], c, f2);
        digits_of<S>(row[3], c, f3);
        __nv_bfloat16* out = dig + (size_t)(r0 + rr) * J.Kp + kk;
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
            *reinterpret_cast<uint2*>(out + (size_t)sl * J.Rp * J.Kp) =
                make_uint2(__byte_perm(f0[sl], f1[sl], 0x7632), __byte_perm(f2[sl], f3[sl], 0x7632));
    }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2D map over `rows` digit rows of kp bf16 each; box = TK x box_rows, swizzled over ROW_BYTES.
int make_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int kp, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return BTA_ERR_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE,
                    ROW_BYTES == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                    : (ROW_BYTES == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B),
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? BTA_OK : BTA_ERR_CUDA;
}

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 148;
    }
    return n;
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

template <int RS, int S>
int split_launch_rs(cudaStream_t s, const SplitJob& ja, const SplitJob& jb, bool same, int nb) {
    const size_t smem = split_smem(RS, ja.Kp);
    BTA_TRY(ensure_dyn_smem((const void*)split_kernel<RS, S>, (int)smem));
    const dim3 grid(ja.Rp / RS + (same ? 0 : jb.Rp / RS), nb);
    split_kernel<RS, S><<<grid, SPLIT_THREADS, smem, s>>>(ja, jb);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

// Digits and row exponents of both operands (of one when they coincide).
template <int S>
int split_launch(cudaStream_t s, const SplitJob& ja, const SplitJob& jb, bool same, int nb) {
    const int rs = split_rows(ja.Kp);
    if (split_smem(rs, ja.Kp) > 227 * 1024) return BTA_ERR_ARG;   // K beyond 29 000
    switch (rs) {
        case 8: return split_launch_rs<8, S>(s, ja, jb, same, nb);
        case 4: return split_launch_rs<4, S>(s, ja, jb, same, nb);
        case 2: return split_launch_rs<2, S>(s, ja, jb, same, nb);
        default: return split_launch_rs<1, S>(s, ja, jb, same, nb);
    }
}

size_t workspace_bytes(int M, int N, int K, int S) {
    // rows of op(B) padded to the widest tile of this slice count
    int tn = 0;
    for (const TileCfg& t : kTiles)
        if (t.S == S) tn = std::max(tn, t.TN);
    const size_t Mp = (size_t)round_up(M, TM), Np = (size_t)round_up(N, tn);
    const size_t Kp = (size_t)std::max(PAD_K, round_up(K, PAD_K));
    return (size_t)S * (Mp + Np) * Kp * 2 + (Mp + Np) * sizeof(int) + 4 * 256;
}

template <int S, int TN, int STG>
int gemm_s(cudaStream_t s, const Gemm64& g, void* ws, int* err, long long epi_wait, int occupancy, int band) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return BTA_OK;
    if (g.M > MAX_MT * TM) return BTA_ERR_ARG;
    const int nb = g.batch;
    const int Mp = round_up(g.M, TM), Np = round_up(g.N, TN);
    const int Kp = std::max(PAD_K, round_up(g.K, PAD_K));
    uint8_t* w = static_cast<uint8_t*>(ws);
    __nv_bfloat16* digA = reinterpret_cast<__nv_bfloat16*>(w);
    __nv_bfloat16* digB = digA + (size_t)nb * S * Mp * Kp;
    int* expA = reinterpret_cast<int*>(digB + (size_t)nb * S * Np * Kp);
    int* expB = expA + (size_t)nb * Mp;
    // rows of op(A): op(A)[i][k] = ta ? A[k + i lda] : A[i + k lda]
    const long long srA = g.ta ? g.lda : 1, skA = g.ta ? 1 : g.lda;
    // rows of op(B)^T: op(B)[k][j] = tb ? B[j + k ldb] : B[k + j ldb]
    const long long srB = g.tb ? 1 : g.ldb, skB = g.tb ? g.ldb : 1;
    // shape of op(B)^T: lower op(B) (zero for j > k) is upper in op(B)^T
    const int shBt = g.shB == 1 ? 2 : (g.shB == 2 ? 1 : 0);
    // op(B)^T = op(A) (A B^T or A^T A shapes on one matrix): one split serves both
    const bool same = g.A == g.B && g.sA == g.sB && g.M == g.N && srA == srB && skA == skB && g.shA == shBt;
    SplitJob ja{g.A, srA, skA, g.sA, g.M, g.K, g.shA, Mp, Kp, expA, digA};
    SplitJob jb{g.B, srB, skB, g.sB, g.N, g.K, shBt, Np, Kp, expB, digB};
    BTA_TRY(split_launch<S>(s, ja, jb, same, nb));
    // digit rows per slice of the B operand as the GEMM kernel reads them
    // (TM is a multiple of TN for S = 7; for S = 5 the last column tile may
    // read rows past Mp, which belong to the next slice and only feed output
    // columns n >= N, never written)
    const int NpB = same ? Mp : Np;
    const __nv_bfloat16* digBr = same ? digA : digB;
    const int* expBr = same ? expA : expB;
    CUtensorMap mA, mB;
    BTA_TRY(make_map(&mA, digA, nb * S * Mp, Kp, TM));
    BTA_TRY(make_map(&mB, digBr, nb * S * NpB, Kp, TN));
    const bool inplace = (g.Cin == g.C && g.ldci == g.ldc && g.beta == 1.0 && g.sCi == g.sC);
    Args a{};
    a.M = g.M; a.N = g.N; a.sC = g.sC;
    a.Mp = Mp; a.Np = NpB; a.kblocks = Kp / TK;
    a.gm = Mp / TM; a.gn = (g.N + TN - 1) / TN;
    if (g.lowerC) {
        a.mcum[0] = 0;
        for (int m = 0; m < a.gm; ++m)
            a.mcum[m + 1] = a.mcum[m] + std::min(a.gn, (m * TM + TM - 1) / TN + 1);
        a.tiles = a.mcum[a.gm];
    } else {
        a.tiles = a.gm * a.gn;
    }
    const long long base = (long long)nb * a.tiles;
    const int sms = num_sms();
    const int nchunks = (a.kblocks + KB_PER_CHUNK - 1) / KB_PER_CHUNK;
    // a K split (atomic adds) only when the tiles cannot give `occupancy` waves
    // of the persistent grid
    long long ksplit = 1;
    const long long want = (long long)sms * std::max(1, occupancy);
    if (base < want) ksplit = std::min<long long>(nchunks, (want + base - 1) / base);
    // the 64-bit fixed-point sums of S = 7 hold at most INT_MAX_CHUNKS chunks
    if (Cfg<S, TN>::INT_ACC) ksplit = std::max<long long>(ksplit, (nchunks + INT_MAX_CHUNKS - 1) / INT_MAX_CHUNKS);
    if (base * ksplit > 0x7FFFFFFFLL) return BTA_ERR_ARG;
    a.ksplit = (int)ksplit;
    a.band = std::max(1, std::min(band, MAX_MT));
    a.units = (int)(base * ksplit);
    // with a K split the parts add into C, which must hold beta Cin first;
    // otherwise the epilogue reads beta Cin itself
    if (ksplit > 1 && !inplace)
        BTA_TRY(scale_into64(s, g.M, g.N, g.Cin, g.ldci, g.beta, g.C, g.ldc, g.lowerC, nb, g.sCi, g.sC));
    a.inplace = (inplace || ksplit > 1) ? 1 : 0;
    // in-place accumulation without a K split goes through bulk reduce-adds,
    // which need 16-byte aligned column starts
    a.bulk = (inplace && ksplit == 1 && (reinterpret_cast<uintptr_t>(g.C) & 15) == 0 && (g.ldc & 1) == 0 &&
              (g.sC & 1) == 0)
                 ? 1
                 : 0;
    a.Cin = g.Cin;
    a.ldci = g.ldci;
    a.sCi = g.sCi;
    a.beta = g.Cin ? g.beta : 0.0;
    a.expA = expA; a.expB = expBr;
    a.C = g.C; a.ldc = g.ldc; a.alpha = g.alpha;
    a.lowerC = g.lowerC;
    a.shA = g.shA;
    a.shB = g.shB;
    a.err = err;
    a.epi_wait = epi_wait > 0 ? epi_wait : WAIT_LIMIT_CYCLES;
    using G = Geo<S, TN, STG>;
    BTA_TRY(ensure_dyn_smem((const void*)ozaki_gemm_kernel<S, TN, STG>, (int)G::SMEM_BYTES));
    const int grid = (int)std::min<long long>(a.units, sms);
    ozaki_gemm_kernel<S, TN, STG><<<grid, THREADS, G::SMEM_BYTES, s>>>(mA, mB, a);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

}  // namespace oz

// Workspace needed by ozaki_gemm for one M x N x K product with `slices`
// digit slices (bytes; a batch of products needs batch times this).
size_t ozaki_workspace_bytes(int M, int N, int K, int slices) { return oz::workspace_bytes(M, N, K, slices); }

// Largest M the tensor-core path accepts (row tiles per matrix).
int ozaki_max_rows() { return oz::MAX_MT * oz::TM; }

// C = beta Cin + alpha op(A) op(B) through the digit-split tensor-core path
// with 5 or 7 digit slices.  ws: device workspace of batch *
// ozaki_workspace_bytes(M, N, K, slices); err: device int; epi_wait: wait
// limit (cycles) of the epilogue's accumulator hand-off, <= 0 for the default;
// band: row tiles per band of the tile order (1: row by row).
int ozaki_gemm(cudaStream_t s, const Gemm64& g, void* ws, int* err, int slices, long long epi_wait, int tile,
               int occupancy, int band) {
    using namespace oz;
    if (slices == 7) return gemm_s<7, 64, 2>(s, g, ws, err, epi_wait, occupancy, band);
    if (slices == 5)
        return tile == 1 ? gemm_s<5, 64, 3>(s, g, ws, err, epi_wait, occupancy, band)
                         : gemm_s<5, 96, 2>(s, g, ws, err, epi_wait, occupancy, band);
    return BTA_ERR_ARG;
}

// Tile configurations the autotuner may choose for a slice count: writes up
// to `cap` tile indices (index into the configuration table) and returns the
// count; ozaki_tile_desc names one.
int ozaki_tiles_for(int slices, int* out, int cap) {
    int n = 0;
    for (int i = 0; i < oz::NUM_TILES && n < cap; ++i)
        if (oz::kTiles[i].S == slices) out[n++] = (slices == 5 ? i : 0);
    return n;
}

// GEMM executor of the mixed path: products whose output is at least
// min_dim x min_dim go to the tensor cores (a short K, as in the rank-a
// updates of the selected inversion, is padded to one 64-wide K block); the
// smaller panels of the recursive diagonal factorisation go to the
// double-float GEMM on the FP32 pipe, arrow and tip products stay FP64.
bool gemm_mixed_takes(const GemmExec* ex, const Gemm64& g) {
    return ex && ex->fn == gemm_mixed_fn && g.M >= ex->min_dim && g.N >= ex->min_dim && g.K >= 1 &&
           g.M <= ozaki_max_rows() &&
           (size_t)g.batch * ozaki_workspace_bytes(g.M, g.N, g.K, ex->slices) <= ex->ws_bytes;
}

int gemm_mixed_fn(const GemmExec* ex, cudaStream_t s, const Gemm64& g) {
    if (gemm_mixed_takes(ex, g)) {
        // test hook: BTA_OZ_EPI_WAIT (cycles) shortens the epilogue's wait for
        // the accumulators, so that a test can make it run out
        long long epi_wait = ex->epi_wait;
        if (const char* e = std::getenv("BTA_OZ_EPI_WAIT")) epi_wait = std::atoll(e);
        const int band = g.lowerC ? ex->band_low : ((g.shA != 0 || g.shB != 0) ? ex->band_tri : ex->band_gen);
        return ozaki_gemm(s, g, ex->ws, ex->err, ex->slices, epi_wait, ex->tile, ex->occupancy, band);
    }
    // below the tensor-core threshold: square-ish products of the diagonal
    // recursion in double-float on the FP32 pipe, thin or tiny ones in FP64
    if (g.M >= 32 && g.N >= 32 && g.K >= 32 && g.batch <= 65535) return gemm_df32(s, g);
    return gemm64(s, g);
}
