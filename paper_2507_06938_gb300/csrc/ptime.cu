// Parallel-in-time BTA factorisation, solve and selected inversion on one
// GPU: the time-domain partitioning of Sections IV-C and IV-D.3 (nested
// dissection over the time blocks, which breaks the sequential dependency of
// the block recurrences) restated for a single device, where the P
// partitions of every matrix run together as the batch of every launch
// instead of on P processes.
//
// Time blocks 0..n-1 are cut by P - 1 separator blocks sigma_p = p h - 1
// (p = 1..P-1, h = ceil((n + 1) / P)); partition p's interior is the blocks
// between sigma_p and sigma_{p+1} (partition 0 starts at block 0; partition
// P-1 ends at block n-1 and may be shorter).  Eliminating the interiors
// first leaves a BTA system on the separators (P - 1 blocks and the arrow
// tip), factored by the ordinary recurrence.  For interior block i of
// partition p, with X_i = L_ii^{-1}:
//   L_ii from chol(D~_i)                        D~ accumulates the Schur updates
//   L_{i+1,i} = B_i X_i^T;  D~_{i+1} -= L_{i+1,i} L_{i+1,i}^T   (block i+1 is the next
//                                                  interior block or sigma_{p+1})
//   p >= 1: L_{sigma_p,i} = U_i X_i^T, U_first = Q[sigma_p, first] = B_{sigma_p}^T;
//           D~_{sigma_p} -= L_{sigma_p,i} L_{sigma_p,i}^T;
//           next interior: U_{i+1} = -L_{sigma_p,i} L_{i+1,i}^T        (fill)
//           next is sigma_{p+1}: Q~[sigma_{p+1}, sigma_p] = -L_{i+1,i} L_{sigma_p,i}^T
//   arrow:  L_{t,i} = R~_i X_i^T;  T~ -= L_{t,i} L_{t,i}^T;  R~_{i+1} -= L_{t,i} L_{i+1,i}^T;
//           p >= 1: R~_{sigma_p} -= L_{t,i} L_{sigma_p,i}^T
// The fill rows L_{sigma_p,i} live in a block array F; the reduced coupling
// Q~[sigma_{p+1}, sigma_p] in the otherwise unused B slot of sigma_p.  The
// selected inversion runs the reduced system first, then every interior
// backwards, with the rows {i+1, sigma_p, tip} of column i:
//   G = L_{i+1,i} X_i, H = L_{sigma_p,i} X_i, F = L_{t,i} X_i
//   Sigma_{i+1,i}     = -(Sigma_{i+1,i+1} G + Sigma_{i+1,sigma_p} H + Sigma_{t,i+1}^T F)
//   Sigma_{sigma_p,i} = -(Sigma_{sigma_p,i+1} G + Sigma_{sigma_p,sigma_p} H + Sigma_{t,sigma_p}^T F)
//   Sigma_{t,i}       = -(Sigma_{t,i+1} G + Sigma_{t,sigma_p} H + Sigma_tt F)
//   Sigma_ii          = X_i^T X_i - G^T Sigma_{i+1,i} - H^T Sigma_{sigma_p,i} - F^T Sigma_{t,i}
// (from Sigma L = L^{-T} on block column i); Sigma_{sigma_p,i} is kept in a
// second block array SF, and the BTA-pattern block (first_p, sigma_p) is its
// transpose.
//
// Layout.  Every block array holds P h slots per matrix (n real blocks, the
// rest padding) after one leading padding slot, so that block k of
// partition p of matrix m sits at slot (m P + p) h + k: one stride, h
// blocks, runs over every (matrix, partition) instance, and each step of the
// interiors is one batched launch over all of them.  The padding makes the
// instances uniform: partition 0's "top separator" is the slot before it (a
// padding slot whose fill stays zero, because B there is zero), and the
// last partition's steps past block n - 1 factor identity diagonal blocks
// against zero couplings, which changes nothing.  The inverse of the tip
// factor sits in the last slot of each matrix's L^{-1} blocks.
//
// Work per interior step of a middle partition: five b x b x b products in
// the factorisation (two for the sequential recurrence) and nine in the
// selected inversion (five): more flops, but about n/P + P instead of n
// sequential steps, which pays where the blocks are small and every product
// is latency-bound.

#include <algorithm>

#include "common.cuh"

namespace {

__global__ void transpose_copy_kernel(const double* src, double* dst, int b, long long ss, long long sd) {
    src += blockIdx.y * ss;
    dst += blockIdx.y * sd;
    const long long total = (long long)b * b;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % b), j = (int)(e / b);
        dst[i + (long long)j * b] = src[j + (long long)i * b];
    }
}

// T_m += sum_p Tacc_{m P + p} (lower entries); blockIdx.y = matrix
__global__ void add_tacc_kernel(double* T, long long sT, const double* Tacc, int a, int P) {
    const int m = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a * a) return;
    const int i = e % a, j = e / a;
    if (i < j) return;
    double s = 0.0;
    for (int p = 0; p < P; ++p) s += Tacc[((long long)m * P + p) * a * a + e];
    T[m * sT + e] += s;
}

// identity in the diagonal blocks of slots [s0, s1) of every matrix (and the
// leading slot when lead): the padding of the time-partitioned layout
__global__ void padding_identity_kernel(double* D, long long sD, int b, int s0, int s1, int lead) {
    const int m = blockIdx.y;
    const long long bb = (long long)b * b;
    const int nslot = s1 - s0 + lead;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)nslot * b;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e / b), i = (int)(e % b);
        double* blk = (lead && q == nslot - 1) ? D - bb : D + m * sD + (long long)(s0 + q) * bb;
        if (!(lead && q == nslot - 1 && m > 0)) blk[i + (long long)i * b] = 1.0;
    }
}

struct PLay {
    int n, b, a, P, h, l, l_last, blk;
    long long bb, ab;
};

PLay layout(const bta_ctx_s* c, int P) {
    PLay L;
    L.n = c->n; L.b = c->b; L.a = c->a; L.P = P;
    L.h = (c->n + P) / P;              // ceil((n + 1) / P)
    L.l = L.h - 1;
    L.l_last = c->n - (P - 1) * L.h;
    L.blk = P * L.h;
    L.bb = (long long)c->b * c->b;
    L.ab = (long long)c->a * c->b;
    return L;
}

// One GEMM of the descriptor shape used everywhere below.
struct G {
    Gemm64 g{};
    G(int M, int N, int K) { g.M = M; g.N = N; g.K = K; g.alpha = 1.0; }
    G& A(const double* p, long long ld, int ta = 0, int sh = 0, long long s = 0) { g.A = p; g.lda = ld; g.ta = ta; g.shA = sh; g.sA = s; return *this; }
    G& B(const double* p, long long ld, int tb = 0, int sh = 0, long long s = 0) { g.B = p; g.ldb = ld; g.tb = tb; g.shB = sh; g.sB = s; return *this; }
    G& C(double* p, long long ld, long long s = 0) { g.C = p; g.ldc = ld; g.sC = s; return *this; }
    G& Cin(const double* p, long long ld, double beta, long long s = 0) { g.Cin = p; g.ldci = ld; g.beta = beta; g.sCi = s; return *this; }
    G& alpha(double a) { g.alpha = a; return *this; }
    G& lower() { g.lowerC = 1; return *this; }
    G& batch(int n) { g.batch = n; return *this; }
};

// C -= op(A) op(B) accumulated into C (in place)
G& acc(G& x, double* C, long long ldc, long long sC) { return x.C(C, ldc, sC).Cin(C, ldc, 1.0, sC).alpha(-1.0); }

}  // namespace

// Block arrays of the partitioned path (fill rows of the factor and of the
// selected inverse, in the padded layout) and per-instance scratch for all
// (matrix, partition) instances.
struct PTimeStore {
    double* F = nullptr;      // lead + nmat P h slots: L_{sigma_p, i}
    double* SF = nullptr;     // lead + nmat P h slots: Sigma_{sigma_p, i}
    double* U = nullptr;      // nmat P b^2: fill coupling U_i (also G of the selected inversion)
    double* Racc = nullptr;   // nmat P a b: arrow rows before their product (also F of the selected inversion)
    double* Tacc = nullptr;   // nmat P a^2
    double* RS = nullptr;     // nmat P b^2: reduced Sigma_{sigma_{p+1}, sigma_p}
    double* W = nullptr;      // nmat P x sW: recursion scratch (also H of the selected inversion)
    double* Wg = nullptr;     // nmat (b^2 + a b): in-place product scratch of the reduced chain
    long long sW = 0;
    int P = 1;
};

void ptime_free(bta_ctx_t c) {
    if (!c->pts) return;
    PTimeStore* st = c->pts;
    const long long bb = (long long)c->b * c->b;
    if (st->F) cudaFree(st->F - bb);
    if (st->SF) cudaFree(st->SF - bb);
    double* ps[] = {st->U, st->Racc, st->Tacc, st->RS, st->W, st->Wg};
    for (double* p : ps)
        if (p) cudaFree(p);
    delete st;
    c->pts = nullptr;
}

static int palloc(double** p, size_t n, size_t lead = 0) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(n + lead, 1) * sizeof(double));
    if (e != cudaSuccess) {
        *p = nullptr;
        return bta_cuda_fail(e);
    }
    BTA_CUDA_TRY(cudaMemset(*p, 0, std::max<size_t>(n + lead, 1) * sizeof(double)));
    *p += lead;
    return BTA_OK;
}

// Q in a layout of `blk` slots per matrix, its assembled blocks carried over
// (block t of every layout sits at slot t of its matrix).
static int move_q(bta_ctx_t c, int blk, int lead) {
    BtaStore nq;
    const int n = c->n, nm = c->nmat;
    const long long bb = (long long)c->b * c->b, ab = (long long)c->a * c->b;
    int rc = store_alloc(nq, nm, n, c->b, c->a, blk, lead);
    if (rc != BTA_OK) {
        store_release(nq);
        return rc;
    }
    const BtaStore& o = c->Q;
    const size_t w = sizeof(double);
    BTA_CUDA_TRY(cudaMemcpy2D(nq.D, nq.sD * w, o.D, o.sD * w, n * bb * w, nm, cudaMemcpyDeviceToDevice));
    if (n > 1)
        BTA_CUDA_TRY(cudaMemcpy2D(nq.B, nq.sB * w, o.B, o.sB * w, (n - 1) * bb * w, nm, cudaMemcpyDeviceToDevice));
    if (c->a > 0) {
        BTA_CUDA_TRY(cudaMemcpy2D(nq.R, nq.sR * w, o.R, o.sR * w, n * ab * w, nm, cudaMemcpyDeviceToDevice));
        BTA_CUDA_TRY(cudaMemcpy(nq.T, o.T, nm * o.sT * w, cudaMemcpyDeviceToDevice));
    }
    store_release(c->Q);
    c->Q = nq;
    return BTA_OK;
}

// Storage of the context in the layout of P partitions (P = 1: the compact
// sequential layout), with the partitioned path's own arrays.  The assembled
// Q matrices are kept; factors and selected inverses are not.
static int relayout(bta_ctx_t c, int P) {
    ptime_free(c);
    const bool had_sigma = c->S.D != nullptr;
    store_release(c->L);
    store_release(c->S);
    if (c->Linv) cudaFree(c->Linv);
    c->Linv = nullptr;
    const int n = c->n, b = c->b, a = c->a, nm = c->nmat;
    const long long bb = (long long)b * b;
    if (P == 1) {
        c->blk = n;
        c->tip_off = (long long)n * bb;
        c->sLinv = (long long)n * bb + (long long)a * a;
        BTA_TRY(move_q(c, n, 0));
        BTA_TRY(store_alloc(c->L, nm, n, b, a, n, 0));
        if (had_sigma) BTA_TRY(store_alloc(c->S, nm, n, b, a, n, 0));
        BTA_TRY(palloc(&c->Linv, (size_t)nm * c->sLinv));
        c->tparts = 1;
        return BTA_OK;
    }
    const PLay L = layout(c, P);
    c->blk = L.blk;
    c->tip_off = (long long)(L.blk - 1) * bb;   // the last padding slot: never an interior block
    c->sLinv = (long long)L.blk * bb;
    BTA_TRY(move_q(c, L.blk, 1));
    BTA_TRY(store_alloc(c->L, nm, n, b, a, L.blk, 1));
    if (had_sigma) BTA_TRY(store_alloc(c->S, nm, n, b, a, L.blk, 1));
    BTA_TRY(palloc(&c->Linv, (size_t)nm * c->sLinv));
    // the padding diagonal blocks of L are identities (factored alongside the
    // real blocks, they stay identities)
    padding_identity_kernel<<<dim3(152, nm), 256>>>(c->L.D, c->L.sD, b, n, L.blk, 1);
    BTA_LAUNCH_CHECK();
    PTimeStore* st = c->pts = new PTimeStore();
    st->P = P;
    const size_t inst = (size_t)nm * P;
    st->sW = bb + bb / 2 + 2LL * b + 64;
    BTA_TRY(palloc(&st->F, (size_t)nm * L.blk * bb, (size_t)bb));
    BTA_TRY(palloc(&st->SF, (size_t)nm * L.blk * bb, (size_t)bb));
    BTA_TRY(palloc(&st->U, inst * bb));
    BTA_TRY(palloc(&st->Racc, inst * a * b));
    BTA_TRY(palloc(&st->Tacc, inst * a * a));
    BTA_TRY(palloc(&st->RS, inst * bb));
    BTA_TRY(palloc(&st->W, inst * st->sW));
    BTA_TRY(palloc(&st->Wg, (size_t)nm * (bb + (size_t)a * b)));
    // the products of a step run over nmat P instances: as many digit workspaces
    if (c->precision != BTA_FP64) {
        const size_t wsb = inst * ozaki_workspace_bytes(b, b, b, c->exec.slices);
        if (wsb > c->exec.ws_bytes) {
            for (GemmExec* e : {&c->exec, &c->fork->ex2}) {
                if (e->ws) cudaFree(e->ws);
                e->ws = nullptr;
                if (cudaMalloc(&e->ws, wsb) != cudaSuccess) {
                    e->ws = nullptr;
                    return BTA_ERR_OOM;
                }
                e->ws_bytes = wsb;
            }
        }
    }
    BTA_CUDA_TRY(cudaDeviceSynchronize());
    c->tparts = P;
    return BTA_OK;
}

// ---------------------------------------------------------------------------- factorisation

// Interior step k of every partition of matrices m0 .. m0 + cnt - 1: the cnt P
// instances are h slots apart, instance z = (m - m0) P + p starting at slot
// m0 P h + k, its top separator at slot m0 P h - 1 + z h.  Per-instance
// scratch (U, Racc, Tacc, recursion W) is indexed by m P + p.
static int pfactor_step(bta_ctx_t c, const PLay& L, int m0, int cnt, int k, cudaStream_t s) {
    const int b = L.b, a = L.a, I = cnt * L.P;
    const long long bb = L.bb, ab = L.ab, sP = (long long)L.h * bb, sPR = (long long)L.h * ab;
    const long long s0 = (long long)m0 * L.blk + k, t0 = (long long)m0 * L.blk - 1;
    const long long z0 = (long long)m0 * L.P;
    const BtaStore &Q = c->Q, &Lf = c->L;
    const GemmExec* ex = &c->exec;
    PTimeStore* st = c->pts;
    double* X = c->Linv;
    double* F = st->F;
    double* U = st->U + z0 * bb;
    // 1. L_ii and X_i
    BTA_TRY(chol_inv64(s, Lf.D + s0 * bb, b, X + s0 * bb, b, b, (long long)k * b, c->status, st->W + z0 * st->sW,
                       c->leaf, ex, I, sP, sP, st->sW, m0, c->batch, c->fork, 0, L.P));
    // 2. L_{i+1,i} = B_i X_i^T ; D~_{i+1} -= L_{i+1,i} L_{i+1,i}^T
    G g1(b, b, b);
    g1.A(Q.B + s0 * bb, b, 0, 0, sP).B(X + s0 * bb, b, 1, 2, sP).C(Lf.B + s0 * bb, b, sP).batch(I);
    BTA_TRY(gemm_exec(ex, s, g1.g));
    G g2(b, b, b);
    g2.A(Lf.B + s0 * bb, b, 0, 0, sP).B(Lf.B + s0 * bb, b, 1, 0, sP).lower().batch(I);
    acc(g2, Lf.D + (s0 + 1) * bb, b, sP);
    BTA_TRY(gemm_exec(ex, s, g2.g));
    // 3. fill rows to the top separator: L_{sigma,i} = U X_i^T, U_first = B_{sigma}^T
    G g3(b, b, b);
    if (k == 0) g3.A(Q.B + (s0 - 1) * bb, b, 1, 0, sP);
    else g3.A(U, b, 0, 0, bb);
    g3.B(X + s0 * bb, b, 1, 2, sP).C(F + s0 * bb, b, sP).batch(I);
    BTA_TRY(gemm_exec(ex, s, g3.g));
    G g4(b, b, b);
    g4.A(F + s0 * bb, b, 0, 0, sP).B(F + s0 * bb, b, 1, 0, sP).lower().batch(I);
    acc(g4, Lf.D + t0 * bb, b, sP);
    BTA_TRY(gemm_exec(ex, s, g4.g));
    if (k < L.l - 1) {
        // the next block is interior: U_{i+1} = -L_{sigma,i} L_{i+1,i}^T
        G g5(b, b, b);
        g5.A(F + s0 * bb, b, 0, 0, sP).B(Lf.B + s0 * bb, b, 1, 0, sP).C(U, b, bb).alpha(-1.0).batch(I);
        BTA_TRY(gemm_exec(ex, s, g5.g));
    } else {
        // the next block is the bottom separator: reduced coupling in the B slot of the top one
        G g6(b, b, b);
        g6.A(Lf.B + s0 * bb, b, 0, 0, sP).B(F + s0 * bb, b, 1, 0, sP).C(Lf.B + t0 * bb, b, sP).alpha(-1.0)
            .batch(I);
        BTA_TRY(gemm_exec(ex, s, g6.g));
    }
    // 4. arrow rows
    if (a > 0) {
        double* Racc = st->Racc + z0 * ab;
        BTA_TRY(copy_mat64(s, Lf.R + s0 * ab, a, Racc, a, a, b, 0, I, sPR, ab));
        G g7(a, b, b);
        g7.A(Racc, a, 0, 0, ab).B(X + s0 * bb, b, 1, 2, sP).C(Lf.R + s0 * ab, a, sPR).batch(I);
        BTA_TRY(gemm64(s, g7.g));
        G g8(a, a, b);
        g8.A(Lf.R + s0 * ab, a, 0, 0, sPR).B(Lf.R + s0 * ab, a, 1, 0, sPR).lower().batch(I);
        acc(g8, st->Tacc + z0 * a * a, a, (long long)a * a);
        BTA_TRY(gemm64(s, g8.g));
        G g9(a, b, b);
        g9.A(Lf.R + s0 * ab, a, 0, 0, sPR).B(F + s0 * bb, b, 1, 0, sP).batch(I);
        acc(g9, Lf.R + t0 * ab, a, sPR);
        BTA_TRY(gemm64(s, g9.g));
        G g10(a, b, b);
        g10.A(Lf.R + s0 * ab, a, 0, 0, sPR).B(Lf.B + s0 * bb, b, 1, 0, sP).batch(I);
        acc(g10, Lf.R + (s0 + 1) * ab, a, sPR);
        BTA_TRY(gemm64(s, g10.g));
    }
    return BTA_OK;
}

int pfactor_impl(bta_ctx_t c, int m0, int cnt, cudaStream_t s) {
    const PLay L = layout(c, c->tparts);
    const int b = L.b, a = L.a;
    const long long bb = L.bb, ab = L.ab;
    const BtaStore &Q = c->Q, &Lf = c->L;
    PTimeStore* st = c->pts;
    const long long sD = Lf.sD, sR = Lf.sR, sT = Lf.sT, sX = c->sLinv, z0 = (long long)m0 * L.P;
    // the real diagonal blocks, arrow rows and tip start from Q (the padding keeps its identities)
    for (int m = m0; m < m0 + cnt; ++m) {
        BTA_TRY(copy_mat64(s, Q.D + m * Q.sD, b, Lf.D + m * sD, b, b, b, 1, L.n, bb, bb));
        if (a > 0) BTA_TRY(copy_mat64(s, Q.R + m * Q.sR, a, Lf.R + m * sR, a, a, b, 0, L.n, ab, ab));
    }
    if (a > 0) {
        BTA_TRY(copy_mat64(s, Q.T + m0 * Q.sT, a, Lf.T + m0 * sT, a, a, a, 1, cnt, Q.sT, sT));
        BTA_CUDA_TRY(cudaMemsetAsync(st->Tacc + z0 * a * a, 0, (size_t)cnt * L.P * a * a * sizeof(double), s));
    }
    // interiors: every partition of every matrix in the same launches
    for (int k = 0; k < L.l; ++k) BTA_TRY(pfactor_step(c, L, m0, cnt, k, s));
    if (a > 0) {
        add_tacc_kernel<<<dim3((a * a + 255) / 256, cnt), 256, 0, s>>>(Lf.T + m0 * sT, sT, st->Tacc + z0 * a * a, a,
                                                                      L.P);
        BTA_LAUNCH_CHECK();
    }
    // the reduced BTA system on the separators, all matrices together
    double* WgB = st->Wg + (long long)m0 * bb;
    double* WgR = st->Wg + (long long)c->nmat * bb + (long long)m0 * ab;
    for (int j = 1; j < L.P; ++j) {
        const long long sj = (long long)m0 * L.blk + (long long)j * L.h - 1;
        const bool more = j < L.P - 1;
        const long long sn = sj + L.h;
        BTA_TRY(chol_inv64(s, Lf.D + sj * bb, b, c->Linv + sj * bb, b, b, (long long)(j * L.h - 1) * b, c->status,
                           st->W + z0 * st->sW, c->leaf, &c->exec, cnt, sD, sX, st->sW, m0, c->batch, c->fork));
        if (more) {
            BTA_TRY(copy_mat64(s, Lf.B + sj * bb, b, WgB, b, b, b, 0, cnt, Lf.sB, bb));
            G g1(b, b, b);
            g1.A(WgB, b, 0, 0, bb).B(c->Linv + sj * bb, b, 1, 2, sX).C(Lf.B + sj * bb, b, Lf.sB).batch(cnt);
            BTA_TRY(gemm_exec(&c->exec, s, g1.g));
            G g2(b, b, b);
            g2.A(Lf.B + sj * bb, b, 0, 0, Lf.sB).B(Lf.B + sj * bb, b, 1, 0, Lf.sB).lower().batch(cnt);
            acc(g2, Lf.D + sn * bb, b, sD);
            BTA_TRY(gemm_exec(&c->exec, s, g2.g));
        }
        if (a > 0) {
            BTA_TRY(copy_mat64(s, Lf.R + sj * ab, a, WgR, a, a, b, 0, cnt, sR, ab));
            G g3(a, b, b);
            g3.A(WgR, a, 0, 0, ab).B(c->Linv + sj * bb, b, 1, 2, sX).C(Lf.R + sj * ab, a, sR).batch(cnt);
            BTA_TRY(gemm64(s, g3.g));
            G g4(a, a, b);
            g4.A(Lf.R + sj * ab, a, 0, 0, sR).B(Lf.R + sj * ab, a, 1, 0, sR).lower().batch(cnt);
            acc(g4, Lf.T + m0 * sT, a, sT);
            BTA_TRY(gemm64(s, g4.g));
            if (more) {
                G g5(a, b, b);
                g5.A(Lf.R + sj * ab, a, 0, 0, sR).B(Lf.B + sj * bb, b, 1, 0, Lf.sB).batch(cnt);
                acc(g5, Lf.R + sn * ab, a, sR);
                BTA_TRY(gemm64(s, g5.g));
            }
        }
    }
    if (a > 0)
        BTA_TRY(chol_inv64(s, Lf.T + m0 * sT, a, c->Linv + m0 * sX + c->tip_off, a, a, (long long)L.n * b, c->status,
                           st->W + z0 * st->sW, c->leaf, nullptr, cnt, sT, sX, st->sW, m0, c->batch));
    for (int m = m0; m < m0 + cnt; ++m) c->factored[m] = 1;
    return BTA_OK;
}

// ---------------------------------------------------------------------------- solve

// x_j = Q_{m0+j}^{-1} r_j with the partitioned factors (vectors N apart, not
// padded): per matrix, forward over the interiors (the partitions of a step
// together), the separators and the tip, then backward in the reverse order.
// Step k covers partitions 0..P-1 while k < l_last and 0..P-2 after; the
// last partition's block n-1 has no successor; the fill terms need p >= 1.
int psolve_impl(bta_ctx_t c, int m0, int cnt, const double* r, double* x, cudaStream_t s) {
    const PLay L = layout(c, c->tparts);
    const int b = L.b, a = L.a, P = L.P;
    const long long bb = L.bb, N = c->N, nb = (long long)L.n * b;
    const long long sP = (long long)L.h * bb, sPv = (long long)L.h * b;
    const BtaStore& Lf = c->L;
    auto pc_of = [&](int k) { return k < L.l_last ? P : P - 1; };
    auto pnext_of = [&](int k) { return k == L.l_last - 1 ? P - 1 : pc_of(k); };
    for (int j = 0; j < cnt; ++j) {
        const int m = m0 + j;
        const long long base = (long long)m * L.blk;      // slot of block 0
        const double* LB = Lf.B + base * bb;
        const double* LR = Lf.R + m * Lf.sR;
        const double* X = c->Linv + m * c->sLinv;
        const double* XT = X + c->tip_off;
        const double* F = c->pts->F + base * bb;
        double* z = vec_row(c, VEC_Z, m);
        double* tmp = vec_row(c, VEC_TMP, m);
        const double* rj = r + j * N;
        double* xj = x + j * N;
        BTA_CUDA_TRY(cudaMemcpyAsync(tmp, rj, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        // forward, interiors: z_i = X_i tmp_i; tmp_{i+1} -= L_{i+1,i} z_i; tmp_{sigma_p} -= L_{sigma_p,i} z_i
        for (int k = 0; k < L.l; ++k) {
            const int pc = pc_of(k), pn = pnext_of(k);
            BTA_TRY(gemv64(s, b, b, X + k * bb, b, 0, 1, tmp + (long long)k * b, 1.0, nullptr, 0.0,
                           z + (long long)k * b, pc, sP, sPv, sPv));
            if (pn > 0)
                BTA_TRY(gemv64(s, b, b, LB + k * bb, b, 0, 0, z + (long long)k * b, -1.0, tmp + (long long)(k + 1) * b,
                               1.0, tmp + (long long)(k + 1) * b, pn, sP, sPv, sPv));
            if (pc > 1) {
                const long long i1 = L.h + k, s1 = L.h - 1;   // partition 1's block and top separator
                BTA_TRY(gemv64(s, b, b, F + i1 * bb, b, 0, 0, z + i1 * b, -1.0, tmp + s1 * b, 1.0, tmp + s1 * b,
                               pc - 1, sP, sPv, sPv));
            }
        }
        // forward, separators
        for (int jj = 1; jj < P; ++jj) {
            const long long sj = (long long)jj * L.h - 1;
            BTA_TRY(gemv64(s, b, b, X + sj * bb, b, 0, 1, tmp + sj * b, 1.0, nullptr, 0.0, z + sj * b));
            if (jj < P - 1)
                BTA_TRY(gemv64(s, b, b, LB + sj * bb, b, 0, 0, z + sj * b, -1.0, tmp + (sj + L.h) * b, 1.0,
                               tmp + (sj + L.h) * b));
        }
        // tip: z_t = X_t (r_t - sum_i L_{t,i} z_i), x_t = X_t^T z_t, then z_i -= L_{t,i}^T x_t
        if (a > 0) {
            BTA_TRY(gemv64(s, a, (int)nb, LR, a, 0, 0, z, -1.0, rj + nb, 1.0, tmp + nb));
            BTA_TRY(gemv64(s, a, a, XT, a, 0, 1, tmp + nb, 1.0, nullptr, 0.0, z + nb));
            BTA_TRY(gemv64(s, a, a, XT, a, 1, 2, z + nb, 1.0, nullptr, 0.0, xj + nb));
            BTA_TRY(gemv64(s, (int)nb, a, LR, a, 1, 0, xj + nb, -1.0, z, 1.0, z));
        }
        // backward, separators: x_s = X_s^T (z_s - L_{s+,s}^T x_{s+})
        for (int jj = P - 1; jj >= 1; --jj) {
            const long long sj = (long long)jj * L.h - 1;
            const double* zs = z + sj * b;
            if (jj < P - 1) {
                BTA_TRY(gemv64(s, b, b, LB + sj * bb, b, 1, 0, xj + (sj + L.h) * b, -1.0, zs, 1.0, tmp + sj * b));
                zs = tmp + sj * b;
            }
            BTA_TRY(gemv64(s, b, b, X + sj * bb, b, 1, 2, zs, 1.0, nullptr, 0.0, xj + sj * b));
        }
        // backward, interiors: x_i = X_i^T (z_i - L_{i+1,i}^T x_{i+1} - L_{sigma_p,i}^T x_{sigma_p})
        for (int k = L.l - 1; k >= 0; --k) {
            const int pc = pc_of(k), pn = pnext_of(k);
            BTA_CUDA_TRY(cudaMemcpy2DAsync(tmp + (long long)k * b, sPv * sizeof(double), z + (long long)k * b,
                                           sPv * sizeof(double), b * sizeof(double), pc, cudaMemcpyDeviceToDevice, s));
            if (pn > 0)
                BTA_TRY(gemv64(s, b, b, LB + k * bb, b, 1, 0, xj + (long long)(k + 1) * b, -1.0, tmp + (long long)k * b,
                               1.0, tmp + (long long)k * b, pn, sP, sPv, sPv));
            if (pc > 1) {
                const long long i1 = L.h + k, s1 = L.h - 1;
                BTA_TRY(gemv64(s, b, b, F + i1 * bb, b, 1, 0, xj + s1 * b, -1.0, tmp + i1 * b, 1.0, tmp + i1 * b,
                               pc - 1, sP, sPv, sPv));
            }
            BTA_TRY(gemv64(s, b, b, X + k * bb, b, 1, 2, tmp + (long long)k * b, 1.0, nullptr, 0.0,
                           xj + (long long)k * b, pc, sP, sPv, sPv));
        }
    }
    return BTA_OK;
}

// ---------------------------------------------------------------------------- selected inversion

// Sigma_tt of matrix z / P copied to instance z (the products with Sigma_tt
// run over instances, whose stride is not the matrices')
static __global__ void replicate_tip_kernel(const double* ST, long long sT, int a, int P, double* out) {
    const int z = blockIdx.y;
    const double* src = ST + (long long)(z / P) * sT;
    for (int e = threadIdx.x; e < a * a; e += blockDim.x) out[(long long)z * a * a + e] = src[e];
}

int pselinv_impl(bta_ctx_t c, int m0, int cnt, cudaStream_t s) {
    const PLay L = layout(c, c->tparts);
    const int b = L.b, a = L.a, I = cnt * L.P;
    const long long bb = L.bb, ab = L.ab, sP = (long long)L.h * bb, sPR = (long long)L.h * ab;
    const BtaStore &Lf = c->L, &S = c->S;
    const GemmExec* ex = &c->exec;
    PTimeStore* st = c->pts;
    const long long z0 = (long long)m0 * L.P, sX = c->sLinv, sD = S.sD, sR = S.sR, sT = S.sT;
    const double* X = c->Linv;
    const double* F = st->F;
    double* SF = st->SF;
    // per-instance scratch: G (in U), H (in the recursion scratch), Fa (in Racc),
    // Sigma_tt per instance (in Tacc), reduced Sigma_{sigma_{p+1},sigma_p} (RS)
    double* Gs = st->U + z0 * bb;
    double* Hs = st->W + z0 * st->sW;
    const long long sH = st->sW;
    double* Fa = st->Racc + z0 * ab;
    double* STi = st->Tacc + z0 * a * a;
    double* RS = st->RS + z0 * bb;
    BTA_CUDA_TRY(cudaMemsetAsync(RS, 0, (size_t)I * bb * sizeof(double), s));
    // Sigma_tt = X_t^T X_t
    if (a > 0) {
        G g(a, a, a);
        g.A(X + m0 * sX + c->tip_off, a, 1, 2, sX).B(X + m0 * sX + c->tip_off, a, 0, 1, sX).C(S.T + m0 * sT, a, sT)
            .batch(cnt);
        BTA_TRY(gemm64(s, g.g));
    }
    // ---- the reduced system, separators P-1 .. 1, all matrices together
    for (int j = L.P - 1; j >= 1; --j) {
        const long long sj = (long long)m0 * L.blk + (long long)j * L.h - 1;
        const bool more = j < L.P - 1;
        const long long sn = sj + L.h;
        double* RSj = RS + (long long)j * bb;                 // instance (m, j), P b^2 apart
        const long long sRS = (long long)L.P * bb;
        if (a > 0) {
            G g(a, b, b);
            g.A(Lf.R + sj * ab, a, 0, 0, Lf.sR).B(X + sj * bb, b, 0, 1, sX).C(Fa, a, ab).batch(cnt);
            BTA_TRY(gemm64(s, g.g));
        }
        if (more) {
            G g(b, b, b);
            g.A(Lf.B + sj * bb, b, 0, 0, Lf.sB).B(X + sj * bb, b, 0, 1, sX).C(Gs, b, bb).batch(cnt);
            BTA_TRY(gemm_exec(ex, s, g.g));
            G g1(b, b, b);
            g1.A(S.D + sn * bb, b, 0, 0, sD).B(Gs, b, 0, 0, bb).C(RSj, b, sRS).alpha(-1.0).batch(cnt);
            BTA_TRY(gemm_exec(ex, s, g1.g));
            if (a > 0) {
                G g2(b, b, a);
                g2.A(S.R + sn * ab, a, 1, 0, sR).B(Fa, a, 0, 0, ab).batch(cnt);
                acc(g2, RSj, b, sRS);
                BTA_TRY(gemm_exec(ex, s, g2.g));
            }
        }
        if (a > 0) {
            G g3(a, b, a);
            g3.A(S.T + m0 * sT, a, 0, 0, sT).B(Fa, a, 0, 0, ab).C(S.R + sj * ab, a, sR).alpha(-1.0).batch(cnt);
            BTA_TRY(gemm64(s, g3.g));
            if (more) {
                G g4(a, b, b);
                g4.A(S.R + sn * ab, a, 0, 0, sR).B(Gs, b, 0, 0, bb).batch(cnt);
                acc(g4, S.R + sj * ab, a, sR);
                BTA_TRY(gemm64(s, g4.g));
            }
        }
        G g5(b, b, b);
        g5.A(X + sj * bb, b, 1, 2, sX).B(X + sj * bb, b, 0, 1, sX).C(S.D + sj * bb, b, sD).lower().batch(cnt);
        BTA_TRY(gemm_exec(ex, s, g5.g));
        if (more) {
            G g6(b, b, b);
            g6.A(Gs, b, 1, 0, bb).B(RSj, b, 0, 0, sRS).lower().batch(cnt);
            acc(g6, S.D + sj * bb, b, sD);
            BTA_TRY(gemm_exec(ex, s, g6.g));
        }
        if (a > 0) {
            G g7(b, b, a);
            g7.A(Fa, a, 1, 0, ab).B(S.R + sj * ab, a, 0, 0, sR).lower().batch(cnt);
            acc(g7, S.D + sj * bb, b, sD);
            BTA_TRY(gemm_exec(ex, s, g7.g));
        }
        BTA_TRY(symmetrize_lower64(s, S.D + sj * bb, b, b, cnt, sD));
    }
    if (a > 0) {
        replicate_tip_kernel<<<dim3(1, I), 256, 0, s>>>(S.T + m0 * sT, sT, a, L.P, STi);
        BTA_LAUNCH_CHECK();
    }
    // ---- interiors, backwards, every partition of every matrix together
    for (int k = L.l - 1; k >= 0; --k) {
        const long long s0 = (long long)m0 * L.blk + k, t0 = (long long)m0 * L.blk - 1;
        const bool next_sep = k == L.l - 1;
        // G = L_{i+1,i} X_i, H = L_{sigma,i} X_i, Fa = L_{t,i} X_i
        G gg(b, b, b);
        gg.A(Lf.B + s0 * bb, b, 0, 0, sP).B(X + s0 * bb, b, 0, 1, sP).C(Gs, b, bb).batch(I);
        BTA_TRY(gemm_exec(ex, s, gg.g));
        G gh(b, b, b);
        gh.A(F + s0 * bb, b, 0, 0, sP).B(X + s0 * bb, b, 0, 1, sP).C(Hs, b, sH).batch(I);
        BTA_TRY(gemm_exec(ex, s, gh.g));
        if (a > 0) {
            G gf(a, b, b);
            gf.A(Lf.R + s0 * ab, a, 0, 0, sPR).B(X + s0 * bb, b, 0, 1, sP).C(Fa, a, ab).batch(I);
            BTA_TRY(gemm64(s, gf.g));
        }
        // Sigma_{i+1,i} = -(Sigma_{i+1,i+1} G + Sigma_{i+1,sigma} H + Sigma_{t,i+1}^T Fa)
        G g1(b, b, b);
        g1.A(S.D + (s0 + 1) * bb, b, 0, 0, sP).B(Gs, b, 0, 0, bb).C(S.B + s0 * bb, b, sP).alpha(-1.0).batch(I);
        BTA_TRY(gemm_exec(ex, s, g1.g));
        G g2(b, b, b);
        if (next_sep) g2.A(RS, b, 0, 0, bb);                     // Sigma_{sigma_{p+1},sigma_p}
        else g2.A(SF + (s0 + 1) * bb, b, 1, 0, sP);             // Sigma_{sigma_p,i+1}^T
        g2.B(Hs, b, 0, 0, sH).batch(I);
        acc(g2, S.B + s0 * bb, b, sP);
        BTA_TRY(gemm_exec(ex, s, g2.g));
        if (a > 0) {
            G g3(b, b, a);
            g3.A(S.R + (s0 + 1) * ab, a, 1, 0, sPR).B(Fa, a, 0, 0, ab).batch(I);
            acc(g3, S.B + s0 * bb, b, sP);
            BTA_TRY(gemm_exec(ex, s, g3.g));
        }
        // Sigma_{sigma,i} = -(Sigma_{sigma,i+1} G + Sigma_{sigma,sigma} H + Sigma_{t,sigma}^T Fa)
        G g4(b, b, b);
        g4.A(S.D + t0 * bb, b, 0, 0, sP).B(Hs, b, 0, 0, sH).C(SF + s0 * bb, b, sP).alpha(-1.0).batch(I);
        BTA_TRY(gemm_exec(ex, s, g4.g));
        G g5(b, b, b);
        if (next_sep) g5.A(RS, b, 1, 0, bb);                     // Sigma_{sigma_p,sigma_{p+1}}
        else g5.A(SF + (s0 + 1) * bb, b, 0, 0, sP);
        g5.B(Gs, b, 0, 0, bb).batch(I);
        acc(g5, SF + s0 * bb, b, sP);
        BTA_TRY(gemm_exec(ex, s, g5.g));
        if (a > 0) {
            G g6(b, b, a);
            g6.A(S.R + t0 * ab, a, 1, 0, sPR).B(Fa, a, 0, 0, ab).batch(I);
            acc(g6, SF + s0 * bb, b, sP);
            BTA_TRY(gemm_exec(ex, s, g6.g));
            // Sigma_{t,i} = -(Sigma_{t,i+1} G + Sigma_{t,sigma} H + Sigma_tt Fa)
            G g7(a, b, a);
            g7.A(STi, a, 0, 0, (long long)a * a).B(Fa, a, 0, 0, ab).C(S.R + s0 * ab, a, sPR).alpha(-1.0).batch(I);
            BTA_TRY(gemm64(s, g7.g));
            G g8(a, b, b);
            g8.A(S.R + (s0 + 1) * ab, a, 0, 0, sPR).B(Gs, b, 0, 0, bb).batch(I);
            acc(g8, S.R + s0 * ab, a, sPR);
            BTA_TRY(gemm64(s, g8.g));
            G g9(a, b, b);
            g9.A(S.R + t0 * ab, a, 0, 0, sPR).B(Hs, b, 0, 0, sH).batch(I);
            acc(g9, S.R + s0 * ab, a, sPR);
            BTA_TRY(gemm64(s, g9.g));
        }
        // Sigma_ii = X^T X - G^T Sigma_{i+1,i} - H^T Sigma_{sigma,i} - Fa^T Sigma_{t,i}
        G g10(b, b, b);
        g10.A(X + s0 * bb, b, 1, 2, sP).B(X + s0 * bb, b, 0, 1, sP).C(S.D + s0 * bb, b, sP).lower().batch(I);
        BTA_TRY(gemm_exec(ex, s, g10.g));
        G g11(b, b, b);
        g11.A(Gs, b, 1, 0, bb).B(S.B + s0 * bb, b, 0, 0, sP).lower().batch(I);
        acc(g11, S.D + s0 * bb, b, sP);
        BTA_TRY(gemm_exec(ex, s, g11.g));
        G g12(b, b, b);
        g12.A(Hs, b, 1, 0, sH).B(SF + s0 * bb, b, 0, 0, sP).lower().batch(I);
        acc(g12, S.D + s0 * bb, b, sP);
        BTA_TRY(gemm_exec(ex, s, g12.g));
        if (a > 0) {
            G g13(b, b, a);
            g13.A(Fa, a, 1, 0, ab).B(S.R + s0 * ab, a, 0, 0, sPR).lower().batch(I);
            acc(g13, S.D + s0 * bb, b, sP);
            BTA_TRY(gemm_exec(ex, s, g13.g));
        }
        BTA_TRY(symmetrize_lower64(s, S.D + s0 * bb, b, b, I, sP));
    }
    // BTA-pattern block (first_p, sigma_p) = Sigma_{sigma_p, first_p}^T (partition 0 writes its padding slot)
    transpose_copy_kernel<<<dim3((int)std::min<long long>((bb + 255) / 256, 1216), I), 256, 0, s>>>(
        SF + (long long)m0 * L.blk * bb, S.B + ((long long)m0 * L.blk - 1) * bb, b, sP, sP);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

// ---------------------------------------------------------------------------- entry point

extern "C" int bta_set_time_partitions(bta_ctx_t ctx, int P) {
    if (!ctx || P < 1) return BTA_ERR_ARG;
    if (P > 1 && ctx->lowmem) return BTA_ERR_STATE;   // the low-memory layout is sequential only
    if (P > 1) {
        // every partition holds an interior block, and L_tt^{-1} fits one block slot
        const PLay L = layout(ctx, P);
        if (L.l_last < 1 || ctx->a > ctx->b) return BTA_ERR_ARG;
    }
    if (P == ctx->tparts) return BTA_OK;
    BTA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    BTA_CUDA_TRY(cudaDeviceSynchronize());
    if (ctx->fobj_graph) {
        cudaGraphExecDestroy(ctx->fobj_graph);
        ctx->fobj_graph = nullptr;
        ctx->graph_calls = 1;
    }
    std::fill(ctx->factored.begin(), ctx->factored.end(), 0);
    const int rc = relayout(ctx, P);
    if (rc != BTA_OK) {
        // back to the sequential layout (which needs less memory); if even that
        // fails the context has no storage and is only fit for bta_destroy
        ptime_free(ctx);
        ctx->tparts = 1;
        relayout(ctx, 1);
    }
    return rc;
}
