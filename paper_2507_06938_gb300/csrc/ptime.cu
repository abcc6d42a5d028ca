// Parallel-in-time BTA factorisation, solve and selected inversion on one
// GPU: the time-domain partitioning of Sections IV-C and IV-D.3 (nested
// dissection over the time blocks, which breaks the sequential dependency of
// the block recurrences) restated for a single device, where the P partitions
// run together as one batch of every launch instead of on P processes.
//
// Time blocks 0..n-1 are cut by P - 1 separator blocks sigma_p = p h - 1
// (p = 1..P-1, h = floor((n + 1) / P)); partition p's interior is the blocks
// between sigma_p and sigma_{p+1} (partition 0 starts at block 0, partition
// P-1 runs to block n-1 and may be longer).  Eliminating the interiors first
// leaves a BTA system on the separators (P - 1 blocks and the arrow tip),
// which is factored by the ordinary recurrence.  For interior block i of
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
// The fill rows L_{sigma_p,i} live in a per-matrix block array F; the reduced
// coupling Q~[sigma_{p+1}, sigma_p] in the otherwise unused B slot of sigma_p.
// The selected inversion runs the reduced system first, then every interior
// backwards, with the rows {i+1, sigma_p, tip} of column i:
//   G = L_{i+1,i} X_i, H = L_{sigma_p,i} X_i, F = L_{t,i} X_i
//   Sigma_{i+1,i}     = -(Sigma_{i+1,i+1} G + Sigma_{i+1,sigma_p} H + Sigma_{t,i+1}^T F)
//   Sigma_{sigma_p,i} = -(Sigma_{sigma_p,i+1} G + Sigma_{sigma_p,sigma_p} H + Sigma_{t,sigma_p}^T F)
//   Sigma_{t,i}       = -(Sigma_{t,i+1} G + Sigma_{t,sigma_p} H + Sigma_tt F)
//   Sigma_ii          = X_i^T X_i - G^T Sigma_{i+1,i} - H^T Sigma_{sigma_p,i} - F^T Sigma_{t,i}
// (from Sigma L = L^{-T} on block column i); Sigma_{sigma_p,i} is kept in a
// second block array, and the BTA-pattern block (first_p, sigma_p) is its
// transpose.  Work per interior step of a middle partition: five b x b x b
// products in the factorisation (two for the sequential recurrence) and nine
// in the selected inversion (five): more flops, but n/P + P instead of n
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

// T += sum_p Tacc_p (lower entries), one thread per entry
__global__ void add_tacc_kernel(double* T, const double* Tacc, int a, int P) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a * a) return;
    const int i = e % a, j = e / a;
    if (i < j) return;
    double s = 0.0;
    for (int p = 0; p < P; ++p) s += Tacc[(long long)p * a * a + e];
    T[e] += s;
}

struct PLay {
    int n, b, a, P, h, l, l_last;
    long long bb, ab;
    int sep(int p) const { return p * h - 1; }        // separator sigma_p, p = 1..P-1
    int first(int p) const { return p * h; }          // first interior block of partition p
};

PLay layout(const bta_ctx_s* c) {
    PLay L;
    L.n = c->n; L.b = c->b; L.a = c->a; L.P = c->tparts;
    L.h = (c->n + 1) / c->tparts;
    L.l = L.h - 1;
    L.l_last = c->n - (c->tparts - 1) * L.h;
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

// Block-array storage of the partitioned path for every matrix (fill rows of
// the factor and of the selected inverse) and its scratch (one matrix at a
// time): allocated by bta_set_time_partitions.
struct PTimeStore {
    double* F = nullptr;      // nmat x n b^2: L_{sigma_p, i}
    double* SF = nullptr;     // nmat x n b^2: Sigma_{sigma_p, i}
    double* U = nullptr;      // P b^2: fill coupling U_i
    double* Racc = nullptr;   // P a b: arrow rows before their product
    double* Tacc = nullptr;   // P a^2
    double* RS = nullptr;     // P b^2: reduced Sigma_{sigma_{p+1}, sigma_p}
    double* W = nullptr;      // P x sW: recursion scratch of the batched diagonal factorisations
    double* Wg = nullptr;     // b^2 (+ a b): in-place product scratch
    long long sW = 0;
};

int ptime_alloc(bta_ctx_t c, int P) {
    PTimeStore* st = c->pts;
    if (!st) st = c->pts = new PTimeStore();
    const long long bb = (long long)c->b * c->b, nb2 = (long long)c->n * bb;
    auto al = [](double** p, size_t n) -> int {
        if (*p) cudaFree(*p);
        *p = nullptr;
        cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(double));
        if (e != cudaSuccess) {
            *p = nullptr;
            return bta_cuda_fail(e);
        }
        return BTA_OK;
    };
    st->sW = bb + bb / 2 + 2LL * c->b + 64;
    BTA_TRY(al(&st->F, (size_t)c->nmat * nb2));
    BTA_TRY(al(&st->SF, (size_t)c->nmat * nb2));
    BTA_TRY(al(&st->U, (size_t)P * bb));
    BTA_TRY(al(&st->Racc, (size_t)P * c->a * c->b));
    BTA_TRY(al(&st->Tacc, (size_t)P * c->a * c->a));
    BTA_TRY(al(&st->RS, (size_t)P * bb));
    BTA_TRY(al(&st->W, (size_t)P * st->sW));
    BTA_TRY(al(&st->Wg, (size_t)bb + (size_t)c->a * c->b));
    return BTA_OK;
}

void ptime_free(bta_ctx_t c) {
    if (!c->pts) return;
    double* ps[] = {c->pts->F, c->pts->SF, c->pts->U, c->pts->Racc, c->pts->Tacc, c->pts->RS, c->pts->W, c->pts->Wg};
    for (double* p : ps)
        if (p) cudaFree(p);
    delete c->pts;
    c->pts = nullptr;
}

// Which partitions of a step continue into an interior block, and which end
// at their bottom separator.  A step (k, p0, pc) runs interior step k of
// partitions p0 .. p0 + pc - 1 (all P for k < l, only the last one after).
struct StepRanges {
    int last;            // last partition of the step
    int pnext;           // partitions p0 .. p0 + pnext - 1 have a block i + 1
    int q0, qc;          // partitions with a top separator (p >= 1)
    int ni0, nic;        // p >= 1 partitions whose block i + 1 is interior
    int ns0, nsc;        // p >= 1 partitions whose block i + 1 is their bottom separator
};

StepRanges ranges(const PLay& L, int k, int p0, int pc) {
    StepRanges r;
    r.last = p0 + pc - 1;
    const bool final_in = r.last == L.P - 1;
    r.pnext = (final_in && k == L.l_last - 1) ? pc - 1 : pc;
    r.q0 = std::max(p0, 1);
    r.qc = std::max(0, r.last - r.q0 + 1);
    r.ni0 = r.q0; r.nic = 0; r.ns0 = r.q0; r.nsc = 0;
    if (r.qc == 0) return r;
    if (k < L.l - 1) {
        r.nic = r.qc;                                  // every partition continues
    } else if (k == L.l - 1) {
        const int se = std::min(r.last, L.P - 2);      // partitions P-1 has no bottom separator
        r.nsc = std::max(0, se - r.q0 + 1);
        if (final_in && L.l_last > L.l) { r.ni0 = L.P - 1; r.nic = 1; }
    } else {
        if (k < L.l_last - 1) { r.ni0 = L.P - 1; r.nic = 1; }   // the last partition's extra steps
    }
    return r;
}

// ---------------------------------------------------------------------------- factorisation

// Interior step k of partitions p0 .. p0 + pc - 1 of matrix m.  Scratch per
// partition: U (absolute partition index, it lives across steps), Racc and
// Tacc (relative to p0).
static int pfactor_step(bta_ctx_t c, const PLay& L, int m, int k, int p0, int pc, cudaStream_t s) {
    const int b = L.b, a = L.a;
    const long long bb = L.bb, ab = L.ab, sP = (long long)L.h * bb, sPR = (long long)L.h * ab;
    const BtaStore &Q = c->Q, &Lf = c->L;
    const GemmExec* ex = &c->exec;
    PTimeStore* st = c->pts;
    const StepRanges R = ranges(L, k, p0, pc);
    const int i0 = p0 * L.h + k;
    auto blk = [&](int p) { return p * L.h + k; };
    double* LD = Lf.D + m * Lf.sD;
    double* LB = Lf.B + m * Lf.sB;
    double* LR = Lf.R + m * Lf.sR;
    const double* QB = Q.B + m * Q.sB;
    double* X = c->Linv + m * c->sLinv;
    double* F = st->F + (long long)m * L.n * bb;
    // 1. L_ii and X_i
    BTA_TRY(chol_inv64(s, LD + i0 * bb, b, X + i0 * bb, b, b, (long long)i0 * b, c->status, st->W, c->leaf, ex, pc,
                       sP, sP, st->sW, m, c->batch, c->fork));
    // 2. L_{i+1,i} = B_i X_i^T ; D~_{i+1} -= L_{i+1,i} L_{i+1,i}^T (block i+1 interior or separator)
    if (R.pnext > 0) {
        G g1(b, b, b);
        g1.A(QB + i0 * bb, b, 0, 0, sP).B(X + i0 * bb, b, 1, 2, sP).C(LB + i0 * bb, b, sP).batch(R.pnext);
        BTA_TRY(gemm_exec(ex, s, g1.g));
        G g2(b, b, b);
        g2.A(LB + i0 * bb, b, 0, 0, sP).B(LB + i0 * bb, b, 1, 0, sP).lower().batch(R.pnext);
        acc(g2, LD + (i0 + 1) * bb, b, sP);
        BTA_TRY(gemm_exec(ex, s, g2.g));
    }
    // 3. fill rows to the top separator (p >= 1)
    if (R.qc > 0) {
        const int iq = blk(R.q0);
        G g3(b, b, b);
        if (k == 0) g3.A(QB + (iq - 1) * bb, b, 1, 0, sP);   // U = Q[sigma_p, first] = B_{sigma_p}^T
        else g3.A(st->U + R.q0 * bb, b, 0, 0, bb);
        g3.B(X + iq * bb, b, 1, 2, sP).C(F + iq * bb, b, sP).batch(R.qc);
        BTA_TRY(gemm_exec(ex, s, g3.g));
        G g4(b, b, b);
        g4.A(F + iq * bb, b, 0, 0, sP).B(F + iq * bb, b, 1, 0, sP).lower().batch(R.qc);
        acc(g4, LD + L.sep(R.q0) * bb, b, sP);
        BTA_TRY(gemm_exec(ex, s, g4.g));
        if (R.nic > 0) {
            // U_{i+1} = -L_{sigma_p,i} L_{i+1,i}^T
            const int in = blk(R.ni0);
            G g5(b, b, b);
            g5.A(F + in * bb, b, 0, 0, sP).B(LB + in * bb, b, 1, 0, sP).C(st->U + R.ni0 * bb, b, bb).alpha(-1.0)
                .batch(R.nic);
            BTA_TRY(gemm_exec(ex, s, g5.g));
        }
        if (R.nsc > 0) {
            // reduced coupling Q~[sigma_{p+1}, sigma_p] = -L_{i+1,i} L_{sigma_p,i}^T, in the B slot of sigma_p
            const int is = blk(R.ns0);
            G g6(b, b, b);
            g6.A(LB + is * bb, b, 0, 0, sP).B(F + is * bb, b, 1, 0, sP).C(LB + L.sep(R.ns0) * bb, b, sP)
                .alpha(-1.0).batch(R.nsc);
            BTA_TRY(gemm_exec(ex, s, g6.g));
        }
    }
    // 4. arrow rows: L_{t,i} = R~_i X_i^T ; T~ -= L_{t,i} L_{t,i}^T ; R~_{sigma_p} -= L_{t,i} L_{sigma_p,i}^T ;
    //    R~_{i+1} -= L_{t,i} L_{i+1,i}^T
    if (a > 0) {
        BTA_TRY(copy_mat64(s, LR + i0 * ab, a, st->Racc, a, a, b, 0, pc, sPR, ab));
        G g7(a, b, b);
        g7.A(st->Racc, a, 0, 0, ab).B(X + i0 * bb, b, 1, 2, sP).C(LR + i0 * ab, a, sPR).batch(pc);
        BTA_TRY(gemm64(s, g7.g));
        G g8(a, a, b);
        g8.A(LR + i0 * ab, a, 0, 0, sPR).B(LR + i0 * ab, a, 1, 0, sPR).lower().batch(pc);
        acc(g8, st->Tacc, a, (long long)a * a);
        BTA_TRY(gemm64(s, g8.g));
        if (R.qc > 0) {
            const int iq = blk(R.q0);
            G g9(a, b, b);
            g9.A(LR + iq * ab, a, 0, 0, sPR).B(F + iq * bb, b, 1, 0, sP).batch(R.qc);
            acc(g9, LR + L.sep(R.q0) * ab, a, sPR);
            BTA_TRY(gemm64(s, g9.g));
        }
        if (R.pnext > 0) {
            G g10(a, b, b);
            g10.A(LR + i0 * ab, a, 0, 0, sPR).B(LB + i0 * bb, b, 1, 0, sP).batch(R.pnext);
            acc(g10, LR + (i0 + 1) * ab, a, sPR);
            BTA_TRY(gemm64(s, g10.g));
        }
    }
    return BTA_OK;
}

int pfactor_impl(bta_ctx_t c, int m0, int cnt, cudaStream_t s) {
    const PLay L = layout(c);
    const int b = L.b, a = L.a;
    const long long bb = L.bb, ab = L.ab;
    const BtaStore &Q = c->Q, &Lf = c->L;
    PTimeStore* st = c->pts;
    for (int m = m0; m < m0 + cnt; ++m) {
        double* LD = Lf.D + m * Lf.sD;
        double* LB = Lf.B + m * Lf.sB;
        double* LR = Lf.R + m * Lf.sR;
        double* LT = Lf.T + m * Lf.sT;
        double* X = c->Linv + m * c->sLinv;
        // every diagonal block, arrow row and the tip start from Q
        BTA_TRY(copy_mat64(s, Q.D + m * Q.sD, b, LD, b, b, b, 1, L.n, bb, bb));
        if (a > 0) {
            BTA_TRY(copy_mat64(s, Q.R + m * Q.sR, a, LR, a, a, b, 0, L.n, ab, ab));
            BTA_TRY(copy_mat64(s, Q.T + m * Q.sT, a, LT, a, a, a, 1));
            BTA_CUDA_TRY(cudaMemsetAsync(st->Tacc, 0, (size_t)L.P * a * a * sizeof(double), s));
        }
        // interiors, all partitions together
        for (int k = 0; k < L.l; ++k) BTA_TRY(pfactor_step(c, L, m, k, 0, L.P, s));
        for (int k = L.l; k < L.l_last; ++k) BTA_TRY(pfactor_step(c, L, m, k, L.P - 1, 1, s));
        if (a > 0) {
            add_tacc_kernel<<<(a * a + 255) / 256, 256, 0, s>>>(LT, st->Tacc, a, L.P);
            BTA_LAUNCH_CHECK();
        }
        // the reduced BTA system on the separators: the sequential recurrence
        for (int j = 1; j < L.P; ++j) {
            const int sj = L.sep(j);
            BTA_TRY(chol_inv64(s, LD + sj * bb, b, X + sj * bb, b, b, (long long)sj * b, c->status, st->W, c->leaf,
                               &c->exec, 1, 0, 0, 0, m, c->batch, c->fork));
            const bool more = j < L.P - 1;
            const int sn = more ? L.sep(j + 1) : -1;
            if (more) {
                BTA_TRY(copy_mat64(s, LB + sj * bb, b, st->Wg, b, b, b, 0));
                G g1(b, b, b);
                g1.A(st->Wg, b).B(X + sj * bb, b, 1, 2).C(LB + sj * bb, b);
                BTA_TRY(gemm_exec(&c->exec, s, g1.g));
                G g2(b, b, b);
                g2.A(LB + sj * bb, b).B(LB + sj * bb, b, 1).lower();
                acc(g2, LD + sn * bb, b, 0);
                BTA_TRY(gemm_exec(&c->exec, s, g2.g));
            }
            if (a > 0) {
                BTA_TRY(copy_mat64(s, LR + sj * ab, a, st->Wg, a, a, b, 0));
                G g3(a, b, b);
                g3.A(st->Wg, a).B(X + sj * bb, b, 1, 2).C(LR + sj * ab, a);
                BTA_TRY(gemm64(s, g3.g));
                G g4(a, a, b);
                g4.A(LR + sj * ab, a).B(LR + sj * ab, a, 1).lower();
                acc(g4, LT, a, 0);
                BTA_TRY(gemm64(s, g4.g));
                if (more) {
                    G g5(a, b, b);
                    g5.A(LR + sj * ab, a).B(LB + sj * bb, b, 1);
                    acc(g5, LR + sn * ab, a, 0);
                    BTA_TRY(gemm64(s, g5.g));
                }
            }
        }
        if (a > 0)
            BTA_TRY(chol_inv64(s, LT, a, X + (long long)L.n * bb, a, a, (long long)L.n * b, c->status, st->W, c->leaf,
                               nullptr, 1, 0, 0, 0, m, c->batch));
        c->factored[m] = 1;
    }
    return BTA_OK;
}

// ---------------------------------------------------------------------------- solve

// x_j = Q_{m0+j}^{-1} r_j with the partitioned factors (vectors N apart):
// forward over the interiors (all partitions together), the separators and
// the tip, then backward in the reverse order.
int psolve_impl(bta_ctx_t c, int m0, int cnt, const double* r, double* x, cudaStream_t s) {
    const PLay L = layout(c);
    const int b = L.b, a = L.a;
    const long long bb = L.bb, N = c->N, nb = (long long)L.n * b;
    const long long sP = (long long)L.h * bb, sPv = (long long)L.h * b;
    const BtaStore& Lf = c->L;
    for (int j = 0; j < cnt; ++j) {
        const int m = m0 + j;
        const double* LB = Lf.B + m * Lf.sB;
        const double* LR = Lf.R + m * Lf.sR;
        const double* X = c->Linv + m * c->sLinv;
        const double* F = c->pts->F + (long long)m * L.n * bb;
        double* z = vec_row(c, VEC_Z, m);
        double* tmp = vec_row(c, VEC_TMP, m);
        const double* rj = r + j * N;
        double* xj = x + j * N;
        BTA_CUDA_TRY(cudaMemcpyAsync(tmp, rj, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        auto fwd = [&](int k, int p0, int pc) -> int {
            const StepRanges R = ranges(L, k, p0, pc);
            const int i0 = p0 * L.h + k;
            // z_i = X_i tmp_i ; tmp_{i+1} -= L_{i+1,i} z_i ; tmp_{sigma_p} -= L_{sigma_p,i} z_i
            BTA_TRY(gemv64(s, b, b, X + i0 * bb, b, 0, 1, tmp + (long long)i0 * b, 1.0, nullptr, 0.0,
                           z + (long long)i0 * b, pc, sP, sPv, sPv));
            if (R.pnext > 0)
                BTA_TRY(gemv64(s, b, b, LB + i0 * bb, b, 0, 0, z + (long long)i0 * b, -1.0,
                               tmp + (long long)(i0 + 1) * b, 1.0, tmp + (long long)(i0 + 1) * b, R.pnext, sP, sPv,
                               sPv));
            if (R.qc > 0) {
                const int iq = R.q0 * L.h + k;
                BTA_TRY(gemv64(s, b, b, F + iq * bb, b, 0, 0, z + (long long)iq * b, -1.0,
                               tmp + (long long)L.sep(R.q0) * b, 1.0, tmp + (long long)L.sep(R.q0) * b, R.qc, sP, sPv,
                               sPv));
            }
            return BTA_OK;
        };
        for (int k = 0; k < L.l; ++k) BTA_TRY(fwd(k, 0, L.P));
        for (int k = L.l; k < L.l_last; ++k) BTA_TRY(fwd(k, L.P - 1, 1));
        for (int jj = 1; jj < L.P; ++jj) {
            const int sj = L.sep(jj);
            BTA_TRY(gemv64(s, b, b, X + sj * bb, b, 0, 1, tmp + (long long)sj * b, 1.0, nullptr, 0.0,
                           z + (long long)sj * b));
            if (jj < L.P - 1) {
                const int sn = L.sep(jj + 1);
                BTA_TRY(gemv64(s, b, b, LB + sj * bb, b, 0, 0, z + (long long)sj * b, -1.0, tmp + (long long)sn * b,
                               1.0, tmp + (long long)sn * b));
            }
        }
        // tip: z_t = X_t (r_t - sum_i L_{t,i} z_i), x_t = X_t^T z_t, then z_i -= L_{t,i}^T x_t for every block
        if (a > 0) {
            BTA_TRY(gemv64(s, a, (int)nb, LR, a, 0, 0, z, -1.0, rj + nb, 1.0, tmp + nb));
            BTA_TRY(gemv64(s, a, a, X + L.n * bb, a, 0, 1, tmp + nb, 1.0, nullptr, 0.0, z + nb));
            BTA_TRY(gemv64(s, a, a, X + L.n * bb, a, 1, 2, z + nb, 1.0, nullptr, 0.0, xj + nb));
            BTA_TRY(gemv64(s, (int)nb, a, LR, a, 1, 0, xj + nb, -1.0, z, 1.0, z));
        }
        // backward, separators: x_s = X_s^T (z_s - L_{s+,s}^T x_{s+})
        for (int jj = L.P - 1; jj >= 1; --jj) {
            const int sj = L.sep(jj);
            const double* zs = z + (long long)sj * b;
            if (jj < L.P - 1) {
                const int sn = L.sep(jj + 1);
                BTA_TRY(gemv64(s, b, b, LB + sj * bb, b, 1, 0, xj + (long long)sn * b, -1.0, zs, 1.0,
                               tmp + (long long)sj * b));
                zs = tmp + (long long)sj * b;
            }
            BTA_TRY(gemv64(s, b, b, X + sj * bb, b, 1, 2, zs, 1.0, nullptr, 0.0, xj + (long long)sj * b));
        }
        // backward, interiors: x_i = X_i^T (z_i - L_{i+1,i}^T x_{i+1} - L_{sigma_p,i}^T x_{sigma_p})
        auto bwd = [&](int k, int p0, int pc) -> int {
            const StepRanges R = ranges(L, k, p0, pc);
            const int i0 = p0 * L.h + k;
            BTA_CUDA_TRY(cudaMemcpy2DAsync(tmp + (long long)i0 * b, sPv * sizeof(double), z + (long long)i0 * b,
                                           sPv * sizeof(double), b * sizeof(double), pc, cudaMemcpyDeviceToDevice, s));
            if (R.pnext > 0)
                BTA_TRY(gemv64(s, b, b, LB + i0 * bb, b, 1, 0, xj + (long long)(i0 + 1) * b, -1.0,
                               tmp + (long long)i0 * b, 1.0, tmp + (long long)i0 * b, R.pnext, sP, sPv, sPv));
            if (R.qc > 0) {
                const int iq = R.q0 * L.h + k;
                BTA_TRY(gemv64(s, b, b, F + iq * bb, b, 1, 0, xj + (long long)L.sep(R.q0) * b, -1.0,
                               tmp + (long long)iq * b, 1.0, tmp + (long long)iq * b, R.qc, sP, sPv, sPv));
            }
            BTA_TRY(gemv64(s, b, b, X + i0 * bb, b, 1, 2, tmp + (long long)i0 * b, 1.0, nullptr, 0.0,
                           xj + (long long)i0 * b, pc, sP, sPv, sPv));
            return BTA_OK;
        };
        for (int k = L.l_last - 1; k >= L.l; --k) BTA_TRY(bwd(k, L.P - 1, 1));
        for (int k = L.l - 1; k >= 0; --k) BTA_TRY(bwd(k, 0, L.P));
    }
    return BTA_OK;
}

// ---------------------------------------------------------------------------- selected inversion

int pselinv_impl(bta_ctx_t c, int m0, int cnt, cudaStream_t s) {
    const PLay L = layout(c);
    const int b = L.b, a = L.a;
    const long long bb = L.bb, ab = L.ab, sP = (long long)L.h * bb, sPR = (long long)L.h * ab;
    const BtaStore &Lf = c->L, &S = c->S;
    const GemmExec* ex = &c->exec;
    PTimeStore* st = c->pts;
    // per-partition scratch of a step, indexed by partition - p0: G (in U),
    // H (in the recursion scratch, sW apart), Fa (in Racc)
    double* Gs = st->U;
    double* Hs = st->W;
    const long long sH = st->sW;
    double* Fa = st->Racc;
    for (int m = m0; m < m0 + cnt; ++m) {
        const double* LB = Lf.B + m * Lf.sB;
        const double* LR = Lf.R + m * Lf.sR;
        const double* X = c->Linv + m * c->sLinv;
        const double* XT = X + (long long)L.n * bb;
        const double* F = st->F + (long long)m * L.n * bb;
        double* SF = st->SF + (long long)m * L.n * bb;
        double* SD = S.D + m * S.sD;
        double* SB = S.B + m * S.sB;
        double* SR = S.R + m * S.sR;
        double* ST = S.T + m * S.sT;
        if (a > 0) {
            G g(a, a, a);
            g.A(XT, a, 1, 2).B(XT, a, 0, 1).C(ST, a);
            BTA_TRY(gemm64(s, g.g));
        }
        // ---- reduced system, separators P-1 .. 1
        for (int j = L.P - 1; j >= 1; --j) {
            const int sj = L.sep(j);
            const bool more = j < L.P - 1;
            const int sn = more ? L.sep(j + 1) : -1;
            double* RSj = st->RS + (long long)j * bb;           // Sigma_{sigma_{j+1}, sigma_j}
            if (a > 0) {
                G g(a, b, b);
                g.A(LR + sj * ab, a).B(X + sj * bb, b, 0, 1).C(Fa, a);
                BTA_TRY(gemm64(s, g.g));
            }
            if (more) {
                G g(b, b, b);
                g.A(LB + sj * bb, b).B(X + sj * bb, b, 0, 1).C(Gs, b);
                BTA_TRY(gemm_exec(ex, s, g.g));
                G g1(b, b, b);
                g1.A(SD + sn * bb, b).B(Gs, b).C(RSj, b).alpha(-1.0);
                BTA_TRY(gemm_exec(ex, s, g1.g));
                if (a > 0) {
                    G g2(b, b, a);
                    g2.A(SR + sn * ab, a, 1).B(Fa, a);
                    acc(g2, RSj, b, 0);
                    BTA_TRY(gemm_exec(ex, s, g2.g));
                }
            }
            if (a > 0) {
                G g3(a, b, a);
                g3.A(ST, a).B(Fa, a).C(SR + sj * ab, a).alpha(-1.0);
                BTA_TRY(gemm64(s, g3.g));
                if (more) {
                    G g4(a, b, b);
                    g4.A(SR + sn * ab, a).B(Gs, b);
                    acc(g4, SR + sj * ab, a, 0);
                    BTA_TRY(gemm64(s, g4.g));
                }
            }
            G g5(b, b, b);
            g5.A(X + sj * bb, b, 1, 2).B(X + sj * bb, b, 0, 1).C(SD + sj * bb, b).lower();
            BTA_TRY(gemm_exec(ex, s, g5.g));
            if (more) {
                G g6(b, b, b);
                g6.A(Gs, b, 1).B(RSj, b).lower();
                acc(g6, SD + sj * bb, b, 0);
                BTA_TRY(gemm_exec(ex, s, g6.g));
            }
            if (a > 0) {
                G g7(b, b, a);
                g7.A(Fa, a, 1).B(SR + sj * ab, a).lower();
                acc(g7, SD + sj * bb, b, 0);
                BTA_TRY(gemm_exec(ex, s, g7.g));
            }
            BTA_TRY(symmetrize_lower64(s, SD + sj * bb, b, b));
        }
        // ---- interiors, backwards, all partitions together
        auto step = [&](int k, int p0, int pc) -> int {
            const StepRanges R = ranges(L, k, p0, pc);
            const int i0 = p0 * L.h + k;
            auto blk = [&](int p) { return p * L.h + k; };
            const int iq = blk(R.q0);
            // G = L_{i+1,i} X_i, H = L_{sigma_p,i} X_i, Fa = L_{t,i} X_i
            if (R.pnext > 0) {
                G g(b, b, b);
                g.A(LB + i0 * bb, b, 0, 0, sP).B(X + i0 * bb, b, 0, 1, sP).C(Gs, b, bb).batch(R.pnext);
                BTA_TRY(gemm_exec(ex, s, g.g));
            }
            if (R.qc > 0) {
                G g(b, b, b);
                g.A(F + iq * bb, b, 0, 0, sP).B(X + iq * bb, b, 0, 1, sP).C(Hs + (R.q0 - p0) * sH, b, sH)
                    .batch(R.qc);
                BTA_TRY(gemm_exec(ex, s, g.g));
            }
            if (a > 0) {
                G g(a, b, b);
                g.A(LR + i0 * ab, a, 0, 0, sPR).B(X + i0 * bb, b, 0, 1, sP).C(Fa, a, ab).batch(pc);
                BTA_TRY(gemm64(s, g.g));
            }
            // Sigma_{i+1,i} = -(Sigma_{i+1,i+1} G + Sigma_{i+1,sigma_p} H + Sigma_{t,i+1}^T Fa)
            if (R.pnext > 0) {
                G g(b, b, b);
                g.A(SD + (i0 + 1) * bb, b, 0, 0, sP).B(Gs, b, 0, 0, bb).C(SB + i0 * bb, b, sP).alpha(-1.0)
                    .batch(R.pnext);
                BTA_TRY(gemm_exec(ex, s, g.g));
                if (R.nic > 0) {
                    // Sigma_{i+1,sigma_p} = Sigma_{sigma_p,i+1}^T
                    const int in = blk(R.ni0);
                    G g2(b, b, b);
                    g2.A(SF + (in + 1) * bb, b, 1, 0, sP).B(Hs + (R.ni0 - p0) * sH, b, 0, 0, sH).batch(R.nic);
                    acc(g2, SB + in * bb, b, sP);
                    BTA_TRY(gemm_exec(ex, s, g2.g));
                }
                if (R.nsc > 0) {
                    // Sigma_{sigma_{p+1},sigma_p} of the reduced system
                    const int is = blk(R.ns0);
                    G g2(b, b, b);
                    g2.A(st->RS + (long long)R.ns0 * bb, b, 0, 0, bb).B(Hs + (R.ns0 - p0) * sH, b, 0, 0, sH)
                        .batch(R.nsc);
                    acc(g2, SB + is * bb, b, sP);
                    BTA_TRY(gemm_exec(ex, s, g2.g));
                }
                if (a > 0) {
                    G g3(b, b, a);
                    g3.A(SR + (i0 + 1) * ab, a, 1, 0, sPR).B(Fa, a, 0, 0, ab).batch(R.pnext);
                    acc(g3, SB + i0 * bb, b, sP);
                    BTA_TRY(gemm_exec(ex, s, g3.g));
                }
            }
            // Sigma_{sigma_p,i} = -(Sigma_{sigma_p,i+1} G + Sigma_{sigma_p,sigma_p} H + Sigma_{t,sigma_p}^T Fa)
            if (R.qc > 0) {
                G g(b, b, b);
                g.A(SD + L.sep(R.q0) * bb, b, 0, 0, sP).B(Hs + (R.q0 - p0) * sH, b, 0, 0, sH).C(SF + iq * bb, b, sP)
                    .alpha(-1.0).batch(R.qc);
                BTA_TRY(gemm_exec(ex, s, g.g));
                if (R.nic > 0) {
                    const int in = blk(R.ni0);
                    G g2(b, b, b);
                    g2.A(SF + (in + 1) * bb, b, 0, 0, sP).B(Gs + (R.ni0 - p0) * bb, b, 0, 0, bb).batch(R.nic);
                    acc(g2, SF + in * bb, b, sP);
                    BTA_TRY(gemm_exec(ex, s, g2.g));
                }
                if (R.nsc > 0) {
                    // Sigma_{sigma_p,sigma_{p+1}} = Sigma_{sigma_{p+1},sigma_p}^T
                    const int is = blk(R.ns0);
                    G g2(b, b, b);
                    g2.A(st->RS + (long long)R.ns0 * bb, b, 1, 0, bb).B(Gs + (R.ns0 - p0) * bb, b, 0, 0, bb)
                        .batch(R.nsc);
                    acc(g2, SF + is * bb, b, sP);
                    BTA_TRY(gemm_exec(ex, s, g2.g));
                }
                if (a > 0) {
                    G g3(b, b, a);
                    g3.A(SR + L.sep(R.q0) * ab, a, 1, 0, sPR).B(Fa + (R.q0 - p0) * ab, a, 0, 0, ab).batch(R.qc);
                    acc(g3, SF + iq * bb, b, sP);
                    BTA_TRY(gemm_exec(ex, s, g3.g));
                }
            }
            // Sigma_{t,i} = -(Sigma_{t,i+1} G + Sigma_{t,sigma_p} H + Sigma_tt Fa)
            if (a > 0) {
                G g(a, b, a);
                g.A(ST, a).B(Fa, a, 0, 0, ab).C(SR + i0 * ab, a, sPR).alpha(-1.0).batch(pc);
                BTA_TRY(gemm64(s, g.g));
                if (R.pnext > 0) {
                    G g2(a, b, b);
                    g2.A(SR + (i0 + 1) * ab, a, 0, 0, sPR).B(Gs, b, 0, 0, bb).batch(R.pnext);
                    acc(g2, SR + i0 * ab, a, sPR);
                    BTA_TRY(gemm64(s, g2.g));
                }
                if (R.qc > 0) {
                    G g3(a, b, b);
                    g3.A(SR + L.sep(R.q0) * ab, a, 0, 0, sPR).B(Hs + (R.q0 - p0) * sH, b, 0, 0, sH).batch(R.qc);
                    acc(g3, SR + iq * ab, a, sPR);
                    BTA_TRY(gemm64(s, g3.g));
                }
            }
            // Sigma_ii = X^T X - G^T Sigma_{i+1,i} - H^T Sigma_{sigma_p,i} - Fa^T Sigma_{t,i}
            G g(b, b, b);
            g.A(X + i0 * bb, b, 1, 2, sP).B(X + i0 * bb, b, 0, 1, sP).C(SD + i0 * bb, b, sP).lower().batch(pc);
            BTA_TRY(gemm_exec(ex, s, g.g));
            if (R.pnext > 0) {
                G g2(b, b, b);
                g2.A(Gs, b, 1, 0, bb).B(SB + i0 * bb, b, 0, 0, sP).lower().batch(R.pnext);
                acc(g2, SD + i0 * bb, b, sP);
                BTA_TRY(gemm_exec(ex, s, g2.g));
            }
            if (R.qc > 0) {
                G g3(b, b, b);
                g3.A(Hs + (R.q0 - p0) * sH, b, 1, 0, sH).B(SF + iq * bb, b, 0, 0, sP).lower().batch(R.qc);
                acc(g3, SD + iq * bb, b, sP);
                BTA_TRY(gemm_exec(ex, s, g3.g));
            }
            if (a > 0) {
                G g4(b, b, a);
                g4.A(Fa, a, 1, 0, ab).B(SR + i0 * ab, a, 0, 0, sPR).lower().batch(pc);
                acc(g4, SD + i0 * bb, b, sP);
                BTA_TRY(gemm_exec(ex, s, g4.g));
            }
            BTA_TRY(symmetrize_lower64(s, SD + i0 * bb, b, b, pc, sP));
            return BTA_OK;
        };
        for (int k = L.l_last - 1; k >= L.l; --k) BTA_TRY(step(k, L.P - 1, 1));
        for (int k = L.l - 1; k >= 0; --k) BTA_TRY(step(k, 0, L.P));
        // BTA-pattern block (first_p, sigma_p) = Sigma_{sigma_p, first_p}^T
        transpose_copy_kernel<<<dim3((int)std::min<long long>((bb + 255) / 256, 1216), L.P - 1), 256, 0, s>>>(
            SF + (long long)L.first(1) * bb, SB + (long long)L.sep(1) * bb, b, sP, sP);
        BTA_LAUNCH_CHECK();
    }
    return BTA_OK;
}

extern "C" int bta_set_time_partitions(bta_ctx_t ctx, int P) {
    if (!ctx || P < 1) return BTA_ERR_ARG;
    if (P > 1 && (ctx->n + 1) / P < 2) return BTA_ERR_ARG;   // every interior needs one block
    if (P == ctx->tparts) return BTA_OK;
    BTA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (ctx->fobj_graph) {
        cudaGraphExecDestroy(ctx->fobj_graph);
        ctx->fobj_graph = nullptr;
        ctx->graph_calls = 1;
    }
    std::fill(ctx->factored.begin(), ctx->factored.end(), 0);
    if (P == 1) {
        ptime_free(ctx);
        ctx->tparts = 1;
        return BTA_OK;
    }
    int rc = ptime_alloc(ctx, P);
    if (rc == BTA_OK && ctx->precision != BTA_FP64 && P > ctx->nmat) {
        // the batched products of P partitions need P digit workspaces
        const size_t wsb = (size_t)P * ozaki_workspace_bytes(ctx->b, ctx->b, ctx->b, ctx->exec.slices);
        if (wsb > ctx->exec.ws_bytes) {
            for (GemmExec* e : {&ctx->exec, &ctx->fork->ex2}) {
                if (e->ws) cudaFree(e->ws);
                e->ws = nullptr;
                if (cudaMalloc(&e->ws, wsb) != cudaSuccess) {
                    e->ws = nullptr;
                    rc = BTA_ERR_OOM;
                }
                e->ws_bytes = wsb;
            }
        }
    }
    if (rc != BTA_OK) {
        ptime_free(ctx);
        ctx->tparts = 1;
        return rc;
    }
    ctx->tparts = P;
    return BTA_OK;
}
