// Autotuning of the launch shapes of the BTA factorisation and selected
// inversion for a context's block order, precision and batch.  Every
// candidate is timed on the context's own storage and the fastest is kept:
//   1. the diagonal-block chain, the latency-bound critical path of the block
//      Cholesky (one batched Cholesky + inverse of a b x b block per step):
//        FP64:  the leaf order of the recursive Cholesky + inverse (16, 32, 64)
//        mixed: the double-float leaf order (32, 64, 128) x the smallest
//               product dimension sent to the tensor cores (128, 256, 384, 512)
//   2. the b x b x b products (Schur updates, selected inversion), timed on
//      the lower-output update D -= L L^T of every matrix:
//        FP64:  the CTAs per SM the DFMA GEMM aims for through its K split
//               (1, 2, 4), which sets its micro-tile and split
//        mixed: the tile configuration of the split product (for 35-bit
//               digits 128 x 96 with 2 TMA stages or 128 x 64 with 3; for
//               49-bit digits 128 x 64 with 2) x the waves of the persistent
//               grid below which it splits K (1, 2)
//   3. mixed only: the tile order of the split product (row tiles per band:
//      1, 4, 8, 16), separately for products with a triangular operand (timed
//      on B X^T with X = L^{-1} lower, as in L_{i+1,i} = B_i X_i^T), for
//      general ones (timed on a dense product, as in Sigma_{i+1,i+1} G_i) and
//      for lower-triangle outputs (timed on the update of stage 2)
// The timed matrices are synthetic SPD blocks written into the first
// diagonal blocks of every matrix of the context (their contents are lost).

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

// A_ij = 2 delta_ij + 1 / ((1 + |i - j|) n): diagonally dominant, SPD.
__global__ void fill_spd_kernel(double* A, int n, long long lda, long long sA) {
    A += blockIdx.y * sA;
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        A[i + (long long)j * lda] = (i == j ? 2.0 : 0.0) + 1.0 / ((1.0 + abs(i - j)) * n);
}

}  // namespace

extern "C" int bta_autotune(bta_ctx_t ctx, int reps, int* chosen) {
    if (!ctx || !chosen || reps < 1) return BTA_ERR_ARG;
    const int b = ctx->b, nm = ctx->nmat;
    cudaStream_t s = ctx->stream;
    // the storage is about to be overwritten: nothing stays factored, and a
    // captured f_obj graph would carry the old launch shapes
    if (ctx->fobj_graph) {
        cudaStreamSynchronize(s);
        cudaGraphExecDestroy(ctx->fobj_graph);
        ctx->fobj_graph = nullptr;
        ctx->graph_calls = 1;
    }
    std::fill(ctx->factored.begin(), ctx->factored.end(), 0);
    fill_spd_kernel<<<dim3(b, nm), 256, 0, s>>>(ctx->Q.D, b, b, ctx->Q.sD);
    BTA_LAUNCH_CHECK();

    struct Cand {
        int leaf, df_leaf, min_dim;
    };
    std::vector<Cand> cands;
    if (ctx->precision != BTA_FP64) {
        for (int dl : {32, 64, 128})
            for (int md : {128, 256, 384, 512}) cands.push_back({ctx->leaf, dl, md});
    } else {
        for (int lf : {16, 32, 64}) cands.push_back({lf, ctx->exec.df_leaf, ctx->exec.min_dim});
    }
    cudaEvent_t e0, e1;
    BTA_CUDA_TRY(cudaEventCreate(&e0));
    BTA_CUDA_TRY(cudaEventCreate(&e1));
    auto run = [&](const Cand& c) -> int {
        ctx->leaf = c.leaf;
        ctx->exec.df_leaf = c.df_leaf;
        ctx->exec.min_dim = c.min_dim;
        if (ctx->fork) {
            ctx->fork->ex2.df_leaf = c.df_leaf;
            ctx->fork->ex2.min_dim = c.min_dim;
        }
        BTA_TRY(copy_mat64(s, ctx->Q.D, b, ctx->L.D, b, b, b, 1, nm, ctx->Q.sD, ctx->L.sD));
        // the low-memory layout keeps X apart from L only in its X buffer
        double* X = ctx->lowmem ? ctx->xtmp : ctx->Linv;
        const long long sX = ctx->lowmem ? (long long)b * b : ctx->sLinv;
        return chol_inv64(s, ctx->L.D, b, X, b, b, 0, ctx->status, ctx->work, c.leaf, &ctx->exec, nm,
                          ctx->L.sD, sX, ctx->sWork, 0, ctx->batch, ctx->fork);
    };
    float best = -1.f;
    Cand pick = cands[0];
    int rc = BTA_OK;
    for (const Cand& c : cands) {
        if ((rc = run(c)) != BTA_OK) break;   // warm-up (first use of each launch shape)
        if (cudaEventRecord(e0, s) != cudaSuccess) { rc = BTA_ERR_CUDA; break; }
        for (int r = 0; r < reps && rc == BTA_OK; ++r) rc = run(c);
        if (rc != BTA_OK) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = BTA_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0.f || ms < best) {
            best = ms;
            pick = c;
        }
    }
    ctx->leaf = pick.leaf;
    ctx->exec.df_leaf = pick.df_leaf;
    ctx->exec.min_dim = pick.min_dim;
    if (ctx->fork) {
        ctx->fork->ex2.df_leaf = pick.df_leaf;
        ctx->fork->ex2.min_dim = pick.min_dim;
    }

    // ---- 2. the b x b x b products: D_0 -= X X^T (lower) on every matrix, with
    // X the synthetic block of Q and D_0 of L as the output
    struct PCand {
        int tile, occ, ctas;
    };
    std::vector<PCand> pc;
    if (ctx->precision != BTA_FP64) {
        int tiles[4];
        const int nt = ozaki_tiles_for(ctx->exec.slices, tiles, 4);
        for (int t = 0; t < nt; ++t)
            for (int occ : {1, 2}) pc.push_back({tiles[t], occ, ctx->exec.fp64_ctas});
    } else {
        for (int c : {1, 2, 4}) pc.push_back({ctx->exec.tile, ctx->exec.occupancy, c});
    }
    Gemm64 g{};
    g.M = b; g.N = b; g.K = b;
    g.A = ctx->Q.D; g.lda = b;
    g.B = ctx->Q.D; g.ldb = b; g.tb = 1;
    g.Cin = ctx->L.D; g.ldci = b; g.beta = 1.0;
    g.C = ctx->L.D; g.ldc = b; g.alpha = -1.0; g.lowerC = 1;
    g.batch = nm; g.sA = ctx->Q.sD; g.sB = ctx->Q.sD; g.sCi = ctx->L.sD; g.sC = ctx->L.sD;
    auto prun = [&](const PCand& c) -> int {
        ctx->exec.tile = c.tile;
        ctx->exec.occupancy = c.occ;
        ctx->exec.fp64_ctas = c.ctas;
        return gemm_exec(&ctx->exec, s, g);
    };
    float pbest = -1.f;
    PCand ppick = pc[0];
    for (const PCand& c : pc) {
        if (rc != BTA_OK) break;
        if ((rc = prun(c)) != BTA_OK) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) { rc = BTA_ERR_CUDA; break; }
        for (int r = 0; r < reps && rc == BTA_OK; ++r) rc = prun(c);
        if (rc != BTA_OK) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = BTA_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (pbest < 0.f || ms < pbest) {
            pbest = ms;
            ppick = c;
        }
    }
    ctx->exec.tile = ppick.tile;
    ctx->exec.occupancy = ppick.occ;
    ctx->exec.fp64_ctas = ppick.ctas;
    if (ctx->fork) {
        ctx->fork->ex2.tile = ppick.tile;
        ctx->fork->ex2.occupancy = ppick.occ;
        ctx->fork->ex2.fp64_ctas = ppick.ctas;
    }

    // ---- 3. tile order of the split products (mixed precision only)
    if (rc == BTA_OK && ctx->precision != BTA_FP64) {
        for (int kind = 0; kind < 3 && rc == BTA_OK; ++kind) {
            const bool tri = kind == 0;
            Gemm64 h{};
            h.M = b; h.N = b; h.K = b;
            h.A = ctx->Q.D; h.lda = b; h.sA = ctx->Q.sD;
            if (tri) {
                // C = A X^T with X the lower inverse factor of the chain stage
                h.B = ctx->lowmem ? ctx->xtmp : ctx->Linv; h.ldb = b; h.tb = 1; h.shB = 2;
                h.sB = ctx->lowmem ? (long long)b * b : ctx->sLinv;
            } else {
                h.B = ctx->Q.D; h.ldb = b; h.sB = ctx->Q.sD;
            }
            h.C = ctx->L.D; h.ldc = b; h.sC = ctx->L.sD; h.alpha = 1.0;
            h.batch = nm;
            if (kind == 2) h = g;   // the lower-output update of stage 2
            int& slot = kind == 0 ? ctx->exec.band_tri : (kind == 1 ? ctx->exec.band_gen : ctx->exec.band_low);
            float bbest = -1.f;
            int bpick = slot;
            for (int band : {1, 4, 8, 16}) {
                slot = band;
                if ((rc = gemm_exec(&ctx->exec, s, h)) != BTA_OK) break;
                if (cudaEventRecord(e0, s) != cudaSuccess) { rc = BTA_ERR_CUDA; break; }
                for (int r = 0; r < reps && rc == BTA_OK; ++r) rc = gemm_exec(&ctx->exec, s, h);
                if (rc != BTA_OK) break;
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = BTA_ERR_CUDA;
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (bbest < 0.f || ms < bbest) {
                    bbest = ms;
                    bpick = band;
                }
            }
            slot = bpick;
        }
        if (ctx->fork) {
            ctx->fork->ex2.band_tri = ctx->exec.band_tri;
            ctx->fork->ex2.band_gen = ctx->exec.band_gen;
            ctx->fork->ex2.band_low = ctx->exec.band_low;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != BTA_OK) return rc;
    BTA_TRY(bta_sync(ctx));
    chosen[0] = pick.leaf;
    chosen[1] = pick.df_leaf;
    chosen[2] = pick.min_dim;
    chosen[3] = ppick.tile;
    chosen[4] = ppick.occ;
    chosen[5] = ppick.ctas;
    chosen[6] = ctx->exec.band_tri;
    chosen[7] = ctx->exec.band_gen;
    chosen[8] = ctx->exec.band_low;
    return BTA_OK;
}
