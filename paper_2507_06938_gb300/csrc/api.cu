// Context life cycle, storage accessors, status and error reporting of the
// C ABI declared in include/bta.h.

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

static thread_local cudaError_t g_last_cuda = cudaSuccess;
static std::atomic<long long> g_launches{0};

void bta_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void bta_note_launches(long long delta) { g_launches.fetch_add(delta, std::memory_order_relaxed); }

extern "C" long long bta_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int bta_cuda_fail(cudaError_t e) {
    g_last_cuda = e;
    if (e == cudaErrorMemoryAllocation) return BTA_ERR_OOM;
    return BTA_ERR_CUDA;
}

namespace {
struct SmemAttr { const void* fn; int dev; int bytes; };
std::mutex g_attr_mutex;
std::vector<SmemAttr> g_attr;
}  // namespace

int ensure_dyn_smem(const void* fn, int bytes) {
    if (bytes <= 48 * 1024) return BTA_OK;
    int dev = 0;
    BTA_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    for (SmemAttr& e : g_attr) {
        if (e.fn != fn || e.dev != dev) continue;
        if (e.bytes >= bytes) return BTA_OK;
        BTA_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        e.bytes = bytes;
        return BTA_OK;
    }
    BTA_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    g_attr.push_back(SmemAttr{fn, dev, bytes});
    return BTA_OK;
}

namespace {

int dalloc(double** p, size_t elems) {
    *p = nullptr;
    if (elems == 0) elems = 1;
    cudaError_t e = cudaMalloc((void**)p, elems * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? BTA_ERR_OOM : bta_cuda_fail(e);
    }
    return BTA_OK;
}

void store_free(BtaStore& M) {
    if (M.D) cudaFree(M.D - M.oD);
    if (M.B) cudaFree(M.B - M.oB);
    if (M.R) cudaFree(M.R - M.oR);
    if (M.T) cudaFree(M.T);
    M = BtaStore{};
}

}  // namespace

// `blk` block slots per matrix (blk == n: the compact layout, n - 1 slots for
// B) and `lead` leading padding slots before matrix 0; everything zeroed.
int store_alloc(BtaStore& M, int nmat, int n, int b, int a, int blk, int lead) {
    const long long bb = (long long)b * b, ab = (long long)a * b;
    const bool compact = blk == n && lead == 0;
    M.sD = blk * bb;
    M.sB = (compact ? (n > 1 ? n - 1 : 0) : blk) * bb;
    M.sR = (long long)blk * ab;
    M.sT = (long long)a * a;
    M.oD = lead * bb;
    M.oB = lead * bb;
    M.oR = lead * ab;
    double* p = nullptr;
    BTA_TRY(dalloc(&p, (size_t)(M.oD + nmat * M.sD)));
    M.D = p + M.oD;
    BTA_TRY(dalloc(&p, (size_t)(M.oB + nmat * M.sB)));
    M.B = p + M.oB;
    BTA_TRY(dalloc(&p, (size_t)(M.oR + nmat * M.sR)));
    M.R = p + M.oR;
    BTA_TRY(dalloc(&p, (size_t)nmat * M.sT));
    M.T = p;
    BTA_CUDA_TRY(cudaMemset(M.D - M.oD, 0, (size_t)(M.oD + nmat * M.sD) * sizeof(double)));
    BTA_CUDA_TRY(cudaMemset(M.B - M.oB, 0, (size_t)std::max<long long>(1, M.oB + nmat * M.sB) * sizeof(double)));
    BTA_CUDA_TRY(cudaMemset(M.R - M.oR, 0, (size_t)std::max<long long>(1, M.oR + nmat * M.sR) * sizeof(double)));
    BTA_CUDA_TRY(cudaMemset(M.T, 0, (size_t)std::max<long long>(1, nmat * M.sT) * sizeof(double)));
    return BTA_OK;
}

void store_release(BtaStore& M) { store_free(M); }

int ensure_sigma(bta_ctx_t ctx) {
    if (ctx->lowmem) {
        ctx->S = ctx->L;   // the selected inverse overwrites the factor
        return BTA_OK;
    }
    if (ctx->S.D) return BTA_OK;
    int rc = store_alloc(ctx->S, ctx->nmat, ctx->n, ctx->b, ctx->a, ctx->blk, ctx->blk != ctx->n ? 1 : 0);
    if (rc != BTA_OK) store_free(ctx->S);
    return rc;
}

// The default factor storage: L blocks, and the inverse diagonal blocks apart.
static int alloc_default_factor(bta_ctx_t c) {
    const int n = c->n, b = c->b, a = c->a, nm = c->nmat;
    const long long bb = (long long)b * b;
    BTA_TRY(store_alloc(c->L, nm, n, b, a, n, 0));
    c->sLinv = n * bb + (long long)a * a;
    c->tip_off = n * bb;
    BTA_TRY(dalloc(&c->Linv, (size_t)nm * c->sLinv));
    // the strict upper triangles of the inverse blocks are never written by the factor
    BTA_CUDA_TRY(cudaMemset(c->Linv, 0, (size_t)nm * c->sLinv * sizeof(double)));
    return BTA_OK;
}

// The low-memory factor storage: a spare diagonal slot per matrix for
// L_tt^{-1}, the inverse blocks in the diagonal slots, one X buffer per matrix.
static int alloc_low_factor(bta_ctx_t c) {
    const int n = c->n, b = c->b, a = c->a, nm = c->nmat;
    const long long bb = (long long)b * b;
    BTA_TRY(store_alloc(c->L, nm, n, b, a, n + 1, 0));
    BTA_TRY(dalloc(&c->xtmp, (size_t)nm * bb));
    BTA_TRY(dalloc(&c->ldacc, (size_t)nm));
    BTA_CUDA_TRY(cudaMemset(c->xtmp, 0, (size_t)nm * bb * sizeof(double)));
    c->Linv = c->L.D;
    c->sLinv = c->L.sD;
    c->tip_off = n * bb;
    c->lowmem = 1;
    return BTA_OK;
}

extern "C" int bta_create_ex(int n, int b, int a, int precision, int batch, int flags, void* stream,
                             bta_ctx_t* out) {
    if (!out || n < 1 || b < 1 || a < 0 || batch < 1 || (flags & ~BTA_CREATE_LOW_MEMORY) != 0 ||
        (precision != BTA_FP64 && precision != BTA_MIXED && precision != BTA_MIXED_HI))
        return BTA_ERR_ARG;
    const bool mixed = precision != BTA_FP64;
    *out = nullptr;
    bta_ctx_s* c = new bta_ctx_s();
    c->n = n; c->b = b; c->a = a; c->precision = precision;
    c->batch = batch; c->nmat = 2 * batch;
    c->N = (long long)n * b + a;
    c->stream = (cudaStream_t)stream;
    c->leaf = 32;
    if (const char* e = std::getenv("BTA_LEAF")) c->leaf = std::atoi(e);
    c->status = nullptr; c->params = nullptr;
    c->aux = nullptr; c->ev_fork = nullptr; c->ev_join = nullptr;
    c->exec = GemmExec{};
    c->factored.assign(c->nmat, 0);
    c->mu_valid.assign(c->batch, 0);
    int rc = BTA_OK;
    auto fail = [&](int r) { bta_destroy(c); return r; };
    if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess) return fail(BTA_ERR_CUDA);
    if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) return fail(BTA_ERR_CUDA);
    if (cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) return fail(BTA_ERR_CUDA);
    const long long bb = (long long)b * b;
    const int nm = c->nmat;
    c->blk = n;
    c->tip_off = (long long)n * bb;
    if ((rc = store_alloc(c->Q, nm, n, b, a, n, 0)) != BTA_OK) return fail(rc);
    rc = (flags & BTA_CREATE_LOW_MEMORY) ? alloc_low_factor(c) : alloc_default_factor(c);
    if (rc != BTA_OK) return fail(rc);
    c->sWork = bb + bb / 2 + 2LL * b + 2LL * a * b + (long long)a * a + 64;
    if ((rc = dalloc(&c->work, (size_t)nm * c->sWork)) != BTA_OK) return fail(rc);
    if ((rc = dalloc(&c->vec, (size_t)VEC_ROWS * nm * c->N)) != BTA_OK) return fail(rc);
    c->red_chunks = 256;
    if ((rc = dalloc(&c->red, (size_t)nm * c->red_chunks)) != BTA_OK) return fail(rc);
    if ((rc = dalloc(&c->ld, nm)) != BTA_OK) return fail(rc);
    if ((rc = dalloc(&c->dots, 3 * (size_t)nm)) != BTA_OK) return fail(rc);
    if ((rc = dalloc(&c->params, (size_t)batch * BTA_PSTRIDE)) != BTA_OK) return fail(rc);
    if ((rc = dalloc(&c->theta_buf, (size_t)batch * BTA_PSTRIDE)) != BTA_OK) return fail(rc);
    if ((rc = dalloc(&c->f_buf, (size_t)batch)) != BTA_OK) return fail(rc);
    if (const char* e = std::getenv("BTA_GRAPH")) c->use_graph = std::atoi(e);
    if (cudaMemset(c->params, 0, (size_t)batch * BTA_PSTRIDE * sizeof(double)) != cudaSuccess)
        return fail(BTA_ERR_CUDA);
    if (cudaMalloc((void**)&c->status, 4 * sizeof(long long)) != cudaSuccess) return fail(BTA_ERR_OOM);
    if (cudaMemset(c->status, 0, 4 * sizeof(long long)) != cudaSuccess) return fail(BTA_ERR_CUDA);
    c->refine = 0;
    if (mixed) {
        if (cudaMalloc((void**)&c->oz_err, sizeof(int)) != cudaSuccess) return fail(BTA_ERR_OOM);
        if (cudaMemset(c->oz_err, 0, sizeof(int)) != cudaSuccess) return fail(BTA_ERR_CUDA);
        int min_dim = 128;
        if (const char* e = std::getenv("BTA_OZ_MIN")) min_dim = std::atoi(e);
        c->exec.df_leaf = 64;
        if (const char* e = std::getenv("BTA_DF_LEAF")) c->exec.df_leaf = std::atoi(e);
        c->exec.slices = precision == BTA_MIXED_HI ? 7 : 5;
        if (const char* e = std::getenv("BTA_OZ_TILE")) c->exec.tile = std::atoi(e) == 1 && c->exec.slices == 5 ? 1 : 0;
        if (const char* e = std::getenv("BTA_OZ_BAND")) {
            // test and profiling hook: one band for all products, or "tri,gen,low"
            int v[3] = {0, 0, 0};
            const int k = std::sscanf(e, "%d,%d,%d", &v[0], &v[1], &v[2]);
            if (k == 1) v[1] = v[2] = v[0];
            if (k == 1 || k == 3) {
                c->exec.band_tri = std::max(1, v[0]);
                c->exec.band_gen = std::max(1, v[1]);
                c->exec.band_low = std::max(1, v[2]);
            }
        }
        const size_t wsb = (size_t)nm * ozaki_workspace_bytes(b, b, b, c->exec.slices);
        if (cudaMalloc(&c->exec.ws, wsb) != cudaSuccess) {
            c->exec.ws = nullptr;
            return fail(BTA_ERR_OOM);
        }
        c->exec.fn = gemm_mixed_fn;
        c->exec.ws_bytes = wsb;
        c->exec.err = c->oz_err;
        c->exec.min_dim = min_dim;
        c->refine = 2;
    }
    // side stream of the diagonal-block recursion (products off its critical
    // path), with a digit workspace of its own in mixed precision
    c->fork = new CholFork();
    if (cudaStreamCreateWithFlags(&c->fork->s2, cudaStreamNonBlocking) != cudaSuccess) return fail(BTA_ERR_CUDA);
    for (int k = 0; k < 2 * CHOL_FORK_DEPTH; ++k)
        if (cudaEventCreateWithFlags(&c->fork->ev[k], cudaEventDisableTiming) != cudaSuccess)
            return fail(BTA_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&c->fork->s3, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork->ev3_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork->ev3_join, cudaEventDisableTiming) != cudaSuccess)
        return fail(BTA_ERR_CUDA);
    c->fork->ex2 = c->exec;
    if (mixed) {
        c->fork->ex2.ws = nullptr;
        if (cudaMalloc(&c->fork->ex2.ws, c->exec.ws_bytes) != cudaSuccess) {
            c->fork->ex2.ws = nullptr;
            return fail(BTA_ERR_OOM);
        }
    }
    if (const char* e = std::getenv("BTA_REFINE")) c->refine = std::atoi(e);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(BTA_ERR_CUDA);
    *out = c;
    return BTA_OK;
}

extern "C" int bta_create_batched(int n, int b, int a, int precision, int batch, void* stream, bta_ctx_t* out) {
    return bta_create_ex(n, b, a, precision, batch, 0, stream, out);
}

extern "C" int bta_create(int n, int b, int a, int precision, void* stream, bta_ctx_t* out) {
    return bta_create_batched(n, b, a, precision, 1, stream, out);
}

extern "C" int bta_batch_size(bta_ctx_t c, int* batch) {
    if (!c || !batch) return BTA_ERR_ARG;
    *batch = c->batch;
    return BTA_OK;
}

extern "C" int bta_destroy(bta_ctx_t c) {
    if (!c) return BTA_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->aux) cudaStreamSynchronize(c->aux);
    if (c->fork) {
        if (c->fork->s2) cudaStreamSynchronize(c->fork->s2);
        for (int q = 0; q < 2 * CHOL_FORK_DEPTH; ++q)
            if (c->fork->ev[q]) cudaEventDestroy(c->fork->ev[q]);
        if (c->fork->s2) cudaStreamDestroy(c->fork->s2);
        if (c->fork->s3) {
            cudaStreamSynchronize(c->fork->s3);
            cudaStreamDestroy(c->fork->s3);
        }
        if (c->fork->ev3_fork) cudaEventDestroy(c->fork->ev3_fork);
        if (c->fork->ev3_join) cudaEventDestroy(c->fork->ev3_join);
        if (c->precision != BTA_FP64 && c->fork->ex2.ws) cudaFree(c->fork->ex2.ws);
        delete c->fork;
        c->fork = nullptr;
    }
    ptime_free(c);
    if (c->lowmem) {
        // S and Linv alias the factor's storage
        c->S = BtaStore{};
        c->Linv = nullptr;
    }
    for (double* p : {c->xtmp, c->ldacc})
        if (p) cudaFree(p);
    store_free(c->Q);
    store_free(c->L);
    store_free(c->S);
    if (c->fobj_graph) cudaGraphExecDestroy(c->fobj_graph);
    double* bufs[] = {c->Linv, c->work, c->vec, c->red, c->ld, c->dots, c->params, c->theta_buf, c->f_buf,
                      c->adj, c->hs_theta, c->hs_f, c->hs_grad, c->hs_var, c->lap};
    for (double* p : bufs)
        if (p) cudaFree(p);
    if (c->exec.ws) cudaFree(c->exec.ws);
    if (c->oz_err) cudaFree(c->oz_err);
    if (c->status) cudaFree(c->status);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->phase_ev)
        if (e) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->aux) cudaStreamDestroy(c->aux);
    delete c;
    return BTA_OK;
}

extern "C" int bta_block_ptr(bta_ctx_t c, int which, int store, int kind, int i, double** ptr_out, int* ld_out) {
    if (!c || !ptr_out) return BTA_ERR_ARG;
    const int m = storage_index(c, which);
    if (m < 0) return BTA_ERR_ARG;
    const long long bb = (long long)c->b * c->b, ab = (long long)c->a * c->b;
    if (store == BTA_STORE_LINV) {
        double* base = c->Linv + m * c->sLinv;
        if (kind == BTA_BLK_D && i >= 0 && i < c->n) {
            *ptr_out = base + i * bb;
            if (ld_out) *ld_out = c->b;
            return BTA_OK;
        }
        if (kind == BTA_BLK_T) {
            *ptr_out = base + c->tip_off;
            if (ld_out) *ld_out = c->a;
            return BTA_OK;
        }
        return BTA_ERR_ARG;
    }
    const BtaStore* M = nullptr;
    if (store == BTA_STORE_Q) M = &c->Q;
    else if (store == BTA_STORE_L) M = &c->L;
    else if (store == BTA_STORE_SIGMA) M = &c->S;
    else return BTA_ERR_ARG;
    if (!M->D) return BTA_ERR_STATE;
    switch (kind) {
        case BTA_BLK_D:
            if (i < 0 || i >= c->n) return BTA_ERR_ARG;
            *ptr_out = M->D + m * M->sD + i * bb;
            if (ld_out) *ld_out = c->b;
            return BTA_OK;
        case BTA_BLK_B:
            if (i < 0 || i >= c->n - 1) return BTA_ERR_ARG;
            *ptr_out = M->B + m * M->sB + i * bb;
            if (ld_out) *ld_out = c->b;
            return BTA_OK;
        case BTA_BLK_R:
            if (i < 0 || i >= c->n) return BTA_ERR_ARG;
            *ptr_out = M->R + m * M->sR + i * ab;
            if (ld_out) *ld_out = c->a;
            return BTA_OK;
        case BTA_BLK_T:
            *ptr_out = M->T + m * M->sT;
            if (ld_out) *ld_out = c->a;
            return BTA_OK;
        default:
            return BTA_ERR_ARG;
    }
}

// Record a timing event; inside a stream capture as an external event-record
// node of the graph (a plain record there would only order the capture).
int prof_record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BTA_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusActive) BTA_CUDA_TRY(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
    else BTA_CUDA_TRY(cudaEventRecord(e, s));
    return BTA_OK;
}

int prof_begin(bta_ctx_t ctx, cudaStream_t s, double flops, cudaEvent_t* stop_out) {
    *stop_out = nullptr;
    if (!ctx->prof) return BTA_OK;
    if (ctx->prof_used + 2 > ctx->prof_ev.size()) {
        for (int q = 0; q < 256; ++q) {
            cudaEvent_t e;
            BTA_CUDA_TRY(cudaEventCreate(&e));
            ctx->prof_ev.push_back(e);
        }
    }
    cudaEvent_t start = ctx->prof_ev[ctx->prof_used], stop = ctx->prof_ev[ctx->prof_used + 1];
    ctx->prof_used += 2;
    ctx->prof_flops += flops;
    BTA_TRY(prof_record(start, s));
    *stop_out = stop;
    return BTA_OK;
}

extern "C" int bta_profile(bta_ctx_t c, int enable) {
    if (!c) return BTA_ERR_ARG;
    enable = enable ? 1 : 0;
    if (enable == c->prof) return BTA_OK;
    // a captured f_obj graph has the event records of the old setting baked in
    if (c->fobj_graph) {
        cudaStreamSynchronize(c->stream);
        cudaGraphExecDestroy(c->fobj_graph);
        c->fobj_graph = nullptr;
        c->graph_calls = 1;
    }
    c->prof = enable;
    c->prof_used = 0;
    c->prof_flops = 0.0;
    c->phase_seen = 0;
    if (enable)
        for (cudaEvent_t& e : c->phase_ev)
            if (!e) BTA_CUDA_TRY(cudaEventCreate(&e));
    return BTA_OK;
}

int prof_phase(bta_ctx_t ctx, int k, cudaStream_t s) {
    if (!ctx->prof || !ctx->phase_ev[k]) return BTA_OK;
    BTA_TRY(prof_record(ctx->phase_ev[k], s));
    ctx->phase_seen |= 1 << k;
    return BTA_OK;
}

extern "C" int bta_profile_phases(bta_ctx_t c, double* ms_out, int count) {
    if (!c || !ms_out || count < 1) return BTA_ERR_ARG;
    const int all = (1 << (BTA_PHASES + 1)) - 1;
    if ((c->phase_seen & all) != all) return BTA_ERR_STATE;
    BTA_CUDA_TRY(cudaEventSynchronize(c->phase_ev[BTA_PHASES]));
    for (int k = 0; k < std::min(count, BTA_PHASES); ++k) {
        float ms = 0.f;
        BTA_CUDA_TRY(cudaEventElapsedTime(&ms, c->phase_ev[k], c->phase_ev[k + 1]));
        ms_out[k] = ms;
    }
    return BTA_OK;
}

extern "C" int bta_profile_read(bta_ctx_t c, double* ms_total, long long* launches, double* flops_total) {
    if (!c || !ms_total || !launches || !flops_total) return BTA_ERR_ARG;
    double ms = 0.0;
    for (size_t q = 0; q + 1 < c->prof_used; q += 2) {
        BTA_CUDA_TRY(cudaEventSynchronize(c->prof_ev[q + 1]));
        float t = 0.f;
        BTA_CUDA_TRY(cudaEventElapsedTime(&t, c->prof_ev[q], c->prof_ev[q + 1]));
        ms += t;
    }
    *ms_total = ms;
    *launches = (long long)(c->prof_used / 2);
    *flops_total = c->prof_flops;
    return BTA_OK;
}

extern "C" int bta_sync(bta_ctx_t c) {
    if (!c) return BTA_ERR_ARG;
    if (cudaStreamSynchronize(c->aux) != cudaSuccess) return bta_cuda_fail(cudaGetLastError());
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bta_cuda_fail(e);
    long long st[3];
    e = cudaMemcpy(st, c->status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bta_cuda_fail(e);
    if (c->oz_err) {
        int oz = 0;
        e = cudaMemcpy(&oz, c->oz_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bta_cuda_fail(e);
        if (oz) {
            // the products after the time-out are void, and so is any pivot
            // error they caused: clear both records
            cudaMemset(c->oz_err, 0, sizeof(int));
            long long zero[3] = {0, 0, 0};
            cudaMemcpy(c->status, zero, sizeof(zero), cudaMemcpyHostToDevice);
            c->last_info = -1;
            c->last_matrix = -1;
            return BTA_ERR_TIMEOUT;
        }
    }
    if (st[0] != 0) {
        c->last_info = st[1];
        c->last_matrix = (int)st[2];
        long long zero[3] = {0, 0, 0};
        cudaMemcpy(c->status, zero, sizeof(zero), cudaMemcpyHostToDevice);
        return (int)st[0];
    }
    c->last_info = -1;
    c->last_matrix = -1;
    return BTA_OK;
}

extern "C" int bta_last_info(bta_ctx_t c, long long* info) {
    if (!c || !info) return BTA_ERR_ARG;
    *info = c->last_info;
    return BTA_OK;
}

extern "C" int bta_last_error_matrix(bta_ctx_t c, int* which) {
    if (!c || !which) return BTA_ERR_ARG;
    *which = c->last_matrix;
    return BTA_OK;
}

extern "C" const char* bta_strerror(int code) {
    switch (code) {
        case BTA_OK: return "ok";
        case BTA_ERR_ARG: return "invalid argument";
        case BTA_ERR_OOM: return "device memory exhausted";
        case BTA_ERR_NOT_PD: return "matrix is not positive definite (non-positive pivot)";
        case BTA_ERR_TIMEOUT: return "bounded device wait ran out";
        case BTA_ERR_NONFINITE: return "non-finite value";
        case BTA_ERR_CUDA: return cudaGetErrorString(g_last_cuda);
        case BTA_ERR_STATE: return "call out of order";
        default: return "unknown error";
    }
}

// Switch between the default storage (factor, selected inverse and inverse
// diagonal blocks apart) and the low-memory one (see bta.h).  Assembled Q
// blocks are kept; factors and selected inverses are dropped.
extern "C" int bta_set_low_memory(bta_ctx_t c, int enable) {
    if (!c) return BTA_ERR_ARG;
    enable = enable ? 1 : 0;
    if (enable == c->lowmem) return BTA_OK;
    if (c->tparts > 1) return BTA_ERR_STATE;
    BTA_CUDA_TRY(cudaStreamSynchronize(c->stream));
    BTA_CUDA_TRY(cudaDeviceSynchronize());
    if (c->fobj_graph) {
        cudaGraphExecDestroy(c->fobj_graph);
        c->fobj_graph = nullptr;
        c->graph_calls = 1;
    }
    std::fill(c->factored.begin(), c->factored.end(), 0);
    if (c->lowmem) {
        c->S = BtaStore{};
        c->Linv = nullptr;
    } else {
        store_free(c->S);
        if (c->Linv) cudaFree(c->Linv);
        c->Linv = nullptr;
    }
    store_free(c->L);
    for (double** p : {&c->xtmp, &c->ldacc}) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    c->lowmem = 0;
    if (enable) {
        const int rc = alloc_low_factor(c);
        if (rc == BTA_OK) return BTA_OK;
        // fall back to the default layout
        c->lowmem = 0;
        c->Linv = nullptr;
        store_free(c->L);
        for (double** p : {&c->xtmp, &c->ldacc}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
        const int rc2 = alloc_default_factor(c);
        return rc2 == BTA_OK ? rc : rc2;
    }
    return alloc_default_factor(c);
}
