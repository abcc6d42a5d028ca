// Context life cycle, storage accessors, status and error reporting of the
// C ABI declared in include/bta.h.

#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"

#include <atomic>

static thread_local cudaError_t g_last_cuda = cudaSuccess;
static std::atomic<long long> g_launches{0};

void bta_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" long long bta_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int bta_cuda_fail(cudaError_t e) {
    g_last_cuda = e;
    if (e == cudaErrorMemoryAllocation) return BTA_ERR_OOM;
    return BTA_ERR_CUDA;
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

void mat_free(BtaMat& M) {
    if (M.D) cudaFree(M.D);
    if (M.B) cudaFree(M.B);
    if (M.R) cudaFree(M.R);
    if (M.T) cudaFree(M.T);
    M = BtaMat{};
}

int mat_alloc(BtaMat& M, int n, int b, int a) {
    const size_t bb = (size_t)b * b;
    BTA_TRY(dalloc(&M.D, (size_t)n * bb));
    BTA_TRY(dalloc(&M.B, (size_t)(n > 1 ? n - 1 : 0) * bb));
    BTA_TRY(dalloc(&M.R, (size_t)n * a * b));
    BTA_TRY(dalloc(&M.T, (size_t)a * a));
    return BTA_OK;
}

}  // namespace

int ensure_sigma(bta_ctx_t ctx, int which) {
    if (ctx->S[which].D) return BTA_OK;
    int rc = mat_alloc(ctx->S[which], ctx->n, ctx->b, ctx->a);
    if (rc != BTA_OK) mat_free(ctx->S[which]);
    return rc;
}

extern "C" int bta_create(int n, int b, int a, int precision, void* stream, bta_ctx_t* out) {
    if (!out || n < 1 || b < 1 || a < 0 || (precision != BTA_FP64 && precision != BTA_MIXED)) return BTA_ERR_ARG;
    *out = nullptr;
    bta_ctx_s* c = new bta_ctx_s();
    c->n = n; c->b = b; c->a = a; c->precision = precision;
    c->N = (long long)n * b + a;
    c->stream = (cudaStream_t)stream;
    c->leaf = 32;
    if (const char* e = std::getenv("BTA_LEAF")) c->leaf = std::atoi(e);
    c->vec = nullptr; c->red = nullptr; c->scal = nullptr; c->status = nullptr; c->params = nullptr;
    c->aux = nullptr; c->ev_fork = nullptr; c->ev_join = nullptr;
    c->exec[0] = GemmExec{};
    c->exec[1] = GemmExec{};
    int rc = BTA_OK;
    auto fail = [&](int r) { bta_destroy(c); return r; };
    if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess) return fail(BTA_ERR_CUDA);
    if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) return fail(BTA_ERR_CUDA);
    if (cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) return fail(BTA_ERR_CUDA);
    const size_t bb = (size_t)b * b;
    c->work_elems = bb + bb / 2 + 2 * (size_t)b + 2 * (size_t)a * b + (size_t)a * a + 64;
    for (int w = 0; w < 2; ++w) {
        if ((rc = mat_alloc(c->Q[w], n, b, a)) != BTA_OK) return fail(rc);
        if ((rc = mat_alloc(c->L[w], n, b, a)) != BTA_OK) return fail(rc);
        if ((rc = dalloc(&c->Linv[w], (size_t)n * bb + (size_t)a * a)) != BTA_OK) return fail(rc);
        if ((rc = dalloc(&c->work[w], c->work_elems)) != BTA_OK) return fail(rc);
        // the strict upper triangles of the inverse blocks are never written by the factor
        if (cudaMemset(c->Linv[w], 0, ((size_t)n * bb + (size_t)a * a) * sizeof(double)) != cudaSuccess)
            return fail(BTA_ERR_CUDA);
    }
    c->exec[0] = GemmExec{};
    c->exec[1] = GemmExec{};
    c->refine = 0;
    if (precision == BTA_MIXED) {
        if (cudaMalloc((void**)&c->oz_err, sizeof(int)) != cudaSuccess) return fail(BTA_ERR_OOM);
        if (cudaMemset(c->oz_err, 0, sizeof(int)) != cudaSuccess) return fail(BTA_ERR_CUDA);
        int min_dim = 256;
        if (const char* e = std::getenv("BTA_OZ_MIN")) min_dim = std::atoi(e);
        const size_t wsb = ozaki_workspace_bytes(b, b, b);
        for (int w = 0; w < 2; ++w) {
            if (cudaMalloc(&c->exec[w].ws, wsb) != cudaSuccess) {
                c->exec[w].ws = nullptr;
                return fail(BTA_ERR_OOM);
            }
            c->exec[w].fn = gemm_mixed_fn;
            c->exec[w].ws_bytes = wsb;
            c->exec[w].err = c->oz_err;
            c->exec[w].min_dim = min_dim;
        }
        c->refine = 2;
    }
    if (const char* e = std::getenv("BTA_REFINE")) c->refine = std::atoi(e);
    if ((rc = dalloc(&c->vec, 9 * (size_t)c->N)) != BTA_OK) return fail(rc);
    c->red_len = 2 * 1216;
    if ((rc = dalloc(&c->red, c->red_len)) != BTA_OK) return fail(rc);
    if ((rc = dalloc(&c->scal, SCAL_COUNT)) != BTA_OK) return fail(rc);
    if ((rc = dalloc(&c->params, 5 * BTA_MAX_NV + BTA_MAX_NV * BTA_MAX_NV)) != BTA_OK) return fail(rc);
    if (cudaMalloc((void**)&c->status, 2 * sizeof(long long)) != cudaSuccess) return fail(BTA_ERR_OOM);
    if (cudaMemset(c->status, 0, 2 * sizeof(long long)) != cudaSuccess) return fail(BTA_ERR_CUDA);
    if (cudaMemset(c->scal, 0, SCAL_COUNT * sizeof(double)) != cudaSuccess) return fail(BTA_ERR_CUDA);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(BTA_ERR_CUDA);
    *out = c;
    return BTA_OK;
}

extern "C" int bta_destroy(bta_ctx_t c) {
    if (!c) return BTA_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->aux) cudaStreamSynchronize(c->aux);
    for (int w = 0; w < 2; ++w) {
        mat_free(c->Q[w]);
        mat_free(c->L[w]);
        mat_free(c->S[w]);
        if (c->Linv[w]) cudaFree(c->Linv[w]);
        if (c->work[w]) cudaFree(c->work[w]);
    }
    for (int w = 0; w < 2; ++w)
        if (c->exec[w].ws) cudaFree(c->exec[w].ws);
    if (c->oz_err) cudaFree(c->oz_err);
    if (c->vec) cudaFree(c->vec);
    if (c->red) cudaFree(c->red);
    if (c->scal) cudaFree(c->scal);
    if (c->params) cudaFree(c->params);
    if (c->status) cudaFree(c->status);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->aux) cudaStreamDestroy(c->aux);
    delete c;
    return BTA_OK;
}

extern "C" int bta_block_ptr(bta_ctx_t c, int which, int store, int kind, int i, double** ptr_out, int* ld_out) {
    if (!c || !ptr_out || (which != BTA_QP && which != BTA_QC)) return BTA_ERR_ARG;
    const size_t bb = (size_t)c->b * c->b, ab = (size_t)c->a * c->b;
    const BtaMat* M = nullptr;
    if (store == BTA_STORE_Q) M = &c->Q[which];
    else if (store == BTA_STORE_L) M = &c->L[which];
    else if (store == BTA_STORE_SIGMA) M = &c->S[which];
    else if (store != BTA_STORE_LINV) return BTA_ERR_ARG;
    if (store == BTA_STORE_LINV) {
        if (kind == BTA_BLK_D && i >= 0 && i < c->n) {
            *ptr_out = c->Linv[which] + i * bb;
            if (ld_out) *ld_out = c->b;
            return BTA_OK;
        }
        if (kind == BTA_BLK_T) {
            *ptr_out = c->Linv[which] + (size_t)c->n * bb;
            if (ld_out) *ld_out = c->a;
            return BTA_OK;
        }
        return BTA_ERR_ARG;
    }
    if (!M->D) return BTA_ERR_STATE;
    switch (kind) {
        case BTA_BLK_D:
            if (i < 0 || i >= c->n) return BTA_ERR_ARG;
            *ptr_out = M->D + i * bb;
            if (ld_out) *ld_out = c->b;
            return BTA_OK;
        case BTA_BLK_B:
            if (i < 0 || i >= c->n - 1) return BTA_ERR_ARG;
            *ptr_out = M->B + i * bb;
            if (ld_out) *ld_out = c->b;
            return BTA_OK;
        case BTA_BLK_R:
            if (i < 0 || i >= c->n) return BTA_ERR_ARG;
            *ptr_out = M->R + i * ab;
            if (ld_out) *ld_out = c->a;
            return BTA_OK;
        case BTA_BLK_T:
            *ptr_out = M->T;
            if (ld_out) *ld_out = c->a;
            return BTA_OK;
        default:
            return BTA_ERR_ARG;
    }
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
    BTA_CUDA_TRY(cudaEventRecord(start, s));
    *stop_out = stop;
    return BTA_OK;
}

extern "C" int bta_profile(bta_ctx_t c, int enable) {
    if (!c) return BTA_ERR_ARG;
    c->prof = enable ? 1 : 0;
    c->prof_used = 0;
    c->prof_flops = 0.0;
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
    long long st[2];
    e = cudaMemcpy(st, c->status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bta_cuda_fail(e);
    if (c->oz_err) {
        int oz = 0;
        e = cudaMemcpy(&oz, c->oz_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bta_cuda_fail(e);
        if (oz) {
            cudaMemset(c->oz_err, 0, sizeof(int));
            c->last_info = -1;
            return BTA_ERR_TIMEOUT;
        }
    }
    if (st[0] != 0) {
        c->last_info = st[1];
        long long zero[2] = {0, 0};
        cudaMemcpy(c->status, zero, sizeof(zero), cudaMemcpyHostToDevice);
        return (int)st[0];
    }
    c->last_info = -1;
    return BTA_OK;
}

extern "C" int bta_last_info(bta_ctx_t c, long long* info) {
    if (!c || !info) return BTA_ERR_ARG;
    *info = c->last_info;
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
