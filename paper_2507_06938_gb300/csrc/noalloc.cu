// Allocation-free Cholesky + inverse of one dense SPD block.
//
// The paper has no counterpart to this entry point: it exists for callers of
// this library that may not call cudaMalloc, for example a host framework
// whose own memory pool already owns the device memory budget (a raw
// cudaMalloc beside it can fail or fragment the pool), or a latency-bound
// serving loop that cannot afford the device-wide synchronisation a
// cudaMalloc/cudaFree pair can cause.  Such a caller passes only its input
// and output buffers; the workspace of the recursive factorisation lives in
// one file-scope __device__ array of fixed size that every GPU loading this
// library holds until the process exits.

#include <mutex>

#include "common.cuh"

namespace {

// Largest block order accepted, and the scratch it needs: the top level of
// the recursion uses an n2 x n1 panel with n1 <= ceil(b/2) rounded up to the
// leaf size and n2 <= b/2.
constexpr int NOALLOC_LEAF = 32;
constexpr int NOALLOC_MAX_B = 2048;
constexpr long long NOALLOC_STATUS_ELEMS = 32;   // 256 bytes: [0] code, [1] row (as long long)
constexpr long long NOALLOC_W_ELEMS = (long long)(NOALLOC_MAX_B / 2 + NOALLOC_LEAF) * (NOALLOC_MAX_B / 2);
constexpr long long NOALLOC_ELEMS = NOALLOC_STATUS_ELEMS + NOALLOC_W_ELEMS;   // 8.5 MiB of doubles

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_ELEMS];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[MAX_DEVICES] = {nullptr};

long long top_panel_elems(int b, int leaf) {
    if (b <= leaf) return 0;
    const int half = (b + 1) / 2;
    int n1 = ((half + leaf - 1) / leaf) * leaf;
    if (n1 >= b) n1 = leaf;
    return (long long)n1 * (b - n1);
}

// info[0] = -1 if every pivot was positive, else the 0-based row of the first
// non-positive pivot.
__global__ void noalloc_finish_kernel(const long long* status, long long* info) {
    info[0] = status[0] != 0 ? status[1] : -1;
}

// X's strict upper triangle is not touched by the factorisation; make it zero.
__global__ void noalloc_zero_upper_kernel(double* X, long long ldx, int b) {
    const long long total = (long long)b * b;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % b), j = (int)(e / b);
        if (i < j) X[i + j * ldx] = 0.0;
    }
}

}  // namespace

extern "C" int bta_chol_inv_noalloc(double* A, int b, int lda, double* X, int ldx, long long* info_dev,
                                    void* stream) {
    if (!A || !X || !info_dev || b < 1 || lda < b || ldx < b) return BTA_ERR_ARG;
    if (b > NOALLOC_MAX_B || top_panel_elems(b, NOALLOC_LEAF) > NOALLOC_W_ELEMS) return BTA_ERR_ARG;
    int dev = 0;
    BTA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return BTA_ERR_ARG;
    double* base = nullptr;
    {
        // one-time set-up per device, with that device current: the host-side
        // name of the array is not a device address, so ask the runtime for it
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            BTA_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_scratch_ptr[dev] = static_cast<double*>(p);
        }
        base = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    long long* status = reinterpret_cast<long long*>(base);
    double* W = base + NOALLOC_STATUS_ELEMS;
    // the status words keep the previous call's contents: clear them
    BTA_CUDA_TRY(cudaMemsetAsync(status, 0, 2 * sizeof(long long), s));
    BTA_TRY(chol_inv64(s, A, lda, X, ldx, b, 0, status, W, NOALLOC_LEAF));
    noalloc_zero_upper_kernel<<<(int)std::min<long long>(((long long)b * b + 255) / 256, 152 * 8), 256, 0, s>>>(
        X, ldx, b);
    BTA_LAUNCH_CHECK();
    noalloc_finish_kernel<<<1, 1, 0, s>>>(status, info_dev);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}
