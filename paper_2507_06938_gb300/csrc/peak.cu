// FP64 throughput probes: the measured denominators of the FP64 path's
// roofline (the measured peaks the benchmark reads cover HBM and bf16 only).

#include "common.cuh"

namespace {

constexpr int PEAK_CHAINS = 16;   // independent FMA chains per thread (covers the FP64 latency)

__global__ void dfma_probe_kernel(double* out, int iters, double b, double c) {
    double acc[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) acc[k] = 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) acc[k] = fma(acc[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += acc[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int DMMA_SETS = 4;   // independent accumulator tiles per warp

// D = A B + D with m8n8k4 FP64 MMAs (each thread holds one A and one B
// element and two accumulator elements per tile).
__global__ void dmma_probe_kernel(double* out, int iters, double av, double bv) {
    double d[DMMA_SETS][2];
#pragma unroll
    for (int k = 0; k < DMMA_SETS; ++k) d[k][0] = d[k][1] = 0.0;
    const double a = av * (1 + threadIdx.x % 3), b = bv;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < DMMA_SETS; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(d[k][0]), "+d"(d[k][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < DMMA_SETS; ++k) s += d[k][0] + d[k][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int bta_fp64_peak(int use_dmma, double* tflops_out) {
    if (!tflops_out) return BTA_ERR_ARG;
    int dev = 0, sms = 0;
    BTA_CUDA_TRY(cudaGetDevice(&dev));
    BTA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = sms * 8;
    double* out = nullptr;
    BTA_CUDA_TRY(cudaMalloc((void**)&out, (size_t)blocks * threads * sizeof(double)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = BTA_OK;
    float ms = 0.f;
    double flops_per_iter = 0.0;
    const int iters = use_dmma ? 4096 : 8192;
    for (int rep = 0; rep < 2 && rc == BTA_OK; ++rep) {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rc = BTA_ERR_CUDA;
            break;
        }
        cudaEventRecord(e0, 0);
        if (use_dmma) {
            dmma_probe_kernel<<<blocks, threads>>>(out, iters, 1.0000001, 0.999999);
            flops_per_iter = (double)blocks * (threads / 32) * DMMA_SETS * 2.0 * 8 * 8 * 4;
        } else {
            dfma_probe_kernel<<<blocks, threads>>>(out, iters, 0.9999999, 1e-7);
            flops_per_iter = (double)blocks * threads * PEAK_CHAINS * 2.0;
        }
        bta_note_launch();
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = BTA_ERR_CUDA;
        else cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        e0 = e1 = nullptr;
    }
    cudaFree(out);
    if (rc != BTA_OK) return rc;
    *tflops_out = flops_per_iter * iters / (ms * 1e-3) / 1e12;
    return BTA_OK;
}
