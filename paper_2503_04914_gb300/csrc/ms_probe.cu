// Instruction-rate probes: the FP32, FP64 and XU (special-function) peaks of this GPU as
// the library's own kernels reach them, the denominators of the ALU-bound rooflines (the
// matrix-free mat-vec is bound by FP32 and XU issue, the FP64 CSR kernels by FP64 issue).
// Every thread runs kChains independent dependent chains, enough to hide the pipes'
// latency, on a grid of kBlocksPerSM blocks per SM.
#include <algorithm>

#include "ms_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kProbeBS = 256;
constexpr int kBlocksPerSM = 4;

template <int KIND>
__global__ void __launch_bounds__(kProbeBS) k_probe(float* out, int iters) {
    const float seed = 1.0f + 1e-3f * (float)(threadIdx.x & 7);
    if (KIND == MS_PROBE_FP64) {
        double a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = (double)seed + c;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], 0.999999999, 1e-9);
        }
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += a[c];
        if (s == 12345.0) out[0] = (float)s;  // keeps the chains live; never true
    } else {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = seed + c;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if (KIND == MS_PROBE_FP32) a[c] = fmaf(a[c], 0.9999999f, 1e-7f);
                else a[c] = rsqrtf(a[c]);  // stays near 1 (rsqrt of ~1)
            }
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += a[c];
        if (s == 12345.0f) out[0] = s;
    }
}

}  // namespace

extern "C" ms_status ms_peak_probe(int kind, double* per_s) {
    if (!per_s || kind < MS_PROBE_FP32 || kind > MS_PROBE_XU) {
        ms_set_error(MS_ERR_ARG, "kind must be MS_PROBE_FP32, MS_PROBE_FP64 or MS_PROBE_XU and per_s non-NULL");
        return MS_ERR_ARG;
    }
    int dev = 0, sms = 0;
    MS_CUDA(cudaGetDevice(&dev));
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const void* fn = kind == MS_PROBE_FP32 ? (const void*)k_probe<MS_PROBE_FP32>
                   : kind == MS_PROBE_FP64 ? (const void*)k_probe<MS_PROBE_FP64>
                                           : (const void*)k_probe<MS_PROBE_XU>;
    // about 10 ms per launch on GB300 (FP64 issues at 1/64 of the FP32 rate)
    int iters = kind == MS_PROBE_FP64 ? 2000 : (kind == MS_PROBE_XU ? 20000 : 100000);
    float* out = nullptr;
    MS_CUDA(cudaMalloc((void**)&out, sizeof(float)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const dim3 grid(sms * kBlocksPerSM);
    void* args[] = {&out, &iters};
    float best = 0.f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // the first launch warms up
        cudaEventRecord(e0);
        err = cudaLaunchKernel(fn, grid, dim3(kProbeBS), args, 0, 0);
        ms_count_launch();
        cudaEventRecord(e1);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
            best = best == 0.f ? ms : std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return ms_cuda_error(err, "instruction-rate probe", __FILE__, __LINE__);
    const double ops = (double)grid.x * kProbeBS * (double)iters * kChains;
    *per_s = best > 0.f ? ops / (best * 1e-3) : 0.0;
    return MS_OK;
}
