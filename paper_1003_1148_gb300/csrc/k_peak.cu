// FP32 FMA throughput of the device (the denominator of the FP32 roofline of the batched
// kernels). Every thread runs eight independent FMA chains, so the FMA pipes, not the
// dependency latency, bound the rate; the grid holds four CTAs of 256 threads per SM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "sop_internal.h"

namespace sop {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_ffma(float *out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true: keeps the chains live
}

}  // namespace
}  // namespace sop

extern "C" {

sop_status sop_fp32_peak(double seconds, double *tflops, double *elapsed_ms, int32_t *sm_count) {
    if (!tflops || !(seconds > 0) || seconds > 10) {
        sop::set_global_error("sop_fp32_peak: tflops required, 0 < seconds <= 10");
        return SOP_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float *out = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * 256 * 4 * (size_t)sms);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int grid = 4 * sms;
    double rate = 0.0, ms_last = 0.0;
    int iters = 1 << 12;
    for (int round = 0; round < 8 && e == cudaSuccess; ++round) {
        cudaEventRecord(e0);
        sop::k_ffma<<<grid, 256>>>(out, iters, 0.999999f, 1e-6f);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * 4 * sop::kChains * (double)iters * 256.0 * grid;
        if (ms > 0) rate = std::max(rate, flops / (ms * 1e-3) / 1e12);
        ms_last = ms;
        if (ms >= 1e3 * seconds) break;
        // grow the launch toward the requested duration
        const double scale = ms > 0 ? std::min(64.0, 1e3 * seconds / ms) : 64.0;
        const double next = (double)iters * scale;
        iters = next > 1e9 ? 1000000000 : (int)next;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        sop::set_global_error(std::string("sop_fp32_peak: ") + cudaGetErrorString(e));
        return SOP_ERR_CUDA;
    }
    *tflops = rate;
    if (elapsed_ms) *elapsed_ms = ms_last;
    if (sm_count) *sm_count = sms;
    return SOP_OK;
}

}  // extern "C"
