// The noise of the Langevin step (Sec. III.C) on its own, for checking: the Box-Muller
// map from four 32-bit words to three normals, and the Philox draw of a bead at a step,
// by the same device functions every step kernel calls (box_muller3, bead_noise).
#include <cuda_runtime.h>

#include <string>

#include "sop_internal.h"

namespace sop {
namespace {

constexpr int kNoiseThreads = 256;

__global__ void k_box_muller(const uint4 *__restrict__ x, int64_t n, float4 *__restrict__ g) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float3 v = box_muller3(x[k]);
    g[k] = make_float4(v.x, v.y, v.z, 0.f);
}

__global__ void k_bead_noise(uint64_t seed, int64_t step, uint32_t bead_lo, int64_t n, float4 *__restrict__ g) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float3 v = bead_noise(seed, step, bead_lo + (uint32_t)k);
    g[k] = make_float4(v.x, v.y, v.z, 0.f);
}

// Runs `launch` over n items with device buffers of in_bytes (copied from `in`, may be 0)
// and n float4 results, widened into out[3n]; synchronises the stream.
template <class Launch>
sop_status run_noise(const char *who, const void *in, size_t in_bytes, int64_t n, double *out, void *cuda_stream,
                     Launch launch) {
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    void *d_in = nullptr;
    float4 *d_out = nullptr;
    auto cuda_fail = [&](cudaError_t e) {
        set_global_error(std::string(who) + ": " + cudaGetErrorString(e));
        if (d_in) cudaFree(d_in);
        if (d_out) cudaFree(d_out);
        return e == cudaErrorMemoryAllocation ? SOP_ERR_OOM : SOP_ERR_CUDA;
    };
    cudaError_t e = cudaSuccess;
    if (in_bytes) {
        e = cudaMalloc(&d_in, in_bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_in, in, in_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    e = cudaMalloc(&d_out, sizeof(float4) * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(e);
    const int64_t blocks = (n + kNoiseThreads - 1) / kNoiseThreads;
    launch(d_in, d_out, (unsigned)blocks, s);
    e = cudaGetLastError();
    std::vector<float4> host((size_t)n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), d_out, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int64_t k = 0; k < n; ++k) {
        out[3 * k] = host[k].x;
        out[3 * k + 1] = host[k].y;
        out[3 * k + 2] = host[k].z;
    }
    if (d_in) cudaFree(d_in);
    cudaFree(d_out);
    return SOP_OK;
}

constexpr int64_t kMaxNoiseItems = (int64_t)1 << 26;   // 1 GiB of FP32 results at most

}  // namespace
}  // namespace sop

extern "C" sop_status sop_box_muller(const uint32_t *x, int64_t n, double *out, void *cuda_stream) {
    using namespace sop;
    if (n < 0 || n > kMaxNoiseItems || (n > 0 && (!x || !out))) {
        set_global_error("sop_box_muller: n in 0 .. 2^26 and non-NULL arrays required");
        return SOP_ERR_INVALID_ARG;
    }
    if (n == 0) return SOP_OK;
    return run_noise("sop_box_muller", x, sizeof(uint4) * (size_t)n, n, out, cuda_stream,
                     [n](void *d_in, float4 *d_out, unsigned blocks, cudaStream_t s) {
                         k_box_muller<<<blocks, kNoiseThreads, 0, s>>>(static_cast<const uint4 *>(d_in), n, d_out);
                     });
}

extern "C" sop_status sop_bead_noise(uint64_t key, int64_t step, uint32_t bead_lo, int64_t n, double *out,
                                     void *cuda_stream) {
    using namespace sop;
    if (n < 0 || n > kMaxNoiseItems || (n > 0 && !out) || (uint64_t)bead_lo + (uint64_t)n > 0x100000000ull) {
        set_global_error("sop_bead_noise: n in 0 .. 2^26, bead_lo + n <= 2^32, non-NULL out required");
        return SOP_ERR_INVALID_ARG;
    }
    if (n == 0) return SOP_OK;
    return run_noise("sop_bead_noise", nullptr, 0, n, out, cuda_stream,
                     [=](void *, float4 *d_out, unsigned blocks, cudaStream_t s) {
                         k_bead_noise<<<blocks, kNoiseThreads, 0, s>>>(key, step, bead_lo, n, d_out);
                     });
}
