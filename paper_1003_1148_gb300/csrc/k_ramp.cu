// Integrator-accuracy experiment of Sec. IV.C on the GPU (sm_103a).
//
// Each thread advances one run of the Brownian particle in the harmonic potential
// K X^2 / 2 under the ramp force r_f t with the first-order update (Eq. 4's drift, or
// Eq. 5's) plus noise, in FP32 with a compensated (Kahan) position. The runs are
// independent: no communication until a checkpoint, where every CTA sums X and X^2 of
// its runs in FP64 and the host adds the CTA sums in a fixed order (the result does not
// depend on scheduling). Noise comes four steps at a time from one Philox block.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "sop_internal.h"

namespace sop {
namespace {

constexpr int kRampThreads = 256;

struct RampArgs {
    float c_n;      // coefficient of n in the drift
    float c_x;      // coefficient of -X
    float c_0;      // constant part
    float amp;      // sqrt(2 kT h / xi)
    uint32_t key0, key1;
    int32_t n_runs;
};

// Four normals of block b of run `run`: Box-Muller on (x0, x1) and (x2, x3), cos then sin.
__device__ __forceinline__ float4 ramp_normals(const RampArgs &a, uint64_t b, uint32_t run) {
    const uint4 x = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(b >> 32), run, 1u), a.key0, a.key1);
    const float two_m31 = 4.656612873077393e-10f;
    const float ra = sqrtf(minus_two_log_u(x.x));
    const float rb = sqrtf(minus_two_log_u(x.z));
    float s1, c1, s2, c2;
    sincospif((float)x.y * two_m31, &s1, &c1);
    sincospif((float)x.w * two_m31, &s2, &c2);
    return make_float4(ra * c1, ra * s1, rb * c2, rb * s2);
}

__device__ __forceinline__ float pick(const float4 &g, int k) {
    return k == 0 ? g.x : (k == 1 ? g.y : (k == 2 ? g.z : g.w));
}

// Steps [n0, n1) of every run; with `partial`, the CTA's FP64 sums of X and X^2 after them.
__global__ void __launch_bounds__(kRampThreads) k_ramp(RampArgs a, float2 *__restrict__ state, int64_t n0,
                                                      int64_t n1, double *__restrict__ partial) {
    const int run = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = run < a.n_runs;
    double xd = 0.0;
    if (live) {
        float2 s = state[run];   // (X, compensation)
        float X = s.x, c = s.y;
        int64_t n = n0;
        if (a.amp == 0.f) {
            for (; n < n1; ++n) kahan_add(X, c, fmaf(-a.c_x, X, fmaf(a.c_n, (float)n, a.c_0)));
        } else {
            float4 g = ramp_normals(a, (uint64_t)(n >> 2), (uint32_t)run);
            for (; n < n1 && (n & 3); ++n)   // the rest of a block begun in the previous launch
                kahan_add(X, c, fmaf(a.amp, pick(g, (int)(n & 3)), fmaf(-a.c_x, X, fmaf(a.c_n, (float)n, a.c_0))));
            for (; n + 4 <= n1; n += 4) {   // whole blocks
                g = ramp_normals(a, (uint64_t)(n >> 2), (uint32_t)run);
                const float fn = (float)n;
                kahan_add(X, c, fmaf(a.amp, g.x, fmaf(-a.c_x, X, fmaf(a.c_n, fn, a.c_0))));
                kahan_add(X, c, fmaf(a.amp, g.y, fmaf(-a.c_x, X, fmaf(a.c_n, (float)(n + 1), a.c_0))));
                kahan_add(X, c, fmaf(a.amp, g.z, fmaf(-a.c_x, X, fmaf(a.c_n, (float)(n + 2), a.c_0))));
                kahan_add(X, c, fmaf(a.amp, g.w, fmaf(-a.c_x, X, fmaf(a.c_n, (float)(n + 3), a.c_0))));
            }
            if (n < n1) {   // a final partial block
                g = ramp_normals(a, (uint64_t)(n >> 2), (uint32_t)run);
                for (; n < n1; ++n)
                    kahan_add(X, c, fmaf(a.amp, pick(g, (int)(n & 3)), fmaf(-a.c_x, X, fmaf(a.c_n, (float)n, a.c_0))));
            }
        }
        state[run] = make_float2(X, c);
        xd = (double)X - (double)c;
    }
    if (!partial) return;
    __shared__ double sh[2][kRampThreads / 32];
    double s1 = live ? xd : 0.0, s2 = live ? xd * xd : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s1;
        sh[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < kRampThreads / 32; ++w) {
            t1 += sh[0][w];
            t2 += sh[1][w];
        }
        partial[2 * blockIdx.x] = t1;
        partial[2 * blockIdx.x + 1] = t2;
    }
}

__global__ void k_ramp_init(float2 *state, int n, float X0) {
    const int run = blockIdx.x * blockDim.x + threadIdx.x;
    if (run < n) state[run] = make_float2(X0, 0.f);
}

__global__ void k_ramp_final(const float2 *state, int n, double *out) {
    const int run = blockIdx.x * blockDim.x + threadIdx.x;
    if (run < n) out[run] = (double)state[run].x - (double)state[run].y;
}

}  // namespace
}  // namespace sop

extern "C" sop_status sop_brownian_ramp(const sop_ramp_params *p, double *mean, double *var, double *x_final,
                                        void *cuda_stream) {
    using namespace sop;
    auto bad = [](const char *msg) {
        set_global_error(std::string("sop_brownian_ramp: ") + msg);
        return SOP_ERR_INVALID_ARG;
    };
    if (!p || !mean || !var) return bad("params, mean and var are required");
    if (!(p->K > 0) || !(p->xi > 0) || !(p->kT >= 0) || !(p->h > 0) || !std::isfinite(p->K) ||
        !std::isfinite(p->xi) || !std::isfinite(p->kT) || !std::isfinite(p->h) || !std::isfinite(p->r_f) ||
        !std::isfinite(p->X0))
        return bad("K, xi, h > 0, kT >= 0, all finite");
    if (p->n_runs < 1 || p->n_runs > 0x7fffffff) return bad("n_runs in 1 .. 2^31 - 1");
    if (p->n_steps < 1 || p->n_out < 1 || p->n_out > p->n_steps) return bad("n_steps >= 1, 1 <= n_out <= n_steps");
    if (p->order < 1 || p->order > 3) return bad("order 1, 2 or 3");
    // drift = c_n n + c_0 - c_x X, the coefficients folded in FP64
    const double tau = p->xi / p->K, h = p->h;
    double c_n = p->r_f * h * h / p->xi, c_x = h / tau, c_0 = 0.0;
    if (p->order >= 2) {
        c_n -= p->r_f * h * h * h / (2.0 * tau * p->xi);
        c_x -= h * h / (2.0 * tau * tau);
    }
    if (p->order == 3) c_0 = p->r_f * h * h / (2.0 * p->xi);
    RampArgs a;
    a.c_n = (float)c_n;
    a.c_x = (float)c_x;
    a.c_0 = (float)c_0;
    a.amp = (float)std::sqrt(2.0 * p->kT * h / p->xi);
    a.key0 = (uint32_t)p->seed;
    a.key1 = (uint32_t)(p->seed >> 32);
    a.n_runs = (int32_t)p->n_runs;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int n = (int)p->n_runs;
    const int blocks = (n + kRampThreads - 1) / kRampThreads;
    float2 *state = nullptr;
    double *partial = nullptr, *fin = nullptr;
    auto cuda_fail = [&](cudaError_t e) {
        set_global_error(std::string("sop_brownian_ramp: ") + cudaGetErrorString(e));
        if (state) cudaFree(state);
        if (partial) cudaFree(partial);
        if (fin) cudaFree(fin);
        return e == cudaErrorMemoryAllocation ? SOP_ERR_OOM : SOP_ERR_CUDA;
    };
    cudaError_t e = cudaMalloc(&state, sizeof(float2) * n);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaMalloc(&partial, sizeof(double) * 2 * blocks);
    if (e != cudaSuccess) return cuda_fail(e);
    k_ramp_init<<<blocks, kRampThreads, 0, s>>>(state, n, (float)p->X0);
    // launches of about 2^35 run-steps each (tens of milliseconds), aligned to the checkpoints
    const int64_t chunk = std::max<int64_t>(4, ((int64_t)1 << 35) / p->n_runs / 4 * 4);
    std::vector<double> host(2 * blocks);
    int64_t n0 = 0;
    for (int k = 0; k < p->n_out; ++k) {
        const int64_t stop = p->n_steps * (k + 1) / p->n_out;
        while (n0 < stop) {
            const int64_t n1 = std::min(stop, n0 + chunk);
            k_ramp<<<blocks, kRampThreads, 0, s>>>(a, state, n0, n1, n1 == stop ? partial : nullptr);
            n0 = n1;
        }
        e = cudaMemcpyAsync(host.data(), partial, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e);
        double s1 = 0.0, s2 = 0.0;
        for (int b = 0; b < blocks; ++b) {
            s1 += host[2 * b];
            s2 += host[2 * b + 1];
        }
        const double m = s1 / (double)n;
        mean[k] = m;
        var[k] = std::max(0.0, s2 / (double)n - m * m);
    }
    if (x_final) {
        e = cudaMalloc(&fin, sizeof(double) * n);
        if (e != cudaSuccess) return cuda_fail(e);
        k_ramp_final<<<blocks, kRampThreads, 0, s>>>(state, n, fin);
        e = cudaMemcpyAsync(x_final, fin, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    cudaFree(state);
    cudaFree(partial);
    if (fin) cudaFree(fin);
    return SOP_OK;
}
