// Device pieces shared by the one-CTA forms of the batched schedule: the particle-based
// gather (k_batched.cu) and the pair-based form (k_bpair.cu). Each form keeps one work
// item (a system of one replica) in one CTA's shared memory for a whole chunk of steps.
#pragma once

#include <cuda_runtime.h>

#include "sop_internal.h"
#include "sop_step.cuh"

namespace sop {
namespace {

constexpr int kKeys = 257;   // row lengths 0..256

// Head of a work item's shared memory for CTAs of up to 32 W threads.
template <int W>
struct HeadT {
    int fail;               // first sop_status raised in this CTA
    int hist[kKeys];        // counting sort of slots by row length
    double red[W][6];       // FP64 block reductions, one row per warp
};
using SharedHead = HeadT<32>;

// The arrays follow the head at a 16-byte aligned offset (float4 accesses).
constexpr size_t kHeadBytes = (sizeof(SharedHead) + 15) / 16 * 16;

template <class H>
__device__ __forceinline__ void cta_fail(H *h, int code) { atomicCAS(&h->fail, 0, code); }

// The CTA's dynamic shared memory; each form lays out its work item in it.
extern __shared__ __align__(16) unsigned char g_smem[];

// FP64 block sum of 6 values; result valid in thread 0.
template <class H>
__device__ __forceinline__ void block_sum6(double v[6], H *h) {
#pragma unroll
    for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < 6; ++k) h->red[w][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 6; ++k) {
            double s = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += h->red[q][k];
            v[k] = s;
        }
    }
}

// Bounding boxes of the blocks of 32 consecutive beads of layer src (one warp per block).
template <class Lay>
__device__ void block_boxes(const Lay &L, const float4 *src, int n_s) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float4 *bb = L.bbox();
    for (int blk = w; blk * 32 < n_s; blk += nw) {
        const int b = blk * 32 + lane;
        float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
        if (b < n_s) {
            const float4 p = src[b];
            lx = hx = p.x; ly = hy = p.y; lz = hz = p.z;
        }
        for (int o = 16; o > 0; o >>= 1) {
            lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
            ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
            lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
            hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
            hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
            hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        }
        if (lane == 0) {
            bb[2 * blk] = make_float4(lx, ly, lz, 0.f);
            bb[2 * blk + 1] = make_float4(hx, hy, hz, 0.f);
        }
    }
}

// Hand the slots to beads by decreasing row length of the last build (counting sort).
// Returns the index (0/1) of the new order buffer. Must be called by all threads.
template <class Lay>
__device__ int reorder_slots(const Lay &L, int n_s, int cur_order, int round = 0) {
    const int T = blockDim.x;
    const int U = round > 0 ? round : T;   // slots handed out per round (threads, or groups of lanes)
    auto *h = L.h();
    for (int k = threadIdx.x; k < kKeys; k += T) h->hist[k] = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < n_s; p += T) atomicAdd(&h->hist[kKeys - 1 - min((int)L.n_tot()[p], kKeys - 1)], 1);
    __syncthreads();
    if (threadIdx.x < 32) {   // exclusive scan of the histogram by one warp
        const int lane = threadIdx.x;
        const int per = (kKeys + 31) / 32;
        int local = 0;
        for (int k = lane * per; k < min(kKeys, lane * per + per); ++k) local += h->hist[k];
        int inc = local;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        int run = inc - local;
        for (int k = lane * per; k < min(kKeys, lane * per + per); ++k) {
            const int c = h->hist[k];
            h->hist[k] = run;
            run += c;
        }
    }
    __syncthreads();
    const uint16_t *src = L.order(cur_order);
    uint16_t *dst = L.order(cur_order ^ 1);
    const int full = n_s - n_s % U;   // slots in complete rounds of U
    for (int p = threadIdx.x; p < n_s; p += T) {
        int pos = atomicAdd(&h->hist[kKeys - 1 - min((int)L.n_tot()[p], kKeys - 1)], 1);
        // boustrophedon: odd rounds run backwards, so a thread owning several slots gets
        // long and short rows alike and the warps of the CTA finish together
        if (pos < full && ((pos / U) & 1)) pos = (pos / U) * U + (U - 1 - pos % U);
        dst[pos] = src[p];
    }
    __syncthreads();
    return cur_order ^ 1;
}

// Systems of at most this many beads keep x, y, z arrays for the rebuild scan (12 bytes
// per bead of shared memory); larger ones scan the float4 layer directly.
constexpr int kSoaMaxBeads = 1024;

// One block of 32 candidates base .. base + 31 read from a float4 layer: bit t is set when
// the FP32 squared distance to candidate base + t is below hi; bits at or beyond lim clear.
__device__ __forceinline__ uint32_t scan_block_f4(const float4 *src, int base, int lim, float4 pb, float hi) {
    uint32_t w = 0u;
    if (lim >= 32) {
#pragma unroll 8
        for (int t = 0; t < 32; ++t) {
            const float4 pj = src[base + t];
            const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            w |= (r2 < hi ? 1u : 0u) << t;
        }
    } else {
        for (int t = 0; t < lim; ++t) {
            const float4 pj = src[base + t];
            const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            w |= (r2 < hi ? 1u : 0u) << t;
        }
    }
    return w;
}

// Positions of layer src as three arrays x, y, z of stride S (a multiple of 32, S >= n_s),
// zero beyond n_s, for the rebuild scan. The caller publishes them with a barrier.
__device__ __forceinline__ void soa_fill(const float4 *src, float *soa, int n_s, int S) {
    const int n32 = (n_s + 31) & ~31;
    for (int b = threadIdx.x; b < n32; b += blockDim.x) {
        const float4 q = b < n_s ? src[b] : make_float4(0.f, 0.f, 0.f, 0.f);
        soa[b] = q.x;
        soa[S + b] = q.y;
        soa[2 * S + b] = q.z;
    }
}

// One block of 32 candidates base .. base + 31 of the all-pairs scan (Algorithm 3): bit t of
// .y is set when the FP32 squared distance to candidate base + t is below hi (the cutoff plus
// its guard band), bit t of .x when it is below lo (the cutoff minus the band): those are
// inside whatever the rounding; the bits of .y alone are decided exactly by within_cut (FP64
// inside the band). Candidates are taken in pairs from the x, y, z arrays, in packed FP32x2
// arithmetic. Bits at or beyond lim are cleared.
__device__ __forceinline__ uint2 scan_block(const float *soa, int S, int base, int lim, float4 pb, float lo,
                                            float hi) {
    const float2 *X = reinterpret_cast<const float2 *>(soa + base);
    const float2 *Y = reinterpret_cast<const float2 *>(soa + S + base);
    const float2 *Z = reinterpret_cast<const float2 *>(soa + 2 * S + base);
    const float2 px = make_float2(pb.x, pb.x), py = make_float2(pb.y, pb.y), pz = make_float2(pb.z, pb.z);
    const float2 m1 = make_float2(-1.f, -1.f);
    uint32_t wl = 0u, wh = 0u;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const float2 dx = __ffma2_rn(X[t], m1, px);   // pb - pj, exactly rounded
        const float2 dy = __ffma2_rn(Y[t], m1, py);
        const float2 dz = __ffma2_rn(Z[t], m1, pz);
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        wh |= (r2.x < hi ? 1u : 0u) << (2 * t);
        wh |= (r2.y < hi ? 1u : 0u) << (2 * t + 1);
        wl |= (r2.x < lo ? 1u : 0u) << (2 * t);
        wl |= (r2.y < lo ? 1u : 0u) << (2 * t + 1);
    }
    const uint32_t m = lim >= 32 ? 0xffffffffu : ((1u << lim) - 1u);
    return make_uint2(wl & m, wh & m);
}

// Verlet partners of bead b (at pb) among the candidates of one block: the candidates inside
// the cutoff (`cand`, from scan_block) that are not excluded, the guard band decided in FP64.
__device__ __forceinline__ uint32_t block_partners(uint2 cand, uint32_t ex_mask, const float4 *src, int base,
                                                  float4 pb, float cut2_f, double cut2_d) {
    uint32_t within = cand.x & ~ex_mask;
    uint32_t band = cand.y & ~cand.x & ~ex_mask;
    while (band) {   // rare
        const int t = __ffs(band) - 1;
        band &= band - 1;
        if (within_cut(pb, src[base + t], cut2_f, cut2_d)) within |= 1u << t;
    }
    return within;
}

// Cantilever / indenter force on replica-local bead i.
__device__ __forceinline__ float3 ext_force(const StepArgs &sa, int r, int i, uint8_t flags, float4 pi, int64_t step,
                                            bool *overlap) {
    float3 f = make_float3(0.f, 0.f, 0.f);
    const DevExternal &e = sa.ext;
    if (flags & kFlagPulled) {
        const int q = e.pull_of_sys[sa.topo.sys[i]];
        if (q >= 0 && e.pull_bead[q] == i) {
            const double tt = e.pull_v[q] * ((double)step - e.pull_n0[q]);
            const double *tip0 = e.pull_tip0 + ((size_t)r * e.n_pull + q) * 3;
            const float ks = (float)e.pull_ks[q];
            f.x = ks * (float)(tip0[0] + tt * e.pull_dir[3 * q] - (double)pi.x);
            f.y = ks * (float)(tip0[1] + tt * e.pull_dir[3 * q + 1] - (double)pi.y);
            f.z = ks * (float)(tip0[2] + tt * e.pull_dir[3 * q + 2] - (double)pi.z);
        }
    }
    if (e.has_indenter) {
        const double tt = e.ind_v * ((double)step - e.ind_n0);
        const float ex = pi.x - (float)(e.ind_c0[0] + tt * e.ind_dir[0]);
        const float ey = pi.y - (float)(e.ind_c0[1] + tt * e.ind_dir[1]);
        const float ez = pi.z - (float)(e.ind_c0[2] + tt * e.ind_dir[2]);
        const float rr = sqrtf(fmaf(ez, ez, fmaf(ey, ey, ex * ex)));
        const float rho = rr - (float)e.ind_radius;
        if (!(rho > 0.f)) {
            *overlap = true;
        } else {
            const float q = sqrtf(sa.fp.sigma2) / rho;
            const float q2 = q * q;
            const float c = sa.fp.eps6_l * (q2 * q2 * q2) / (rho * rr);
            f.x = fmaf(c, ex, f.x); f.y = fmaf(c, ey, f.y); f.z = fmaf(c, ez, f.z);
        }
    }
    return f;
}

// Records of the cadence events after `step` to the end of the chunk that this CTA will not
// take (frozen replica): step, replica and system are set, the values are NaN.
__device__ void missing_records(const BatchedArgs &a, int r, int s, int g, int64_t step0, int64_t step,
                                int64_t event) {
    if (a.obs_every <= 0) return;
    const int64_t end = step0 + a.n_steps;
    for (int64_t t = (step / a.obs_every + 1) * a.obs_every; t <= end; t += a.obs_every) {
        sop_record rec;
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        rec.step = (double)t;
        rec.replica = (double)r;
        rec.system = (double)s;
        rec.energy = rec.f_ext = rec.extension = rec.q = rec.r_ee = nan;
        a.obs.ring[(event * a.n_seg + g) % a.obs.cap] = rec;
        ++event;
    }
}

// Sum of the Eq. 1 pair forces on a bead at pb over its merged row: entries 0 .. nn-1 are
// native partners (12-6 with r0^2 from natr, stride nat_stride), entries nn .. tot-1
// Verlet partners ((sigma/r)^6); entry k at row[k * row_stride]. Two loops walking
// pointers, so that no entry pays for a select or an index multiply.
__device__ __forceinline__ float3 row_force(const float4 *P, float4 pb, const uint16_t *row, const float *natr,
                                            int nn, int tot, int row_stride, int nat_stride, const ForceParams &fp,
                                            float3 acc = make_float3(0.f, 0.f, 0.f)) {
    float fx = acc.x, fy = acc.y, fz = acc.z;   // the sum continues from acc
    const float A = fp.eps12_h, K = fp.rep_k;
    int k = 0;
#pragma unroll 2
    for (; k < nn; ++k) {
        const int j = *row;
        row += row_stride;
        const float s0 = __ldg(natr);
        natr += nat_stride;
        const float4 pj = P[j];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float inv = __fdividef(1.0f, r2);
        const float s = s0 * inv;
        const float s3 = s * s * s;
        const float c = inv * s3 * fmaf(A, s3, -A);   // (12 eps_h / r^2)(s^6 - s^3), s = r0^2 / r^2
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
#pragma unroll 2
    for (; k < tot; ++k) {
        const int j = *row;
        row += row_stride;
        const float4 pj = P[j];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float inv = __fdividef(1.0f, r2);
        const float i2 = inv * inv;
        const float c = K * (i2 * i2);                  // 6 eps_l sigma^6 / r^8
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    return make_float3(fx, fy, fz);
}

// FP64 observable sums of system-local bead b (replica-local index b0 + b) at layer P that
// do not depend on the Verlet rows: the FENE energy of the bond (b, b + 1) when it exists,
// and the native energy and formed contacts over the native pairs (i, j > i) (Eq. 1; Q).
__device__ __forceinline__ void obs_bonded(const StepArgs &sa, const float4 *P, int b, int b0, bool bond_right,
                                           double v[6]) {
    const DevTopo &t = sa.topo;
    const int i = b0 + b;
    const float4 pb = P[b];
    const double R02 = sa.R0 * sa.R0;
    if (bond_right) {
        const float4 pj = P[b + 1];
        float d2f;
        const double d2 = dist2_two(pb, pj, &d2f);
        const double rr = sqrt_seeded(d2, d2f);
        const double dr = rr - t.bond_r0d[i];
        const double arg = 1.0 - dr * dr / R02;
        if (arg > 0.0) v[0] += -0.5 * sa.k_fene * R02 * log(arg);
    }
    for (int q = t.nat_row[i]; q < t.nat_row[i + 1]; ++q) {
        const int j = t.nat_col[q];
        if (j < i) continue;
        const float4 pj = P[j - b0];
        float d2f;
        const double d2 = dist2_two(pb, pj, &d2f);
        const double r0 = t.nat_r0[q];
        const double u = r0 * r0 * rcp_seeded(d2, d2f);
        const double u3 = u * u * u;
        v[0] = fma(sa.eps_h, u3 * u3 - 2.0 * u3, v[0]);
        if (native_formed(d2, r0, pb, pj)) v[3] += 1.0;
    }
}

// FP64 readouts of bead b of replica r, system s at `step` (Sec. IV.B): the spring force along
// the pulling direction and the anchor-to-pulled distance when b is the pulled bead, the
// indenter's force along its direction of travel, and the end-to-end distance of the
// system's first chain from its first bead.
__device__ __forceinline__ void obs_external(const StepArgs &sa, const float4 *P, int b, int b0, int r, int s,
                                             int64_t step, uint8_t fl, double v[6]) {
    const DevTopo &t = sa.topo;
    const DevExternal &e = sa.ext;
    const int i = b0 + b;
    const float4 pb = P[b];
    const double xi = pb.x, yi = pb.y, zi = pb.z;
    if (fl & kFlagPulled) {
        const int qq = e.pull_of_sys[s];
        if (qq >= 0 && e.pull_bead[qq] == i) {
            const double tt = e.pull_v[qq] * ((double)step - e.pull_n0[qq]);
            const double *tip0 = e.pull_tip0 + ((size_t)r * e.n_pull + qq) * 3;
            const double *dir = e.pull_dir + 3 * qq;
            const double x[3] = {xi, yi, zi};
            double f = 0.0;
            for (int c = 0; c < 3; ++c) f += e.pull_ks[qq] * (tip0[c] + tt * dir[c] - x[c]) * dir[c];
            v[1] += f;
            const float4 pa = P[e.pull_anchor[qq] - b0];
            v[2] += __dsqrt_rn(dist2_d(xi, yi, zi, pa.x, pa.y, pa.z));
        }
    }
    if (e.has_indenter) {
        const double tt = e.ind_v * ((double)step - e.ind_n0);
        const double c[3] = {e.ind_c0[0] + tt * e.ind_dir[0], e.ind_c0[1] + tt * e.ind_dir[1],
                             e.ind_c0[2] + tt * e.ind_dir[2]};
        const double ex = xi - c[0], ey = yi - c[1], ez = zi - c[2];
        const double rr = sqrt_fast((ex * ex + ey * ey) + ez * ez);
        const double rho = rr - e.ind_radius;
        if (rho > 0.0) {
            const double qq = sa.sigma * rcp_fast(rho);
            const double q2 = qq * qq;
            const double coef = 6.0 * sa.eps_l * (q2 * q2 * q2) * rcp_fast(rho * rr);
            v[4] += coef * ((ex * e.ind_dir[0] + ey * e.ind_dir[1]) + ez * e.ind_dir[2]);
        }
    }
    if (fl & kFlagFirstOfSystem) {
        const float4 pl_ = P[t.sys_ree_last[s] - b0];
        v[5] += __dsqrt_rn(dist2_d(xi, yi, zi, pl_.x, pl_.y, pl_.z));
    }
}

// Write the observable record of (replica r, system s) at `step` from the CTA sums v (E,
// f_pull, extension, formed natives, f_wall, r_ee), valid in thread 0.
__device__ __forceinline__ void write_record(const BatchedArgs &a, const double v[6], int r, int s, int g,
                                             int64_t step, int64_t event) {
    const DevTopo &t = a.sa.topo;
    const DevExternal &e = a.sa.ext;
    sop_record rec;
    rec.step = (double)step;
    rec.replica = (double)r;
    rec.system = (double)s;
    rec.energy = v[0];
    const bool pulled = e.pull_of_sys[s] >= 0;
    rec.f_ext = pulled ? v[1] : (e.has_indenter ? v[4] : 0.0);
    rec.extension = pulled ? v[2] : (e.has_indenter ? e.ind_v * ((double)step - e.ind_n0) : 0.0);
    const int np = t.sys_nat_pairs[s];
    rec.q = np > 0 ? v[3] / (double)np : 0.0;
    if (a.obs.q_every > 0 && step % a.obs.q_every != 0) rec.q = __longlong_as_double(0x7ff8000000000000LL);
    rec.r_ee = v[5];
    a.obs.ring[(event * a.n_seg + g) % a.obs.cap] = rec;
}

}  // namespace
}  // namespace sop
