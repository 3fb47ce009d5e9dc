// Batched schedule: one persistent fused kernel for many small systems (sm_103a).
//
// One CTA owns one work item (a system of one replica) for a whole chunk of
// steps. Its positions (two time layers, as in Algorithm 7) and its Verlet
// list live in shared memory; each thread owns up to BPT beads and keeps their
// compensation terms and bond lengths in registers. Per step a thread gathers
// the Eq. 1 forces of its beads (particle-based, Algorithm 2), adds the
// cantilever/indenter force, draws Philox noise and applies the compensated
// first-order update into the other time layer; one __syncthreads() separates
// steps. Every K steps the list is rebuilt in shared memory by an all-pairs
// scan of the system (Algorithm 3 with the whole system as candidate set),
// kept in a column-major ELL layout (entry k of bead b at k*n + b) so that a
// warp reads consecutive addresses. Natives come from a column-major table in
// global memory that all replicas of a system share (L1/L2 resident).
// Observables (FP64) are reduced inside the CTA at their cadence.
#include <cuda_runtime.h>

#include "sop_internal.h"

namespace sop {

namespace {

constexpr int kMaxThreads = 512;

struct SharedHead {
    int fail;          // first sop_status raised in this CTA
    double red[kMaxThreads / 32][6];
};

// The position layers follow the head at a 16-byte aligned offset (float4 accesses).
constexpr size_t kHeadBytes = (sizeof(SharedHead) + 15) / 16 * 16;

__device__ __forceinline__ void cta_fail(SharedHead *h, int code) { atomicCAS(&h->fail, 0, code); }

// FP64 block sum of 6 values; result valid in thread 0.
__device__ __forceinline__ void block_sum6(double v[6], SharedHead *h) {
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

template <int BPT>
struct Owned {
    float4 c[BPT];        // Kahan compensation
    float r0_prev[BPT];   // bond (b-1, b) length or < 0
    float r0_next[BPT];   // bond (b, b+1) length or < 0
    int npl[BPT];         // Verlet entries
    int nnat[BPT];        // native entries
    uint8_t flags[BPT];
};

// All-pairs Verlet rebuild of the system in shared memory from layer src.
template <int BPT>
__device__ void rebuild_list(const BatchedArgs &a, const float4 *src, uint16_t *pl, int n_s, int nat_off, int b0,
                             Owned<BPT> &o, SharedHead *h) {
    const int T = blockDim.x;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
        const int b = threadIdx.x + k * T;
        if (b >= n_s) continue;
        const float4 pb = src[b];
        const uint16_t *natc = a.nat_ell_col + nat_off + b;
        int nk = 0;
        int next_nat = o.nnat[k] > 0 ? (int)natc[0] : 0x7fffffff;
        int cnt = 0;
        for (int j = 0; j < n_s; ++j) {
            while (next_nat < j) {
                ++nk;
                next_nat = nk < o.nnat[k] ? (int)natc[(size_t)nk * n_s] : 0x7fffffff;
            }
            if (j == b || j == next_nat) continue;
            if ((j == b + 1 && o.r0_next[k] > 0.f) || (j == b - 1 && o.r0_prev[k] > 0.f)) continue;
            if (within_cut(pb, src[j], a.sa.cut2_f, a.sa.cut2_d)) {
                if (cnt < a.cap) pl[cnt * n_s + b] = (uint16_t)j;
                ++cnt;
            }
        }
        if (cnt > a.cap) cta_fail(h, SOP_ERR_PAIRLIST_OVERFLOW);
        o.npl[k] = cnt < a.cap ? cnt : a.cap;
    }
    (void)b0;
}

template <int BPT>
__device__ __forceinline__ float3 bead_force(const BatchedArgs &a, const float4 *P, const uint16_t *pl, int n_s,
                                             int nat_off, int b, int k, const Owned<BPT> &o, bool *broken) {
    const ForceParams &fp = a.sa.fp;
    const float4 pb = P[b];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (o.r0_prev[k] > 0.f) {
        const float4 pj = P[b - 1];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float c = fene_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), o.r0_prev[k], fp, broken);
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    if (o.r0_next[k] > 0.f) {
        const float4 pj = P[b + 1];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float c = fene_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), o.r0_next[k], fp, broken);
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    const uint16_t *natc = a.nat_ell_col + nat_off + b;
    const float *natr = a.nat_ell_r0sq + nat_off + b;
    for (int q = 0; q < o.nnat[k]; ++q) {
        const int j = __ldg(natc + (size_t)q * n_s);
        const float r0sq = __ldg(natr + (size_t)q * n_s);
        const float4 pj = P[j];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float c = native_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), r0sq, fp);
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    for (int q = 0; q < o.npl[k]; ++q) {
        const float4 pj = P[pl[q * n_s + b]];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float c = repulsive_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), fp);
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    return make_float3(fx, fy, fz);
}

// Cantilever / indenter force on replica-local bead i (global layout of ext).
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

// FP64 observables of the CTA's system at layer P (same definitions as the streamed kernels).
template <int BPT>
__device__ void observe(const BatchedArgs &a, const float4 *P, const uint16_t *pl, int n_s, int b0, int r, int s,
                        int g, int64_t step, int64_t event, const Owned<BPT> &o, SharedHead *h) {
    const StepArgs &sa = a.sa;
    const DevTopo &t = sa.topo;
    const DevExternal &e = sa.ext;
    const int T = blockDim.x;
    double v[6] = {0, 0, 0, 0, 0, 0};   // E, f_pull, ext, formed, f_wall, r_ee
    const double R02 = sa.R0 * sa.R0, sig2 = sa.sigma * sa.sigma;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
        const int b = threadIdx.x + k * T;
        if (b >= n_s) continue;
        const int i = b0 + b;
        const float4 pb = P[b];
        const double xi = pb.x, yi = pb.y, zi = pb.z;
        if (o.r0_next[k] > 0.f) {
            const float4 pj = P[b + 1];
            const double rr = __dsqrt_rn(dist2_d(xi, yi, zi, pj.x, pj.y, pj.z));
            const double dr = rr - t.bond_r0d[i];
            const double arg = 1.0 - dr * dr / R02;
            if (arg > 0.0) v[0] += -0.5 * sa.k_fene * R02 * log(arg);
        }
        for (int p = t.nat_row[i]; p < t.nat_row[i + 1]; ++p) {
            const int j = t.nat_col[p];
            if (j < i) continue;
            const float4 pj = P[j - b0];
            const double d2 = dist2_d(xi, yi, zi, pj.x, pj.y, pj.z);
            const double r0 = t.nat_r0[p];
            const double q = r0 * r0 / d2;
            const double q3 = q * q * q;
            v[0] += sa.eps_h * (q3 * q3 - 2.0 * q3);
            if (__dsqrt_rn(d2) < r0 + 2.0) v[3] += 1.0;
        }
        for (int q = 0; q < o.npl[k]; ++q) {
            const int j = pl[q * n_s + b];
            if (j < b) continue;
            const float4 pj = P[j];
            const double c = sig2 / dist2_d(xi, yi, zi, pj.x, pj.y, pj.z);
            v[0] += sa.eps_l * c * c * c;
        }
        if (o.flags[k] & kFlagPulled) {
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
            const double rr = __dsqrt_rn((ex * ex + ey * ey) + ez * ez);
            const double rho = rr - e.ind_radius;
            if (rho > 0.0) {
                const double qq = sa.sigma / rho;
                const double q2 = qq * qq;
                const double coef = 6.0 * sa.eps_l * (q2 * q2 * q2) / rho / rr;
                v[4] += coef * ((ex * e.ind_dir[0] + ey * e.ind_dir[1]) + ez * e.ind_dir[2]);
            }
        }
        if (o.flags[k] & kFlagFirstOfSystem) {
            const float4 pl_ = P[t.sys_ree_last[s] - b0];
            v[5] += __dsqrt_rn(dist2_d(xi, yi, zi, pl_.x, pl_.y, pl_.z));
        }
    }
    block_sum6(v, h);
    if (threadIdx.x == 0) {
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
        rec.r_ee = v[5];
        a.obs.ring[(event * a.n_seg + g) % a.obs.cap] = rec;
    }
    __syncthreads();
}

// Records of the cadence events from `step` to the end of the chunk that this CTA will not
// take (frozen or stopped replica): step, replica and system are set, the values are NaN.
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

template <int BPT>
__global__ void __launch_bounds__(kMaxThreads) k_batched(BatchedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    SharedHead *h = reinterpret_cast<SharedHead *>(smem);
    const int item = blockIdx.x;
    const int r = a.item_rep[item], s = a.item_sys[item];
    const StepArgs &sa = a.sa;
    const DevTopo &t = sa.topo;
    const int b0 = t.sys_lo[s], n_s = t.sys_lo[s + 1] - b0;
    const int n = t.n;
    const size_t gbase = (size_t)r * n + b0;
    const int g = r * t.n_sys + s;
    float4 *lay0 = reinterpret_cast<float4 *>(smem + kHeadBytes);
    float4 *lay1 = lay0 + a.max_n;
    uint16_t *pl = reinterpret_cast<uint16_t *>(lay1 + a.max_n);
    const int nat_off = a.nat_ell_off[s];
    const int T = blockDim.x;

    if (threadIdx.x == 0) h->fail = 0;
    // the chunk starts at the device step counter; records continue the device event count
    const int64_t step0 = *a.d_step;
    const int64_t event0 = a.d_events ? *a.d_events : 0;
    const bool forces_only = (a.n_steps == 0 && a.force_out != nullptr);
    if (sa.rep_status[r] != 0 || *sa.halt != 0) {   // CTA-uniform: a frozen replica only marks its records
        if (!forces_only && threadIdx.x == 0) missing_records(a, r, s, g, step0, step0, event0);
        return;
    }

    Owned<BPT> o;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
        const int b = threadIdx.x + k * T;
        o.npl[k] = 0;
        o.nnat[k] = 0;
        o.flags[k] = 0;
        o.r0_prev[k] = -1.f;
        o.r0_next[k] = -1.f;
        o.c[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (b < n_s) {
            const int i = b0 + b;
            lay0[b] = a.pos[gbase + b];
            o.c[k] = a.comp[gbase + b];
            o.flags[k] = t.flags[i];
            o.r0_next[k] = t.bond_r0[i];
            o.r0_prev[k] = b > 0 ? t.bond_r0[i - 1] : -1.f;
            o.nnat[k] = a.nat_ell_cnt[i];
            // the list of the first step comes from the positions at the last rebuild step
            if (step0 % a.K != 0) lay1[b] = a.snap[gbase + b];
        }
    }
    __syncthreads();

    int cur = 0;
    int64_t step = step0;
    int64_t list_step = -1;
    int64_t event = event0;
    for (int it = 0; it < a.n_steps || (forces_only && it == 0); ++it) {
        float4 *P = cur ? lay1 : lay0;
        float4 *Q = cur ? lay0 : lay1;
        if (it == 0 && step % a.K != 0 && !forces_only) {
            rebuild_list<BPT>(a, Q, pl, n_s, nat_off, b0, o, h);   // Q holds the snapshot here
            list_step = step;
            __syncthreads();
        } else if (step % a.K == 0 && list_step != step || forces_only) {
            rebuild_list<BPT>(a, P, pl, n_s, nat_off, b0, o, h);
            list_step = step;
#pragma unroll
            for (int k = 0; k < BPT; ++k) {
                const int b = threadIdx.x + k * T;
                if (b < n_s && !forces_only) a.snap[gbase + b] = P[b];
            }
            __syncthreads();
        }
        if (forces_only) {
#pragma unroll
            for (int k = 0; k < BPT; ++k) {
                const int b = threadIdx.x + k * T;
                if (b >= n_s) continue;
                bool broken = false, overlap = false;
                const float3 f = bead_force<BPT>(a, P, pl, n_s, nat_off, b, k, o, &broken);
                const float3 fe = ext_force(sa, r, b0 + b, o.flags[k], P[b], step, &overlap);
                a.force_out[gbase + b] = make_float4(f.x + fe.x, f.y + fe.y, f.z + fe.z, (broken || overlap) ? 1.f : 0.f);
                if (a.pl_dump_col) {
                    const size_t row = gbase + b;
                    a.pl_dump_start[row] = (int)(row * a.pl_dump_stride);
                    a.pl_dump_len[row] = o.npl[k];
                    for (int q = 0; q < o.npl[k]; ++q)
                        a.pl_dump_col[row * a.pl_dump_stride + q] = b0 + (int)pl[q * n_s + b];
                }
            }
            break;
        }
#pragma unroll
        for (int k = 0; k < BPT; ++k) {
            const int b = threadIdx.x + k * T;
            if (b >= n_s) continue;
            bool broken = false, overlap = false;
            const float3 f = bead_force<BPT>(a, P, pl, n_s, nat_off, b, k, o, &broken);
            const float4 p_old = P[b];
            const float3 fe = ext_force(sa, r, b0 + b, o.flags[k], p_old, step, &overlap);
            float4 pb = p_old;
            if (broken || overlap) {
                // a bead whose force cannot be evaluated stays where it is; the replica freezes
                cta_fail(h, broken ? SOP_ERR_FENE_BREAK : SOP_ERR_INDENTER_OVERLAP);
            } else if (!(o.flags[k] & kFlagFixed)) {
                const float3 gn = bead_noise(sa.seed + (uint64_t)r, step, (uint32_t)(b0 + b));
                float4 c = o.c[k];
                kahan_add(pb.x, c.x, fmaf(f.x + fe.x, sa.fp.mob, gn.x * sa.fp.amp));
                kahan_add(pb.y, c.y, fmaf(f.y + fe.y, sa.fp.mob, gn.y * sa.fp.amp));
                kahan_add(pb.z, c.z, fmaf(f.z + fe.z, sa.fp.mob, gn.z * sa.fp.amp));
                if (isfinite(pb.x) && isfinite(pb.y) && isfinite(pb.z)) {
                    o.c[k] = c;
                } else {
                    cta_fail(h, SOP_ERR_NONFINITE);
                    pb = p_old;
                }
            }
            Q[b] = pb;
        }
        __syncthreads();
        cur ^= 1;
        ++step;
        if (h->fail != 0) break;   // the replica freezes after the step in which it failed
        if (a.obs_every > 0 && step % a.obs_every == 0) {
            float4 *Pn = cur ? lay1 : lay0;
            if (step % a.K == 0) {
                rebuild_list<BPT>(a, Pn, pl, n_s, nat_off, b0, o, h);
                list_step = step;
#pragma unroll
                for (int k = 0; k < BPT; ++k) {
                    const int b = threadIdx.x + k * T;
                    if (b < n_s) a.snap[gbase + b] = Pn[b];
                }
                __syncthreads();
            }
            observe<BPT>(a, Pn, pl, n_s, b0, r, s, g, step, event, o, h);
            ++event;
        }
    }
    if (forces_only) return;
    if (threadIdx.x == 0 && h->fail != 0) missing_records(a, r, s, g, step0, step, event);
    const float4 *P = cur ? lay1 : lay0;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
        const int b = threadIdx.x + k * T;
        if (b >= n_s) continue;
        a.pos[gbase + b] = P[b];
        a.comp[gbase + b] = o.c[k];
    }
    if (threadIdx.x == 0 && h->fail != 0) atomicCAS(&sa.rep_status[r], 0, h->fail);
}

template <int BPT>
cudaError_t launch_t(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s) {
    auto kern = k_batched<BPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    kern<<<a.n_items, cfg.threads, cfg.smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool batched_config(int max_n, int cap, int threads_hint, BatchedConfig *cfg) {
    if (max_n <= 0 || max_n > 65535) return false;
    int threads = threads_hint > 0 ? threads_hint : 0;
    if (threads == 0) {
        threads = ((max_n + 31) / 32) * 32;
        if (threads > 256) threads = 256;
        if (threads < 64) threads = 64;
    }
    const int bpt = (max_n + threads - 1) / threads;
    if (bpt > 8) return false;
    cfg->threads = threads;
    cfg->beads_per_thread = bpt <= 1 ? 1 : bpt <= 2 ? 2 : bpt <= 4 ? 4 : 8;
    cfg->smem = kHeadBytes + 2 * sizeof(float4) * (size_t)max_n + sizeof(uint16_t) * (size_t)cap * max_n;
    cfg->smem = (cfg->smem + 15) / 16 * 16;
    return cfg->smem <= 227 * 1024;
}

cudaError_t launch_batched(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s, int64_t *launches) {
    if (a.n_items <= 0) return cudaSuccess;
    if (launches) *launches += 1;
    switch (cfg.beads_per_thread) {
    case 1: return launch_t<1>(a, cfg, s);
    case 2: return launch_t<2>(a, cfg, s);
    case 4: return launch_t<4>(a, cfg, s);
    default: return launch_t<8>(a, cfg, s);
    }
}

}  // namespace sop
