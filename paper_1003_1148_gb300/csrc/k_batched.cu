// Batched schedule: one persistent fused kernel for many small systems (sm_103a).
//
// One CTA owns one work item (a system of one replica) for a whole chunk of
// steps. The two time layers of positions (Algorithm 7), the compensation
// terms, bond lengths and the neighbour rows live in shared memory; thread t
// owns beads t, t + T, ... (BPT of them). Per step a thread gathers the Eq. 1
// forces of its beads (particle-based, Algorithm 2) over one merged row per
// bead -- its native partners first, then its Verlet partners -- so that one
// loop of nearly equal length per lane covers both pair terms. It adds the
// cantilever/indenter force, draws Philox noise and applies the compensated
// first-order update into the other layer; one __syncthreads() separates steps.
//
// Rows are column-major (entry k of bead b at k*n + b: a warp reads
// consecutive 16-bit words). Every K steps the Verlet part of the rows is
// rebuilt from the current layer by an all-pairs scan of the system
// (Algorithm 3 with the whole system as candidate set): for 32 candidates at
// a time each thread forms a bit mask of "closer than the cutoff", clears the
// bits of itself, its bonded neighbours and its native partners, and appends
// the remaining bits in ascending order. Every thread of a warp reads the
// same candidate at the same time (a shared-memory broadcast). The natives'
// r0^2 come from a column-major table in global memory that all replicas of a
// system share (L1/L2 resident). Observables (FP64) are reduced in the CTA.
#include <cuda_runtime.h>

#include "sop_internal.h"

namespace sop {

namespace {

constexpr int kMaxThreads = 256;

struct SharedHead {
    int fail;   // first sop_status raised in this CTA
    double red[kMaxThreads / 32][6];
};

// The arrays follow the head at a 16-byte aligned offset (float4 accesses).
constexpr size_t kHeadBytes = (sizeof(SharedHead) + 15) / 16 * 16;

__device__ __forceinline__ void cta_fail(SharedHead *h, int code) { atomicCAS(&h->fail, 0, code); }

// Shared-memory layout of one work item, for systems of at most max_n beads.
struct Layout {
    SharedHead *h;
    float4 *lay[2];       // positions, two time layers
    float4 *comp;         // Kahan compensation (w unused)
    float2 *bond;         // (r0 of bond b-1,b ; r0 of bond b,b+1), < 0 when absent
    uint16_t *n_nat;      // native partners of each bead
    uint16_t *n_tot;      // natives + Verlet partners
    uint8_t *flags;
    uint16_t *row;        // merged rows, entry k of bead b at row[k * n + b]
};

__host__ __device__ inline size_t layout_bytes(int max_n, int row_width) {
    size_t s = kHeadBytes;
    s += 3 * sizeof(float4) * (size_t)max_n;   // two layers + compensation
    s += sizeof(float2) * (size_t)max_n;       // bond lengths
    s += 2 * sizeof(uint16_t) * (size_t)max_n; // counts
    s += (size_t)max_n;                        // flags
    s = (s + 15) / 16 * 16;
    s += sizeof(uint16_t) * (size_t)row_width * max_n;
    return s;
}

__device__ inline Layout make_layout(unsigned char *smem, int max_n) {
    Layout L;
    L.h = reinterpret_cast<SharedHead *>(smem);
    float4 *f4 = reinterpret_cast<float4 *>(smem + kHeadBytes);
    L.lay[0] = f4;
    L.lay[1] = f4 + max_n;
    L.comp = f4 + 2 * max_n;
    L.bond = reinterpret_cast<float2 *>(f4 + 3 * max_n);
    L.n_nat = reinterpret_cast<uint16_t *>(L.bond + max_n);
    L.n_tot = L.n_nat + max_n;
    L.flags = reinterpret_cast<uint8_t *>(L.n_tot + max_n);
    size_t off = (size_t)(reinterpret_cast<unsigned char *>(L.flags + max_n) - smem);
    off = (off + 15) / 16 * 16;
    L.row = reinterpret_cast<uint16_t *>(smem + off);
    return L;
}

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

// Verlet part of the rows of the thread's beads from layer src (all-pairs scan).
template <int BPT>
__device__ void rebuild_rows(const BatchedArgs &a, const Layout &L, const float4 *src, int n_s, int nat_off) {
    const int T = blockDim.x;
    const float cut2 = a.sa.cut2_f;
    const float band = cut2 * 1e-4f;
#pragma unroll 1
    for (int k = 0; k < BPT; ++k) {
        const int b = threadIdx.x + k * T;
        if (b >= n_s) continue;
        const float4 pb = src[b];
        const int nn = L.n_nat[b];
        const uint16_t *natc = a.nat_ell_col + nat_off + b;
        const float2 bd = L.bond[b];
        int q = 0;                                  // next native to exclude
        int next_nat = nn > 0 ? (int)__ldg(natc) : 0x7fffffff;
        int cnt = 0;
        for (int base = 0; base < n_s; base += 32) {
            const int lim = min(32, n_s - base);
            uint32_t within = 0u, near = 0u;
#pragma unroll 8
            for (int t = 0; t < lim; ++t) {
                const float4 pj = src[base + t];
                const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                within |= (uint32_t)(r2 < cut2 - band) << t;
                near |= (uint32_t)(fabsf(r2 - cut2) <= band) << t;
            }
            // exclusions in [base, base + 32): self, bonded neighbours, native partners
            uint32_t ex = 0u;
            if (b >= base && b < base + 32) ex |= 1u << (b - base);
            if (bd.x > 0.f && b - 1 >= base && b - 1 < base + 32) ex |= 1u << (b - 1 - base);
            if (bd.y > 0.f && b + 1 >= base && b + 1 < base + 32) ex |= 1u << (b + 1 - base);
            while (next_nat < base + 32) {
                ex |= 1u << (next_nat - base);
                ++q;
                next_nat = q < nn ? (int)__ldg(natc + (size_t)q * n_s) : 0x7fffffff;
            }
            within &= ~ex;
            near &= ~ex;
            while (near) {   // rare: decide within the guard band in FP64
                const int t = __ffs(near) - 1;
                near &= near - 1;
                if (within_cut(pb, src[base + t], cut2, a.sa.cut2_d)) within |= 1u << t;
            }
            while (within) {
                const int t = __ffs(within) - 1;
                within &= within - 1;
                if (cnt < a.cap) L.row[(size_t)(nn + cnt) * n_s + b] = (uint16_t)(base + t);
                ++cnt;
            }
        }
        if (cnt > a.cap) cta_fail(L.h, SOP_ERR_PAIRLIST_OVERFLOW);
        L.n_tot[b] = (uint16_t)(nn + min(cnt, a.cap));
    }
}

// Sum of the Eq. 1 pair forces on bead b at layer P over its bonds and merged row.
// Entries k < n_nat are native (12-6 with r0^2 from the table), the rest repulsive.
__device__ __forceinline__ float3 bead_force(const BatchedArgs &a, const Layout &L, const float4 *P, int n_s,
                                             int nat_off, int b, bool *broken) {
    const ForceParams &fp = a.sa.fp;
    const float4 pb = P[b];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const float2 bd = L.bond[b];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const float r0 = side ? bd.y : bd.x;
        if (r0 > 0.f) {
            const float4 pj = P[side ? b + 1 : b - 1];
            const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float r = r2 * rsqrtf(r2);
            const float dr = r - r0;
            const float arg = fmaf(-dr * dr, fp.inv_R02, 1.0f);
            float c = 0.f;
            if (arg > 0.f) c = __fdividef(-fp.k_fene * dr, arg * r);
            else *broken = true;
            fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
        }
    }
    const int nn = L.n_nat[b], tot = L.n_tot[b];
    const float *natr = a.nat_ell_r0sq + nat_off + b;
    const float A = fp.eps12_h, B = fp.eps6_l;
#pragma unroll 2
    for (int k = 0; k < tot; ++k) {
        const bool nat = k < nn;
        const int j = L.row[(size_t)k * n_s + b];
        const float s0 = nat ? __ldg(natr + (size_t)k * n_s) : fp.sigma2;
        const float4 pj = P[j];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float inv = __fdividef(1.0f, r2);
        const float s = s0 * inv;
        const float s3 = s * s * s;
        // native: (12 eps_h / r^2)(s^6 - s^3); repulsive: (6 eps_l / r^2) s^3 with s = sigma^2/r^2
        const float c = inv * s3 * (nat ? fmaf(A, s3, -A) : B);
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    return make_float3(fx, fy, fz);
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

// FP64 observables of the CTA's system at layer P (same definitions as the streamed kernels).
template <int BPT>
__device__ __noinline__ void observe(const BatchedArgs &a, const Layout &L, const float4 *P, int n_s, int b0, int r,
                                     int s, int g, int64_t step, int64_t event) {
    const StepArgs &sa = a.sa;
    const DevTopo &t = sa.topo;
    const DevExternal &e = sa.ext;
    const int T = blockDim.x;
    double v[6] = {0, 0, 0, 0, 0, 0};   // E, f_pull, ext, formed, f_wall, r_ee
    const double R02 = sa.R0 * sa.R0, sig2 = sa.sigma * sa.sigma;
    for (int k = 0; k < BPT; ++k) {
        const int b = threadIdx.x + k * T;
        if (b >= n_s) continue;
        const int i = b0 + b;
        const float4 pb = P[b];
        const double xi = pb.x, yi = pb.y, zi = pb.z;
        if (L.bond[b].y > 0.f) {
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
        for (int q = L.n_nat[b]; q < L.n_tot[b]; ++q) {
            const int j = L.row[(size_t)q * n_s + b];
            if (j < b) continue;
            const float4 pj = P[j];
            const double c = sig2 / dist2_d(xi, yi, zi, pj.x, pj.y, pj.z);
            v[0] += sa.eps_l * c * c * c;
        }
        const uint8_t fl = L.flags[b];
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
            const double rr = __dsqrt_rn((ex * ex + ey * ey) + ez * ez);
            const double rho = rr - e.ind_radius;
            if (rho > 0.0) {
                const double qq = sa.sigma / rho;
                const double q2 = qq * qq;
                const double coef = 6.0 * sa.eps_l * (q2 * q2 * q2) / rho / rr;
                v[4] += coef * ((ex * e.ind_dir[0] + ey * e.ind_dir[1]) + ez * e.ind_dir[2]);
            }
        }
        if (fl & kFlagFirstOfSystem) {
            const float4 pl_ = P[t.sys_ree_last[s] - b0];
            v[5] += __dsqrt_rn(dist2_d(xi, yi, zi, pl_.x, pl_.y, pl_.z));
        }
    }
    block_sum6(v, L.h);
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

// MINB: CTAs of kMaxThreads threads that must fit an SM, i.e. the register cap
// 65536 / (kMaxThreads * MINB): 2 -> 128, 3 -> 85, 4 -> 64 registers per thread.
template <int BPT, int MINB>
__global__ void __launch_bounds__(kMaxThreads, MINB) k_batched(BatchedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Layout L = make_layout(smem, a.max_n);
    const int item = blockIdx.x;
    const int r = a.item_rep[item], s = a.item_sys[item];
    const StepArgs &sa = a.sa;
    const DevTopo &t = sa.topo;
    const int b0 = t.sys_lo[s], n_s = t.sys_lo[s + 1] - b0;
    const int n = t.n;
    const size_t gbase = (size_t)r * n + b0;
    const int g = r * t.n_sys + s;
    const int nat_off = a.nat_ell_off[s];
    const int T = blockDim.x;
    const int64_t step0 = *a.d_step;
    const int64_t event0 = a.d_events ? *a.d_events : 0;
    const bool forces_only = (a.n_steps == 0 && a.force_out != nullptr);

    if (threadIdx.x == 0) L.h->fail = 0;
    if (!forces_only && (sa.rep_status[r] != 0 || *sa.halt != 0)) {   // CTA-uniform: a frozen replica
        if (threadIdx.x == 0) missing_records(a, r, s, g, step0, step0, event0);        // only marks its records
        return;
    }
    // load the item: positions, compensation, bonds, flags, native part of the rows
    for (int b = threadIdx.x; b < n_s; b += T) {
        const int i = b0 + b;
        L.lay[0][b] = a.pos[gbase + b];
        L.comp[b] = a.comp[gbase + b];
        L.bond[b] = make_float2(b > 0 ? t.bond_r0[i - 1] : -1.f, t.bond_r0[i]);
        L.flags[b] = t.flags[i];
        const int nn = a.nat_ell_cnt[i];
        L.n_nat[b] = (uint16_t)nn;
        L.n_tot[b] = (uint16_t)nn;
        for (int k = 0; k < nn; ++k)
            L.row[(size_t)k * n_s + b] = a.nat_ell_col[nat_off + (size_t)k * n_s + b];
        // the list of the first step comes from the positions at the last rebuild step
        if (step0 % a.K != 0) L.lay[1][b] = a.snap[gbase + b];
    }
    __syncthreads();

    int cur = 0;
    int64_t step = step0;
    int64_t list_step = -1;
    int64_t event = event0;
    for (int it = 0; it < a.n_steps || (forces_only && it == 0); ++it) {
        const float4 *P = L.lay[cur];
        float4 *Q = L.lay[cur ^ 1];
        if (it == 0 && step % a.K != 0 && !forces_only) {
            rebuild_rows<BPT>(a, L, Q, n_s, nat_off);   // Q holds the snapshot here
            list_step = step;
            __syncthreads();
        } else if ((step % a.K == 0 && list_step != step) || forces_only) {
            rebuild_rows<BPT>(a, L, P, n_s, nat_off);
            list_step = step;
            if (!forces_only)
                for (int b = threadIdx.x; b < n_s; b += T) a.snap[gbase + b] = P[b];
            __syncthreads();
        }
        if (forces_only) {
            for (int b = threadIdx.x; b < n_s; b += T) {
                bool broken = false, overlap = false;
                const float3 f = bead_force(a, L, P, n_s, nat_off, b, &broken);
                const float3 fe = ext_force(sa, r, b0 + b, L.flags[b], P[b], step, &overlap);
                a.force_out[gbase + b] = make_float4(f.x + fe.x, f.y + fe.y, f.z + fe.z, (broken || overlap) ? 1.f : 0.f);
                if (a.pl_dump_col) {
                    const size_t rowi = gbase + b;
                    const int nn = L.n_nat[b], np = L.n_tot[b] - nn;
                    a.pl_dump_start[rowi] = (int)(rowi * a.pl_dump_stride);
                    a.pl_dump_len[rowi] = np;
                    for (int q = 0; q < np; ++q)
                        a.pl_dump_col[rowi * a.pl_dump_stride + q] = b0 + (int)L.row[(size_t)(nn + q) * n_s + b];
                }
            }
            break;
        }
#pragma unroll 1
        for (int k = 0; k < BPT; ++k) {
            const int b = threadIdx.x + k * T;
            if (b >= n_s) continue;
            bool broken = false, overlap = false;
            const float3 f = bead_force(a, L, P, n_s, nat_off, b, &broken);
            const float4 p_old = P[b];
            const uint8_t fl = L.flags[b];
            const float3 fe = ext_force(sa, r, b0 + b, fl, p_old, step, &overlap);
            float4 pb = p_old;
            if (broken || overlap) {
                // a bead whose force cannot be evaluated stays where it is; the replica freezes
                cta_fail(L.h, broken ? SOP_ERR_FENE_BREAK : SOP_ERR_INDENTER_OVERLAP);
            } else if (!(fl & kFlagFixed)) {
                const float3 gn = bead_noise(sa.seed + (uint64_t)r, step, (uint32_t)(b0 + b));
                float4 c = L.comp[b];
                kahan_add(pb.x, c.x, fmaf(f.x + fe.x, sa.fp.mob, gn.x * sa.fp.amp));
                kahan_add(pb.y, c.y, fmaf(f.y + fe.y, sa.fp.mob, gn.y * sa.fp.amp));
                kahan_add(pb.z, c.z, fmaf(f.z + fe.z, sa.fp.mob, gn.z * sa.fp.amp));
                if (isfinite(pb.x) && isfinite(pb.y) && isfinite(pb.z)) {
                    L.comp[b] = c;
                } else {
                    cta_fail(L.h, SOP_ERR_NONFINITE);
                    pb = p_old;
                }
            }
            Q[b] = pb;
        }
        __syncthreads();
        cur ^= 1;
        ++step;
        if (L.h->fail != 0) break;   // the replica freezes after the step in which it failed
        if (a.obs_every > 0 && step % a.obs_every == 0) {
            const float4 *Pn = L.lay[cur];
            if (step % a.K == 0) {
                rebuild_rows<BPT>(a, L, Pn, n_s, nat_off);
                list_step = step;
                for (int b = threadIdx.x; b < n_s; b += T) a.snap[gbase + b] = Pn[b];
                __syncthreads();
            }
            observe<BPT>(a, L, Pn, n_s, b0, r, s, g, step, event);
            ++event;
        }
    }
    if (forces_only) return;
    if (threadIdx.x == 0 && L.h->fail != 0) missing_records(a, r, s, g, step0, step, event);
    const float4 *P = L.lay[cur];
    for (int b = threadIdx.x; b < n_s; b += T) {
        a.pos[gbase + b] = P[b];
        a.comp[gbase + b] = L.comp[b];
    }
    if (threadIdx.x == 0 && L.h->fail != 0) atomicCAS(&sa.rep_status[r], 0, L.h->fail);
}

template <int BPT, int MINB>
cudaError_t launch_t(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s) {
    auto kern = k_batched<BPT, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    kern<<<a.n_items, cfg.threads, cfg.smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

int batched_max_threads() { return kMaxThreads; }

bool batched_config(int max_n, int row_width, int threads_hint, BatchedConfig *cfg) {
    if (max_n <= 0 || max_n > 65535) return false;
    int threads = threads_hint > 0 ? threads_hint : 0;
    if (threads == 0) {
        threads = ((max_n + 31) / 32) * 32;
        if (threads > 256) threads = 256;
        if (threads < 64) threads = 64;
    }
    if (threads > kMaxThreads || threads % 32) return false;
    const int bpt = (max_n + threads - 1) / threads;
    if (bpt > 8) return false;
    cfg->threads = threads;
    cfg->beads_per_thread = bpt <= 1 ? 1 : bpt <= 2 ? 2 : bpt <= 4 ? 4 : 8;
    cfg->smem = layout_bytes(max_n, row_width);
    return cfg->smem <= 227 * 1024;
}

template <int BPT>
cudaError_t launch_b(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s) {
    switch (cfg.min_blocks) {
    case 2: return launch_t<BPT, 2>(a, cfg, s);
    case 3: return launch_t<BPT, 3>(a, cfg, s);
    default: return launch_t<BPT, 4>(a, cfg, s);
    }
}

cudaError_t launch_batched(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s, int64_t *launches) {
    if (a.n_items <= 0) return cudaSuccess;
    if (launches) *launches += 1;
    switch (cfg.beads_per_thread) {
    case 1: return launch_b<1>(a, cfg, s);
    case 2: return launch_b<2>(a, cfg, s);
    case 4: return launch_b<4>(a, cfg, s);
    default: return launch_b<8>(a, cfg, s);
    }
}

}  // namespace sop
