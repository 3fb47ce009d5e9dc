// Batched schedule: one persistent fused kernel for many small systems (sm_103a).
//
// One CTA owns one work item (a system of one replica) for a whole chunk of
// steps. The two time layers of positions (Algorithm 7), the compensation
// terms and bond lengths live in shared memory, and so do the neighbour rows
// unless the system is too large (then each item's rows live in global
// memory, L2-resident). Per step a thread gathers the Eq. 1 forces of its
// beads (particle-based, Algorithm 2) over one merged row per bead -- its
// native partners first, then its Verlet partners -- adds the
// cantilever/indenter force, draws Philox noise and applies the compensated
// first-order update into the other layer; one __syncthreads() separates
// steps.
//
// Work balance. Threads own "slots" (slot p = thread + k * blockDim). At each
// Verlet rebuild the slots are handed to beads in order of decreasing row
// length of the previous build (a counting sort in shared memory), so that a
// warp holds beads with rows of similar length and its lanes finish their
// force loops together. The row of the bead in slot p is stored in column p
// (entry k at k*n + p): a warp reads consecutive 16-bit words. A bead's force
// is summed in its row's order whatever slot it lands in, so the assignment
// does not change any result.
//
// Rebuild (every K steps, Algorithm 3 with the whole system as candidate set):
// the beads are taken 32 at a time in index order; consecutive beads of a
// chain are close in space, so each block of 32 gets a bounding box and a
// thread skips every block whose box lies beyond the cutoff. Otherwise it
// tests the 32 candidates, forming a bit mask; clears itself, its bonded
// neighbours and its native partners; and appends the remaining bits in
// ascending order. All lanes of a warp read the same candidate (a
// shared-memory broadcast). The natives' r0^2 come from a column-major table
// in global memory shared by all replicas of a system. Observables (FP64) are
// reduced in the CTA.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "sop_internal.h"
#include "sop_step.cuh"

namespace cg = cooperative_groups;

namespace sop {

namespace {

constexpr int kKeys = 257;   // row lengths 0..256

struct SharedHead {
    int fail;               // first sop_status raised in this CTA
    int hist[kKeys];        // counting sort of slots by row length
    double red[32][6];      // FP64 block reductions (up to 1024 threads)
};

// The arrays follow the head at a 16-byte aligned offset (float4 accesses).
constexpr size_t kHeadBytes = (sizeof(SharedHead) + 15) / 16 * 16;

__device__ __forceinline__ void cta_fail(SharedHead *h, int code) { atomicCAS(&h->fail, 0, code); }

// Shared-memory layout of one work item, for systems of at most max_n beads. The
// accessors recompute each array's address from the dynamic shared-memory symbol, so
// that only a few integers stay live and every access is a 32-bit shared address.
extern __shared__ __align__(16) unsigned char g_smem[];

__host__ __device__ inline size_t state_bytes(int max_n) {
    size_t s = kHeadBytes;
    s += 3 * sizeof(float4) * (size_t)max_n;       // two layers + compensation
    s += sizeof(float2) * (size_t)max_n;           // bond lengths
    s += 5 * sizeof(uint16_t) * (size_t)max_n;     // two orders, counts, slot of each bead
    s += (size_t)max_n;                            // flags
    s = (s + 15) / 16 * 16;
    s += 2 * sizeof(float4) * (size_t)((max_n + 31) / 32);   // block bounding boxes
    return s;
}

__host__ __device__ inline size_t layout_bytes(int max_n, int row_width, bool rows_global) {
    return state_bytes(max_n) + (rows_global ? 0 : sizeof(uint16_t) * (size_t)row_width * max_n);
}

template <bool RG>
struct Layout {
    int mx;          // max_n
    uint16_t *grow;  // RG: this item's rows in global memory
    __device__ __forceinline__ SharedHead *h() const { return reinterpret_cast<SharedHead *>(g_smem); }
    // positions by bead, two time layers; lay(2) is the Kahan compensation (w unused)
    __device__ __forceinline__ float4 *lay(int i) const {
        return reinterpret_cast<float4 *>(g_smem + kHeadBytes) + i * mx;
    }
    __device__ __forceinline__ float4 *comp() const { return lay(2); }
    // by bead: (r0 of bond b-1,b ; r0 of bond b,b+1), < 0 when absent
    __device__ __forceinline__ float2 *bond() const { return reinterpret_cast<float2 *>(lay(3)); }
    // slot -> bead (current, spare)
    __device__ __forceinline__ uint16_t *order(int i) const {
        return reinterpret_cast<uint16_t *>(bond() + mx) + i * mx;
    }
    // by slot: native entries of the row, and natives + Verlet entries
    __device__ __forceinline__ uint16_t *n_nat() const { return order(2); }
    __device__ __forceinline__ uint16_t *n_tot() const { return order(3); }
    // by bead: its slot in the current order (kept for systems of more than 256 beads)
    __device__ __forceinline__ uint16_t *slot_of() const { return order(4); }
    // by bead
    __device__ __forceinline__ uint8_t *flags() const { return reinterpret_cast<uint8_t *>(order(5)); }
    // per block of 32 beads: (lo, hi) corners of the bounding box
    __device__ __forceinline__ float4 *bbox() const {
        const size_t off = (kHeadBytes + 3 * 16 * (size_t)mx + 8 * (size_t)mx + 10 * (size_t)mx + mx + 15) / 16 * 16;
        return reinterpret_cast<float4 *>(g_smem + off);
    }
    // by slot: entry k of slot p at row[k * n + p] (bead indices)
    __device__ __forceinline__ uint16_t *row() const {
        if (RG) return grow;
        return reinterpret_cast<uint16_t *>(g_smem + state_bytes(mx));
    }
};

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
__device__ int reorder_slots(const Lay &L, int n_s, int cur_order) {
    const int T = blockDim.x;
    SharedHead *h = L.h();
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
    const int full = n_s - n_s % T;   // slots in complete rounds of T
    for (int p = threadIdx.x; p < n_s; p += T) {
        int pos = atomicAdd(&h->hist[kKeys - 1 - min((int)L.n_tot()[p], kKeys - 1)], 1);
        // boustrophedon: odd rounds run backwards, so a thread owning several slots gets
        // long and short rows alike and the warps of the CTA finish together
        if (pos < full && ((pos / T) & 1)) pos = (pos / T) * T + (T - 1 - pos % T);
        dst[pos] = src[p];
    }
    __syncthreads();
    return cur_order ^ 1;
}

// One 32-candidate block of the all-pairs scan: bit t of *within is set when
// candidate base + t is closer than the cutoff, bit t of *near when it lies in
// the guard band around it (decided later in FP64).
template <bool kFull>
__device__ __forceinline__ void scan32(const float4 *src, int base, int lim, float4 pb, float lo, float hi,
                                       uint32_t *within, uint32_t *near) {
    uint32_t w = 0u, nr = 0u;
    if (kFull) {
        // groups of four candidates form a nibble with constant bit positions
#pragma unroll 2
        for (int g = 0; g < 8; ++g) {
            uint32_t wn = 0u, nn = 0u;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float4 pj = src[base + 4 * g + t];
                const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                if (r2 < lo) wn |= 1u << t;
                if (r2 < hi) nn |= 1u << t;
            }
            w |= wn << (4 * g);
            nr |= nn << (4 * g);
        }
    } else {
        for (int t = 0; t < lim; ++t) {
            const float4 pj = src[base + t];
            const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (r2 < lo) w |= 1u << t;
            if (r2 < hi) nr |= 1u << t;
        }
    }
    *within = w;
    *near = nr & ~w;
}

// Rows from layer src: the bead in slot p gets its native partners and its Verlet
// partners in column p. Block boxes must be current. In systems of up to 256 beads a
// thread builds the rows of its own slots. In larger ones it builds the rows of beads
// threadIdx.x + k * blockDim (slot_of must be current): a warp then scans for 32
// consecutive beads, which lie close together, so the box test skips blocks for all its
// lanes at once (with slots, ordered by row length, the lanes are spread over the whole
// system and some lane needs nearly every block). The rows are the same either way.
template <int BPT, bool RG>
__device__ void rebuild_rows(const BatchedArgs &a, const Layout<RG> &L, const uint16_t *order, const float4 *src,
                             int n_s, int nat_off, int b0) {
    const int T = blockDim.x;
    const float cut2 = a.sa.cut2_f;
    const float lo = cut2 - cut2 * 1e-4f, hi = cut2 + cut2 * 1e-4f;
    const float4 *bb = L.bbox();
    uint16_t *row = L.row();
    // instances with one bead per thread and shared-memory rows never hold more than 256 beads
    constexpr bool kLarge = RG || BPT > 1;
    const bool by_bead = kLarge && n_s > 256;
#pragma unroll 1
    for (int k = 0; k < BPT; ++k) {
        const int idx = threadIdx.x + k * T;
        if (idx >= n_s) continue;
        const int p = by_bead ? (int)L.slot_of()[idx] : idx;
        const int b = by_bead ? idx : (int)order[p];
        const float4 pb = src[b];
        const int nn = a.nat_ell_cnt[b0 + b];
        const uint16_t *natc = a.nat_ell_col + nat_off + b;
        for (int q = 0; q < nn; ++q) row[q * n_s + p] = __ldg(natc + q * n_s);
        const float2 bd = L.bond()[b];
        int q = 0;   // next native to exclude
        int next_nat = nn > 0 ? (int)__ldg(natc) : 0x7fffffff;
        int cnt = 0;
        for (int base = 0; base < n_s; base += 32) {
            // exact cull: every bead of the block is at least as far as its box
            const float4 blo = bb[base >> 4], bhi = bb[(base >> 4) + 1];
            const float ex = fmaxf(fmaxf(blo.x - pb.x, pb.x - bhi.x), 0.f);
            const float ey = fmaxf(fmaxf(blo.y - pb.y, pb.y - bhi.y), 0.f);
            const float ez = fmaxf(fmaxf(blo.z - pb.z, pb.z - bhi.z), 0.f);
            uint32_t within = 0u, near = 0u;
            // in a system of a few blocks nearly every box is in range for some lane of the
            // warp: the test only costs there, so it is skipped
            if (!kLarge || n_s <= 256 || fmaf(ez, ez, fmaf(ey, ey, ex * ex)) < hi) {
                if (base + 32 <= n_s) scan32<true>(src, base, 32, pb, lo, hi, &within, &near);
                else scan32<false>(src, base, n_s - base, pb, lo, hi, &within, &near);
            }
            // exclusions in [base, base + 32): self, bonded neighbours, native partners
            uint32_t ex_mask = 0u;
            if (b >= base && b < base + 32) ex_mask |= 1u << (b - base);
            if (bd.x > 0.f && b - 1 >= base && b - 1 < base + 32) ex_mask |= 1u << (b - 1 - base);
            if (bd.y > 0.f && b + 1 >= base && b + 1 < base + 32) ex_mask |= 1u << (b + 1 - base);
            while (next_nat < base + 32) {
                ex_mask |= 1u << (next_nat - base);
                ++q;
                next_nat = q < nn ? (int)__ldg(natc + q * n_s) : 0x7fffffff;
            }
            within &= ~ex_mask;
            near &= ~ex_mask;
            while (near) {   // rare: decide within the guard band in FP64
                const int t = __ffs(near) - 1;
                near &= near - 1;
                if (within_cut(pb, src[base + t], cut2, a.sa.cut2_d)) within |= 1u << t;
            }
            while (within) {
                const int t = __ffs(within) - 1;
                within &= within - 1;
                if (cnt < a.cap) row[(nn + cnt) * n_s + p] = (uint16_t)(base + t);
                ++cnt;
            }
        }
        if (cnt > a.cap) cta_fail(L.h(), SOP_ERR_PAIRLIST_OVERFLOW);
        L.n_nat()[p] = (uint16_t)nn;
        L.n_tot()[p] = (uint16_t)(nn + min(cnt, a.cap));
    }
}

// A full rebuild from layer src: boxes, slot order, rows. Ends with a barrier.
template <int BPT, bool RG>
__device__ int rebuild(const BatchedArgs &a, const Layout<RG> &L, const float4 *src, int n_s, int nat_off, int b0,
                       int ord) {
    constexpr bool kLarge = RG || BPT > 1;   // as in rebuild_rows
    block_boxes(L, src, n_s);
    ord = reorder_slots(L, n_s, ord);   // its barriers also publish the boxes
    if (kLarge && n_s > 256) {
        const uint16_t *o = L.order(ord);
        for (int p = threadIdx.x; p < n_s; p += blockDim.x) L.slot_of()[o[p]] = (uint16_t)p;
        __syncthreads();
    }
    rebuild_rows<BPT>(a, L, L.order(ord), src, n_s, nat_off, b0);
    __syncthreads();
    return ord;
}

// Sum of the Eq. 1 pair forces on bead b (in slot p) at layer P over its bonds and row.
// Entries k < n_nat are native (12-6 with r0^2 from the table), the rest repulsive.
template <bool RG>
__device__ __forceinline__ float3 bead_force(const BatchedArgs &a, const Layout<RG> &L, const float4 *P, int n_s,
                                             int nat_off, int b, int p, bool *broken) {
    const ForceParams &fp = a.sa.fp;
    const float4 pb = P[b];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const float2 bd = L.bond()[b];
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
    const int nn = L.n_nat()[p], tot = L.n_tot()[p];
    const float *natr = a.nat_ell_r0sq + nat_off + b;
    const uint16_t *rowp = L.row() + p;
    const float A = fp.eps12_h, B = fp.eps6_l;
#pragma unroll 2
    for (int k = 0; k < tot; ++k) {
        const bool nat = k < nn;
        const int j = rowp[k * n_s];
        const float s0 = nat ? __ldg(natr + k * n_s) : fp.sigma2;
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
template <int BPT, bool RG>
__device__ __noinline__ void observe(const BatchedArgs &a, const Layout<RG> &L, const uint16_t *order,
                                     const float4 *P, int n_s, int b0, int r, int s, int g, int64_t step,
                                     int64_t event) {
    const StepArgs &sa = a.sa;
    const DevTopo &t = sa.topo;
    const DevExternal &e = sa.ext;
    const int T = blockDim.x;
    const uint16_t *row = L.row();
    double v[6] = {0, 0, 0, 0, 0, 0};   // E, f_pull, ext, formed, f_wall, r_ee
    const double R02 = sa.R0 * sa.R0, sig2 = sa.sigma * sa.sigma;
    for (int k = 0; k < BPT; ++k) {
        const int p = threadIdx.x + k * T;
        if (p >= n_s) continue;
        const int b = order[p];
        const int i = b0 + b;
        const float4 pb = P[b];
        const double xi = pb.x, yi = pb.y, zi = pb.z;
        if (L.bond()[b].y > 0.f) {
            const float4 pj = P[b + 1];
            const double rr = __dsqrt_rn(dist2_d(xi, yi, zi, pj.x, pj.y, pj.z));
            const double dr = rr - t.bond_r0d[i];
            const double arg = 1.0 - dr * dr / R02;
            if (arg > 0.0) v[0] += -0.5 * sa.k_fene * R02 * log(arg);
        }
        for (int q = t.nat_row[i]; q < t.nat_row[i + 1]; ++q) {
            const int j = t.nat_col[q];
            if (j < i) continue;
            const float4 pj = P[j - b0];
            const double d2 = dist2_d(xi, yi, zi, pj.x, pj.y, pj.z);
            const double r0 = t.nat_r0[q];
            const double u = r0 * r0 / d2;
            const double u3 = u * u * u;
            v[0] += sa.eps_h * (u3 * u3 - 2.0 * u3);
            if (__dsqrt_rn(d2) < r0 + 2.0) v[3] += 1.0;
        }
        for (int q = L.n_nat()[p]; q < L.n_tot()[p]; ++q) {
            const int j = row[q * n_s + p];
            if (j < b) continue;
            const float4 pj = P[j];
            const double c = sig2 / dist2_d(xi, yi, zi, pj.x, pj.y, pj.z);
            v[0] += sa.eps_l * c * c * c;
        }
        const uint8_t fl = L.flags()[b];
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
    block_sum6(v, L.h());
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

// MAXT: largest CTA the instance is compiled for; MINB: CTAs of MAXT threads that must
// fit an SM, i.e. the register cap 65536 / (MAXT * MINB). RG: rows in global memory.
template <int BPT, int MINB, int MAXT, bool RG>
__global__ void __launch_bounds__(MAXT, MINB) k_batched(BatchedArgs a) {
    const int item = blockIdx.x;
    Layout<RG> L;
    L.mx = a.max_n;
    L.grow = RG ? a.row_global + (size_t)item * a.row_width * a.max_n : nullptr;
    const int r = a.item_rep[item], s = a.item_sys[item];
    const StepArgs &sa = a.sa;
    const DevTopo &t = sa.topo;
    const int b0 = t.sys_lo[s], n_s = t.sys_lo[s + 1] - b0;
    const int gbase = r * t.n + b0;   // replicas x beads < 2^28
    const int g = r * t.n_sys + s;
    const int nat_off = a.nat_ell_off[s];
    const int T = blockDim.x;
    const int64_t step0 = *a.d_step;
    const bool forces_only = (a.n_steps == 0 && a.force_out != nullptr);

    if (threadIdx.x == 0) L.h()->fail = 0;
    if (!forces_only && (sa.rep_status[r] != 0 || *sa.halt != 0)) {   // CTA-uniform: a frozen replica
        if (threadIdx.x == 0)                                           // only marks its records
            missing_records(a, r, s, g, step0, step0, a.d_events ? *a.d_events : 0);
        return;
    }
    // phases of the step counter, kept as wrapped counters instead of 64-bit modulos
    int k_phase = (int)(step0 % a.K);                                   // step mod K
    int o_phase = a.obs_every > 0 ? (int)(step0 % a.obs_every) : 0;     // step mod obs_every
    // load the item; the first order is by native row length
    for (int b = threadIdx.x; b < n_s; b += T) {
        const int i = b0 + b;
        L.lay(0)[b] = a.pos[gbase + b];
        L.comp()[b] = a.comp[gbase + b];
        L.bond()[b] = make_float2(b > 0 ? t.bond_r0[i - 1] : -1.f, t.bond_r0[i]);
        L.flags()[b] = t.flags[i];
        L.order(0)[b] = (uint16_t)b;
        L.n_tot()[b] = (uint16_t)a.nat_ell_cnt[i];
        // the list of the first step comes from the positions at the last rebuild step
        if (k_phase != 0) L.lay(1)[b] = a.snap[gbase + b];
    }
    __syncthreads();

    int cur = 0, ord = 0;
    int n_events = 0;
    bool built_now = false;   // the list was built at the current step
    int it = 0;
    for (; it < a.n_steps || (forces_only && it == 0); ++it) {
        const float4 *P = L.lay(cur);
        float4 *Q = L.lay(cur ^ 1);
        if (it == 0 && k_phase != 0 && !forces_only) {
            ord = rebuild<BPT>(a, L, Q, n_s, nat_off, b0, ord);   // Q holds the snapshot here
        } else if ((k_phase == 0 && !built_now) || forces_only) {
            ord = rebuild<BPT>(a, L, P, n_s, nat_off, b0, ord);
            if (!forces_only)
                for (int b = threadIdx.x; b < n_s; b += T) a.snap[gbase + b] = P[b];
        }
        built_now = false;
        const int64_t step = step0 + it;
        const uint16_t *order = L.order(ord);
        if (forces_only) {
            for (int p = threadIdx.x; p < n_s; p += T) {
                const int b = order[p];
                bool broken = false, overlap = false;
                const float3 f = bead_force(a, L, P, n_s, nat_off, b, p, &broken);
                const float3 fe = ext_force(sa, r, b0 + b, L.flags()[b], P[b], step, &overlap);
                a.force_out[gbase + b] = make_float4(f.x + fe.x, f.y + fe.y, f.z + fe.z, (broken || overlap) ? 1.f : 0.f);
                if (a.pl_dump_col) {
                    const size_t rowi = (size_t)gbase + b;
                    const int nn = L.n_nat()[p], np = L.n_tot()[p] - nn;
                    a.pl_dump_start[rowi] = (int)(rowi * a.pl_dump_stride);
                    a.pl_dump_len[rowi] = np;
                    for (int q = 0; q < np; ++q)
                        a.pl_dump_col[rowi * a.pl_dump_stride + q] = b0 + (int)L.row()[(nn + q) * n_s + p];
                }
            }
            break;
        }
#pragma unroll 1
        for (int k = 0; k < BPT; ++k) {
            const int p = threadIdx.x + k * T;
            if (p >= n_s) continue;
            const int b = order[p];
            bool broken = false, overlap = false;
            const float3 f = bead_force(a, L, P, n_s, nat_off, b, p, &broken);
            const float4 p_old = P[b];
            const uint8_t fl = L.flags()[b];
            const float3 fe = ext_force(sa, r, b0 + b, fl, p_old, step, &overlap);
            float4 pb = p_old;
            if (broken || overlap) {
                // a bead whose force cannot be evaluated stays where it is; the replica freezes
                cta_fail(L.h(), broken ? SOP_ERR_FENE_BREAK : SOP_ERR_INDENTER_OVERLAP);
            } else if (!(fl & kFlagFixed)) {
                float4 c = L.comp()[b];
                if (update_position(sa, r, b0 + b, (size_t)gbase + b, pb, c,
                                    make_float3(f.x + fe.x, f.y + fe.y, f.z + fe.z), step))
                    L.comp()[b] = c;
                else
                    cta_fail(L.h(), SOP_ERR_NONFINITE);
            }
            Q[b] = pb;
        }
        __syncthreads();
        cur ^= 1;
        k_phase = k_phase + 1 == a.K ? 0 : k_phase + 1;
        if (a.obs_every > 0) o_phase = o_phase + 1 == a.obs_every ? 0 : o_phase + 1;
        if (L.h()->fail != 0) { ++it; break; }   // the replica freezes after the step in which it failed
        if (a.obs_every > 0 && o_phase == 0) {
            const float4 *Pn = L.lay(cur);
            if (k_phase == 0) {
                ord = rebuild<BPT>(a, L, Pn, n_s, nat_off, b0, ord);
                built_now = true;
                for (int b = threadIdx.x; b < n_s; b += T) a.snap[gbase + b] = Pn[b];
            }
            const int64_t ev = (a.d_events ? *a.d_events : 0) + n_events;
            observe<BPT>(a, L, L.order(ord), Pn, n_s, b0, r, s, g, step + 1, ev);
            ++n_events;
        }
    }
    if (forces_only) return;
    if (threadIdx.x == 0 && L.h()->fail != 0)
        missing_records(a, r, s, g, step0, step0 + it, (a.d_events ? *a.d_events : 0) + n_events);
    const float4 *P = L.lay(cur);
    for (int b = threadIdx.x; b < n_s; b += T) {
        a.pos[gbase + b] = P[b];
        a.comp[gbase + b] = L.comp()[b];
    }
    if (threadIdx.x == 0 && L.h()->fail != 0) atomicCAS(&sa.rep_status[r], 0, L.h()->fail);
}

// ===========================================================================
// Cluster form: one system over a thread-block cluster (distributed shared
// memory). CTA q of a cluster of C owns the system's beads [q m, (q + 1) m),
// m = 2^m_shift a multiple of 32: their compensation, bond lengths, slot orders
// and rows live in its shared memory, next to a full copy of the positions of the
// whole system (both time layers). All reads are local: a CTA gathers forces and
// builds rows exactly as the one-CTA form does, from its own copy. After the
// update each CTA writes the new positions of its own beads into every copy in
// the cluster (stores to distributed shared memory), and one cluster barrier
// (release/acquire) ends the step. A copy's layer is only ever written while
// every CTA reads the other layer, so no read meets a remote write. Every CTA of
// a cluster takes the same sequence of cluster barriers: each control decision
// (a frozen replica, a failure, the rebuild and observable cadence) comes from
// values every CTA reads after the same barrier.
// ===========================================================================
constexpr int kMaxCluster = 16;
constexpr int kNoFail = 0x7fffffff;

struct ClusterExtra {
    int fail_step;                        // first step of the launch at which this CTA failed
    int frozen;                           // rank 0: the replica was frozen at launch
    double part[6];                       // this CTA's observable sums
    float4 *rpos[2][kMaxCluster];         // every rank's two position layers (generic addresses)
    const ClusterExtra *peer[kMaxCluster];
};

// Shared-memory layout of one CTA of the cluster form: positions of all n_max = C m
// beads (two layers), then own-bead state for m beads, block boxes of the whole
// system, rows of the own slots, and the cluster bookkeeping.
struct CLayout {
    int nmax, m, rw;
    __device__ __forceinline__ SharedHead *h() const { return reinterpret_cast<SharedHead *>(g_smem); }
    __device__ __forceinline__ float4 *pos(int layer) const {
        return reinterpret_cast<float4 *>(g_smem + kHeadBytes) + (size_t)layer * nmax;
    }
    __device__ __forceinline__ float4 *comp() const { return pos(2); }
    __device__ __forceinline__ float2 *bond() const { return reinterpret_cast<float2 *>(comp() + m); }
    __device__ __forceinline__ uint16_t *order(int i) const {
        return reinterpret_cast<uint16_t *>(bond() + m) + i * m;
    }
    __device__ __forceinline__ uint16_t *n_nat() const { return order(2); }
    __device__ __forceinline__ uint16_t *n_tot() const { return order(3); }
    __device__ __forceinline__ uint16_t *slot_of() const { return order(4); }   // by own bead: its slot
    __device__ __forceinline__ uint8_t *flags() const { return reinterpret_cast<uint8_t *>(order(5)); }
    __device__ __forceinline__ float4 *bbox() const {
        const size_t off = (kHeadBytes + 32 * (size_t)nmax + 16 * (size_t)m + 8 * (size_t)m + 10 * (size_t)m + m + 15)
                           / 16 * 16;
        return reinterpret_cast<float4 *>(g_smem + off);
    }
    __device__ __forceinline__ uint16_t *row() const { return reinterpret_cast<uint16_t *>(bbox() + nmax / 16); }
    __device__ __forceinline__ ClusterExtra *extra() const {
        const size_t off = ((reinterpret_cast<unsigned char *>(row() + (size_t)rw * m) - g_smem) + 15) / 16 * 16;
        return reinterpret_cast<ClusterExtra *>(g_smem + off);
    }
};

__host__ __device__ inline size_t cluster_smem(int m, int nmax, int row_width) {
    size_t s = kHeadBytes + 32 * (size_t)nmax + 16 * (size_t)m + 8 * (size_t)m + 10 * (size_t)m + m;
    s = (s + 15) / 16 * 16;
    s += 2 * sizeof(float4) * (size_t)(nmax / 32);
    s += sizeof(uint16_t) * (size_t)row_width * m;
    s = (s + 15) / 16 * 16;
    return s + (sizeof(ClusterExtra) + 15) / 16 * 16;
}

// Rows of this CTA's slots from layer `layer` of its copy (system-local bead indices).
// The block boxes of the whole system and slot_of must be current. A thread builds the
// rows of own beads threadIdx.x + k * blockDim, so that a warp scans for 32 consecutive
// beads and the box test skips blocks for all its lanes at once (as in rebuild_rows).
template <int BPT>
__device__ void cluster_rows(const BatchedArgs &a, const CLayout &L, const uint16_t *order, int layer, int n_loc,
                             int lo, int n_s, int nat_off, int b0) {
    const int T = blockDim.x, m = L.m;
    const float cut2 = a.sa.cut2_f;
    const float lo2 = cut2 - cut2 * 1e-4f, hi2 = cut2 + cut2 * 1e-4f;
    const float4 *src = L.pos(layer);
    const float4 *bb = L.bbox();
    uint16_t *row = L.row();
    (void)order;
#pragma unroll 1
    for (int k = 0; k < BPT; ++k) {
        const int l = threadIdx.x + k * T;
        if (l >= n_loc) continue;
        const int p = L.slot_of()[l];
        const int b = lo + l;
        const float4 pb = src[b];
        const int nn = a.nat_ell_cnt[b0 + b];
        const uint16_t *natc = a.nat_ell_col + nat_off + b;
        for (int q = 0; q < nn; ++q) row[q * m + p] = __ldg(natc + q * n_s);
        const float2 bd = L.bond()[l];
        int q = 0;
        int next_nat = nn > 0 ? (int)__ldg(natc) : 0x7fffffff;
        int cnt = 0;
        for (int base = 0; base < n_s; base += 32) {
            const float4 blo = bb[base >> 4], bhi = bb[(base >> 4) + 1];
            const float ex = fmaxf(fmaxf(blo.x - pb.x, pb.x - bhi.x), 0.f);
            const float ey = fmaxf(fmaxf(blo.y - pb.y, pb.y - bhi.y), 0.f);
            const float ez = fmaxf(fmaxf(blo.z - pb.z, pb.z - bhi.z), 0.f);
            uint32_t within = 0u, near = 0u;
            if (fmaf(ez, ez, fmaf(ey, ey, ex * ex)) < hi2) {
                if (base + 32 <= n_s) scan32<true>(src, base, 32, pb, lo2, hi2, &within, &near);
                else scan32<false>(src, base, n_s - base, pb, lo2, hi2, &within, &near);
            }
            uint32_t ex_mask = 0u;
            if (b >= base && b < base + 32) ex_mask |= 1u << (b - base);
            if (bd.x > 0.f && b - 1 >= base && b - 1 < base + 32) ex_mask |= 1u << (b - 1 - base);
            if (bd.y > 0.f && b + 1 >= base && b + 1 < base + 32) ex_mask |= 1u << (b + 1 - base);
            while (next_nat < base + 32) {
                ex_mask |= 1u << (next_nat - base);
                ++q;
                next_nat = q < nn ? (int)__ldg(natc + q * n_s) : 0x7fffffff;
            }
            within &= ~ex_mask;
            near &= ~ex_mask;
            while (near) {
                const int t = __ffs(near) - 1;
                near &= near - 1;
                if (within_cut(pb, src[base + t], cut2, a.sa.cut2_d)) within |= 1u << t;
            }
            while (within) {
                const int t = __ffs(within) - 1;
                within &= within - 1;
                if (cnt < a.cap) row[(nn + cnt) * m + p] = (uint16_t)(base + t);
                ++cnt;
            }
        }
        if (cnt > a.cap) cta_fail(L.h(), SOP_ERR_PAIRLIST_OVERFLOW);
        L.n_nat()[p] = (uint16_t)nn;
        L.n_tot()[p] = (uint16_t)(nn + min(cnt, a.cap));
    }
}

// Rebuild from layer `layer` of the local copy: boxes of every block of the system, the
// own slot order and rows. Local only; ends with a CTA barrier.
template <int BPT>
__device__ int cluster_rebuild(const BatchedArgs &a, const CLayout &L, int layer, int n_loc, int lo, int n_s,
                               int nat_off, int b0, int ord) {
    block_boxes(L, L.pos(layer), n_s);
    ord = reorder_slots(L, n_loc, ord);   // its barriers also publish the boxes
    const uint16_t *o = L.order(ord);
    for (int p = threadIdx.x; p < n_loc; p += blockDim.x) L.slot_of()[o[p]] = (uint16_t)p;
    __syncthreads();
    cluster_rows<BPT>(a, L, L.order(ord), layer, n_loc, lo, n_s, nat_off, b0);
    __syncthreads();
    return ord;
}

// Eq. 1 pair forces on own bead l (system bead b, slot p) at layer P of the local copy.
__device__ __forceinline__ float3 cluster_force(const BatchedArgs &a, const CLayout &L, const float4 *P, int n_s,
                                                int nat_off, int l, int b, int p, bool *broken) {
    const ForceParams &fp = a.sa.fp;
    const int m = L.m;
    const float4 pb = P[b];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const float2 bd = L.bond()[l];
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
    const int nn = L.n_nat()[p], tot = L.n_tot()[p];
    const float *natr = a.nat_ell_r0sq + nat_off + b;
    const uint16_t *rowp = L.row() + p;
    const float A = fp.eps12_h, B = fp.eps6_l;
#pragma unroll 2
    for (int k = 0; k < tot; ++k) {
        const bool nat = k < nn;
        const int j = rowp[k * m];
        const float s0 = nat ? __ldg(natr + k * n_s) : fp.sigma2;
        const float4 pj = P[j];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float inv = __fdividef(1.0f, r2);
        const float s = s0 * inv;
        const float s3 = s * s * s;
        const float c = inv * s3 * (nat ? fmaf(A, s3, -A) : B);
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    return make_float3(fx, fy, fz);
}

// FP64 observables of the cluster's system at layer P: every CTA sums its own beads, rank
// 0 adds the CTA sums after a cluster barrier and writes the record.
template <int BPT>
__device__ __noinline__ void cluster_observe(const BatchedArgs &a, const CLayout &L, ClusterExtra *X,
                                             const uint16_t *order, const float4 *P, int n_loc, int lo, int b0,
                                             int r, int s, int g, int64_t step, int64_t event, int rank, int C) {
    const StepArgs &sa = a.sa;
    const DevTopo &t = sa.topo;
    const DevExternal &e = sa.ext;
    const int T = blockDim.x, m = L.m;
    const uint16_t *row = L.row();
    double v[6] = {0, 0, 0, 0, 0, 0};   // E, f_pull, ext, formed, f_wall, r_ee
    const double R02 = sa.R0 * sa.R0, sig2 = sa.sigma * sa.sigma;
    for (int k = 0; k < BPT; ++k) {
        const int p = threadIdx.x + k * T;
        if (p >= n_loc) continue;
        const int l = order[p];
        const int b = lo + l;
        const int i = b0 + b;
        const float4 pb = P[b];
        const double xi = pb.x, yi = pb.y, zi = pb.z;
        if (L.bond()[l].y > 0.f) {
            const float4 pj = P[b + 1];
            const double rr = __dsqrt_rn(dist2_d(xi, yi, zi, pj.x, pj.y, pj.z));
            const double dr = rr - t.bond_r0d[i];
            const double arg = 1.0 - dr * dr / R02;
            if (arg > 0.0) v[0] += -0.5 * sa.k_fene * R02 * log(arg);
        }
        for (int q = t.nat_row[i]; q < t.nat_row[i + 1]; ++q) {
            const int j = t.nat_col[q];
            if (j < i) continue;
            const float4 pj = P[j - b0];
            const double d2 = dist2_d(xi, yi, zi, pj.x, pj.y, pj.z);
            const double r0 = t.nat_r0[q];
            const double u = r0 * r0 / d2;
            const double u3 = u * u * u;
            v[0] += sa.eps_h * (u3 * u3 - 2.0 * u3);
            if (__dsqrt_rn(d2) < r0 + 2.0) v[3] += 1.0;
        }
        for (int q = L.n_nat()[p]; q < L.n_tot()[p]; ++q) {
            const int j = row[q * m + p];
            if (j < b) continue;
            const float4 pj = P[j];
            const double c = sig2 / dist2_d(xi, yi, zi, pj.x, pj.y, pj.z);
            v[0] += sa.eps_l * c * c * c;
        }
        const uint8_t fl = L.flags()[l];
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
    block_sum6(v, L.h());
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) X->part[k] = v[k];
    cg::this_cluster().sync();
    if (rank == 0 && threadIdx.x == 0) {
        double w[6] = {0, 0, 0, 0, 0, 0};
        for (int q = 0; q < C; ++q)
            for (int k = 0; k < 6; ++k) w[k] += X->peer[q]->part[k];
        sop_record rec;
        rec.step = (double)step;
        rec.replica = (double)r;
        rec.system = (double)s;
        rec.energy = w[0];
        const bool pulled = e.pull_of_sys[s] >= 0;
        rec.f_ext = pulled ? w[1] : (e.has_indenter ? w[4] : 0.0);
        rec.extension = pulled ? w[2] : (e.has_indenter ? e.ind_v * ((double)step - e.ind_n0) : 0.0);
        const int np = t.sys_nat_pairs[s];
        rec.q = np > 0 ? w[3] / (double)np : 0.0;
        rec.r_ee = w[5];
        a.obs.ring[(event * a.n_seg + g) % a.obs.cap] = rec;
    }
    __syncthreads();
}

template <int BPT, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_cluster(BatchedArgs a, int sh) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int C = (int)cl.num_blocks();
    const int item = blockIdx.x / C;
    CLayout L;
    L.m = 1 << sh;
    L.nmax = C << sh;
    L.rw = a.row_width;
    ClusterExtra *X = L.extra();
    const int r = a.item_rep[item], s = a.item_sys[item];
    const StepArgs &sa = a.sa;
    const DevTopo &t = sa.topo;
    const int b0 = t.sys_lo[s], n_s = t.sys_lo[s + 1] - b0;
    const int lo = rank * L.m;
    const int n_loc = max(0, min(L.m, n_s - lo));
    const int gbase = r * t.n + b0;
    const int g = r * t.n_sys + s;
    const int nat_off = a.nat_ell_off[s];
    const int T = blockDim.x;
    const int64_t step0 = *a.d_step;
    const bool forces_only = (a.n_steps == 0 && a.force_out != nullptr);
    if (threadIdx.x == 0) {
        L.h()->fail = 0;
        X->fail_step = kNoFail;
        X->frozen = (!forces_only && (sa.rep_status[r] != 0 || *sa.halt != 0)) ? 1 : 0;
    }
    for (int k = threadIdx.x; k < 3 * C; k += T) {
        if (k < 2 * C) X->rpos[k / C][k % C] = cl.map_shared_rank(L.pos(k / C), k % C);
        else X->peer[k - 2 * C] = cl.map_shared_rank(X, k - 2 * C);
    }
    int k_phase = (int)(step0 % a.K);
    int o_phase = a.obs_every > 0 ? (int)(step0 % a.obs_every) : 0;
    // the whole system into the local copy (and the snapshot of the last rebuild into layer 1)
    for (int b = threadIdx.x; b < n_s; b += T) {
        L.pos(0)[b] = a.pos[gbase + b];
        if (k_phase != 0 && !forces_only) L.pos(1)[b] = a.snap[gbase + b];
    }
    for (int l = threadIdx.x; l < n_loc; l += T) {
        const int b = lo + l, i = b0 + b;
        L.comp()[l] = a.comp[gbase + b];
        L.bond()[l] = make_float2(b > 0 ? t.bond_r0[i - 1] : -1.f, t.bond_r0[i]);
        L.flags()[l] = t.flags[i];
        L.order(0)[l] = (uint16_t)l;
        L.n_tot()[l] = (uint16_t)a.nat_ell_cnt[i];
    }
    cl.sync();   // every copy is loaded before any CTA writes into another
    const bool frozen = X->peer[0]->frozen != 0;   // rank 0's reading, the same for every CTA
    if (frozen) {
        if (rank == 0 && threadIdx.x == 0)
            missing_records(a, r, s, g, step0, step0, a.d_events ? *a.d_events : 0);
        cl.sync();   // no CTA leaves while another may still read its shared memory
        return;
    }

    int cur = 0, ord = 0, n_events = 0;
    bool built_now = false;
    int it = 0;
    for (; it < a.n_steps || (forces_only && it == 0); ++it) {
        if (it == 0 && k_phase != 0 && !forces_only) {
            ord = cluster_rebuild<BPT>(a, L, 1, n_loc, lo, n_s, nat_off, b0, ord);   // from the snapshot
            cl.sync();   // layer 1 is read by every CTA before the step writes it
        } else if ((k_phase == 0 && !built_now) || forces_only) {
            ord = cluster_rebuild<BPT>(a, L, cur, n_loc, lo, n_s, nat_off, b0, ord);
            if (!forces_only)
                for (int l = threadIdx.x; l < n_loc; l += T) a.snap[gbase + lo + l] = L.pos(cur)[lo + l];
        }
        built_now = false;
        const int64_t step = step0 + it;
        const uint16_t *order = L.order(ord);
        const float4 *P = L.pos(cur);
        if (forces_only) {
            for (int p = threadIdx.x; p < n_loc; p += T) {
                const int l = order[p], b = lo + l;
                bool broken = false, overlap = false;
                const float3 f = cluster_force(a, L, P, n_s, nat_off, l, b, p, &broken);
                const float3 fe = ext_force(sa, r, b0 + b, L.flags()[l], P[b], step, &overlap);
                a.force_out[gbase + b] = make_float4(f.x + fe.x, f.y + fe.y, f.z + fe.z, (broken || overlap) ? 1.f : 0.f);
                if (a.pl_dump_col) {
                    const size_t rowi = (size_t)gbase + b;
                    const int nn = L.n_nat()[p], np = L.n_tot()[p] - nn;
                    a.pl_dump_start[rowi] = (int)(rowi * a.pl_dump_stride);
                    a.pl_dump_len[rowi] = np;
                    for (int q = 0; q < np; ++q)
                        a.pl_dump_col[rowi * a.pl_dump_stride + q] = b0 + (int)L.row()[(nn + q) * L.m + p];
                }
            }
            break;
        }
        const int nxt = cur ^ 1;
#pragma unroll 1
        for (int k = 0; k < BPT; ++k) {
            const int p = threadIdx.x + k * T;
            if (p >= n_loc) continue;
            const int l = order[p], b = lo + l;
            bool broken = false, overlap = false;
            const float3 f = cluster_force(a, L, P, n_s, nat_off, l, b, p, &broken);
            const float4 p_old = P[b];
            const uint8_t fl = L.flags()[l];
            const float3 fe = ext_force(sa, r, b0 + b, fl, p_old, step, &overlap);
            float4 pb = p_old;
            if (broken || overlap) {
                cta_fail(L.h(), broken ? SOP_ERR_FENE_BREAK : SOP_ERR_INDENTER_OVERLAP);
            } else if (!(fl & kFlagFixed)) {
                float4 c = L.comp()[l];
                if (update_position(sa, r, b0 + b, (size_t)gbase + b, pb, c,
                                    make_float3(f.x + fe.x, f.y + fe.y, f.z + fe.z), step))
                    L.comp()[l] = c;
                else
                    cta_fail(L.h(), SOP_ERR_NONFINITE);
            }
            // the new position into every copy of the cluster
            for (int q = 0; q < C; ++q) X->rpos[nxt][q][b] = pb;
        }
        __syncthreads();
        if (threadIdx.x == 0 && L.h()->fail != 0 && X->fail_step == kNoFail) X->fail_step = it;
        cl.sync();   // the next layer is complete in every copy
        cur = nxt;
        k_phase = k_phase + 1 == a.K ? 0 : k_phase + 1;
        if (a.obs_every > 0) o_phase = o_phase + 1 == a.obs_every ? 0 : o_phase + 1;
        // the replica freezes after the step in which any CTA failed (every CTA decides
        // from the same values: a CTA's fail_step is written once, before a barrier)
        bool stop = false;
        for (int q = 0; q < C; ++q) stop |= X->peer[q]->fail_step <= it;
        if (stop) { ++it; break; }
        if (a.obs_every > 0 && o_phase == 0) {
            if (k_phase == 0) {
                ord = cluster_rebuild<BPT>(a, L, cur, n_loc, lo, n_s, nat_off, b0, ord);
                built_now = true;
                for (int l = threadIdx.x; l < n_loc; l += T) a.snap[gbase + lo + l] = L.pos(cur)[lo + l];
            }
            const int64_t ev = (a.d_events ? *a.d_events : 0) + n_events;
            cluster_observe<BPT>(a, L, X, L.order(ord), L.pos(cur), n_loc, lo, b0, r, s, g, step + 1, ev, rank, C);
            ++n_events;
        }
    }
    if (!forces_only) {
        bool failed = false;
        for (int q = 0; q < C; ++q) failed |= X->peer[q]->fail_step != kNoFail;
        if (failed && rank == 0 && threadIdx.x == 0)
            missing_records(a, r, s, g, step0, step0 + it, (a.d_events ? *a.d_events : 0) + n_events);
        for (int l = threadIdx.x; l < n_loc; l += T) {
            a.pos[gbase + lo + l] = L.pos(cur)[lo + l];
            a.comp[gbase + lo + l] = L.comp()[l];
        }
        if (threadIdx.x == 0 && L.h()->fail != 0) atomicCAS(&sa.rep_status[r], 0, L.h()->fail);
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

template <int BPT, int MAXT>
cudaError_t launch_cl(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s) {
    auto kern = k_cluster<BPT, MAXT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    if (cfg.cluster > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(a.n_items * cfg.cluster), 1, 1);
    lc.blockDim = dim3((unsigned)cfg.threads, 1, 1);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cfg.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, kern, a, cfg.m_shift);
}

template <int BPT, int MINB, int MAXT, bool RG>
cudaError_t launch_t(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s) {
    auto kern = k_batched<BPT, MINB, MAXT, RG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    kern<<<a.n_items, cfg.threads, cfg.smem, s>>>(a);
    return cudaGetLastError();
}

// Shared-memory rows, CTAs of up to 256 threads.
template <int BPT>
cudaError_t launch_small(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s) {
    switch (cfg.min_blocks) {
    case 2: return launch_t<BPT, 2, 256, false>(a, cfg, s);
    case 3: return launch_t<BPT, 3, 256, false>(a, cfg, s);
    default: return launch_t<BPT, 4, 256, false>(a, cfg, s);
    }
}

}  // namespace

// The compiled instances: shared-memory rows with CTAs of at most 256 threads and
// 1, 2 or 4 beads per thread under a register cap of 128, 85 or 64; global-memory
// rows with CTAs of at most 1024 threads, 1 to 8 beads per thread, 64 registers.
bool batched_config(int max_n, int row_width, int threads, bool rows_global, int min_blocks, BatchedConfig *cfg) {
    if (max_n <= 0 || max_n > 8192 || row_width > kKeys - 1 || threads % 32 || threads < 32) return false;
    const int bpt = (max_n + threads - 1) / threads;
    const int bpt_c = bpt <= 1 ? 1 : bpt <= 2 ? 2 : bpt <= 4 ? 4 : 8;
    if (bpt > 8) return false;
    if (!rows_global && (threads > 256 || bpt_c > 4 || min_blocks < 2 || min_blocks > 4)) return false;
    if (rows_global && (threads > 1024 || min_blocks != 1)) return false;
    cfg->threads = threads;
    cfg->beads_per_thread = bpt_c;
    cfg->min_blocks = min_blocks;
    cfg->rows_global = rows_global;
    cfg->row_width = row_width;
    cfg->smem = layout_bytes(max_n, row_width, rows_global);
    return cfg->smem <= 227 * 1024;
}

bool cluster_config(int max_n, int row_width, int threads, int m_shift, BatchedConfig *cfg) {
    if (m_shift < 5 || m_shift > 9 || max_n <= 0 || max_n > 8192 || row_width > kKeys - 1) return false;
    const int m = 1 << m_shift;
    const int C = (max_n + m - 1) / m;
    if (C < 2 || C > kMaxCluster || threads % 32 || threads < 32 || threads > 512) return false;
    const int bpt = (m + threads - 1) / threads;
    if (bpt > 2) return false;
    cfg->threads = threads;
    cfg->beads_per_thread = bpt;
    cfg->min_blocks = 1;
    cfg->rows_global = false;
    cfg->row_width = row_width;
    cfg->smem = cluster_smem(m, C * m, row_width);
    cfg->cluster = C;
    cfg->m_shift = m_shift;
    return cfg->smem <= 227 * 1024;
}

// Clusters of this configuration that can be resident at once (0: it cannot launch).
int cluster_capacity(const BatchedConfig &cfg) {
    if (cfg.cluster <= 0) return 0;
    auto kern = cfg.beads_per_thread == 1 ? k_cluster<1, 512> : k_cluster<2, 512>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem) != cudaSuccess ||
        (cfg.cluster > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)cfg.cluster, 1, 1);
    lc.blockDim = dim3((unsigned)cfg.threads, 1, 1);
    lc.dynamicSmemBytes = cfg.smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cfg.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &lc) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_batched(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s, int64_t *launches) {
    if (a.n_items <= 0) return cudaSuccess;
    if (launches) *launches += 1;
    if (cfg.cluster > 0)
        return cfg.beads_per_thread == 1 ? launch_cl<1, 512>(a, cfg, s) : launch_cl<2, 512>(a, cfg, s);
    if (cfg.rows_global) {
        switch (cfg.beads_per_thread) {
        case 1: return launch_t<1, 1, 1024, true>(a, cfg, s);
        case 2: return launch_t<2, 1, 1024, true>(a, cfg, s);
        case 4: return launch_t<4, 1, 1024, true>(a, cfg, s);
        default: return launch_t<8, 1, 1024, true>(a, cfg, s);
        }
    }
    switch (cfg.beads_per_thread) {
    case 1: return launch_small<1>(a, cfg, s);
    case 2: return launch_small<2>(a, cfg, s);
    default: return launch_small<4>(a, cfg, s);
    }
}

// CTAs of this configuration that the device holds at once (0: unknown).
namespace {
template <int BPT, int MINB, int MAXT, bool RG>
int resident_t(const BatchedConfig &cfg) {
    auto kern = k_batched<BPT, MINB, MAXT, RG>;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cfg.threads, cfg.smem) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}
}  // namespace

int batched_resident_ctas(const BatchedConfig &cfg) {
    if (cfg.cluster > 0) return cluster_capacity(cfg) * cfg.cluster;
    if (cfg.rows_global) {
        switch (cfg.beads_per_thread) {
        case 1: return resident_t<1, 1, 1024, true>(cfg);
        case 2: return resident_t<2, 1, 1024, true>(cfg);
        case 4: return resident_t<4, 1, 1024, true>(cfg);
        default: return resident_t<8, 1, 1024, true>(cfg);
        }
    }
    const int b = cfg.beads_per_thread;
    switch (cfg.min_blocks) {
    case 2: return b == 1 ? resident_t<1, 2, 256, false>(cfg) : b == 2 ? resident_t<2, 2, 256, false>(cfg)
                                                                      : resident_t<4, 2, 256, false>(cfg);
    case 3: return b == 1 ? resident_t<1, 3, 256, false>(cfg) : b == 2 ? resident_t<2, 3, 256, false>(cfg)
                                                                      : resident_t<4, 3, 256, false>(cfg);
    default: return b == 1 ? resident_t<1, 4, 256, false>(cfg) : b == 2 ? resident_t<2, 4, 256, false>(cfg)
                                                                       : resident_t<4, 4, 256, false>(cfg);
    }
}

}  // namespace sop
