// Pair-based parallelisation of the force evaluation (Sec. III.B, Algorithms 4 and 5), sm_103a.
//
// Each thread of the pair kernel evaluates one interacting pair -- a bond, a native
// contact or a Verlet pair, each taken once with i < j -- and stores +df in the slot of
// the entry (i -> j) and -df in the slot of the reverse entry (j -> i) of a force table
// that is laid out like the rows: bond slots 2 gb (bond to the left) and 2 gb + 1 (bond to
// the right), native slots aligned with the native CSR (one table per replica), Verlet
// slots aligned with the Verlet columns. Every slot has exactly one writer, so there are
// no atomics and the result does not depend on thread timing. The gathering of
// Algorithm 5 -- the sum over a bead's slots -- is fused into the update kernel, with L
// lanes per bead reading the bead's contiguous slots.
//
// The Verlet half list is rebuilt with the list: rows are ascending, so the entries with
// j > i form the tail of row i; they are counted, offset by a scan, and each one finds
// its reverse entry by binary search in the row of j (the list is symmetric).
#include <cuda_runtime.h>

#include "sop_internal.h"
#include "sop_step.cuh"

namespace sop {

namespace {

inline int blocks_for(int64_t work, int threads) { return (int)((work + threads - 1) / threads); }

constexpr int kPairThreads = 256;
constexpr int kPairMaxBlocks = 152 * 8;   // grid-stride beyond one wave of 8 CTAs per SM

// First position of row [s, s + len) whose column exceeds i (columns ascending).
__device__ __forceinline__ int first_above(const int32_t *col, int s, int len, int i) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (col[s + mid] > i) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void k_pair_count(DevPairList pl, int32_t *count, int n, int b_lo, int b_hi) {
    const int gb = b_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (gb >= b_hi) return;
    const int i = gb % n;
    const int s = pl.start[gb], len = pl.len[gb];
    count[gb - b_lo] = len - first_above(pl.col, s, len, i);
}

__global__ void k_pair_fill(DevPairList pl, DevPairTables t, int32_t *rep_status, int n, int b_lo, int b_hi) {
    const int gb = b_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (gb >= b_hi) return;
    const int r = gb / n, i = gb - r * n;
    const int s = pl.start[gb], len = pl.len[gb];
    const int lo = first_above(pl.col, s, len, i);
    const int64_t base = t.voff[gb - b_lo];
    for (int u = 0; lo + u < len; ++u) {
        const int k = s + lo + u;
        const int gj = r * n + pl.col[k];
        // reverse entry: i in the ascending row of j
        const int sj = pl.start[gj], lj = pl.len[gj];
        int a0 = 0, a1 = lj;
        while (a0 < a1) {
            const int mid = (a0 + a1) >> 1;
            if (pl.col[sj + mid] < i) a0 = mid + 1;
            else a1 = mid;
        }
        const int kr = (a0 < lj && pl.col[sj + a0] == i) ? sj + a0 : -1;
        if (base + u < t.vcap) t.vpair[base + u] = make_int4(k, kr, gb, gj);
        else set_status(&rep_status[r], (int32_t)SOP_ERR_PAIRLIST_OVERFLOW);
    }
}

// Algorithm 4 over the pairs of the beads [b_lo, b_hi) (whole replicas): bonds first, then
// the natives of every replica of the range, then the Verlet half list.
__global__ void __launch_bounds__(kPairThreads) k_pairs(StepArgs a, DevPairTables t, const float4 *__restrict__ pos,
                                                        int b_lo, int b_hi) {
    const int n = a.topo.n;
    const int nb = b_hi - b_lo;
    const int r_lo = b_lo / n;
    const int64_t n_nat = (int64_t)(nb / n) * t.n_nat_half;
    const int64_t n_ver = min((int64_t)t.voff[nb], t.vcap);
    const int64_t n_all = nb + n_nat + n_ver;
    const ForceParams &fp = a.fp;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_all;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (p < nb) {   // bond (gb, gb + 1)
            const int gb = b_lo + (int)p;
            const int i = gb % n;
            const float r0 = a.topo.bond_r0[i];
            if (!(r0 > 0.f)) continue;
            const float4 pi = pos[gb], pj = pos[gb + 1];
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            bool brk = false;
            const float c = fene_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), r0, fp, &brk);
            const float w = brk ? 1.f : 0.f;
            const float fx = c * dx, fy = c * dy, fz = c * dz;
            t.fb[2 * (size_t)gb + 1] = make_float4(fx, fy, fz, w);
            t.fb[2 * (size_t)gb + 2] = make_float4(-fx, -fy, -fz, w);
        } else if (p < nb + n_nat) {   // native contact (i, j), i < j
            const int64_t m = p - nb;
            const int rr = r_lo + (int)(m / t.n_nat_half);
            const int q = t.nat_half[m % t.n_nat_half];
            const int i = t.nat_owner[q], j = a.topo.nat_col[q];
            const float4 pi = pos[(size_t)rr * n + i], pj = pos[(size_t)rr * n + j];
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const float c = native_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), a.topo.nat_r0sq[q], fp);
            const float fx = c * dx, fy = c * dy, fz = c * dz;
            float4 *fn = t.fn + (size_t)rr * t.nnz;
            fn[q] = make_float4(fx, fy, fz, 0.f);
            fn[t.nat_mirror[q]] = make_float4(-fx, -fy, -fz, 0.f);
        } else {   // Verlet pair
            const int4 e = t.vpair[p - nb - n_nat];
            const float4 pi = pos[e.z], pj = pos[e.w];
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const float c = repulsive_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), fp);
            const float fx = c * dx, fy = c * dy, fz = c * dz;
            t.fv[e.x] = make_float4(fx, fy, fz, 0.f);
            if (e.y >= 0) t.fv[e.y] = make_float4(-fx, -fy, -fz, 0.f);
        }
    }
}

// Algorithm 5: the sum of bead gb's slots, L lanes per bead (lanes 0 and 1 take the two
// bond slots, all lanes stride over the native and Verlet slots), reduced by shuffles.
template <int L>
__device__ __forceinline__ float3 gather_slots(const StepArgs &a, const DevPairList &pl, const DevPairTables &t, int r,
                                               int i, int gb, int lane, const float4 *P, bool *broken) {
    float fx = 0.f, fy = 0.f, fz = 0.f;
    bool brk = false;
    xlink_force<L>(a.topo, a.fp, P, i, P[i], lane, fx, fy, fz, &brk);   // cross-links, gathered
    if (lane < 2) {
        const float4 v = t.fb[2 * (size_t)gb + lane];
        fx += v.x; fy += v.y; fz += v.z;
        brk = v.w != 0.f;
    }
    const float4 *fn = t.fn + (size_t)r * t.nnz;
    for (int q = a.topo.nat_row[i] + lane; q < a.topo.nat_row[i + 1]; q += L) {
        const float4 v = fn[q];
        fx += v.x; fy += v.y; fz += v.z;
    }
    const int p0 = pl.start[gb], p1 = p0 + pl.len[gb];
    for (int q = p0 + lane; q < p1; q += L) {
        const float4 v = t.fv[q];
        fx += v.x; fy += v.y; fz += v.z;
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(group_mask<L>(), fx, o, L);
        fy += __shfl_xor_sync(group_mask<L>(), fy, o, L);
        fz += __shfl_xor_sync(group_mask<L>(), fz, o, L);
    }
    *broken = brk;
    return make_float3(fx, fy, fz);
}

template <int L>
__global__ void __launch_bounds__(256) k_pairs_step(StepArgs a, DevPairList pl, DevPairTables t,
                                                    const float4 *__restrict__ pos_in, float4 *__restrict__ pos_out,
                                                    float4 *__restrict__ comp, int b_lo, int b_hi, int k_off) {
    const int th = blockIdx.x * blockDim.x + threadIdx.x;
    const int gb = b_lo + th / L;
    const int lane = th % L;
    if (gb >= b_hi) return;   // whole groups of L lanes leave together
    const int n = a.topo.n;
    const int r = gb / n, i = gb - r * n;
    const float4 *P = pos_in + (size_t)r * n;
    if (__any_sync(group_mask<L>(), *a.halt != 0 || a.rep_status[r] != 0)) {   // one decision per group
        if (lane == 0) pos_out[gb] = P[i];
        return;
    }
    const int64_t step = *a.d_step + k_off;
    bool broken = false;
    const float3 f = gather_slots<L>(a, pl, t, r, i, gb, lane, P, &broken);
    broken = __any_sync(group_mask<L>(), broken);
    if (lane != 0) return;
    advance_bead(a, r, i, gb, P, f, broken, step, pos_out, comp);
}

template <int L>
__global__ void __launch_bounds__(256) k_pairs_forces(StepArgs a, DevPairList pl, DevPairTables t,
                                                      const float4 *__restrict__ pos, float4 *__restrict__ force,
                                                      int b_lo, int b_hi, int64_t step) {
    const int th = blockIdx.x * blockDim.x + threadIdx.x;
    const int gb = b_lo + th / L;
    const int lane = th % L;
    if (gb >= b_hi) return;
    const int n = a.topo.n;
    const int r = gb / n, i = gb - r * n;
    bool broken = false;
    const float3 f = gather_slots<L>(a, pl, t, r, i, gb, lane, pos + (size_t)r * n, &broken);
    broken = __any_sync(group_mask<L>(), broken);
    if (lane != 0) return;
    bool overlap = false;
    const float3 fe = external_force(a, r, i, pos[gb], step, &overlap);
    force[gb] = make_float4(f.x + fe.x, f.y + fe.y, f.z + fe.z, (broken || overlap) ? 1.f : 0.f);
}

int pair_grid(const StepArgs &a, const DevPairTables &t, const SegRange &rg) {
    const int nb = rg.b_hi - rg.b_lo;
    const int64_t guess = (int64_t)nb + (int64_t)(nb / a.topo.n) * t.n_nat_half + 16 * (int64_t)nb;
    const int g = blocks_for(guess, kPairThreads);
    return g < 1 ? 1 : (g > kPairMaxBlocks ? kPairMaxBlocks : g);
}

}  // namespace

void launch_pair_index(const StepArgs &a, const DevPairList &pl, const DevPairTables &t, const SegRange &rg,
                       cudaStream_t s, int64_t *launches) {
    const int nb = rg.b_hi - rg.b_lo;
    if (nb <= 0) return;
    k_pair_count<<<blocks_for(nb, 256), 256, 0, s>>>(pl, t.vcount, a.topo.n, rg.b_lo, rg.b_hi);
    scan_exclusive(t.vcount, t.voff, nb, t.scan_tmp, s, launches);
    k_pair_fill<<<blocks_for(nb, 128), 128, 0, s>>>(pl, t, a.rep_status, a.topo.n, rg.b_lo, rg.b_hi);
    if (launches) *launches += 2;
}

void launch_pairs_step(const StepArgs &a, const DevPairList &pl, const DevPairTables &t, const float4 *pos_in,
                       float4 *pos_out, float4 *comp, const SegRange &rg, int32_t k_off, int lanes, cudaStream_t s,
                       int64_t *launches) {
    const int nb = rg.b_hi - rg.b_lo;
    if (nb <= 0) return;
    k_pairs<<<pair_grid(a, t, rg), kPairThreads, 0, s>>>(a, t, pos_in, rg.b_lo, rg.b_hi);
    const int blocks = blocks_for((int64_t)nb * lanes, 256);
    switch (lanes) {
    case 4: k_pairs_step<4><<<blocks, 256, 0, s>>>(a, pl, t, pos_in, pos_out, comp, rg.b_lo, rg.b_hi, k_off); break;
    case 16: k_pairs_step<16><<<blocks, 256, 0, s>>>(a, pl, t, pos_in, pos_out, comp, rg.b_lo, rg.b_hi, k_off); break;
    default: k_pairs_step<8><<<blocks, 256, 0, s>>>(a, pl, t, pos_in, pos_out, comp, rg.b_lo, rg.b_hi, k_off); break;
    }
    if (launches) *launches += 2;
}

void launch_pairs_forces(const StepArgs &a, const DevPairList &pl, const DevPairTables &t, const float4 *pos,
                         float4 *force, const SegRange &rg, int64_t step, cudaStream_t s, int64_t *launches) {
    const int nb = rg.b_hi - rg.b_lo;
    if (nb <= 0) return;
    k_pairs<<<pair_grid(a, t, rg), kPairThreads, 0, s>>>(a, t, pos, rg.b_lo, rg.b_hi);
    k_pairs_forces<8><<<blocks_for((int64_t)nb * 8, 256), 256, 0, s>>>(a, pl, t, pos, force, rg.b_lo, rg.b_hi, step);
    if (launches) *launches += 2;
}

}  // namespace sop
