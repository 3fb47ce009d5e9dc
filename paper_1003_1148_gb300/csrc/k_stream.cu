// Streamed schedule: per-step kernels over global memory (sm_103a).
//
//   setup      bonds and the native contact map (Eq. 1, Sec. IV.A), FP64 exact
//   rebuild    Verlet list (Sec. III.A, Algorithm 3) from a cell list built by
//              counting sort: per-segment bounding box -> cell id per bead ->
//              histogram -> exclusive scan -> scatter (one CTA per segment in shared
//              memory when every segment of the launch is small, else one kernel per
//              stage over global memory); then one warp per bead scans its 27 cells
//              and writes its row, ranked ascending
//   step       fused forces (Eq. 1 over bonds, natives and the list, each bead
//              gathered by a group of L lanes with a shuffle reduction, as in
//              the particle-based Algorithm 2) + cantilever/indenter + Philox
//              noise + compensated first-order update (Algorithm 7)
//   observables FP64 energy, pulling force, extension, Q and end-to-end distance
//
// A "segment" is one system of one replica; its beads are a contiguous range of
// the replica-major global bead index.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "sop_internal.h"
#include "sop_step.cuh"

namespace sop {

namespace {

// ---------------------------------------------------------------------------
// Setup: bonds and native map
// ---------------------------------------------------------------------------
__global__ void k_setup_bonds(const double *X, const int32_t *chain, float *bond_r0, double *bond_r0d, int32_t n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i + 1 < n && chain[i] == chain[i + 1]) {
        const double d2 = dist2_d(X[3 * i], X[3 * i + 1], X[3 * i + 2], X[3 * i + 3], X[3 * i + 4], X[3 * i + 5]);
        const double r0 = __dsqrt_rn(d2);
        bond_r0[i] = (float)r0;
        bond_r0d[i] = r0;
    } else {
        bond_r0[i] = -1.0f;
        bond_r0d[i] = -1.0;
    }
}

// Native candidates: same system, and |i-j| > 2 when in the same chain.
// Decided on the FP64 native coordinates: d^2 < cut^2 with d^2 = ((dx*dx+dy*dy)+dz*dz).
// An FP32 distance screens out pairs that are clearly beyond the cutoff.
template <bool kFill>
__global__ void k_native(const double *X, const int32_t *chain, const int32_t *sys, const int32_t *sys_lo,
                         int32_t n, double cut, int32_t *count, const int32_t *row, int32_t *col, double *r0,
                         float *r0sq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = sys[i];
    const int lo = sys_lo[s], hi = sys_lo[s + 1];
    const double xi = X[3 * i], yi = X[3 * i + 1], zi = X[3 * i + 2];
    const float fxi = (float)xi, fyi = (float)yi, fzi = (float)zi;
    const double cut2 = __dmul_rn(cut, cut);
    const float screen = (float)cut2 * 1.001f + 1e-3f;
    const int ci = chain[i];
    int c = 0;
    int out = kFill ? row[i] : 0;
    for (int j = lo; j < hi; ++j) {
        if (j == i) continue;
        const double xj = X[3 * j], yj = X[3 * j + 1], zj = X[3 * j + 2];
        const float dx = fxi - (float)xj, dy = fyi - (float)yj, dz = fzi - (float)zj;
        if (dx * dx + dy * dy + dz * dz > screen) continue;
        if (chain[j] == ci && (j - i <= 2 && i - j <= 2)) continue;
        const double d2 = dist2_d(xi, yi, zi, xj, yj, zj);
        if (d2 < cut2) {
            if (kFill) {
                col[out] = j;
                const double r = __dsqrt_rn(d2);
                r0[out] = r;
                r0sq[out] = (float)__dmul_rn(r, r);
                ++out;
            } else {
                ++c;
            }
        }
    }
    if (!kFill) count[i] = c;
}

// ---------------------------------------------------------------------------
// Exclusive scan (three passes: block sums, scan of sums, block scans)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanTile = 2 * kScanThreads;
static_assert(kScanTile == kScanTileElems, "scan_tmp_elems and the no-alloc scratch assume this tile");

__device__ __forceinline__ int warp_inclusive_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread across the block; returns the prefix and
// writes the block total to *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int *total) {
    __shared__ int warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int inc = warp_inclusive_scan(v);
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
        s = warp_inclusive_scan(s);
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const int before = (w > 0 ? warp_sums[w - 1] : 0) + inc - v;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void k_scan_reduce(const int32_t *in, int64_t n, int32_t *sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + 2 * threadIdx.x;
    int v = 0;
    if (base < n) v += in[base];
    if (base + 1 < n) v += in[base + 1];
    int total;
    block_exclusive_scan(v, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int32_t *sums, int64_t nb) {
    int carry = 0;
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        const int64_t k = base + threadIdx.x;
        const int v = k < nb ? sums[k] : 0;
        int total;
        const int ex = block_exclusive_scan(v, &total);
        if (k < nb) sums[k] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_scan_final(const int32_t *in, int32_t *out, int64_t n, const int32_t *sums, int64_t nb) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + 2 * threadIdx.x;
    const int a = base < n ? in[base] : 0;
    const int b = base + 1 < n ? in[base + 1] : 0;
    int total;
    const int ex = block_exclusive_scan(a + b, &total) + sums[blockIdx.x];
    if (base < n) out[base] = ex;
    if (base + 1 < n) out[base + 1] = ex + a;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[nb];
}

// ---------------------------------------------------------------------------
// Rebuild
// ---------------------------------------------------------------------------
struct RebuildArgs {
    const float4 *pos;
    float4 *snap;
    const int32_t *sys;
    const int32_t *chain;
    int32_t n, n_sys;
    int32_t g_lo, g_hi;
    float cell_edge;
    const int32_t *seg_bead_lo;
    const int32_t *seg_cell_base;
    float4 *seg_lo;
    int4 *seg_dims;
    int32_t *cell_of;
    int32_t *cell_cnt;
    int32_t *cell_start;   // range-relative offsets
    float4 *sorted;        // sorted[sorted_base + k]: position, bead index (int bits) in w
    int32_t sorted_base;   // first bead of the range
    int32_t cell_base0;    // first cell of the range
    int32_t *rep_status;
    int32_t *seg_box;
};

// Dims d and edge of the grid over [l, h]: cubic cells, edge from edge0 growing by a
// quarter (at most 64 times) until at most `budget` cells cover the box. False if none does.
__device__ bool fit_grid(const float l[3], const float h[3], float edge0, int budget, int d[3], float *edge) {
    float e0 = edge0;
    for (int it = 0; it < 64; ++it) {
        long long prod = 1;
        for (int k = 0; k < 3; ++k) {
            const float e = (h[k] - l[k]) / e0;
            d[k] = e < 1e6f ? (int)floorf(e) + 1 : 1000000;
            prod *= d[k];
        }
        if (prod <= budget) {
            *edge = e0;
            return true;
        }
        e0 *= 1.25f;
    }
    *edge = e0;
    return false;
}

// The cell grid of segment g from its bounding box [l, h]: cubic cells of edge >= cutoff,
// at most the segment's cell budget of them (fit_grid). A skipped segment (bad = true, or
// no grid fits) gets one empty cell and, when it holds beads, fails its replica.
__device__ void seg_grid(const RebuildArgs &a, int g, float l[3], const float h[3], bool bad, bool has_beads) {
    const int budget = a.seg_cell_base[g + 1] - a.seg_cell_base[g];
    float edge = a.cell_edge;
    int d[3] = {1, 1, 1};
    bool skip = bad;
    if (!skip && !fit_grid(l, h, a.cell_edge, budget, d, &edge)) {
        d[0] = d[1] = d[2] = 1;
        skip = true;
    }
    if (skip) {
        l[0] = l[1] = l[2] = 0.0f;
        if (has_beads) atomicCAS(&a.rep_status[g / a.n_sys], 0, (int32_t)SOP_ERR_NONFINITE);
    }
    a.seg_lo[g] = make_float4(l[0], l[1], l[2], 1.0f / edge);
    a.seg_dims[g] = make_int4(d[0], d[1], d[2], skip ? 0 : d[0] * d[1] * d[2]);
}

// Order-preserving integer key of a float (a < b <=> key(a) < key(b) for non-NaN values),
// so that several CTAs can merge minima and maxima with integer atomics.
__device__ __forceinline__ int f2key(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float key2f(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// Empty accumulator: minima at the largest key, maxima at the smallest, no bad position.
__device__ __forceinline__ void seg_box_reset(int32_t *bx) {
    bx[0] = bx[1] = bx[2] = INT_MAX;
    bx[3] = bx[4] = bx[5] = INT_MIN;
    bx[6] = 0;
    bx[7] = 0;
}

__global__ void k_seg_box_init(int32_t *seg_box, int n_seg) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n_seg) seg_box_reset(seg_box + 8 * g);
}

// Bounding boxes of large segments, gridDim.y CTAs per segment: each CTA reduces one slice
// of the segment's beads and merges it into the segment's accumulator (min and max are
// independent of the order of the merges).
__global__ void __launch_bounds__(256) k_seg_bbox(RebuildArgs a) {
    const int g = a.g_lo + blockIdx.x;
    if (a.rep_status[g / a.n_sys] != 0) return;   // CTA-uniform; k_seg_grid skips the segment
    const int lo = a.seg_bead_lo[g], hi = a.seg_bead_lo[g + 1];
    const int per = (hi - lo + gridDim.y - 1) / gridDim.y;
    const int s0 = lo + blockIdx.y * per, s1 = min(hi, s0 + per);
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    constexpr int kLd = 4;   // loads in flight per thread
    const int T = blockDim.x;
    for (int b0 = s0 + threadIdx.x; b0 < s1; b0 += kLd * T) {
        float4 pv[kLd];
#pragma unroll
        for (int u = 0; u < kLd; ++u) pv[u] = b0 + u * T < s1 ? a.pos[b0 + u * T] : a.pos[b0];
#pragma unroll
        for (int u = 0; u < kLd; ++u) {
            const float v[3] = {pv[u].x, pv[u].y, pv[u].z};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (!isfinite(v[k])) bad = true;
                mn[k] = fminf(mn[k], v[k]);
                mx[k] = fmaxf(mx[k], v[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = fminf(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
            mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
        }
    bad = __any_sync(0xffffffffu, bad);
    __shared__ float smn[3][8], smx[3][8];
    __shared__ int sbad[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        for (int k = 0; k < 3; ++k) { smn[k][w] = mn[k]; smx[k][w] = mx[k]; }
        sbad[w] = bad ? 1 : 0;
    }
    __syncthreads();
    if (threadIdx.x != 0 || s1 <= s0) return;
    int32_t *bx = a.seg_box + 8 * g;
    int any_bad = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) any_bad |= sbad[q];
    for (int k = 0; k < 3; ++k) {
        float l = smn[k][0], h = smx[k][0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) { l = fminf(l, smn[k][q]); h = fmaxf(h, smx[k][q]); }
        atomicMin(&bx[k], f2key(l));
        atomicMax(&bx[3 + k], f2key(h));
    }
    if (any_bad) atomicOr(&bx[6], 1);
}

// One thread per segment: the grid from the merged box (or the skip of a failed replica's
// segment: no bead is binned and its rows stay empty; its frozen positions may lie
// anywhere), then the accumulator back to its empty state. A live segment with a
// non-finite position or an extent that no grid of the budget covers fails its replica
// and is skipped too (seg_grid).
__global__ void k_seg_grid(RebuildArgs a, int n_seg_range, int32_t *pl_cursor, const int64_t *pl_seg_base) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_seg_range) return;
    const int g = a.g_lo + k;
    int32_t *bx = a.seg_box + 8 * g;
    if (a.rep_status[g / a.n_sys] != 0) {
        a.seg_lo[g] = make_float4(0.f, 0.f, 0.f, 1.0f / a.cell_edge);
        a.seg_dims[g] = make_int4(1, 1, 1, 0);
    } else {
        const int lo = a.seg_bead_lo[g], hi = a.seg_bead_lo[g + 1];
        float l[3], h[3];
        for (int q = 0; q < 3; ++q) { l[q] = key2f(bx[q]); h[q] = key2f(bx[3 + q]); }
        seg_grid(a, g, l, h, bx[6] != 0 || hi <= lo, hi > lo);
    }
    if (pl_cursor) pl_cursor[g] = (int32_t)pl_seg_base[g];
    seg_box_reset(bx);
}

__device__ __forceinline__ int cell_coord(float x, float lo, float inv, int dim) {
    int c = (int)((x - lo) * inv);
    c = c < 0 ? 0 : c;
    return c >= dim ? dim - 1 : c;
}

// Cell id of every bead, per-cell counts (histogram), and the snapshot of the
// positions the list is built from.
__global__ void k_cell_count(RebuildArgs a, int b_lo, int b_hi) {
    const int gb = b_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (gb >= b_hi) return;
    const int r = gb / a.n, i = gb - r * a.n;
    const int g = r * a.n_sys + a.sys[i];
    const float4 p = a.pos[gb];
    if (a.snap) a.snap[gb] = p;
    const float4 lo = a.seg_lo[g];
    const int4 d = a.seg_dims[g];
    if (d.w == 0) {   // skipped segment: the bead is not binned
        a.cell_of[gb] = -1;
        return;
    }
    int cx = 0, cy = 0, cz = 0;
    if (isfinite(p.x) && isfinite(p.y) && isfinite(p.z)) {
        cx = cell_coord(p.x, lo.x, lo.w, d.x);
        cy = cell_coord(p.y, lo.y, lo.w, d.y);
        cz = cell_coord(p.z, lo.z, lo.w, d.z);
    }
    const int gc = a.seg_cell_base[g] + (cz * d.y + cy) * d.x + cx;
    // the grid never exceeds the segment's budget (seg_grid); a cell outside it is
    // recorded as a failure of the replica and the bead goes to the segment's first cell
    if (gc < a.seg_cell_base[g] || gc >= a.seg_cell_base[g + 1]) {
        atomicCAS(&a.rep_status[r], 0, (int32_t)SOP_ERR_NONFINITE);
        a.cell_of[gb] = a.seg_cell_base[g];
        atomicAdd(&a.cell_cnt[a.seg_cell_base[g]], 1);
        return;
    }
    a.cell_of[gb] = gc;
    atomicAdd(&a.cell_cnt[gc], 1);
}

// Counting-sort scatter. Counts are consumed (they return to zero for the next rebuild).
__global__ void k_cell_scatter(RebuildArgs a, int b_lo, int b_hi) {
    const int gb = b_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (gb >= b_hi) return;
    const int gc = a.cell_of[gb];
    if (gc < 0) return;   // skipped segment
    const int slot = atomicSub(&a.cell_cnt[gc], 1) - 1;
    const float4 p = a.pos[gb];
    a.sorted[a.sorted_base + a.cell_start[gc - a.cell_base0] + slot] = make_float4(p.x, p.y, p.z, __int_as_float(gb));
}

constexpr int kBuildWarps = 8;
constexpr int kRowBuf = kRowCandidates;   // candidates a row may hold before it is an overflow
constexpr int kNatBuf = 64;    // native partners kept in shared memory per warp

struct BuildExtra {
    const int32_t *nat_row;
    const int32_t *nat_col;
    const int32_t *xb_row;      // cross-links (NULL: none): partners excluded like bonded ones
    const int32_t *xb_col;
    double cut2_d;
    float cut2_f;
    int32_t *pl_start;
    int32_t *pl_len;
    int32_t *pl_col;
    int32_t *pl_cursor;         // [n_seg]
    const int64_t *pl_seg_base; // [n_seg] first column of each segment
    const int64_t *pl_seg_end;  // [n_seg] capacity limit of each segment
    int32_t *rep_status;
};

// Is j a cross-link partner of bead i (a covalent bond, so not a Verlet-list pair)?
__device__ __forceinline__ bool xlinked(const BuildExtra &x, int i, int j) {
    for (int p = x.xb_row[i]; p < x.xb_row[i + 1]; ++p)
        if (x.xb_col[p] == j) return true;
    return false;
}

// Append the row of bead gb (cnt kept partners in the warp's buffer, in any order) to
// segment g's column range, ranked ascending; a row of more than kRowBuf partners, or one
// that does not fit the segment's capacity, is an overflow of replica r and stays empty.
// Called by the whole warp.
__device__ __forceinline__ void emit_row(const BuildExtra &x, const int32_t *buf, int cnt, int g, int r, int gb,
                                         int lane, int32_t *rep_status) {
    __syncwarp();
    int base = 0;
    bool ok = cnt <= kRowBuf;
    if (lane == 0 && ok) {
        base = atomicAdd(&x.pl_cursor[g], cnt);
        if ((int64_t)base + cnt > x.pl_seg_end[g]) ok = false;
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    if (!ok) {
        if (lane == 0) {
            set_status(&rep_status[r], (int32_t)SOP_ERR_PAIRLIST_OVERFLOW);
            x.pl_start[gb] = 0;
            x.pl_len[gb] = 0;
        }
        return;
    }
    for (int k = lane; k < cnt; k += 32) {
        const int v = buf[k];
        int rank = 0;
        for (int m2 = 0; m2 < cnt; ++m2) rank += buf[m2] < v;
        x.pl_col[base + rank] = v;
    }
    if (lane == 0) {
        x.pl_start[gb] = base;
        x.pl_len[gb] = cnt;
    }
}

// One warp per bead: scan the 27 neighbouring cells, keep partners j with |i-j| != 1 in
// a chain, j not native, j != i and r^2 < cut^2; order them ascending (rank sort) and
// append the row to the segment's column range. The 27 cells are 9 runs of 3 cells
// consecutive along x, hence 9 contiguous ranges of the cell-sorted positions; the warp
// walks their concatenation 32 candidates at a time, so every load of a pass is a
// coalesced read of sorted positions and no lane idles at the end of a short run.
__global__ void __launch_bounds__(kBuildWarps * 32) k_pl_build(RebuildArgs a, BuildExtra x, int b_lo, int b_hi) {
    __shared__ int32_t buf[kBuildWarps][kRowBuf];
    __shared__ int32_t nat[kBuildWarps][kNatBuf];
    __shared__ int32_t run_t0[kBuildWarps][9];   // first candidate of each run in the walk
    __shared__ int32_t run_q0[kBuildWarps][9];   // its first sorted slot
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = b_lo + blockIdx.x * kBuildWarps + w;
    if (gb >= b_hi) return;
    const int r = gb / a.n, i = gb - r * a.n;
    const int g = r * a.n_sys + a.sys[i];
    if (a.rep_status[r] != 0) {
        if (lane == 0) { x.pl_start[gb] = 0; x.pl_len[gb] = 0; }
        return;
    }
    const float4 pi = a.pos[gb];
    const int nlo = x.nat_row[i], nhi = x.nat_row[i + 1];
    const int nn = nhi - nlo;
    for (int k = lane; k < nn && k < kNatBuf; k += 32) nat[w][k] = x.nat_col[nlo + k];
    const int ci = a.chain[i];
    // bonded neighbours are excluded when they lie in the same chain
    const bool ex_lo = i > 0 && a.chain[i - 1] == ci;
    const bool ex_hi = i + 1 < a.n && a.chain[i + 1] == ci;
    const float4 lo = a.seg_lo[g];
    const int4 d = a.seg_dims[g];
    const int cx = cell_coord(pi.x, lo.x, lo.w, d.x);
    const int cy = cell_coord(pi.y, lo.y, lo.w, d.y);
    const int cz = cell_coord(pi.z, lo.z, lo.w, d.z);
    const int cbase = a.seg_cell_base[g] - a.cell_base0;
    const int rbase = r * a.n;
    // lane k < 9 reads run k (z = cz - 1 + k / 3, y = cy - 1 + k % 3): its slots [q0, q1)
    int q0 = 0, len = 0;
    if (lane < 9) {
        const int zz = cz - 1 + lane / 3, yy = cy - 1 + lane % 3;
        if (zz >= 0 && zz < d.z && yy >= 0 && yy < d.y) {
            const int x0 = cx > 0 ? cx - 1 : 0, x1 = cx + 1 < d.x ? cx + 1 : d.x - 1;
            const int c0 = cbase + (zz * d.y + yy) * d.x + x0;
            const int c1 = cbase + (zz * d.y + yy) * d.x + x1;
            q0 = a.cell_start[c0];
            len = a.cell_start[c1 + 1] - q0;
        }
    }
    int pre = len;   // inclusive prefix over the runs
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += t;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 8);
    if (lane < 9) {
        run_t0[w][lane] = pre - len;
        run_q0[w][lane] = q0;
    }
    __syncwarp();
    const bool nat_shared = nn <= kNatBuf;
    const float4 *S = a.sorted + a.sorted_base;
    int cnt = 0;
    for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        bool keep = false;
        int jl = 0;
        if (t < total) {
            // the last run starting at or before t (empty runs share their start with the
            // next run, so the last one is the non-empty run holding t)
            int k = t >= run_t0[w][8] ? 8 : 0;
            if (k == 0) {
                if (t >= run_t0[w][4]) k = 4;
                if (t >= run_t0[w][k + 2]) k += 2;
                if (t >= run_t0[w][k + 1]) k += 1;
            }
            const float4 pj = S[run_q0[w][k] + (t - run_t0[w][k])];
            jl = __float_as_int(pj.w) - rbase;
            if (jl != i && !(jl == i + 1 && ex_hi) && !(jl == i - 1 && ex_lo) &&
                within_cut(pi, pj, x.cut2_f, x.cut2_d)) {
                if (nat_shared) {   // the native row is ascending: binary search
                    int a0 = 0, a1 = nn;
                    while (a0 < a1) {
                        const int mid = (a0 + a1) >> 1;
                        if (nat[w][mid] < jl) a0 = mid + 1;
                        else a1 = mid;
                    }
                    keep = !(a0 < nn && nat[w][a0] == jl);
                } else {
                    keep = true;
                    for (int k2 = 0; k2 < nn; ++k2)
                        if (x.nat_col[nlo + k2] == jl) { keep = false; break; }
                }
                if (keep && x.xb_row) keep = !xlinked(x, i, jl);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int slot = cnt + __popc(m & ((1u << lane) - 1u));
            if (slot < kRowBuf) buf[w][slot] = jl;
        }
        cnt += __popc(m);
    }
    emit_row(x, buf[w], cnt, g, r, gb, lane, a.rep_status);
}

constexpr int kBruteBeads = kBruteMaxBeads;   // segments up to this size: k_pl_brute (no cell list)
constexpr int kBruteBlock = 16;   // beads per culling block (even: candidate pairs stay in one block)
constexpr int kBruteWarps = 16;   // warps per k_pl_brute CTA, one bead each
constexpr int kBruteSlice = kBruteSliceBeads;

struct BruteArgs {
    const int32_t *cta_lo;   // [n_seg+1] first k_pl_brute CTA of each segment
    int32_t *done;           // [n_seg] CTAs finished in the current build (0 between builds)
    int32_t *used;           // [n_seg] entries of the segment after its last build
    int32_t k_lo;            // cta_lo[g_lo]: first CTA of the launch
};

// The Verlet rows of segments of at most kBruteBeads beads without a cell list. Every CTA
// holds the positions of its segment in shared memory (x, y, z arrays, each padded to an
// even length with a point at infinity) and the bounding boxes of its blocks of 64
// consecutive beads; each warp takes one bead at a time and scans the blocks whose box lies
// within the screen distance of it, two candidates per lane with packed FP32x2 arithmetic.
// A candidate whose FP32 squared distance exceeds cut^2 (1 + 1e-4) is out by the FP32
// screen of within_cut; the others queue in shared memory and, 32 at a time (one per lane,
// so that the rare survivors of the screen do not idle the warp), take within_cut itself,
// the bonded, native and cross-link exclusions and the same compaction, ranking and
// overflow rules as k_pl_build, so the rows equal the cell-list rows. Each CTA also takes
// its segment's bounding box and fails the replica, as the cell list does, when a position
// is not finite or no grid of the segment's cell budget covers it. kBruteSlice beads per
// CTA; the last CTA of a segment to finish records the entries used and puts the segment's
// column cursor back to its first column for the next build.
__global__ void __launch_bounds__(kBruteWarps * 32) k_pl_brute(RebuildArgs a, BuildExtra x, BruteArgs bz) {
    extern __shared__ float soa[];
    __shared__ int32_t buf[kBruteWarps][kRowBuf];
    __shared__ int32_t nat[kBruteWarps][kNatBuf];
    __shared__ int32_t cand[kBruteWarps][96];   // screened candidates waiting for the exact tests
    __shared__ int32_t near_list[kBruteWarps][32];   // near blocks of the warp's current group
    __shared__ float smn[3][kBruteWarps], smx[3][kBruteWarps];
    __shared__ int sbad[kBruteWarps];
    __shared__ int s_ok;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cta = bz.k_lo + blockIdx.x;
    // the segment of this CTA: cta_lo[g] <= cta < cta_lo[g + 1] (empty segments own no CTA)
    int g = a.g_lo, g1 = a.g_hi;
    while (g1 - g > 1) {
        const int mid = (g + g1) >> 1;
        if (bz.cta_lo[mid] <= cta) g = mid;
        else g1 = mid;
    }
    const int lo = a.seg_bead_lo[g], hi = a.seg_bead_lo[g + 1], m = hi - lo, m2 = (m + 1) & ~1;
    float *sx = soa, *sy = soa + m2, *sz = soa + 2 * m2;
    const int nblk = (m + kBruteBlock - 1) / kBruteBlock;
    float *bx = soa + 3 * m2;   // box of block q: lo (x, y, z) at bx[q], bx[nblk + q], bx[2 nblk + q], hi after
    const int r = g / a.n_sys;
    const bool failed = a.rep_status[r] != 0;   // CTA-uniform
    if (!failed) {
        float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
        bool bad = false;
        // four loads in flight per thread (a loop of one load each would wait out the
        // latency of every load in turn)
        constexpr int kLd = 4;
        const int T = blockDim.x;
        for (int k0 = threadIdx.x; k0 < m; k0 += kLd * T) {
            float4 pv[kLd];
#pragma unroll
            for (int u = 0; u < kLd; ++u) pv[u] = k0 + u * T < m ? a.pos[lo + k0 + u * T] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < kLd; ++u) {
                const int k = k0 + u * T;
                if (k >= m) break;
                sx[k] = pv[u].x;
                sy[k] = pv[u].y;
                sz[k] = pv[u].z;
                const float v[3] = {pv[u].x, pv[u].y, pv[u].z};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (!isfinite(v[c])) bad = true;
                    mn[c] = fminf(mn[c], v[c]);
                    mx[c] = fmaxf(mx[c], v[c]);
                }
            }
        }
        if (threadIdx.x == 0 && m2 > m) sx[m] = sy[m] = sz[m] = INFINITY;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            for (int o = 16; o > 0; o >>= 1) {
                mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
                mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
            }
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            for (int c = 0; c < 3; ++c) { smn[c][w] = mn[c]; smx[c][w] = mx[c]; }
            sbad[w] = bad ? 1 : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float l[3], h[3];
            int any_bad = 0;
            for (int c = 0; c < 3; ++c) {
                l[c] = smn[c][0];
                h[c] = smx[c][0];
            }
            for (int q = 0; q < kBruteWarps; ++q) {
                any_bad |= sbad[q];
                for (int c = 0; c < 3; ++c) { l[c] = fminf(l[c], smn[c][q]); h[c] = fmaxf(h[c], smx[c][q]); }
            }
            int d[3];
            float edge;
            const bool ok = !any_bad && fit_grid(l, h, a.cell_edge, a.seg_cell_base[g + 1] - a.seg_cell_base[g], d, &edge);
            if (!ok) atomicCAS(&a.rep_status[r], 0, (int32_t)SOP_ERR_NONFINITE);
            s_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    const bool skip = failed || s_ok == 0;
    // bounding boxes of the blocks of kBruteBlock consecutive beads (consecutive beads of a
    // chain lie close together), one thread per block
    if (!skip)
        for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
            float l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int k = q * kBruteBlock; k < min(m, (q + 1) * kBruteBlock); ++k) {
                const float v[3] = {sx[k], sy[k], sz[k]};
#pragma unroll
                for (int c = 0; c < 3; ++c) { l[c] = fminf(l[c], v[c]); h[c] = fmaxf(h[c], v[c]); }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                bx[c * nblk + q] = l[c];
                bx[(3 + c) * nblk + q] = h[c];
            }
        }
    __syncthreads();
    const int b0 = lo + (cta - bz.cta_lo[g]) * kBruteSlice, b1 = min(hi, b0 + kBruteSlice);
    if (a.snap)
        for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) a.snap[b] = a.pos[b];
    const int rbase = r * a.n, jbase = lo - rbase;   // replica-local index of the segment's first bead
    const float band = x.cut2_f * 1e-4f, screen = x.cut2_f + band;
    const float2 m1 = make_float2(-1.f, -1.f);
    for (int gb = b0 + w; gb < b1; gb += kBruteWarps) {
        if (skip) {
            if (lane == 0) { x.pl_start[gb] = 0; x.pl_len[gb] = 0; }
            continue;
        }
        const int i = gb - rbase;
        const int nlo = x.nat_row[i], nn = x.nat_row[i + 1] - nlo;
        __syncwarp();   // the previous bead's row is out of buf and nat
        for (int k = lane; k < nn && k < kNatBuf; k += 32) nat[w][k] = x.nat_col[nlo + k];
        const int ci = a.chain[i];
        const bool ex_lo = i > 0 && a.chain[i - 1] == ci;
        const bool ex_hi = i + 1 < a.n && a.chain[i + 1] == ci;
        const bool nat_shared = nn <= kNatBuf;
        const float4 pi = make_float4(sx[gb - lo], sy[gb - lo], sz[gb - lo], 0.f);
        const float2 px = make_float2(pi.x, pi.x), py = make_float2(pi.y, pi.y), pz = make_float2(pi.z, pi.z);
        __syncwarp();
        int cnt = 0, pend = 0;
        // the exact tests of the candidates that passed the FP32 screen, cand[w][0 .. np)
        // with np <= 32, one per lane; kept partners are compacted into buf[w]
        auto settle = [&](int np) {
            bool keep = false;
            int jl = 0;
            if (lane < np) {
                const int kk = cand[w][lane];
                jl = jbase + kk;
                if (jl != i && !(jl == i + 1 && ex_hi) && !(jl == i - 1 && ex_lo) &&
                    within_cut(pi, make_float4(sx[kk], sy[kk], sz[kk], 0.f), x.cut2_f, x.cut2_d)) {
                    if (nat_shared) {   // the native row is ascending: binary search
                        int a0 = 0, a1 = nn;
                        while (a0 < a1) {
                            const int mid = (a0 + a1) >> 1;
                            if (nat[w][mid] < jl) a0 = mid + 1;
                            else a1 = mid;
                        }
                        keep = !(a0 < nn && nat[w][a0] == jl);
                    } else {
                        keep = true;
                        for (int q = 0; q < nn; ++q)
                            if (x.nat_col[nlo + q] == jl) { keep = false; break; }
                    }
                    if (keep && x.xb_row) keep = !xlinked(x, i, jl);
                }
            }
            const unsigned msk = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int slot = cnt + __popc(msk & ((1u << lane) - 1u));
                if (slot < kRowBuf) buf[w][slot] = jl;
            }
            cnt += __popc(msk);
        };
        const unsigned below = (1u << lane) - 1u;
        // candidates k0 and k0 + 1 (k0 even, or k0 >= m2 for none): screened, survivors queued
        auto scan_pair = [&](int k0) {
            bool in0 = false, in1 = false;
            if (k0 < m2) {
                const float2 X = *reinterpret_cast<const float2 *>(sx + k0);
                const float2 Y = *reinterpret_cast<const float2 *>(sy + k0);
                const float2 Z = *reinterpret_cast<const float2 *>(sz + k0);
                const float2 dx = __ffma2_rn(X, m1, px);   // pi - pj, exactly rounded
                const float2 dy = __ffma2_rn(Y, m1, py);
                const float2 dz = __ffma2_rn(Z, m1, pz);
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                in0 = r2.x <= screen;
                in1 = r2.y <= screen;
            }
            const unsigned q0 = __ballot_sync(0xffffffffu, in0), q1 = __ballot_sync(0xffffffffu, in1);
            if ((q0 | q1) == 0u) return;
            if (in0) cand[w][pend + __popc(q0 & below)] = k0;
            pend += __popc(q0);
            if (in1) cand[w][pend + __popc(q1 & below)] = k0 + 1;
            pend += __popc(q1);
            if (pend >= 32) {
                __syncwarp();
                settle(32);
                // move the rest (at most 63) to the front
                const int v0 = lane + 32 < pend ? cand[w][lane + 32] : 0;
                const int v1 = lane + 64 < pend ? cand[w][lane + 64] : 0;
                __syncwarp();
                if (lane + 32 < pend) cand[w][lane] = v0;
                if (lane + 64 < pend) cand[w][lane + 32] = v1;
                pend -= 32;
                __syncwarp();
            }
        };
        // blocks whose box lies within the screen distance of bead i (the box is no farther
        // than any of its beads, so no candidate the exact test keeps is culled), 32 blocks at a
        // time: their near blocks are listed, and the warp walks the concatenation of their
        // beads 64 at a time, two per lane
        for (int q = 0; q < nblk; q += 32) {
            bool near = false;
            if (q + lane < nblk) {
                const float v[3] = {pi.x, pi.y, pi.z};
                float d2 = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float e = fmaxf(fmaxf(bx[c * nblk + q + lane] - v[c], v[c] - bx[(3 + c) * nblk + q + lane]), 0.f);
                    d2 = fmaf(e, e, d2);
                }
                near = d2 <= screen;
            }
            const unsigned bm = __ballot_sync(0xffffffffu, near);
            if (bm == 0u) continue;
            if (near) near_list[w][__popc(bm & below)] = q + lane;
            __syncwarp();
            const int nc = __popc(bm) * kBruteBlock;
            for (int t0 = 0; t0 < nc; t0 += 64) {
                const int t = t0 + 2 * lane;
                scan_pair(t < nc ? near_list[w][t / kBruteBlock] * kBruteBlock + t % kBruteBlock : m2);
            }
            __syncwarp();   // near_list is rewritten by the next group
        }
        __syncwarp();
        if (pend > 0) settle(pend);
        emit_row(x, buf[w], cnt, g, r, gb, lane, a.rep_status);
    }
    // the last CTA of the segment records its entries and resets its cursor
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int n_cta = bz.cta_lo[g + 1] - bz.cta_lo[g];
        if (atomicAdd(&bz.done[g], 1) == n_cta - 1) {
            __threadfence();
            const int32_t base = (int32_t)x.pl_seg_base[g];
            bz.used[g] = atomicAdd(&x.pl_cursor[g], 0) - base;
            x.pl_cursor[g] = base;
            bz.done[g] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Forces and the fused step
// ---------------------------------------------------------------------------
// Sum of the Eq. 1 pair forces on bead i of replica r, gathered by L lanes
// (particle-based, Algorithm 2): lanes stride over the native row and the
// Verlet row, bonds go to lanes 0 and 1, a shuffle reduction leaves the sum in
// every lane. pi = P[i]; [n0, n1) and [p0, p1) are the bead's native and Verlet rows.
template <int L>
__device__ __forceinline__ float3 gather_force_at(const StepArgs &a, const DevPairList &pl, const float4 *P, int i,
                                                  int lane, float4 pi, int n0, int n1, int p0, int p1,
                                                  bool *broken) {
    const DevTopo &t = a.topo;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    bool brk = false;
    if (lane == 0 && i > 0) {
        const float r0 = t.bond_r0[i - 1];
        if (r0 > 0.f) {
            const float4 pj = P[i - 1];
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const float c = fene_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), r0, a.fp, &brk);
            fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
        }
    }
    if (lane == (1 % L) && i + 1 < t.n) {
        const float r0 = t.bond_r0[i];
        if (r0 > 0.f) {
            const float4 pj = P[i + 1];
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const float c = fene_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), r0, a.fp, &brk);
            fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
        }
    }
    xlink_force<L>(t, a.fp, P, i, pi, lane, fx, fy, fz, &brk);
#pragma unroll 2
    for (int p = n0 + lane; p < n1; p += L) {
        const uint2 e = t.nat_ent[p];   // partner and r0^2 in one load
        const float4 pj = P[e.x];
        const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        const float c = native_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), __uint_as_float(e.y), a.fp);
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
#pragma unroll 2
    for (int p = p0 + lane; p < p1; p += L) {
        const float4 pj = P[pl.col[p]];
        const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        const float c = repulsive_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), a.fp);
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
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
__device__ __forceinline__ float3 gather_force(const StepArgs &a, const DevPairList &pl, const float4 *P, int i,
                                               int gb, int lane, bool *broken) {
    const int p0 = pl.start[gb];
    return gather_force_at<L>(a, pl, P, i, lane, P[i], a.topo.nat_row[i], a.topo.nat_row[i + 1], p0,
                              p0 + pl.len[gb], broken);
}

// advance_bead for an overdamped step with Philox noise, given the bead's position
// pi = P[i], compensation c = comp[gb] and flags fl loaded, and its noise g drawn, before
// the force gather, so that none of them waits behind it. The same decisions as
// advance_bead and the same Algorithm 7 update as update_position, in the same order.
__device__ __forceinline__ void advance_bead_pre(const StepArgs &a, int r, int i, int gb, float4 pi, float4 c,
                                                 uint8_t fl, float3 g, float3 f, bool broken, int64_t step,
                                                 float4 *pos_out, float4 *comp) {
    if (broken) {
        set_status(&a.rep_status[r], (int32_t)SOP_ERR_FENE_BREAK);
        pos_out[gb] = pi;
        return;
    }
    bool overlap = false;
    const float3 fe = external_force(a, r, i, pi, step, &overlap);
    if (overlap) {
        set_status(&a.rep_status[r], (int32_t)SOP_ERR_INDENTER_OVERLAP);
        pos_out[gb] = pi;
        return;
    }
    if (fl & kFlagFixed) {
        pos_out[gb] = pi;
        return;
    }
    const float3 F = make_float3(f.x + fe.x, f.y + fe.y, f.z + fe.z);
    float4 pn = pi, cn = c;
    kahan_add(pn.x, cn.x, fmaf(F.x, a.fp.mob, g.x * a.fp.amp));
    kahan_add(pn.y, cn.y, fmaf(F.y, a.fp.mob, g.y * a.fp.amp));
    kahan_add(pn.z, cn.z, fmaf(F.z, a.fp.mob, g.z * a.fp.amp));
    if (!(isfinite(pn.x) && isfinite(pn.y) && isfinite(pn.z))) {
        set_status(&a.rep_status[r], (int32_t)SOP_ERR_NONFINITE);
        pos_out[gb] = pi;
        return;
    }
    comp[gb] = cn;
    pos_out[gb] = pn;
}

// One step of bead gb by its group of L lanes (lane = this thread's lane in the group).
template <int L>
// (No __restrict__ here: in k_step_coop the same layers are read and written by different
// steps of one launch, so no load may take the read-only path.)
__device__ __forceinline__ void step_bead(const StepArgs &a, const DevPairList &pl, const float4 *pos_in,
                                          float4 *pos_out, float4 *comp, int gb, int lane, int k_off) {
    const int n = a.topo.n;
    const int r = gb / n, i = gb - r * n;
    const float4 *P = pos_in + (size_t)r * n;
    // Loads issued together, all in bounds whatever the replica's state: the stop decision,
    // the step, and the bead's position, row bounds, compensation and flags, so that the
    // stop test, the update and the gather's first loads do not each wait in turn.
    const bool stop = *a.halt != 0 || a.rep_status[r] != 0;
    const int64_t step = *a.d_step + k_off;
    const float4 pi = P[i];
    const int n0 = a.topo.nat_row[i], n1 = a.topo.nat_row[i + 1];
    const int p0 = pl.start[gb], p1 = p0 + pl.len[gb];
    const float4 c = comp[gb];
    const uint8_t fl = a.topo.flags[i];
    if (__any_sync(group_mask<L>(), stop)) {   // one decision per group
        if (lane == 0) pos_out[gb] = pi;
        return;
    }
    // The Philox noise does not depend on the forces: in an overdamped step every lane of
    // the group draws it here (the same words), off the path that follows the reduction.
    // Hybrid Taus noise (drawn only when the bead moves) and the underdamped update stay
    // in advance_bead.
    const bool pre = a.taus == nullptr && a.vel == nullptr;
    float3 g = make_float3(0.f, 0.f, 0.f);
    if (pre) g = bead_noise(a.seed + (uint64_t)r, step, (uint32_t)i);
    bool broken = false;
    const float3 f = gather_force_at<L>(a, pl, P, i, lane, pi, n0, n1, p0, p1, &broken);
    broken = __any_sync(group_mask<L>(), broken);
    if (lane != 0) return;
    if (pre) advance_bead_pre(a, r, i, gb, pi, c, fl, g, f, broken, step, pos_out, comp);
    else advance_bead(a, r, i, gb, P, f, broken, step, pos_out, comp);
}

template <int L>
__global__ void __launch_bounds__(256) k_step(StepArgs a, DevPairList pl, const float4 *__restrict__ pos_in,
                                              float4 *__restrict__ pos_out, float4 *__restrict__ comp, int b_lo,
                                              int b_hi, int k_off) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int gb = b_lo + t / L;
    if (gb >= b_hi) return;   // whole groups of L lanes leave together
    step_bead<L>(a, pl, pos_in, pos_out, comp, gb, t % L, k_off);
}

// Grid-wide barrier of a cooperative launch (all CTAs co-resident). Thread 0 of each CTA
// reads the generation, arrives on the counter with an acquire-release add (releasing the
// CTA's writes, which the __syncthreads before it orders first); the last arrival resets
// the counter and publishes the next generation with a release add; the others poll the
// generation with acquire loads (first without sleeping, then with a short back-off) up to
// a bound. False when the wait gave up (a CTA that never arrived): the caller marks its
// replicas SOP_ERR_TIMEOUT and returns.
constexpr long long kBarrierSpins = 1ll << 22;   // about a second with the back-off below
constexpr int kBarrierHotPolls = 2048;           // polls before the back-off starts

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned *p, unsigned x) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(x) : "memory");
    return old;
}

__device__ __forceinline__ void red_add_release_gpu(unsigned *p, unsigned x) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}

__device__ __forceinline__ void st_relaxed_gpu(unsigned *p, unsigned x) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}

__device__ bool grid_barrier(unsigned *bar) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned *gen = bar + 1;
        const unsigned g = ld_acquire_gpu(gen);   // before arriving: the last arrival changes it only after
        ok = 1;
        if (atom_add_acq_rel_gpu(bar, 1u) == gridDim.x - 1) {
            st_relaxed_gpu(bar, 0u);              // nobody arrives again before the next generation
            red_add_release_gpu(gen, 1u);
        } else {
            long long it = 0;
            while (ld_acquire_gpu(gen) == g) {
                if (++it > kBarrierSpins) {
                    ok = 0;
                    break;
                }
                if (it > kBarrierHotPolls) __nanosleep(64);
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

// k_steps steps of the beads [b_lo, b_hi) in one cooperative launch: a grid-stride loop of
// k_step's work per step, a grid barrier between steps; the layers alternate from pos_a.
// The same arithmetic as k_step, so the results are bit-identical to k_steps launches.
template <int L>
__global__ void __launch_bounds__(256) k_step_coop(StepArgs a, DevPairList pl, float4 *pos_a, float4 *pos_b,
                                                   float4 *comp, int b_lo, int b_hi, int k_off, int k_steps,
                                                   unsigned *bar) {
    const int64_t n_thr = (int64_t)(b_hi - b_lo) * L;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;   // a multiple of L: groups stay whole
    for (int k = 0; k < k_steps; ++k) {
        const float4 *pin = (k & 1) ? pos_b : pos_a;
        float4 *pout = (k & 1) ? pos_a : pos_b;
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_thr; t += stride)
            step_bead<L>(a, pl, pin, pout, comp, b_lo + (int)(t / L), (int)(t % L), k_off + k);
        if (k + 1 < k_steps && !grid_barrier(bar)) {
            if (threadIdx.x == 0)
                for (int r = b_lo / a.topo.n; r * a.topo.n < b_hi; ++r)
                    atomicCAS(&a.rep_status[r], 0, (int32_t)SOP_ERR_TIMEOUT);
            return;
        }
    }
}

// The same step for large systems, with the tail spread over the lanes: a group of L
// lanes gathers the forces of L consecutive beads one after another (the same gather and
// reduction as k_step, so every force is bit-identical), lane q keeps bead q's sum, and
// then every lane draws the noise and updates its own bead. k_step leaves L - 1 lanes of
// each group idle through the noise and the update; here none is.
template <int L>
__global__ void __launch_bounds__(256) k_step_spread(StepArgs a, DevPairList pl, const float4 *__restrict__ pos_in,
                                                     float4 *__restrict__ pos_out, float4 *__restrict__ comp,
                                                     int b_lo, int b_hi, int k_off) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = t % L;
    const int gb0 = b_lo + (t - lane);   // first bead of the group
    if (gb0 >= b_hi) return;             // whole groups of L lanes leave together
    const int n = a.topo.n;
    const bool halted = *a.halt != 0;
    float3 mine = make_float3(0.f, 0.f, 0.f);
    bool mine_broken = false;
    for (int q = 0; q < L && gb0 + q < b_hi; ++q) {   // the same trip count in every lane of the group
        const int gb = gb0 + q;
        const int r = gb / n, i = gb - r * n;
        // one decision for the group (its lanes then shuffle together)
        if (__any_sync(group_mask<L>(), halted || a.rep_status[r] != 0)) continue;
        bool broken = false;
        const float3 f = gather_force<L>(a, pl, pos_in + (size_t)r * n, i, gb, lane, &broken);
        broken = __any_sync(group_mask<L>(), broken);
        if (lane == q) {
            mine = f;
            mine_broken = broken;
        }
    }
    const int gb = gb0 + lane;
    if (gb >= b_hi) return;
    const int r = gb / n, i = gb - r * n;
    const float4 *P = pos_in + (size_t)r * n;
    if (halted || a.rep_status[r] != 0) {
        pos_out[gb] = P[i];
        return;
    }
    advance_bead(a, r, i, gb, P, mine, mine_broken, *a.d_step + k_off, pos_out, comp);
}

template <int L>
__global__ void __launch_bounds__(256) k_forces(StepArgs a, DevPairList pl, const float4 *__restrict__ pos,
                                                float4 *__restrict__ force, int b_lo, int b_hi, int64_t step) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int gb = b_lo + t / L;
    const int lane = t % L;
    if (gb >= b_hi) return;
    const int n = a.topo.n;
    const int r = gb / n, i = gb - r * n;
    const float4 *P = pos + (size_t)r * n;
    bool broken = false;
    float3 f = gather_force<L>(a, pl, P, i, gb, lane, &broken);
    broken = __any_sync(group_mask<L>(), broken);
    if (lane != 0) return;
    bool overlap = false;
    const float3 fe = external_force(a, r, i, P[i], step, &overlap);
    force[gb] = make_float4(f.x + fe.x, f.y + fe.y, f.z + fe.z, (broken || overlap) ? 1.f : 0.f);
}

// ---------------------------------------------------------------------------
// Observables (FP64)
// ---------------------------------------------------------------------------
constexpr int kObsLanes = 4;                        // lanes per bead in k_obs_partial's counting
constexpr int kObsThreads = kObsChunkBeads * kObsLanes;
static_assert(kObsChunkBeads == 32, "k_obs_partial scans its chunk's beads in one warp");

// Sum of v[0..5] over the CTA, valid in thread 0: a fixed shuffle tree in each warp, then
// thread 0 adds the warps in order. The grouping depends only on the launch shape, so
// the result is the same on every run. sh holds 6 doubles per warp.
__device__ __forceinline__ void block_sum6_d(double v[6], double *sh) {
#pragma unroll
    for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < 6; ++k) sh[w * 6 + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
            for (int k = 0; k < 6; ++k) v[k] += sh[q * 6 + k];
}

struct ObsArgs {
    StepArgs a;
    DevPairList pl;
    DevObs o;
    const float4 *pos;
    int32_t k_off;
    int32_t gate;
    int32_t chunk0;           // first chunk of the launch
    double eps_h, eps_l, sigma, k_fene, R0;
    const double *bond_r0d;   // [n] FP64 bond lengths
};

// Partial FP64 sums of one chunk of beads (energy, pull force, extension, formed native
// contacts, indenter force, end-to-end distance). Each pair is taken once, from its lower
// index: rows are ascending (the list builders and the native map write them so), so the
// partners j > i of bead i are a suffix of each of its rows. The CTA counts those suffixes
// (kObsLanes lanes per bead), lays them end to end, and its threads then stride over the
// concatenation, native pairs first: the FP64 pipe, narrow on this GPU and busy for a
// whole warp instruction whatever the number of active lanes, sees full warps except at
// the tails. The terms of the beads themselves (bond, pulling, indenter, end-to-end
// distance) take one thread per bead. The grouping of every sum depends only on the
// chunk, so the result is the same on every run.
__global__ void __launch_bounds__(kObsThreads) k_obs_partial(ObsArgs q) {
    constexpr int kB = kObsThreads / kObsLanes;   // beads of a chunk
    __shared__ int s_nat0[kB], s_ver0[kB];        // first suffix entry of each bead's rows
    __shared__ int s_natp[kB + 1], s_verp[kB + 1]; // exclusive prefix of the suffix lengths
    const int64_t step = *q.a.d_step + q.k_off;
    if (q.gate > 0 && step % q.gate != 0) return;
    const int ch = q.chunk0 + blockIdx.x;
    const int lo = q.o.chunk_lo[ch], hi = q.o.chunk_hi[ch];
    const DevTopo &t = q.a.topo;
    const DevExternal &e = q.a.ext;
    const int n = t.n;
    const int lane = threadIdx.x & 31;
    // a chunk lies in one segment, hence in one replica r; bead b of the chunk is i0 + b
    const int r = lo / n, i0 = lo - r * n;
    const float4 *P = q.pos + (size_t)r * n;
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // E, fpull, ext, formed, fwall, ree
    {   // suffix lengths: kObsLanes lanes per bead count the entries above the bead's index
        const int bl = threadIdx.x / kObsLanes, gl = threadIdx.x % kObsLanes;
        const int gb = lo + bl;
        int cn = 0, cv = 0, n1 = 0, v1 = 0;
        if (gb < hi) {
            const int i = i0 + bl;
            n1 = t.nat_row[i + 1];
            for (int p = t.nat_row[i] + gl; p < n1; p += kObsLanes) cn += t.nat_col[p] > i;
            v1 = q.pl.start[gb] + q.pl.len[gb];
            for (int p = q.pl.start[gb] + gl; p < v1; p += kObsLanes) cv += q.pl.col[p] > i;
        }
#pragma unroll
        for (int o = kObsLanes / 2; o > 0; o >>= 1) {
            cn += __shfl_xor_sync(0xffffffffu, cn, o, kObsLanes);
            cv += __shfl_xor_sync(0xffffffffu, cv, o, kObsLanes);
        }
        if (gl == 0) {
            s_nat0[bl] = n1 - cn;
            s_ver0[bl] = v1 - cv;
            s_natp[bl + 1] = cn;
            s_verp[bl + 1] = cv;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {   // inclusive scans of the lengths (kB <= 32)
        int a = lane < kB ? s_natp[lane + 1] : 0, b = lane < kB ? s_verp[lane + 1] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ta = __shfl_up_sync(0xffffffffu, a, o), tb = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) { a += ta; b += tb; }
        }
        if (lane < kB) { s_natp[lane + 1] = a; s_verp[lane + 1] = b; }
        if (lane == 0) { s_natp[0] = 0; s_verp[0] = 0; }
    }
    __syncthreads();
    // the bead of flat entry f: the last b with prefix[b] <= f
    auto bead_of = [](const int *pre, int f) {
        int b = 0;
#pragma unroll
        for (int step2 = kB / 2; step2 > 0; step2 >>= 1)
            if (pre[b + step2] <= f) b += step2;
        return b;
    };
    const double sig2 = q.sigma * q.sigma;
    const int tot_nat = s_natp[kB], tot_ver = s_verp[kB];
    for (int f = threadIdx.x; f < tot_nat; f += kObsThreads) {
        const int b = bead_of(s_natp, f);
        const int p = s_nat0[b] + (f - s_natp[b]);
        const float4 pi = P[i0 + b], pj = P[t.nat_col[p]];
        float d2f;
        const double d2 = dist2_two(pi, pj, &d2f);
        const double r0 = t.nat_r0[p];
        const double s = r0 * r0 * rcp_seeded(d2, d2f);
        const double s3 = s * s * s;
        acc[0] = fma(q.eps_h, s3 * s3 - 2.0 * s3, acc[0]);
        if (native_formed(d2, r0, pi, pj)) acc[3] += 1.0;
    }
    for (int f = threadIdx.x; f < tot_ver; f += kObsThreads) {
        const int b = bead_of(s_verp, f);
        const float4 pi = P[i0 + b], pj = P[q.pl.col[s_ver0[b] + (f - s_verp[b])]];
        float d2f;
        const double d2 = dist2_two(pi, pj, &d2f);
        const double c = sig2 * rcp_seeded(d2, d2f);
        acc[0] = fma(q.eps_l, c * c * c, acc[0]);
    }
    const int gb = lo + (int)threadIdx.x;
    if (threadIdx.x < kB && gb < hi) {   // the terms of the bead itself
        const int i = i0 + (int)threadIdx.x;
        const float4 pi = P[i];
        const double xi = pi.x, yi = pi.y, zi = pi.z;
        if (t.bond_r0[i] > 0.f) {
            const float4 pj = P[i + 1];
            float d2f;
            const double d2 = dist2_two(pi, pj, &d2f);
            const double rr = sqrt_seeded(d2, d2f);
            const double R02 = q.R0 * q.R0;
            const double dr = rr - q.bond_r0d[i];
            const double arg = 1.0 - dr * dr * (1.0 / R02);
            if (arg > 0.0) acc[0] += -0.5 * q.k_fene * R02 * log(arg);
        }
        if (t.xb_row)   // cross-links, each from its lower index
            for (int p = t.xb_row[i]; p < t.xb_row[i + 1]; ++p) {
                const int j = t.xb_col[p];
                if (j < i) continue;
                float d2f;
                const double d2 = dist2_two(pi, P[j], &d2f);
                const double R02 = q.R0 * q.R0;
                const double dr = sqrt_seeded(d2, d2f) - t.xb_r0d[p];
                const double arg = 1.0 - dr * dr * (1.0 / R02);
                if (arg > 0.0) acc[0] += -0.5 * q.k_fene * R02 * log(arg);
            }
        if (t.flags[i] & kFlagPulled) {
            const int qq = e.pull_of_sys[t.sys[i]];
            if (qq >= 0 && e.pull_bead[qq] == i) {
                const double tt = e.pull_v[qq] * ((double)step - e.pull_n0[qq]);
                const double *tip0 = e.pull_tip0 + ((size_t)r * e.n_pull + qq) * 3;
                const double *dir = e.pull_dir + 3 * qq;
                const double x[3] = {xi, yi, zi};
                double fs = 0.0;
                for (int k = 0; k < 3; ++k) fs += e.pull_ks[qq] * (tip0[k] + tt * dir[k] - x[k]) * dir[k];
                acc[1] += fs;
                const float4 pa = P[e.pull_anchor[qq]];
                acc[2] += __dsqrt_rn(dist2_d(xi, yi, zi, pa.x, pa.y, pa.z));
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
                const double qq = q.sigma * rcp_fast(rho);
                const double q2 = qq * qq;
                const double q6 = q2 * q2 * q2;
                const double coef = 6.0 * q.eps_l * q6 * rcp_fast(rho * rr);
                acc[4] += coef * ((ex * e.ind_dir[0] + ey * e.ind_dir[1]) + ez * e.ind_dir[2]);
            }
        }
        if (t.flags[i] & kFlagFirstOfSystem) {
            const float4 pl_ = P[t.sys_ree_last[t.sys[i]]];
            acc[5] += __dsqrt_rn(dist2_d(xi, yi, zi, pl_.x, pl_.y, pl_.z));
        }
    }
    __shared__ double sh[6 * (kObsThreads / 32)];
    block_sum6_d(acc, sh);
    if (threadIdx.x == 0) {
        double *out = q.o.partial + (size_t)ch * 8;
        for (int k = 0; k < 6; ++k) out[k] = acc[k];
        out[6] = 0;
        out[7] = 0;
    }
}

// Sum of the chunk partials [ch_lo, ch_hi) over the CTA (thread t adds chunks t, t + T, ...
// in order, then block_sum6_d); valid in thread 0.
__device__ __forceinline__ void chunk_sums(const DevObs &o, int ch_lo, int ch_hi, double acc[6], double *sh) {
    for (int k = 0; k < 6; ++k) acc[k] = 0.0;
    for (int ch = ch_lo + threadIdx.x; ch < ch_hi; ch += blockDim.x)
        for (int k = 0; k < 6; ++k) acc[k] += o.partial[(size_t)ch * 8 + k];
    block_sum6_d(acc, sh);
}

constexpr int kObsFinalMaxThreads = 256;

// The record of segment g at `step` from its chunks' partial sums, into ring slot `slot`.
// Called by the whole CTA; thread 0 writes the record.
__device__ void write_record(const ObsArgs &q, int g, int64_t step, int64_t slot) {
    __shared__ double sh[6 * (kObsFinalMaxThreads / 32)];
    double acc[6];
    chunk_sums(q.o, q.o.seg_chunk_lo[g], q.o.seg_chunk_lo[g + 1], acc, sh);
    if (threadIdx.x != 0) return;
    const int ns = q.a.topo.n_sys;
    const int r = g / ns, s = g - r * ns;
    const DevExternal &e = q.a.ext;
    sop_record rec;
    rec.step = (double)step;
    rec.replica = (double)r;
    rec.system = (double)s;
    rec.energy = acc[0];
    const bool pulled = e.pull_of_sys[s] >= 0;
    rec.f_ext = pulled ? acc[1] : (e.has_indenter ? acc[4] : 0.0);
    rec.extension = pulled ? acc[2] : (e.has_indenter ? e.ind_v * ((double)step - e.ind_n0) : 0.0);
    const int np = q.a.topo.sys_nat_pairs[s];
    rec.q = np > 0 ? acc[3] / (double)np : 0.0;
    if (q.o.q_every > 0 && step % q.o.q_every != 0) rec.q = __longlong_as_double(0x7ff8000000000000LL);
    rec.r_ee = acc[5];
    q.o.ring[slot] = rec;
}

// One CTA per segment.
__global__ void __launch_bounds__(kObsFinalMaxThreads) k_obs_final(ObsArgs q, int n_seg) {
    const int64_t step = *q.a.d_step + q.k_off;
    if (q.gate > 0 && step % q.gate != 0) return;
    const int g = blockIdx.x;
    write_record(q, g, step, (*q.o.events * n_seg + g) % q.o.cap);
}

// One segment's record (the plain form, which runs the segments one after another): the
// event is the device counter plus event_off. One CTA.
__global__ void __launch_bounds__(kObsFinalMaxThreads) k_obs_final_one(ObsArgs q, int g, int n_seg,
                                                                        int64_t event_off) {
    write_record(q, g, *q.a.d_step + q.k_off, ((*q.o.events + event_off) * n_seg + g) % q.o.cap);
}

// Per-replica energy (for sop_forces): sum of the energy partials of segments [g_lo, g_hi).
__global__ void __launch_bounds__(kObsFinalMaxThreads) k_energy_sum(DevObs o, int g_lo, int g_hi, double *out) {
    __shared__ double sh[6 * (kObsFinalMaxThreads / 32)];
    double acc[6];
    chunk_sums(o, o.seg_chunk_lo[g_lo], o.seg_chunk_lo[g_hi], acc, sh);
    if (threadIdx.x == 0) *out = acc[0];
}

// Threads of the final reductions: a warp when segments hold few chunks, else a full CTA.
inline int final_threads(const DevObs &o) { return o.max_seg_chunks > 64 ? kObsFinalMaxThreads : 32; }

__global__ void k_tick(int64_t *d_step, int64_t k, int64_t *events, int32_t gate, int64_t n_events) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int64_t s = *d_step + k;
        if (events) *events += gate > 0 ? (s % gate == 0 ? 1 : 0) : n_events;
        *d_step = s;
    }
}

inline int blocks_for(int64_t work, int threads) { return (int)((work + threads - 1) / threads); }

// From this many beads in one launch the step runs one thread per bead (k_step_spread).
constexpr int64_t kSpreadMinBeads = 152 * 256;

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

void scan_exclusive(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s, int64_t *launches) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb > 0) k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp, nb);
    k_scan_final<<<(unsigned)(nb > 0 ? nb : 1), kScanThreads, 0, s>>>(in, out, n, tmp, nb);
    if (launches) *launches += nb > 0 ? 3 : 2;
}

void launch_setup_bonds(const double *X, const int32_t *chain, float *bond_r0, double *bond_r0d, int32_t n,
                        cudaStream_t s) {
    k_setup_bonds<<<blocks_for(n, 256), 256, 0, s>>>(X, chain, bond_r0, bond_r0d, n);
}

void launch_native_count(const double *X, const int32_t *chain, const int32_t *sys, const int32_t *sys_lo, int32_t n,
                         double cut, int32_t *count, cudaStream_t s) {
    k_native<false><<<blocks_for(n, 128), 128, 0, s>>>(X, chain, sys, sys_lo, n, cut, count, nullptr, nullptr,
                                                       nullptr, nullptr);
}

void launch_native_fill(const double *X, const int32_t *chain, const int32_t *sys, const int32_t *sys_lo, int32_t n,
                        double cut, const int32_t *row, int32_t *col, double *r0, float *r0sq, cudaStream_t s) {
    k_native<true><<<blocks_for(n, 128), 128, 0, s>>>(X, chain, sys, sys_lo, n, cut, nullptr, row, col, r0, r0sq);
}

void launch_seg_box_init(int32_t *seg_box, int32_t n_seg, cudaStream_t s) {
    if (n_seg > 0) k_seg_box_init<<<blocks_for(n_seg, 128), 128, 0, s>>>(seg_box, n_seg);
}

void launch_rebuild(const StepArgs &sa, const DevCells &c, const DevPairList &pl, const float4 *pos, float4 *snap,
                    const SegRange &rg, cudaStream_t s, int64_t *launches) {
    if (rg.g_hi <= rg.g_lo) return;
    RebuildArgs a;
    a.pos = pos;
    a.snap = snap;
    a.sys = sa.topo.sys;
    a.chain = sa.topo.chain;
    a.n = sa.topo.n;
    a.n_sys = sa.topo.n_sys;
    a.g_lo = rg.g_lo;
    a.g_hi = rg.g_hi;
    a.cell_edge = sqrtf(sa.cut2_f);
    a.seg_bead_lo = c.seg_bead_lo;
    a.seg_cell_base = c.seg_cell_base;
    a.seg_lo = c.seg_lo;
    a.seg_dims = c.seg_dims;
    a.cell_of = c.cell_of;
    a.cell_cnt = c.cell_cnt;
    a.cell_start = c.cell_start;
    a.sorted = c.sorted;
    a.sorted_base = rg.b_lo;
    a.cell_base0 = rg.c_lo;
    a.rep_status = sa.rep_status;
    a.seg_box = c.seg_box;
    const int nb = rg.b_hi - rg.b_lo, nc = rg.c_hi - rg.c_lo;
    BuildExtra x;
    x.nat_row = sa.topo.nat_row;
    x.nat_col = sa.topo.nat_col;
    x.xb_row = sa.topo.xb_row;
    x.xb_col = sa.topo.xb_col;
    x.cut2_d = sa.cut2_d;
    x.cut2_f = sa.cut2_f;
    x.pl_start = pl.start;
    x.pl_len = pl.len;
    x.pl_col = pl.col;
    x.pl_cursor = pl.cursor;
    x.pl_seg_base = pl.seg_base;
    x.pl_seg_end = pl.seg_end;
    x.rep_status = sa.rep_status;
    if (rg.max_seg > 0 && rg.max_seg <= kBruteBeads && c.brute_cta_lo && rg.k_hi > rg.k_lo) {
        // small segments: every bead against every bead, no cell list
        static bool brute_attr = false;
        if (!brute_attr) {
            cudaFuncSetAttribute(k_pl_brute, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(float) * (3 * kBruteBeads + 6 * (kBruteBeads / kBruteBlock)));
            brute_attr = true;
        }
        BruteArgs bz;
        bz.cta_lo = c.brute_cta_lo;
        bz.done = c.brute_done;
        bz.used = c.brute_used;
        bz.k_lo = rg.k_lo;
        // positions (x, y, z padded to even) and the boxes of the culling blocks
        const size_t smem = sizeof(float) * (3 * (size_t)((rg.max_seg + 1) & ~1) +
                                             6 * (size_t)((rg.max_seg + kBruteBlock - 1) / kBruteBlock));
        k_pl_brute<<<rg.k_hi - rg.k_lo, kBruteWarps * 32, smem, s>>>(a, x, bz);
        if (launches) *launches += 1;
        return;
    }
    {
        // bounding boxes: one CTA per 4096 beads of the largest segment (at most 128 per
        // segment), merged by atomics, then the grids
        const int slices = std::min(128, std::max(1, (rg.max_seg + 4095) / 4096));
        k_seg_bbox<<<dim3(rg.g_hi - rg.g_lo, slices), 256, 0, s>>>(a);
        k_seg_grid<<<blocks_for(rg.g_hi - rg.g_lo, 128), 128, 0, s>>>(a, rg.g_hi - rg.g_lo, pl.cursor, pl.seg_base);
        k_cell_count<<<blocks_for(nb, 256), 256, 0, s>>>(a, rg.b_lo, rg.b_hi);
        scan_exclusive(c.cell_cnt + rg.c_lo, c.cell_start, nc, c.scan_tmp, s, launches);
        k_cell_scatter<<<blocks_for(nb, 256), 256, 0, s>>>(a, rg.b_lo, rg.b_hi);
        if (launches) *launches += 4;
    }
    k_pl_build<<<blocks_for(nb, kBuildWarps), kBuildWarps * 32, 0, s>>>(a, x, rg.b_lo, rg.b_hi);
    if (launches) *launches += 1;
}

void launch_step(const StepArgs &a, const DevPairList &pl, const float4 *pos_in, float4 *pos_out, float4 *comp,
                 int32_t b_lo, int32_t b_hi, int32_t k_off, int lanes, cudaStream_t s, int64_t *launches) {
    const int64_t nb = b_hi - b_lo;
    if (nb >= kSpreadMinBeads) {   // enough beads to fill the GPU with one thread per bead
        const int blocks = blocks_for(nb, 256);
        switch (lanes) {
        case 4: k_step_spread<4><<<blocks, 256, 0, s>>>(a, pl, pos_in, pos_out, comp, b_lo, b_hi, k_off); break;
        case 16: k_step_spread<16><<<blocks, 256, 0, s>>>(a, pl, pos_in, pos_out, comp, b_lo, b_hi, k_off); break;
        case 32: k_step_spread<32><<<blocks, 256, 0, s>>>(a, pl, pos_in, pos_out, comp, b_lo, b_hi, k_off); break;
        default: k_step_spread<8><<<blocks, 256, 0, s>>>(a, pl, pos_in, pos_out, comp, b_lo, b_hi, k_off); break;
        }
        if (launches) *launches += 1;
        return;
    }
    const int64_t threads = nb * lanes;
    const int blocks = blocks_for(threads, 256);
    if (blocks <= 0) return;
    switch (lanes) {
    case 4: k_step<4><<<blocks, 256, 0, s>>>(a, pl, pos_in, pos_out, comp, b_lo, b_hi, k_off); break;
    case 16: k_step<16><<<blocks, 256, 0, s>>>(a, pl, pos_in, pos_out, comp, b_lo, b_hi, k_off); break;
    case 32: k_step<32><<<blocks, 256, 0, s>>>(a, pl, pos_in, pos_out, comp, b_lo, b_hi, k_off); break;
    default: k_step<8><<<blocks, 256, 0, s>>>(a, pl, pos_in, pos_out, comp, b_lo, b_hi, k_off); break;
    }
    if (launches) *launches += 1;
}

int coop_grid(int lanes, int64_t nb) {
    static int per_sm[3] = {-1, -1, -1};   // co-resident CTAs of 256 threads per SM, by lanes 4/8/16
    const int li = lanes == 4 ? 0 : lanes == 16 ? 2 : 1;
    if (per_sm[li] < 0) {
        int v = 0;
        const cudaError_t e = lanes == 4    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_step_coop<4>, 256, 0)
                              : lanes == 16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_step_coop<16>, 256, 0)
                                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_step_coop<8>, 256, 0);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        per_sm[li] = (e == cudaSuccess) ? v * sms : 0;
        cudaGetLastError();
    }
    const int need = blocks_for(nb * lanes, 256);
    return need < per_sm[li] ? need : per_sm[li];
}

cudaError_t launch_step_coop(const StepArgs &a, const DevPairList &pl, float4 *pos_a, float4 *pos_b, float4 *comp,
                             int32_t b_lo, int32_t b_hi, int32_t k_off, int32_t k_steps, int lanes, unsigned *bar,
                             cudaStream_t s, int64_t *launches) {
    const int64_t nb = b_hi - b_lo;
    const int grid = coop_grid(lanes, nb);
    if (nb <= 0 || k_steps <= 0) return cudaSuccess;
    if (grid <= 0) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid, 1, 1);
    lc.blockDim = dim3(256, 1, 1);
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t e;
    switch (lanes) {
    case 4: e = cudaLaunchKernelEx(&lc, k_step_coop<4>, a, pl, pos_a, pos_b, comp, b_lo, b_hi, k_off, k_steps, bar); break;
    case 16: e = cudaLaunchKernelEx(&lc, k_step_coop<16>, a, pl, pos_a, pos_b, comp, b_lo, b_hi, k_off, k_steps, bar); break;
    default: e = cudaLaunchKernelEx(&lc, k_step_coop<8>, a, pl, pos_a, pos_b, comp, b_lo, b_hi, k_off, k_steps, bar); break;
    }
    if (launches) *launches += 1;
    return e;
}

void launch_forces(const StepArgs &a, const DevPairList &pl, const float4 *pos, float4 *force, int32_t b_lo,
                   int32_t b_hi, int64_t step, cudaStream_t s, int64_t *launches, int lanes) {
    const int64_t threads = (int64_t)(b_hi - b_lo) * lanes;
    const int blocks = blocks_for(threads, 256);
    if (blocks <= 0) return;
    switch (lanes) {
    case 4: k_forces<4><<<blocks, 256, 0, s>>>(a, pl, pos, force, b_lo, b_hi, step); break;
    case 16: k_forces<16><<<blocks, 256, 0, s>>>(a, pl, pos, force, b_lo, b_hi, step); break;
    case 32: k_forces<32><<<blocks, 256, 0, s>>>(a, pl, pos, force, b_lo, b_hi, step); break;
    default: k_forces<8><<<blocks, 256, 0, s>>>(a, pl, pos, force, b_lo, b_hi, step); break;
    }
    if (launches) *launches += 1;
}

static ObsArgs make_obs_args(const StepArgs &a, const DevPairList &pl, const DevObs &o, const float4 *pos,
                             int32_t k_off, int32_t gate) {
    ObsArgs q;
    q.a = a;
    q.pl = pl;
    q.o = o;
    q.pos = pos;
    q.k_off = k_off;
    q.gate = gate;
    q.chunk0 = 0;
    q.eps_h = a.eps_h;
    q.eps_l = a.eps_l;
    q.sigma = a.sigma;
    q.k_fene = a.k_fene;
    q.R0 = a.R0;
    q.bond_r0d = a.topo.bond_r0d;
    return q;
}

void launch_observables(const StepArgs &a, const DevPairList &pl, const DevObs &o, const float4 *pos, int32_t n_seg,
                        int32_t k_off, int32_t gate, cudaStream_t s, int64_t *launches) {
    if (o.n_chunks <= 0) return;
    ObsArgs q = make_obs_args(a, pl, o, pos, k_off, gate);
    k_obs_partial<<<o.n_chunks, kObsThreads, 0, s>>>(q);
    k_obs_final<<<n_seg, final_threads(o), 0, s>>>(q, n_seg);
    if (launches) *launches += 2;
}

void launch_energy(const StepArgs &a, const DevPairList &pl, const DevObs &o, const float4 *pos, int32_t g_lo,
                   int32_t g_hi, int32_t ch_lo, int32_t ch_hi, double *out, cudaStream_t s, int64_t *launches) {
    if (ch_hi <= ch_lo) return;
    // only the chunks of segments [g_lo, g_hi): the list pl may be built for those alone
    ObsArgs q = make_obs_args(a, pl, o, pos, 0, 0);
    q.chunk0 = ch_lo;
    k_obs_partial<<<ch_hi - ch_lo, kObsThreads, 0, s>>>(q);
    k_energy_sum<<<1, kObsFinalMaxThreads, 0, s>>>(o, g_lo, g_hi, out);
    if (launches) *launches += 2;
}

void launch_observables_seg(const StepArgs &a, const DevPairList &pl, const DevObs &o, const float4 *pos, int32_t g,
                            int32_t n_seg, int32_t ch_lo, int32_t ch_hi, int32_t k_off, int64_t event_off,
                            cudaStream_t s, int64_t *launches) {
    if (ch_hi <= ch_lo) return;
    ObsArgs q = make_obs_args(a, pl, o, pos, k_off, 0);
    q.chunk0 = ch_lo;
    k_obs_partial<<<ch_hi - ch_lo, kObsThreads, 0, s>>>(q);
    k_obs_final_one<<<1, final_threads(o), 0, s>>>(q, g, n_seg, event_off);
    if (launches) *launches += 2;
}

void launch_tick(int64_t *d_step, int64_t k, int64_t *events, int32_t gate, int64_t n_events, cudaStream_t s,
                 int64_t *launches) {
    k_tick<<<1, 32, 0, s>>>(d_step, k, events, gate, n_events);
    if (launches) *launches += 1;
}

}  // namespace sop
