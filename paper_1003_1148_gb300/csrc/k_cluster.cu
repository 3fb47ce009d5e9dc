// Batched schedule, cluster form: one system over a thread-block cluster (sm_103a).
//
// CTA q of a cluster of C owns the system's beads [q m, (q + 1) m), m = 2^m_shift a
// multiple of 32: their compensation, bond lengths, slot orders and rows live in its
// shared memory, next to a full copy of the positions of the whole system (both time
// layers). All reads are local: a CTA gathers forces and builds rows from its own copy.
// After the update each CTA writes the new positions of its own beads into every copy in
// the cluster (stores to distributed shared memory), and one cluster barrier
// (release/acquire) ends the step. A copy's layer is only ever written while every CTA
// reads the other layer, so no read meets a remote write. Every CTA of a cluster takes the
// same sequence of cluster barriers: each control decision (a frozen replica, a failure,
// the rebuild and observable cadence) comes from values every CTA reads after the same
// barrier.
//
// A single system of a few thousand beads leaves the SMs of its cluster short of work,
// and a step is a chain of dependent loads and arithmetic. So a bead is served by a group
// of LN lanes (1, 2 or 4): lane l of the group takes the native partners q = l, l + LN, ...
// and, at each rebuild, scans the candidates t = l, l + LN, ... of every block of 32 beads
// in range and keeps the Verlet partners among them. Its partners form its own sub-row
// (natives first, then Verlet partners ascending); the group adds the sub-row sums by a
// shuffle tree, lane 0 draws the noise and updates the bead, and the lanes share the
// stores of the new position into the C copies. Every sum has a fixed order, so runs are
// reproducible bit for bit; with one lane per bead the arithmetic and its order are those
// of the one-CTA particle-based form (k_batched.cu).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "batched_common.cuh"

namespace cg = cooperative_groups;

namespace sop {

namespace {

constexpr int kMaxCluster = 16;
constexpr int kNoFail = 0x7fffffff;

struct ClusterExtra {
    int fail_step;                        // first step of the launch at which this CTA failed
    int frozen;                           // rank 0: the replica was frozen at launch
    double part[6];                       // this CTA's observable sums
    float4 *rpos[2][kMaxCluster];         // every rank's two position layers (generic addresses)
    const ClusterExtra *peer[kMaxCluster];
};

// Entries of one lane's sub-row: its share of a row of row_width entries, with room for an
// uneven split of the partners over the lanes.
__host__ __device__ inline int lane_width(int row_width, int ln) {
    return ln == 1 ? row_width : (5 * row_width + 4 * ln - 1) / (4 * ln) + 2;
}

// Shared-memory layout of one CTA: positions of all nmax = C m beads (two layers), then
// own-bead state for m beads (compensation, bond lengths, two slot orders, the sort key,
// the slot of each bead, flags, and per lane the native and total entries of its
// sub-row), block boxes of the whole system, the sub-rows of the own slots (entry e of
// lane l of slot p at (e LN + l) m + p), and the cluster bookkeeping.
struct CLayout {
    int nmax, m, ln, lw;   // lw: entries of one lane's sub-row
    __device__ __forceinline__ SharedHead *h() const { return reinterpret_cast<SharedHead *>(g_smem); }
    __device__ __forceinline__ float4 *pos(int layer) const {
        return reinterpret_cast<float4 *>(g_smem + kHeadBytes) + (size_t)layer * nmax;
    }
    __device__ __forceinline__ float4 *comp() const { return pos(2); }
    __device__ __forceinline__ float2 *bond() const { return reinterpret_cast<float2 *>(comp() + m); }
    __device__ __forceinline__ uint16_t *u16(int i) const { return reinterpret_cast<uint16_t *>(bond() + m) + i * m; }
    __device__ __forceinline__ uint16_t *order(int i) const { return u16(i); }   // slot -> own bead
    __device__ __forceinline__ uint16_t *n_tot() const { return u16(2); }        // by slot: sort key (longest sub-row)
    __device__ __forceinline__ uint16_t *slot_of() const { return u16(3); }      // by own bead: its slot
    __device__ __forceinline__ uint16_t *lane_nat() const { return u16(4); }     // [ln][m] natives of the sub-row
    __device__ __forceinline__ uint16_t *lane_tot() const { return u16(4 + ln); }   // [ln][m] all entries
    __device__ __forceinline__ uint8_t *flags() const { return reinterpret_cast<uint8_t *>(u16(4 + 2 * ln)); }
    __device__ __forceinline__ float4 *bbox() const {
        const size_t off = (kHeadBytes + 32 * (size_t)nmax + 16 * (size_t)m + 8 * (size_t)m +
                            2 * (size_t)(4 + 2 * ln) * m + m + 15) / 16 * 16;
        return reinterpret_cast<float4 *>(g_smem + off);
    }
    __device__ __forceinline__ uint16_t *row() const { return reinterpret_cast<uint16_t *>(bbox() + nmax / 16); }
    __device__ __forceinline__ ClusterExtra *extra() const {
        const size_t off = ((reinterpret_cast<unsigned char *>(row() + (size_t)lw * ln * m) - g_smem) + 15) / 16 * 16;
        return reinterpret_cast<ClusterExtra *>(g_smem + off);
    }
};

__host__ __device__ inline size_t cluster_smem(int m, int nmax, int row_width, int ln) {
    size_t s = kHeadBytes + 32 * (size_t)nmax + 16 * (size_t)m + 8 * (size_t)m + 2 * (size_t)(4 + 2 * ln) * m + m;
    s = (s + 15) / 16 * 16;
    s += 2 * sizeof(float4) * (size_t)(nmax / 32);
    s += sizeof(uint16_t) * (size_t)lane_width(row_width, ln) * ln * m;
    s = (s + 15) / 16 * 16;
    return s + (sizeof(ClusterExtra) + 15) / 16 * 16;
}

// Lanes of this thread's group of LN (groups are aligned within the warp).
template <int LN>
__device__ __forceinline__ unsigned lane_group_mask() {
    return LN == 32 ? 0xffffffffu : (((1u << LN) - 1u) << ((threadIdx.x & 31) & ~(LN - 1)));
}

// Sub-rows of this CTA's own beads from layer `layer` of its copy (system-local bead
// indices). The block boxes of the whole system and slot_of must be current. Group grp
// builds the rows of own beads grp + k G (G groups), so that a warp scans for consecutive
// beads, which lie close together, and the box test skips blocks for all its lanes at once.
template <int BPT, int LN>
__device__ void cluster_rows(const BatchedArgs &a, const CLayout &L, int layer, int n_loc, int lo, int n_s,
                             int nat_off, int b0) {
    const int G = blockDim.x / LN, m = L.m;
    const int grp = threadIdx.x / LN, ln = threadIdx.x % LN;
    const float cut2 = a.sa.cut2_f;
    const float hi2 = cut2 + cut2 * 1e-4f;
    const float4 *src = L.pos(layer);
    const float4 *bb = L.bbox();
    const int stride = LN * m;
#pragma unroll 1
    for (int k = 0; k < BPT; ++k) {
        const int l = grp + k * G;
        if (l >= n_loc) continue;   // the same for every lane of the group
        const int p = L.slot_of()[l];
        const int b = lo + l;
        const float4 pb = src[b];
        const int nn = a.nat_ell_cnt[b0 + b];
        const uint16_t *natc = a.nat_ell_col + nat_off + b;
        uint16_t *rl = L.row() + ln * m + p;   // entry e of this lane's sub-row at rl[e * stride]
        int e = 0;
        for (int q = ln; q < nn; q += LN, ++e)
            if (e < L.lw) rl[e * stride] = __ldg(natc + q * n_s);
        const int nn_l = e;
        const float2 bd = L.bond()[l];
        int q = 0;
        int next_nat = nn > 0 ? (int)__ldg(natc) : 0x7fffffff;
        int cnt = 0;
        for (int base = 0; base < n_s; base += 32) {
            const float4 blo = bb[base >> 4], bhi = bb[(base >> 4) + 1];
            const float ex = fmaxf(fmaxf(blo.x - pb.x, pb.x - bhi.x), 0.f);
            const float ey = fmaxf(fmaxf(blo.y - pb.y, pb.y - bhi.y), 0.f);
            const float ez = fmaxf(fmaxf(blo.z - pb.z, pb.z - bhi.z), 0.f);
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
            if (!(fmaf(ez, ez, fmaf(ey, ey, ex * ex)) < hi2)) continue;
            // this lane's candidates base + ln, base + ln + LN, ...
            const int lim = min(32, n_s - base);
            uint32_t cand = 0u;
#pragma unroll 4
            for (int t = ln; t < lim; t += LN) {
                const float4 pj = src[base + t];
                const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                cand |= (r2 < hi2 ? 1u : 0u) << t;
            }
            cand &= ~ex_mask;
            while (cand) {   // ascending: the exact decision, then the entry
                const int t = __ffs(cand) - 1;
                cand &= cand - 1;
                if (!within_cut(pb, src[base + t], cut2, a.sa.cut2_d)) continue;
                if (nn_l + cnt < L.lw) rl[(nn_l + cnt) * stride] = (uint16_t)(base + t);
                ++cnt;
            }
        }
        // the bead's Verlet count over the group, and its longest sub-row (the sort key)
        int total = cnt, longest = nn_l + cnt;
#pragma unroll
        for (int o = LN / 2; o > 0; o >>= 1) {
            total += __shfl_xor_sync(lane_group_mask<LN>(), total, o, LN);
            longest = max(longest, __shfl_xor_sync(lane_group_mask<LN>(), longest, o, LN));
        }
        if (total > a.cap || nn_l + cnt > L.lw) cta_fail(L.h(), SOP_ERR_PAIRLIST_OVERFLOW);
        L.lane_nat()[ln * m + p] = (uint16_t)min(nn_l, L.lw);
        L.lane_tot()[ln * m + p] = (uint16_t)min(nn_l + cnt, L.lw);
        if (ln == 0) L.n_tot()[p] = (uint16_t)min(longest, kKeys - 1);
    }
}

// Rebuild from layer `layer` of the local copy: boxes of every block of the system, the
// own slot order (groups of slots handed out by decreasing longest sub-row) and rows.
// Local only; ends with a CTA barrier.
template <int BPT, int LN>
__device__ int cluster_rebuild(const BatchedArgs &a, const CLayout &L, int layer, int n_loc, int lo, int n_s,
                               int nat_off, int b0, int ord) {
    block_boxes(L, L.pos(layer), n_s);
    ord = reorder_slots(L, n_loc, ord, blockDim.x / LN);   // its barriers also publish the boxes
    const uint16_t *o = L.order(ord);
    for (int p = threadIdx.x; p < n_loc; p += blockDim.x) L.slot_of()[o[p]] = (uint16_t)p;
    __syncthreads();
    cluster_rows<BPT, LN>(a, L, layer, n_loc, lo, n_s, nat_off, b0);
    __syncthreads();
    return ord;
}

// Eq. 1 pair forces on own bead l (system bead b, slot p) at layer P of the local copy:
// lane ln sums its bond and its sub-row, the group adds the lanes' sums (every lane gets
// the total). With one lane the bonds and the row are summed as in the one-CTA form.
template <int LN>
__device__ __forceinline__ float3 cluster_force(const BatchedArgs &a, const CLayout &L, const float4 *P, int n_s,
                                                int nat_off, int l, int b, int p, int ln, bool *broken) {
    const ForceParams &fp = a.sa.fp;
    const int m = L.m;
    const float4 pb = P[b];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const float2 bd = L.bond()[l];
    bool brk = false;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const float r0 = side ? bd.y : bd.x;
        if (r0 > 0.f && (LN == 1 || ln == side)) {
            const float4 pj = P[side ? b + 1 : b - 1];
            const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float r = r2 * rsqrtf(r2);
            const float dr = r - r0;
            const float arg = fmaf(-dr * dr, fp.inv_R02, 1.0f);
            float c = 0.f;
            if (arg > 0.f) c = __fdividef(-fp.k_fene * dr, arg * r);
            else brk = true;
            fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
        }
    }
    const float3 fr = row_force(P, pb, L.row() + ln * m + p, a.nat_ell_r0sq + nat_off + b + ln * n_s,
                                L.lane_nat()[ln * m + p], L.lane_tot()[ln * m + p], LN * m, LN * n_s, fp);
    fx += fr.x; fy += fr.y; fz += fr.z;
    if (LN > 1) {
#pragma unroll
        for (int o = LN / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(lane_group_mask<LN>(), fx, o, LN);
            fy += __shfl_xor_sync(lane_group_mask<LN>(), fy, o, LN);
            fz += __shfl_xor_sync(lane_group_mask<LN>(), fz, o, LN);
        }
        brk = __any_sync(lane_group_mask<LN>(), brk);
    }
    *broken = brk;
    return make_float3(fx, fy, fz);
}

// FP64 observables of the cluster's system at layer P: every CTA sums its own beads (lane 0
// of a group the bonded terms and readouts, every lane the Verlet energy of its sub-row),
// rank 0 adds the CTA sums after a cluster barrier and writes the record.
template <int BPT, int LN>
__device__ __noinline__ void cluster_observe(const BatchedArgs &a, const CLayout &L, ClusterExtra *X,
                                             const uint16_t *order, const float4 *P, int n_loc, int lo, int b0,
                                             int r, int s, int g, int64_t step, int64_t event, int rank, int C) {
    const StepArgs &sa = a.sa;
    const int G = blockDim.x / LN, m = L.m;
    const int grp = threadIdx.x / LN, ln = threadIdx.x % LN;
    double v[6] = {0, 0, 0, 0, 0, 0};   // E, f_pull, ext, formed, f_wall, r_ee
    const double sig2 = sa.sigma * sa.sigma;
    for (int k = 0; k < BPT; ++k) {
        const int p = grp + k * G;
        if (p >= n_loc) continue;
        const int l = order[p];
        const int b = lo + l;
        const float4 pb = P[b];
        if (ln == 0) obs_bonded(sa, P, b, b0, L.bond()[l].y > 0.f, v);
        const uint16_t *rl = L.row() + ln * m + p;
        for (int e = L.lane_nat()[ln * m + p]; e < L.lane_tot()[ln * m + p]; ++e) {
            const int j = rl[e * LN * m];
            if (j < b) continue;
            const float4 pj = P[j];
            float d2f;
            const double d2 = dist2_two(pb, pj, &d2f);
            const double c = sig2 * rcp_seeded(d2, d2f);
            v[0] = fma(sa.eps_l, c * c * c, v[0]);
        }
        if (ln == 0) obs_external(sa, P, b, b0, r, s, step, L.flags()[l], v);
    }
    block_sum6(v, L.h());
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) X->part[k] = v[k];
    cg::this_cluster().sync();
    if (rank == 0 && threadIdx.x == 0) {
        double w[6] = {0, 0, 0, 0, 0, 0};
        for (int q = 0; q < C; ++q)
            for (int k = 0; k < 6; ++k) w[k] += X->peer[q]->part[k];
        write_record(a, w, r, s, g, step, event);
    }
    __syncthreads();
}

// BPT: own beads per group of LN lanes; MAXT: largest CTA the instance is compiled for.
template <int BPT, int LN, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_cluster(BatchedArgs a, int sh, int lw) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int C = (int)cl.num_blocks();
    const int item = blockIdx.x / C;
    CLayout L;
    L.m = 1 << sh;
    L.nmax = C << sh;
    L.ln = LN;
    L.lw = lw;
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
    const int T = blockDim.x, G = T / LN;
    const int grp = threadIdx.x / LN, ln = threadIdx.x % LN;
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
        L.n_tot()[l] = (uint16_t)min(a.nat_ell_cnt[i], kKeys - 1);
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
            ord = cluster_rebuild<BPT, LN>(a, L, 1, n_loc, lo, n_s, nat_off, b0, ord);   // from the snapshot
            cl.sync();   // layer 1 is read by every CTA before the step writes it
        } else if ((k_phase == 0 && !built_now) || forces_only) {
            ord = cluster_rebuild<BPT, LN>(a, L, cur, n_loc, lo, n_s, nat_off, b0, ord);
            if (!forces_only && it + a.K >= a.n_steps)
                for (int l = threadIdx.x; l < n_loc; l += T) a.snap[gbase + lo + l] = L.pos(cur)[lo + l];
        }
        built_now = false;
        const int64_t step = step0 + it;
        const uint16_t *order = L.order(ord);
        const float4 *P = L.pos(cur);
        if (forces_only) {
            for (int k = 0; k < BPT; ++k) {
                const int p = grp + k * G;
                if (p >= n_loc) continue;
                const int l = order[p], b = lo + l;
                bool broken = false, overlap = false;
                const float3 f = cluster_force<LN>(a, L, P, n_s, nat_off, l, b, p, ln, &broken);
                if (ln != 0) continue;
                const float3 fe = ext_force(sa, r, b0 + b, L.flags()[l], P[b], step, &overlap);
                a.force_out[gbase + b] = make_float4(f.x + fe.x, f.y + fe.y, f.z + fe.z, (broken || overlap) ? 1.f : 0.f);
                if (a.pl_dump_col) {   // the Verlet partners of every lane, up to the stride
                    const size_t rowi = (size_t)gbase + b;
                    int w = 0, np = 0;
                    for (int q = 0; q < LN; ++q) {
                        const int e0 = L.lane_nat()[q * L.m + p], e1 = L.lane_tot()[q * L.m + p];
                        np += e1 - e0;
                        for (int e = e0; e < e1 && w < a.pl_dump_stride; ++e)
                            a.pl_dump_col[rowi * a.pl_dump_stride + w++] = b0 + (int)L.row()[(e * LN + q) * L.m + p];
                    }
                    a.pl_dump_start[rowi] = (int)(rowi * a.pl_dump_stride);
                    a.pl_dump_len[rowi] = np;
                }
            }
            break;
        }
        const int nxt = cur ^ 1;
#pragma unroll 1
        for (int k = 0; k < BPT; ++k) {
            const int p = grp + k * G;
            if (p >= n_loc) continue;   // the same for every lane of the group
            const int l = order[p], b = lo + l;
            bool broken = false, overlap = false;
            const float3 f = cluster_force<LN>(a, L, P, n_s, nat_off, l, b, p, ln, &broken);
            float4 pb = P[b];
            if (ln == 0) {
                const float4 p_old = pb;
                const uint8_t fl = L.flags()[l];
                const float3 fe = ext_force(sa, r, b0 + b, fl, p_old, step, &overlap);
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
            }
            if (LN > 1) {   // lane 0's result to the group, which shares the remote stores
                const unsigned gm = lane_group_mask<LN>();
                pb.x = __shfl_sync(gm, pb.x, 0, LN);
                pb.y = __shfl_sync(gm, pb.y, 0, LN);
                pb.z = __shfl_sync(gm, pb.z, 0, LN);
                pb.w = __shfl_sync(gm, pb.w, 0, LN);
            }
            // the new position into every copy of the cluster
            for (int q = ln; q < C; q += LN) X->rpos[nxt][q][b] = pb;
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
                ord = cluster_rebuild<BPT, LN>(a, L, cur, n_loc, lo, n_s, nat_off, b0, ord);
                built_now = true;
                if (it + 1 + a.K >= a.n_steps)
                    for (int l = threadIdx.x; l < n_loc; l += T) a.snap[gbase + lo + l] = L.pos(cur)[lo + l];
            }
            const int64_t ev = (a.d_events ? *a.d_events : 0) + n_events;
            cluster_observe<BPT, LN>(a, L, X, L.order(ord), L.pos(cur), n_loc, lo, b0, r, s, g, step + 1, ev, rank,
                                     C);
            ++n_events;
        }
    }
    if (!forces_only) {
        bool failed = false;
        for (int q = 0; q < C; ++q) failed |= X->peer[q]->fail_step != kNoFail;
        if (failed && rank == 0 && threadIdx.x == 0)
            missing_records(a, r, s, g, step0, step0 + it - 1, (a.d_events ? *a.d_events : 0) + n_events);
        for (int l = threadIdx.x; l < n_loc; l += T) {
            a.pos[gbase + lo + l] = L.pos(cur)[lo + l];
            a.comp[gbase + lo + l] = L.comp()[l];
        }
        if (threadIdx.x == 0 && L.h()->fail != 0) atomicCAS(&sa.rep_status[r], 0, L.h()->fail);
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

template <int BPT, int LN, int MAXT>
cudaError_t launch_cl(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s) {
    auto kern = k_cluster<BPT, LN, MAXT>;
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
    return cudaLaunchKernelEx(&lc, kern, a, cfg.m_shift, lane_width(cfg.row_width, LN));
}

template <int BPT, int LN, int MAXT>
int capacity_cl(const BatchedConfig &cfg) {
    auto kern = k_cluster<BPT, LN, MAXT>;
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

}  // namespace

// The compiled instances: one or two own beads per group of 1, 2 or 4 lanes; CTAs of up to
// 512 threads with one or two lanes per bead, up to 1024 with four.
bool cluster_config(int max_n, int row_width, int threads, int m_shift, int lanes, BatchedConfig *cfg) {
    if (m_shift < 5 || m_shift > 9 || max_n <= 0 || max_n > 8192 || row_width > kKeys - 1) return false;
    if (lanes != 1 && lanes != 2 && lanes != 4) return false;
    const int m = 1 << m_shift;
    const int C = (max_n + m - 1) / m;
    const int maxt = lanes == 4 ? 1024 : 512;
    if (C < 2 || C > kMaxCluster || threads % 32 || threads < 32 || threads > maxt) return false;
    const int groups = threads / lanes;
    const int bpt = (m + groups - 1) / groups;
    if (bpt > 2 || groups * bpt < m) return false;
    cfg->threads = threads;
    cfg->beads_per_thread = bpt;
    cfg->min_blocks = 1;
    cfg->rows_global = false;
    cfg->row_width = row_width;
    cfg->smem = cluster_smem(m, C * m, row_width, lanes);
    cfg->cluster = C;
    cfg->m_shift = m_shift;
    cfg->lanes = lanes;
    cfg->pair_form = false;
    return cfg->smem <= 227 * 1024;
}

cudaError_t launch_cluster(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s) {
    const bool two = cfg.beads_per_thread > 1;
    switch (cfg.lanes) {
    case 2: return two ? launch_cl<2, 2, 512>(a, cfg, s) : launch_cl<1, 2, 512>(a, cfg, s);
    case 4: return two ? launch_cl<2, 4, 1024>(a, cfg, s) : launch_cl<1, 4, 1024>(a, cfg, s);
    default: return two ? launch_cl<2, 1, 512>(a, cfg, s) : launch_cl<1, 1, 512>(a, cfg, s);
    }
}

int cluster_capacity(const BatchedConfig &cfg) {
    if (cfg.cluster <= 0) return 0;
    const bool two = cfg.beads_per_thread > 1;
    switch (cfg.lanes) {
    case 2: return two ? capacity_cl<2, 2, 512>(cfg) : capacity_cl<1, 2, 512>(cfg);
    case 4: return two ? capacity_cl<2, 4, 1024>(cfg) : capacity_cl<1, 4, 1024>(cfg);
    default: return two ? capacity_cl<2, 1, 512>(cfg) : capacity_cl<1, 1, 512>(cfg);
    }
}

}  // namespace sop
