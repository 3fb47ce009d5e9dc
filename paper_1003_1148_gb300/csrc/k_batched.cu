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
#include <cuda_runtime.h>

#include "batched_common.cuh"

namespace sop {

namespace {

// Shared-memory layout of one work item, for systems of at most max_n beads. The
// accessors recompute each array's address from the dynamic shared-memory symbol, so
// that only a few integers stay live and every access is a 32-bit shared address.
__host__ __device__ inline size_t state_bytes(int max_n) {
    size_t s = kHeadBytes;
    s += 3 * sizeof(float4) * (size_t)max_n;       // two layers + compensation
    s += sizeof(float2) * (size_t)max_n;           // bond lengths
    s += 5 * sizeof(uint16_t) * (size_t)max_n;     // two orders, counts, slot of each bead
    s += (size_t)max_n;                            // flags
    s = (s + 15) / 16 * 16;
    s += 2 * sizeof(float4) * (size_t)((max_n + 31) / 32);   // block bounding boxes
    if (max_n <= kSoaMaxBeads) s += 3 * sizeof(float) * (size_t)((max_n + 31) & ~31);   // x, y, z arrays
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
    // rebuild scan: x, y, z of the layer being scanned, stride soa_stride()
    __device__ __forceinline__ int soa_stride() const { return (mx + 31) & ~31; }
    __device__ __forceinline__ float *soa() const { return reinterpret_cast<float *>(bbox() + 2 * ((mx + 31) / 32)); }
    // by slot: entry k of slot p at row[k * n + p] (bead indices)
    __device__ __forceinline__ uint16_t *row() const {
        if (RG) return grow;
        return reinterpret_cast<uint16_t *>(g_smem + state_bytes(mx));
    }
};





// Rows from layer src: the bead in slot p gets its native partners and its Verlet
// partners in column p. Block boxes must be current. In systems of up to 256 beads a
// thread builds the rows of its own slots. In larger ones it builds the rows of beads
// threadIdx.x + k * blockDim (slot_of must be current): a warp then scans for 32
// consecutive beads, which lie close together, so the box test skips blocks for all its
// lanes at once (with slots, ordered by row length, the lanes are spread over the whole
// system and some lane needs nearly every block). The rows are the same either way.
template <int BPT, bool RG>
__device__ void rebuild_rows(const BatchedArgs &a, const Layout<RG> &L, const uint16_t *order, const float4 *src,
                             int n_s, int nat_off, int b0, int exo) {
    const int T = blockDim.x;
    const float cut2 = a.sa.cut2_f;
    const float lo = cut2 - cut2 * 1e-4f, hi = cut2 + cut2 * 1e-4f;
    const float4 *bb = L.bbox();
    const float *soa = L.soa();
    const int S = L.soa_stride();
    uint16_t *row = L.row();
    const uint32_t *excl = exo >= 0 ? a.excl + exo : nullptr;
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
        // the row holds the Verlet partners only: the natives are read from the
        // slot-ordered native table in the native phase of the step
        const int nn = a.nat_ell_cnt[b0 + b];
        const uint16_t *natc = a.nat_ell_col + nat_off + b;
        constexpr int row0 = 0;
        const float2 bd = L.bond()[b];
        int q = 0;   // next native to exclude
        int next_nat = nn > 0 ? (int)__ldg(natc) : 0x7fffffff;
        int cnt = 0;
        for (int base = 0; base < n_s; base += 32) {
            // exact cull: every bead of the block is at least as far as its box. In a system of
            // a few blocks nearly every box is in range for some lane of the warp: the test only
            // costs there, so it is skipped
            bool scan = !kLarge || n_s <= 256;
            if (!scan) {
                const float4 blo = bb[base >> 4], bhi = bb[(base >> 4) + 1];
                const float ex = fmaxf(fmaxf(blo.x - pb.x, pb.x - bhi.x), 0.f);
                const float ey = fmaxf(fmaxf(blo.y - pb.y, pb.y - bhi.y), 0.f);
                const float ez = fmaxf(fmaxf(blo.z - pb.z, pb.z - bhi.z), 0.f);
                scan = fmaf(ez, ez, fmaf(ey, ey, ex * ex)) < hi;
            }
            // exclusions in [base, base + 32): self, bonded neighbours, native partners
            uint32_t ex_mask = 0u;
            if (excl) {
                ex_mask = __ldg(excl + (base >> 5) * n_s + b);
            } else {
                if (b >= base && b < base + 32) ex_mask |= 1u << (b - base);
                if (bd.x > 0.f && b - 1 >= base && b - 1 < base + 32) ex_mask |= 1u << (b - 1 - base);
                if (bd.y > 0.f && b + 1 >= base && b + 1 < base + 32) ex_mask |= 1u << (b + 1 - base);
                while (next_nat < base + 32) {
                    ex_mask |= 1u << (next_nat - base);
                    ++q;
                    next_nat = q < nn ? (int)__ldg(natc + q * n_s) : 0x7fffffff;
                }
            }
            if (!scan) continue;
            uint32_t within;
            if (L.mx <= kSoaMaxBeads) {
                within = block_partners(scan_block(soa, S, base, n_s - base, pb, lo, hi), ex_mask, src, base, pb, cut2,
                                        a.sa.cut2_d);
            } else {
                uint32_t cand = scan_block_f4(src, base, n_s - base, pb, hi) & ~ex_mask;
                within = 0u;
                while (cand) {
                    const int t = __ffs(cand) - 1;
                    cand &= cand - 1;
                    if (within_cut(pb, src[base + t], cut2, a.sa.cut2_d)) within |= 1u << t;
                }
            }
            while (within) {   // ascending
                const int t = __ffs(within) - 1;
                within &= within - 1;
                if (cnt < a.cap) row[(row0 + cnt) * n_s + p] = (uint16_t)(base + t);
                ++cnt;
            }
        }
        if (cnt > a.cap) cta_fail(L.h(), SOP_ERR_PAIRLIST_OVERFLOW);
        L.n_nat()[p] = (uint16_t)row0;
        L.n_tot()[p] = (uint16_t)(row0 + min(cnt, a.cap));
    }
}

// A full rebuild from layer src: boxes, slot order, rows. Ends with a barrier.
template <int BPT, bool RG>
__device__ int rebuild(const BatchedArgs &a, const Layout<RG> &L, const float4 *src, int n_s, int nat_off, int b0,
                       int ord, int exo) {
    constexpr bool kLarge = RG || BPT > 1;   // as in rebuild_rows
    if (kLarge && n_s > 256) block_boxes(L, src, n_s);
    if (L.mx <= kSoaMaxBeads) soa_fill(src, L.soa(), n_s, L.soa_stride());
    ord = reorder_slots(L, n_s, ord);   // its barriers also publish the boxes and the x, y, z arrays
    if (kLarge && n_s > 256) {
        const uint16_t *o = L.order(ord);
        for (int p = threadIdx.x; p < n_s; p += blockDim.x) L.slot_of()[o[p]] = (uint16_t)p;
        __syncthreads();
    }
    rebuild_rows<BPT>(a, L, L.order(ord), src, n_s, nat_off, b0, exo);
    __syncthreads();
    return ord;
}

// Sum of the Eq. 1 pair forces on bead b (in slot p) at layer P over its bonds and row.
// Entries k < n_nat are native (12-6 with r0^2 from the table), the rest repulsive.
// Native phase of a step (Eq. 1's 12-6 term): the bead in native slot t of the system (slots
// ordered by native count, so that the warps' loops are balanced) gets the sum of its native
// forces, entries from the slot-ordered native table in global memory (consecutive lanes read
// consecutive words). Returns its local index. The entries are those of its row in their
// order, and the Verlet phase continues the same sum, so every force has the bits of one
// loop over the whole row.
__device__ __forceinline__ int native_force(const BatchedArgs &a, const float4 *P, int n_s, int nat_off, int b0,
                                            int t, float3 *f) {
    const ForceParams &fp = a.sa.fp;
    const int b = a.nat_slot_bead[b0 + t];
    const float4 pb = P[b];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const int nn = a.nat_slot_cnt[b0 + t];
    const uint2 *ent = a.nat_slot_ent + nat_off + t;
    const float A = fp.eps12_h;
#pragma unroll 2
    for (int k = 0; k < nn; ++k) {
        const uint2 e = __ldg(ent);   // partner and r0^2 in one load
        ent += n_s;
        const int j = (int)e.x;
        const float s0 = __uint_as_float(e.y);
        const float4 pj = P[j];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float inv = __fdividef(1.0f, r2);
        const float s = s0 * inv;
        const float s3 = s * s * s;
        const float c = inv * s3 * fmaf(A, s3, -A);   // (12 eps_h / r^2)(s^6 - s^3), s = r0^2 / r^2
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    *f = make_float3(fx, fy, fz);
    return b;
}

// Verlet phase: the bead in slot p adds its repulsive terms (its row holds Verlet partners
// only) to its native sum `nat`, and the FENE force of its two bonds is summed apart and added
// last (Eq. 1; the grouping of the former one-pass bead_force).
template <bool RG>
__device__ __forceinline__ float3 verlet_force(const BatchedArgs &a, const Layout<RG> &L, const float4 *P, int n_s,
                                               int b, int p, float3 nat, bool *broken) {
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
    const float3 fr = row_force(P, pb, L.row() + p, nullptr, 0, L.n_tot()[p], n_s, n_s, fp, nat);
    return make_float3(fx + fr.x, fy + fr.y, fz + fr.z);
}

// The native phase over the CTA's native slots: each bead's native sum into F[b]. Ends with
// a barrier.
template <int BPT, bool RG>
__device__ __forceinline__ void native_phase(const BatchedArgs &a, const Layout<RG> &L, const float4 *P, float4 *F,
                                             int n_s, int nat_off, int b0) {
#pragma unroll 1
    for (int k = 0; k < BPT; ++k) {
        const int t = threadIdx.x + k * blockDim.x;
        if (t >= n_s) continue;
        float3 f;
        const int b = native_force(a, P, n_s, nat_off, b0, t, &f);
        F[b] = make_float4(f.x, f.y, f.z, 0.f);
    }
    __syncthreads();
}

// FP64 observables of the CTA's system at layer P (same definitions as the streamed kernels).
template <int BPT, bool RG>
__device__ __noinline__ void observe(const BatchedArgs &a, const Layout<RG> &L, const uint16_t *order,
                                     const float4 *P, int n_s, int b0, int r, int s, int g, int64_t step,
                                     int64_t event) {
    const StepArgs &sa = a.sa;
    const int T = blockDim.x;
    const uint16_t *row = L.row();
    double v[6] = {0, 0, 0, 0, 0, 0};   // E, f_pull, ext, formed, f_wall, r_ee
    const double sig2 = sa.sigma * sa.sigma;
    for (int k = 0; k < BPT; ++k) {
        const int p = threadIdx.x + k * T;
        if (p >= n_s) continue;
        const int b = order[p];
        const float4 pb = P[b];
        obs_bonded(sa, P, b, b0, L.bond()[b].y > 0.f, v);
        for (int q = L.n_nat()[p]; q < L.n_tot()[p]; ++q) {
            const int j = row[q * n_s + p];
            if (j < b) continue;
            const float4 pj = P[j];
            float d2f;
            const double d2 = dist2_two(pb, pj, &d2f);
            const double c = sig2 * rcp_seeded(d2, d2f);
            v[0] = fma(sa.eps_l, c * c * c, v[0]);
        }
        obs_external(sa, P, b, b0, r, s, step, L.flags()[b], v);
    }
    block_sum6(v, L.h());
    if (threadIdx.x == 0) write_record(a, v, r, s, g, step, event);
    __syncthreads();
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
    const int exo = a.excl_off[s];
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
        L.n_tot()[b] = 0;   // the first slot order (no row built yet)
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
            ord = rebuild<BPT>(a, L, Q, n_s, nat_off, b0, ord, exo);   // Q holds the snapshot here
        } else if ((k_phase == 0 && !built_now) || forces_only) {
            ord = rebuild<BPT>(a, L, P, n_s, nat_off, b0, ord, exo);
            // the snapshot is kept only from the launch's last rebuild: a later launch that
            // starts between rebuilds builds its first list from it
            if (!forces_only && it + a.K >= a.n_steps)
                for (int b = threadIdx.x; b < n_s; b += T) a.snap[gbase + b] = P[b];
        }
        built_now = false;
        const int64_t step = step0 + it;
        const uint16_t *order = L.order(ord);
        // native phase: bonds and natives of every bead into Q (the next layer, free until
        // the Verlet phase below writes each bead's new position over its own entry)
        native_phase<BPT>(a, L, P, Q, n_s, nat_off, b0);
        if (forces_only) {
            for (int p = threadIdx.x; p < n_s; p += T) {
                const int b = order[p];
                bool overlap = false, broken = false;
                const float4 fn = Q[b];
                const float3 f = verlet_force(a, L, P, n_s, b, p, make_float3(fn.x, fn.y, fn.z), &broken);
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
            bool overlap = false, broken = false;
            const float4 fn = Q[b];
            const float3 f = verlet_force(a, L, P, n_s, b, p, make_float3(fn.x, fn.y, fn.z), &broken);
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
                ord = rebuild<BPT>(a, L, Pn, n_s, nat_off, b0, ord, exo);
                built_now = true;
                if (it + 1 + a.K >= a.n_steps)
                    for (int b = threadIdx.x; b < n_s; b += T) a.snap[gbase + b] = Pn[b];
            }
            const int64_t ev = (a.d_events ? *a.d_events : 0) + n_events;
            observe<BPT>(a, L, L.order(ord), Pn, n_s, b0, r, s, g, step + 1, ev);
            ++n_events;
        }
    }
    if (forces_only) return;
    if (threadIdx.x == 0 && L.h()->fail != 0)
        missing_records(a, r, s, g, step0, step0 + it - 1, (a.d_events ? *a.d_events : 0) + n_events);
    const float4 *P = L.lay(cur);
    for (int b = threadIdx.x; b < n_s; b += T) {
        a.pos[gbase + b] = P[b];
        a.comp[gbase + b] = L.comp()[b];
    }
    if (threadIdx.x == 0 && L.h()->fail != 0) atomicCAS(&sa.rep_status[r], 0, L.h()->fail);
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

cudaError_t launch_batched(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s, int64_t *launches) {
    if (a.n_items <= 0) return cudaSuccess;
    if (launches) *launches += 1;
    if (cfg.pair_form) return launch_bpair(a, cfg, s);
    if (cfg.cluster > 0) return launch_cluster(a, cfg, s);
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
    if (cfg.pair_form) return bpair_resident_ctas(cfg);
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
