// Batched schedule, pair form: every pair evaluated once, inside one CTA (sm_103a).
//
// The paper's pair-based parallelisation (Sec. III.B, Algorithms 4 and 5) computes each
// interacting pair once and adds +df and -df to its two particles. Here the whole system of
// one work item (a system of one replica, at most 256 beads) lives in one CTA's shared
// memory for a chunk of steps, as in the particle-based form (k_batched.cu), and each pair
// belongs to the row of one of its two beads:
//
// * a native pair by a balanced orientation chosen on the host (every bead owns about half
//   of its native pairs);
// * a Verlet pair (i, j), i < j, by i when i + j is odd and by j when i + j is even, which
//   also gives every bead about half of its Verlet pairs.
//
// A step has two phases separated by a barrier. Phase A: the thread of bead b evaluates
// the pairs of its own row (and the bond (b, b+1)), adds each force to b and stores the
// pair's scalar coefficient c (F_b = c (r_b - r_j)) in a slot beside the entry. Phase B:
// the same thread reads, through its reverse list, the coefficients of the pairs that other
// beads own with b and adds c (r_b - r_i), the exact negation of the owner's term; then the
// cantilever/indenter force, Philox noise and the compensated update follow as in every
// form. A bead's force is summed in a fixed order (own bond, own natives, own Verlet
// partners ascending, then the bond to b - 1, reverse natives, reverse Verlet partners
// ascending), whatever slot or thread it is given, so runs are reproducible bit for bit.
//
// Rows are stored sliced by groups of 32 slots (entry k of slot p at base[p/32] + 32 k +
// p % 32, base from the widths of the groups), so lanes of a warp read consecutive words and
// little space is spent on padding. The reverse entry of b for a pair owned by i holds i and
// the position of the pair in i's row. Rebuild (every K steps, Algorithm 3 with the whole
// system as candidate set): slots are handed to beads by decreasing degree of the last build;
// each thread tests all candidates of its bead in blocks of 32 (bit masks, FP64 decision in
// the guard band), splits the partners by ownership, counts, and after the group widths and
// bases are known writes its row and its reverse list. The position of b in the row of its
// owner i follows from i's masks: i's own natives first, then the own Verlet partners of i
// below b.
#include <cuda_runtime.h>

#include "batched_common.cuh"

namespace sop {

namespace {

constexpr int kPairGroups = kPairMaxBeads / 32;

// Head of the work item: the common head for CTAs of up to 256 threads, then the layout of
// the pair pool fixed at each rebuild.
struct PairHead {
    int fail;                            // first sop_status raised in this CTA
    int hist[kKeys];                     // counting sort of slots by degree
    double red[kPairGroups][6];          // FP64 block reductions, one row per warp
    int b_own[kPairGroups + 1];          // first entry of each group of 32 slots (own rows)
    int b_rev[kPairGroups + 1];          // the same for the reverse lists
    int w_own[kPairGroups], w_rev[kPairGroups];   // widths of the groups
    int off_rev, off_coef;               // byte offsets of the reverse lists and coefficients in the pool
};

constexpr size_t kPHeadBytes = (sizeof(PairHead) + 15) / 16 * 16;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) / 16 * 16; }

// Bytes of the rebuild's partner masks (one u32 per block of 32 candidates per bead).
__host__ __device__ inline size_t pair_mask_bytes(int n) { return 4 * (size_t)((n + 31) / 32) * (size_t)n; }

__host__ __device__ inline size_t pair_state_bytes(int mx) {
    size_t s = kPHeadBytes;
    s += 3 * sizeof(float4) * (size_t)mx;     // two layers + compensation
    s += sizeof(float2) * (size_t)mx;         // bond lengths
    s += sizeof(float) * (size_t)mx;          // coefficient of the bond (b, b+1)
    s += 8 * sizeof(uint16_t) * (size_t)mx;   // two orders, degree, own, own natives, rev, rev natives, slot of bead
    s += (size_t)mx;                          // flags
    s = align16(s);
    s += 3 * sizeof(float) * (size_t)((mx + 31) & ~31);   // x, y, z arrays of the rebuild scan
    return align16(s);
}

// Bytes the pool needs for so own entries and sr reverse entries: the rows (u16), the
// reverse lists (u32) and the coefficients (f32).
__host__ __device__ inline size_t pair_pool_need(int so, int sr) {
    return (2 * (size_t)so + 3) / 4 * 4 + 4 * (size_t)sr + 4 * (size_t)so;
}

struct PLayout {
    int mx;      // largest system of the launch
    int pool;    // bytes of the pair pool
    __device__ __forceinline__ PairHead *h() const { return reinterpret_cast<PairHead *>(g_smem); }
    __device__ __forceinline__ float4 *lay(int i) const {
        return reinterpret_cast<float4 *>(g_smem + kPHeadBytes) + i * mx;
    }
    __device__ __forceinline__ float4 *comp() const { return lay(2); }
    // by bead: (r0 of bond b-1,b ; r0 of bond b,b+1), < 0 when absent
    __device__ __forceinline__ float2 *bond() const { return reinterpret_cast<float2 *>(lay(3)); }
    // by bead: coefficient of the bond (b, b+1) in this step, NaN when it broke
    __device__ __forceinline__ float *cb() const { return reinterpret_cast<float *>(bond() + mx); }
    __device__ __forceinline__ uint16_t *u16(int i) const { return reinterpret_cast<uint16_t *>(cb() + mx) + i * mx; }
    __device__ __forceinline__ uint16_t *order(int i) const { return u16(i); }   // slot -> bead (two buffers)
    __device__ __forceinline__ uint16_t *n_tot() const { return u16(2); }        // by slot: degree
    __device__ __forceinline__ uint16_t *n_own() const { return u16(3); }        // by slot: own entries
    __device__ __forceinline__ uint16_t *n_own_nat() const { return u16(4); }    // by slot: own natives
    __device__ __forceinline__ uint16_t *n_rev() const { return u16(5); }        // by slot: reverse entries
    __device__ __forceinline__ uint16_t *n_rev_nat() const { return u16(6); }    // by slot: reverse natives
    __device__ __forceinline__ uint16_t *slot_of() const { return u16(7); }      // by bead
    __device__ __forceinline__ uint8_t *flags() const { return reinterpret_cast<uint8_t *>(u16(8)); }
    // rebuild scan: x, y, z of the layer being scanned, stride soa_stride()
    __device__ __forceinline__ int soa_stride() const { return (mx + 31) & ~31; }
    __device__ __forceinline__ float *soa() const {
        return reinterpret_cast<float *>(g_smem + pair_state_bytes(mx) - 3 * sizeof(float) * (size_t)soa_stride());
    }
    __device__ __forceinline__ unsigned char *pool_base() const { return g_smem + pair_state_bytes(mx); }
    // own rows: entry k of slot p at b_own[p / 32] + 32 k + p % 32 (partner bead)
    __device__ __forceinline__ uint16_t *rows() const { return reinterpret_cast<uint16_t *>(pool_base()); }
    // reverse lists: entry q of slot p at b_rev[p / 32] + 32 q + p % 32 (partner | own entry << 16)
    __device__ __forceinline__ uint32_t *rev() const {
        return reinterpret_cast<uint32_t *>(pool_base() + h()->off_rev);
    }
    // coefficient of own entry e in this step
    __device__ __forceinline__ float *coef() const { return reinterpret_cast<float *>(pool_base() + h()->off_coef); }
    // rebuild: Verlet partners of bead b among candidates 32 blk ... 32 blk + 31 at blk * n_s + b,
    // kept at the end of the pool (they are read while rows and reverse lists are written)
    __device__ __forceinline__ uint32_t *masks(int n_s) const {
        return reinterpret_cast<uint32_t *>(pool_base() + ((size_t)pool - pair_mask_bytes(n_s)));
    }
};

// Bits t of the block of candidates base + t (base a multiple of 32) whose pair with bead b
// belongs to b's row: j = base + t > b with b + j odd, or j < b with b + j even.
__device__ __forceinline__ uint32_t own_mask(int b, int base) {
    const uint32_t opp = (b & 1) ? 0x55555555u : 0xAAAAAAAAu;   // j of the other parity
    const int d = b - base;
    const uint32_t above = d < 0 ? 0xffffffffu : (d >= 31 ? 0u : (0xffffffffu << (d + 1)));
    const uint32_t below = d <= 0 ? 0u : (d >= 32 ? 0xffffffffu : ((1u << d) - 1u));
    return (opp & above) | (~opp & below);
}

// Rebuild from layer src: slot order by degree, partner masks, group widths, the pool
// layout, own rows and reverse lists. Ends with a barrier. When the pool is too small the
// CTA's failure code is set and the rows are not written.
template <int BPT>
__device__ __noinline__ int pair_rebuild(const BatchedArgs &a, const PLayout &L, const float4 *src, int n_s, int s, int b0,
                            int ord) {
    const int T = blockDim.x;
    PairHead *H = L.h();
    soa_fill(src, L.soa(), n_s, L.soa_stride());
    ord = reorder_slots(L, n_s, ord);   // ends with a barrier (publishes the x, y, z arrays)
    const uint16_t *order = L.order(ord);
    for (int p = threadIdx.x; p < n_s; p += T) L.slot_of()[order[p]] = (uint16_t)p;
    const int nblk = (n_s + 31) >> 5;
    const float cut2 = a.sa.cut2_f;
    const float lo = cut2 - cut2 * 1e-4f, hi = cut2 + cut2 * 1e-4f;
    const float *soa = L.soa();
    const uint32_t *excl = a.excl + a.excl_off[s];   // systems of the pair form have at most 256 beads
    const int S = L.soa_stride();
    uint32_t *M = L.masks(n_s);
#pragma unroll 1
    for (int k = 0; k < BPT; ++k) {
        const int p = threadIdx.x + k * T;
        int no = 0, nr = 0;
        if (p < n_s) {
            const int b = order[p];
            const int i = b0 + b;
            const float4 pb = src[b];
            for (int blk = 0; blk < nblk; ++blk) {
                const int base = blk << 5;
                // exclusions (self, bonded neighbours, native partners) from the static table
                const uint32_t within = block_partners(scan_block(soa, S, base, n_s - base, pb, lo, hi),
                                                       __ldg(excl + blk * n_s + b), src, base, pb, cut2, a.sa.cut2_d);
                M[blk * n_s + b] = within;
                const uint32_t om = own_mask(b, base);
                no += __popc(within & om);
                nr += __popc(within & ~om);
            }
            const int ono = a.nat_own_cnt[i], onr = a.nat_rev_cnt[i];
            no += ono;
            nr += onr;
            L.n_own()[p] = (uint16_t)no;
            L.n_own_nat()[p] = (uint16_t)ono;
            L.n_rev()[p] = (uint16_t)nr;
            L.n_rev_nat()[p] = (uint16_t)onr;
            L.n_tot()[p] = (uint16_t)min(2 * no + nr, kKeys - 1);   // slot order: the cost of both phases
        }
        // widths of this group of 32 slots (every lane of the warp takes part)
        const int wo = (int)__reduce_max_sync(0xffffffffu, (unsigned)no);
        const int wr = (int)__reduce_max_sync(0xffffffffu, (unsigned)nr);
        const int g = p >> 5;
        if ((threadIdx.x & 31) == 0 && g < nblk) {
            H->w_own[g] = wo;
            H->w_rev[g] = wr;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int so = 0, sr = 0;
        for (int g = 0; g < nblk; ++g) {
            H->b_own[g] = so;
            H->b_rev[g] = sr;
            so += 32 * H->w_own[g];
            sr += 32 * H->w_rev[g];
        }
        H->b_own[nblk] = so;
        H->b_rev[nblk] = sr;
        const int off_rev = (2 * so + 3) / 4 * 4;
        H->off_rev = off_rev;
        H->off_coef = off_rev + 4 * sr;
        // the rows and reverse lists must not reach the masks, which the fill still reads
        if ((size_t)L.pool < pair_pool_need(so, sr) || (size_t)(off_rev + 4 * sr) > (size_t)L.pool - pair_mask_bytes(n_s))
            cta_fail(H, SOP_ERR_PAIRLIST_OVERFLOW);
    }
    __syncthreads();
    if (H->fail != 0) return ord;
    const uint16_t *own_col = a.nat_own_col + a.nat_own_off[s];
    const uint16_t *rev_col = a.nat_rev_col + a.nat_rev_off[s];
    const uint16_t *rev_k = a.nat_rev_k + a.nat_rev_off[s];
    uint16_t *rows = L.rows();
    uint32_t *revl = L.rev();
#pragma unroll 1
    for (int k = 0; k < BPT; ++k) {
        const int p = threadIdx.x + k * T;
        if (p >= n_s) continue;
        const int b = order[p];
        const int g = p >> 5, l = p & 31;
        uint16_t *ro = rows + H->b_own[g] + l;
        const int ono = L.n_own_nat()[p];
        for (int q = 0; q < ono; ++q) ro[32 * q] = __ldg(own_col + q * n_s + b);
        int kk = ono;
        for (int blk = 0; blk < nblk; ++blk) {
            uint32_t m = M[blk * n_s + b] & own_mask(b, blk << 5);
            while (m) {
                const int t = __ffs(m) - 1;
                m &= m - 1;
                ro[32 * kk++] = (uint16_t)((blk << 5) + t);
            }
        }
        uint32_t *rv = revl + H->b_rev[g] + l;
        const int onr = L.n_rev_nat()[p];
        for (int q = 0; q < onr; ++q) {
            const int j = __ldg(rev_col + q * n_s + b);
            const int kj = __ldg(rev_k + q * n_s + b);
            const int sj = L.slot_of()[j];
            const int e = H->b_own[sj >> 5] + 32 * kj + (sj & 31);
            rv[32 * q] = (uint32_t)j | ((uint32_t)e << 16);
        }
        int qq = onr;
        const int bb = b >> 5;
        const uint32_t below_b = (1u << (b & 31)) - 1u;
        for (int blk = 0; blk < nblk; ++blk) {
            uint32_t m = M[blk * n_s + b] & ~own_mask(b, blk << 5);
            while (m) {
                const int t = __ffs(m) - 1;
                m &= m - 1;
                const int j = (blk << 5) + t;
                const int sj = L.slot_of()[j];
                // b's place in the row of its owner j: j's own natives, then j's own Verlet
                // partners below b
                int kj = L.n_own_nat()[sj] + __popc(M[bb * n_s + j] & own_mask(j, bb << 5) & below_b);
                for (int c = 0; c < bb; ++c) kj += __popc(M[c * n_s + j] & own_mask(j, c << 5));
                const int e = H->b_own[sj >> 5] + 32 * kj + (sj & 31);
                rv[32 * qq++] = (uint32_t)j | ((uint32_t)e << 16);
            }
        }
    }
    __syncthreads();
    return ord;
}

// Phase A for bead b in slot p at layer P: the bond (b, b+1) and the pairs of b's own row.
// Stores each pair's coefficient (and the bond's, NaN when it broke) and returns the sum.
__device__ __forceinline__ float3 own_force(const BatchedArgs &a, const PLayout &L, const float4 *P, int n_s,
                                            const float *natr, int b, int p, bool *broken) {
    const ForceParams &fp = a.sa.fp;
    const float4 pb = P[b];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const float r0 = L.bond()[b].y;
    if (r0 > 0.f) {
        const float4 pj = P[b + 1];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float r = r2 * rsqrtf(r2);
        const float dr = r - r0;
        const float arg = fmaf(-dr * dr, fp.inv_R02, 1.0f);
        float c = 0.f;
        if (arg > 0.f) {
            c = __fdividef(-fp.k_fene * dr, arg * r);
            L.cb()[b] = c;
        } else {
            *broken = true;
            L.cb()[b] = __int_as_float(0x7fc00000);
        }
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    const int off = L.h()->b_own[p >> 5] + (p & 31);
    const uint16_t *rp = L.rows() + off;
    float *cp = L.coef() + off;
    const int nno = L.n_own_nat()[p], no = L.n_own()[p];
    const float A = fp.eps12_h, K = fp.rep_k;
    int k = 0;
#pragma unroll 2
    for (; k < nno; ++k) {
        const int j = *rp;
        rp += 32;
        const float s0 = __ldg(natr);
        natr += n_s;
        const float4 pj = P[j];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float inv = __fdividef(1.0f, r2);
        const float s = s0 * inv;
        const float s3 = s * s * s;
        const float c = inv * s3 * fmaf(A, s3, -A);   // (12 eps_h / r^2)(s^6 - s^3)
        *cp = c;
        cp += 32;
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
#pragma unroll 2
    for (; k < no; ++k) {
        const int j = *rp;
        rp += 32;
        const float4 pj = P[j];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float inv = __fdividef(1.0f, r2);
        const float i2 = inv * inv;
        const float c = K * (i2 * i2);                  // 6 eps_l sigma^6 / r^8
        *cp = c;
        cp += 32;
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    return make_float3(fx, fy, fz);
}

// Phase B for bead b in slot p: adds the bond (b-1, b) and the pairs other beads own with b,
// each as c (r_b - r_i) with the owner's coefficient c.
__device__ __forceinline__ float3 rev_force(const PLayout &L, const float4 *P, int b, int p, float3 f, bool *broken) {
    const float4 pb = P[b];
    float fx = f.x, fy = f.y, fz = f.z;
    if (L.bond()[b].x > 0.f) {
        const float c = L.cb()[b - 1];
        if (!(c == c)) {
            *broken = true;
        } else {
            const float4 pj = P[b - 1];
            const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
            fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
        }
    }
    const uint32_t *vp = L.rev() + L.h()->b_rev[p >> 5] + (p & 31);
    const float *C = L.coef();
    const int nr = L.n_rev()[p];
#pragma unroll 2
    for (int q = 0; q < nr; ++q) {
        const uint32_t v = *vp;
        vp += 32;
        const float c = C[v >> 16];
        const float4 pj = P[v & 0xffffu];
        const float dx = pb.x - pj.x, dy = pb.y - pj.y, dz = pb.z - pj.z;
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
    return make_float3(fx, fy, fz);
}

// FP64 observables of the CTA's system at layer P; the Verlet energy over the own rows (each
// pair once).
template <int BPT>
__device__ __noinline__ void pair_observe(const BatchedArgs &a, const PLayout &L, const uint16_t *order,
                                          const float4 *P, int n_s, int b0, int r, int s, int g, int64_t step,
                                          int64_t event) {
    const StepArgs &sa = a.sa;
    const int T = blockDim.x;
    double v[6] = {0, 0, 0, 0, 0, 0};   // E, f_pull, ext, formed, f_wall, r_ee
    const double sig2 = sa.sigma * sa.sigma;
    for (int k = 0; k < BPT; ++k) {
        const int p = threadIdx.x + k * T;
        if (p >= n_s) continue;
        const int b = order[p];
        const float4 pb = P[b];
        obs_bonded(sa, P, b, b0, L.bond()[b].y > 0.f, v);
        const uint16_t *rp = L.rows() + L.h()->b_own[p >> 5] + (p & 31);
        for (int q = L.n_own_nat()[p]; q < L.n_own()[p]; ++q) {
            const float4 pj = P[rp[32 * q]];
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

template <int BPT, int MINB, int MAXT>
__global__ void __launch_bounds__(MAXT, MINB) k_bpair(BatchedArgs a) {
    const int item = blockIdx.x;
    PLayout L;
    L.mx = a.max_n;
    L.pool = a.pair_pool;
    const int r = a.item_rep[item], s = a.item_sys[item];
    const StepArgs &sa = a.sa;
    const DevTopo &t = sa.topo;
    const int b0 = t.sys_lo[s], n_s = t.sys_lo[s + 1] - b0;
    const int gbase = r * t.n + b0;   // replicas x beads < 2^28
    const int g = r * t.n_sys + s;
    const float *natr0 = a.nat_own_r0sq + a.nat_own_off[s];
    const int T = blockDim.x;
    const int64_t step0 = *a.d_step;
    const bool forces_only = (a.n_steps == 0 && a.force_out != nullptr);

    if (threadIdx.x == 0) L.h()->fail = 0;
    if (!forces_only && (sa.rep_status[r] != 0 || *sa.halt != 0)) {   // CTA-uniform: a frozen replica
        if (threadIdx.x == 0)                                           // only marks its records
            missing_records(a, r, s, g, step0, step0, a.d_events ? *a.d_events : 0);
        return;
    }
    int k_phase = (int)(step0 % a.K);
    int o_phase = a.obs_every > 0 ? (int)(step0 % a.obs_every) : 0;
    for (int b = threadIdx.x; b < n_s; b += T) {
        const int i = b0 + b;
        L.lay(0)[b] = a.pos[gbase + b];
        L.comp()[b] = a.comp[gbase + b];
        L.bond()[b] = make_float2(b > 0 ? t.bond_r0[i - 1] : -1.f, t.bond_r0[i]);
        L.flags()[b] = t.flags[i];
        L.order(0)[b] = (uint16_t)b;
        L.n_tot()[b] = (uint16_t)min(2 * a.nat_own_cnt[i] + a.nat_rev_cnt[i], kKeys - 1);
        if (k_phase != 0) L.lay(1)[b] = a.snap[gbase + b];
    }
    __syncthreads();

    int cur = 0, ord = 0, n_events = 0;
    bool built_now = false;
    int it = 0;
    // a replica that fails takes no record after this step (the records of later cadence
    // events of the chunk are written as NaN)
    int64_t miss_after = 0;
    for (; it < a.n_steps || (forces_only && it == 0); ++it) {
        const float4 *P = L.lay(cur);
        float4 *Q = L.lay(cur ^ 1);
        if (it == 0 && k_phase != 0 && !forces_only) {
            ord = pair_rebuild<BPT>(a, L, Q, n_s, s, b0, ord);   // Q holds the snapshot here
        } else if ((k_phase == 0 && !built_now) || forces_only) {
            ord = pair_rebuild<BPT>(a, L, P, n_s, s, b0, ord);
            // the snapshot is kept only from the launch's last rebuild: a later launch that
            // starts between rebuilds builds its first list from it
            if (!forces_only && it + a.K >= a.n_steps)
                for (int b = threadIdx.x; b < n_s; b += T) a.snap[gbase + b] = P[b];
        }
        built_now = false;
        if (L.h()->fail != 0) {   // the rows did not fit: the replica stops before this step
            miss_after = step0 + it;
            break;
        }
        const int64_t step = step0 + it;
        const uint16_t *order = L.order(ord);
        float3 fa[BPT];
        bool brk[BPT];
#pragma unroll
        for (int k = 0; k < BPT; ++k) {
            const int p = threadIdx.x + k * T;
            brk[k] = false;
            fa[k] = make_float3(0.f, 0.f, 0.f);
            if (p < n_s) {
                const int b = order[p];
                fa[k] = own_force(a, L, P, n_s, natr0 + b, b, p, &brk[k]);
            }
        }
        __syncthreads();
        if (forces_only) {
#pragma unroll
            for (int k = 0; k < BPT; ++k) {
                const int p = threadIdx.x + k * T;
                if (p >= n_s) continue;
                const int b = order[p];
                bool broken = brk[k], overlap = false;
                const float3 f = rev_force(L, P, b, p, fa[k], &broken);
                const float3 fe = ext_force(sa, r, b0 + b, L.flags()[b], P[b], step, &overlap);
                a.force_out[gbase + b] = make_float4(f.x + fe.x, f.y + fe.y, f.z + fe.z, (broken || overlap) ? 1.f : 0.f);
                if (a.pl_dump_col) {
                    const size_t rowi = (size_t)gbase + b;
                    const int nno = L.n_own_nat()[p], no = L.n_own()[p];
                    const int nrn = L.n_rev_nat()[p], nr = L.n_rev()[p];
                    a.pl_dump_start[rowi] = (int)(rowi * a.pl_dump_stride);
                    // the full row (both directions); a row longer than the stride is reported
                    // by its length and written only up to the stride
                    a.pl_dump_len[rowi] = (no - nno) + (nr - nrn);
                    int w = 0;
                    const uint16_t *rp = L.rows() + L.h()->b_own[p >> 5] + (p & 31);
                    for (int q = nno; q < no && w < a.pl_dump_stride; ++q)
                        a.pl_dump_col[rowi * a.pl_dump_stride + w++] = b0 + (int)rp[32 * q];
                    const uint32_t *vp = L.rev() + L.h()->b_rev[p >> 5] + (p & 31);
                    for (int q = nrn; q < nr && w < a.pl_dump_stride; ++q)
                        a.pl_dump_col[rowi * a.pl_dump_stride + w++] = b0 + (int)(vp[32 * q] & 0xffffu);
                }
            }
            break;
        }
#pragma unroll
        for (int k = 0; k < BPT; ++k) {
            const int p = threadIdx.x + k * T;
            if (p >= n_s) continue;
            const int b = order[p];
            bool broken = brk[k], overlap = false;
            const float3 f = rev_force(L, P, b, p, fa[k], &broken);
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
        if (L.h()->fail != 0) {   // the replica freezes after the step in which it failed
            miss_after = step0 + it;
            ++it;
            break;
        }
        if (a.obs_every > 0 && o_phase == 0) {
            const float4 *Pn = L.lay(cur);
            if (k_phase == 0) {
                ord = pair_rebuild<BPT>(a, L, Pn, n_s, s, b0, ord);
                built_now = true;
                if (it + 1 + a.K >= a.n_steps)
                    for (int b = threadIdx.x; b < n_s; b += T) a.snap[gbase + b] = Pn[b];
                if (L.h()->fail != 0) {
                    miss_after = step0 + it;
                    ++it;
                    break;
                }
            }
            const int64_t ev = (a.d_events ? *a.d_events : 0) + n_events;
            pair_observe<BPT>(a, L, L.order(ord), Pn, n_s, b0, r, s, g, step + 1, ev);
            ++n_events;
        }
    }
    if (forces_only) return;
    if (threadIdx.x == 0 && L.h()->fail != 0)
        missing_records(a, r, s, g, step0, miss_after, (a.d_events ? *a.d_events : 0) + n_events);
    const float4 *P = L.lay(cur);
    for (int b = threadIdx.x; b < n_s; b += T) {
        a.pos[gbase + b] = P[b];
        a.comp[gbase + b] = L.comp()[b];
    }
    if (threadIdx.x == 0 && L.h()->fail != 0) atomicCAS(&sa.rep_status[r], 0, L.h()->fail);
}

template <int BPT, int MINB>
cudaError_t launch_p(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s) {
    auto kern = k_bpair<BPT, MINB, 256>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    kern<<<a.n_items, cfg.threads, cfg.smem, s>>>(a);
    return cudaGetLastError();
}

template <int BPT, int MINB>
int resident_p(const BatchedConfig &cfg) {
    auto kern = k_bpair<BPT, MINB, 256>;
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

bool pair_config(int max_n, int pool, int threads, int min_blocks, BatchedConfig *cfg) {
    if (max_n <= 0 || max_n > kPairMaxBeads || threads % 32 || threads < 32 || threads > 256) return false;
    if (pool <= (int)pair_mask_bytes(max_n) || pool % 16) return false;
    if (min_blocks < 2 || min_blocks > 4) return false;
    const int bpt = (max_n + threads - 1) / threads;
    const int bpt_c = bpt <= 1 ? 1 : bpt <= 2 ? 2 : bpt <= 4 ? 4 : 8;
    if (bpt_c > 4) return false;
    cfg->threads = threads;
    cfg->beads_per_thread = bpt_c;
    cfg->min_blocks = min_blocks;
    cfg->rows_global = false;
    cfg->row_width = 0;
    cfg->cluster = 0;
    cfg->m_shift = 0;
    cfg->pair_form = true;
    cfg->smem = pair_state_bytes(max_n) + (size_t)pool;
    return cfg->smem <= 227 * 1024;
}

size_t pair_pool_bytes(int so, int sr, int n) {
    const size_t need = pair_pool_need(so, sr);
    const size_t with_masks = (2 * (size_t)so + 3) / 4 * 4 + 4 * (size_t)sr + pair_mask_bytes(n);
    return align16(need > with_masks ? need : with_masks);
}

cudaError_t launch_bpair(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s) {
    const int b = cfg.beads_per_thread;
    switch (cfg.min_blocks) {
    case 2: return b == 1 ? launch_p<1, 2>(a, cfg, s) : b == 2 ? launch_p<2, 2>(a, cfg, s) : launch_p<4, 2>(a, cfg, s);
    case 3: return b == 1 ? launch_p<1, 3>(a, cfg, s) : b == 2 ? launch_p<2, 3>(a, cfg, s) : launch_p<4, 3>(a, cfg, s);
    default: return b == 1 ? launch_p<1, 4>(a, cfg, s) : b == 2 ? launch_p<2, 4>(a, cfg, s) : launch_p<4, 4>(a, cfg, s);
    }
}

int bpair_resident_ctas(const BatchedConfig &cfg) {
    const int b = cfg.beads_per_thread;
    switch (cfg.min_blocks) {
    case 2: return b == 1 ? resident_p<1, 2>(cfg) : b == 2 ? resident_p<2, 2>(cfg) : resident_p<4, 2>(cfg);
    case 3: return b == 1 ? resident_p<1, 3>(cfg) : b == 2 ? resident_p<2, 3>(cfg) : resident_p<4, 3>(cfg);
    default: return b == 1 ? resident_p<1, 4>(cfg) : b == 2 ? resident_p<2, 4>(cfg) : resident_p<4, 4>(cfg);
    }
}

}  // namespace sop
