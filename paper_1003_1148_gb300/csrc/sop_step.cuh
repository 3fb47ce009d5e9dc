// Per-bead pieces of a streamed step shared by the particle-based form (k_stream.cu)
// and the pair-based form (k_pairs.cu): the cantilever and indenter forces, the failure
// checks, the Philox noise and the compensated first-order update of Algorithm 7.
#pragma once

#include "sop_internal.h"

namespace sop {

__device__ __forceinline__ void set_status(int32_t *st, int32_t code) { atomicCAS(st, 0, code); }

// Lanes of this thread's group of L (groups are aligned within the warp).
template <int L>
__device__ __forceinline__ unsigned group_mask() {
    return L == 32 ? 0xffffffffu : (((1u << L) - 1u) << ((threadIdx.x & 31) & ~(L - 1)));
}

// FENE forces of bead i's cross-links (the topology's extra bonds, Eq. 1's first term
// with each link's native length), added to (fx, fy, fz) by lane `lane` of a group of L
// lanes striding over the bead's cross-link row; *broken is set at |r - r0| >= R0.
template <int L>
__device__ __forceinline__ void xlink_force(const DevTopo &t, const ForceParams &fp, const float4 *P, int i,
                                            float4 pi, int lane, float &fx, float &fy, float &fz, bool *broken) {
    if (!t.xb_row) return;
    for (int p = t.xb_row[i] + lane; p < t.xb_row[i + 1]; p += L) {
        const float4 pj = P[t.xb_col[p]];
        const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        const float c = fene_coef(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), t.xb_r0[p], fp, broken);
        fx = fmaf(c, dx, fx); fy = fmaf(c, dy, fy); fz = fmaf(c, dz, fz);
    }
}

// Cantilever and indenter forces on bead i (FP64 tip / centre, FP32 force).
__device__ __forceinline__ float3 external_force(const StepArgs &a, int r, int i, float4 pi, int64_t step,
                                                 bool *overlap) {
    float3 f = make_float3(0.f, 0.f, 0.f);
    const DevTopo &t = a.topo;
    const DevExternal &e = a.ext;
    if (t.flags[i] & kFlagPulled) {
        const int q = e.pull_of_sys[t.sys[i]];
        if (q >= 0 && e.pull_bead[q] == i) {
            const double tt = e.pull_v[q] * ((double)step - e.pull_n0[q]);
            const double *tip0 = e.pull_tip0 + ((size_t)r * e.n_pull + q) * 3;
            const float ks = (float)e.pull_ks[q];
            f.x += ks * (float)(tip0[0] + tt * e.pull_dir[3 * q] - (double)pi.x);
            f.y += ks * (float)(tip0[1] + tt * e.pull_dir[3 * q + 1] - (double)pi.y);
            f.z += ks * (float)(tip0[2] + tt * e.pull_dir[3 * q + 2] - (double)pi.z);
        }
    }
    if (e.has_indenter) {
        const double tt = e.ind_v * ((double)step - e.ind_n0);
        const float cx = (float)(e.ind_c0[0] + tt * e.ind_dir[0]);
        const float cy = (float)(e.ind_c0[1] + tt * e.ind_dir[1]);
        const float cz = (float)(e.ind_c0[2] + tt * e.ind_dir[2]);
        const float ex = pi.x - cx, ey = pi.y - cy, ez = pi.z - cz;
        const float rr = sqrtf(fmaf(ez, ez, fmaf(ey, ey, ex * ex)));
        const float rho = rr - (float)e.ind_radius;
        if (!(rho > 0.f)) {
            *overlap = true;
        } else {
            const float q = a.fp.sigma2 > 0.f ? sqrtf(a.fp.sigma2) / rho : 0.f;
            const float q2 = q * q;
            const float q6 = q2 * q2 * q2;
            const float c = a.fp.eps6_l * q6 / (rho * rr);
            f.x = fmaf(c, ex, f.x); f.y = fmaf(c, ey, f.y); f.z = fmaf(c, ez, f.z);
        }
    }
    return f;
}

// Algorithm 7 (or the BAOAB step of the underdamped integrator) for one bead that moves:
// F is the total force (pair terms plus external), i the bead's index in its replica (the
// Philox counter), gidx its index in the per-bead arrays of all replicas (Hybrid Taus
// state, velocities). p and c are the position and its compensation, updated in place when
// the result is finite; false (p, c and the velocity untouched) otherwise. Every schedule
// calls this one function, so all of them take the same arithmetic in the same order.
__device__ __forceinline__ bool update_position(const StepArgs &a, int r, int i, size_t gidx, float4 &p, float4 &c,
                                                float3 F, int64_t step) {
    float3 g;
    if (a.taus) {
        uint4 st = a.taus[gidx];
        g = taus_noise(st);
        a.taus[gidx] = st;
    } else {
        g = bead_noise(a.seed + (uint64_t)r, step, (uint32_t)i);
    }
    float4 pn = p, cn = c, w;
    if (a.vel) {   // underdamped: BAOAB with the stored post-O velocity w
        w = a.vel[gidx];
        const float v1x = fmaf(F.x, a.h_m, w.x), v1y = fmaf(F.y, a.h_m, w.y), v1z = fmaf(F.z, a.h_m, w.z);
        w.x = fmaf(a.c1, v1x, a.c2 * g.x);
        w.y = fmaf(a.c1, v1y, a.c2 * g.y);
        w.z = fmaf(a.c1, v1z, a.c2 * g.z);
        kahan_add(pn.x, cn.x, a.half_h * (v1x + w.x));
        kahan_add(pn.y, cn.y, a.half_h * (v1y + w.y));
        kahan_add(pn.z, cn.z, a.half_h * (v1z + w.z));
    } else {
        kahan_add(pn.x, cn.x, fmaf(F.x, a.fp.mob, g.x * a.fp.amp));
        kahan_add(pn.y, cn.y, fmaf(F.y, a.fp.mob, g.y * a.fp.amp));
        kahan_add(pn.z, cn.z, fmaf(F.z, a.fp.mob, g.z * a.fp.amp));
    }
    if (!(isfinite(pn.x) && isfinite(pn.y) && isfinite(pn.z))) return false;
    if (a.vel) a.vel[gidx] = w;
    p = pn;
    c = cn;
    return true;
}

// The end of one step for bead i of replica r (global index gb) given the sum f of its
// pair forces at layer P: a broken bond or an indenter overlap leaves the bead where it
// is and marks the replica; a fixed bead stays; otherwise it moves (update_position).
__device__ __forceinline__ void advance_bead(const StepArgs &a, int r, int i, int gb, const float4 *P, float3 f,
                                             bool broken, int64_t step, float4 *pos_out, float4 *comp) {
    float4 pi = P[i];
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
    if (a.topo.flags[i] & kFlagFixed) {
        pos_out[gb] = pi;
        return;
    }
    float4 c = comp[gb];
    if (!update_position(a, r, i, gb, pi, c, make_float3(f.x + fe.x, f.y + fe.y, f.z + fe.z), step)) {
        set_status(&a.rep_status[r], (int32_t)SOP_ERR_NONFINITE);
        pos_out[gb] = P[i];
        return;
    }
    comp[gb] = c;
    pos_out[gb] = pi;
}

}  // namespace sop
