// Device-side building blocks of the SOP-model Langevin step (sm_103a).
//
// Pair terms of Eq. 1 (FENE, native 12-6, (sigma/r)^6 repulsion) in FP32,
// counter-based Philox4x32-10 noise with a Box-Muller transform (Sec. III.C),
// and the first-order update of Algorithm 7 with a compensated (Kahan) sum.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sop {

// Philox4x32 multipliers and Weyl key increments (Salmon et al., SC'11).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Philox4x32-10: ten rounds; each multiplies words 0 and 2, crosses the
// product halves over the lanes and xors in the key; the key advances between
// rounds by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        const uint32_t lo0 = kPhiloxM0 * c.x;
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
        const uint32_t lo1 = kPhiloxM1 * c.z;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// -2 ln(u) for u = (x + 1) 2^-32 in (0, 1], without branches, to a few ulp. Write
// u = 2^e (1 - t) with t in [0, 1/2]: then ln u = e ln 2 + ln(1 - t), and
// ln(1 - t) = -2 atanh(z) with z = t / (2 - t) in [0, 1/3], where atanh is summed by its
// odd power series z + z^3/3 + ... + z^13/13 (the identity ln((1 + z)/(1 - z)) = 2 atanh z;
// the first omitted term is below 2^-26 of the sum at z = 1/3). For u >= 1/2 the
// complement 1 - u = (2^32 - 1 - x) 2^-32 is known exactly (e = 0), so u near 1 keeps its
// relative accuracy; below, u is rounded to FP32 and its mantissa f in [1/2, 1) gives
// t = 1 - f exactly. Both terms of the result are >= 0: no cancellation.
__device__ __forceinline__ float minus_two_log_u(uint32_t x) {
    const float two_m32 = 2.3283064365386963e-10f;  // 2^-32
    const bool upper = x >= 0x80000000u;
    const float u = fmaf((float)x, two_m32, two_m32);
    const uint32_t ub = __float_as_uint(u);
    const int e_lo = (int)(ub >> 23) - 126;         // u = f 2^e_lo
    const float f = __uint_as_float((ub & 0x007FFFFFu) | 0x3F000000u);
    const float t = upper ? (float)(~x) * two_m32 : 1.0f - f;
    const float e = upper ? 0.0f : (float)e_lo;
    const float z = __fdividef(t, 2.0f - t);
    const float w = z * z;
    float p = 1.0f / 13.0f;
    p = fmaf(p, w, 1.0f / 11.0f);
    p = fmaf(p, w, 1.0f / 9.0f);
    p = fmaf(p, w, 1.0f / 7.0f);
    p = fmaf(p, w, 1.0f / 5.0f);
    p = fmaf(p, w, 1.0f / 3.0f);
    p = fmaf(p, w, 1.0f);                           // atanh(z) = z p
    const float ln2 = 0.6931471805599453f;
    return fmaf(-2.0f * e, ln2, 4.0f * z * p);
}

// Three standard normals from one Philox block (Box-Muller): the pair
// (x0, x1) gives radius sqrt(-2 ln u1) and angle 2 pi u2 (cos, sin); the pair
// (x2, x3) gives the third normal from its cosine. The fourth is not used.
__device__ __forceinline__ float3 box_muller3(uint4 x) {
    const float two_m31 = 4.656612873077393e-10f;  // 2^-31, so that 2 pi u = pi * (x 2^-31)
    const float ra = sqrtf(minus_two_log_u(x.x));
    const float rb = sqrtf(minus_two_log_u(x.z));
    float s, c;
    sincospif((float)x.y * two_m31, &s, &c);
    const float c2 = cospif((float)x.w * two_m31);
    return make_float3(ra * c, ra * s, rb * c2);
}

// Gaussian 3-vector of bead `bead` at step `step` of the replica keyed by `seed`:
// key = seed (lo, hi), counter = (step lo, step hi, bead, 0).
__device__ __forceinline__ float3 bead_noise(uint64_t seed, int64_t step, uint32_t bead) {
    const uint64_t s = (uint64_t)step;
    const uint4 ctr = make_uint4((uint32_t)s, (uint32_t)(s >> 32), bead, 0u);
    return box_muller3(philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Hybrid Taus (Algorithm 6): three Tausworthe components in L'Ecuyer's shift form
// b = ((y << q) ^ y) >> (k - s), y = ((y & mask) << s) ^ b with (q, k - s, s, mask) =
// (13, 19, 12, 0xFFFFFFFE), (2, 25, 4, 0xFFFFFFF8), (3, 11, 17, 0xFFFFFFF0), and the LCG
// y4 = 1664525 y4 + 1013904223 (mod 2^32); the output is y1 ^ y2 ^ y3 ^ y4.
__device__ __forceinline__ uint32_t taus_next(uint4 &s) {
    s.x = (((s.x & 0xFFFFFFFEu) << 12) ^ (((s.x << 13) ^ s.x) >> 19));
    s.y = (((s.y & 0xFFFFFFF8u) << 4) ^ (((s.y << 2) ^ s.y) >> 25));
    s.z = (((s.z & 0xFFFFFFF0u) << 17) ^ (((s.z << 3) ^ s.z) >> 11));
    s.w = 1664525u * s.w + 1013904223u;
    return s.x ^ s.y ^ s.z ^ s.w;
}

// Three normals from four successive outputs, mapped like one Philox block.
__device__ __forceinline__ float3 taus_noise(uint4 &s) {
    uint4 x;
    x.x = taus_next(s);
    x.y = taus_next(s);
    x.z = taus_next(s);
    x.w = taus_next(s);
    return box_muller3(x);
}

// Physical constants of one run, FP32 copies for the force loop.
struct ForceParams {
    float k_fene;     // k
    float inv_R02;    // 1 / R0^2
    float eps12_h;    // 12 eps_h
    float eps6_l;     // 6 eps_l
    float rep_k;      // 6 eps_l sigma^6 (repulsion: F = rep_k / r^8 d)
    float sigma2;     // sigma^2
    float mob;        // h / zeta
    float amp;        // sqrt(2 kT h / zeta)
};

// FENE: F_i = -k (r - r0) / (1 - (r - r0)^2 / R0^2) * d / r, d = r_i - r_j.
// Returns the coefficient multiplying d; sets *broken when |r - r0| >= R0.
__device__ __forceinline__ float fene_coef(float r2, float r0, const ForceParams &fp, bool *broken) {
    const float r = sqrtf(r2);
    const float dr = r - r0;
    const float arg = 1.0f - dr * dr * fp.inv_R02;
    if (!(arg > 0.0f)) {
        *broken = true;
        return 0.0f;
    }
    return -fp.k_fene * dr / (arg * r);
}

// Native 12-6: F_i = (12 eps_h / r^2) (s^6 - s^3) d with s = r0^2 / r^2. The reciprocal is
// the fast approximate one (within 2 ulp), as in the batched forms' row_force.
__device__ __forceinline__ float native_coef(float r2, float r0sq, const ForceParams &fp) {
    const float inv_r2 = __fdividef(1.0f, r2);
    const float s = r0sq * inv_r2;
    const float s3 = s * s * s;
    return inv_r2 * s3 * fmaf(fp.eps12_h, s3, -fp.eps12_h);
}

// Repulsion: F_i = (6 eps_l / r^2) (sigma^2 / r^2)^3 d = 6 eps_l sigma^6 / r^8 d.
__device__ __forceinline__ float repulsive_coef(float r2, const ForceParams &fp) {
    const float inv_r2 = __fdividef(1.0f, r2);
    const float i4 = inv_r2 * inv_r2;
    return fp.rep_k * (i4 * i4);
}

// Compensated (Kahan) accumulation of one step's displacement.
__device__ __forceinline__ void kahan_add(float &x, float &c, float delta) {
    const float y = delta - c;
    const float t = x + y;
    c = (t - x) - y;
    x = t;
}

// Is the squared distance below cut^2? FP32 decides unless the value lies within a
// relative 1e-4 of the cutoff; there the FP64 expression ((dx*dx + dy*dy) + dz*dz)
// of the same FP32 positions decides (round-to-nearest, no contraction), so the
// outcome equals an FP64 evaluation of the definition.
__device__ __forceinline__ bool within_cut(float4 a, float4 b, float cut2_f, double cut2_d) {
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float band = cut2_f * 1e-4f;
    if (r2 < cut2_f - band) return true;
    if (r2 > cut2_f + band) return false;
    const double ex = __dsub_rn((double)a.x, (double)b.x);
    const double ey = __dsub_rn((double)a.y, (double)b.y);
    const double ez = __dsub_rn((double)a.z, (double)b.z);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    return d2 < cut2_d;
}

// 1/x in FP64 for finite x > 0: the FP32 reciprocal (24 bits) refined by two Newton steps
// y <- y + y (1 - x y), each of which squares the relative error (to about 1e-15 here).
// Cheaper than an FP64 division on a GPU whose FP64 pipe runs at a small fraction of its
// FP32 rate; used for the terms of the FP64 readouts, which are compared at 1e-9 relative.
__device__ __forceinline__ double rcp_fast(double x) {
    double y = (double)__frcp_rn((float)x);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// sqrt(x) in FP64 for finite x > 0: the FP32 1/sqrt refined by two Newton steps
// y <- y (3 - x y^2) / 2, times x (relative error about 1e-15), for the same readouts.
__device__ __forceinline__ double sqrt_fast(double x) {
    double y = (double)rsqrtf((float)x);
    y = y * fma(-0.5 * x * y, y, 1.5);
    y = y * fma(-0.5 * x * y, y, 1.5);
    return x * y;
}

// FP32 -> FP64 from the IEEE-754 encodings, in integer operations: a normal float's
// exponent is rebiased (127 -> 1023) and its 23 fraction bits become the top of the 52.
// Zero, subnormal, infinite and NaN inputs take the conversion instruction. Exact, like
// the conversion, but off the FP64 pipe, which is narrow on this GPU (about 2 operations
// per cycle per SM) and also executes the conversions.
__device__ __forceinline__ double f2d(float f) {
    const unsigned b = __float_as_uint(f);
    if (((b >> 23) & 0xffu) - 1u >= 254u) return (double)f;
    const unsigned hi = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(b << 29));
}

// Knuth's TwoSum: returns s = fl(a + b) and sets e with s + e = a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// |a - b|^2 of two FP32 points as an FP64 value, computed in FP32: each difference exactly
// as s + e (TwoSum, |e| <= 2^-24 |s|), each s^2 exactly as p + q (an FMA gives q), the three
// p summed exactly into a two-float P + (u + v), and the small terms u + v + q + 2 s e
// (at most about 2^-21 of the total) added in FP32. The result is within about 2^-42
// (2e-13) relative of the exact squared distance; *d2f is the same value in FP32 (relative
// 2^-24), a seed for rcp_seeded. Against the FP64 evaluation of the definition it trades
// nine FP64 operations and six conversions for some thirty FP32 ones.
__device__ __forceinline__ double dist2_two(float4 a, float4 b, float *d2f) {
    float e0, e1, e2;
    const float s0 = two_sum(a.x, -b.x, e0);
    const float s1 = two_sum(a.y, -b.y, e1);
    const float s2 = two_sum(a.z, -b.z, e2);
    const float p0 = __fmul_rn(s0, s0), p1 = __fmul_rn(s1, s1), p2 = __fmul_rn(s2, s2);
    const float q0 = __fmaf_rn(s0, s0, -p0), q1 = __fmaf_rn(s1, s1, -p1), q2 = __fmaf_rn(s2, s2, -p2);
    float u, v;
    const float t = two_sum(p0, p1, u);
    const float P = two_sum(t, p2, v);
    const float cross = __fmaf_rn(s0, e0, __fmaf_rn(s1, e1, __fmul_rn(s2, e2)));
    const float lo = __fmaf_rn(2.0f, cross, __fadd_rn(__fadd_rn(u, v), __fadd_rn(__fadd_rn(q0, q1), q2)));
    *d2f = __fadd_rn(P, lo);
    return __dadd_rn(f2d(P), f2d(lo));
}

// 1/x in FP64 for finite x > 0, given xf, x rounded to FP32: the FP32 reciprocal of xf
// (relative error below 2^-23) refined by one Newton step y + y (1 - x y), which squares
// the error (to about 1e-14).
__device__ __forceinline__ double rcp_seeded(double x, float xf) {
    const double y = f2d(__frcp_rn(xf));
    return fma(y, fma(-x, y, 1.0), y);
}

// sqrt(x) in FP64 for finite x > 0, given xf, x rounded to FP32: 1/sqrt(xf) refined by two
// Newton steps y <- y (3 - x y^2) / 2, times x (relative error about 1e-15).
__device__ __forceinline__ double sqrt_seeded(double x, float xf) {
    double y = f2d(rsqrtf(xf));
    y = y * fma(-0.5 * x * y, y, 1.5);
    y = y * fma(-0.5 * x * y, y, 1.5);
    return x * y;
}

// FP64 squared distance ((dx*dx + dy*dy) + dz*dz) with no contraction.
__device__ __forceinline__ double dist2_d(double ax, double ay, double az, double bx, double by, double bz) {
    const double ex = __dsub_rn(ax, bx);
    const double ey = __dsub_rn(ay, by);
    const double ez = __dsub_rn(az, bz);
    return __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
}

// Is the native pair (a, b) formed, r < r0 + 2 A (Q)? d2 is their squared distance to a
// relative 1e-12 or better (dist2_d, dist2_two). Away from the threshold d2 against
// (r0 + 2)^2 decides; within a relative 1e-10 of it the correctly rounded square root of
// the FP64 definition ((dx*dx + dy*dy) + dz*dz) of the same FP32 positions does, so the
// outcome is always that of the definition evaluated in FP64.
__device__ __forceinline__ bool native_formed(double d2, double r0, float4 a, float4 b) {
    const double t = r0 + 2.0, t2 = t * t;
    if (d2 < t2 * (1.0 - 1e-10)) return true;
    if (d2 > t2 * (1.0 + 1e-10)) return false;
    return __dsqrt_rn(dist2_d(f2d(a.x), f2d(a.y), f2d(a.z), f2d(b.x), f2d(b.y), f2d(b.z))) < t;
}

}  // namespace sop
