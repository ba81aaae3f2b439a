// wn_kernels.cu -- query kernels of the containment library (sm_103a).
//
// Mixed path (WN_PREC_MIXED), per call:
//   k_bin_*       spatial bucketing: each domain's queries sorted into small
//                 cells, so that a warp's queries lie close together.
//   k_sweep_tree  persistent warps pop (domain, query-tile) units and walk
//                 the record tree of every instance their queries see (the
//                 flat k_sweep instead stages the records in shared memory).
//                 Per record reached, the root step of Algorithm 1 in FP32:
//                 a circle that contains the ellipse of Eq. 4, then the
//                 ellipse of Eq. 5, then the box of the segment's control
//                 points (each inflated by its FP32 error bound) decide
//                 "far"; a far chord then contributes its signed crossing of
//                 the +x ray from the query (the chord's Eq. 3 angle is an
//                 integer multiple of 2 pi plus endpoint angles that cancel
//                 around each loop), and every gap between consecutive
//                 segments contributes its own crossing and its exact small
//                 angle.  A node whose records are all far contributes its
//                 crossings in O(1) and its gap angles by an expansion.
//                 Pairs that are not far go to a queue.
//   k_near        FP32 Algorithm 1 on each queued pair in query-relative
//                 coordinates; every test carries an error band, and a pair
//                 whose band cannot settle a decision hands its tail to FP64.
//   k_f64items    Algorithm 1 in FP64 on those tails.  (Both walks also test
//                 a rational segment's nodes against the derivative bound of
//                 the eighth of [0, 1] they lie in.)
//   k_finalize    omega = crossings + line terms / 2 - sum(gap angles) / 2 pi;
//                 a query whose omega lies within 1e-4 of 1/2, or that any
//                 kernel flagged, is recomputed in FP64 (k_finalize4 and
//                 k_finalize_bits4: the same, four queries per thread, for
//                 aligned outputs and for bitmasks).
//   k_f64query    the FP64 recomputation of those queries (crossing form).
// Plain path (WN_PREC_PLAIN_FP64): k_plain, one thread per query running
// Algorithm 1 in FP64 on every segment the query sees, chord angles summed
// with atan2 (Eq. 3) -- the paper's method ported as is.
#include <algorithm>

#include <cooperative_groups.h>

#include "wn_internal.h"

namespace cg = cooperative_groups;

namespace wn {

constexpr float kTwoM22 = 2.384185791015625e-7f;   // 2^-22
constexpr float kTwoM24 = 5.9604644775390625e-8f;  // 2^-24
constexpr float kTwoM44 = 5.684341886080802e-14f;  // 2^-44
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float kOmegaBandF = 1e-4f;               // classification band of the mixed path
constexpr float kInv2PiF = 0.15915494309189533577f;
constexpr float kInv2PiLoF = 6.4206382432985265e-09f;   // 1/(2 pi) - kInv2PiF
constexpr int kChunk = 64;                          // records per shared-memory stage

__device__ __forceinline__ void get_point(const PointSrc &s, uint32_t q, double &x, double &y)
{
    if (s.pts) {
        double2 v = __ldg(reinterpret_cast<const double2 *>(s.pts) + q);
        x = v.x;
        y = v.y;
    } else {
        uint32_t i = q % (uint32_t)s.nu, j = q / (uint32_t)s.nu;
        x = ((double)i + 0.5) / (double)s.nu * s.su;
        y = ((double)j + 0.5) / (double)s.nv * s.sv;
    }
}

// FP64 instructions, conversions included, run on GB300's narrow FP64 unit;
// the two conversions below use integer instructions only.
//
// The double whose value is the float f (exact): the exponent re-biased and
// the fraction widened; zeros, infinities and NaNs keep their kind, a
// subnormal float becomes a normal double.
__device__ __forceinline__ double f32_to_f64_exact(float f)
{
    const uint32_t u = __float_as_uint(f);
    const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
    const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    if (e == 0xffu) return __longlong_as_double(s | 0x7ff0000000000000ULL | ((unsigned long long)m << 29));
    if (e == 0u) {
        if (m == 0u) return __longlong_as_double(s);
        const int p = 31 - __clz(m);                           // m = 2^p (1 + r), value m 2^-149
        const uint32_t r = (m << (23 - p)) & 0x7fffffu;
        return __longlong_as_double(s | ((unsigned long long)(p + 874) << 52) | ((unsigned long long)r << 29));
    }
    return __longlong_as_double(s | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29));
}

// The double x truncated to FP32 (toward zero), for choices that need no
// exactness: magnitudes below FP32's normal range give 0, above it (and
// infinities and NaNs) an infinity of x's sign.
__device__ __forceinline__ float f64_to_f32_trunc(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// The remainder x - f64_to_f32_trunc(x) (the low 29 bits of x's fraction)
// as an FP32 value, with integer instructions and one conversion: within
// 2^-24 of itself, so the pair (trunc, remainder) is x within 2^-47 |x|.
// For |x| < 2^-74 the remainder (below 2^-97) is dropped; for |x| >= 2^180
// it is not formed (such a query is escalated).
__device__ __forceinline__ float f64_rem_f32(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu);
    if (e < 949 || e > 1202) return 0.f;
    const float r = __uint2float_rn((uint32_t)b & 0x1fffffffu) * __int_as_float((e - 948) << 23);   // * 2^(e-1075)
    return (b >> 63) ? -r : r;
}

// An interval of FP32 values around a truncated coordinate r (within 2^-23
// of the double it came from, or below 2^-126) that holds that double.
__device__ __forceinline__ float pt_lo(float r) { return r - fabsf(r) * 2.384185791015625e-7f - 1e-30f; }
__device__ __forceinline__ float pt_hi(float r) { return r + fabsf(r) * 2.384185791015625e-7f + 1e-30f; }

// (h, l) = (ah + al) - (bh + bl) as an FP32 pair: Knuth's TwoSum of the high
// parts, the low parts and the rounding error added, then TwoSum again, so
// h + l is the difference to about 2^-47 of the operands' magnitudes.
__device__ __forceinline__ void df_sub(float ah, float al, float bh, float bl, float &h, float &l)
{
    const float s = ah - bh;
    const float bb = s - ah;
    const float e = (ah - (s - bb)) + (-bh - bb);
    const float t = e + (al - bl);
    h = s + t;
    const float b2 = h - s;
    l = (s - (h - b2)) + (t - b2);
}

__device__ __forceinline__ double exact_cross(double2 a, double2 b, double px, double py)
{
    double ax = a.x - px, ay = a.y - py, bx = b.x - px, by = b.y - py;
    return ax * by - ay * bx;
}

__device__ __forceinline__ void write_out(const OutDst &o, uint32_t q, double om, int st, bool atomic_bits)
{
    if (o.w) o.w[q] = om;
    if (o.st) o.st[q] = (uint8_t)st;
    if (o.bits && atomic_bits) {
        if (st != 0) atomicOr(&o.bits[q >> 5], 1u << (q & 31));
        if (st == 2 && o.nbound) atomicAdd(o.nbound, 1ull);
    }
}

// The final step of one query in the mixed path (Sec. 4.1's decision, the
// finalize kernel):
// omega = a2 / 2 - theta / 2 pi from the doubled crossings and line halves
// a2 and the sum of gap angles theta.  Returns the state (0 outside, 1
// inside, 2 boundary) and omega in *om (when want_w), or -1 when the query
// must be recomputed in FP64: a kernel flagged it, or omega lies within the
// classification band of 1/2.  The classification runs in FP32 (its error,
// ~1e-7 of the terms, is far inside the band); omega is formed as an exact
// FP32 pair (product residual, TwoSum, 1/(2 pi) split in two floats) so
// that its FP64 value costs one FP64 addition.
// (float)n for |n| < 2^22 without a conversion instruction (conversions
// share GB300's narrow FP64 unit): 1.5 * 2^23 + n is exact in FP32 with n in
// the low bits of its fraction.
__device__ __forceinline__ float small_i2f(int n) { return __int_as_float(0x4B400000 + n) - 12582912.0f; }

__device__ __forceinline__ int settle(int32_t a2, float th, uint32_t f, bool want_w, double &om)
{
    om = 0.0;
    if (f & QF_ESCALATE) return -1;
    if (f & QF_BOUNDARY) {
        om = __longlong_as_double(0x7ff8000000000000ULL);
        return 2;
    }
    const float fa2 = (a2 > -4194304 && a2 < 4194304) ? small_i2f(a2) : (float)a2;
    const float om32 = fmaf(-th, kInv2PiF, 0.5f * fa2);
    const float band = kOmegaBandF + 1e-6f * (fabsf(0.5f * fa2) + fabsf(th) * kInv2PiF);
    if (fabsf(om32 - 0.5f) < band) return -1;
    if (want_w) {
        const float h = 0.5f * fa2;
        const float p = th * kInv2PiF;
        const float pe = fmaf(th, kInv2PiF, -p);
        const float s = h - p;
        const float bb = s - h;
        const float e = (h - (s - bb)) + (-p - bb);
        const float lo = (e - pe) - th * kInv2PiLoF;
        om = f32_to_f64_exact(s) + f32_to_f64_exact(lo);
    }
    return om32 >= 0.5f ? 1 : 0;
}

// Asynchronous global -> shared copies (cp.async): 16 bytes, both addresses
// 16-byte aligned; commit closes a group, wait_all waits for the thread's
// copies.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The per-query accumulator of the mixed path: the doubled crossings and
// line halves times 4 with the QF_* flags in the two low bits, so that one
// word is written per query and the near walks' atomic adds (multiples of
// 4) and ORs (the low bits) never disturb each other.
static_assert((QF_BOUNDARY | QF_ESCALATE) == 3u, "the flags fill the two low bits");
__device__ __forceinline__ int32_t pack_acc(int acc2, uint32_t flags) { return acc2 * 4 + (int32_t)flags; }
__device__ __forceinline__ int unpack_acc(int32_t v) { return (v - (v & 3)) / 4; }

// ------------------------------------------------------------------ sweep
struct SweepArgs {
    const DomDev *doms;
    const int4 *units;
    int n_units;
    const int *perm;            // position -> query index (spatially bucketed), or null
    PointSrc src;
    int32_t *acc2;              // packed per query: (2 crossings + line halves) * 4 | QF_* flags
    float *theta;
    Item *near_items;
    long long cap_near;
    unsigned long long *counters;
    unsigned long long *work;   // WK_* tallies of the counting build, or null
    int unit_ctr;               // the counter (CNT_*) the kernel's CTAs draw units from
};

// Exact recomputation of one record's crossings and gap angle in FP64, for a
// (query, record) whose FP32 error bands could not settle a sign.  Out of
// line so that the FP64 instructions never issue on the fast path.
__device__ __noinline__ void sweep_record_exact(int ridx, uint32_t fl, bool near,
                                                const DomDev *__restrict__ Dp, double pxp,
                                                double pyp, int &c, float &dth)
{
    const double2 a = Dp->rec_a64[ridx], b = Dp->rec_b64[ridx], n = Dp->rec_n64[ridx];
    const bool sa = a.y > pyp, sb = b.y > pyp, sn = n.y > pyp;
    c = 0;
    dth = 0.f;
    if (!near && sa != sb) {
        const bool pos = exact_cross(a, b, pxp, pyp) > 0;
        c = (!sa && sb && pos) ? 1 : ((sa && !sb && !pos) ? -1 : 0);
    }
    if (fl & RF_GAP) {
        const double ux = b.x - pxp, uy = b.y - pyp, vx = n.x - pxp, vy = n.y - pyp;
        const double d = ux * vy - uy * vx;
        if (sb != sn) {
            const bool pos = d > 0;
            c += (!sb && sn && pos) ? 1 : ((sb && !sn && !pos) ? -1 : 0);
        }
        dth = (float)atan2(d, ux * vx + uy * vy);
    }
}

// The exact FP64 window test and line-term sign of instance j, out of line:
// the sweep's FP32 pre-tests settle almost every query, and inlined these
// would only crowd the instruction cache.
__device__ __noinline__ bool inst_sees_exact(const DomDev *__restrict__ Dp, int j, double x, double y)
{
    const InstDev &in = Dp->inst[j];
    return inst_sees(*Dp, in, Dp->loops[in.loop], x, y);
}

__device__ __noinline__ int line_side_exact(const DomDev *__restrict__ Dp, int j, double x, double y)
{
    const InstDev &in = Dp->inst[j];
    return line_side(*Dp, in, Dp->loops[in.loop], x, y);
}

// Signed crossings of the +x ray from p by a node's whole polyline when the
// polyline lies right of p: [end above p] - [start above p], with the exact
// FP64 comparison for a sign inside its band.  Out of line.
__device__ __noinline__ int node_span_exact(const DomDev *__restrict__ Dp, int R0, int R1, double pyp)
{
    const bool s0 = Dp->rec_a64[R0].y > pyp, s1 = Dp->rec_n64[R1 - 1].y > pyp;
    return (s1 ? 1 : 0) - (s0 ? 1 : 0);
}

__device__ __noinline__ float atan2_wide(float y, float x) { return atan2f(y, x); }

// Signed angle atan2(y, x) of a gap seen from the query.  For |y| <= x/4 the
// odd Gregory series of atan(t), t = y/x, truncated after t^11 (remainder
// below t^13/13 < 5e-9 |t|); otherwise the library atan2f, out of line.
__device__ __forceinline__ float gap_angle(float y, float x)
{
    if (fabsf(y) <= 0.25f * x) {
        const float t = __fdividef(y, x);
        const float t2 = t * t;
        float p = -1.0f / 11.0f;
        p = fmaf(p, t2, 1.0f / 9.0f);
        p = fmaf(p, t2, -1.0f / 7.0f);
        p = fmaf(p, t2, 1.0f / 5.0f);
        p = fmaf(p, t2, -1.0f / 3.0f);
        p = fmaf(p, t2, 1.0f);
        return t * p;
    }
    return atan2_wide(y, x);
}

// A query inside a record's circle: is it inside the ellipse of Eq. 5 and
// inside the box of the segment's control points (the root step's "near")?
//   ellipse: the circle's inflated focal sum 2R, |p - a| + |p - b| > 2R is
//     far; 4T covers the FP32 coordinate errors and R's two 2^-20 inflations
//     the relative rounding of the distances, their sum and the square, so
//     "far" here implies far in Alg. 1's own test;
//   box: in the chord's frame (t along b - a, d across it, widened by eps);
//     outside it the query is more than eps from the curve, which lies in
//     the control points' hull and so is seen under its chord's angle.  The
//     band covers the FP32 errors of a - p = (ux, uy) (T per coordinate), of
//     b - a and of the products.
// Inlined (measured faster than a call on the batched workload, though only
// a few (query, record) pairs get here).  Returns 0 (far by the ellipse), 1
// (far by the box) or 2 (near).
__device__ __forceinline__ int root_near(const float4 R0, float R2c, float ux, float uy, float wx, float wy, float T,
                                      const float4 *obb)
{
    const float da = sqrtf(fmaf(ux, ux, uy * uy)), db = sqrtf(fmaf(wx, wx, wy * wy));
    const float s = (da + db) - 4.f * T;
    if ((s > 0.f) & (s * s > 4.f * R2c)) return 0;
    const float4 O = __ldg(obb);
    const float ex = R0.z - R0.x, ey = R0.w - R0.y;
    const float tq = -fmaf(ux, ex, uy * ey), dq = fmaf(uy, ex, -ux * ey);
    const float bd = 4.f * T * (fabsf(ex) + fabsf(ey) + fabsf(ux) + fabsf(uy));
    return ((tq < O.x - bd) | (tq > O.y + bd) | (dq < O.z - bd) | (dq > O.w + bd)) ? 1 : 2;
}

// One record against one query in FP32: the root step of Alg. 1 (a circle
// that contains the ellipse of Eq. 4 and the eps discs, then, inside it, the
// ellipse itself, then, inside that, the control points' box; `ell` and
// `box` say which of the later tests ran), the chord's
// crossing of the +x ray from p, the gap chord's crossing and the gap angle.
// `slow` is set when an error band cannot settle a sign; the caller then
// redoes the record with sweep_record_exact.
__device__ __forceinline__ void sweep_record(const float4 R0, const float4 R1, const float4 R2,
                                             const float4 R3, float fx, float fy, float fxl,
                                             float fyl, float T, const float4 *obb, int &c, float &dth,
                                             bool &near, bool &slow, bool &ell, bool &box)
{
    const float uy = R0.y - fy, wy = R0.w - fy;
    const bool sa = uy > 0.f, sb = wy > 0.f;
    slow = (fabsf(uy) <= T) | (fabsf(wy) <= T);
    const uint32_t fl = __float_as_uint(R1.w);
    const float wx = R0.z - fx;
    near = false;
    ell = false;
    box = false;
    c = 0;
    dth = 0.f;
    const float ux = R0.x - fx;
    if (!(fl & RF_CHORD)) {
        const float dcx = R1.x - fx, dcy = R1.y - fy;
        near = fmaf(dcx, dcx, dcy * dcy) <= R1.z;
        if (near) {
            const int rn = root_near(R0, R1.z, ux, uy, wx, wy, T, obb);
            near = rn == 2;
            ell = true;
            box = rn != 0;
        }
    }
    if (!near && sa != sb) {
        const float D = fmaf(ux, wy, -uy * wx);
        const float TD = T * (fabsf(ux) + fabsf(uy) + fabsf(wx) + fabsf(wy)) +
                         kTwoM22 * (fabsf(ux * wy) + fabsf(uy * wx));
        slow |= fabsf(D) <= TD;
        const bool pos = D > 0.f;
        c = (!sa && sb && pos) ? 1 : ((sa && !sb && !pos) ? -1 : 0);
    }
    if (fl & RF_GAP) {
        const float gx = R2.x, gy = R2.y;
        const float ny = R2.w - fy;
        const bool sn = ny > 0.f;
        slow |= fabsf(ny) <= T;
        // b - p and n - p from the hi/lo split of the points: each accurate to
        // ~2^-23 relative, so no cancellation when the query is near b or n
        const float bx = wx + (R3.x - fxl), by = wy + (R3.y - fyl);
        const float vx = (R2.z - fx) + (R3.z - fxl), vy = ny + (R3.w - fyl);
        // cross(b-p, n-p) = cross(b-p, g): use the short side for accuracy
        const bool use_g = fmaf(gx, gx, gy * gy) <= fmaf(vx, vx, vy * vy);
        const float ex = use_g ? gx : vx, ey = use_g ? gy : vy;
        const float Dg = fmaf(bx, ey, -by * ex);
        if (sb != sn) {
            slow |= fabsf(Dg) <= 4.0f * kTwoM22 * (fabsf(bx) + fabsf(by)) * (fabsf(ex) + fabsf(ey));
            const bool pos = Dg > 0.f;
            c += (!sb && sn && pos) ? 1 : ((sb && !sn && !pos) ? -1 : 0);
        }
        dth = gap_angle(Dg, fmaf(bx, vx, by * vy));
    }
}

// One record against a query that is outside every circle of its cluster
// (so no near pair can arise): chord crossing, gap crossing and gap angle.
__device__ __forceinline__ void sweep_record_far(const float4 R0, const float4 R1, const float4 R2,
                                                 const float4 R3, float fx, float fy, float fxl,
                                                 float fyl, float T, int &c, float &dth, bool &slow)
{
    const float uy = R0.y - fy, wy = R0.w - fy;
    const bool sa = uy > 0.f, sb = wy > 0.f;
    slow = (fabsf(uy) <= T) | (fabsf(wy) <= T);
    const uint32_t fl = __float_as_uint(R1.w);
    const float wx = R0.z - fx;
    c = 0;
    dth = 0.f;
    if (sa != sb) {
        const float ux = R0.x - fx;
        const float D = fmaf(ux, wy, -uy * wx);
        const float TD = T * (fabsf(ux) + fabsf(uy) + fabsf(wx) + fabsf(wy)) +
                         kTwoM22 * (fabsf(ux * wy) + fabsf(uy * wx));
        slow |= fabsf(D) <= TD;
        const bool pos = D > 0.f;
        c = (!sa && sb && pos) ? 1 : ((sa && !sb && !pos) ? -1 : 0);
    }
    if (fl & RF_GAP) {
        const float gx = R2.x, gy = R2.y;
        const float ny = R2.w - fy;
        const bool sn = ny > 0.f;
        slow |= fabsf(ny) <= T;
        const float bx = wx + (R3.x - fxl), by = wy + (R3.y - fyl);
        const float vx = (R2.z - fx) + (R3.z - fxl), vy = ny + (R3.w - fyl);
        const bool use_g = fmaf(gx, gx, gy * gy) <= fmaf(vx, vx, vy * vy);
        const float ex = use_g ? gx : vx, ey = use_g ? gy : vy;
        const float Dg = fmaf(bx, ey, -by * ex);
        if (sb != sn) {
            slow |= fabsf(Dg) <= 4.0f * kTwoM22 * (fabsf(bx) + fabsf(by)) * (fabsf(ex) + fabsf(ey));
            const bool pos = Dg > 0.f;
            c += (!sb && sn && pos) ? 1 : ((sb && !sn && !pos) ? -1 : 0);
        }
        dth = gap_angle(Dg, fmaf(bx, vx, by * vy));
    }
}

// Compensated addition of a float into a (hi, lo) pair (Knuth's TwoSum).
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float v)
{
    const float s = hi + v;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (v - bb);
    hi = s;
    lo += err;
}

// Crossings only (chord and gap chord) of one record, for a query known to be
// outside every circle of the record's cluster.
__device__ __forceinline__ void sweep_record_cross(const float4 R0, const float4 R1, const float4 R2,
                                                   float fx, float fy, float T, int &c, bool &slow)
{
    const float uy = R0.y - fy, wy = R0.w - fy;
    const bool sa = uy > 0.f, sb = wy > 0.f;
    slow = (fabsf(uy) <= T) | (fabsf(wy) <= T);
    const uint32_t fl = __float_as_uint(R1.w);
    const float wx = R0.z - fx;
    c = 0;
    if (sa != sb) {
        const float ux = R0.x - fx;
        const float D = fmaf(ux, wy, -uy * wx);
        const float TD = T * (fabsf(ux) + fabsf(uy) + fabsf(wx) + fabsf(wy)) +
                         kTwoM22 * (fabsf(ux * wy) + fabsf(uy * wx));
        slow |= fabsf(D) <= TD;
        const bool pos = D > 0.f;
        c = (!sa && sb && pos) ? 1 : ((sa && !sb && !pos) ? -1 : 0);
    }
    if (fl & RF_GAP) {
        const float ny = R2.w - fy;
        const bool sn = ny > 0.f;
        slow |= fabsf(ny) <= T;
        if (sb != sn) {
            const float vx = R2.z - fx;
            const float Dg = fmaf(wx, ny, -wy * vx);
            const float TDg = T * (fabsf(wx) + fabsf(wy) + fabsf(vx) + fabsf(ny)) +
                              kTwoM22 * (fabsf(wx * ny) + fabsf(wy * vx));
            slow |= fabsf(Dg) <= TDg;
            const bool pos = Dg > 0.f;
            c += (!sb && sn && pos) ? 1 : ((sb && !sn && !pos) ? -1 : 0);
        }
    }
}

// Sum of a node's gap angles at each of the QPT queries of a thread from the
// node's Laurent expansion, Im sum_{t<Kq} c_t w^(t+1) with w = r_c / (z_c - p),
// by Horner's rule; slot k only when use[k] (uniform across the warp).  One
// coefficient load per term serves every slot: the loop runs the warp's
// largest K in blocks of 4 terms (every K is a multiple of 4), and a slot
// takes a block only when it lies below its own length kq[k] (the series
// length its query's distance needs; starting from 0, its sum is the
// Horner sum of its own terms), so a query's sum does not depend on which
// queries share its warp.
template <int QPT>
__device__ __forceinline__ void node_gap_sums(const float4 *__restrict__ N, const float *fx, const float *fy,
                                              const float *fxl, const float *fyl, const bool *use,
                                              const int *kq, int K, float *out)
{
    const float4 z = __ldg(N + 2);
    const float rc = __ldg(&N[3].x);
    float wr[QPT], wi[QPT], sr[QPT], si[QPT];
    const float4 *cf = N + kCluCoef;              // two complex coefficients per float4
#pragma unroll
    for (int k = 0; k < QPT; k++) {
        const float dx = (z.x - fx[k]) + (z.z - fxl[k]);
        const float dy = (z.y - fy[k]) + (z.w - fyl[k]);
        const float inv = __fdividef(rc, fmaf(dx, dx, dy * dy));
        wr[k] = dx * inv;
        wi[k] = -dy * inv;
        sr[k] = 0.f;
        si[k] = 0.f;
    }
    for (int b = K / 4 - 1; b >= 0; b--) {
        const float4 c01 = __ldg(cf + 2 * b), c23 = __ldg(cf + 2 * b + 1);
        const float cr[4] = {c23.z, c23.x, c01.z, c01.x}, ci[4] = {c23.w, c23.y, c01.w, c01.y};
#pragma unroll
        for (int k = 0; k < QPT; k++) {
            if (!use[k] || 4 * b >= kq[k]) continue;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float tr = fmaf(sr[k], wr[k], fmaf(-si[k], wi[k], cr[j]));
                const float ti = fmaf(sr[k], wi[k], fmaf(si[k], wr[k], ci[j]));
                sr[k] = tr;
                si[k] = ti;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < QPT; k++) out[k] = fmaf(sr[k], wi[k], si[k] * wr[k]);
}


// Warp-synchronous walk of the record trees of every loop an instance
// covers.  Each query slot carries a status per tree level: 1 = full (gap
// angles and near pairs still needed below), 2 = crossings only, 0 = done.
// At a node, a full slot outside the near box whose distance accepts the
// node's expansion takes the node's gap angles from it and keeps only the
// crossings (if its +x ray can meet the node); a slot inside the box, or too
// close, stays full.  Leaves sweep their records for the slots that still
// need them.  The stack lives in the lanes' registers (entry i in lane i).
//
// The CNT build adds per-lane tallies of the work done (WK_*), summed per
// warp into A.work when the warp runs out of units; its decisions and
// arithmetic are those of the plain build.  MINB CTAs per SM set the
// register budget (64 registers at 4, 80 at 3, 128 at 2): fewer resident
// warps, fewer spills.
template <int QPT, bool CNT, int MINB>
__global__ void __launch_bounds__(kSweepThreads, MINB) k_sweep_tree(const SweepArgs A)
{
    constexpr int SB = 2 * QPT;                     // status bits per level
    constexpr uint64_t SMASK = (1ull << SB) - 1ull;
    static_assert(SB * kTreeMaxLevels <= 64, "level flags must fit 64 bits");
    __shared__ double2 s_p[QPT][kSweepThreads];       // reduced queries (FP64), read on the slow paths
    __shared__ float4 s_ph[QPT][kSweepThreads];       // p - o as FP32 hi/lo pairs (x hi, x lo, y hi, y lo)
    __shared__ float2 s_pr[QPT][kSweepThreads];       // reduced query in FP32 (within 2^-23)
    __shared__ float s_wb[kSweepThreads / 32][8];     // per warp: query box, |max|, family normal
    // the next unit of a warp's claimed run, staged while the current one
    // runs: its unit record, its queries' indices and (by cp.async) points
    __shared__ double2 s_nq[QPT][kSweepThreads];
    __shared__ int s_nid[QPT][kSweepThreads];
    __shared__ int4 s_nu[kSweepThreads / 32];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t wk[WK_SWEEP_N];
#pragma unroll
    for (int i = 0; i < WK_SWEEP_N; i++) wk[i] = 0u;

    // every warp works on its own units (32*QPT queries): no block barrier.
    // A warp claims `batch` consecutive units per atomic on the shared
    // counter, more when there are many units per warp (the units come in
    // decreasing cost order, so neighbours cost about the same)
    const int n_warps = (int)(gridDim.x * (kSweepThreads / 32));
    const int batch = max(1, min(8, A.n_units / (64 * n_warps)));
    int u_next = 0, u_end = 0;          // the warp's claimed units (warp-uniform)
    bool staged = false;                // the unit about to start is staged in shared memory (warp-uniform)
    for (;;) {
        if (u_next >= u_end) {
            unsigned long long uu = 0;
            if (lane == 0) uu = atomicAdd(&A.counters[CNT_UNIT], (unsigned long long)batch);
            u_next = (int)__shfl_sync(0xffffffffu, uu, 0);
            u_end = u_next + batch;
            staged = false;
        }
        const int u = u_next++;
        if (u >= A.n_units) {
            if constexpr (CNT) {
#pragma unroll
                for (int i = 0; i < WK_SWEEP_N; i++) {
                    const unsigned s = __reduce_add_sync(0xffffffffu, wk[i]);
                    if (lane == 0 && s) atomicAdd(&A.work[i], (unsigned long long)s);
                }
            }
            return;
        }
        if (staged) {
            cp_async_wait_all();
            __syncwarp();
        }
        const int4 U = staged ? s_nu[warp] : __ldg(&A.units[u]);
        const DomDev *__restrict__ Dp = A.doms + U.x;
        const double Pu = Dp->Pu, Pv = Dp->Pv;
        const float M = Dp->M, Mq = Dp->Mq;
        const int n_inst = Dp->n_inst;
        const float4 *__restrict__ rec = Dp->rec;
        const float4 *__restrict__ nodes = Dp->nodes;
        // the next unit of the run (bucketed queries): its record and query
        // indices are loaded now, their latency hidden by this unit's start,
        // and staged below once this unit's own staged data has been read
        const bool stage_next = A.perm && u_next < u_end && u_next < A.n_units;
        int4 Un = make_int4(0, 0, 0, 0);
        int qn[QPT];
#pragma unroll
        for (int k = 0; k < QPT; k++) qn[k] = -1;
        if (stage_next) {
            Un = __ldg(&A.units[u_next]);
#pragma unroll
            for (int k = 0; k < QPT; k++)
                if (lane * QPT + k < Un.z) qn[k] = __ldg(&A.perm[(uint32_t)(Un.w + lane * QPT + k)]);
        }

        float fx[QPT], fy[QPT], fxl[QPT], fyl[QPT], T[QPT], th[QPT], thl[QPT];
        int acc[QPT];
        uint32_t fl[QPT], qid[QPT];
        bool valid[QPT], inc[QPT];
#pragma unroll
        for (int k = 0; k < QPT; k++) {
            const int ql = lane * QPT + k;          // the warp owns the unit's 32*QPT positions
            valid[k] = ql < U.z;
            qid[k] = 0;
            double x = 0.0, y = 0.0;
            if (valid[k]) {
                const uint32_t pos = (uint32_t)(U.y + ql);
                if (A.perm) {
                    // bucketed: the unit's positions start at U.w in the
                    // bucketed order (tree domains only)
                    qid[k] = staged ? (uint32_t)s_nid[k][tid] : (uint32_t)__ldg(&A.perm[(uint32_t)(U.w + ql)]);
                } else if (A.src.tiles_x) {
                    // grid in tiles of 64 cells (w x 64/w), row-major:
                    // position -> cell
                    const uint32_t t = pos >> 6, j = pos & 63u, lw = (uint32_t)A.src.tile_lw;
                    const uint32_t ci = (t % (uint32_t)A.src.tiles_x << lw) + (j & ((1u << lw) - 1u));
                    const uint32_t cj = (t / (uint32_t)A.src.tiles_x << (6u - lw)) + (j >> lw);
                    valid[k] = ci < (uint32_t)A.src.nu && cj < (uint32_t)A.src.nv;
                    qid[k] = valid[k] ? cj * (uint32_t)A.src.nu + ci : 0u;
                } else {
                    qid[k] = pos;
                }
                if (valid[k]) {
                    if (staged) {
                        const double2 v = s_nq[k][tid];
                        x = v.x;
                        y = v.y;
                    } else {
                        get_point(A.src, qid[k], x, y);
                    }
                }
            }
            x = reduce_period(x, Pu);
            y = reduce_period(y, Pv);
            s_p[k][tid] = make_double2(x, y);
            // the query in FP32 without FP64 instructions (GB300's FP64
            // unit is narrow and every query passes here): p as a truncated
            // FP32 value (the window pre-tests' point) plus its remainder,
            // then p - o as an FP32 pair by TwoSum against the origin's pair;
            // each instance then subtracts its lattice shift the same way.
            // Within 2^-46 (|p - o| + |o|) of p - o.
            const float xt = f64_to_f32_trunc(x), yt = f64_to_f32_trunc(y);
            float hx, lx, hy, ly;
            df_sub(xt, f64_rem_f32(x), Dp->oxh, Dp->oxl, hx, lx);
            df_sub(yt, f64_rem_f32(y), Dp->oyh, Dp->oyl, hy, ly);
            s_ph[k][tid] = make_float4(hx, lx, hy, ly);
            s_pr[k][tid] = make_float2(xt, yt);
            acc[k] = 0;
            th[k] = 0.f;
            thl[k] = 0.f;
            fl[k] = 0u;
        }
        // stage the next unit: each lane writes its own slots (it has just
        // read this unit's from them), lane 0 the unit record
        if (stage_next) {
            if (lane == 0) s_nu[warp] = Un;
#pragma unroll
            for (int k = 0; k < QPT; k++)
                if (qn[k] >= 0) {
                    s_nid[k][tid] = qn[k];
                    cp_async16(&s_nq[k][tid], A.src.pts + 2 * (size_t)qn[k]);
                }
            cp_async_commit();
        }
        staged = stage_next;

        // warp box of the reduced queries (FP32, rounded outward): instances
        // whose window misses it are skipped by the whole warp, 32 tested
        // per round (a domain with one instance needs no test).  The box
        // waits in shared memory, not in registers, during the tree walks.
        if (n_inst > 1) {
            float wb0 = INFINITY, wb1 = -INFINITY, wb2 = INFINITY, wb3 = -INFINITY;
#pragma unroll
            for (int k = 0; k < QPT; k++)
                if (valid[k]) {
                    const float2 r = s_pr[k][tid];
                    wb0 = fminf(wb0, pt_lo(r.x));
                    wb1 = fmaxf(wb1, pt_hi(r.x));
                    wb2 = fminf(wb2, pt_lo(r.y));
                    wb3 = fmaxf(wb3, pt_hi(r.y));
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                wb0 = fminf(wb0, __shfl_xor_sync(0xffffffffu, wb0, o));
                wb1 = fmaxf(wb1, __shfl_xor_sync(0xffffffffu, wb1, o));
                wb2 = fminf(wb2, __shfl_xor_sync(0xffffffffu, wb2, o));
                wb3 = fmaxf(wb3, __shfl_xor_sync(0xffffffffu, wb3, o));
            }
            if (lane == 0) {
                s_wb[warp][0] = wb0;
                s_wb[warp][1] = wb1;
                s_wb[warp][2] = wb2;
                s_wb[warp][3] = wb3;
                s_wb[warp][4] = fmaxf(fmaxf(fabsf(wb0), fabsf(wb1)), fmaxf(fabsf(wb2), fabsf(wb3)));
            }
        }
        if (lane == 0) {
            s_wb[warp][5] = Dp->nxf;
            s_wb[warp][6] = Dp->nyf;
        }
        __syncwarp();
        for (int jb = 0; jb < n_inst; jb += 32) {
            const int jl = jb + lane;
            unsigned vis = 1u;
            if (n_inst > 1) {
                const float *wb = s_wb[warp];
                vis = __ballot_sync(0xffffffffu, jl < n_inst && cull_sees(Dp->cull[jl], wb[5], wb[6], wb[0], wb[1],
                                                                          wb[2], wb[3], wb[4]));
            }
            while (vis) {
                const int j = jb + __ffs(vis) - 1;
                vis &= vis - 1;
                const InstDev &in = Dp->inst[j];
                const int itype = in.type;
                const InstF32 F = Dp->instf[j];
                bool any = false;
#pragma unroll
                for (int k = 0; k < QPT; k++) {
                    inc[k] = valid[k] && !(fl[k] & (QF_BOUNDARY | QF_ESCALATE));
                    const float2 r = s_pr[k][tid];
                    if (inc[k] && itype != IT_ALL) {
                        // FP32 pre-test of the window: outside the widened
                        // window -> not seen, inside the shrunk one -> seen,
                        // in between -> the exact FP64 test
                        const float bx0 = pt_lo(r.x), bx1 = pt_hi(r.x), by0 = pt_lo(r.y), by1 = pt_hi(r.y);
                        const float wm = fmaxf(fmaxf(fabsf(bx0), fabsf(bx1)), fmaxf(fabsf(by0), fabsf(by1)));
                        const float *wb = s_wb[warp];
                        if (!cull_sees(Dp->cull[j], wb[5], wb[6], bx0, bx1, by0, by1, wm)) {
                            inc[k] = false;
                        } else if (!inner_sees(Dp->cull[j], F, wb[5], wb[6], bx0, bx1, by0, by1, wm)) {
                            const double2 p = s_p[k][tid];
                            inc[k] = inst_sees_exact(Dp, j, p.x, p.y);
                            if constexpr (CNT) wk[WK_EXACT]++;
                        }
                    }
                    if (itype == IT_LINE) {
                        if (inc[k]) {
                            int sd = line_side_f32(F, r.x, r.y);
                            if (sd == 0) {
                                const double2 p = s_p[k][tid];
                                sd = line_side_exact(Dp, j, p.x, p.y);
                                if constexpr (CNT) wk[WK_EXACT]++;
                            }
                            if (sd == 0) fl[k] |= QF_BOUNDARY;
                            acc[k] += sd;
                        }
                        inc[k] = false;
                        continue;
                    }
                    // p' - o = (p - o) - T in FP32 double-float arithmetic
                    const float4 ph = s_ph[k][tid];
                    df_sub(ph.x, ph.y, F.txh, F.txl, fx[k], fxl[k]);
                    df_sub(ph.z, ph.w, F.tyh, F.tyl, fy[k], fyl[k]);
                    const float mag = fmaxf(fabsf(fx[k]), fabsf(fy[k]));
                    if (inc[k] && !(mag <= Mq)) {
                        fl[k] |= QF_ESCALATE;
                        inc[k] = false;
                    }
                    T[k] = kTwoM22 * (M + mag);
                    any |= inc[k];
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                // a planar domain's loops hang below one root; otherwise each
                // loop the instance covers is walked from its own root
                const bool one_root = in.type == IT_ALL && Dp->all_root >= 0;
                const int l0 = (in.type == IT_ALL) ? 0 : in.loop;
                const int l1 = one_root ? 1 : (in.type == IT_ALL) ? Dp->n_loops : in.loop + 1;
                for (int l = l0; l < l1; l++) {
                    const int root = one_root ? Dp->all_root : Dp->loops[l].root;
                    if (root < 0) continue;
                    uint64_t lf = 0;
#pragma unroll
                    for (int k = 0; k < QPT; k++)
                        if (inc[k]) lf |= 1ull << (2 * k);
                    int st_cur = root, st_end = root + 1, st_lvl = 0;    // stack entry `lane`
                    int sp = 0;
                    while (sp >= 0) {
                        const int cur = __shfl_sync(0xffffffffu, st_cur, sp);
                        const int end = __shfl_sync(0xffffffffu, st_end, sp);
                        const int lvl = __shfl_sync(0xffffffffu, st_lvl, sp);
                        if (lane == sp) st_cur = cur + 1;
                        if (cur + 1 >= end) sp--;
                        const uint32_t f = (uint32_t)((lf >> (lvl * SB)) & SMASK);
                        if (!__any_sync(0xffffffffu, f != 0u)) continue;
                        if constexpr (CNT) wk[WK_WARP_NODE] += lane == 0 ? 1u : 0u;
                        const float4 *__restrict__ N = nodes + (size_t)kCluF4 * cur;
                        const float4 nb = __ldg(N), yx = __ldg(N + 1), meta = __ldg(N + 3), sp6 = __ldg(N + 6);
                        const int nflags = __float_as_int(meta.y);
                        const bool gaps = nflags & 1, leaf = (nflags & 2) != 0;
                        uint32_t cf = 0u, nearb = 0u, mpb = 0u;
                        int kneed = 0, kqs[QPT];
                        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (gaps) z = __ldg(N + 2);
#pragma unroll
                        for (int k = 0; k < QPT; k++) {
                            kqs[k] = 0;
                            const uint32_t sk = (f >> (2 * k)) & 3u;
                            if (!sk) continue;
                            if constexpr (CNT) wk[WK_NODE]++;
                            const bool outside = (fx[k] < nb.x - T[k]) | (fx[k] > nb.y + T[k]) |
                                                 (fy[k] < nb.z - T[k]) | (fy[k] > nb.w + T[k]);
                            // does the +x ray from p meet the node's extent at all?
                            const bool meets = !((fy[k] > yx.y + T[k]) | (fy[k] < yx.x - T[k]) | (fx[k] > yx.z + T[k]));
                            bool full = false;     // stays in full mode: descend, crossings at the leaves
                            if (sk == 1u) {
                                if (!outside) {
                                    full = true;
                                    nearb |= 1u << k;
                                } else if (gaps) {
                                    const float dx = (z.x - fx[k]) + (z.z - fxl[k]);
                                    const float dy = (z.y - fy[k]) + (z.w - fyl[k]);
                                    const float d2 = fmaf(dx, dx, dy * dy);
                                    if (d2 >= yx.w) {
                                        const float4 t0 = __ldg(N + 4), t1 = __ldg(N + 5);
                                        const int kq = d2 >= t0.x ? 4 : d2 >= t0.y ? 8 : d2 >= t0.z ? 12 : d2 >= t0.w ? 16
                                                     : d2 >= t1.x ? 20 : d2 >= t1.y ? 24 : d2 >= t1.z ? 28 : kCluTerms;
                                        kneed = max(kneed, kq);
                                        kqs[k] = kq;
                                        mpb |= 1u << k;
                                    } else {
                                        full = true;
                                    }
                                }
                            }
                            uint32_t child = full ? 1u : 0u;
                            if (!full && meets) {
                                if (fx[k] < sp6.x - T[k]) {
                                    // the node lies right of p: its polyline's crossings
                                    // telescope to [end above] - [start above]
                                    const float d0 = sp6.y - fy[k], d1 = sp6.z - fy[k];
                                    int span = (d1 > 0.f ? 1 : 0) - (d0 > 0.f ? 1 : 0);
                                    if ((fabsf(d0) <= T[k]) | (fabsf(d1) <= T[k])) {
                                        const double2 p = s_p[k][tid];
                                        span = node_span_exact(Dp, __float_as_int(sp6.w), __float_as_int(__ldg(&N[7].x)),
                                                               xsub(p.y, in.Ty));
                                        if constexpr (CNT) wk[WK_EXACT]++;
                                    }
                                    if constexpr (CNT) wk[WK_TELE]++;
                                    acc[k] += 2 * span;
                                } else {
                                    child = 2u;    // crossings only, below
                                }
                            }
                            cf |= child << (2 * k);
                        }
                        if (gaps) {
                            const int K = __reduce_max_sync(0xffffffffu, kneed);
                            if (K > 0) {
                                bool use[QPT];
#pragma unroll
                                for (int k = 0; k < QPT; k++) use[k] = __any_sync(0xffffffffu, (mpb >> k) & 1u);
                                float gs[QPT];
                                node_gap_sums<QPT>(N, fx, fy, fxl, fyl, use, kqs, K, gs);
#pragma unroll
                                for (int k = 0; k < QPT; k++)
                                    if (mpb >> k & 1u) {
                                        two_sum_add(th[k], thl[k], gs[k]);
                                        if constexpr (CNT) {
                                            wk[WK_EXPANSION]++;
                                            wk[WK_TERMS] += (uint32_t)kqs[k];
                                        }
                                    }
                            }
                        }
                        if (!leaf) {
                            if (__any_sync(0xffffffffu, cf != 0u)) {
                                sp++;
                                if (lane == sp) {
                                    st_cur = __float_as_int(meta.z);
                                    st_end = __float_as_int(meta.w);
                                    st_lvl = lvl + 1;
                                }
                                const int sh = (lvl + 1) * SB;
                                lf = (lf & ~(SMASK << sh)) | ((uint64_t)cf << sh);
                            }
                            continue;
                        }
                        // leaf: records [first, end) for the slots that still need them
                        bool need_near = nearb != 0u, need_full = false, need_cross = false;
#pragma unroll
                        for (int k = 0; k < QPT; k++) {
                            const uint32_t ck = (cf >> (2 * k)) & 3u;
                            need_full |= ck == 1u;
                            need_cross |= ck == 2u;
                        }
                        const bool wn = __any_sync(0xffffffffu, need_near);
                        const bool we = __any_sync(0xffffffffu, need_full);
                        const bool wc = __any_sync(0xffffffffu, need_cross);
                        if (!we && !wc) continue;
                        const int r0 = __float_as_int(meta.z), r1 = __float_as_int(meta.w);
                        float tcl[QPT];
#pragma unroll
                        for (int k = 0; k < QPT; k++) tcl[k] = 0.f;
                        for (int r = r0; r < r1; r++) {
                            if constexpr (CNT) wk[WK_WARP_REC] += lane == 0 ? 1u : 0u;
                            // the gap data (R2, R3) only where the leaf has gaps
                            // (closed C0 loops have none)
                            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                            const float4 R0 = __ldg(rec + 4 * r), R1 = __ldg(rec + 4 * r + 1),
                                         R2 = gaps ? __ldg(rec + 4 * r + 2) : z4;
                            if (wn) {
                                const float4 R3 = gaps ? __ldg(rec + 4 * r + 3) : z4;
                                bool nr[QPT];
                                bool any_near = false;
#pragma unroll
                                for (int k = 0; k < QPT; k++) {
                                    const uint32_t ck = (cf >> (2 * k)) & 3u;
                                    int cc;
                                    float dth;
                                    bool slow, ell, box;
                                    sweep_record(R0, R1, R2, R3, fx[k], fy[k], fxl[k], fyl[k], T[k], Dp->rec_obb + r, cc,
                                                 dth, nr[k], slow, ell, box);
                                    if (slow && ck) {
                                        const double2 p = s_p[k][tid];
                                        sweep_record_exact(r, __float_as_uint(R1.w), nr[k], Dp, xsub(p.x, in.Tx),
                                                           xsub(p.y, in.Ty), cc, dth);
                                        if constexpr (CNT) wk[WK_EXACT]++;
                                    }
                                    if constexpr (CNT) {
                                        if (ck == 1u && ell) wk[WK_ELLIPSE]++;
                                        if (ck == 1u && box) wk[WK_BOX]++;
                                        if (ck == 1u) wk[WK_REC_NEAR]++;
                                        else if (ck == 2u) wk[WK_REC_CROSS]++;
                                    }
                                    nr[k] = nr[k] && ck == 1u;
                                    if (ck) {
                                        acc[k] += 2 * cc;
                                        if (ck == 1u) tcl[k] += dth;
                                    }
                                    any_near |= nr[k];
                                }
                                if (__any_sync(0xffffffffu, any_near)) {
#pragma unroll
                                    for (int k = 0; k < QPT; k++) {
                                        const unsigned m = __ballot_sync(0xffffffffu, nr[k]);
                                        if (!m) continue;
                                        const int leader = __ffs(m) - 1;
                                        unsigned long long base = 0;
                                        if (lane == leader) base = atomicAdd(&A.counters[CNT_NEAR], (unsigned long long)__popc(m));
                                        base = __shfl_sync(0xffffffffu, base, leader);
                                        if (nr[k]) {
                                            const unsigned long long idx = base + __popc(m & lt_mask);
                                            if (idx < (unsigned long long)A.cap_near) {
                                                Item it;
                                                it.q = qid[k];
                                                it.dom = (uint32_t)U.x;
                                                it.inst = (uint32_t)j;
                                                it.seg = __float_as_uint(R1.w) >> RF_SEG_SHIFT;
                                                it.fx = fx[k];
                                                it.fy = fy[k];
                                                it.fxl = fxl[k];
                                                it.fyl = fyl[k];
                                                A.near_items[idx] = it;
                                            } else {
                                                fl[k] |= QF_ESCALATE;
                                            }
                                        }
                                    }
                                }
                            } else if (we) {
                                const float4 R3 = gaps ? __ldg(rec + 4 * r + 3) : z4;
#pragma unroll
                                for (int k = 0; k < QPT; k++) {
                                    const uint32_t ck = (cf >> (2 * k)) & 3u;
                                    int cc;
                                    float dth;
                                    bool slow;
                                    sweep_record_far(R0, R1, R2, R3, fx[k], fy[k], fxl[k], fyl[k], T[k], cc, dth, slow);
                                    if (slow && ck) {
                                        const double2 p = s_p[k][tid];
                                        sweep_record_exact(r, __float_as_uint(R1.w), false, Dp, xsub(p.x, in.Tx),
                                                           xsub(p.y, in.Ty), cc, dth);
                                        if constexpr (CNT) wk[WK_EXACT]++;
                                    }
                                    if constexpr (CNT) {
                                        if (ck == 1u) wk[WK_REC_FAR]++;
                                        else if (ck == 2u) wk[WK_REC_CROSS]++;
                                    }
                                    if (ck) {
                                        acc[k] += 2 * cc;
                                        if (ck == 1u) tcl[k] += dth;
                                    }
                                }
                            } else {
#pragma unroll
                                for (int k = 0; k < QPT; k++) {
                                    const uint32_t ck = (cf >> (2 * k)) & 3u;
                                    int cc;
                                    bool slow;
                                    sweep_record_cross(R0, R1, R2, fx[k], fy[k], T[k], cc, slow);
                                    if (slow && ck) {
                                        const double2 p = s_p[k][tid];
                                        float dth;
                                        sweep_record_exact(r, __float_as_uint(R1.w), false, Dp, xsub(p.x, in.Tx),
                                                           xsub(p.y, in.Ty), cc, dth);
                                        if constexpr (CNT) wk[WK_EXACT]++;
                                    }
                                    if constexpr (CNT) {
                                        if (ck) wk[WK_REC_CROSS]++;
                                    }
                                    if (ck) acc[k] += 2 * cc;
                                }
                            }
                        }
#pragma unroll
                        for (int k = 0; k < QPT; k++) two_sum_add(th[k], thl[k], tcl[k]);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < QPT; k++) {
            if (!valid[k]) continue;
            A.acc2[qid[k]] = pack_acc(acc[k], fl[k]);
            A.theta[qid[k]] = th[k] + thl[k];
        }
    }
}

// ------------------------------------------------------------------ spatial bucketing
// Queries of each domain are counted into a G x G grid of cells over the
// domain's box and scattered cell by cell, so that a sweep tile covers a
// small area.  Only the order of work changes: every query's arithmetic is
// the same in any order.
struct BinArgs {
    const DomDev *doms;
    long long n;
    PointSrc src;
    unsigned long long *counters;   // CNT_BIN_RUN, CNT_SCAT_RUN: the next run of each kernel
    const int4 *dcell;          // per domain: first cell, G
    int *cell_of;               // per query: its cell in the run's domain << kBinRankBits | its rank there in the run
    int *cnt;                   // per cell: count, then first position
    int *run_off;               // per run and cell of its domain (from the run's .w): the run's offset in the cell
    int *chunk;                 // per chunk of kBinChunk cells: its sum, then its first position
    int *perm;
    int n_cells;
    const int4 *bchunks;        // (domain, first query, count, first run_off entry): runs of one domain's queries
    int n_bchunks;
};

constexpr int kBinChunk = 4096;     // cells per block of the chunked scan
constexpr int kBinThreads = 512;

// v rounded to the nearest integer by FP32 addition (ties to even), for
// -2^22 <= v < 2^22 (other values, NaN included, are clamped into that
// range first; the callers clamp the result again): as a float and an int.
__device__ __forceinline__ float round_near(float v)
{
    const float m = 12582912.0f;    // 1.5 * 2^23
    return fminf(fmaxf(v, -4194304.f), 4194303.f) + m - m;
}
__device__ __forceinline__ int round_near_int(float v)
{
    const float t = fminf(fmaxf(v, -4194304.f), 4194303.f) + 12582912.0f;
    return (__float_as_int(t) & 0x7fffff) - 0x400000;
}

// An FP32 value near the double x from its high word alone (its top 20
// fraction bits): within 2^-20 relative for |x| in FP32's normal range, a
// signed zero below it, some other value above it; for cell choices only,
// which clamp whatever they get.
__device__ __forceinline__ float f64_hi_to_f32(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), sign = hi & 0x80000000u;
    return __uint_as_float((hi & 0x7ff00000u) < 0x38100000u ? sign : sign | ((hi - 0x38000000u) << 3));
}

// Cell of every query, counted per cell.  One CTA per run of one domain's
// queries: the run is counted into the domain's cells in shared memory (the
// shared atomic's old value is the query's rank among the run's queries of
// its cell), then one global atomic per non-empty cell adds the run's count
// and returns the run's offset within the cell.  Each query keeps its cell
// and rank in one word (cell < 2^14, rank < 2^kBinRankBits).
// (3 CTAs of 512 threads per SM: measured faster than 2 with more registers or 4 with spills)
__global__ void __launch_bounds__(kBinThreads, 3) k_bin_count(const BinArgs A)
{
    __shared__ int s_cnt[kBinSmemCells];   // zero at the start of every run (each run clears what it used)
    __shared__ float s_box[8];          // the run's cell frame, from the domain's FP64 fields once per run
    __shared__ int4 s_R, s_dc;
    __shared__ int s_run;
    for (int i = threadIdx.x; i < kBinSmemCells; i += blockDim.x) s_cnt[i] = 0;
    for (;;) {
        // the next run from the shared counter (runs come largest first):
        // CTAs finish together whatever the mix of run sizes
        if (threadIdx.x == 0) {
            const int c = (int)atomicAdd(&A.counters[CNT_BIN_RUN], 1ULL);
            s_run = c;
            if (c < A.n_bchunks) {
                const int4 R = __ldg(&A.bchunks[c]);
                const int4 dc = __ldg(&A.dcell[R.x]);
                s_R = R;
                s_dc = dc;
                // G x G cells over the domain's box (the base tile on periodic
                // axes); FP32 is enough to choose a cell.  One thread converts
                // the FP64 fields (the FP64 unit is narrow on GB300)
                const DomDev *Dp = A.doms + R.x;
                const bool pu = Dp->Pu > 0, pv = Dp->Pv > 0;
                const float wx = pu ? (float)Dp->Pu : 2.f * Dp->M;
                const float wy = pv ? (float)Dp->Pv : 2.f * Dp->M;
                s_box[0] = pu ? 0.f : (float)Dp->ox - Dp->M;
                s_box[1] = pv ? 0.f : (float)Dp->oy - Dp->M;
                s_box[2] = wx;
                s_box[3] = wy;
                // periodic axes: the coordinate's tile offset removed in FP32 (a
                // cell choice needs no exactness)
                s_box[4] = pu ? __fdividef(1.f, wx) : 0.f;
                s_box[5] = pv ? __fdividef(1.f, wy) : 0.f;
                s_box[6] = pu ? 1.f : 0.f;
                s_box[7] = pv ? 1.f : 0.f;
            }
        }
        // (the previous run's flush is also ordered before this run's counts here)
        __syncthreads();
        if (s_run >= A.n_bchunks) return;
        const int4 R = s_R, dc = s_dc;
        const int G = dc.y, G2 = G * G;
        const float x0 = s_box[0], y0 = s_box[1], wx = s_box[2], wy = s_box[3], ipu = s_box[4], ipv = s_box[5];
        const bool pu = s_box[6] != 0.f, pv = s_box[7] != 0.f;
        const float sx = __fdividef((float)G, wx), sy = __fdividef((float)G, wy);
        // four queries per thread at a time: their point loads issue together
        for (int i0 = threadIdx.x; i0 < R.z; i0 += 4 * blockDim.x) {
            double px[4], py[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                px[k] = py[k] = 0.0;
                if (i0 + k * (int)blockDim.x < R.z) get_point(A.src, (uint32_t)(R.y + i0 + k * blockDim.x), px[k], py[k]);
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (i0 + k * (int)blockDim.x >= R.z) continue;
                const uint32_t q = (uint32_t)(R.y + i0 + k * blockDim.x);
                float xf = f64_hi_to_f32(px[k]), yf = f64_hi_to_f32(py[k]);
                // integer parts by FP32 rounding (no conversion instructions,
                // which share GB300's narrow FP64 unit): round_near(v) is the
                // low bits of v + 1.5 * 2^23 for |v| < 2^22; a cell choice needs
                // neither floor nor exactness, only the clamp below
                if (pu) xf -= round_near(xf * ipu - 0.5f) * wx;
                if (pv) yf -= round_near(yf * ipv - 0.5f) * wy;
                int cx = round_near_int((xf - x0) * sx - 0.5f), cy = round_near_int((yf - y0) * sy - 0.5f);
                cx = min(max(cx, 0), G - 1);
                cy = min(max(cy, 0), G - 1);
                const int lc = cy * G + ((cy & 1) ? G - 1 - cx : cx);      // serpentine order
                A.cell_of[q] = lc << kBinRankBits | atomicAdd(&s_cnt[lc], 1);
            }
        }
        __syncthreads();
        // four cells per thread at a time, so that four returning atomics
        // are in flight together
        for (int i0 = threadIdx.x; i0 < G2; i0 += 4 * blockDim.x) {
            int v[4], old[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = i0 + k * blockDim.x;
                v[k] = i < G2 ? s_cnt[i] : 0;
            }
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (v[k]) old[k] = atomicAdd(&A.cnt[dc.x + i0 + k * blockDim.x], v[k]);
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (v[k]) {
                    A.run_off[R.w + i0 + k * blockDim.x] = old[k];
                    s_cnt[i0 + k * blockDim.x] = 0;
                }
        }
        // no barrier: thread 0 rewrites s_run, s_R, s_dc and s_box only after
        // every thread has passed the barrier above, past its last read of them
    }
}

// Exclusive scan of the cell counts in three steps: chunk sums, one CTA
// over the chunk sums, each chunk's local scan plus its offset.
__device__ __forceinline__ int block_excl_scan_1024(int v, int *s_warp, int &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = s_warp[lane];
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        s_warp[lane] = xi - x;                  // exclusive warp offsets
        if (lane == 31) s_warp[32] = xi;        // block total
    }
    __syncthreads();
    const int r = s_warp[w] + incl - v;
    total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) k_bin_chunk_sum(const BinArgs A)
{
    __shared__ int s_warp[33];
    const int c0 = blockIdx.x * kBinChunk;
    int v = 0;
    for (int k = threadIdx.x; k < kBinChunk; k += 1024)
        if (c0 + k < A.n_cells) v += A.cnt[c0 + k];
    int total;
    block_excl_scan_1024(v, s_warp, total);
    if (threadIdx.x == 0) A.chunk[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_bin_chunk_scan(const BinArgs A, int n_chunks)
{
    __shared__ int s_warp[33];
    int run = 0;
    for (int base = 0; base < n_chunks; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < n_chunks ? A.chunk[i] : 0;
        int total;
        const int ex = block_excl_scan_1024(v, s_warp, total);
        if (i < n_chunks) A.chunk[i] = run + ex;
        run += total;
    }
}

__global__ void __launch_bounds__(1024) k_bin_chunk_apply(const BinArgs A)
{
    __shared__ int s_warp[33];
    const int c0 = blockIdx.x * kBinChunk;
    int run = A.chunk[blockIdx.x];
    for (int base = 0; base < kBinChunk; base += 1024) {
        const int c = c0 + base + threadIdx.x;
        const int v = c < A.n_cells ? A.cnt[c] : 0;
        int total;
        const int ex = block_excl_scan_1024(v, s_warp, total);
        if (c < A.n_cells) A.cnt[c] = run + ex;
        run += total;
    }
}

// Every query to its slot, with no atomics: per run of one domain's
// queries, the run's first slot in each cell (the cell's first position plus
// the run's offset in it) in shared memory, and each query at that slot plus
// its rank.  (Entries of cells the run does not reach were never written and
// are never used.)
__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(const BinArgs A)
{
    __shared__ uint32_t s_slot[kBinSmemCells];
    __shared__ int4 s_R, s_dc;
    __shared__ int s_run;
    for (;;) {
        // runs from a shared counter, as in k_bin_count
        if (threadIdx.x == 0) {
            const int c = (int)atomicAdd(&A.counters[CNT_SCAT_RUN], 1ULL);
            s_run = c;
            if (c < A.n_bchunks) {
                const int4 R = __ldg(&A.bchunks[c]);
                s_R = R;
                s_dc = __ldg(&A.dcell[R.x]);
            }
        }
        __syncthreads();
        if (s_run >= A.n_bchunks) return;
        const int4 R = s_R, dc = s_dc;
        const int G2 = dc.y * dc.y;
        for (int i0 = threadIdx.x; i0 < G2; i0 += 4 * blockDim.x) {
            uint32_t a[4], b[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = i0 + k * blockDim.x;
                a[k] = i < G2 ? (uint32_t)__ldg(&A.cnt[dc.x + i]) : 0u;
                b[k] = i < G2 ? (uint32_t)__ldg(&A.run_off[R.w + i]) : 0u;
            }
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (i0 + k * (int)blockDim.x < G2) s_slot[i0 + k * blockDim.x] = a[k] + b[k];
        }
        __syncthreads();
        // four queries per thread at a time: their loads issue together
        for (int i0 = threadIdx.x; i0 < R.z; i0 += 4 * blockDim.x) {
            uint32_t v[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = i0 + k * blockDim.x;
                v[k] = i < R.z ? (uint32_t)__ldg(&A.cell_of[R.y + i]) : 0u;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = i0 + k * blockDim.x;
                if (i < R.z) A.perm[s_slot[v[k] >> kBinRankBits] + (v[k] & (kBinRunMax - 1u))] = R.y + i;
            }
        }
        __syncthreads();
    }
}

template <int QPT>
__global__ void __launch_bounds__(kSweepThreads, (QPT <= 2 ? 3 : 2)) k_sweep(const SweepArgs A)
{
    __shared__ float4 s_rec[4 * kChunk];
    __shared__ double2 s_p[QPT][kSweepThreads];   // reduced queries (FP64), read on the slow paths
    __shared__ int s_unit;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const unsigned lt_mask = (1u << lane) - 1u;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_unit = (int)atomicAdd(&A.counters[A.unit_ctr], 1ULL);
        __syncthreads();
        const int u = s_unit;
        if (u >= A.n_units) return;
        const int4 U = __ldg(&A.units[u]);
        const DomDev *__restrict__ Dp = A.doms + U.x;
        const double Pu = Dp->Pu, Pv = Dp->Pv, ox = Dp->ox, oy = Dp->oy;
        const float M = Dp->M, Mq = Dp->Mq;
        const int n_inst = Dp->n_inst;
        const float4 *__restrict__ rec = Dp->rec;

        float fx[QPT], fy[QPT], fxl[QPT], fyl[QPT], T[QPT], th[QPT], thl[QPT];
        int acc[QPT];
        uint32_t fl[QPT];
        bool valid[QPT], inc[QPT];
#pragma unroll
        for (int k = 0; k < QPT; k++) {
            const int ql = tid + k * kSweepThreads;
            valid[k] = ql < U.z;
            double x = 0.0, y = 0.0;
            if (valid[k]) get_point(A.src, (uint32_t)(U.y + ql), x, y);
            s_p[k][tid] = make_double2(reduce_period(x, Pu), reduce_period(y, Pv));
            acc[k] = 0;
            th[k] = 0.f;
            thl[k] = 0.f;
            fl[k] = 0u;
        }
        for (int j = 0; j < n_inst; j++) {
            const InstDev in = Dp->inst[j];
            const LoopDev &L = Dp->loops[in.loop];
            int any = 0;
#pragma unroll
            for (int k = 0; k < QPT; k++) {
                const double2 p = s_p[k][tid];
                inc[k] = valid[k] && !(fl[k] & (QF_BOUNDARY | QF_ESCALATE)) &&
                         inst_sees(*Dp, in, L, p.x, p.y);
                if (in.type == IT_LINE) {
                    if (inc[k]) {
                        const int s = line_side(*Dp, in, L, p.x, p.y);
                        if (s == 0) fl[k] |= QF_BOUNDARY;
                        acc[k] += s;
                    }
                    inc[k] = false;
                    continue;
                }
                const double dx = xsub(p.x, in.Tx) - ox, dy = xsub(p.y, in.Ty) - oy;
                fx[k] = (float)dx;
                fy[k] = (float)dy;
                fxl[k] = (float)(dx - (double)fx[k]);
                fyl[k] = (float)(dy - (double)fy[k]);
                const float mag = fmaxf(fabsf(fx[k]), fabsf(fy[k]));
                if (inc[k] && !(mag <= Mq)) {
                    fl[k] |= QF_ESCALATE;
                    inc[k] = false;
                }
                T[k] = kTwoM22 * (M + mag);
                any |= inc[k];
            }
            if (!__syncthreads_or(any)) continue;
            if (A.work) {
                // counting: every included query meets every record of the instance
                int n_inc = 0;
#pragma unroll
                for (int k = 0; k < QPT; k++) n_inc += __syncthreads_count(inc[k]);
                if (tid == 0) atomicAdd(&A.work[WK_REC_NEAR], (unsigned long long)n_inc * (unsigned long long)(in.r1 - in.r0));
            }
            for (int r0 = in.r0; r0 < in.r1; r0 += kChunk) {
                const int cnt = min(kChunk, in.r1 - r0);
                // the records of the chunk into shared memory by cp.async
                // (float4 records, 16-byte aligned), shared by every query
                // of the tile
                for (int i = tid; i < 4 * cnt; i += kSweepThreads) cp_async16(&s_rec[i], rec + 4 * r0 + i);
                cp_async_commit();
                cp_async_wait_all();
                __syncthreads();
                float tc[QPT];
#pragma unroll
                for (int k = 0; k < QPT; k++) tc[k] = 0.f;
                for (int r = 0; r < cnt; r++) {
                    const float4 R0 = s_rec[4 * r], R1 = s_rec[4 * r + 1], R2 = s_rec[4 * r + 2],
                                 R3 = s_rec[4 * r + 3];
                    bool nr[QPT];
                    bool any_near = false;
#pragma unroll
                    for (int k = 0; k < QPT; k++) {
                        int c;
                        float dth;
                        bool slow, ell, box;
                        sweep_record(R0, R1, R2, R3, fx[k], fy[k], fxl[k], fyl[k], T[k], Dp->rec_obb + r0 + r, c, dth,
                                     nr[k], slow, ell, box);
                        if (slow && inc[k]) {
                            const double2 p = s_p[k][tid];
                            sweep_record_exact(r0 + r, __float_as_uint(R1.w), nr[k], Dp, xsub(p.x, in.Tx),
                                               xsub(p.y, in.Ty), c, dth);
                        }
                        nr[k] = nr[k] && inc[k];
                        if (inc[k]) {
                            acc[k] += 2 * c;
                            tc[k] += dth;
                        }
                        any_near |= nr[k];
                    }
                    if (__any_sync(0xffffffffu, any_near)) {
#pragma unroll
                        for (int k = 0; k < QPT; k++) {
                            const unsigned m = __ballot_sync(0xffffffffu, nr[k]);
                            if (!m) continue;
                            const int leader = __ffs(m) - 1;
                            unsigned long long base = 0;
                            if (lane == leader) base = atomicAdd(&A.counters[CNT_NEAR], (unsigned long long)__popc(m));
                            base = __shfl_sync(0xffffffffu, base, leader);
                            if (nr[k]) {
                                const unsigned long long idx = (unsigned long long)base + __popc(m & lt_mask);
                                if (idx < (unsigned long long)A.cap_near) {
                                    Item it;
                                    it.q = (uint32_t)(U.y + tid + k * kSweepThreads);
                                    it.dom = (uint32_t)U.x;
                                    it.inst = (uint32_t)j;
                                    it.seg = __float_as_uint(R1.w) >> RF_SEG_SHIFT;
                                    it.fx = fx[k];
                                    it.fy = fy[k];
                                    it.fxl = fxl[k];
                                    it.fyl = fyl[k];
                                    A.near_items[idx] = it;
                                } else {
                                    fl[k] |= QF_ESCALATE;
                                }
                            }
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < QPT; k++) two_sum_add(th[k], thl[k], tc[k]);
                __syncthreads();
            }
        }
#pragma unroll
        for (int k = 0; k < QPT; k++) {
            if (!valid[k]) continue;
            const uint32_t q = (uint32_t)(U.y + tid + k * kSweepThreads);
            A.acc2[q] = pack_acc(acc[k], fl[k]);
            A.theta[q] = th[k] + thl[k];
        }
    }
}

// ------------------------------------------------------------------ near pairs, FP32
// Algorithm 1 in FP32 on query-relative control points, one node per step,
// with every test under an error band: E bounds the absolute error of each
// evaluated point against its FP64 value.  When a band cannot settle a
// decision (eps test, ellipse test, chord sign, depth) the pair becomes an
// FP64 work item and its FP32 walk stops.
struct NearWalk {                      // scalars and control points (registers)
    float qx[kNcp], qy[kNcp];           // q_k = P_k - p; times w_k for a rational segment
    const float *qw;                    // rational segment: its FP32 weights (global, read per evaluation)
    const float *bsub;                  // rational segment: bounds on its eighths (global), see below
    float a, ax, ay, ra, B, E, eps;
    int n, nmax, sp, cnt;
    bool sa, b_tested, rat;
};

struct NearStack {                     // the walk's stack (dynamically indexed: local memory)
    float t[kDepthCap32Max + 2], x[kDepthCap32Max + 2], y[kDepthCap32Max + 2];
    int d[kDepthCap32Max + 2];
};

struct NearArgs {
    const DomDev *doms;
    PointSrc src;
    const Item *items;
    long long cap_near;
    int32_t *acc2;              // packed, see SweepArgs
    SubItem *f64_items;
    long long cap_f64;
    unsigned long long *counters;
    int depth_cap;              // FP32 walk depth cap (kDepthCap32Min..kDepthCap32Max)
    int chunk;                  // pairs a warp draws per atomic (multiple of 32)
    int refill;                 // idle lanes that trigger a refill
    unsigned long long *work;   // WK_NEAR_* tallies of the counting build, or null
};

__device__ __forceinline__ void item_query(const DomDev *Dp, const PointSrc &src, const Item &it,
                                           double &pxp, double &pyp)
{
    double x, y;
    get_point(src, it.q, x, y);
    x = reduce_period(x, Dp->Pu);
    y = reduce_period(y, Dp->Pv);
    const InstDev &in = Dp->inst[it.inst];
    pxp = xsub(x, in.Tx);
    pyp = xsub(y, in.Ty);
}

__device__ __forceinline__ void emit_f64(const NearArgs &A, const Item &it, float a, float b, uint32_t signs)
{
    const unsigned long long idx = atomicAdd(&A.counters[CNT_F64], 1ULL);
    if (idx < (unsigned long long)A.cap_f64) {
        SubItem si;
        si.it = it;
        si.a = a;
        si.b = b;
        si.signs = signs;
        si.pad = 0;
        A.f64_items[idx] = si;
    } else {
        atomicOr(&A.acc2[it.q], (int)QF_ESCALATE);
    }
}

// (a_hi + a_lo) - (b_hi + b_lo) rounded once to FP32: Knuth's TwoSum of the
// high parts carries their rounding error into the sum of the low parts.
__device__ __forceinline__ float hilo_diff(float ah, float al, float bh, float bl)
{
    const float d = ah - bh;
    const float bb = d - ah;
    const float e = (ah - (d - bb)) + (-bh - bb);
    return d + ((al - bl) + e);
}

// gamma(t) - p of a rational segment in FP32, out of line so that the
// polynomial walk keeps its registers: the homogeneous control points come
// by value (x, y already times w), the weights from global memory.
__device__ __noinline__ float2 near_eval_rat(float4 x0, float4 x1, float4 y0, float4 y1, const float *qw, int n,
                                             int nmax, float t)
{
    const float hx[kNcp] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
    const float hy[kNcp] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
    float mx, my;
    bez_eval_h<float>(hx, hy, qw, n, nmax, t, mx, my);
    return make_float2(mx, my);
}

// Set up the walk of one near pair.  Returns false when the item needs no
// walk (already decided: *result 0 done, 1 boundary).  The query-relative
// control points come from FP32 hi/lo pairs (control point and query, both
// relative to the domain origin), within 2^-24 |q| + eabs of P - p: the
// control point's pair is within 2^-48 |P - o| <= 2^-48 M, the query's
// (p - o from p's truncation and remainder and the origin's pair, within
// 2^-46 (|p - o| + |o|), then the lattice shift T subtracted in
// double-float arithmetic, within 2^-47 (|p - o| + |T|) more) within
// 2^-45 (|p' - o| + 2 |T| + |o|) <= 2^-45 (Mq + 2 Tm + Om), with Mq = 2 M (a
// query beyond Mq goes to FP64) and Om = |o|; eabs = 2^-44 (6 M + 2 Tm +
// Om) covers both and joins the evaluation bound E.
template <bool RAT>
__device__ __forceinline__ bool near_start(const NearArgs &A, const Item &it, NearWalk &W, NearStack &S,
                                           int &result)
{
    const DomDev *Dp = A.doms + it.dom;
    const int4 si = __ldg(&Dp->seg_info[it.seg]);
    const int deg = si.y;
    const float4 *P = Dp->cp32 + si.x;
    float mq = 0.f;
#pragma unroll
    for (int k = 0; k < kNcp; k++) {
        if (k <= deg) {
            const float4 c = __ldg(P + k);
            W.qx[k] = hilo_diff(c.x, c.z, it.fx, it.fxl);
            W.qy[k] = hilo_diff(c.y, c.w, it.fy, it.fyl);
            mq = fmaxf(mq, fabsf(W.qx[k]) + fabsf(W.qy[k]));
        } else {
            W.qx[k] = 0.f;
            W.qy[k] = 0.f;
        }
    }
    const float eabs = kTwoM44 * (6.f * Dp->M + 2.f * Dp->Tm + Dp->Om);
    // the endpoint signs must be those of the exact differences (the sweep
    // decides the same vertices exactly): inside the representation error,
    // the pair goes to FP64, which takes them from the FP64 control points
    if ((fabsf(W.qy[0]) <= eabs) | (fabsf(W.qy[deg]) <= eabs)) {
        emit_f64(A, it, 0.f, 1.f, 0u);
        result = 0;
        return false;
    }
    W.n = deg;
    W.nmax = Dp->max_deg;
    W.B = __int_as_float(si.z);
    W.rat = RAT && si.w != 0;             // RAT: the batch holds rational segments
    // evaluation error bound: de Casteljau on q (2n + 4 ulps of mq); for a
    // rational segment the homogeneous sums and the division scale it by
    // the weight ratio W/w (with a factor 2 to spare)
    W.E = W.rat ? kTwoM24 * mq * (small_i2f(8 * deg + 8) * __int_as_float(si.w) + 8.f) + eabs
                : small_i2f(2 * deg + 4) * kTwoM24 * mq + eabs;
    W.eps = Dp->eps32;
    W.cnt = 0;
    W.a = 0.f;
    W.ax = W.qx[0];
    W.ay = W.qy[0];
    W.sa = W.ay > 0.f;                      // exact: the sign of P0.y - p.y
    W.ra = sqrtf(fmaf(W.ax, W.ax, W.ay * W.ay));
    const float er = W.E + W.ra * kTwoM22;
    if (W.ra + er < W.eps) {
        result = 1;
        return false;
    }
    if (W.ra - er < W.eps) {
        emit_f64(A, it, 0.f, 1.f, (W.sa ? 1u : 0u) | (W.qy[deg] > 0.f ? 2u : 0u));
        result = 0;
        return false;
    }
    S.t[0] = 1.f;
    S.x[0] = W.qx[deg];
    S.y[0] = W.qy[deg];
    S.d[0] = 0;
    if (W.rat) {
        W.qw = Dp->w32 + si.x;
        W.bsub = Dp->seg_bsub32 + 8 * (size_t)it.seg;
#pragma unroll
        for (int k = 0; k < kNcp; k++) {
            const float w = k <= deg ? __ldg(W.qw + k) : 1.f;
            W.qx[k] *= w;
            W.qy[k] *= w;
        }
    }
    W.sp = 1;
    W.b_tested = false;
    return true;
}

// One node of the walk.  Returns 0 while walking, 1 when finished, 2 when the
// query is certainly on the boundary.  The counting build (CNT) adds the
// node's work to wk: one far test per node, a chord per far node, one
// evaluation of gamma(m) (and its degree) per split.
template <bool RAT, bool CNT>
__device__ __forceinline__ int near_step(const NearArgs &A, const Item &it, NearWalk &W, NearStack &S,
                                         uint32_t *wk)
{
    const int sp = W.sp;
    const float b = S.t[sp - 1], bx = S.x[sp - 1], by = S.y[sp - 1];
    const int d = S.d[sp - 1];
    const bool sb = by > 0.f;
    const float rb = sqrtf(fmaf(bx, bx, by * by));
    bool undecided = false;
    if (!W.b_tested) {
        const float er = W.E + rb * kTwoM22;
        if (rb + er < W.eps) return 2;
        undecided = rb - er < W.eps;
        W.b_tested = true;
    }
    float lim = W.B * (b - W.a);
    if (RAT && W.rat && d >= 3) {
        // a node of the walk from [0, 1] lies in the eighth of its start from
        // depth 3 on: the eighth's bound with a margin of 2 eps (the FP64
        // walk's tighter test; es covers the roundings)
        lim = fminf(lim, fmaf(__ldg(W.bsub + eighth_lo(W.a)), b - W.a, 2.f * W.eps));
    }
    const float s = (W.ra + rb) - lim;
    const float es = 2.f * W.E + (W.ra + rb + lim) * (2.f * kTwoM22);
    bool far = false;
    if (!undecided) {
        if (s > es) {
            far = true;
            if (W.sa != sb) {
                const float D = fmaf(W.ax, by, -W.ay * bx);
                if (fabsf(D) <= kTwoM22 * (fabsf(W.ax * by) + fabsf(W.ay * bx))) undecided = true;
                else if (!W.sa && sb && D > 0.f) W.cnt++;
                else if (W.sa && !sb && D < 0.f) W.cnt--;
            }
        } else if (s >= -es || d >= A.depth_cap) {
            undecided = true;
        }
    }
    if constexpr (CNT) {
        wk[0]++;
        if (far && !undecided) wk[1]++;
    }
    if (undecided) {
        // [0, a] is done (its crossings stay in W.cnt); [a, 1] goes to FP64
        // with the walk's sign of gamma(a), so the two parts count the
        // crossings at gamma(a) consistently.  (Handing over only [a, b] and
        // walking on costs more: the walk then continues next to the query.)
        emit_f64(A, it, W.a, 1.f, W.sa ? 1u : 0u);
        W.sp = 0;
        return 1;
    }
    if (far) {
        W.a = b;
        W.ax = bx;
        W.ay = by;
        W.ra = rb;
        W.sa = sb;
        W.sp = sp - 1;
        W.b_tested = true;  // the next top was tested when it was pushed
        return W.sp == 0 ? 1 : 0;
    }
    const float m = 0.5f * (W.a + b);
    float mx, my;
    if (RAT && W.rat) {
        const float2 r = near_eval_rat(make_float4(W.qx[0], W.qx[1], W.qx[2], W.qx[3]),
                                       make_float4(W.qx[4], W.qx[5], W.qx[6], W.qx[7]),
                                       make_float4(W.qy[0], W.qy[1], W.qy[2], W.qy[3]),
                                       make_float4(W.qy[4], W.qy[5], W.qy[6], W.qy[7]), W.qw, W.n, W.nmax, m);
        mx = r.x;
        my = r.y;
    } else {
        bez_eval<float>(W.qx, W.qy, W.n, W.nmax, m, mx, my);
    }
    if constexpr (CNT) {
        wk[2]++;
        wk[3] += (uint32_t)W.n;
    }
    S.d[sp - 1] = d + 1;
    S.t[sp] = m;
    S.x[sp] = mx;
    S.y[sp] = my;
    S.d[sp] = d + 1;
    W.sp = sp + 1;
    W.b_tested = false;
    return 0;
}

// Persistent lanes: walks differ a lot in length (a few nodes for most
// pairs, 30 or more for a query next to the curve), so a lane that finishes
// its walk takes a new pair instead of waiting for the warp's longest walk.
// Starting a pair costs three dependent global loads (pair, segment, control
// points), so idle lanes are refilled together, once at least kNearRefill of
// them wait (A.refill, a tuning knob), and one load latency serves them
// all; every iteration then advances each busy lane by one node.  A warp
// draws up to A.chunk pairs at a time from the queue (one atomic per draw,
// a tuning knob), fewer when the queue is short, so that every warp of the
// grid gets pairs; consecutive pairs come from neighbouring queries of one
// tile, so the lanes' walks stay close in memory.
template <bool RAT, bool CNT>
__global__ void __launch_bounds__(256, 4) k_near(const NearArgs A)
{
    unsigned long long n = A.counters[CNT_NEAR];
    if (n > (unsigned long long)A.cap_near) n = (unsigned long long)A.cap_near;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    // pairs per draw: the queue spread over the grid's warps, 32 to A.chunk
    const unsigned long long n_warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long chunk =
        min((unsigned long long)A.chunk, max(32ULL, (n / n_warps) & ~31ULL));
    uint32_t wk[4] = {0u, 0u, 0u, 0u};
    NearWalk W;
    NearStack S;
    Item it;
    bool busy = false, dry = false;                   // dry: the queue is used up (warp-uniform)
    unsigned long long pool = 0, pool_end = 0;        // the warp's drawn range (warp-uniform)
    for (;;) {
        const unsigned idle = __ballot_sync(0xffffffffu, !busy);
        if (__popc(idle) >= A.refill && !dry) {
            if (pool >= pool_end) {
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(&A.counters[CNT_NEAR_CURSOR], chunk);
                b = __shfl_sync(0xffffffffu, b, 0);
                if (b >= n) {
                    dry = true;
                } else {
                    pool = b;
                    pool_end = min(b + chunk, n);
                }
            }
            if (!dry) {
                if (!busy) {
                    const unsigned long long i = pool + __popc(idle & lt_mask);
                    if (i < pool_end) {
                        it = A.items[i];
                        int res = 0;
                        busy = near_start<RAT>(A, it, W, S, res);
                        if (!busy && res == 1) atomicOr(&A.acc2[it.q], (int)QF_BOUNDARY);
                    }
                }
                pool = min(pool + (unsigned long long)__popc(idle), pool_end);
            }
        }
        if (!__any_sync(0xffffffffu, busy)) {
            if (dry) break;
            continue;
        }
        if (busy) {
            const int r = near_step<RAT, CNT>(A, it, W, S, wk);
            if (r != 0) {
                if (r == 2) atomicOr(&A.acc2[it.q], (int)QF_BOUNDARY);
                else if (W.cnt) atomicAdd(&A.acc2[it.q], 8 * W.cnt);        // 2 crossings each, packed
                busy = false;
            }
        }
    }
    if constexpr (CNT) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const unsigned v = __reduce_add_sync(0xffffffffu, wk[i]);
            if (lane == 0 && v) atomicAdd(&A.work[WK_NEAR_NODE + i], (unsigned long long)v);
        }
    }
}

// ------------------------------------------------------------------ FP64 pairs
__global__ void __launch_bounds__(128) k_f64items(const NearArgs A)
{
    unsigned long long n = A.counters[CNT_F64];
    if (n > (unsigned long long)A.cap_f64) n = (unsigned long long)A.cap_f64;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const SubItem si = A.f64_items[i];
        const Item &it = si.it;
        const DomDev *Dp = A.doms + it.dom;
        double pxp, pyp;
        item_query(Dp, A.src, it, pxp, pyp);
        const int s = (int)it.seg;
        const int deg = Dp->seg_deg[s];
        const double *P = Dp->cp + 2 * (size_t)Dp->seg_cp[s];
        // a sub-interval's end signs are the FP32 walk's (consistent with
        // its counts so far); the curve's own ends are decided exactly here
        const bool sa = si.a == 0.f ? P[1] > pyp : (si.signs & 1u) != 0;
        const bool sb = si.b == 1.f ? P[2 * deg + 1] > pyp : (si.signs & 2u) != 0;
        int cnt = 0;
        const int res = alg1_fp64_sub(P, seg_weights(*Dp, s), deg, Dp->max_deg, Dp->seg_B[s], pxp, pyp, Dp->eps,
                                      (double)si.a, (double)si.b, sa, sb, seg_bsub(*Dp, s), cnt);
        if (res != WALK_DONE) {
            atomicOr(&A.acc2[it.q], (int)QF_BOUNDARY);
            if (res == WALK_DEPTH) atomicAdd(&A.counters[CNT_DEPTH], 1ULL);
        } else if (cnt) {
            atomicAdd(&A.acc2[it.q], 8 * cnt);
        }
    }
}

// ------------------------------------------------------------------ plain FP64
// Sum over every instance the query sees of Algorithm 1 (FP64, atan2 chord
// angles), the chord corrections and line terms of Eq. 9.
__device__ void plain_query(const DomDev *Dp, double x0, double y0, double &om, int &state, bool &depth)
{
    const double x = reduce_period(x0, Dp->Pu), y = reduce_period(y0, Dp->Pv);
    FarAngle fa;
    long long half = 0;
    bool bnd = false;
    depth = false;
    const double eps = Dp->eps;
    for (int j = 0; j < Dp->n_inst && !bnd; j++) {
        const InstDev in = Dp->inst[j];
        const LoopDev &L = Dp->loops[in.loop];
        if (!inst_sees(*Dp, in, L, x, y)) continue;
        if (in.type == IT_LINE) {
            const int s = line_side(*Dp, in, L, x, y);
            if (s == 0) bnd = true;
            half += s;
            continue;
        }
        const double qx = xsub(x, in.Tx), qy = xsub(y, in.Ty);
        // the planar instance covers every loop of the domain
        const int sb = (in.type == IT_ALL) ? 0 : L.s0, se = (in.type == IT_ALL) ? Dp->n_segs : L.s1;
        for (int s = sb; s < se && !bnd; s++) {
            const int res = alg1_fp64(Dp->cp + 2 * (size_t)__ldg(&Dp->seg_cp[s]), seg_weights(*Dp, s),
                                      __ldg(&Dp->seg_deg[s]), Dp->max_deg, __ldg(&Dp->seg_B[s]), qx, qy, eps, fa);
            bnd = res != WALK_DONE;
            depth = res == WALK_DEPTH;
        }
        if (in.type == IT_PE && !bnd) {
            const double ax = L.g0x - qx, ay = L.g0y - qy, bx = L.g0vx - qx, by = L.g0vy - qy;
            fa.ang -= atan2(ax * by - ay * bx, ax * bx + ay * by);
        }
    }
    if (bnd) {
        om = __longlong_as_double(0x7ff8000000000000ULL);
        state = 2;
    } else {
        om = fa.ang / kTwoPi + 0.5 * (double)half;
        state = om >= 0.5 ? 1 : 0;
    }
}


__global__ void __launch_bounds__(128) k_plain(const DomDev *Dp, long long q0, long long n,
                                               PointSrc src, OutDst out, unsigned long long *counters)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t q = (uint32_t)(q0 + i);
        double x, y, om;
        int st;
        bool depth;
        get_point(src, q, x, y);
        plain_query(Dp, x, y, om, st, depth);
        if (depth && counters) atomicAdd(&counters[CNT_DEPTH], 1ULL);
        write_out(out, q, om, st, true);
    }
}

// ------------------------------------------------------------------ finalize
struct FinArgs {
    long long n;
    const int64_t *offsets;
    int n_doms;
    const int32_t *acc2;        // packed, see SweepArgs
    const float *theta;
    uint2 *esc;
    unsigned long long *counters;
    OutDst out;
};

__device__ __forceinline__ uint32_t find_dom(const int64_t *off, int n_doms, long long q)
{
    int lo = 0, hi = n_doms - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    return (uint32_t)lo;
}

__global__ void __launch_bounds__(256) k_finalize(const FinArgs A)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long nround = (A.n + 31) & ~31LL;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nround; i += stride) {
        const bool in_range = i < A.n;
        const uint32_t q = (uint32_t)i;
        int st = 0;
        double om = 0.0;
        bool esc = false;
        if (in_range) {
            const int32_t v = A.acc2[q];
            st = settle(unpack_acc(v), A.theta[q], (uint32_t)v & 3u, A.out.w != nullptr, om);
            esc = st < 0;
            if (esc) {
                const unsigned long long idx = atomicAdd(&A.counters[CNT_ESC], 1ULL);
                A.esc[idx] = make_uint2(q, find_dom(A.offsets, A.n_doms, (long long)q));
            } else {
                write_out(A.out, q, om, st, false);
            }
        }
        if (A.out.bits) {
            const unsigned m = __ballot_sync(0xffffffffu, in_range && !esc && st != 0);
            const unsigned mb = __ballot_sync(0xffffffffu, in_range && !esc && st == 2);
            if ((threadIdx.x & 31) == 0) {
                A.out.bits[i >> 5] = m;
                if (mb && A.out.nbound) atomicAdd(A.out.nbound, (unsigned long long)__popc(mb));
            }
        }
    }
}

// The same for outputs in windings and states (no bitmask), four queries
// per thread and iteration with 16-byte loads and stores (two double2 for
// omega, one word for the states); the outputs must be 16- and 4-byte
// aligned.  The last n mod 4 queries take one thread each.
__global__ void __launch_bounds__(256) k_finalize4(const FinArgs A)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = A.n >> 2;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long j = t0; j < n4; j += stride) {
        const int4 v = __ldg(reinterpret_cast<const int4 *>(A.acc2) + j);
        const float4 th = __ldg(reinterpret_cast<const float4 *>(A.theta) + j);
        const int32_t vv[4] = {v.x, v.y, v.z, v.w};
        const float tt[4] = {th.x, th.y, th.z, th.w};
        double om[4];
        uint32_t stw = 0u;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint32_t q = (uint32_t)(4 * j + k);
            const int st = settle(unpack_acc(vv[k]), tt[k], (uint32_t)vv[k] & 3u, A.out.w != nullptr, om[k]);
            if (st < 0) {
                const unsigned long long idx = atomicAdd(&A.counters[CNT_ESC], 1ULL);
                A.esc[idx] = make_uint2(q, find_dom(A.offsets, A.n_doms, (long long)q));
                om[k] = 0.0;            // rewritten by the FP64 recomputation
            } else {
                stw |= (uint32_t)st << (8 * k);
            }
        }
        if (A.out.w) {
            double2 *w2 = reinterpret_cast<double2 *>(A.out.w) + 2 * j;
            w2[0] = make_double2(om[0], om[1]);
            w2[1] = make_double2(om[2], om[3]);
        }
        if (A.out.st) reinterpret_cast<uint32_t *>(A.out.st)[j] = stw;
    }
    const long long i = 4 * n4 + t0;
    if (i < A.n) {
        const uint32_t q = (uint32_t)i;
        const int32_t v = A.acc2[q];
        double om = 0.0;
        const int st = settle(unpack_acc(v), A.theta[q], (uint32_t)v & 3u, A.out.w != nullptr, om);
        if (st < 0) {
            const unsigned long long idx = atomicAdd(&A.counters[CNT_ESC], 1ULL);
            A.esc[idx] = make_uint2(q, find_dom(A.offsets, A.n_doms, (long long)q));
        } else {
            write_out(A.out, q, om, st, false);
        }
    }
}

// Bit i of a byte to bit 4 i of a word.
__device__ __forceinline__ uint32_t spread4(uint32_t x)
{
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    return (x | (x << 3)) & 0x11111111u;
}

// The bitmask form (a grid's cells, no windings or states out): each warp
// takes 128 consecutive queries, four per lane by 16-byte loads, and writes
// their four words (bit 4 j + k of word w is query 4 (8 w + j) + k of the
// warp's lane 8 w + j, interleaved from four ballots); escalated queries
// keep 0 here and are ORed in by the FP64 recomputation.
__global__ void __launch_bounds__(256) k_finalize_bits4(const FinArgs A)
{
    const int lane = threadIdx.x & 31;
    const long long n_tasks = (A.n + 127) >> 7;
    const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; t < n_tasks; t += n_warps) {
        const long long q0 = 128 * t + 4 * lane;
        int32_t v[4] = {0, 0, 0, 0};
        float th[4] = {0.f, 0.f, 0.f, 0.f};
        if (q0 + 3 < A.n) {
            const int4 a = __ldg(reinterpret_cast<const int4 *>(A.acc2) + (q0 >> 2));
            const float4 b = __ldg(reinterpret_cast<const float4 *>(A.theta) + (q0 >> 2));
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            th[0] = b.x; th[1] = b.y; th[2] = b.z; th[3] = b.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (q0 + k < A.n) {
                    v[k] = A.acc2[q0 + k];
                    th[k] = A.theta[q0 + k];
                }
        }
        unsigned m[4], mb[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const bool in_range = q0 + k < A.n;
            bool esc = false;
            int st = 0;
            if (in_range) {
                double om;
                st = settle(unpack_acc(v[k]), th[k], (uint32_t)v[k] & 3u, false, om);
                esc = st < 0;
                if (esc) {
                    const uint32_t q = (uint32_t)(q0 + k);
                    const unsigned long long idx = atomicAdd(&A.counters[CNT_ESC], 1ULL);
                    A.esc[idx] = make_uint2(q, find_dom(A.offsets, A.n_doms, (long long)q));
                }
            }
            m[k] = __ballot_sync(0xffffffffu, in_range && !esc && st != 0);
            mb[k] = __ballot_sync(0xffffffffu, in_range && !esc && st == 2);
        }
        if (lane < 4) {
            uint32_t word = 0u;
#pragma unroll
            for (int k = 0; k < 4; k++) word |= spread4((m[k] >> (8 * lane)) & 0xffu) << k;
            const long long wi = 4 * t + lane;
            if (32 * wi < A.n) A.out.bits[wi] = word;
        }
        if (lane == 0 && A.out.nbound) {
            const int nb = __popc(mb[0]) + __popc(mb[1]) + __popc(mb[2]) + __popc(mb[3]);
            if (nb) atomicAdd(A.out.nbound, (unsigned long long)nb);
        }
    }
}

struct EscArgs {
    const DomDev *doms;
    PointSrc src;
    const uint2 *esc;
    unsigned long long *counters;
    OutDst out;
};

// FP64 recomputation of the escalated queries in the crossing form of the
// mixed path, every step exact up to FP64 rounding: per record of every
// instance the query sees, the signed crossings of the +x ray by the chords
// Algorithm 1 leaves of its segment (root step first, the FP64 walk only when
// the query is inside the root ellipse), then its gap's crossing and angle;
// omega = crossings + line halves - sum(gap angles) / 2 pi.  (Summing Eq. 3's
// chord angles instead, as k_plain does, costs an FP64 atan2 at every node
// of the walks next to the query.)  FP64 is the slow unit, so each query is
// spread over one cluster of kEscCluster CTAs, i.e. as many SMs: every CTA's
// threads share a slice of the records and reduce their sums in shared
// memory; the cluster's first CTA then adds the CTAs' partial sums from their
// shared memory and writes the result.
constexpr int kEscThreads = 128;
constexpr int kEscCluster = 8;              // CTAs (one per SM) per escalated query

// One record against the query (p relative to the instance) in FP64: the
// crossings of its segment's Algorithm 1 chords (or of the closing chord),
// its gap's crossing and angle.  Returns WALK_DONE, or WALK_BOUNDARY /
// WALK_DEPTH when the query is on the boundary.
__device__ __noinline__ int record_f64(const DomDev *__restrict__ Dp, int r, double pxp, double pyp, int &c,
                                        double &dth)
{
    const uint32_t fl = __float_as_uint(Dp->rec[4 * r + 1].w);
    const double2 a = Dp->rec_a64[r], b = Dp->rec_b64[r], nx = Dp->rec_n64[r];
    const bool sa = a.y > pyp, sb = b.y > pyp, sn = nx.y > pyp;
    c = 0;
    dth = 0.0;
    bool chord = true;              // the straight chord a -> b decides the crossings
    if (!(fl & RF_CHORD)) {
        const int s = (int)(fl >> RF_SEG_SHIFT);
        const double ax = a.x - pxp, ay = a.y - pyp, bx = b.x - pxp, by = b.y - pyp;
        const double qa = ax * ax + ay * ay, qb = bx * bx + by * by;
        const double eps = Dp->eps;
        if (qa < eps * eps || qb < eps * eps) return WALK_BOUNDARY;
        const double L = Dp->seg_B[s];
        const double S = L * L - (qa + qb);
        if (!(S < 0.0 || 4.0 * qa * qb > S * S)) {
            // inside the root ellipse: the FP64 walk
            int cnt = 0;
            const int res = alg1_fp64_sub(Dp->cp + 2 * (size_t)Dp->seg_cp[s], seg_weights(*Dp, s), Dp->seg_deg[s],
                                          Dp->max_deg, L, pxp, pyp, eps, 0.0, 1.0, sa, sb, seg_bsub(*Dp, s), cnt);
            if (res != WALK_DONE) return res;
            c = cnt;
            chord = false;
        }
    }
    if (chord && sa != sb) {
        const bool pos = exact_cross(a, b, pxp, pyp) > 0;
        c += (!sa && sb && pos) ? 1 : ((sa && !sb && !pos) ? -1 : 0);
    }
    if (fl & RF_GAP) {
        const double ux = b.x - pxp, uy = b.y - pyp, vx = nx.x - pxp, vy = nx.y - pyp;
        const double d = ux * vy - uy * vx;
        if (sb != sn) {
            const bool pos = d > 0;
            c += (!sb && sn && pos) ? 1 : ((sb && !sn && !pos) ? -1 : 0);
        }
        dth = atan2(d, ux * vx + uy * vy);
    }
    return WALK_DONE;
}

__global__ void __cluster_dims__(kEscCluster, 1, 1) __launch_bounds__(kEscThreads) k_f64query(const EscArgs A)
{
    __shared__ double s_th[kEscThreads];
    __shared__ long long s_acc[kEscThreads];
    __shared__ int s_bnd[kEscThreads];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x;
    const unsigned long long n = A.counters[CNT_ESC];
    const unsigned long long n_cl = gridDim.x / kEscCluster;
    for (unsigned long long i = blockIdx.x / kEscCluster; i < n; i += n_cl) {
        const uint2 e = A.esc[i];
        const DomDev *Dp = A.doms + e.y;
        double x0, y0;
        get_point(A.src, e.x, x0, y0);
        const double x = reduce_period(x0, Dp->Pu), y = reduce_period(y0, Dp->Pv);
        double th = 0.0;
        long long acc = 0;            // 2 * crossings + line sides
        bool bnd = false;
        for (int j = 0; j < Dp->n_inst; j++) {
            const InstDev in = Dp->inst[j];
            const LoopDev &L = Dp->loops[in.loop];
            if (!inst_sees(*Dp, in, L, x, y)) continue;
            if (in.type == IT_LINE) {
                if (tid == 0 && rank == 0) {
                    const int sd = line_side(*Dp, in, L, x, y);
                    bnd |= sd == 0;
                    acc += sd;
                }
                continue;
            }
            const double qx = xsub(x, in.Tx), qy = xsub(y, in.Ty);
            for (int r = in.r0 + rank * kEscThreads + tid; r < in.r1 && !bnd; r += kEscCluster * kEscThreads) {
                int c;
                double dth;
                const int res = record_f64(Dp, r, qx, qy, c, dth);
                if (res == WALK_DEPTH) atomicAdd(&A.counters[CNT_DEPTH], 1ULL);
                bnd |= res != WALK_DONE;
                acc += 2 * c;
                th += dth;
            }
        }
        s_th[tid] = th;
        s_acc[tid] = acc;
        s_bnd[tid] = bnd ? 1 : 0;
        __syncthreads();
        for (int w = kEscThreads / 2; w > 0; w >>= 1) {
            if (tid < w) {
                s_th[tid] += s_th[tid + w];
                s_acc[tid] += s_acc[tid + w];
                s_bnd[tid] |= s_bnd[tid + w];
            }
            __syncthreads();
        }
        cl.sync();
        if (rank == 0 && tid == 0) {
            double tsum = 0.0;
            long long asum = 0;
            int bd = 0;
            for (int r = 0; r < kEscCluster; r++) {
                tsum += *cl.map_shared_rank(&s_th[0], r);
                asum += *cl.map_shared_rank(&s_acc[0], r);
                bd |= *cl.map_shared_rank(&s_bnd[0], r);
            }
            double om;
            int st;
            if (bd) {
                om = __longlong_as_double(0x7ff8000000000000ULL);
                st = 2;
            } else {
                om = 0.5 * (double)asum - tsum / kTwoPi;
                st = om >= 0.5 ? 1 : 0;
            }
            write_out(A.out, e.x, om, st, true);
        }
        cl.sync();      // the partial sums stay until the first CTA has read them
    }
}

// ------------------------------------------------------------------ pairing support
// PE(x, loop a at family shift (IA, JA)) for x = mid(loop b) + (IB Pu, JB Pv),
// Eq. 9 in FP64 with the slab window (App. C, Alg. 8 ToLeft).

__global__ void k_pe_eval(const DomDev *Dp, const PeReq *req, int n, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const PeReq R = req[i];
    const LoopDev &Lb = Dp->loops[R.b];
    const int m = Lb.s1 - Lb.s0;
    const int s = Lb.s0 + m / 2;
    const double t = (m % 2) ? 0.5 : 0.0;
    const int deg = Dp->seg_deg[s];
    const double *P = Dp->cp + 2 * (size_t)Dp->seg_cp[s];
    SegF64 sgm;
    sgm.load(P, seg_weights(*Dp, s), deg, Dp->max_deg);
    double mx, my;
    sgm.eval(t, mx, my);
    const double Pu = Dp->Pu, Pv = Dp->Pv;
    const double x = xadd(mx, xmul((double)R.IB, Pu)), y = xadd(my, xmul((double)R.JB, Pv));
    const LoopDev &L = Dp->loops[R.a];
    const double xf = (Pu > 0) ? xsub(x, xmul((double)R.IA, Pu)) : x;
    const double yf = (Pv > 0) ? xsub(y, xmul((double)R.JA, Pv)) : y;
    const double cr = xsub(xmul(L.vx, xsub(yf, L.g0y)), xmul(L.vy, xsub(xf, L.g0x)));
    if (cr == 0) {
        out[i] = __longlong_as_double(0x7ff8000000000000ULL);
        return;
    }
    FarAngle fa;
    const double sp = xdiv(xadd(xmul(xf, L.vx), xmul(yf, L.vy)), L.vv);
    const double klo = ceil(xsub(sp, L.smax)), khi = floor(xsub(sp, L.smin));
    for (double k = klo; k <= khi; k += 1.0) {
        const long long kk = (long long)k;
        const double qx = (Pu > 0) ? xsub(x, xmul((double)(R.IA + kk * L.hp), Pu)) : x;
        const double qy = (Pv > 0) ? xsub(y, xmul((double)(R.JA + kk * L.hq), Pv)) : y;
        for (int sg = L.s0; sg < L.s1; sg++) {
            if (alg1_fp64(Dp->cp + 2 * (size_t)Dp->seg_cp[sg], seg_weights(*Dp, sg), Dp->seg_deg[sg], Dp->max_deg,
                          Dp->seg_B[sg], qx, qy,
                          Dp->eps, fa)) {
                out[i] = __longlong_as_double(0x7ff8000000000000ULL);
                return;
            }
        }
        const double ax = L.g0x - qx, ay = L.g0y - qy, bx = L.g0vx - qx, by = L.g0vy - qy;
        fa.ang -= atan2(ax * by - ay * bx, ax * bx + ay * by);
    }
    out[i] = fa.ang / kTwoPi + (cr > 0 ? 0.5 : -0.5);
}

// ------------------------------------------------------------------ launchers
int bin_blocks_per_sm(int scatter)
{
    static int per_sm[2] = {0, 0};
    if (!per_sm[scatter]) {
        int n = 0;
        const cudaError_t e = scatter ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bin_scatter, kBinThreads, 0)
                                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bin_count, kBinThreads, 0);
        per_sm[scatter] = (e == cudaSuccess && n > 0) ? n : 1;
    }
    return per_sm[scatter];
}

bool mixed_buckets(const Work &W, const LaunchCfg &cfg)
{
    return cfg.tun.tree && cfg.tun.bucket && !cfg.grid_tiled && W.perm && W.cell_of && W.cell_cnt && W.dcell &&
           W.bin_chunk && W.bchunks && W.run_off && W.n_cells > 0 && W.n_bchunks > 0;
}

int mixed_kernel_count(const Work &W, const LaunchCfg &cfg)
{
    return 5 + (mixed_buckets(W, cfg) ? 5 : 0) + (cfg.tun.tree && cfg.n_flat > 0 ? 1 : 0);
}

cudaError_t launch_mixed(const Work &W, const DomDev *d_doms, int n_doms, const int4 *d_units,
                         int n_units, const int64_t *d_offsets, int64_t n_queries, PointSrc src,
                         OutDst out, const LaunchCfg &cfg, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(W.counters, 0, CNT_N * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    cudaEvent_t ev[kProfEvents] = {};
    if (cfg.events) {
        for (int i = 0; i < kProfEvents; i++) {
            if ((e = cudaEventCreate(&ev[i])) != cudaSuccess) return e;
            cfg.events->push_back(ev[i]);
        }
    }
    auto mark = [&](int i) {
        if (cfg.events) cudaEventRecord(ev[i], s);
    };
    if (out.nbound) {
        e = cudaMemsetAsync(out.nbound, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    const bool bucket = mixed_buckets(W, cfg);
    mark(0);
    if (bucket) {
        BinArgs ba;
        ba.doms = d_doms;
        ba.n = n_queries;
        ba.chunk = W.bin_chunk;
        ba.src = src;
        ba.dcell = W.dcell;
        ba.cell_of = W.cell_of;
        ba.cnt = W.cell_cnt;
        ba.run_off = W.run_off;
        ba.counters = W.counters;
        ba.perm = W.perm;
        ba.n_cells = W.n_cells;
        if ((e = cudaMemsetAsync(W.cell_cnt, 0, (size_t)W.n_cells * sizeof(int), s)) != cudaSuccess) return e;
        ba.bchunks = W.bchunks;
        ba.n_bchunks = W.n_bchunks;
        // one wave: as many CTAs as fit on the SMs at once (they draw runs
        // from a counter, so no CTA waits for a slot while others idle)
        const int count_blocks = std::max(1, std::min(W.n_bchunks, cfg.n_sm * bin_blocks_per_sm(0)));
        const int scatter_blocks = std::max(1, std::min(W.n_bchunks, cfg.n_sm * bin_blocks_per_sm(1)));
        const int n_chunks = (W.n_cells + kBinChunk - 1) / kBinChunk;
        k_bin_count<<<count_blocks, kBinThreads, 0, s>>>(ba);
        k_bin_chunk_sum<<<n_chunks, 1024, 0, s>>>(ba);
        k_bin_chunk_scan<<<1, 1024, 0, s>>>(ba, n_chunks);
        k_bin_chunk_apply<<<n_chunks, 1024, 0, s>>>(ba);
        k_bin_scatter<<<scatter_blocks, kBinThreads, 0, s>>>(ba);
    }
    SweepArgs sa;
    sa.doms = d_doms;
    sa.units = d_units;
    sa.n_units = n_units;
    sa.perm = bucket ? W.perm : nullptr;
    sa.src = src;
    sa.acc2 = W.acc2;
    sa.theta = W.theta;
    sa.near_items = W.near_items;
    sa.cap_near = W.cap_near;
    sa.counters = W.counters;
    sa.work = cfg.work;
    sa.unit_ctr = CNT_UNIT;
    const int sweep_grid = max(1, min(n_units, cfg.n_sm * cfg.tun.sweep_ctas_per_sm));
    mark(1);
    if (cfg.tun.tree && cfg.n_flat > 0) {
        // the small planar domains: the flat sweep over their own units
        SweepArgs fa_ = sa;
        fa_.units = d_units + n_units;
        fa_.n_units = cfg.n_flat;
        fa_.perm = nullptr;
        fa_.unit_ctr = CNT_FLAT_UNIT;
        k_sweep<kFlatQpt><<<max(1, min(cfg.n_flat, cfg.n_sm * 3)), kSweepThreads, 0, s>>>(fa_);
    }
    if (cfg.tun.tree) {
        // the level flags fit 2 slots; the register budget follows the CTAs
        // per SM (2: 128 registers, 3: 80, more: 64)
        const int cps = cfg.tun.sweep_ctas_per_sm;
        if (cfg.work) {
            if (cfg.tun.qpt == 1) k_sweep_tree<1, true, 4><<<sweep_grid, kSweepThreads, 0, s>>>(sa);
            else k_sweep_tree<2, true, 4><<<sweep_grid, kSweepThreads, 0, s>>>(sa);
        } else if (cfg.tun.qpt == 1) {
            if (cps <= 2) k_sweep_tree<1, false, 2><<<sweep_grid, kSweepThreads, 0, s>>>(sa);
            else if (cps == 3) k_sweep_tree<1, false, 3><<<sweep_grid, kSweepThreads, 0, s>>>(sa);
            else k_sweep_tree<1, false, 4><<<sweep_grid, kSweepThreads, 0, s>>>(sa);
        } else {
            if (cps <= 2) k_sweep_tree<2, false, 2><<<sweep_grid, kSweepThreads, 0, s>>>(sa);
            else if (cps == 3) k_sweep_tree<2, false, 3><<<sweep_grid, kSweepThreads, 0, s>>>(sa);
            else k_sweep_tree<2, false, 4><<<sweep_grid, kSweepThreads, 0, s>>>(sa);
        }
    } else {
        switch (cfg.tun.qpt) {
        case 1: k_sweep<1><<<sweep_grid, kSweepThreads, 0, s>>>(sa); break;
        case 4: k_sweep<4><<<sweep_grid, kSweepThreads, 0, s>>>(sa); break;
        default: k_sweep<2><<<sweep_grid, kSweepThreads, 0, s>>>(sa); break;
        }
    }
    NearArgs na;
    na.doms = d_doms;
    na.src = src;
    na.items = W.near_items;
    na.cap_near = W.cap_near;
    na.acc2 = W.acc2;
    na.f64_items = W.f64_items;
    na.cap_f64 = W.cap_f64;
    na.counters = W.counters;
    na.depth_cap = std::min(std::max(cfg.tun.near_depth, kDepthCap32Min), kDepthCap32Max);
    na.chunk = std::min(std::max(cfg.tun.near_chunk, kNearChunkMin), kNearChunkMax) & ~31;
    na.refill = std::min(std::max(cfg.tun.near_refill, 1), 32);
    na.work = cfg.work;
    mark(2);
    {
        const int g = cfg.n_sm * cfg.tun.near_ctas_per_sm;
        if (cfg.work) {
            if (cfg.rational) k_near<true, true><<<g, 256, 0, s>>>(na);
            else k_near<false, true><<<g, 256, 0, s>>>(na);
        } else {
            if (cfg.rational) k_near<true, false><<<g, 256, 0, s>>>(na);
            else k_near<false, false><<<g, 256, 0, s>>>(na);
        }
    }
    mark(3);
    k_f64items<<<cfg.n_sm * 16, 128, 0, s>>>(na);
    mark(4);
    FinArgs fa;
    fa.n = n_queries;
    fa.offsets = d_offsets;
    fa.n_doms = n_doms;
    fa.acc2 = W.acc2;
    fa.theta = W.theta;
    fa.esc = W.esc_q;
    fa.counters = W.counters;
    fa.out = out;
    const long long fin_blocks = std::max(1LL, std::min((long long)(n_queries + 255) / 256, (long long)cfg.n_sm * 16));
    if (!out.bits && ((uintptr_t)out.w & 15u) == 0 && ((uintptr_t)out.st & 3u) == 0)
        k_finalize4<<<(int)std::max(1LL, std::min((long long)(n_queries / 4 + 255) / 256, (long long)cfg.n_sm * 16)),
                      256, 0, s>>>(fa);
    else if (out.bits && !out.w && !out.st)
        k_finalize_bits4<<<(int)std::max(1LL, std::min((long long)(n_queries / 4 + 255) / 256,
                                                         (long long)cfg.n_sm * 16)),
                           256, 0, s>>>(fa);
    else
        k_finalize<<<(int)fin_blocks, 256, 0, s>>>(fa);
    mark(5);
    EscArgs ea;
    ea.doms = d_doms;
    ea.src = src;
    ea.esc = W.esc_q;
    ea.counters = W.counters;
    ea.out = out;
    k_f64query<<<std::max(1, cfg.n_sm * 2 / kEscCluster) * kEscCluster, kEscThreads, 0, s>>>(ea);
    mark(6);
    return cudaGetLastError();
}

__global__ void k_gap_angle(const float *y, const float *x, float *out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = gap_angle(y[i], x[i]);
}

cudaError_t launch_gap_angle(const float *y, const float *x, float *out, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min((n + 255) / 256, (int64_t)4096);
    k_gap_angle<<<(int)blocks, 256, 0, s>>>(y, x, out, n);
    return cudaGetLastError();
}

cudaError_t launch_plain(const DomDev *d_dom, int64_t q0, int64_t n, PointSrc src, OutDst out,
                         unsigned long long *counters, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min((long long)(n + 127) / 128, 1LL << 20);
    k_plain<<<(int)blocks, 128, 0, s>>>(d_dom, q0, n, src, out, counters);
    return cudaGetLastError();
}

cudaError_t launch_pe_eval(const DomDev *d_dom, const PeReq *d_req, int n, double *d_out,
                           cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_pe_eval<<<(n + 63) / 64, 64, 0, s>>>(d_dom, d_req, n, d_out);
    return cudaGetLastError();
}

}  // namespace wn
