// wn_dev.cuh -- device data layout and arithmetic primitives of the
// containment-query library (internal; not part of the C ABI).
//
// Terminology follows Bao, Shen & Wang, "Fast and Robust Point Containment
// Queries on Trimmed Surface":
//   segment  a Bezier curve gamma with control points P_0..P_n (Sec. 4.2)
//   B        the hodograph bound max_i n|P_i - P_{i-1}| (Lemma 1, App. A.1)
//   loop     consecutive segments; lifted to the covering space (Sec. 4.3)
//   instance one lattice copy of a loop that a query may see: the loop itself
//            (planar), a contractible copy (Alg. 4-5 reading), one copy of a
//            periodically extended curve (Eq. 9), or a line term (Sec. 4.4)
//
// Every copy is a lattice translation T = (I Pu, J Pv) applied to the query
// (p' = p - T, the translation identity of App. C.1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <math.h>

namespace wn {

constexpr int kMaxDeg = 7;
constexpr int kNcp = kMaxDeg + 1;
constexpr int kDepthCap64 = 64;   // FP64 recursion cap: reported as BOUNDARY
constexpr int kDepthCap32Max = 30;  // largest FP32 recursion cap: the pair then goes to FP64
// What an FP64 walk of Algorithm 1 ended in.
enum : int { WALK_DONE = 0, WALK_BOUNDARY = 1, WALK_DEPTH = 2 };

enum : int { DK_PLANAR = 0, DK_UNI_U = 1, DK_UNI_V = 2, DK_BI = 3 };
enum : int { IT_ALL = 0, IT_BOX = 1, IT_PE = 2, IT_LINE = 3 };
enum : uint32_t { QF_BOUNDARY = 1u, QF_ESCALATE = 2u };
enum : uint32_t { RF_CHORD = 1u, RF_GAP = 2u };
// Record flags carry the record's segment in their upper 30 bits
// (RF_NO_SEG for a closing chord).
constexpr int RF_SEG_SHIFT = 2;
constexpr uint32_t RF_NO_SEG = 0x3FFFFFFFu;

// One lifted loop (FP64).
struct LoopDev {
    int s0, s1;                 // segments [s0, s1)
    int r0, r1;                 // FP32 records [r0, r1)
    int hp, hq;                 // homology
    int cls, root;              // 0 plain, 1 contractible, 2 extended; record-tree root (-1: none)
    double vx, vy;              // lattice vector (hp Pu, hq Pv)
    double g0x, g0y;            // gamma(0)
    double g0vx, g0vy;          // gamma(0) + v
    double smin, smax, vv;      // slab of the curve along v, v.v
    double box[4];              // xmin xmax ymin ymax of control points
    double nlo, nhi;            // extent along the family normal (bi-periodic)
};

// One instance (FP64 predicate data).
struct InstDev {
    int type;                   // IT_*
    int loop;
    int pair;                   // bi-periodic pair for the family window, -1 none
    int axes;                   // IT_BOX: bit0 window x, bit1 window y
    int r0, r1;                 // FP32 records swept for this instance
    double Tx, Ty;              // query shift: p' = p - (Tx, Ty)
    double Fx, Fy;              // family shift for the slab / line: x_f = p - (Fx, Fy)
    long long I, J;             // lattice units of (Fx, Fy)
    long long c;                // family index
    long long k;                // copy index along v
};

struct PairDev {
    double plo, phi;            // hull of the n-extents of alpha and shifted beta
};

// Where in query space (reduced to the base tile) an instance can see a
// query: a box, a strip along the family normal n and a strip along the
// loop's lattice vector v (each +-inf where it does not constrain), widened
// so that every query its exact test accepts lies inside, and rounded
// outward to FP32.  Used to skip an instance for a whole warp at once.
struct InstCull {
    float x0, x1, y0, y1;       // box
    float n0, n1;               // n.p range (family window)
    float v0, v1;               // v.p range (copy slab)
    float vx, vy;               // v (0 when the instance has no slab)
    float pad0, pad1;
};

// The FP32 side of one instance, so that the sweep decides most (query,
// instance) pairs without FP64 instructions (GB300's FP64 unit is narrow):
// its lattice shift as hi/lo pairs, the exact window shrunk well beyond the
// rounding of its test and rounded inward (a query inside it is seen), and
// for a line term the base point and direction of its line.
struct InstF32 {
    float txh, txl, tyh, tyl;   // (Tx, Ty) = (txh + txl, tyh + tyl) to ~2^-48
    float x0, x1, y0, y1;       // inner box
    float n0, n1, v0, v1;       // inner n.p and v.p ranges
    float lx, ly, lvx, lvy;     // line term: (Fx + g0x, Fy + g0y) (F on periodic axes), v
};

// Everything a kernel needs about one domain (copied per batch entry).
struct DomDev {
    int kind, n_loops, n_segs, n_inst, n_rec, n_pairs;
    int total_cp, max_deg;              // largest segment degree
    double Pu, Pv, eps;
    double ox, oy;              // origin of the FP32 coordinates
    double nx, ny, PP;          // family normal and Pu*Pv (bi-periodic)
    float M;                    // max |P - o|_inf over lifted control points
    float Tm;                   // max |lattice shift|_inf over the instances (0 planar)
    float Mq;                   // queries with |p' - o|_inf > Mq go to FP64
    float Om;                   // max(|ox|, |oy|)
    float nxf, nyf;             // nx, ny rounded to FP32
    float oxh, oxl, oyh, oyl;   // the origin as FP32 pairs (to ~2^-48)
    const int *seg_deg;         // [n_segs]
    const int *seg_cp;          // [n_segs] first control point (in points)
    const double *cp;           // [2 * total_cp] lifted control points
    const double *seg_B;        // [n_segs]
    const LoopDev *loops;       // [n_loops]
    const InstDev *inst;        // [n_inst]
    const InstCull *cull;       // [n_inst]
    const InstF32 *instf;       // [n_inst]
    const PairDev *pairs;       // [n_pairs]
    const float4 *rec;          // [4 * n_rec]: (a, b), (centre, R^2, flags), (gap, next), (b low)
    const int *rec_seg;         // [n_rec] segment, -1 for a closing chord
    const float4 *rec_obb;      // [n_rec] (t0, t1, d0, d1): control points' box in the chord's frame
    const double2 *rec_a64;     // [n_rec] exact chord start
    const double2 *rec_b64;     // [n_rec] exact chord end
    const double2 *rec_n64;     // [n_rec] exact next vertex
    const float4 *nodes;        // [kCluF4 * n_nodes] record tree, see below
    int n_nodes;
    int all_root;               // planar: root over every loop (-1: per-loop roots)
    const float4 *cp32;         // [total_cp] P - origin as FP32 (hi.x, hi.y, lo.x, lo.y)
    const int4 *seg_info;       // [n_segs] (first control point, degree, B as FP32 bits, weight
                                //   ratio W/w as FP32 bits for a rational segment, else 0)
    const double *w;            // [total_cp] weights, or null when no segment is rational
    const float *w32;           // [total_cp] the weights rounded to FP32, or null
    const double *seg_bsub;     // [8 n_segs] bound of |gamma'| on each eighth [j/8, (j+1)/8]
                                //   of a segment (rational domains only, else null)
    const float *seg_bsub32;    // [8 n_segs] the same rounded up to FP32, or null
    float eps32;                // eps rounded to FP32
    int pad4;
};

// Record tree: per loop, leaves over runs of at most kCluRecs consecutive
// records and internal nodes over kTreeArity consecutive children.  Each node
// covers a contiguous record range; per node, kCluF4 float4 (FP32, relative
// to the domain origin):
//   [0] near box (xmin, xmax, ymin, ymax): outside it, by the query's error
//       band, a query is outside every record's circle below the node (so far
//       from every segment's ellipse and eps discs);
//   [1] (ymin, ymax, xmax) of every vertex of its pieces (a query above,
//       below or right of them cannot meet them with its +x ray), and the
//       squared distance from z_c beyond which the gap-angle expansion is used;
//   [2] expansion centre z_c, hi and lo parts;
//   [3] (r_c, flags: bit 0 gaps, bit 1 leaf, first, end) -- the last three as
//       int bits; first/end index records (leaf) or child nodes;
//   [4] squared distances beyond which 4, 8, 12, 16 terms suffice;
//   [5] squared distances beyond which 20, 24, 28 terms suffice;
//   [6] (xmin of every vertex, y of the first record's start, y of the last
//       record's next vertex, first record as int bits): the pieces below the
//       node form one polyline from that start to that end, so a query left
//       of xmin sees crossings = [end above] - [start above];
//   [7] (end record as int bits, 0, 0, 0);
//   [8 ..] kCluTerms complex coefficients c_k of the Laurent expansion of the
//       sum of the cluster's gap angles:
//         sum_gaps theta = Im sum_k c_k w^k,   w = r_c / (z_c - p),
//       truncated after K terms with error at most C |w|^(K+1) / (1 - |w|),
//       C = max_k |c_k| <= sum |gap| / r_c; the distances in [1], [4], [5]
//       keep that below kCluTol radians.
constexpr int kCluRecs = 8;
constexpr int kTreeArity = 4;
constexpr int kTreeMaxLevels = 16;
constexpr int kCluTerms = 32;
constexpr int kCluCoef = 8;                 // first float4 of the coefficients
constexpr int kCluF4 = kCluCoef + (kCluTerms + 1) / 2;
// Truncation error allowed per expansion sum, radians.  Even a query that
// takes 150 expansion sums stays below 1.5e-5 rad (2.4e-6 in omega): inside
// the 1e-5 omega tolerance of the mixed path and far inside its 1e-4
// classification band.
constexpr double kCluTol = 1e-7;

// Near / FP64 work item.
struct Item {
    uint32_t q;                 // global query index
    uint32_t dom;               // batch entry
    uint32_t inst;
    uint32_t seg;               // the record's segment
    float fx, fy, fxl, fyl;     // p - (Tx, Ty) - origin as FP32 hi + lo (from the sweep)
};

// FP64 work item: the sub-interval [a, b] of a near pair whose FP32 error
// band could not settle a decision, with the signs (bit 0: gamma(a) above
// the query, bit 1: gamma(b) above) that the FP32 chain already used for
// its end points.
struct SubItem {
    Item it;
    float a, b;
    uint32_t signs;
    uint32_t pad;
};

// ---------------------------------------------------------------- exact FP64
// Predicates that decide which copies a query sees are evaluated with
// explicitly rounded operations (no FMA contraction), in the order the
// definitions state them.
__host__ __device__ __forceinline__ double xmul(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
__host__ __device__ __forceinline__ double xadd(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
__host__ __device__ __forceinline__ double xsub(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}
__host__ __device__ __forceinline__ double xdiv(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __ddiv_rn(a, b);
#else
    return a / b;
#endif
}

// Reduce a coordinate into [0, P) (identity when P <= 0).
__host__ __device__ __forceinline__ double reduce_period(double x, double P)
{
#ifdef __CUDA_ARCH__
    // the common cases decided with integer instructions (GB300's FP64 unit
    // is narrow): the bit patterns of non-negative doubles order as their
    // values, and P is never NaN
    const long long pb = __double_as_longlong(P), xb = __double_as_longlong(x);
    if (pb <= 0) return x;                  // P <= 0: no period on this axis
    if (xb >= 0 && xb < pb) return x;       // +0 <= x < P (NaN and -0 take the general path)
#endif
    if (!(P > 0)) return x;
    if (x >= 0.0 && x < P) return x;        // already in the base tile: fmod(x, P) == x
    double r = fmod(x, P);
    if (r < 0) r = xadd(r, P);
    if (r >= P) r = 0.0;
    return r;
}

// Does instance `in` see the reduced query (x, y)?  Exactly the windows of
// the contractible copies, the slab of Eq. 9 and the family window.
__device__ __forceinline__ bool inst_sees(const DomDev &D, const InstDev &in, const LoopDev &L,
                                          double x, double y)
{
    if (in.type == IT_ALL) return true;
    if (in.type == IT_BOX) {
        if (in.axes & 1) {
            double xs = xsub(x, in.Tx);
            if (!(xs >= L.box[0] && xs <= L.box[1])) return false;
        }
        if (in.axes & 2) {
            double ys = xsub(y, in.Ty);
            if (!(ys >= L.box[2] && ys <= L.box[3])) return false;
        }
        return true;
    }
    if (in.pair >= 0) {
        const PairDev P = D.pairs[in.pair];
        double np = xadd(xmul(D.nx, x), xmul(D.ny, y));
        double clo = ceil(xdiv(xsub(np, P.phi), D.PP));
        double chi = floor(xdiv(xsub(np, P.plo), D.PP));
        double c = (double)in.c;
        if (!(c >= clo && c <= chi)) return false;
    }
    if (in.type == IT_LINE) return true;
    // IT_PE: copy k lies in the slab window of the family base point
    double xf = (D.Pu > 0) ? xsub(x, in.Fx) : x;
    double yf = (D.Pv > 0) ? xsub(y, in.Fy) : y;
    double sp = xdiv(xadd(xmul(xf, L.vx), xmul(yf, L.vy)), L.vv);
    double klo = ceil(xsub(sp, L.smax)), khi = floor(xsub(sp, L.smin));
    double k = (double)in.k;
    return k >= klo && k <= khi;
}

// Can an instance see any query in the box [bx0, bx1] x [by0, by1] (FP32,
// rounded outward; wmag = the largest |coordinate| of the box)?  True
// whenever the exact test (inst_sees) accepts some query of the box: the
// projections carry a slack above their FP32 rounding.
__device__ __forceinline__ bool cull_sees(const InstCull &c, float nx, float ny, float bx0, float bx1,
                                          float by0, float by1, float wmag)
{
    if (bx1 < c.x0 || bx0 > c.x1 || by1 < c.y0 || by0 > c.y1) return false;
    const float sn = 4e-7f * (fabsf(nx) + fabsf(ny)) * wmag;
    const float n_lo = fmaf(nx, nx >= 0.f ? bx0 : bx1, ny * (ny >= 0.f ? by0 : by1));
    const float n_hi = fmaf(nx, nx >= 0.f ? bx1 : bx0, ny * (ny >= 0.f ? by1 : by0));
    if (n_hi + sn < c.n0 || n_lo - sn > c.n1) return false;
    const float sv = 4e-7f * (fabsf(c.vx) + fabsf(c.vy)) * wmag;
    const float v_lo = fmaf(c.vx, c.vx >= 0.f ? bx0 : bx1, c.vy * (c.vy >= 0.f ? by0 : by1));
    const float v_hi = fmaf(c.vx, c.vx >= 0.f ? bx1 : bx0, c.vy * (c.vy >= 0.f ? by1 : by0));
    return !(v_hi + sv < c.v0 || v_lo - sv > c.v1);
}

// Is the box [bx0, bx1] x [by0, by1] (rounded outward) inside the inner
// window of an instance, projections' rounding included?  Then the exact
// test (inst_sees) accepts every query of the box.
__device__ __forceinline__ bool inner_sees(const InstCull &c, const InstF32 &f, float nx, float ny, float bx0,
                                           float bx1, float by0, float by1, float wmag)
{
    if (bx0 < f.x0 || bx1 > f.x1 || by0 < f.y0 || by1 > f.y1) return false;
    if (f.n0 > -INFINITY || f.n1 < INFINITY) {
        const float sn = 4e-7f * (fabsf(nx) + fabsf(ny)) * wmag;
        const float n_lo = fmaf(nx, nx >= 0.f ? bx0 : bx1, ny * (ny >= 0.f ? by0 : by1));
        const float n_hi = fmaf(nx, nx >= 0.f ? bx1 : bx0, ny * (ny >= 0.f ? by1 : by0));
        if (n_lo - sn < f.n0 || n_hi + sn > f.n1) return false;
    }
    if (f.v0 > -INFINITY || f.v1 < INFINITY) {
        const float sv = 4e-7f * (fabsf(c.vx) + fabsf(c.vy)) * wmag;
        const float v_lo = fmaf(c.vx, c.vx >= 0.f ? bx0 : bx1, c.vy * (c.vy >= 0.f ? by0 : by1));
        const float v_hi = fmaf(c.vx, c.vx >= 0.f ? bx1 : bx0, c.vy * (c.vy >= 0.f ? by1 : by0));
        if (v_lo - sv < f.v0 || v_hi + sv > f.v1) return false;
    }
    return true;
}

// Line term sign in FP32 for the query (xr, yr) (the reduced point within
// 2^-23 relative): +1 / -1 when the cross product clears its error band
// (the coordinates' and the line data's rounding, four times over), 0 when
// only the exact test (line_side) can decide.
__device__ __forceinline__ int line_side_f32(const InstF32 &f, float xr, float yr)
{
    const float dx = xr - f.lx, dy = yr - f.ly;
    const float cr = fmaf(f.lvx, dy, -f.lvy * dx);
    const float band = 4.76837158203125e-7f *      // 2^-21
                       (fabsf(f.lvx) * (fabsf(yr) + fabsf(f.ly)) + fabsf(f.lvy) * (fabsf(xr) + fabsf(f.lx)));
    return cr > band ? 1 : (cr < -band ? -1 : 0);
}

// Line term of Eq. 9 (+1 on the left of L, -1 on the right, 0 on L) for the
// family base point of a line instance.
__device__ __forceinline__ int line_side(const DomDev &D, const InstDev &in, const LoopDev &L,
                                         double x, double y)
{
    double xf = (D.Pu > 0) ? xsub(x, in.Fx) : x;
    double yf = (D.Pv > 0) ? xsub(y, in.Fy) : y;
    double cr = xsub(xmul(L.vx, xsub(yf, L.g0y)), xmul(L.vy, xsub(xf, L.g0x)));
    return cr > 0 ? 1 : (cr < 0 ? -1 : 0);
}

// ---------------------------------------------------------------- Bezier
// gamma(t) by repeated linear interpolation of the control points, unrolled
// for degrees up to NM (lanes with a lower degree n mask the extra steps).
template <typename T, int NM>
__device__ __forceinline__ void bez_eval_n(const T *cx, const T *cy, int n, T t, T &ox, T &oy)
{
    T qx[NM + 1], qy[NM + 1];
#pragma unroll
    for (int i = 0; i <= NM; i++) {
        qx[i] = cx[i];
        qy[i] = cy[i];
    }
    const T s = T(1) - t;
#pragma unroll
    for (int r = 1; r <= NM; r++) {
#pragma unroll
        for (int i = 0; i <= NM - r; i++) {
            if (i <= n - r) {
                qx[i] = s * qx[i] + t * qx[i + 1];
                qy[i] = s * qy[i] + t * qy[i + 1];
            }
        }
    }
    ox = qx[0];
    oy = qy[0];
}

// Dispatch on an upper bound of the degree (the domain's largest degree,
// the same for every lane that works on one domain).
template <typename T>
__device__ __forceinline__ void bez_eval(const T *cx, const T *cy, int n, int nmax, T t, T &ox, T &oy)
{
    switch (nmax) {
    case 1: bez_eval_n<T, 1>(cx, cy, n, t, ox, oy); break;
    case 2: bez_eval_n<T, 2>(cx, cy, n, t, ox, oy); break;
    case 3: bez_eval_n<T, 3>(cx, cy, n, t, ox, oy); break;
    case 4: bez_eval_n<T, 4>(cx, cy, n, t, ox, oy); break;
    case 5: bez_eval_n<T, 5>(cx, cy, n, t, ox, oy); break;
    case 6: bez_eval_n<T, 6>(cx, cy, n, t, ox, oy); break;
    default: bez_eval_n<T, kMaxDeg>(cx, cy, n, t, ox, oy); break;
    }
}

// A rational segment: de Casteljau on the homogeneous control points
// (w x, w y, w) -- the curve is their central projection -- then the
// division by the weight coordinate.
template <typename T, int NM>
__device__ __forceinline__ void bez_eval_h_n(const T *hx, const T *hy, const T *hw, int n, T t, T &ox, T &oy)
{
    T qx[NM + 1], qy[NM + 1], qw[NM + 1];
#pragma unroll
    for (int i = 0; i <= NM; i++) {
        qx[i] = hx[i];
        qy[i] = hy[i];
        qw[i] = i <= n ? hw[i] : T(1);     // hw may point into a longer array
    }
    const T s = T(1) - t;
#pragma unroll
    for (int r = 1; r <= NM; r++) {
#pragma unroll
        for (int i = 0; i <= NM - r; i++) {
            if (i <= n - r) {
                qx[i] = s * qx[i] + t * qx[i + 1];
                qy[i] = s * qy[i] + t * qy[i + 1];
                qw[i] = s * qw[i] + t * qw[i + 1];
            }
        }
    }
    const T r = T(1) / qw[0];          // one division per point
    ox = qx[0] * r;
    oy = qy[0] * r;
}

template <typename T>
__device__ __forceinline__ void bez_eval_h(const T *hx, const T *hy, const T *hw, int n, int nmax, T t, T &ox,
                                           T &oy)
{
    switch (nmax) {
    case 1: bez_eval_h_n<T, 1>(hx, hy, hw, n, t, ox, oy); break;
    case 2: bez_eval_h_n<T, 2>(hx, hy, hw, n, t, ox, oy); break;
    case 3: bez_eval_h_n<T, 3>(hx, hy, hw, n, t, ox, oy); break;
    case 4: bez_eval_h_n<T, 4>(hx, hy, hw, n, t, ox, oy); break;
    case 5: bez_eval_h_n<T, 5>(hx, hy, hw, n, t, ox, oy); break;
    case 6: bez_eval_h_n<T, 6>(hx, hy, hw, n, t, ox, oy); break;
    default: bez_eval_h_n<T, kMaxDeg>(hx, hy, hw, n, t, ox, oy); break;
    }
}

// Control points of one segment for the FP64 recursions: plain, or
// homogeneous (w x, w y, w) when Wt (its weights) is not null.
struct SegF64 {
    double cx[kNcp], cy[kNcp], cw[kNcp];
    int n, nmax;
    bool rat;
    __device__ __forceinline__ void load(const double *P, const double *Wt, int n_, int nmax_)
    {
        n = n_;
        nmax = nmax_;
        rat = Wt != nullptr;
#pragma unroll
        for (int i = 0; i < kNcp; i++) {
            const double w = (rat && i <= n) ? Wt[i] : 1.0;
            cx[i] = (i <= n) ? w * P[2 * i] : 0.0;
            cy[i] = (i <= n) ? w * P[2 * i + 1] : 0.0;
            cw[i] = w;
        }
    }
    __device__ __forceinline__ void eval(double t, double &x, double &y) const
    {
        if (rat) bez_eval_h<double>(cx, cy, cw, n, nmax, t, x, y);
        else bez_eval<double>(cx, cy, n, nmax, t, x, y);
    }
};

// Weights of segment s, or null when it is polynomial.
__device__ __forceinline__ const double *seg_weights(const DomDev &D, int s)
{
    if (!D.w) return nullptr;
    const int4 si = D.seg_info[s];
    return si.w ? D.w + si.x : nullptr;
}

// Bounds of |gamma'| on the eighths of a rational segment, or null
__device__ __forceinline__ const double *seg_bsub(const DomDev &D, int s)
{
    return D.seg_bsub ? D.seg_bsub + 8 * (size_t)s : nullptr;
}

// ---------------------------------------------------------------- Alg. 1, FP64
// Far actions of Algorithm 1: the chord of an excluded sub-segment either adds
// its signed angle (Eq. 3, the plain method) or its signed crossing of the
// +x ray from p (the exact reformulation used by the mixed path).
struct FarAngle {
    double ang = 0.0;
    __device__ __forceinline__ void chord(double ax, double ay, double bx, double by)
    {
        ang += atan2(ax * by - ay * bx, ax * bx + ay * by);
    }
};

struct FarCross {
    int cnt = 0;
    __device__ __forceinline__ void chord(double ax, double ay, double bx, double by)
    {
        bool sa = ay > 0.0, sb = by > 0.0;
        if (sa != sb) {
            double d = ax * by - ay * bx;
            if (!sa && sb && d > 0) cnt++;
            else if (sa && !sb && d < 0) cnt--;
        }
    }
};

// Algorithm 1 over [0,1] of one segment, query (px,py), in FP64.  Points are
// handled relative to p after evaluation in absolute coordinates.  Returns
// WALK_BOUNDARY when an evaluated point is closer than eps, WALK_DEPTH at the
// depth cap (both mean the query is on the boundary), else WALK_DONE.
template <class Far>
__device__ int alg1_fp64(const double *P, const double *Wt, int n, int nmax, double B, double px, double py,
                          double eps, Far &far)
{
    SegF64 sg;              // loaded at the first evaluation: most segments are far at the root
    bool loaded = false;
    double st_t[kDepthCap64 + 2], st_x[kDepthCap64 + 2], st_y[kDepthCap64 + 2];
    int st_d[kDepthCap64 + 2];
    double a = 0.0;
    double ax = P[0] - px, ay = P[1] - py;
    double ra = sqrt(ax * ax + ay * ay);
    int sp = 0;
    {
        double bx = P[2 * n] - px, by = P[2 * n + 1] - py;
        st_t[0] = 1.0; st_x[0] = bx; st_y[0] = by; st_d[0] = 0;
        sp = 1;
    }
    while (sp > 0) {
        double b = st_t[sp - 1], bx = st_x[sp - 1], by = st_y[sp - 1];
        int d = st_d[sp - 1];
        double rb = sqrt(bx * bx + by * by);
        if (ra < eps || rb < eps) return WALK_BOUNDARY;
        if (ra + rb > B * (b - a)) {
            far.chord(ax, ay, bx, by);
            a = b; ax = bx; ay = by; ra = rb;
            sp--;
            continue;
        }
        if (d >= kDepthCap64) return WALK_DEPTH;
        if (!loaded) {
            sg.load(P, Wt, n, nmax);
            loaded = true;
        }
        double m = 0.5 * (a + b), mx, my;
        sg.eval(m, mx, my);
        st_d[sp - 1] = d + 1;
        st_t[sp] = m; st_x[sp] = mx - px; st_y[sp] = my - py; st_d[sp] = d + 1;
        sp++;
    }
    return WALK_DONE;
}

// The eighth [j/8, (j+1)/8] of the parameter interval that holds a node:
// j = floor(8 a) for its start a in [0, 1) and ceil(8 b) - 1 for its end b
// in (0, 1]; the node lies in one eighth iff the two agree.  From the bits
// (a, b >= 0 are dyadic node ends), so no conversion instructions.
__device__ __forceinline__ int eighth_lo(float a)
{
    const uint32_t u = __float_as_uint(a);
    const int e = (int)(u >> 23) - 127;                 // a = 1.m 2^e
    if (e < -3) return 0;
    return (int)(((u & 0x7fffffu) | 0x800000u) >> (20 - e));
}
__device__ __forceinline__ int eighth_hi(float b)
{
    const uint32_t u = __float_as_uint(b);
    const int e = (int)(u >> 23) - 127;
    if (e < -3) return 0;
    const uint32_t m = (u & 0x7fffffu) | 0x800000u;
    const int sh = 20 - e;
    return (int)(m >> sh) - ((m & ((1u << sh) - 1u)) == 0u ? 1 : 0);
}
__device__ __forceinline__ int eighth_lo(double a)
{
    const uint32_t hi = (uint32_t)__double2hiint(a);
    const int e = (int)(hi >> 20) - 1023;
    if (e < -3) return 0;
    return (int)(((hi & 0xfffffu) | 0x100000u) >> (17 - e));
}
__device__ __forceinline__ int eighth_hi(double b)
{
    const uint32_t hi = (uint32_t)__double2hiint(b), lo = (uint32_t)__double2loint(b);
    const int e = (int)(hi >> 20) - 1023;
    if (e < -3) return 0;
    const uint32_t m = (hi & 0xfffffu) | 0x100000u;
    const int sh = 17 - e;
    return (int)(m >> sh) - (((m & ((1u << sh) - 1u)) | lo) == 0u ? 1 : 0);
}

// Algorithm 1 in FP64 on the sub-interval [a0, b0] of a polynomial segment
// of degree n <= NM, adding the signed crossings of the +x ray from (px, py)
// by its chords; the end points take the given signs (those of the FP32
// chain around it).  Returns true when the query is on the boundary.
//
// FP64 is the slow unit here, so every node is cheap in FP64 operations:
//   gamma(t) - p by Horner's rule in the power basis of the query-relative
//     control points q_i = P_i - p: gamma(t) - p = sum_k C(n,k) D^k q_0 t^k,
//     D^k the k-th forward difference (2n FMAs per point);
//   the eps test on squared distances, |q|^2 < eps^2;
//   the far test of Eq. 5, ra + rb > L with L = B (b - a), without square
//     roots: with S = L^2 - ra^2 - rb^2 it holds iff S < 0 or
//     4 ra^2 rb^2 > S^2 (both sides of ra + rb > L are non-negative).
// Each decision is the exact one up to FP64 rounding of its operands.
template <int NM>
__device__ __noinline__ int alg1_fp64_sub_pow(const double *P, int n, double B, double px, double py,
                                                  double eps, double a0, double b0, bool sa0, bool sb0, int &cnt)
{
    double cx[NM + 1], cy[NM + 1];
#pragma unroll
    for (int i = 0; i <= NM; i++) {
        cx[i] = i <= n ? P[2 * i] - px : 0.0;
        cy[i] = i <= n ? P[2 * i + 1] - py : 0.0;
    }
#pragma unroll
    for (int k = 1; k <= NM; k++) {
#pragma unroll
        for (int i = NM; i >= k; i--) {
            if (i <= n) {
                cx[i] -= cx[i - 1];
                cy[i] -= cy[i - 1];
            }
        }
    }
    double bin = 1.0;
#pragma unroll
    for (int k = 1; k <= NM; k++) {
        if (k <= n) {
            bin = bin * (double)(n - k + 1) / (double)k;     // C(n, k), exact
            cx[k] *= bin;
            cy[k] *= bin;
        }
    }
    auto eval = [&](double t, double &x, double &y) {
        x = cx[NM];
        y = cy[NM];
#pragma unroll
        for (int k = NM - 1; k >= 0; k--) {
            x = fma(x, t, cx[k]);
            y = fma(y, t, cy[k]);
        }
    };
    const double eps2 = eps * eps;
    double st_t[kDepthCap64 + 2], st_x[kDepthCap64 + 2], st_y[kDepthCap64 + 2];
    int st_d[kDepthCap64 + 2];
    double ax, ay, bx, by;
    if (a0 == 0.0) { ax = P[0] - px; ay = P[1] - py; }
    else eval(a0, ax, ay);
    if (b0 == 1.0) { bx = P[2 * n] - px; by = P[2 * n + 1] - py; }
    else eval(b0, bx, by);
    double a = a0;
    bool sa = sa0;
    double qa = ax * ax + ay * ay;
    int d0 = 0;
    for (double w = b0 - a0; w < 1.0 && d0 < kDepthCap64; w *= 2.0) d0++;
    st_t[0] = b0; st_x[0] = bx; st_y[0] = by; st_d[0] = d0;
    int sp = 1;
    cnt = 0;
    while (sp > 0) {
        const double b = st_t[sp - 1];
        bx = st_x[sp - 1];
        by = st_y[sp - 1];
        const int d = st_d[sp - 1];
        const double qb = bx * bx + by * by;
        if (qa < eps2 || qb < eps2) return WALK_BOUNDARY;
        const bool sb = (b == b0) ? sb0 : (by > 0.0);
        const double L = B * (b - a);
        const double S = L * L - (qa + qb);
        if (S < 0.0 || 4.0 * qa * qb > S * S) {
            if (sa != sb) {
                const double D = ax * by - ay * bx;
                if (!sa && sb && D > 0) cnt++;
                else if (sa && !sb && D < 0) cnt--;
            }
            a = b; ax = bx; ay = by; qa = qb; sa = sb;
            sp--;
            continue;
        }
        if (d >= kDepthCap64) return WALK_DEPTH;
        const double m = 0.5 * (a + b);
        double mx, my;
        eval(m, mx, my);
        st_d[sp - 1] = d + 1;
        st_t[sp] = m; st_x[sp] = mx; st_y[sp] = my; st_d[sp] = d + 1;
        sp++;
    }
    return WALK_DONE;
}

// The same walk for a rational segment (weights w_i > 0): gamma(t) - p =
// Q(t) / W(t) with the homogeneous query-relative control points
// w_i (P_i - p) and weights w_i, each of Q_x, Q_y, W by Horner's rule in its
// power basis.  Since W > 0, signs and cross products take Q alone, and the
// eps and far tests are those of the polynomial walk multiplied through by
// the squared weights (|Q|^2 = |gamma - p|^2 W^2), so no node divides.
//
// A rational segment's bound B (App. A.1) grows with its weight ratio
// (about 2 / w for a circular arc of weights (1, w, 1)), and the walk's
// node count with it.  With bsub (the segment's bounds on its eighths, or
// null), a node inside one eighth is also far when ra + rb > Bj (b - a) + 2 eps
// holds for that eighth's bound Bj: the sub-curve then lies in the smaller
// ellipse, so the chord's crossings are the curve's, and every one of its
// points is more than eps from the query (|q - c| >= (ra + rb - Bj (b - a)) / 2
// for c in that ellipse), so the eps test of the walk with B alone would not
// have fired inside the node either.
template <int NM>
__device__ __noinline__ int alg1_fp64_sub_rpow(const double *P, const double *Wt, int n, double B, double px,
                                                double py, double eps, double a0, double b0, bool sa0, bool sb0,
                                                const double *bsub, int &cnt)
{
    double cx[NM + 1], cy[NM + 1], cw[NM + 1];
#pragma unroll
    for (int i = 0; i <= NM; i++) {
        const double w = i <= n ? Wt[i] : 0.0;
        cx[i] = i <= n ? w * (P[2 * i] - px) : 0.0;
        cy[i] = i <= n ? w * (P[2 * i + 1] - py) : 0.0;
        cw[i] = w;
    }
#pragma unroll
    for (int k = 1; k <= NM; k++) {
#pragma unroll
        for (int i = NM; i >= k; i--) {
            if (i <= n) {
                cx[i] -= cx[i - 1];
                cy[i] -= cy[i - 1];
                cw[i] -= cw[i - 1];
            }
        }
    }
    double bin = 1.0;
#pragma unroll
    for (int k = 1; k <= NM; k++) {
        if (k <= n) {
            bin = bin * (double)(n - k + 1) / (double)k;
            cx[k] *= bin;
            cy[k] *= bin;
            cw[k] *= bin;
        }
    }
    auto eval = [&](double t, double &x, double &y, double &w) {
        x = cx[NM];
        y = cy[NM];
        w = cw[NM];
#pragma unroll
        for (int k = NM - 1; k >= 0; k--) {
            x = fma(x, t, cx[k]);
            y = fma(y, t, cy[k]);
            w = fma(w, t, cw[k]);
        }
    };
    const double eps2 = eps * eps;
    double st_t[kDepthCap64 + 2], st_x[kDepthCap64 + 2], st_y[kDepthCap64 + 2], st_w[kDepthCap64 + 2];
    int st_d[kDepthCap64 + 2];
    double ax, ay, aw, bx, by, bw;
    if (a0 == 0.0) { aw = Wt[0]; ax = aw * (P[0] - px); ay = aw * (P[1] - py); }
    else eval(a0, ax, ay, aw);
    if (b0 == 1.0) { bw = Wt[n]; bx = bw * (P[2 * n] - px); by = bw * (P[2 * n + 1] - py); }
    else eval(b0, bx, by, bw);
    double a = a0;
    bool sa = sa0;
    double na = ax * ax + ay * ay, wa2 = aw * aw;
    int d0 = 0;
    for (double w = b0 - a0; w < 1.0 && d0 < kDepthCap64; w *= 2.0) d0++;
    st_t[0] = b0; st_x[0] = bx; st_y[0] = by; st_w[0] = bw; st_d[0] = d0;
    int sp = 1;
    cnt = 0;
    while (sp > 0) {
        const double b = st_t[sp - 1];
        bx = st_x[sp - 1];
        by = st_y[sp - 1];
        bw = st_w[sp - 1];
        const int d = st_d[sp - 1];
        const double nb = bx * bx + by * by, wb2 = bw * bw;
        if (na < eps2 * wa2 || nb < eps2 * wb2) return WALK_BOUNDARY;
        const bool sb = (b == b0) ? sb0 : (by > 0.0);
        double L = B * (b - a);
        if (bsub) {
            const int j = eighth_lo(a);
            if (j == eighth_hi(b)) L = fmin(L, fma(__ldg(bsub + j), b - a, 2.0 * eps));
        }
        const double S = L * L * wa2 * wb2 - (na * wb2 + nb * wa2);
        if (S < 0.0 || 4.0 * na * nb * wa2 * wb2 > S * S) {
            if (sa != sb) {
                const double D = ax * by - ay * bx;
                if (!sa && sb && D > 0) cnt++;
                else if (sa && !sb && D < 0) cnt--;
            }
            a = b; ax = bx; ay = by; na = nb; wa2 = wb2; sa = sb;
            sp--;
            continue;
        }
        if (d >= kDepthCap64) return WALK_DEPTH;
        const double m = 0.5 * (a + b);
        double mx, my, mw;
        eval(m, mx, my, mw);
        st_d[sp - 1] = d + 1;
        st_t[sp] = m; st_x[sp] = mx; st_y[sp] = my; st_w[sp] = mw; st_d[sp] = d + 1;
        sp++;
    }
    return WALK_DONE;
}

// Algorithm 1 in FP64 on the sub-interval [a0, b0] of one segment, adding
// the signed crossings of the +x ray from (px, py) by its chords; the end
// points take the given signs (those of the FP32 chain around it).  bsub:
// the segment's bounds on its eighths (rational segments), or null.
// Returns WALK_DONE, or WALK_BOUNDARY / WALK_DEPTH when the query is on the
// boundary.
__device__ inline int alg1_fp64_sub(const double *P, const double *Wt, int n, int nmax, double B, double px,
                                     double py, double eps, double a0, double b0, bool sa0, bool sb0,
                                     const double *bsub, int &cnt)
{
    if (!Wt) {
        switch (nmax) {
        case 1: return alg1_fp64_sub_pow<1>(P, n, B, px, py, eps, a0, b0, sa0, sb0, cnt);
        case 2: return alg1_fp64_sub_pow<2>(P, n, B, px, py, eps, a0, b0, sa0, sb0, cnt);
        case 3: return alg1_fp64_sub_pow<3>(P, n, B, px, py, eps, a0, b0, sa0, sb0, cnt);
        case 4: return alg1_fp64_sub_pow<4>(P, n, B, px, py, eps, a0, b0, sa0, sb0, cnt);
        case 5: return alg1_fp64_sub_pow<5>(P, n, B, px, py, eps, a0, b0, sa0, sb0, cnt);
        case 6: return alg1_fp64_sub_pow<6>(P, n, B, px, py, eps, a0, b0, sa0, sb0, cnt);
        default: return alg1_fp64_sub_pow<kMaxDeg>(P, n, B, px, py, eps, a0, b0, sa0, sb0, cnt);
        }
    }
    switch (nmax) {
    case 1: return alg1_fp64_sub_rpow<1>(P, Wt, n, B, px, py, eps, a0, b0, sa0, sb0, bsub, cnt);
    case 2: return alg1_fp64_sub_rpow<2>(P, Wt, n, B, px, py, eps, a0, b0, sa0, sb0, bsub, cnt);
    case 3: return alg1_fp64_sub_rpow<3>(P, Wt, n, B, px, py, eps, a0, b0, sa0, sb0, bsub, cnt);
    case 4: return alg1_fp64_sub_rpow<4>(P, Wt, n, B, px, py, eps, a0, b0, sa0, sb0, bsub, cnt);
    case 5: return alg1_fp64_sub_rpow<5>(P, Wt, n, B, px, py, eps, a0, b0, sa0, sb0, bsub, cnt);
    case 6: return alg1_fp64_sub_rpow<6>(P, Wt, n, B, px, py, eps, a0, b0, sa0, sb0, bsub, cnt);
    default: return alg1_fp64_sub_rpow<kMaxDeg>(P, Wt, n, B, px, py, eps, a0, b0, sa0, sb0, bsub, cnt);
    }
}

}  // namespace wn
