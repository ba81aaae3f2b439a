// wn_domain.cu -- building a domain: validation, lifting to the covering
// space, loop classes, pairing, and the instance / record tables the query
// kernels sweep.
//
//   lifting (Sec. 4.3): every segment after the first of a loop is translated
//     by the lattice vector (I Pu, J Pv), I = round((e.x - s.x) / Pu), that
//     brings its start s nearest to the previous segment's lifted end e;
//     homology = round((end - start) / period) per periodic axis.
//   classes (Prop. 1): planar / contractible / extended; on a torus the
//     extended loops must be +-(p, q) with gcd(p, q) = 1 and |A| = |B|; on a
//     cylinder |homology| <= 1.
//   families (Prop. 2): index c = p j - q i, represented by c (i0, j0) with
//     p j0 - q i0 = 1 (i0 in [0, |p|) for p != 0; i0 = -q, j0 = 0 for p = 0).
//   pairing (App. C, Alg. 8-10): for each alpha in input order, the copies
//     beta + w_c (c within 2 of the shift that brings beta's start within one
//     family spacing of alpha's) that lie left of alpha (PE(beta mid) > 0),
//     and among them the one left of all others in beta's orientation.  The
//     PE values come from a device kernel.
//   instances: for every lattice copy that some query of the base tile can
//     see -- contractible copies with the shifted query inside the control
//     point box (both axes on a torus, the periodic axis on a cylinder),
//     extended-curve copies k inside the slab of Eq. 9, the line term of every
//     extended curve (and family) -- one InstDev; queries test the exact
//     window on the device.
//   records: per loop, one FP32 record per segment (chord endpoints, the
//     inflated circle that contains the ellipse of Lemma 1 and the eps discs,
//     the gap to the next vertex, and beside it the box of the segment's
//     control points in the chord's frame) plus, for an extended curve, the closing
//     chord gamma(0)+v -> gamma(0) that turns W(gamma) - omega(chord) of
//     Eq. 9 into a closed polygon.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "wn_internal.h"

namespace wn {

namespace {

struct HostLoop {
    int s0, s1;
    int hp = 0, hq = 0;
    int cls = 0;
    double v[2] = {0, 0}, g0[2] = {0, 0}, g0v[2] = {0, 0};
    double smin = 0, smax = 0, vv = 0;
    double box[4];
    double nlo = 0, nhi = 0;
};

struct DevBuf {
    std::vector<void *> *list;
    cudaError_t err = cudaSuccess;
    template <typename T>
    T *up(const std::vector<T> &v)
    {
        if (err != cudaSuccess) return nullptr;
        size_t bytes = std::max<size_t>(sizeof(T), v.size() * sizeof(T));
        void *p = nullptr;
        err = cudaMalloc(&p, bytes);
        if (err != cudaSuccess) return nullptr;
        list->push_back(p);
        if (!v.empty()) err = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        return static_cast<T *>(p);
    }
};

long long lround_ll(double x) { return (long long)std::llround(x); }

}  // namespace

// App. A.1's two bounds of |gamma'| for a rational segment of degree n
// (control points P, weights w > 0), the smaller of n (W/w) max |P_i - P_j|
// and n (W/w)^2 max |P_i - P_{i-1}|.
double rational_segment_bound(const double *P, const double *w, int n)
{
    double wmax = w[0], wmin = w[0];
    for (int i = 1; i <= n; i++) {
        wmax = std::fmax(wmax, w[i]);
        wmin = std::fmin(wmin, w[i]);
    }
    const double r = wmax / wmin;
    double dall = 0.0, dnext = 0.0;
    for (int i = 0; i <= n; i++)
        for (int j = i + 1; j <= n; j++) {
            const double dx = P[2 * j] - P[2 * i], dy = P[2 * j + 1] - P[2 * i + 1];
            const double d = std::sqrt(dx * dx + dy * dy);
            dall = std::fmax(dall, d);
            if (j == i + 1) dnext = std::fmax(dnext, d);
        }
    return std::fmin((double)n * r * dall, (double)n * r * r * dnext);
}

// App. A.1's bounds of |gamma'| on each eighth [j/8, (j+1)/8] of a rational
// segment of degree n (control points P, weights w > 0, segment bound B).
// An eighth is itself a rational Bezier curve of degree n, its homogeneous
// control points (w P, w) those of the segment's de Casteljau subdivision;
// App. A.1 bounds its speed in its own parameter, and 8 times that bounds
// |gamma'| there in the segment's parameter.  Near an arc's middle the
// eighths' weights vary far less than the segment's (an arc of weights
// (1, w, 1) has ratio 1 / w, its eighths ratios near 1), so their bounds are
// much smaller than B.  The subdivision's rounding is covered: the
// sub-curve's control points are convex combinations of the segment's, so
// each differs from the computed one by at most
// Delta = 32 n u R max|P| (R the segment's weight ratio, u = 2^-53), its
// weights by a relative 32 n u R; each distance is widened by 2 Delta and
// the ratio by that relative amount.  No result exceeds B.
void rational_eighth_bounds(const double *P, const double *w, int n, double B, double out[8])
{
    constexpr double u = 1.1102230246251565e-16;
    double wmax = w[0], wmin = w[0], Pm = 0.0;
    for (int i = 0; i <= n; i++) {
        wmax = std::fmax(wmax, w[i]);
        wmin = std::fmin(wmin, w[i]);
        Pm = std::fmax(Pm, std::fmax(std::fabs(P[2 * i]), std::fabs(P[2 * i + 1])));
    }
    const double rel = 32.0 * n * u * (wmax / wmin);
    const double Delta = rel * Pm;
    // de Casteljau at t: the left (keep_left) or right part of h
    auto split = [n](double (*h)[3], double t, bool keep_left) {
        double tmp[kMaxDeg + 1][3], part[kMaxDeg + 1][3];
        for (int i = 0; i <= n; i++)
            for (int c = 0; c < 3; c++) tmp[i][c] = h[i][c];
        for (int c = 0; c < 3; c++) {
            part[0][c] = tmp[0][c];
            part[n][c] = tmp[n][c];
        }
        for (int k = 1; k <= n; k++) {
            for (int i = 0; i <= n - k; i++)
                for (int c = 0; c < 3; c++) tmp[i][c] = (1.0 - t) * tmp[i][c] + t * tmp[i + 1][c];
            for (int c = 0; c < 3; c++) {
                if (keep_left) part[k][c] = tmp[0][c];
                else part[n - k][c] = tmp[n - k][c];
            }
        }
        for (int i = 0; i <= n; i++)
            for (int c = 0; c < 3; c++) h[i][c] = part[i][c];
    };
    for (int j = 0; j < 8; j++) {
        double h[kMaxDeg + 1][3];
        for (int i = 0; i <= n; i++) {
            h[i][0] = w[i] * P[2 * i];
            h[i][1] = w[i] * P[2 * i + 1];
            h[i][2] = w[i];
        }
        split(h, (j + 1) / 8.0, true);                       // [0, (j+1)/8]
        if (j > 0) split(h, (double)j / (double)(j + 1), false);     // then its part from j/8
        double smax = h[0][2], smin = h[0][2];
        double q[kMaxDeg + 1][2];
        for (int i = 0; i <= n; i++) {
            smax = std::fmax(smax, h[i][2]);
            smin = std::fmin(smin, h[i][2]);
            q[i][0] = h[i][0] / h[i][2];
            q[i][1] = h[i][1] / h[i][2];
        }
        const double r = (smax / smin) * (1.0 + rel) / (1.0 - rel);
        double dall = 0.0, dnext = 0.0;
        for (int i = 0; i <= n; i++)
            for (int k = i + 1; k <= n; k++) {
                const double d = std::hypot(q[k][0] - q[i][0], q[k][1] - q[i][1]);
                dall = std::fmax(dall, d);
                if (k == i + 1) dnext = std::fmax(dnext, d);
            }
        const double bj = std::fmin((double)n * r * (dall + 2.0 * Delta), (double)n * r * r * (dnext + 2.0 * Delta));
        out[j] = std::fmin(B, 8.0 * bj * (1.0 + 1e-12));
    }
}


int build_domain(const int32_t *loop_offsets, int32_t n_loops, const int32_t *degrees,
                 const double *cps, const double *weights, double Pu, double Pv, double eps,
                 wn_domain **out, std::string &err)
{
    *out = nullptr;
    if (n_loops < 0 || !loop_offsets || (n_loops > 0 && (!degrees || !cps))) {
        err = "null array or negative loop count";
        return 1;
    }
    if (!(Pu >= 0) || !(Pv >= 0) || !std::isfinite(Pu) || !std::isfinite(Pv) || std::isnan(eps)) {
        err = "periods must be finite and >= 0, epsilon not NaN";
        return 1;
    }
    if (loop_offsets[0] != 0) {
        err = "loop_offsets[0] must be 0";
        return 1;
    }
    for (int l = 0; l < n_loops; l++)
        if (loop_offsets[l + 1] < loop_offsets[l]) {
            err = "loop_offsets must be non-decreasing";
            return 1;
        }
    const int ns = loop_offsets[n_loops];
    std::vector<int> seg_cp(ns), seg_deg(ns);
    long long ncp = 0;
    for (int s = 0; s < ns; s++) {
        if (degrees[s] < 1 || degrees[s] > kMaxDeg) {
            err = "segment degree outside 1.." + std::to_string(kMaxDeg);
            return 1;
        }
        seg_deg[s] = degrees[s];
        seg_cp[s] = (int)ncp;
        ncp += degrees[s] + 1;
        if (ncp > (1LL << 30)) {
            err = "too many control points";
            return 5;
        }
    }
    std::vector<double> P(cps, cps + 2 * ncp);
    for (long long i = 0; i < 2 * ncp; i++)
        if (!std::isfinite(P[i])) {
            err = "control points must be finite";
            return 1;
        }
    // rational input: a segment whose weights are not all equal is rational
    // (equal weights give the polynomial curve); weights must be positive
    std::vector<double> Wt;
    std::vector<char> seg_rat(ns, 0);
    bool rational = false;
    if (weights) {
        Wt.assign(weights, weights + ncp);
        for (long long i = 0; i < ncp; i++)
            if (!(Wt[i] > 0) || !std::isfinite(Wt[i])) {
                err = "weights must be finite and > 0";
                return 1;
            }
        for (int s = 0; s < ns; s++)
            for (int i = 1; i <= seg_deg[s]; i++)
                if (Wt[seg_cp[s] + i] != Wt[seg_cp[s]]) seg_rat[s] = 1;
        for (int s = 0; s < ns; s++) rational |= seg_rat[s] != 0;
    }
    const int kind = (Pu > 0 && Pv > 0) ? DK_BI : (Pu > 0) ? DK_UNI_U : (Pv > 0) ? DK_UNI_V : DK_PLANAR;
    if (!(eps > 0)) {
        double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
        for (long long i = 0; i < ncp; i++) {
            x0 = std::fmin(x0, P[2 * i]); x1 = std::fmax(x1, P[2 * i]);
            y0 = std::fmin(y0, P[2 * i + 1]); y1 = std::fmax(y1, P[2 * i + 1]);
        }
        double S = std::fmax(Pu, Pv);
        if (ncp) S = std::fmax(S, std::fmax(x1 - x0, y1 - y0));
        eps = 1e-9 * S;
    }

    // ---- lifting and per-loop data
    std::vector<HostLoop> loops(n_loops);
    std::vector<double> segB(ns);
    for (int l = 0; l < n_loops; l++) {
        HostLoop &L = loops[l];
        L.s0 = loop_offsets[l];
        L.s1 = loop_offsets[l + 1];
        for (int s = L.s0 + 1; s < L.s1; s++) {
            const double *pe = &P[2 * (seg_cp[s - 1] + seg_deg[s - 1])];
            double *ps = &P[2 * seg_cp[s]];
            long long I = (Pu > 0) ? lround_ll((pe[0] - ps[0]) / Pu) : 0;
            long long J = (Pv > 0) ? lround_ll((pe[1] - ps[1]) / Pv) : 0;
            for (int i = 0; i <= seg_deg[s]; i++) {
                if (I) ps[2 * i] = ps[2 * i] + (double)I * Pu;
                if (J) ps[2 * i + 1] = ps[2 * i + 1] + (double)J * Pv;
            }
        }
        if (L.s1 > L.s0) {
            const double *f = &P[2 * seg_cp[L.s0]];
            const double *e = &P[2 * (seg_cp[L.s1 - 1] + seg_deg[L.s1 - 1])];
            if (Pu > 0) L.hp = (int)lround_ll((e[0] - f[0]) / Pu);
            if (Pv > 0) L.hq = (int)lround_ll((e[1] - f[1]) / Pv);
        }
        L.box[0] = L.box[2] = INFINITY;
        L.box[1] = L.box[3] = -INFINITY;
        for (int s = L.s0; s < L.s1; s++) {
            const double *q = &P[2 * seg_cp[s]];
            const int n = seg_deg[s];
            double B = 0.0;
            if (!seg_rat[s]) {
                // Lemma 1: the hodograph's control polygon, n |P_i - P_{i-1}|
                for (int i = 1; i <= n; i++) {
                    double dx = q[2 * i] - q[2 * i - 2], dy = q[2 * i + 1] - q[2 * i - 1];
                    double b = (double)n * std::sqrt(dx * dx + dy * dy);
                    if (b > B) B = b;
                }
            } else {
                // App. A.1 (rational): n (W/w) max |P_i - P_j| and
                // n (W/w)^2 max |P_i - P_{i-1}| both bound |gamma'|; the smaller
                B = rational_segment_bound(q, &Wt[seg_cp[s]], n);
            }
            segB[s] = B;
            for (int i = 0; i <= n; i++) {
                L.box[0] = std::fmin(L.box[0], q[2 * i]);
                L.box[1] = std::fmax(L.box[1], q[2 * i]);
                L.box[2] = std::fmin(L.box[2], q[2 * i + 1]);
                L.box[3] = std::fmax(L.box[3], q[2 * i + 1]);
            }
        }
        if (kind == DK_PLANAR) L.cls = 0;
        else if (L.hp == 0 && L.hq == 0) L.cls = 1;
        else L.cls = 2;
        if (L.cls == 2) {
            if (kind != DK_BI && (std::abs(L.hp) > 1 || std::abs(L.hq) > 1)) {
                err = "a loop winds more than once around the cylinder (Prop. 1)";
                return 2;
            }
            L.v[0] = (Pu > 0) ? (double)L.hp * Pu : 0.0;
            L.v[1] = (Pv > 0) ? (double)L.hq * Pv : 0.0;
            const double *f = &P[2 * seg_cp[L.s0]];
            L.g0[0] = f[0];
            L.g0[1] = f[1];
            L.g0v[0] = L.g0[0] + L.v[0];
            L.g0v[1] = L.g0[1] + L.v[1];
            L.vv = L.v[0] * L.v[0] + L.v[1] * L.v[1];
            L.smin = (L.g0v[0] * L.v[0] + L.g0v[1] * L.v[1]) / L.vv;
            L.smax = L.smin;
            for (int s = L.s0; s < L.s1; s++) {
                const double *q = &P[2 * seg_cp[s]];
                for (int i = 0; i <= seg_deg[s]; i++) {
                    double sv = (q[2 * i] * L.v[0] + q[2 * i + 1] * L.v[1]) / L.vv;
                    L.smin = std::fmin(L.smin, sv);
                    L.smax = std::fmax(L.smax, sv);
                }
            }
        }
    }

    // ---- bi-periodic classes and family generator
    int hp = 0, hq = 0;
    long long i0 = 0, j0 = 0;
    double nx = 0, ny = 0, PP = Pu * Pv;
    std::vector<int> A_idx, B_idx;
    if (kind == DK_BI) {
        int first = -1;
        for (int l = 0; l < n_loops; l++)
            if (loops[l].cls == 2) { first = l; break; }
        if (first >= 0) {
            hp = loops[first].hp;
            hq = loops[first].hq;
            long long a = std::llabs(hp), b = std::llabs(hq);
            while (b) { long long t = a % b; a = b; b = t; }
            if (a != 1) {
                err = "homology coefficients are not coprime (Prop. 1)";
                return 2;
            }
            for (int l = 0; l < n_loops; l++) {
                if (loops[l].cls != 2) continue;
                if (loops[l].hp == hp && loops[l].hq == hq) A_idx.push_back(l);
                else if (loops[l].hp == -hp && loops[l].hq == -hq) B_idx.push_back(l);
                else {
                    err = "non-contractible loops with different homology classes (Prop. 1)";
                    return 2;
                }
            }
            if (A_idx.size() != B_idx.size()) {
                err = "unequal numbers of (p,q) and -(p,q) loops (Prop. 1)";
                return 2;
            }
            if (hp == 0) { i0 = -hq; j0 = 0; }
            else {
                long long ap = std::llabs(hp);
                i0 = -1;
                for (long long i = 0; i < ap; i++)
                    if ((1 + (long long)hq * i) % hp == 0) { i0 = i; break; }
                j0 = (1 + (long long)hq * i0) / hp;
            }
            nx = -(double)hq * Pv;
            ny = (double)hp * Pu;
            for (int l : A_idx) {
                HostLoop &L = loops[l];
                L.nlo = INFINITY; L.nhi = -INFINITY;
                for (int s = L.s0; s < L.s1; s++) {
                    const double *q = &P[2 * seg_cp[s]];
                    for (int i = 0; i <= seg_deg[s]; i++) {
                        double nv = nx * q[2 * i] + ny * q[2 * i + 1];
                        L.nlo = std::fmin(L.nlo, nv);
                        L.nhi = std::fmax(L.nhi, nv);
                    }
                }
            }
        }
    }

    // ---- FP32 origin and scale over every vertex the records use
    double bx0 = INFINITY, bx1 = -INFINITY, by0 = INFINITY, by1 = -INFINITY;
    for (int l = 0; l < n_loops; l++) {
        const HostLoop &L = loops[l];
        if (L.s1 == L.s0) continue;
        bx0 = std::fmin(bx0, L.box[0]); bx1 = std::fmax(bx1, L.box[1]);
        by0 = std::fmin(by0, L.box[2]); by1 = std::fmax(by1, L.box[3]);
        if (L.cls == 2) {
            bx0 = std::fmin(bx0, L.g0v[0]); bx1 = std::fmax(bx1, L.g0v[0]);
            by0 = std::fmin(by0, L.g0v[1]); by1 = std::fmax(by1, L.g0v[1]);
        }
    }
    double ox = 0.0, oy = 0.0, M = 1.0;
    if (bx0 <= bx1) {
        ox = 0.5 * (bx0 + bx1);
        oy = 0.5 * (by0 + by1);
        M = std::fmax(std::fmax(bx1 - ox, ox - bx0), std::fmax(by1 - oy, oy - by0));
        if (!(M > 0)) M = 1.0;
        M = M * (1.0 + 1e-6);
    }
    const double Mq = 2.0 * M;
    const double Trec = std::ldexp(M + Mq, -22);

    // ---- records
    std::vector<float4> rec;
    std::vector<int> rec_seg;
    std::vector<double2> ra64, rb64, rn64;
    std::vector<int> loop_r0(n_loops), loop_r1(n_loops);
    auto f32 = [](double x) { return (float)x; };
    // per record, the box of its segment's control points in the chord's
    // frame: t = (P - a).(b - a), d = (P - a) x (b - a), widened by eps |b - a|
    // (and far beyond FP64 rounding) and rounded outward to FP32.  The curve
    // lies in the control points' hull, so a query outside the box is more
    // than eps from the curve and sees it under its chord's angle.
    std::vector<float4> robb;
    auto seg_box = [&](const double *a, const double *b, int seg) {
        if (seg < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
        const double ex = b[0] - a[0], ey = b[1] - a[1];
        double t0 = INFINITY, t1 = -INFINITY, d0 = INFINITY, d1 = -INFINITY;
        for (int i = 0; i <= seg_deg[seg]; i++) {
            const double px = P[2 * (seg_cp[seg] + i)] - a[0], py = P[2 * (seg_cp[seg] + i) + 1] - a[1];
            const double t = px * ex + py * ey, d = px * ey - py * ex;
            t0 = std::fmin(t0, t); t1 = std::fmax(t1, t);
            d0 = std::fmin(d0, d); d1 = std::fmax(d1, d);
        }
        const double el = std::sqrt(ex * ex + ey * ey);
        const double sl = eps * el * (1.0 + 1e-6) +
                          1e-12 * (std::fabs(t0) + std::fabs(t1) + std::fabs(d0) + std::fabs(d1) + el * el);
        return make_float4(std::nextafter((float)(t0 - sl), -INFINITY), std::nextafter((float)(t1 + sl), INFINITY),
                           std::nextafter((float)(d0 - sl), -INFINITY), std::nextafter((float)(d1 + sl), INFINITY));
    };
    auto push_rec = [&](const double *a, const double *b, const double *nxt, int seg, double B, bool chord) {
        float4 r0, r1, r2;
        r0.x = f32(a[0] - ox); r0.y = f32(a[1] - oy); r0.z = f32(b[0] - ox); r0.w = f32(b[1] - oy);
        const double cx = 0.5 * (a[0] + b[0]), cy = 0.5 * (a[1] + b[1]);
        const double R = (0.5 * B + eps) * (1.0 + std::ldexp(1.0, -20)) + 2.0 * Trec;
        const double gx = nxt[0] - b[0], gy = nxt[1] - b[1];
        uint32_t fl = (chord ? RF_CHORD : 0u) | ((gx != 0.0 || gy != 0.0) ? RF_GAP : 0u) |
                      ((seg >= 0 ? (uint32_t)seg : RF_NO_SEG) << RF_SEG_SHIFT);
        r1.x = f32(cx - ox); r1.y = f32(cy - oy); r1.z = f32(R * R * (1.0 + std::ldexp(1.0, -20)));
        uint32_t flb = fl;
        std::memcpy(&r1.w, &flb, 4);
        r2.x = f32(gx); r2.y = f32(gy); r2.z = f32(nxt[0] - ox); r2.w = f32(nxt[1] - oy);
        // low parts of the chord end and the next vertex: b - o = r0.zw + r3.xy and
        // n - o = r2.zw + r3.zw to ~2^-48 relative
        float4 r3;
        r3.x = f32((b[0] - ox) - (double)r0.z);
        r3.y = f32((b[1] - oy) - (double)r0.w);
        r3.z = f32((nxt[0] - ox) - (double)r2.z);
        r3.w = f32((nxt[1] - oy) - (double)r2.w);
        rec.push_back(r0); rec.push_back(r1); rec.push_back(r2); rec.push_back(r3);
        robb.push_back(seg_box(a, b, seg));
        rec_seg.push_back(seg);
        ra64.push_back(make_double2(a[0], a[1]));
        rb64.push_back(make_double2(b[0], b[1]));
        rn64.push_back(make_double2(nxt[0], nxt[1]));
    };
    for (int l = 0; l < n_loops; l++) {
        const HostLoop &L = loops[l];
        loop_r0[l] = (int)rec_seg.size();
        for (int s = L.s0; s < L.s1; s++) {
            const double *a = &P[2 * seg_cp[s]];
            const double *b = &P[2 * (seg_cp[s] + seg_deg[s])];
            const double *nxt;
            if (s + 1 < L.s1) nxt = &P[2 * seg_cp[s + 1]];
            else nxt = (L.cls == 2) ? L.g0v : &P[2 * seg_cp[L.s0]];
            push_rec(a, b, nxt, s, segB[s], false);
        }
        if (L.cls == 2 && L.s1 > L.s0) push_rec(L.g0v, L.g0, L.g0, -1, 0.0, true);
        loop_r1[l] = (int)rec_seg.size();
    }

    // ---- record tree: per loop, leaves of kCluRecs consecutive records and
    // internal nodes over kTreeArity consecutive children; every node covers a
    // contiguous record range and carries its near box, ray extent and the
    // expansion of its gap angles
    std::vector<float4> nodes;
    std::vector<int> loop_root(n_loops, -1);
    int all_root = -1;          // planar: root of the tree over all loops
    {
        auto dn = [](double x) { return std::nextafter((float)x, -INFINITY); };
        auto upf = [](double x) { return std::nextafter((float)x, INFINITY); };
        // one node over the records of `ranges`; a group node (several whole
        // loops, each a closed chain) has no chain ends: its crossings of a ray
        // that passes right of all its vertices cancel, so its end values are
        // +inf (both above every query)
        auto make_node_r = [&](const std::vector<std::pair<int, int>> &ranges, bool leaf, int first, int end,
                               bool group) {
            const int R0 = ranges.front().first, R1 = ranges.back().second;
            double nb[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
            double yr0 = INFINITY, yr1 = -INFINITY, xr1 = -INFINITY, xr0 = INFINITY;
            double gb[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
            bool gaps = false;
            for (const auto &rg : ranges)
            for (int r = rg.first; r < rg.second; r++) {
                const double2 a = ra64[r], b = rb64[r], n = rn64[r];
                for (const double2 &v : {a, b, n}) {
                    yr0 = std::fmin(yr0, v.y); yr1 = std::fmax(yr1, v.y);
                    xr1 = std::fmax(xr1, v.x); xr0 = std::fmin(xr0, v.x);
                }
                uint32_t fl;
                std::memcpy(&fl, &rec[4 * r + 1].w, 4);
                if (!(fl & RF_CHORD)) {
                    const int sg = rec_seg[r];
                    const double cx = 0.5 * (a.x + b.x), cy = 0.5 * (a.y + b.y);
                    const double R = (0.5 * segB[sg] + eps) * (1.0 + std::ldexp(1.0, -20)) + 4.0 * Trec;
                    nb[0] = std::fmin(nb[0], cx - R); nb[1] = std::fmax(nb[1], cx + R);
                    nb[2] = std::fmin(nb[2], cy - R); nb[3] = std::fmax(nb[3], cy + R);
                }
                if (fl & RF_GAP) {
                    gaps = true;
                    for (const double2 &v : {b, n}) {
                        gb[0] = std::fmin(gb[0], v.x); gb[1] = std::fmax(gb[1], v.x);
                        gb[2] = std::fmin(gb[2], v.y); gb[3] = std::fmax(gb[3], v.y);
                    }
                }
            }
            float4 c[kCluF4];
            std::memset(c, 0, sizeof c);
            if (nb[0] <= nb[1]) c[0] = make_float4(dn(nb[0] - ox), upf(nb[1] - ox), dn(nb[2] - oy), upf(nb[3] - oy));
            else c[0] = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);   // closing chords only
            c[1] = make_float4(dn(yr0 - oy), upf(yr1 - oy), upf(xr1 - ox), 0.f);
            double zx = 0, zy = 0, rc = 0;
            if (gaps) {
                zx = 0.5 * (gb[0] + gb[1]);
                zy = 0.5 * (gb[2] + gb[3]);
                double Cb = 0.0;
                for (const auto &rg : ranges)
                for (int r = rg.first; r < rg.second; r++) {
                    uint32_t fl;
                    std::memcpy(&fl, &rec[4 * r + 1].w, 4);
                    if (!(fl & RF_GAP)) continue;
                    rc = std::fmax(rc, std::hypot(rb64[r].x - zx, rb64[r].y - zy));
                    rc = std::fmax(rc, std::hypot(rn64[r].x - zx, rn64[r].y - zy));
                }
                rc = std::fmax(rc, 1e-300);
                // M_k = sum_gaps (n - z)^k - (b - z)^k ;  c_k = (-1)^(k+1) M_k / (k rc^k),
                // kept to kTail terms for the truncation bound
                constexpr int kTail = 96;
                double Mre[kTail + 1] = {}, Mim[kTail + 1] = {};
                for (const auto &rg : ranges)
                for (int r = rg.first; r < rg.second; r++) {
                    uint32_t fl;
                    std::memcpy(&fl, &rec[4 * r + 1].w, 4);
                    if (!(fl & RF_GAP)) continue;
                    Cb += std::hypot(rn64[r].x - rb64[r].x, rn64[r].y - rb64[r].y) / rc;
                    for (int side = 0; side < 2; side++) {
                        const double2 v = side ? rn64[r] : rb64[r];
                        const double sg = side ? 1.0 : -1.0;
                        const double ux = (v.x - zx) / rc, uy = (v.y - zy) / rc;
                        double pr = 1.0, pi = 0.0;
                        for (int k = 1; k <= kTail; k++) {
                            const double t = pr * ux - pi * uy;
                            pi = pr * uy + pi * ux;
                            pr = t;
                            Mre[k] += sg * pr;
                            Mim[k] += sg * pi;
                        }
                    }
                }
                for (int k = 1; k <= kCluTerms; k++) {
                    const double f = ((k & 1) ? 1.0 : -1.0) / (double)k;
                    float *dst = reinterpret_cast<float *>(&c[kCluCoef]) + 2 * (k - 1);
                    dst[0] = (float)(f * Mre[k]);
                    dst[1] = (float)(f * Mim[k]);
                }
                // Truncation after K terms at |w| = m: the next coefficients as
                // computed, then C >= |c_k| for every k (each gap adds at most
                // |g| / r_c) beyond kTail:
                //   sum_{K<k<=kTail} |c_k| m^k + C m^(kTail+1) / (1 - m).
                // The largest m with that <= tol, by bisection (it grows with m).
                double cabs[kTail + 1];
                for (int k = 1; k <= kTail; k++) cabs[k] = std::hypot(Mre[k], Mim[k]) / (double)k;
                auto tail = [&](int K, double m) {
                    double t = Cb * std::pow(m, kTail + 1) / (1.0 - m), mk = std::pow(m, K + 1);
                    for (int k = K + 1; k <= kTail; k++, mk *= m) t += cabs[k] * mk;
                    return t;
                };
                auto dist2 = [&](int K) {
                    double lo = 0.0, hi = 0.999;
                    for (int it = 0; it < 60; it++) {
                        const double m = 0.5 * (lo + hi);
                        if (tail(K, m) <= kCluTol) lo = m;
                        else hi = m;
                    }
                    const double d = lo > 0 ? rc / lo : INFINITY;
                    return upf(d * d * (1.0 + 1e-6));
                };
                c[1].w = dist2(kCluTerms);
                c[4] = make_float4(dist2(4), dist2(8), dist2(12), dist2(16));
                c[5] = make_float4(dist2(20), dist2(24), dist2(28), dist2(kCluTerms));
            }
            const float zxh = (float)(zx - ox), zyh = (float)(zy - oy);
            c[2] = make_float4(zxh, zyh, (float)((zx - ox) - (double)zxh), (float)((zy - oy) - (double)zyh));
            const int flags = (gaps ? 1 : 0) | (leaf ? 2 : 0);
            float ff, f0, f1;
            std::memcpy(&ff, &flags, 4);
            std::memcpy(&f0, &first, 4);
            std::memcpy(&f1, &end, 4);
            c[3] = make_float4((float)rc, ff, f0, f1);
            // the chain's start (record R0's a) and end (record R1-1's next
            // vertex): the same FP32 values the records hold
            float rb0, rb1;
            std::memcpy(&rb0, &R0, 4);
            std::memcpy(&rb1, &R1, 4);
            if (group) c[6] = make_float4(dn(xr0 - ox), INFINITY, INFINITY, 0.f);
            else c[6] = make_float4(dn(xr0 - ox), rec[4 * R0].y, rec[4 * (R1 - 1) + 2].w, rb0);
            c[7] = make_float4(rb1, 0.f, 0.f, 0.f);
            const int id = (int)(nodes.size() / kCluF4);
            for (int i = 0; i < kCluF4; i++) nodes.push_back(c[i]);
            return id;
        };
        auto make_node = [&](int R0, int R1, bool leaf, int first, int end) {
            return make_node_r({{R0, R1}}, leaf, first, end, false);
        };
        int max_depth = 0;
        for (int l = 0; l < n_loops; l++) {
            if (loop_r1[l] == loop_r0[l]) continue;
            std::vector<int> level, lr0, lr1;       // node ids and their record ranges
            for (int r0 = loop_r0[l]; r0 < loop_r1[l]; r0 += kCluRecs) {
                const int r1 = std::min(r0 + kCluRecs, loop_r1[l]);
                level.push_back(make_node(r0, r1, true, r0, r1));
                lr0.push_back(r0);
                lr1.push_back(r1);
            }
            int depth = 1;
            while (level.size() > 1) {
                depth++;
                std::vector<int> up_level, u0, u1;
                for (size_t i = 0; i < level.size(); i += kTreeArity) {
                    const size_t j = std::min(level.size(), i + kTreeArity);
                    up_level.push_back(make_node(lr0[i], lr1[j - 1], false, level[i], level[j - 1] + 1));
                    u0.push_back(lr0[i]);
                    u1.push_back(lr1[j - 1]);
                }
                level.swap(up_level);
                lr0.swap(u0);
                lr1.swap(u1);
            }
            loop_root[l] = level[0];
            max_depth = std::max(max_depth, depth);
        }
        // planar domains: a tree over the loops themselves, so that a query
        // far from a group of loops (holes, islands) tests the group once.
        // Loops in Morton order of their box centres; the loop roots are
        // copied into one contiguous run to serve as the first level.
        std::vector<int> live;
        for (int l = 0; l < n_loops; l++)
            if (loop_root[l] >= 0) live.push_back(l);
        int group_levels = 0;
        for (size_t m = live.size(); m > 1; m = (m + kTreeArity - 1) / kTreeArity) group_levels++;
        if (kind == DK_PLANAR && live.size() == 1) {
            all_root = loop_root[live[0]];
        } else if (kind == DK_PLANAR && live.size() > 1 && max_depth + group_levels <= kTreeMaxLevels) {
            auto morton = [&](int l) {
                const HostLoop &L = loops[l];
                const double cx = 0.5 * (L.box[0] + L.box[1]), cy = 0.5 * (L.box[2] + L.box[3]);
                const double w = std::fmax(bx1 - bx0, 1e-300), h = std::fmax(by1 - by0, 1e-300);
                const uint32_t ix = (uint32_t)std::fmin(65535.0, std::fmax(0.0, (cx - bx0) / w * 65536.0));
                const uint32_t iy = (uint32_t)std::fmin(65535.0, std::fmax(0.0, (cy - by0) / h * 65536.0));
                uint64_t code = 0;
                for (int bit = 0; bit < 16; bit++)
                    code |= (uint64_t)((ix >> bit) & 1u) << (2 * bit) | (uint64_t)((iy >> bit) & 1u) << (2 * bit + 1);
                return code;
            };
            std::vector<uint64_t> key(n_loops, 0);
            for (int l : live) key[l] = morton(l);
            std::stable_sort(live.begin(), live.end(), [&](int x, int y) { return key[x] < key[y]; });
            std::vector<int> level;
            std::vector<std::vector<std::pair<int, int>>> lrng;
            for (int l : live) {
                const int id = (int)(nodes.size() / kCluF4);
                for (int i = 0; i < kCluF4; i++) nodes.push_back(nodes[(size_t)kCluF4 * loop_root[l] + i]);
                level.push_back(id);
                lrng.push_back({{loop_r0[l], loop_r1[l]}});
            }
            while (level.size() > 1) {
                std::vector<int> up_level;
                std::vector<std::vector<std::pair<int, int>>> urng;
                for (size_t i = 0; i < level.size(); i += kTreeArity) {
                    const size_t j = std::min(level.size(), i + kTreeArity);
                    std::vector<std::pair<int, int>> rg;
                    for (size_t t = i; t < j; t++) rg.insert(rg.end(), lrng[t].begin(), lrng[t].end());
                    up_level.push_back(make_node_r(rg, false, level[i], level[j - 1] + 1, true));
                    urng.push_back(rg);
                }
                level.swap(up_level);
                lrng.swap(urng);
            }
            all_root = level[0];
        }
    }

    // ---- device upload of the geometry (pairing needs it)
    wn_domain *D = new wn_domain();
    cudaGetDevice(&D->device);
    DevBuf up{&D->allocs};
    auto fail = [&](int code, const std::string &msg) {
        for (void *p : D->allocs) cudaFree(p);
        delete D;
        err = msg;
        return code;
    };
    std::vector<LoopDev> hl(n_loops);
    for (int l = 0; l < n_loops; l++) {
        const HostLoop &L = loops[l];
        LoopDev &o = hl[l];
        std::memset(&o, 0, sizeof o);
        o.s0 = L.s0; o.s1 = L.s1; o.r0 = loop_r0[l]; o.r1 = loop_r1[l];
        o.hp = L.hp; o.hq = L.hq; o.cls = L.cls;
        o.vx = L.v[0]; o.vy = L.v[1]; o.g0x = L.g0[0]; o.g0y = L.g0[1];
        o.g0vx = L.g0v[0]; o.g0vy = L.g0v[1];
        o.smin = L.smin; o.smax = L.smax; o.vv = L.vv;
        for (int i = 0; i < 4; i++) o.box[i] = L.box[i];
        o.nlo = L.nlo; o.nhi = L.nhi;
        o.root = loop_root[l];
    }
    DomDev &dv = D->dev;
    std::memset(&dv, 0, sizeof dv);
    dv.kind = kind; dv.n_loops = n_loops; dv.n_segs = ns; dv.total_cp = (int)ncp;
    dv.max_deg = 1;
    for (int sgi = 0; sgi < ns; sgi++) dv.max_deg = std::max(dv.max_deg, seg_deg[sgi]);
    dv.Pu = Pu; dv.Pv = Pv; dv.eps = eps; dv.ox = ox; dv.oy = oy;
    dv.nx = nx; dv.ny = ny; dv.PP = PP;
    dv.M = (float)M;
    dv.Mq = (float)Mq;
    dv.Om = (float)std::fmax(std::fabs(ox), std::fabs(oy));
    dv.nxf = (float)nx;
    dv.nyf = (float)ny;
    dv.oxh = (float)ox;
    dv.oxl = (float)(ox - (double)dv.oxh);
    dv.oyh = (float)oy;
    dv.oyl = (float)(oy - (double)dv.oyh);
    dv.seg_deg = up.up(seg_deg);
    dv.seg_cp = up.up(seg_cp);
    dv.cp = up.up(P);
    dv.seg_B = up.up(segB);
    dv.loops = up.up(hl);
    dv.n_rec = (int)rec_seg.size();
    dv.rec = up.up(rec);
    dv.rec_obb = up.up(robb);
    dv.rec_seg = up.up(rec_seg);
    dv.rec_a64 = up.up(ra64);
    dv.rec_b64 = up.up(rb64);
    dv.rec_n64 = up.up(rn64);
    dv.n_nodes = (int)(nodes.size() / kCluF4);
    dv.all_root = all_root;
    {
        // FP32 hi/lo of every lifted control point relative to the origin,
        // for the near walk's query-relative control points
        std::vector<float4> cp32(ncp);
        for (size_t i = 0; i < (size_t)ncp; i++) {
            const double dx = P[2 * i] - ox, dy = P[2 * i + 1] - oy;
            const float hx = (float)dx, hy = (float)dy;
            cp32[i] = make_float4(hx, hy, (float)(dx - (double)hx), (float)(dy - (double)hy));
        }
        std::vector<int4> info(ns);
        for (int i = 0; i < ns; i++) {
            const float b32 = (float)segB[i];
            int bi, ri = 0;
            std::memcpy(&bi, &b32, 4);
            if (seg_rat[i]) {
                // weight ratio W/w of the segment, rounded up, for the FP32 error bound
                const double *w = &Wt[seg_cp[i]];
                double wmax = w[0], wmin = w[0];
                for (int k = 1; k <= seg_deg[i]; k++) {
                    wmax = std::fmax(wmax, w[k]);
                    wmin = std::fmin(wmin, w[k]);
                }
                const float r32 = std::nextafter((float)(wmax / wmin), INFINITY);
                std::memcpy(&ri, &r32, 4);
            }
            info[i] = make_int4(seg_cp[i], seg_deg[i], bi, ri);
        }
        dv.cp32 = up.up(cp32);
        dv.seg_info = up.up(info);
        if (rational) {
            // weights of the rational segments (1 elsewhere: those evaluate as
            // polynomials, the seg_info ratio says which)
            std::vector<float> w32(ncp);
            for (long long i = 0; i < ncp; i++) w32[i] = (float)Wt[i];
            dv.w = up.up(Wt);
            dv.w32 = up.up(w32);
            // bounds on the eighths of the rational segments (the polynomial
            // ones repeat B; only rational walks read these)
            std::vector<double> bs(8 * (size_t)ns);
            std::vector<float> bs32(8 * (size_t)ns);
            for (int i = 0; i < ns; i++) {
                double e8[8];
                if (seg_rat[i]) rational_eighth_bounds(&P[2 * seg_cp[i]], &Wt[seg_cp[i]], seg_deg[i], segB[i], e8);
                else std::fill(e8, e8 + 8, segB[i]);
                for (int j = 0; j < 8; j++) {
                    float f = (float)e8[j];
                    if ((double)f < e8[j]) f = std::nextafter(f, INFINITY);
                    bs[8 * (size_t)i + j] = e8[j];
                    bs32[8 * (size_t)i + j] = f;
                }
            }
            dv.seg_bsub = up.up(bs);
            dv.seg_bsub32 = up.up(bs32);
        }
        dv.eps32 = (float)eps;
    }
    dv.nodes = up.up(nodes);
    if (up.err != cudaSuccess) return fail(up.err == cudaErrorMemoryAllocation ? 4 : 3,
                                           std::string("CUDA: ") + cudaGetErrorString(up.err));
    {
        std::vector<DomDev> one(1, dv);
        D->d_self = up.up(one);
        if (up.err != cudaSuccess) return fail(3, std::string("CUDA: ") + cudaGetErrorString(up.err));
    }

    // ---- pairing (bi-periodic)
    struct Pair { int a, b; long long I, J; double plo, phi; };
    std::vector<Pair> pairs;
    if (!A_idx.empty()) {
        std::vector<char> used(n_loops, 0);
        auto run_pe = [&](const std::vector<PeReq> &req, std::vector<double> &res) -> cudaError_t {
            res.assign(req.size(), 0.0);
            if (req.empty()) return cudaSuccess;
            PeReq *dreq = nullptr;
            double *dres = nullptr;
            cudaError_t e = cudaMalloc(&dreq, req.size() * sizeof(PeReq));
            if (e == cudaSuccess) e = cudaMalloc(&dres, req.size() * sizeof(double));
            if (e == cudaSuccess) e = cudaMemcpy(dreq, req.data(), req.size() * sizeof(PeReq), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = launch_pe_eval(D->d_self, dreq, (int)req.size(), dres, 0);
            if (e == cudaSuccess) e = cudaMemcpy(res.data(), dres, req.size() * sizeof(double), cudaMemcpyDeviceToHost);
            cudaFree(dreq);
            cudaFree(dres);
            return e;
        };
        for (int a : A_idx) {
            const HostLoop &LA = loops[a];
            const double nA = nx * LA.g0[0] + ny * LA.g0[1];
            struct Cand { int b; long long I, J; };
            std::vector<Cand> cand;
            for (int b : B_idx) {
                if (used[b]) continue;
                const HostLoop &LB = loops[b];
                const double nB = nx * LB.g0[0] + ny * LB.g0[1];
                const long long c0 = lround_ll((nA - nB) / PP);
                for (long long c = c0 - 2; c <= c0 + 2; c++) cand.push_back({b, c * i0, c * j0});
            }
            std::vector<PeReq> req;
            for (const Cand &c : cand) req.push_back({a, c.b, 0, 0, c.I, c.J});
            std::vector<double> left;
            cudaError_t e = run_pe(req, left);
            if (e != cudaSuccess) return fail(3, std::string("CUDA: ") + cudaGetErrorString(e));
            std::vector<int> L;
            for (size_t i = 0; i < cand.size(); i++) {
                if (std::isnan(left[i])) return fail(2, "trimming loops intersect (pairing met a boundary point)");
                if (left[i] > 0) L.push_back((int)i);
            }
            // relation: cand X left of cand Y in Y's (beta) orientation
            req.clear();
            for (int x : L)
                for (int y : L)
                    req.push_back({cand[y].b, cand[x].b, cand[y].I, cand[y].J, cand[x].I, cand[x].J});
            std::vector<double> rel;
            e = run_pe(req, rel);
            if (e != cudaSuccess) return fail(3, std::string("CUDA: ") + cudaGetErrorString(e));
            int best = -1;
            for (size_t xi = 0; xi < L.size(); xi++) {
                if (best >= 0) {
                    size_t bi = std::find(L.begin(), L.end(), best) - L.begin();
                    double w = rel[xi * L.size() + bi];
                    if (std::isnan(w)) return fail(2, "trimming loops intersect (pairing met a boundary point)");
                    if (!(w > 0)) continue;
                }
                best = L[xi];
            }
            if (best < 0) return fail(2, "no partner found for a non-contractible loop (App. C pairing)");
            const Cand &bc = cand[best];
            used[bc.b] = 1;
            Pair pr{a, bc.b, bc.I, bc.J, LA.nlo, LA.nhi};
            const HostLoop &LB = loops[bc.b];
            for (int s = LB.s0; s < LB.s1; s++) {
                const double *q = &P[2 * seg_cp[s]];
                for (int i = 0; i <= seg_deg[s]; i++) {
                    double x = q[2 * i] + (double)bc.I * Pu, y = q[2 * i + 1] + (double)bc.J * Pv;
                    double nv = nx * x + ny * y;
                    pr.plo = std::fmin(pr.plo, nv);
                    pr.phi = std::fmax(pr.phi, nv);
                }
            }
            pairs.push_back(pr);
        }
    }

    // ---- instances
    std::vector<InstDev> inst;
    auto base_inst = [&](int type, int l) {
        InstDev in;
        std::memset(&in, 0, sizeof in);
        in.type = type;
        in.loop = l;
        in.pair = -1;
        in.r0 = loop_r0[l];
        in.r1 = loop_r1[l];
        return in;
    };
    const double tile_x[2] = {0.0, (Pu > 0) ? Pu : 0.0}, tile_y[2] = {0.0, (Pv > 0) ? Pv : 0.0};
    // slab window of copies k of loop l seen from x_f = p - F, p in the base tile
    auto add_extended = [&](int l, long long I, long long J, int pair, long long c) {
        const HostLoop &L = loops[l];
        InstDev ln = base_inst(IT_LINE, l);
        ln.Fx = (double)I * Pu; ln.Fy = (double)J * Pv;
        if (!(Pu > 0)) ln.Fx = 0.0;
        if (!(Pv > 0)) ln.Fy = 0.0;
        ln.I = I; ln.J = J; ln.pair = pair; ln.c = c;
        ln.r0 = ln.r1 = 0;
        inst.push_back(ln);
        // sp range over the base tile (a cylinder tile is unbounded across the
        // axis, but v has no component along it)
        double smn = INFINITY, smx = -INFINITY;
        for (double tx : tile_x)
            for (double ty : tile_y) {
                double xf = tx - ln.Fx, yf = ty - ln.Fy;
                double sp = (xf * L.v[0] + yf * L.v[1]) / L.vv;
                smn = std::fmin(smn, sp);
                smx = std::fmax(smx, sp);
            }
        const long long klo = (long long)std::floor(smn - L.smax) - 1;
        const long long khi = (long long)std::ceil(smx - L.smin) + 1;
        for (long long k = klo; k <= khi; k++) {
            InstDev in = base_inst(IT_PE, l);
            in.Fx = ln.Fx; in.Fy = ln.Fy; in.I = I; in.J = J; in.pair = pair; in.c = c; in.k = k;
            in.Tx = (Pu > 0) ? (double)(I + k * L.hp) * Pu : 0.0;
            in.Ty = (Pv > 0) ? (double)(J + k * L.hq) * Pv : 0.0;
            inst.push_back(in);
        }
    };
    if (kind == DK_PLANAR) {
        if (n_loops > 0 && ns > 0) {
            InstDev in = base_inst(IT_ALL, 0);
            in.r0 = 0;
            in.r1 = (int)rec_seg.size();
            inst.push_back(in);
        }
    } else {
        for (int l = 0; l < n_loops; l++) {
            const HostLoop &L = loops[l];
            if (L.s1 == L.s0) continue;
            if (L.cls == 1) {
                long long ia = 0, ib = 0, ja = 0, jb = 0;
                if (Pu > 0) {
                    ia = (long long)std::floor((0.0 - L.box[1]) / Pu) - 1;
                    ib = (long long)std::ceil((Pu - L.box[0]) / Pu) + 1;
                }
                if (Pv > 0) {
                    ja = (long long)std::floor((0.0 - L.box[3]) / Pv) - 1;
                    jb = (long long)std::ceil((Pv - L.box[2]) / Pv) + 1;
                }
                for (long long i = ia; i <= ib; i++)
                    for (long long j = ja; j <= jb; j++) {
                        InstDev in = base_inst(IT_BOX, l);
                        in.axes = (Pu > 0 ? 1 : 0) | (Pv > 0 ? 2 : 0);
                        in.Tx = (Pu > 0) ? (double)i * Pu : 0.0;
                        in.Ty = (Pv > 0) ? (double)j * Pv : 0.0;
                        inst.push_back(in);
                    }
            } else if (L.cls == 2 && kind != DK_BI) {
                add_extended(l, 0, 0, -1, 0);
            }
        }
        for (size_t k = 0; k < pairs.size(); k++) {
            const Pair &pr = pairs[k];
            double nmn = INFINITY, nmx = -INFINITY;
            for (double tx : tile_x)
                for (double ty : tile_y) {
                    double np = nx * tx + ny * ty;
                    nmn = std::fmin(nmn, np);
                    nmx = std::fmax(nmx, np);
                }
            const long long clo = (long long)std::floor((nmn - pr.phi) / PP) - 1;
            const long long chi = (long long)std::ceil((nmx - pr.plo) / PP) + 1;
            for (long long c = clo; c <= chi; c++) {
                add_extended(pr.a, c * i0, c * j0, (int)k, c);
                add_extended(pr.b, c * i0 + pr.I, c * j0 + pr.J, (int)k, c);
            }
        }
    }
    std::vector<PairDev> hp_dev;
    for (const Pair &pr : pairs) hp_dev.push_back({pr.plo, pr.phi});
    // per instance, the query region its exact test can accept (inst_sees),
    // widened far beyond the rounding of that test (InstCull: a query outside
    // it is not seen), and the same region shrunk by as much (InstF32: a query
    // inside it is seen)
    std::vector<InstCull> cull(inst.size());
    std::vector<InstF32> instf(inst.size());
    struct Win64 { double x0, x1, y0, y1, n0, n1, v0, v1; };
    for (size_t j = 0; j < inst.size(); j++) {
        const InstDev &in = inst[j];
        Win64 c, e;                 // c widened, e shrunk
        c.x0 = c.y0 = c.n0 = c.v0 = -INFINITY;
        c.x1 = c.y1 = c.n1 = c.v1 = INFINITY;
        e = c;
        double vx = 0.0, vy = 0.0;
        auto bounds = [](double lo, double hi, double mag, double &wlo, double &whi, double &slo, double &shi) {
            const double sl = 1e-9 * (mag + 1.0);
            wlo = lo - sl;
            whi = hi + sl;
            slo = lo + sl;
            shi = hi - sl;
        };
        if (in.type == IT_BOX) {
            const HostLoop &L = loops[in.loop];
            if (in.axes & 1)
                bounds(L.box[0] + in.Tx, L.box[1] + in.Tx, std::fabs(L.box[0]) + std::fabs(L.box[1]) + std::fabs(in.Tx),
                       c.x0, c.x1, e.x0, e.x1);
            if (in.axes & 2)
                bounds(L.box[2] + in.Ty, L.box[3] + in.Ty, std::fabs(L.box[2]) + std::fabs(L.box[3]) + std::fabs(in.Ty),
                       c.y0, c.y1, e.y0, e.y1);
        } else if (in.type == IT_LINE || in.type == IT_PE) {
            if (in.pair >= 0) {
                const Pair &pr = pairs[in.pair];
                const double cp = (double)in.c * PP;
                bounds(cp + pr.plo, cp + pr.phi,
                       std::fabs(cp) + std::fabs(pr.plo) + std::fabs(pr.phi) + (std::fabs(nx) + std::fabs(ny)) * (Pu + Pv),
                       c.n0, c.n1, e.n0, e.n1);
            }
            if (in.type == IT_PE) {
                const HostLoop &L = loops[in.loop];
                const double fx = (Pu > 0) ? in.Fx : 0.0, fy = (Pv > 0) ? in.Fy : 0.0;
                const double off = fx * L.v[0] + fy * L.v[1];
                vx = L.v[0];
                vy = L.v[1];
                const double v0 = ((double)in.k + L.smin) * L.vv + off, v1 = ((double)in.k + L.smax) * L.vv + off;
                bounds(v0, v1, std::fabs(v0) + std::fabs(v1) + std::fabs(off) + (std::fabs(L.v[0]) + std::fabs(L.v[1])) * (Pu + Pv + 1.0),
                       c.v0, c.v1, e.v0, e.v1);
            }
        }
        auto lo = [](double x) { return std::nextafter((float)x, -INFINITY); };
        auto hi = [](double x) { return std::nextafter((float)x, INFINITY); };
        InstCull f;
        f.x0 = lo(c.x0); f.x1 = hi(c.x1); f.y0 = lo(c.y0); f.y1 = hi(c.y1);
        f.n0 = lo(c.n0); f.n1 = hi(c.n1); f.v0 = lo(c.v0); f.v1 = hi(c.v1);
        f.vx = (float)vx; f.vy = (float)vy;
        f.pad0 = f.pad1 = 0.f;
        cull[j] = f;
        // inner window rounded inward, infinite sides kept (an empty window
        // accepts nothing)
        auto ilo = [](double x) { return std::isinf(x) ? (float)x : std::nextafter((float)x, INFINITY); };
        auto ihi = [](double x) { return std::isinf(x) ? (float)x : std::nextafter((float)x, -INFINITY); };
        InstF32 g;
        g.x0 = ilo(e.x0); g.x1 = ihi(e.x1); g.y0 = ilo(e.y0); g.y1 = ihi(e.y1);
        g.n0 = ilo(e.n0); g.n1 = ihi(e.n1); g.v0 = ilo(e.v0); g.v1 = ihi(e.v1);
        g.txh = (float)in.Tx;
        g.txl = (float)(in.Tx - (double)g.txh);
        g.tyh = (float)in.Ty;
        g.tyl = (float)(in.Ty - (double)g.tyh);
        g.lx = g.ly = g.lvx = g.lvy = 0.f;
        if (in.type == IT_LINE) {
            const HostLoop &L = loops[in.loop];
            g.lx = (float)(((Pu > 0) ? in.Fx : 0.0) + L.g0[0]);
            g.ly = (float)(((Pv > 0) ? in.Fy : 0.0) + L.g0[1]);
            g.lvx = (float)L.v[0];
            g.lvy = (float)L.v[1];
        }
        instf[j] = g;
        dv.Tm = std::fmax(dv.Tm, (float)std::fmax(std::fabs(in.Tx), std::fabs(in.Ty)));
    }
    dv.cull = up.up(cull);
    dv.instf = up.up(instf);
    dv.n_inst = (int)inst.size();
    dv.n_pairs = (int)pairs.size();
    dv.inst = up.up(inst);
    dv.pairs = up.up(hp_dev);
    if (up.err != cudaSuccess) return fail(up.err == cudaErrorMemoryAllocation ? 4 : 3,
                                           std::string("CUDA: ") + cudaGetErrorString(up.err));
    cudaError_t e = cudaMemcpy(D->d_self, &dv, sizeof dv, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(3, std::string("CUDA: ") + cudaGetErrorString(e));
    D->n_records = (int64_t)rec_seg.size();
    D->n_instances = (int64_t)inst.size();
    D->sweep_records = 0;
    for (const InstDev &in : inst) D->sweep_records += in.r1 - in.r0;
    {
        // circle area of every record over the area queries come from (the
        // base tile on periodic axes, else the control-point box), counted
        // once per instance that sweeps it: the near queue is sized from it
        double area = 0.0;
        for (size_t r = 0; r < rec.size() / 4; r++) {
            const double R = std::sqrt((double)rec[4 * r + 1].z);
            area += M_PI * R * R;
        }
        const double wx = Pu > 0 ? Pu : std::fmax(bx1 - bx0, 1e-300);
        const double wy = Pv > 0 ? Pv : std::fmax(by1 - by0, 1e-300);
        const double per_inst = rec.empty() ? 0.0 : (double)D->sweep_records / (double)(rec.size() / 4);
        D->near_density = std::fmin(area / (wx * wy) * std::fmax(per_inst, 1.0), 1e6);
    }
    *out = D;
    return 0;
}

}  // namespace wn
