/*
 * wn_oracle.c -- plain, slow FP64 oracle for point containment against
 * Bezier trimming loops, written from Bao, Shen & Wang, "Fast and Robust
 * Point Containment Queries on Trimmed Surface" (arXiv 2510.25159).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or helper with the CUDA library; it reads the same seeded inputs.
 *
 * Every function follows the paper's definitions in the paper's order, in
 * double precision, with no blocking, fusion or reordering:
 *
 *   or_eval            gamma(t) by de Casteljau (Sec. 4.2 evaluates gamma(m);
 *                      any exact evaluation of the Bernstein form is valid).
 *   or_bound           B = max_i n |P_i - P_{i-1}|   (Lemma 1, App. A.1).
 *   seg_wn             Algorithm 1 with the sub-segment ellipse of Eq. 5 and
 *                      the chord winding of Eq. 3 (signed angle / 2 pi).
 *   or_hull_segment_wn independent second oracle: the same recursion with the
 *                      control-polygon hull bound and de Casteljau splits
 *                      (the prior method the paper compares to, Sec. 4.2,
 *                      Table 1).  Shares only or_eval-free code paths.
 *   pe_wn              periodically extended curve, Eq. 9 (Sec. 4.4) with
 *                      the line term omega(p,L) = +-1/2 and the truncation
 *                      window taken as the slab of the curve along v.
 *   query_one          planar sum (Sec. 4.1), uni-periodic copies and
 *                      extended curves (Sec. 4.5, App. C Alg. 3-4),
 *                      bi-periodic contractible copies (Alg. 5 reading),
 *                      loop classes A/B/C (Prop. 1), families (Prop. 2,
 *                      Eq. 11) and band winding of pairs (Eq. 12, Alg. 6-7),
 *                      pairing (Alg. 8-10 reading).
 *
 * Readings where the paper is silent, garbled or inconsistent (each is also
 * listed in the design notes of the repository):
 *   R1  boundary test is strict (d < eps) and runs before the bound test;
 *       the ellipse is closed, so "far" needs d(p,a)+d(p,b) > B (b-a).
 *   R2  recursion depth cap 64 reports BOUNDARY (unreachable for d > eps by
 *       Lemma 2).
 *   R3  INSIDE iff omega >= 1/2 (outer loops CCW, holes CW).
 *   R4  default eps = 1e-9 * max(Pu, Pv, extent of the control-point box).
 *   R5  lifting translates whole segments by the lattice vector that brings
 *       their start nearest to the previous segment's lifted end; homology
 *       is round((end - start) / period) per periodic axis.
 *   R6  contractible copies: bi-periodic -> every lattice shift with the
 *       shifted query inside the closed control-point box (replaces the
 *       window of Alg. 5); uni-periodic -> every shift along the periodic
 *       axis with the shifted coordinate inside the box's range on that axis
 *       (the loop shape of Alg. 4).
 *   R7  extended curves use the lattice vector v = (p Pu, q Pv) (equal to
 *       gamma(1)-gamma(0) for closed loops), include k = 0 exactly once, and
 *       sum the copies k with s(p) - k inside the slab [smin, smax] of the
 *       control points and gamma(0)+v along v, s(x) = x.v / v.v.  A query on
 *       the line L is BOUNDARY.
 *   R8  bi-periodic families are indexed by c = p j - q i (gcd(p,q) = 1),
 *       represented by the lattice vector c (i0, j0) with p j0 - q i0 = 1
 *       (i0 in [0,|p|) for p != 0; i0 = -q, j0 = 0 for p = 0); a family is
 *       summed when n.(x - w_c) lies in the hull of the n-extents of alpha
 *       and of the paired beta, n = (-q Pv, p Pu).
 *   R10 rational segments (weights w_i > 0): gamma is the projection of the
 *       polynomial curve of (w_i x_i, w_i y_i, w_i); of the two derivative
 *       bounds of App. A.1 the smaller is taken (both hold).
 *   R9  pairing: for each alpha in input order, among the remaining beta and
 *       the shifts c0-2..c0+2 (c0 brings beta's start within one family
 *       spacing of alpha's), take the copies left of alpha (ToLeft, Alg. 8,
 *       on the loop's parameter midpoint) and keep the one that lies left of
 *       the current best in the beta orientation (the nearest one).
 *   R11 a sphere's or cone's singular point, punctured (Sec. 4.3), enters as
 *       a boundary loop along its line in the parameter domain, as B-Rep
 *       models store a degenerate edge there (an input convention: this
 *       file treats it as any other loop).
 *
 * Pins (tests/pins.py, tests/test_oracle.py): exact integer winding of
 * degree-1 polygons, atan2 for a single chord, +-1/0 for circles, the hull
 * oracle, dense polylines, the unit jump, additivity / degree elevation /
 * reversal / translation, Lemma 1 containment, Lemma 2 depth, Table 3's
 * shape, the boundary fraction trend, closed-form cylinder strips and torus
 * bands (which fix lifting, homology, families, line terms and pairing),
 * lattice translation, window enlargement for closed extended curves, the
 * 3x3 unfold, rational segments (exact circular arcs, the bound against
 * sampled speeds, dense polylines, weight scaling and reparametrization),
 * and 19 planted mistakes that the pins reject.
 * Parity unpinned: the contribution of OPEN loops on periodic domains
 * (R6/R7 windows are the definition there and nothing outside this file
 * fixes them), and the BOUNDARY decision for points whose distance to an
 * evaluated curve point is within rounding of eps.
 *
 * Every lattice translation is applied in one step, x - (I Pu, J Pv) with
 * integers I, J, so that shifted points do not depend on summation order.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_DEG 15
#define OR_DEPTH_CAP 64

enum { OR_OUTSIDE = 0, OR_INSIDE = 1, OR_BOUNDARY = 2 };
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_TOPOLOGY = 2, OR_ERR_OOM = 4 };
enum { K_PLANAR = 0, K_UNI_U = 1, K_UNI_V = 2, K_BI = 3 };
enum { L_PLAIN = 0, L_CONTRACTIBLE = 1, L_EXTENDED = 2 };

typedef struct {
    int64_t evals;      /* gamma(m) evaluations (Table 3 "eval count") */
    int64_t nodes;      /* Algorithm 1 invocations */
    int64_t chords;     /* chord contributions taken */
    int64_t max_depth;
    int64_t depth_cap;  /* R2 hits */
} or_stats;

typedef struct {
    double ang;      /* sum of chord angles, radians */
    int64_t half;    /* sum of line terms in units of 1/2 */
    double margin;   /* smallest decision margin on the path */
    int boundary;
    or_stats st;
} acc_t;

typedef struct {
    int deg;
    const double *P;   /* (deg+1) points, xy interleaved, lifted */
    double B;
    const double *W;   /* (deg+1) weights of a rational segment, or NULL */
} oseg_t;

typedef struct {
    int s0, s1;          /* segment range [s0, s1) */
    int cls;
    int hp, hq;          /* homology */
    double v[2];         /* lattice vector of the homology */
    double g0[2], g0v[2];/* gamma(0), gamma(0) + v */
    double box[4];       /* xmin xmax ymin ymax of lifted control points */
    double smin, smax;   /* slab along v */
    double nlo, nhi;     /* extent along the family normal (bi-periodic) */
} oloop_t;

typedef struct {
    int kind;
    double Pu, Pv, eps;
    int n_loops, n_segs;
    oseg_t *seg;
    oloop_t *loop;
    double *cps;         /* lifted control points */
    double *w;           /* weights per control point (rational input), or NULL */
    /* bi-periodic */
    int hp, hq;          /* homology of class A */
    long i0, j0;         /* family generator */
    double nx, ny;       /* family normal n = (-q Pv, p Pu) */
    int n_pairs;
    int *pa, *pb;        /* loop index of alpha / beta */
    long *pI, *pJ;       /* lattice shift of beta in the pair */
    double *plo, *phi;   /* hull of the n-extents of alpha and shifted beta */
} odom_t;

static void acc_margin(acc_t *a, double m)
{
    m = fabs(m);
    if (m < a->margin) a->margin = m;
}

/* ------------------------------------------------------------------ */
/* Bezier primitives                                                   */
/* ------------------------------------------------------------------ */

/* gamma(t) by de Casteljau's repeated linear interpolation. */
int or_eval(int deg, const double *P, double t, double *out)
{
    double q[2 * (OR_MAX_DEG + 1)];
    if (deg < 0 || deg > OR_MAX_DEG) return OR_ERR_ARG;
    memcpy(q, P, sizeof(double) * 2 * (size_t)(deg + 1));
    for (int r = 1; r <= deg; r++)
        for (int i = 0; i <= deg - r; i++) {
            q[2 * i] = (1.0 - t) * q[2 * i] + t * q[2 * i + 2];
            q[2 * i + 1] = (1.0 - t) * q[2 * i + 1] + t * q[2 * i + 3];
        }
    out[0] = q[0];
    out[1] = q[1];
    return OR_OK;
}

/* Derivative bound of Lemma 1: the hodograph has control points
 * n (P_i - P_{i-1}), and its control polygon bounds |gamma'|. */
double or_bound(int deg, const double *P)
{
    double B = 0.0;
    for (int i = 1; i <= deg; i++) {
        double dx = P[2 * i] - P[2 * i - 2], dy = P[2 * i + 1] - P[2 * i - 1];
        double b = (double)deg * sqrt(dx * dx + dy * dy);
        if (b > B) B = b;
    }
    return B;
}

/* gamma(t) of a rational segment (weights W > 0): the curve is the central
 * projection of the polynomial curve with control points (w_i x_i, w_i y_i,
 * w_i), so de Casteljau runs on those and the result is divided by the last
 * coordinate (App. A.1 treats the rational case; W = NULL is polynomial). */
int or_eval_w(int deg, const double *P, const double *W, double t, double *out)
{
    if (!W) return or_eval(deg, P, t, out);
    double h[3 * (OR_MAX_DEG + 1)];
    if (deg < 0 || deg > OR_MAX_DEG) return OR_ERR_ARG;
    for (int i = 0; i <= deg; i++) {
        h[3 * i] = W[i] * P[2 * i];
        h[3 * i + 1] = W[i] * P[2 * i + 1];
        h[3 * i + 2] = W[i];
    }
    for (int r = 1; r <= deg; r++)
        for (int i = 0; i <= deg - r; i++)
            for (int c = 0; c < 3; c++) h[3 * i + c] = (1.0 - t) * h[3 * i + c] + t * h[3 * i + 3 + c];
    out[0] = h[0] / h[2];
    out[1] = h[1] / h[2];
    return OR_OK;
}

/* Derivative bound of a rational segment (App. A.1, after Floater):
 *   |gamma'| <= n (W/w) max_{i,j} |P_i - P_j|  and
 *   |gamma'| <= n (W/w)^2 max_i |P_i - P_{i-1}|,  W = max w_i, w = min w_i;
 * both hold, so the smaller one is taken.  W = NULL: or_bound. */
double or_bound_w(int deg, const double *P, const double *W)
{
    if (!W) return or_bound(deg, P);
    double wmax = W[0], wmin = W[0];
    for (int i = 1; i <= deg; i++) {
        wmax = fmax(wmax, W[i]);
        wmin = fmin(wmin, W[i]);
    }
    const double r = wmax / wmin;
    double dall = 0.0, dnext = 0.0;
    for (int i = 0; i <= deg; i++)
        for (int j = i + 1; j <= deg; j++) {
            double dx = P[2 * j] - P[2 * i], dy = P[2 * j + 1] - P[2 * i + 1];
            double d = sqrt(dx * dx + dy * dy);
            if (d > dall) dall = d;
            if (j == i + 1 && d > dnext) dnext = d;
        }
    const double b1 = (double)deg * r * dall, b2 = (double)deg * r * r * dnext;
    return b1 < b2 ? b1 : b2;
}

/* Eq. 3: winding number of the oriented chord a->b about p, in radians
 * (the signed angle from a-p to b-p). */
static double chord_angle(double px, double py, const double *a, const double *b)
{
    double ax = a[0] - px, ay = a[1] - py, bx = b[0] - px, by = b[1] - py;
    return atan2(ax * by - ay * bx, ax * bx + ay * by);
}

/* Algorithm 1 on the parameter interval [a,b]; ga = gamma(a), gb = gamma(b).
 * Returns 1 when the query is on the boundary. */
static int seg_wn(const oseg_t *s, double px, double py, double a, double b,
                  const double *ga, const double *gb, double eps, int depth, acc_t *acc)
{
    acc->st.nodes++;
    if (depth > acc->st.max_depth) acc->st.max_depth = depth;
    double ax = ga[0] - px, ay = ga[1] - py, bx = gb[0] - px, by = gb[1] - py;
    double da = sqrt(ax * ax + ay * ay), db = sqrt(bx * bx + by * by);
    acc_margin(acc, da - eps);
    acc_margin(acc, db - eps);
    if (da < eps || db < eps) return 1;
    double lim = s->B * (b - a);
    acc_margin(acc, (da + db) - lim);
    if (da + db > lim) {                      /* outside the ellipse of Eq. 5 */
        acc->ang += atan2(ax * by - ay * bx, ax * bx + ay * by);
        acc->st.chords++;
        return 0;
    }
    if (depth >= OR_DEPTH_CAP) {
        acc->st.depth_cap++;
        return 1;
    }
    double m = 0.5 * (a + b), gm[2];
    or_eval_w(s->deg, s->P, s->W, m, gm);
    acc->st.evals++;
    if (seg_wn(s, px, py, a, m, ga, gm, eps, depth + 1, acc)) return 1;
    return seg_wn(s, px, py, m, b, gm, gb, eps, depth + 1, acc);
}

static int seg_root(const oseg_t *s, double px, double py, double eps, acc_t *acc)
{
    return seg_wn(s, px, py, 0.0, 1.0, s->P, s->P + 2 * s->deg, eps, 0, acc);
}

/* Alg. 1 on one segment (weights W, or NULL for a polynomial segment);
 * *angle receives the sum of chord angles (radians). */
int or_segment_wn_w(int deg, const double *P, const double *W, double px, double py, double eps,
                    double *angle, int64_t *stats5)
{
    if (deg < 1 || deg > OR_MAX_DEG) return -1;
    oseg_t s = {deg, P, or_bound_w(deg, P, W), W};
    acc_t acc;
    memset(&acc, 0, sizeof acc);
    acc.margin = INFINITY;
    int bnd = seg_root(&s, px, py, eps, &acc);
    *angle = acc.ang;
    if (stats5) {
        stats5[0] = acc.st.evals; stats5[1] = acc.st.nodes; stats5[2] = acc.st.chords;
        stats5[3] = acc.st.max_depth; stats5[4] = acc.st.depth_cap;
    }
    return bnd;
}

int or_segment_wn(int deg, const double *P, double px, double py, double eps,
                  double *angle, int64_t *stats5)
{
    return or_segment_wn_w(deg, P, NULL, px, py, eps, angle, stats5);
}

/* ------------------------------------------------------------------ */
/* Independent second oracle: control-polygon hull bound               */
/* ------------------------------------------------------------------ */

static double cross3(const double *o, const double *a, const double *b)
{
    return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0]);
}

static int cmp_pt(const void *x, const void *y)
{
    const double *a = (const double *)x, *b = (const double *)y;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    return 0;
}

/* 1 when p is strictly outside the convex hull of the n+1 points. */
static int outside_hull(int n, const double *Q, double px, double py)
{
    double pts[2 * (OR_MAX_DEG + 1)], H[4 * (OR_MAX_DEG + 1)], p[2] = {px, py};
    int m = n + 1, k = 0;
    memcpy(pts, Q, sizeof(double) * 2 * (size_t)m);
    qsort(pts, (size_t)m, 2 * sizeof(double), cmp_pt);
    for (int i = 0; i < m; i++) {                           /* lower chain */
        while (k >= 2 && cross3(H + 2 * (k - 2), H + 2 * (k - 1), pts + 2 * i) <= 0) k--;
        H[2 * k] = pts[2 * i]; H[2 * k + 1] = pts[2 * i + 1]; k++;
    }
    for (int i = m - 2, t = k + 1; i >= 0; i--) {           /* upper chain */
        while (k >= t && cross3(H + 2 * (k - 2), H + 2 * (k - 1), pts + 2 * i) <= 0) k--;
        H[2 * k] = pts[2 * i]; H[2 * k + 1] = pts[2 * i + 1]; k++;
    }
    if (k > 1) k--;                                         /* last == first */
    if (k == 1) return !(px == H[0] && py == H[1]);
    if (k == 2) {
        double c = cross3(H, H + 2, p);
        if (c != 0) return 1;
        double d0 = (px - H[0]) * (H[2] - H[0]) + (py - H[1]) * (H[3] - H[1]);
        double d1 = (px - H[2]) * (H[0] - H[2]) + (py - H[3]) * (H[1] - H[3]);
        return d0 < 0 || d1 < 0;
    }
    for (int i = 0; i < k; i++) {
        const double *a = H + 2 * i, *b = H + 2 * ((i + 1) % k);
        if (cross3(a, b, p) < 0) return 1;
    }
    return 0;
}

static int hull_rec(int n, const double *Q, double px, double py, double eps, int depth,
                    double *ang, int64_t *evals)
{
    const double *a = Q, *b = Q + 2 * n;
    double da = hypot(a[0] - px, a[1] - py), db = hypot(b[0] - px, b[1] - py);
    if (da < eps || db < eps) return 1;
    if (outside_hull(n, Q, px, py)) {
        *ang += chord_angle(px, py, a, b);
        return 0;
    }
    if (depth >= OR_DEPTH_CAP) return 1;
    /* de Casteljau split at 1/2: left = first points of each level,
     * right = last points of each level. */
    double tri[2 * (OR_MAX_DEG + 1)], L[2 * (OR_MAX_DEG + 1)], R[2 * (OR_MAX_DEG + 1)];
    memcpy(tri, Q, sizeof(double) * 2 * (size_t)(n + 1));
    L[0] = tri[0]; L[1] = tri[1];
    R[2 * n] = tri[2 * n]; R[2 * n + 1] = tri[2 * n + 1];
    for (int r = 1; r <= n; r++) {
        for (int i = 0; i <= n - r; i++) {
            tri[2 * i] = 0.5 * tri[2 * i] + 0.5 * tri[2 * i + 2];
            tri[2 * i + 1] = 0.5 * tri[2 * i + 1] + 0.5 * tri[2 * i + 3];
        }
        L[2 * r] = tri[0]; L[2 * r + 1] = tri[1];
        R[2 * (n - r)] = tri[2 * (n - r)]; R[2 * (n - r) + 1] = tri[2 * (n - r) + 1];
    }
    (*evals)++;
    if (hull_rec(n, L, px, py, eps, depth + 1, ang, evals)) return 1;
    return hull_rec(n, R, px, py, eps, depth + 1, ang, evals);
}

int or_hull_segment_wn(int deg, const double *P, double px, double py, double eps,
                       double *angle, int64_t *evals)
{
    if (deg < 1 || deg > OR_MAX_DEG) return -1;
    double a = 0.0;
    int64_t e = 0;
    int bnd = hull_rec(deg, P, px, py, eps, 0, &a, &e);
    *angle = a;
    if (evals) *evals = e;
    return bnd;
}

/* ------------------------------------------------------------------ */
/* Domain: lifting, classification, pairing                            */
/* ------------------------------------------------------------------ */

static double reduce(double x, double P)
{
    if (!(P > 0)) return x;
    double r = fmod(x, P);
    if (r < 0) r += P;
    if (r >= P) r = 0.0;
    return r;
}

static int loop_wn(const odom_t *D, const oloop_t *L, double px, double py, acc_t *acc)
{
    for (int s = L->s0; s < L->s1; s++)
        if (seg_root(&D->seg[s], px, py, D->eps, acc)) return 1;
    return 0;
}

/* Parameter midpoint of a whole loop (App. C, Alg. 8 evaluates gamma(0.5)). */
static void loop_mid(const odom_t *D, const oloop_t *L, double *out)
{
    int m = L->s1 - L->s0;
    int s = L->s0 + m / 2;
    double t = (m % 2) ? 0.5 : 0.0;
    or_eval_w(D->seg[s].deg, D->seg[s].P, D->seg[s].W, t, out);
}

/* Eq. 9: winding number about x of the periodically extended curve made
 * of the lifts L + (I + k lp, J + k lq) (Pu,Pv), k in Z, where x is the
 * base query and (I, J) the family's lattice shift (R7). */
static int pe_wn(const odom_t *D, const oloop_t *L, double bx, double by, long I, long J,
                 acc_t *acc)
{
    double Pu = D->Pu, Pv = D->Pv;
    double xf = bx - (double)I * Pu, yf = by - (double)J * Pv;
    if (!(Pu > 0)) xf = bx;
    if (!(Pv > 0)) yf = by;
    double vx = L->v[0], vy = L->v[1];
    double vn = sqrt(vx * vx + vy * vy);
    /* line term: +1/2 on the left of L (the line through gamma(0) along v) */
    double cr = vx * (yf - L->g0[1]) - vy * (xf - L->g0[0]);
    acc_margin(acc, cr / vn);
    if (cr == 0) return 1;
    acc->half += cr > 0 ? 1 : -1;
    double vv = vx * vx + vy * vy;
    double sp = (xf * vx + yf * vy) / vv;
    double klo = ceil(sp - L->smax), khi = floor(sp - L->smin);
    acc_margin(acc, (klo - (sp - L->smax)) * vn);
    acc_margin(acc, ((sp - L->smax) - (klo - 1.0)) * vn);
    acc_margin(acc, ((sp - L->smin) - khi) * vn);
    acc_margin(acc, ((khi + 1.0) - (sp - L->smin)) * vn);
    for (double k = klo; k <= khi; k += 1.0) {
        long kk = (long)k;
        double qx = (Pu > 0) ? bx - (double)(I + kk * L->hp) * Pu : bx;
        double qy = (Pv > 0) ? by - (double)(J + kk * L->hq) * Pv : by;
        if (loop_wn(D, L, qx, qy, acc)) return 1;
        acc->ang -= chord_angle(qx, qy, L->g0, L->g0v);
    }
    return 0;
}

static double pe_value(const odom_t *D, const oloop_t *L, double x, double y, long I, long J,
                       int *bnd)
{
    acc_t a;
    memset(&a, 0, sizeof a);
    a.margin = INFINITY;
    *bnd = pe_wn(D, L, x, y, I, J, &a);
    return a.ang / (2.0 * M_PI) + 0.5 * (double)a.half;
}

static void free_dom(odom_t *D)
{
    free(D->seg); free(D->loop); free(D->cps); free(D->w);
    free(D->pa); free(D->pb); free(D->pI); free(D->pJ); free(D->plo); free(D->phi);
    memset(D, 0, sizeof *D);
}

static long lround_d(double x) { return (long)round(x); }

static int build_dom(odom_t *D, int n_loops, const int32_t *loop_offsets, const int32_t *degrees,
                     const double *cps, const double *weights, double Pu, double Pv, double eps)
{
    memset(D, 0, sizeof *D);
    if (n_loops < 0 || !(Pu >= 0) || !(Pv >= 0) || isnan(eps)) return OR_ERR_ARG;
    if (loop_offsets[0] != 0) return OR_ERR_ARG;
    for (int l = 0; l < n_loops; l++)
        if (loop_offsets[l + 1] < loop_offsets[l]) return OR_ERR_ARG;
    int ns = loop_offsets[n_loops];
    long ncp = 0;
    for (int s = 0; s < ns; s++) {
        if (degrees[s] < 1 || degrees[s] > OR_MAX_DEG) return OR_ERR_ARG;
        ncp += degrees[s] + 1;
    }
    for (long i = 0; i < 2 * ncp; i++)
        if (!isfinite(cps[i])) return OR_ERR_ARG;
    if (weights)
        for (long i = 0; i < ncp; i++)
            if (!(weights[i] > 0) || !isfinite(weights[i])) return OR_ERR_ARG;
    D->Pu = Pu; D->Pv = Pv;
    D->kind = (Pu > 0 && Pv > 0) ? K_BI : (Pu > 0) ? K_UNI_U : (Pv > 0) ? K_UNI_V : K_PLANAR;
    D->n_loops = n_loops; D->n_segs = ns;
    D->seg = calloc((size_t)(ns ? ns : 1), sizeof(oseg_t));
    D->loop = calloc((size_t)(n_loops ? n_loops : 1), sizeof(oloop_t));
    D->cps = malloc(sizeof(double) * 2 * (size_t)(ncp ? ncp : 1));
    if (!D->seg || !D->loop || !D->cps) { free_dom(D); return OR_ERR_OOM; }
    memcpy(D->cps, cps, sizeof(double) * 2 * (size_t)ncp);
    if (weights) {
        D->w = malloc(sizeof(double) * (size_t)(ncp ? ncp : 1));
        if (!D->w) { free_dom(D); return OR_ERR_OOM; }
        memcpy(D->w, weights, sizeof(double) * (size_t)ncp);
    }

    /* R4: default tolerance */
    if (!(eps > 0)) {
        double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
        for (long i = 0; i < ncp; i++) {
            x0 = fmin(x0, cps[2 * i]); x1 = fmax(x1, cps[2 * i]);
            y0 = fmin(y0, cps[2 * i + 1]); y1 = fmax(y1, cps[2 * i + 1]);
        }
        double S = fmax(Pu, Pv);
        if (ncp) S = fmax(S, fmax(x1 - x0, y1 - y0));
        eps = 1e-9 * S;
    }
    D->eps = eps;

    long off = 0;
    for (int s = 0; s < ns; s++) {
        D->seg[s].deg = degrees[s];
        D->seg[s].P = D->cps + 2 * off;
        D->seg[s].W = D->w ? D->w + off : NULL;
        off += degrees[s] + 1;
    }
    /* R5: lift each loop into the covering space */
    for (int l = 0; l < n_loops; l++) {
        oloop_t *L = &D->loop[l];
        L->s0 = loop_offsets[l];
        L->s1 = loop_offsets[l + 1];
        for (int s = L->s0 + 1; s < L->s1; s++) {
            const oseg_t *pr = &D->seg[s - 1];
            double ex = pr->P[2 * pr->deg], ey = pr->P[2 * pr->deg + 1];
            double *P = (double *)D->seg[s].P;
            long I = (Pu > 0) ? lround_d((ex - P[0]) / Pu) : 0;
            long J = (Pv > 0) ? lround_d((ey - P[1]) / Pv) : 0;
            for (int i = 0; i <= D->seg[s].deg; i++) {
                if (I) P[2 * i] = P[2 * i] + (double)I * Pu;
                if (J) P[2 * i + 1] = P[2 * i + 1] + (double)J * Pv;
            }
        }
        L->hp = L->hq = 0;
        if (L->s1 > L->s0) {
            const oseg_t *f = &D->seg[L->s0], *e = &D->seg[L->s1 - 1];
            if (Pu > 0) L->hp = (int)lround_d((e->P[2 * e->deg] - f->P[0]) / Pu);
            if (Pv > 0) L->hq = (int)lround_d((e->P[2 * e->deg + 1] - f->P[1]) / Pv);
        }
        L->box[0] = L->box[2] = INFINITY;
        L->box[1] = L->box[3] = -INFINITY;
        for (int s = L->s0; s < L->s1; s++) {
            oseg_t *sg = &D->seg[s];
            sg->B = or_bound_w(sg->deg, sg->P, sg->W);
            for (int i = 0; i <= sg->deg; i++) {
                L->box[0] = fmin(L->box[0], sg->P[2 * i]);
                L->box[1] = fmax(L->box[1], sg->P[2 * i]);
                L->box[2] = fmin(L->box[2], sg->P[2 * i + 1]);
                L->box[3] = fmax(L->box[3], sg->P[2 * i + 1]);
            }
        }
        if (D->kind == K_PLANAR) L->cls = L_PLAIN;
        else if (L->hp == 0 && L->hq == 0) L->cls = L_CONTRACTIBLE;
        else L->cls = L_EXTENDED;
        if (L->cls == L_EXTENDED) {
            if (D->kind != K_BI && (abs(L->hp) > 1 || abs(L->hq) > 1)) {
                free_dom(D);
                return OR_ERR_TOPOLOGY;        /* cylinder case of Prop. 1 */
            }
            L->v[0] = (double)L->hp * Pu;
            L->v[1] = (double)L->hq * Pv;
            if (!(Pu > 0)) L->v[0] = 0.0;
            if (!(Pv > 0)) L->v[1] = 0.0;
            L->g0[0] = D->seg[L->s0].P[0];
            L->g0[1] = D->seg[L->s0].P[1];
            L->g0v[0] = L->g0[0] + L->v[0];
            L->g0v[1] = L->g0[1] + L->v[1];
            double vv = L->v[0] * L->v[0] + L->v[1] * L->v[1];
            L->smin = (L->g0v[0] * L->v[0] + L->g0v[1] * L->v[1]) / vv;
            L->smax = L->smin;
            for (int s = L->s0; s < L->s1; s++) {
                const oseg_t *sg = &D->seg[s];
                for (int i = 0; i <= sg->deg; i++) {
                    double sv = (sg->P[2 * i] * L->v[0] + sg->P[2 * i + 1] * L->v[1]) / vv;
                    L->smin = fmin(L->smin, sv);
                    L->smax = fmax(L->smax, sv);
                }
            }
        }
    }
    if (D->kind != K_BI) return OR_OK;

    /* Prop. 1: classes A (homology (p,q)), B (-(p,q)), C (contractible) */
    int first = -1, na = 0, nb = 0;
    for (int l = 0; l < n_loops; l++)
        if (D->loop[l].cls == L_EXTENDED) { first = l; break; }
    if (first < 0) return OR_OK;
    D->hp = D->loop[first].hp;
    D->hq = D->loop[first].hq;
    {
        long a = labs(D->hp), b = labs(D->hq);
        while (b) { long t = a % b; a = b; b = t; }
        if (a != 1) { free_dom(D); return OR_ERR_TOPOLOGY; }
    }
    for (int l = 0; l < n_loops; l++) {
        oloop_t *L = &D->loop[l];
        if (L->cls != L_EXTENDED) continue;
        if (L->hp == D->hp && L->hq == D->hq) na++;
        else if (L->hp == -D->hp && L->hq == -D->hq) nb++;
        else { free_dom(D); return OR_ERR_TOPOLOGY; }
    }
    if (na != nb) { free_dom(D); return OR_ERR_TOPOLOGY; }
    /* R8: family generator and normal */
    if (D->hp == 0) { D->i0 = -D->hq; D->j0 = 0; }
    else {
        long ap = labs(D->hp);
        D->i0 = -1;
        for (long i = 0; i < ap; i++)
            if ((1 + (long)D->hq * i) % D->hp == 0) { D->i0 = i; break; }
        D->j0 = (1 + (long)D->hq * D->i0) / D->hp;
    }
    D->nx = -(double)D->hq * Pv;
    D->ny = (double)D->hp * Pu;
    for (int l = 0; l < n_loops; l++) {
        oloop_t *L = &D->loop[l];
        if (L->cls != L_EXTENDED) continue;
        L->nlo = INFINITY; L->nhi = -INFINITY;
        for (int s = L->s0; s < L->s1; s++) {
            const oseg_t *sg = &D->seg[s];
            for (int i = 0; i <= sg->deg; i++) {
                double nv = D->nx * sg->P[2 * i] + D->ny * sg->P[2 * i + 1];
                L->nlo = fmin(L->nlo, nv);
                L->nhi = fmax(L->nhi, nv);
            }
        }
    }
    /* R9: pairing, Alg. 8-10 */
    D->n_pairs = na;
    D->pa = calloc((size_t)na, sizeof(int));
    D->pb = calloc((size_t)na, sizeof(int));
    D->pI = calloc((size_t)na, sizeof(long));
    D->pJ = calloc((size_t)na, sizeof(long));
    D->plo = calloc((size_t)na, sizeof(double));
    D->phi = calloc((size_t)na, sizeof(double));
    int *used = calloc((size_t)n_loops, sizeof(int));
    if (!D->pa || !D->pb || !D->pI || !D->pJ || !D->plo || !D->phi || !used) {
        free(used); free_dom(D); return OR_ERR_OOM;
    }
    double PP = Pu * Pv;
    int k = 0;
    for (int a = 0; a < n_loops; a++) {
        const oloop_t *A = &D->loop[a];
        if (A->cls != L_EXTENDED || A->hp != D->hp || A->hq != D->hq) continue;
        double nA = D->nx * A->g0[0] + D->ny * A->g0[1];
        int best = -1;
        long bI = 0, bJ = 0;
        for (int b = 0; b < n_loops; b++) {
            const oloop_t *Bl = &D->loop[b];
            if (Bl->cls != L_EXTENDED || used[b] || (Bl->hp == D->hp && Bl->hq == D->hq)) continue;
            double nB = D->nx * Bl->g0[0] + D->ny * Bl->g0[1];
            long c0 = lround_d((nA - nB) / PP);
            double mid[2];
            loop_mid(D, Bl, mid);
            for (long c = c0 - 2; c <= c0 + 2; c++) {
                long I = c * D->i0, J = c * D->j0;
                double x = mid[0] + (double)I * Pu, y = mid[1] + (double)J * Pv;
                int bnd;
                double w = pe_value(D, A, x, y, 0, 0, &bnd);
                if (bnd) { free(used); free_dom(D); return OR_ERR_TOPOLOGY; }
                if (!(w > 0)) continue;
                if (best >= 0) {
                    /* candidate left of the current best (beta orientation):
                     * PE(mid + (I,J)P, best + (bI,bJ)P) = PE(., best) at shift (bI,bJ) */
                    double wb = pe_value(D, &D->loop[best], x, y, bI, bJ, &bnd);
                    if (bnd) { free(used); free_dom(D); return OR_ERR_TOPOLOGY; }
                    if (!(wb > 0)) continue;
                }
                best = b; bI = I; bJ = J;
            }
        }
        if (best < 0) { free(used); free_dom(D); return OR_ERR_TOPOLOGY; }
        used[best] = 1;
        D->pa[k] = a; D->pb[k] = best; D->pI[k] = bI; D->pJ[k] = bJ;
        const oloop_t *Bl = &D->loop[best];
        double lo = A->nlo, hi = A->nhi;
        for (int s = Bl->s0; s < Bl->s1; s++) {
            const oseg_t *sg = &D->seg[s];
            for (int i = 0; i <= sg->deg; i++) {
                double x = sg->P[2 * i] + (double)bI * Pu, y = sg->P[2 * i + 1] + (double)bJ * Pv;
                double nv = D->nx * x + D->ny * y;
                lo = fmin(lo, nv);
                hi = fmax(hi, nv);
            }
        }
        D->plo[k] = lo; D->phi[k] = hi;
        k++;
    }
    free(used);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Query                                                               */
/* ------------------------------------------------------------------ */

static void copies_1d(double x, double lo, double hi, double P, long *a, long *b)
{
    *a = (long)floor((x - hi) / P) - 1;
    *b = (long)ceil((x - lo) / P) + 1;
}

static void query_one(const odom_t *D, double px, double py, double *w, uint8_t *state,
                      double *margin, or_stats *st)
{
    acc_t acc;
    memset(&acc, 0, sizeof acc);
    acc.margin = INFINITY;
    double x = reduce(px, D->Pu), y = reduce(py, D->Pv);
    double Pu = D->Pu, Pv = D->Pv;
    int bnd = 0;
    for (int l = 0; l < D->n_loops && !bnd; l++) {
        const oloop_t *L = &D->loop[l];
        if (L->s1 == L->s0) continue;
        if (L->cls == L_PLAIN) {
            bnd = loop_wn(D, L, x, y, &acc);
        } else if (L->cls == L_CONTRACTIBLE) {
            long ia = 0, ib = 0, ja = 0, jb = 0;
            if (Pu > 0) copies_1d(x, L->box[0], L->box[1], Pu, &ia, &ib);
            if (Pv > 0) copies_1d(y, L->box[2], L->box[3], Pv, &ja, &jb);
            for (long i = ia; i <= ib && !bnd; i++) {
                double xs = (Pu > 0) ? x - (double)i * Pu : x;
                if (Pu > 0) {
                    acc_margin(&acc, xs - L->box[0]);
                    acc_margin(&acc, xs - L->box[1]);
                    if (!(xs >= L->box[0] && xs <= L->box[1])) continue;
                }
                for (long j = ja; j <= jb && !bnd; j++) {
                    double ys = (Pv > 0) ? y - (double)j * Pv : y;
                    if (Pv > 0) {
                        acc_margin(&acc, ys - L->box[2]);
                        acc_margin(&acc, ys - L->box[3]);
                        if (!(ys >= L->box[2] && ys <= L->box[3])) continue;
                    }
                    if (D->kind == K_BI) {
                        /* both coordinates inside the closed box */
                        bnd = loop_wn(D, L, xs, ys, &acc);
                    } else {
                        /* uni-periodic: only the periodic axis is windowed */
                        bnd = loop_wn(D, L, xs, ys, &acc);
                    }
                }
            }
        } else if (D->kind != K_BI) {
            bnd = pe_wn(D, L, x, y, 0, 0, &acc);
        }
    }
    if (D->kind == K_BI && !bnd) {
        double PP = Pu * Pv;
        double np = D->nx * x + D->ny * y;
        for (int k = 0; k < D->n_pairs && !bnd; k++) {
            double clo = ceil((np - D->phi[k]) / PP), chi = floor((np - D->plo[k]) / PP);
            acc_margin(&acc, (np - D->phi[k]) - (clo - 1.0) * PP);
            acc_margin(&acc, clo * PP - (np - D->phi[k]));
            acc_margin(&acc, (np - D->plo[k]) - chi * PP);
            acc_margin(&acc, (chi + 1.0) * PP - (np - D->plo[k]));
            for (double c = clo; c <= chi && !bnd; c += 1.0) {
                long I = (long)c * D->i0, J = (long)c * D->j0;
                bnd = pe_wn(D, &D->loop[D->pa[k]], x, y, I, J, &acc);
                if (!bnd) bnd = pe_wn(D, &D->loop[D->pb[k]], x, y, I + D->pI[k], J + D->pJ[k], &acc);
            }
        }
    }
    double om = acc.ang / (2.0 * M_PI) + 0.5 * (double)acc.half;
    *w = bnd ? NAN : om;
    if (bnd) *state = OR_BOUNDARY;
    else {
        acc_margin(&acc, om - 0.5);
        *state = (om >= 0.5) ? OR_INSIDE : OR_OUTSIDE;
    }
    if (margin) *margin = acc.margin;
    if (st) {
        st->evals += acc.st.evals; st->nodes += acc.st.nodes; st->chords += acc.st.chords;
        if (acc.st.max_depth > st->max_depth) st->max_depth = acc.st.max_depth;
        st->depth_cap += acc.st.depth_cap;
    }
}

typedef struct {
    const odom_t *D;
    const double *pts;
    double *w, *margin;
    uint8_t *state;
    int64_t i0, i1;
    or_stats st;
} job_t;

static void *worker(void *arg)
{
    job_t *J = (job_t *)arg;
    for (int64_t i = J->i0; i < J->i1; i++)
        query_one(J->D, J->pts[2 * i], J->pts[2 * i + 1], &J->w[i], &J->state[i],
                  J->margin ? &J->margin[i] : NULL, &J->st);
    return NULL;
}

/*
 * Winding numbers and states of n points against one domain.
 *   out_w      omega per point (NaN when BOUNDARY)
 *   out_state  0 outside, 1 inside, 2 boundary
 *   out_margin smallest decision margin met by the point (may be NULL)
 *   stats5     evals, nodes, chords, max depth, depth-cap hits (may be NULL)
 * Returns 0, or 1 (bad argument), 2 (topology), 4 (out of memory).
 */
int or_query_w(int32_t n_loops, const int32_t *loop_offsets, const int32_t *degrees,
               const double *cps, const double *weights, double Pu, double Pv, double eps, int64_t n,
               const double *pts, double *out_w, uint8_t *out_state, double *out_margin,
               int32_t n_threads, int64_t *stats5)
{
    odom_t D;
    int rc = build_dom(&D, n_loops, loop_offsets, degrees, cps, weights, Pu, Pv, eps);
    if (rc) return rc;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if ((int64_t)n_threads > n) n_threads = (int32_t)(n > 0 ? n : 1);
    job_t jobs[256];
    pthread_t th[256];
    for (int t = 0; t < n_threads; t++) {
        memset(&jobs[t], 0, sizeof(job_t));
        jobs[t].D = &D; jobs[t].pts = pts; jobs[t].w = out_w; jobs[t].state = out_state;
        jobs[t].margin = out_margin;
        jobs[t].i0 = n * t / n_threads;
        jobs[t].i1 = n * (t + 1) / n_threads;
    }
    for (int t = 1; t < n_threads; t++) pthread_create(&th[t], NULL, worker, &jobs[t]);
    worker(&jobs[0]);
    for (int t = 1; t < n_threads; t++) pthread_join(th[t], NULL);
    if (stats5) {
        memset(stats5, 0, 5 * sizeof(int64_t));
        for (int t = 0; t < n_threads; t++) {
            stats5[0] += jobs[t].st.evals; stats5[1] += jobs[t].st.nodes;
            stats5[2] += jobs[t].st.chords;
            if (jobs[t].st.max_depth > stats5[3]) stats5[3] = jobs[t].st.max_depth;
            stats5[4] += jobs[t].st.depth_cap;
        }
    }
    free_dom(&D);
    return OR_OK;
}

/* or_query_w of a polynomial domain (weights all 1). */
int or_query(int32_t n_loops, const int32_t *loop_offsets, const int32_t *degrees,
             const double *cps, double Pu, double Pv, double eps, int64_t n, const double *pts,
             double *out_w, uint8_t *out_state, double *out_margin, int32_t n_threads,
             int64_t *stats5)
{
    return or_query_w(n_loops, loop_offsets, degrees, cps, NULL, Pu, Pv, eps, n, pts, out_w, out_state,
                      out_margin, n_threads, stats5);
}

/*
 * Lifted control points (same layout as the input), per-loop homology
 * (2 ints per loop) and, for bi-periodic domains, the pairs (alpha loop,
 * beta loop, I, J per pair; *n_pairs set).  Any output may be NULL.
 */
int or_domain_info(int32_t n_loops, const int32_t *loop_offsets, const int32_t *degrees,
                   const double *cps, double Pu, double Pv, double eps, double *lifted,
                   int32_t *homology, int64_t *pairs, int32_t *n_pairs, double *eps_out)
{
    odom_t D;
    int rc = build_dom(&D, n_loops, loop_offsets, degrees, cps, NULL, Pu, Pv, eps);
    if (rc) return rc;
    long ncp = 0;
    for (int s = 0; s < D.n_segs; s++) ncp += D.seg[s].deg + 1;
    if (lifted) memcpy(lifted, D.cps, sizeof(double) * 2 * (size_t)ncp);
    if (homology)
        for (int l = 0; l < n_loops; l++) {
            homology[2 * l] = D.loop[l].hp;
            homology[2 * l + 1] = D.loop[l].hq;
        }
    if (n_pairs) *n_pairs = D.n_pairs;
    if (pairs)
        for (int k = 0; k < D.n_pairs; k++) {
            pairs[4 * k] = D.pa[k]; pairs[4 * k + 1] = D.pb[k];
            pairs[4 * k + 2] = D.pI[k]; pairs[4 * k + 3] = D.pJ[k];
        }
    if (eps_out) *eps_out = D.eps;
    free_dom(&D);
    return OR_OK;
}

/*
 * Periodically extended winding number (Eq. 9) of one open or closed curve
 * given by its lifted segments, about (x, y), with lattice vector v =
 * (hp Pu, hq Pv); the curve is treated as one loop of an otherwise empty
 * domain.  Returns 0 / 1 (boundary); *w receives omega.
 */
int or_extended_wn(int32_t n_segs, const int32_t *degrees, const double *cps, double Pu,
                   double Pv, int32_t hp, int32_t hq, double eps, double x, double y, double *w)
{
    int32_t lo[2] = {0, n_segs};
    odom_t D;
    int rc = build_dom(&D, 1, lo, degrees, cps, NULL, 0.0, 0.0, eps);
    if (rc) return -rc;
    D.Pu = Pu; D.Pv = Pv;
    oloop_t *L = &D.loop[0];
    L->hp = hp; L->hq = hq;
    L->v[0] = (double)hp * Pu; L->v[1] = (double)hq * Pv;
    L->g0[0] = D.seg[0].P[0]; L->g0[1] = D.seg[0].P[1];
    L->g0v[0] = L->g0[0] + L->v[0]; L->g0v[1] = L->g0[1] + L->v[1];
    double vv = L->v[0] * L->v[0] + L->v[1] * L->v[1];
    L->smin = L->smax = (L->g0v[0] * L->v[0] + L->g0v[1] * L->v[1]) / vv;
    for (int s = 0; s < n_segs; s++)
        for (int i = 0; i <= D.seg[s].deg; i++) {
            double sv = (D.seg[s].P[2 * i] * L->v[0] + D.seg[s].P[2 * i + 1] * L->v[1]) / vv;
            L->smin = fmin(L->smin, sv);
            L->smax = fmax(L->smax, sv);
        }
    int bnd;
    *w = pe_value(&D, L, x, y, 0, 0, &bnd);
    free_dom(&D);
    return bnd;
}
