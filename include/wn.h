/*
 * wn.h -- C ABI of the GB300 (sm_103a) containment-query library.
 *
 * The library classifies query points (u,v) of a trimmed surface's
 * parameter domain against the surface's Bezier trimming loops by the
 * generalized winding number, following Bao, Shen & Wang, "Fast and Robust
 * Point Containment Queries on Trimmed Surface" (arXiv 2510.25159):
 *
 *   - the problem statement and the inside/outside rule: Sec. 4.1;
 *   - the winding number and its additivity / homotopy invariance: Sec. 3.2,
 *     Eq. 1-3 (chord winding = signed angle / 2 pi);
 *   - the recursion: Algorithm 1, with the ellipse bound of Lemma 1 (Eq. 4),
 *     its sub-segment form (Eq. 5) and B = max_i n |P_i - P_{i-1}| (App. A.1);
 *   - periodic domains: lifting to the universal covering space (Sec. 4.3),
 *     periodically extended curves with the line term (Sec. 4.4, Eq. 6-9),
 *     uni-/bi-periodic domains, loop classes and families (Sec. 4.5,
 *     Prop. 1-2, Eq. 10-12) and pairing (App. C, Alg. 3-10).
 *
 * All functions are plain C: pointers, sizes and a CUDA stream.  Nothing here
 * names a C++ or PyTorch type.  Every call returns a wn_status; on failure a
 * thread-local message is available from wn_last_error().
 */
#ifndef WN_H
#define WN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle (cudaStream_t); NULL means the legacy default stream. */
typedef struct CUstream_st *wn_stream;

/* Opaque domain: owns device copies of the lifted loops and the query
 * tables built from them, plus host bookkeeping.  Create with
 * wn_create_domain, free with wn_destroy_domain. */
typedef struct wn_domain wn_domain;

typedef enum {
    WN_OK = 0,
    WN_ERR_ARG = 1,       /* bad argument: size, degree, NaN, negative period, pointer */
    WN_ERR_TOPOLOGY = 2,  /* periodic loops violate Prop. 1 (unpaired or mixed homology,
                             non-coprime (p,q), |homology| > 1 on a cylinder) or the
                             pairing of App. C finds no partner */
    WN_ERR_CUDA = 3,      /* a CUDA runtime call failed (message has the CUDA error) */
    WN_ERR_OOM = 4,       /* device or host allocation failed */
    WN_ERR_LIMIT = 5      /* a size exceeds a documented maximum */
} wn_status;

/* out_inside values (Sec. 4.1: classify by omega; on-boundary per Alg. 1). */
enum { WN_OUTSIDE = 0, WN_INSIDE = 1, WN_BOUNDARY = 2 };

/* precision argument of the query calls */
enum {
    WN_PREC_PLAIN_FP64 = 0, /* Algorithm 1 in FP64 per (query, segment), chord angles
                               summed with atan2: the plain port of the paper's method */
    WN_PREC_MIXED = 1       /* FP32 sweep with error bands and exact crossing counts,
                               FP32 recursion on near pairs, FP64 for every decision
                               whose FP32 error band cannot settle it */
};

#define WN_MAX_DEGREE 7           /* highest Bezier degree accepted */
#define WN_MAX_QUERIES_PER_CALL 2147483647LL

/*
 * Build a domain (Sec. 4.1 input: the trimming loops of one face).
 *
 *   loop_offsets    host int32[n_loops+1]; loop l owns segments
 *                   [loop_offsets[l], loop_offsets[l+1]); loop_offsets[0] == 0.
 *   n_loops         >= 0.
 *   degrees         host int32[n_segs], each in 1..WN_MAX_DEGREE
 *                   (n_segs = loop_offsets[n_loops]).
 *   control_points  host double[2 * sum(degrees[s] + 1)], x,y interleaved,
 *                   segment-major; a segment's first and last points are its
 *                   endpoints gamma(0), gamma(1).  Segments of a loop are
 *                   consecutive end to start; gaps are allowed (open loops).
 *   period_u/_v     0 = not periodic on that axis, > 0 = period.  Periodic
 *                   loops may be stored per-segment wrapped; they are lifted
 *                   (each segment translated by the lattice vector that brings
 *                   its start nearest to the previous segment's end).
 *   epsilon         boundary tolerance of Alg. 1 (strict d < eps);
 *                   <= 0 selects 1e-9 * max(period_u, period_v, extent of the
 *                   control-point box).
 *   out             receives the domain.
 *
 * The caller keeps ownership of every input array; the domain copies what it
 * needs.  Needs a current CUDA device; performs synchronous uploads and, for
 * bi-periodic domains, launches the pairing kernel (App. C, Alg. 8-10) and
 * waits for it.  Errors: WN_ERR_ARG, WN_ERR_TOPOLOGY, WN_ERR_OOM, WN_ERR_CUDA.
 */
wn_status wn_create_domain(const int32_t *loop_offsets, int32_t n_loops,
                           const int32_t *degrees, const double *control_points,
                           double period_u, double period_v, double epsilon,
                           wn_domain **out);

/*
 * wn_create_domain for rational Bezier segments (Sec. 3.1 admits rational
 * p-curves; App. A.1 gives their derivative bounds).
 *
 *   weights         host double[sum(degrees[s] + 1)], one per control point,
 *                   each finite and > 0; NULL is wn_create_domain.  A segment
 *                   whose weights are all equal is the polynomial curve.
 *
 * gamma(t) = sum w_i B_i(t) P_i / sum w_i B_i(t).  The bound of Lemma 1 /
 * Eq. 5 for a rational segment is the smaller of n (W/w) max |P_i - P_j| and
 * n (W/w)^2 max |P_i - P_{i-1}| (W, w: largest and smallest weight); the
 * rest of the method is unchanged (the ellipse bound holds for any curve
 * whose speed B bounds).  The other arguments, the errors and the ownership
 * rules are those of wn_create_domain; a non-positive or non-finite weight is
 * WN_ERR_ARG.
 */
wn_status wn_create_domain_rational(const int32_t *loop_offsets, int32_t n_loops,
                                    const int32_t *degrees, const double *control_points,
                                    const double *weights, double period_u, double period_v,
                                    double epsilon, wn_domain **out);

/* Free a domain (NULL is ignored).  Waits for the device to finish. */
void wn_destroy_domain(wn_domain *domain);

/*
 * Classify n points against one domain (Sec. 4.1; Alg. 1 per segment;
 * Sec. 4.3-4.5 for periodic domains).
 *
 *   points       double[2n], x,y interleaved: device memory, or host memory
 *                (pinned or pageable), in which case the library stages the
 *                copies on `stream`.  Periodic coordinates may lie outside
 *                [0, period); they are reduced modulo the period.
 *   n            0 <= n <= WN_MAX_QUERIES_PER_CALL.
 *   out_winding  double[n] (device or host, may be NULL): omega, NaN for
 *                WN_BOUNDARY.
 *   out_inside   uint8[n]  (device or host, may be NULL): WN_OUTSIDE /
 *                WN_INSIDE (omega >= 1/2) / WN_BOUNDARY.
 *   precision    WN_PREC_PLAIN_FP64 or WN_PREC_MIXED.
 *   stream       work is ordered on this stream.  With device buffers the
 *                call is asynchronous; with any host buffer it returns after
 *                the results are in host memory.
 *
 * Scratch memory (per-query accumulators and the near-pair queues) is owned
 * by the library and grown on demand; the first call of a given size
 * allocates.  Errors: WN_ERR_ARG, WN_ERR_OOM, WN_ERR_CUDA.
 */
wn_status wn_query(const wn_domain *domain, const double *points, int64_t n,
                   double *out_winding, uint8_t *out_inside, int precision,
                   wn_stream stream);

/*
 * Classify the points of many domains in one persistent launch: domain d
 * owns points [point_offsets[d], point_offsets[d+1]).
 *
 *   domains        host array of n_domains domain pointers (repeats allowed).
 *   point_offsets  HOST int64[n_domains+1], non-decreasing, point_offsets[0] == 0.
 *   points, out_winding, out_inside: as in wn_query, concatenated.
 *
 * WN_PREC_MIXED runs one persistent sweep over a global (domain, query-tile)
 * work list ordered by decreasing cost, then the near-pair, FP64 and
 * finalize kernels; with WN_PREC_PLAIN_FP64 one plain kernel is launched per
 * domain.  The tile shape and launch sizes come from wn_set_tuning or the
 * defaults.  A large WN_PREC_MIXED batch with host points (millions of
 * queries) runs as groups of consecutive domains, so that the copies of one
 * group overlap the kernels of the others (two library-owned copy streams,
 * ordered after the caller's earlier work on `stream`); the call still
 * returns after the results are in host memory.  Errors as wn_query.
 */
wn_status wn_query_batched(const wn_domain *const *domains, int32_t n_domains,
                           const int64_t *point_offsets, const double *points,
                           double *out_winding, uint8_t *out_inside, int precision,
                           wn_stream stream);

/*
 * Classify the cell centres ((i + 1/2)/nu, (j + 1/2)/nv), i < nu, j < nv, of a
 * uniform grid over [0,1]^2 scaled by the periods (or the unit square for a
 * planar domain) -- the tessellation use of Sec. 5.4.3.  Points are made on
 * the device.  Bit (j*nu + i) of out_bits (device uint32[(nu*nv + 31)/32],
 * bit k of word k/32 at position k%32) is 1 for WN_INSIDE or WN_BOUNDARY.
 * out_boundary (device int64[1], may be NULL) receives the number of
 * WN_BOUNDARY cells.  1 <= nu, nv <= 65536.
 */
wn_status wn_query_grid_bitmask(const wn_domain *domain, int32_t nu, int32_t nv,
                                uint32_t *out_bits, int64_t *out_boundary, int precision,
                                wn_stream stream);

/*
 * Triangles of a trimmed cell-centre grid (the tessellation application of
 * Sec. 5.4.3): the nu x nv cell centres of a wn_query_grid_bitmask call are
 * the vertices, vertex (i, j) has index j*nu + i; each quad with lower-left
 * vertex (i, j) has corners a = (i, j), b = (i+1, j), c = (i, j+1),
 * d = (i+1, j+1) and triangles (a, b, d) then (a, d, c), counter-clockwise
 * in (u, v); a triangle is kept when its three vertices have their bit set.
 * With wrap_u (wrap_v) != 0 the axis is periodic: indices wrap modulo nu
 * (nv) and the seam quads are included.  Quads are emitted row by row, so
 * the output order is fixed.
 *
 *   bits        device uint32[(nu*nv + 31)/32], the layout of
 *               wn_query_grid_bitmask.
 *   out_tris    device int32[3 * capacity]: vertex indices, 3 per triangle;
 *               only the first `capacity` triangles are written.
 *   out_count   device int64[1]: the number of kept triangles (may exceed
 *               capacity: then call again with a larger buffer).
 *
 * Three kernels on `stream` and a small stream-ordered allocation
 * (cudaMallocAsync) for per-block counts.  Errors: WN_ERR_ARG (null or host
 * pointers, capacity < 0), WN_ERR_LIMIT (nu or nv outside 1..65536, more than
 * 2^31-1 vertices), WN_ERR_OOM, WN_ERR_CUDA.  No counterpart in the paper's
 * text beyond the tessellation it describes.
 */
wn_status wn_grid_triangles(const uint32_t *bits, int32_t nu, int32_t nv, int32_t wrap_u,
                            int32_t wrap_v, int32_t *out_tris, int64_t capacity,
                            int64_t *out_count, wn_stream stream);

/*
 * Several trimmed faces on one geometric surface (multi-patch B-Rep
 * processing, Sec. 5.4.2): a point sampled on a surface is inside when it
 * lies inside, or on the boundary of, ANY face that references the surface.
 *
 *   faces          host array of face pointers, grouped by surface.
 *   surface_faces  HOST int32[n_surfaces+1]: surface s owns
 *                  faces[surface_faces[s] .. surface_faces[s+1]) (may be empty).
 *   point_offsets  HOST int64[n_surfaces+1]: surface s owns points
 *                  [point_offsets[s], point_offsets[s+1]).
 *   points         device double[2 * n], x,y interleaved, 16-byte aligned,
 *                  in each surface's parameter domain.
 *   out_inside     device uint8[n]: 1 inside some face of the point's
 *                  surface (WN_INSIDE or WN_BOUNDARY there), else 0.
 *
 * One batched query over (surface, face) pairs (each surface's points are
 * gathered once per face), then an OR per point; scratch comes from the
 * stream-ordered pool (cudaMallocAsync).  Errors as wn_query_batched, and
 * WN_ERR_LIMIT when the pairs hold more than 2^31-1 point copies.
 */
wn_status wn_query_surfaces(const wn_domain *const *faces, const int32_t *surface_faces,
                            int32_t n_surfaces, const int64_t *point_offsets, const double *points,
                            uint8_t *out_inside, int precision, wn_stream stream);

/*
 * Topological filtering of B-Rep intersection curves (Sec. 5.4.2): pieces of
 * the raw intersection curves, already split at the face's trimming
 * boundaries, are classified by their midpoints 0.5 (a + b).
 *
 *   pieces     device double[4 * n]: (ax, ay, bx, by) per piece, 32-byte aligned.
 *   out_state  device uint8[n]: the midpoint's WN_OUTSIDE / WN_INSIDE /
 *              WN_BOUNDARY (keep the piece when it is not WN_OUTSIDE).
 *
 * Errors as wn_query.
 */
wn_status wn_query_midpoints(const wn_domain *domain, const double *pieces, int64_t n,
                             uint8_t *out_state, int precision, wn_stream stream);

/*
 * Tuning knobs of the mixed path (0 keeps the current value for the first
 * three, a negative value keeps it for the last three):
 *   tile_queries_per_thread  1, 2 or 4 queries per sweep thread
 *   sweep_ctas_per_sm        persistent sweep CTAs per SM (1..8)
 *   near_ctas_per_sm         near-pair kernel CTAs per SM (1..16)
 *   use_graph                1 = capture each distinct batched call in a CUDA
 *                            graph and replay it; 0 = plain launches
 *   tree                     1 = sweep record clusters (gap angles of far
 *                            clusters from their series expansion); 0 = sweep
 *                            every record for every query
 *   bucket                   1 = order the queries by spatial cell before the
 *                            sweep (results do not depend on it)
 */
wn_status wn_set_tuning(int32_t tile_queries_per_thread, int32_t sweep_ctas_per_sm,
                        int32_t near_ctas_per_sm, int32_t use_graph, int32_t tree,
                        int32_t bucket);

/*
 * Autotuner of the mixed path.  Times candidate launch shapes on the
 * caller's own batch and keeps the fastest for the following calls:
 * coordinate descent from the current setting over queries per sweep thread
 * {1, 2}, sweep CTAs per SM {2, 3, 4, 6}, near-pair CTAs per SM {4, 8, 16},
 * the spatial bucket size {32, 64, 128} queries, bucketing on / off, the
 * FP32 near-walk depth cap {16, 22, 28}, the near-pair draw {64, 128, 256},
 * the refill threshold {8, 16, 24} (see wn_set_near_tuning) and the
 * flat-sweep record limit {0, 16, 32} (see wn_set_flat_records);
 * each candidate runs one
 * warm-up call and `iterations` timed calls (CUDA events on `stream`).
 *   domains, n_domains, point_offsets, points: as in wn_query_batched, with
 *                points in DEVICE memory (results go to library scratch).
 *   iterations   timed calls per candidate, 1..100.
 *   best_ms      host double[1] or NULL: mean time per call of the kept shape.
 * Synchronises `stream`.  Errors as wn_query_batched.
 */
wn_status wn_autotune(const wn_domain *const *domains, int32_t n_domains,
                      const int64_t *point_offsets, const double *points, int32_t iterations,
                      double *best_ms, wn_stream stream);

/* Current tuning: the first min(n_out, 12) of (queries per sweep thread,
 * sweep CTAs per SM, near-pair CTAs per SM, graph replay, tree sweep, bucket
 * cell size in queries, spatial bucketing on/off, FP32 near-walk depth cap,
 * near-pair draw, refill threshold, flat-sweep record limit, grid tile
 * width) into out (host int32[n_out]). */
wn_status wn_get_tuning(int32_t *out, int32_t n_out);

/*
 * Knobs of the FP32 near-pair walk (Alg. 1 on the pairs the sweep could not
 * settle; 0 keeps the current value):
 *   depth_cap  12..30: subdivision depth after which a pair's undecided tail
 *              goes to the FP64 walk.  Lemma 2 bounds the depth a pair needs
 *              by about log2(B / max(eps, d)) for a query at distance d; a
 *              lower cap moves more near-curve pairs to FP64, a higher one
 *              walks longer in FP32 where the error bands may still fail.
 *              Results do not depend on it (default 22).
 *   chunk      pairs a warp takes from the queue per atomic, a multiple of
 *              32 in 32..1024 (default 128).
 *   refill     idle lanes (1..32) that make a warp load new pairs (default 16).
 * Errors: WN_ERR_ARG for values outside those ranges.
 */
wn_status wn_set_near_tuning(int32_t depth_cap, int32_t chunk, int32_t refill);

/*
 * With the tree sweep on, planar domains of at most max_records records
 * (0..4096; 0 = none) take the flat sweep instead: every query against every
 * record, staged in shared memory, without spatial bucketing.  For a few
 * dozen segments that costs less than the tree's dependent node steps.
 * Results do not depend on it beyond rounding of the gap angles (the flat
 * sweep sums them per record, the tree per record or by expansions).
 * Default 0: on the batched B-Rep-shaped workload the tree sweep was as
 * fast or faster for every limit tried.  Errors: WN_ERR_ARG outside 0..4096.
 */
wn_status wn_set_flat_records(int32_t max_records);

/*
 * Tile shape of the grid queries (wn_query_grid_bitmask) in the tree sweep:
 * a warp sweeps 64 cells, `width` wide (8, 16, 32 or 64) and 64 / width
 * high.  Wide tiles keep a warp's queries on few rows, so their +x rays
 * cross the same segments; square tiles keep them close to one another.
 * Results do not depend on it.  Default 8.  Errors: WN_ERR_ARG.
 */
wn_status wn_set_grid_tile(int32_t width);

/*
 * Test hook: caps on the near-pair and FP64-pair queues of the mixed path
 * (0 = the allocated capacity).  A pair that does not fit sends its query to
 * the FP64 recomputation, as a full queue does, so results do not change;
 * wn_get_stats reports the pairs that did not fit in `overflow`.
 */
wn_status wn_set_queue_limits(int64_t near_pairs, int64_t fp64_pairs);

/* Counters of the last query call on this thread's device, read after the
 * stream is synchronised: queries, near pairs, pairs escalated to FP64,
 * queries recomputed in FP64, pairs that did not fit the near or FP64
 * queue (their queries were recomputed in FP64), FP64 walks that reached
 * the depth cap of 64 and were reported WN_BOUNDARY (unreachable for points
 * farther than eps from the curve, Lemma 2); and the number of kernels the
 * last query call (mixed or plain) launched. */
typedef struct {
    int64_t queries;
    int64_t near_pairs;
    int64_t fp64_pairs;
    int64_t fp64_queries;
    int64_t overflow;
    int64_t depth_cap;
    int64_t kernels;
} wn_stats;

wn_status wn_get_stats(wn_stats *out);

/*
 * The queries the last mixed call on this thread's device recomputed in
 * FP64 (the classification band or a flag of Sec. 4.1's decision, see
 * wn_get_stats fp64_queries), for verification: *n_out receives their
 * number and out_idx (host int64[capacity]) the first min(n, capacity)
 * query indices of the call (cell indices j*nu + i for a grid), in no
 * particular order.  Synchronises the device.  Errors: WN_ERR_ARG.
 */
wn_status wn_last_escalated(int64_t *out_idx, int64_t capacity, int64_t *n_out);

/*
 * Verification hook: the bounds of |gamma'(t)| that the walks of Algorithm 1
 * use for one rational Bezier segment (App. A.1): out9[0] = B, the smaller
 * of App. A.1's two bounds on the whole segment; out9[1 + j] = the bound on
 * the eighth [j/8, (j+1)/8] of its parameter interval (each at most B): 8
 * times App. A.1's bound of that eighth as a rational Bezier curve of its
 * own (homogeneous de Casteljau subdivision), with allowances for the
 * subdivision's rounding.  A node of a walk inside one eighth is far when
 * ra + rb > B_j (b - a) + 2 eps as well as under Eq. 5 with B.
 * control_points: 2 (degree + 1) doubles (x0, y0, x1, y1, ...); weights:
 * degree + 1 doubles > 0; degree 1..7.  Host computation only (no device
 * call).  Errors: WN_ERR_ARG.
 */
wn_status wn_rational_bounds(const double *control_points, const double *weights, int32_t degree, double *out9);

/*
 * Verification hook: the FP32 angle the mixed path assigns to a gap between
 * consecutive segments seen from a query (its share of Eq. 3's chord angles
 * in the crossing form), out[i] = angle of the vector (x[i], y[i]) in
 * (-pi, pi].  For |y| <= x / 4 it is the odd series of atan(y / x) to the
 * t^11 term (remainder below |t|^13 / 13 <= 1.2e-9) in FP32, else atan2f.
 * y, x, out: DEVICE float[n].  Asynchronous on `stream`.  Errors: WN_ERR_ARG.
 */
wn_status wn_eval_gap_angle(const float *y, const float *x, float *out, int64_t n, wn_stream stream);

/*
 * Per-kernel device time of the mixed path, for measurement.  With on != 0
 * every following WN_PREC_MIXED call records CUDA events around each of its
 * kernels on the call's own stream (so the times are those of the stream the
 * kernels run on); on == 0 stops recording and drops what was recorded.
 * wn_kernel_times synchronises the device, writes the summed milliseconds of
 * the six stages [query bucketing (3 kernels), sweep, near pairs FP32, pairs
 * FP64, finalize, queries FP64] into ms6 (host double[6]) and the number of
 * recorded calls into *n_calls, then clears the record.
 */
wn_status wn_set_profiling(int32_t on);
wn_status wn_kernel_times(double *ms6, int64_t *n_calls);

/*
 * Work tallies of the tree sweep, for measurement (no counterpart in the
 * paper).  With on != 0 the following WN_PREC_MIXED calls on this thread's
 * device run a counting build of the sweep kernel -- the same decisions and
 * arithmetic, plus per-warp tallies -- and add to twelve counters, which
 * wn_set_work_counting also clears.  wn_sweep_work synchronises, writes the
 * first min(n_out, 12) into out (host int64[n_out]) and clears them:
 *   [0] (query, node) tests          [1] nodes whose crossings telescoped
 *   [2] gap-angle expansion sums     [3] their terms
 *   [4] (query, record) tests with the near check (Alg. 1's first step)
 *   [5] record tests for crossings and gap angle
 *   [6] record tests for crossings only
 *   [7] exact FP64 recomputations of a sign
 *   [8] ellipse tests (Eq. 5) of records whose enclosing circle held the query
 *   [9] control-point box tests of records whose ellipse held the query
 *   [10] node visits of warps and [11] record iterations of warps in the
 *        leaves (per warp, each serving its 32 or 64 query slots: [0] and
 *        [4]-[6] over these, divided by the slots, is the SIMT efficiency)
 * Zeros when the flat sweep ran (wn_set_tuning tree = 0) or nothing ran.
 */
wn_status wn_set_work_counting(int32_t on);
wn_status wn_sweep_work(int64_t *out, int32_t n_out);

/*
 * Work tallies of the counting build of the FP32 near-pair walk (enabled by
 * wn_set_work_counting with the sweep's): wn_near_work writes into out4
 * (host int64[4]) and clears
 *   [0] nodes tested with the ellipse of Eq. 5   [1] nodes accepted as far
 *   [2] evaluations of gamma(m)                  [3] sum of their degrees
 */
wn_status wn_near_work(int64_t *out4);

/*
 * wn_query_noalloc -- the WN_PREC_MIXED query of wn_query for one domain,
 * without any memory allocation.  (The paper has no counterpart: this is a
 * deployment variant of the same computation.)
 *
 * Some callers cannot let the library call cudaMalloc at query time: code
 * running inside a custom device allocator or memory-pool callback (a nested
 * allocation would re-enter the allocator), real-time or certified loops
 * that forbid allocation once they have started, and processes held to a
 * fixed device-memory budget.  This entry point keeps all of its scratch
 * (per-query accumulators, the near-pair and FP64 queues, the work list)
 * in one fixed-size device array that is part of the library image (about
 * 12.0 MiB per device).  The library is built without relocatable device
 * code and CUDA loads modules lazily by default, so the array and the
 * kernels' code are placed on a device when the FIRST call on that device
 * loads them; that call also launches every kernel a call can use once on
 * an empty work list (loading its code and reserving its local memory), so
 * it may allocate device memory implicitly.
 * Make it at start-up (n = 0 is enough: it does the set-up and returns),
 * outside allocator callbacks and stream capture, or run the process with
 * CUDA_MODULE_LOADING=EAGER; from then on the process holds the array until
 * it exits, and later calls make no cudaMalloc, cudaFree or other
 * allocating call.
 *
 *   domain       from wn_create_domain (not modified).
 *   points       DEVICE double[2n], x,y interleaved, 16-byte aligned.
 *   n            0..WN_NOALLOC_MAX_QUERIES; larger n returns WN_ERR_LIMIT
 *                (split the batch, or use wn_query).
 *   out_winding  DEVICE double[n] or NULL; out_inside DEVICE uint8[n] or NULL
 *                (same meaning as in wn_query).
 *   stream       all work is queued on this stream; the call is asynchronous.
 *
 * Results: the same WN_OUTSIDE / WN_INSIDE / WN_BOUNDARY states as
 * wn_query(..., WN_PREC_MIXED, ...) on the same inputs, and windings within
 * the mixed path's tolerance of its windings (this call runs a fixed launch
 * shape without spatial bucketing, so warps group the queries differently).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call on a device shares the one array, and each call
 * re-initialises what it needs, so calls that may overlap on the GPU (on
 * different streams without ordering between them) race and give wrong
 * results: order them on one stream, or with events.
 * Errors: WN_ERR_ARG (NULL domain, n < 0, host or misaligned pointers, a
 * domain created on another device than the current one), WN_ERR_LIMIT (n
 * too large), WN_ERR_CUDA.  No message is recorded for wn_last_error
 * (recording one could allocate host memory).
 */
#define WN_NOALLOC_MAX_QUERIES 65536
wn_status wn_query_noalloc(const wn_domain *domain, const double *points, int64_t n,
                           double *out_winding, uint8_t *out_inside, wn_stream stream);

/* Thread-local description of the last failure ("" when none). */
const char *wn_last_error(void);

/* Library version string. */
const char *wn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WN_H */
