// wn_api.cu -- the C ABI of include/wn.h: domain lifetime, scratch memory,
// the batched work list, host-buffer staging, tuning and counters.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "wn.h"
#include "wn_internal.h"

using namespace wn;

namespace {

thread_local std::string g_err;
std::mutex g_mu;
Tuning g_tun;
// Test hook: upper limits on the near-pair and FP64-pair queues (0: the
// allocated capacity).  Pairs beyond a limit send their query to the FP64
// recomputation, exactly as a full queue does.
int64_t g_lim_near = 0, g_lim_f64 = 0;

// Batch tables of one list of domains (see build_tables).
struct Tables {
    std::vector<const wn_domain *> key_doms;
    std::vector<int64_t> key_offsets;
    int key = 0;
    int n_units = 0, n_flat = 0, n_cells = 0, n_bchunks = 0;
    int64_t n_runoff = 0;               // run_off entries: the cells of each run's domain, summed over runs
    bool flat0 = false;                 // a one-domain list: its domain takes the flat sweep
    int4 *units = nullptr;
    DomDev *doms = nullptr;
    int64_t *offsets = nullptr;
    int4 *dcell = nullptr;
    int4 *bchunks = nullptr;
    int64_t cap_units = 0, cap_doms = 0, cap_off = 0, cap_dbin = 0, cap_bchunks = 0;
};

// A large mixed batch from host buffers runs as G groups of domains, so that
// each group's copies overlap the other groups' kernels.  With the copies
// taking C (about 25 bytes per query at ~200 GB/s) a split hides C (1 - 1/G)
// and costs about kGroupCostMs per extra group (the latency-bound tails of
// each group's kernels), so G = sqrt(C / kGroupCostMs), at most kMaxGroups.
constexpr int kMaxGroups = 8;
constexpr int kMaxGraphs = 256;
constexpr int64_t kGroupMinQueries = 1 << 21;
constexpr double kGroupCostMs = 0.3;
constexpr double kCopyMsPerQuery = 25.0 / 200e9 * 1e3;

int group_count(int64_t n, int32_t n_domains)
{
    if (n < kGroupMinQueries || n_domains < 2) return 1;
    const int G = (int)std::lround(std::sqrt((double)n * kCopyMsPerQuery / kGroupCostMs));
    return std::max(1, std::min({G, kMaxGroups, (int)n_domains}));
}

struct DevState {
    bool init = false;
    int n_sm = 0;
    Work W;
    // host-buffer staging
    double *st_pts = nullptr;
    double *st_w = nullptr;
    uint8_t *st_st = nullptr;
    int64_t cap_st = 0;
    // batch tables, reused while the batch layout does not change: the
    // whole list's, and those of the groups of a large host-buffer batch
    Tables main;
    Tables grp[kMaxGroups];
    // copy streams and events of a grouped host-buffer batch
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev[2 * kMaxGroups + 2] = {};
    wn_stats last{};
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    // work tallies of the counting build of the tree sweep
    bool counting = false;
    unsigned long long *d_work = nullptr;
    // CUDA graphs of captured mixed calls, each replayed while its launch
    // parameters (batch layout, buffers, stream, tuning) recur; at most
    // kMaxGraphs, the oldest dropped first (a tessellation run replays one
    // graph per face)
    std::vector<std::pair<std::vector<uintptr_t>, cudaGraphExec_t>> graphs;
    int64_t graph_launches = 0;
};
DevState g_dev[64];

// A captured graph names buffers and tables by address: any reallocation
// drops it.
void drop_graphs()
{
    for (DevState &S : g_dev)
        if (!S.graphs.empty()) {
            for (auto &g : S.graphs) cudaGraphExecDestroy(g.second);
            S.graphs.clear();
        }
}

wn_status fail(wn_status s, const std::string &m)
{
    g_err = m;
    return s;
}

wn_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(e == cudaErrorMemoryAllocation ? WN_ERR_OOM : WN_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

bool is_device_ptr(const void *p)
{
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void drop_graphs();

template <typename T>
cudaError_t grow(T *&p, int64_t &cap, int64_t need)
{
    if (need <= cap && p) return cudaSuccess;
    drop_graphs();
    if (p) {
        cudaDeviceSynchronize();
        cudaFree(p);
        p = nullptr;
    }
    cap = 0;
    cudaError_t e = cudaMalloc(&p, (size_t)std::max<int64_t>(need, 1) * sizeof(T));
    if (e == cudaSuccess) cap = need;
    return e;
}

DevState *dev_state(wn_status &st)
{
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess || d < 0 || d >= 64) {
        st = cuda_fail(e == cudaSuccess ? cudaErrorInvalidDevice : e, "cudaGetDevice");
        return nullptr;
    }
    DevState &S = g_dev[d];
    if (!S.init) {
        e = cudaDeviceGetAttribute(&S.n_sm, cudaDevAttrMultiProcessorCount, d);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaDeviceGetAttribute");
            return nullptr;
        }
        e = cudaMalloc(&S.W.counters, CNT_N * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaMalloc counters");
            return nullptr;
        }
        cudaMemset(S.W.counters, 0, CNT_N * sizeof(unsigned long long));
        bin_blocks_per_sm(0);      // the bucketing grids' occupancy, cached before any capture
        bin_blocks_per_sm(1);
        S.init = true;
    }
    st = WN_OK;
    return &S;
}

// Scratch of the mixed path sized for n queries.
cudaError_t ensure_work(Work &W, int64_t n, int64_t near_expected)
{
    cudaError_t e = cudaSuccess;
    int64_t nq = std::max<int64_t>(n, 1024);
    if (nq > W.cap_q) {
        int64_t c0 = W.cap_q, c1 = W.cap_q, c3 = W.cap_q;
        if ((e = grow(W.acc2, c0, nq)) != cudaSuccess) return e;
        if ((e = grow(W.theta, c1, nq)) != cudaSuccess) return e;
        if ((e = grow(W.esc_q, c3, nq)) != cudaSuccess) return e;
        W.cap_q = nq;
    }
    // near pairs: twice the expected count (from the records' circle areas),
    // at least one per four queries and 4M (an overflowing pair sends its
    // query to the FP64 recomputation), but at most a quarter of the free
    // device memory: a smaller queue only moves the pairs that do not fit
    // to that recomputation
    int64_t need_near = std::max<int64_t>(std::max<int64_t>(1 << 22, nq / 4), 2 * near_expected);
    if (need_near > W.cap_near) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            const int64_t room = (int64_t)(free_b / 4 / sizeof(Item)) + W.cap_near;
            need_near = std::max<int64_t>(std::min(need_near, room), std::min<int64_t>(need_near, 1 << 22));
        }
    }
    if ((e = grow(W.near_items, W.cap_near, need_near)) != cudaSuccess) return e;
    const int64_t need_f64 = std::max<int64_t>(1 << 18, nq / 8);
    if ((e = grow(W.f64_items, W.cap_f64, need_f64)) != cudaSuccess) return e;
    if (nq > W.cap_bin_q || !W.perm) {
        int64_t c0 = W.cap_bin_q, c1 = W.cap_bin_q;
        if ((e = grow(W.cell_of, c0, nq)) != cudaSuccess) return e;
        if ((e = grow(W.perm, c1, nq)) != cudaSuccess) return e;
        W.cap_bin_q = nq;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char *wn_last_error(void) { return g_err.c_str(); }

const char *wn_version(void) { return "wn 0.1 (sm_103a)"; }

wn_status wn_create_domain_rational(const int32_t *loop_offsets, int32_t n_loops, const int32_t *degrees,
                                    const double *control_points, const double *weights, double period_u,
                                    double period_v, double epsilon, wn_domain **out)
{
    if (!out) return fail(WN_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::string err;
    int rc;
    try {
        rc = build_domain(loop_offsets, n_loops, degrees, control_points, weights, period_u, period_v,
                          epsilon, out, err);
    } catch (const std::bad_alloc &) {
        return fail(WN_ERR_OOM, "host allocation failed");
    }
    if (rc != 0) return fail((wn_status)rc, err);
    g_err.clear();
    return WN_OK;
}

wn_status wn_rational_bounds(const double *control_points, const double *weights, int32_t degree, double *out9)
{
    if (!control_points || !weights || !out9) return fail(WN_ERR_ARG, "NULL pointer");
    if (degree < 1 || degree > kMaxDeg) return fail(WN_ERR_ARG, "degree must be 1..7");
    for (int i = 0; i <= degree; i++) {
        if (!(weights[i] > 0.0) || !std::isfinite(weights[i])) return fail(WN_ERR_ARG, "weights must be finite and > 0");
        if (!std::isfinite(control_points[2 * i]) || !std::isfinite(control_points[2 * i + 1]))
            return fail(WN_ERR_ARG, "control points must be finite");
    }
    out9[0] = rational_segment_bound(control_points, weights, degree);
    rational_eighth_bounds(control_points, weights, degree, out9[0], out9 + 1);
    g_err.clear();
    return WN_OK;
}

wn_status wn_create_domain(const int32_t *loop_offsets, int32_t n_loops, const int32_t *degrees,
                           const double *control_points, double period_u, double period_v,
                           double epsilon, wn_domain **out)
{
    return wn_create_domain_rational(loop_offsets, n_loops, degrees, control_points, nullptr, period_u,
                                     period_v, epsilon, out);
}

void wn_destroy_domain(wn_domain *d)
{
    if (!d) return;
    std::lock_guard<std::mutex> lk(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != d->device) cudaSetDevice(d->device);
    cudaDeviceSynchronize();
    for (void *p : d->allocs) cudaFree(p);
    if (cur != d->device) cudaSetDevice(cur);
    drop_graphs();
    // batch tables that name this domain must be rebuilt
    for (DevState &S : g_dev)
        for (int t = 0; t <= kMaxGroups; t++) {
            Tables &T = t == 0 ? S.main : S.grp[t - 1];
            for (const wn_domain *k : T.key_doms)
                if (k == d) {
                    T.key_doms.clear();
                    break;
                }
        }
    delete d;
}

wn_status wn_set_tuning(int32_t qpt, int32_t sweep_ctas_per_sm, int32_t near_ctas_per_sm,
                        int32_t use_graph, int32_t tree, int32_t bucket)
{
    std::lock_guard<std::mutex> lk(g_mu);
    drop_graphs();
    if (qpt != 0 && qpt != 1 && qpt != 2 && qpt != 4) return fail(WN_ERR_ARG, "qpt must be 1, 2 or 4");
    if (sweep_ctas_per_sm < 0 || sweep_ctas_per_sm > 8) return fail(WN_ERR_ARG, "sweep_ctas_per_sm 1..8");
    if (near_ctas_per_sm < 0 || near_ctas_per_sm > 16) return fail(WN_ERR_ARG, "near_ctas_per_sm 1..16");
    if (qpt) g_tun.qpt = qpt;
    if (sweep_ctas_per_sm) g_tun.sweep_ctas_per_sm = sweep_ctas_per_sm;
    if (near_ctas_per_sm) g_tun.near_ctas_per_sm = near_ctas_per_sm;
    if (use_graph >= 0) g_tun.use_graph = use_graph;
    if (tree >= 0) g_tun.tree = tree != 0;
    if (bucket >= 0) g_tun.bucket = bucket != 0;
    return WN_OK;
}

wn_status wn_set_near_tuning(int32_t depth_cap, int32_t chunk, int32_t refill)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (depth_cap != 0 && (depth_cap < kDepthCap32Min || depth_cap > kDepthCap32Max))
        return fail(WN_ERR_ARG, "depth_cap outside 12..30");
    if (chunk != 0 && (chunk < kNearChunkMin || chunk > kNearChunkMax || (chunk & 31)))
        return fail(WN_ERR_ARG, "chunk must be a multiple of 32 in 32..1024");
    if (refill != 0 && (refill < 1 || refill > 32)) return fail(WN_ERR_ARG, "refill outside 1..32");
    drop_graphs();
    if (depth_cap) g_tun.near_depth = depth_cap;
    if (chunk) g_tun.near_chunk = chunk;
    if (refill) g_tun.near_refill = refill;
    return WN_OK;
}

wn_status wn_set_flat_records(int32_t max_records)
{
    if (max_records < 0 || max_records > 4096) return fail(WN_ERR_ARG, "max_records outside 0..4096");
    std::lock_guard<std::mutex> lk(g_mu);
    drop_graphs();
    g_tun.flat_max = max_records;
    return WN_OK;
}

wn_status wn_set_grid_tile(int32_t width)
{
    if (width != 8 && width != 16 && width != 32 && width != 64) return fail(WN_ERR_ARG, "width must be 8, 16, 32 or 64");
    std::lock_guard<std::mutex> lk(g_mu);
    drop_graphs();
    g_tun.grid_tile_w = width;
    return WN_OK;
}

wn_status wn_set_queue_limits(int64_t near_pairs, int64_t fp64_pairs)
{
    if (near_pairs < 0 || fp64_pairs < 0) return fail(WN_ERR_ARG, "limits must be >= 0");
    std::lock_guard<std::mutex> lk(g_mu);
    drop_graphs();
    g_lim_near = near_pairs;
    g_lim_f64 = fp64_pairs;
    return WN_OK;
}

// Small planar domains take the flat sweep (every query against every
// record, staged in shared memory): a handful of records costs less swept
// flat than walked as a tree, whose node steps wait on dependent loads.
static bool flat_domain(const wn_domain *d, bool grid_tiled)
{
    return !grid_tiled && g_tun.tree && g_tun.flat_max > 0 && d->dev.kind == DK_PLANAR &&
           d->sweep_records <= g_tun.flat_max;
}

// The batch tables of one list of domains: the work list of (domain, query
// tile) units in decreasing cost order (the tree sweep's units, then the
// flat sweep's), the domain records, the offsets and the bucketing layout
// (tree domains only), uploaded once and reused while the list, its query
// offsets and the launch shape are unchanged.
static wn_status build_tables(DevState *S, Tables &T, const wn_domain *const *domains, int32_t n_domains,
                              const int64_t *offsets, int key, bool grid_tiled, const PointSrc &src,
                              int32_t grid_nv, int64_t tile)
{
    const bool same = T.key == key && T.key_doms.size() == (size_t)n_domains &&
                      (n_domains == 1 ? T.flat0 == flat_domain(domains[0], grid_tiled)
                                      : std::equal(T.key_doms.begin(), T.key_doms.end(), domains)) &&
                      T.key_offsets.size() == (size_t)n_domains + 1 &&
                      std::equal(T.key_offsets.begin(), T.key_offsets.end(), offsets);
    cudaError_t e;
    if (same) {
        // the shared cell scratch may have been sized for a smaller list since
        if ((e = grow(S->W.cell_cnt, S->W.cap_cells, (int64_t)T.n_cells)) != cudaSuccess ||
            (e = grow(S->W.bin_chunk, S->W.cap_chunk, ((int64_t)T.n_cells + 4095) / 4096)) != cudaSuccess ||
            (e = grow(S->W.run_off, S->W.cap_runoff, std::max<int64_t>(1, T.n_runoff))) != cudaSuccess)
            return cuda_fail(e, "cells");
        return WN_OK;
    }
    T.key_doms.clear();
    std::vector<DomDev> h_doms(n_domains);
    std::vector<std::pair<double, int4>> u, uf;
    std::vector<char> flat(n_domains);
    // a tree unit's .w: its first position in the bucketed order, which
    // holds the tree domains' queries only (the flat ones are not bucketed)
    int64_t pbase = 0;
    for (int d = 0; d < n_domains; d++) {
        h_doms[d] = domains[d]->dev;
        flat[d] = flat_domain(domains[d], grid_tiled);
        // positions to sweep: the queries, or the cells of every tile of the grid
        const int th = 64 >> src.tile_lw;
        const int64_t cnt = grid_tiled ? (int64_t)src.tiles_x * ((grid_nv + th - 1) / th) * 64 : offsets[d + 1] - offsets[d];
        // sweep cost of one query of this domain: records of every instance
        const double work = (double)std::max<int64_t>(domains[d]->sweep_records, 1);
        const int64_t t = flat[d] ? (int64_t)kSweepThreads * kFlatQpt : tile;
        for (int64_t q0 = 0; q0 < cnt; q0 += t) {
            const int64_t c = std::min(t, cnt - q0);
            (flat[d] ? uf : u).push_back({work * (double)c, make_int4(d, (int)(offsets[d] + q0), (int)c,
                                                                      flat[d] ? 0 : (int)(pbase + q0))});
        }
        if (!flat[d]) pbase += cnt;
    }
    auto by_cost = [](const std::pair<double, int4> &a, const std::pair<double, int4> &b) { return a.first > b.first; };
    std::stable_sort(u.begin(), u.end(), by_cost);
    std::stable_sort(uf.begin(), uf.end(), by_cost);
    T.n_units = (int)u.size();
    T.n_flat = (int)uf.size();
    T.flat0 = n_domains == 1 && flat[0];
    u.insert(u.end(), uf.begin(), uf.end());
    std::vector<int4> h_units(u.size());
    for (size_t i = 0; i < u.size(); i++) h_units[i] = u[i].second;
    if ((e = grow(T.units, T.cap_units, (int64_t)u.size())) != cudaSuccess) return cuda_fail(e, "units");
    if ((e = grow(T.doms, T.cap_doms, (int64_t)n_domains)) != cudaSuccess) return cuda_fail(e, "doms");
    if ((e = grow(T.offsets, T.cap_off, (int64_t)n_domains + 1)) != cudaSuccess) return cuda_fail(e, "offsets");
    if ((e = cudaMemcpy(T.units, h_units.data(), u.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "upload units");
    if ((e = cudaMemcpy(T.doms, h_doms.data(), n_domains * sizeof(DomDev), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "upload domains");
    if ((e = cudaMemcpy(T.offsets, offsets, (n_domains + 1) * sizeof(int64_t), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return cuda_fail(e, "upload offsets");
    // spatial buckets: about cell_q queries per cell; G x G cells per
    // domain (the bucketing kernel lays them over the domain's box),
    // G <= kBinMaxG so that one CTA holds a domain's cell counters;
    // the bucketing kernels take each domain's queries in runs of a few
    // queries per cell
    std::vector<int4> dcell(n_domains);
    std::vector<int4> bch;
    int64_t ncell = 0, nro = 0;
    for (int d = 0; d < n_domains; d++) {
        const int64_t cnt = flat[d] ? 0 : offsets[d + 1] - offsets[d];    // the flat sweep needs no bucketing
        const int G = cnt == 0 ? 0 : (int)std::min<double>((double)kBinMaxG, std::max<double>(1.0, std::floor(std::sqrt((double)cnt / (double)g_tun.cell_q))));
        dcell[d] = make_int4((int)ncell, G, 0, 0);
        ncell += (int64_t)G * G;
        // runs of about kBinRunPerCell queries per cell, 4096 to kBinRunMax
        // queries (the kernels draw them largest first from a counter)
        const int64_t csz = std::min<int64_t>(kBinRunMax, std::max<int64_t>(4096, (int64_t)kBinRunPerCell * G * G));
        for (int64_t q0 = 0; q0 < cnt; q0 += csz) {
            bch.push_back(make_int4(d, (int)(offsets[d] + q0), (int)std::min(csz, cnt - q0), (int)std::min<int64_t>(nro, INT32_MAX)));
            nro += (int64_t)G * G;
        }
    }
    // largest runs first: the kernels take them in this order from a counter
    std::stable_sort(bch.begin(), bch.end(), [](const int4 &a, const int4 &b) { return a.z > b.z; });
    if (ncell > INT32_MAX || nro > INT32_MAX) return fail(WN_ERR_LIMIT, "too many query cells");
    if ((e = grow(T.bchunks, T.cap_bchunks, (int64_t)bch.size())) != cudaSuccess) return cuda_fail(e, "cells");
    T.n_bchunks = (int)bch.size();
    if (!bch.empty() &&
        (e = cudaMemcpy(T.bchunks, bch.data(), bch.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "upload cells");
    if ((e = grow(T.dcell, T.cap_dbin, (int64_t)n_domains)) != cudaSuccess) return cuda_fail(e, "cells");
    if ((e = grow(S->W.cell_cnt, S->W.cap_cells, ncell)) != cudaSuccess) return cuda_fail(e, "cells");
    if ((e = grow(S->W.bin_chunk, S->W.cap_chunk, (ncell + 4095) / 4096)) != cudaSuccess)
        return cuda_fail(e, "cells");
    if ((e = grow(S->W.run_off, S->W.cap_runoff, std::max<int64_t>(1, nro))) != cudaSuccess)
        return cuda_fail(e, "cells");
    T.n_cells = (int)ncell;
    T.n_runoff = nro;
    if ((e = cudaMemcpy(T.dcell, dcell.data(), n_domains * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "upload cells");
    T.key_doms.assign(domains, domains + n_domains);
    T.key_offsets.assign(offsets, offsets + n_domains + 1);
    T.key = key;
    drop_graphs();
    return WN_OK;
}

// The shared scratch with one list's tables in place (queue capacities cut
// to the test limits, when set).
static Work work_with(const DevState *S, const Tables &T)
{
    Work W = S->W;
    if (g_lim_near > 0) W.cap_near = std::min(W.cap_near, g_lim_near);
    if (g_lim_f64 > 0) W.cap_f64 = std::min(W.cap_f64, g_lim_f64);
    W.units = T.units;
    W.doms = T.doms;
    W.offsets = T.offsets;
    W.dcell = T.dcell;
    W.bchunks = T.bchunks;
    W.n_cells = T.n_cells;
    W.n_bchunks = T.n_bchunks;
    return W;
}

static double near_expected_of(const wn_domain *const *domains, int32_t n_domains, const int64_t *offsets)
{
    double x = 0.0;
    for (int d = 0; d < n_domains; d++) x += (double)(offsets[d + 1] - offsets[d]) * domains[d]->near_density;
    return std::fmin(x, 4e9);
}

static wn_status query_impl(const wn_domain *const *domains, int32_t n_domains,
                            const int64_t *offsets, const double *points, double *out_w,
                            uint8_t *out_st, int precision, cudaStream_t stream, PointSrc grid,
                            uint32_t *bits, int64_t *nbound)
{
    if (n_domains < 0 || !offsets || (n_domains > 0 && !domains))
        return fail(WN_ERR_ARG, "bad domain list");
    if (precision != WN_PREC_PLAIN_FP64 && precision != WN_PREC_MIXED)
        return fail(WN_ERR_ARG, "precision must be WN_PREC_PLAIN_FP64 or WN_PREC_MIXED");
    if (offsets[0] != 0) return fail(WN_ERR_ARG, "point_offsets[0] must be 0");
    int cur_dev = 0;
    if (cudaGetDevice(&cur_dev) != cudaSuccess) return fail(WN_ERR_CUDA, "cudaGetDevice failed");
    for (int d = 0; d < n_domains; d++) {
        if (!domains[d]) return fail(WN_ERR_ARG, "NULL domain");
        if (domains[d]->device != cur_dev)
            return fail(WN_ERR_ARG, "a domain was created on another device than the current one");
        if (offsets[d + 1] < offsets[d]) return fail(WN_ERR_ARG, "point_offsets must be non-decreasing");
    }
    const int64_t n = offsets[n_domains];
    if (n > WN_MAX_QUERIES_PER_CALL) return fail(WN_ERR_LIMIT, "more than 2^31-1 queries in one call");
    if (n > 0 && !points && !grid.nu) return fail(WN_ERR_ARG, "points is NULL");
    if (n == 0) return WN_OK;

    std::lock_guard<std::mutex> lk(g_mu);
    wn_status st;
    DevState *S = dev_state(st);
    if (!S) return st;
    cudaError_t e;

    // host buffers are staged through library-owned device buffers
    const bool h_pts = points && !is_device_ptr(points);
    const bool h_w = out_w && !is_device_ptr(out_w);
    const bool h_st = out_st && !is_device_ptr(out_st);
    if ((h_pts || h_w || h_st) && (n > S->cap_st || !S->st_pts)) {
        if (S->st_pts) {
            cudaDeviceSynchronize();
            cudaFree(S->st_pts);
            cudaFree(S->st_w);
            cudaFree(S->st_st);
            S->st_pts = nullptr;
            S->st_w = nullptr;
            S->st_st = nullptr;
        }
        S->cap_st = 0;
        if ((e = cudaMalloc(&S->st_pts, 2 * n * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&S->st_w, n * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&S->st_st, n)) != cudaSuccess)
            return cuda_fail(e, "staging buffers");
        S->cap_st = n;
    }
    if (points && !h_pts && (reinterpret_cast<uintptr_t>(points) & 15))
        return fail(WN_ERR_ARG, "device points must be 16-byte aligned");
    // a large mixed batch from host buffers runs as groups of domains whose
    // copies overlap the other groups' kernels
    const int n_groups = group_count(n, n_domains);
    const bool grouped = h_pts && precision == WN_PREC_MIXED && !grid.nu && !bits && !S->profiling &&
                         !S->counting && n_groups >= 2;
    const double *d_pts = points;
    if (h_pts) {
        if (!grouped && (e = cudaMemcpyAsync(S->st_pts, points, 2 * n * sizeof(double), cudaMemcpyHostToDevice,
                                             stream)) != cudaSuccess)
            return cuda_fail(e, "copy points");
        d_pts = S->st_pts;
    }
    OutDst out;
    out.w = h_w ? S->st_w : out_w;
    out.st = h_st ? S->st_st : out_st;
    out.bits = bits;
    out.nbound = reinterpret_cast<unsigned long long *>(nbound);
    PointSrc src = grid;
    src.pts = grid.nu ? nullptr : d_pts;
    // a grid swept by the tree kernel walks tiles of 64 cells, w wide and
    // 64 / w high (spatially coherent warps without the bucketing kernels;
    // wide tiles share the rows, and so the +x rays' crossings)
    const int tw = g_tun.grid_tile_w, th = 64 / tw;
    const bool grid_tiled = grid.nu > 0 && precision != WN_PREC_PLAIN_FP64 && g_tun.tree &&
                            (int64_t)((grid.nu + tw - 1) / tw) * ((grid.nv + th - 1) / th) * 64 <= (int64_t)INT32_MAX;
    src.tiles_x = grid_tiled ? (grid.nu + tw - 1) / tw : 0;
    src.tile_lw = tw == 64 ? 6 : tw == 32 ? 5 : tw == 16 ? 4 : 3;

    if (precision == WN_PREC_PLAIN_FP64) {
        if (bits && (e = cudaMemsetAsync(bits, 0, (size_t)((n + 31) / 32) * 4, stream)) != cudaSuccess)
            return cuda_fail(e, "memset bits");
        if (nbound && (e = cudaMemsetAsync(nbound, 0, 8, stream)) != cudaSuccess)
            return cuda_fail(e, "memset");
        if ((e = cudaMemsetAsync(S->W.counters, 0, CNT_N * sizeof(unsigned long long), stream)) != cudaSuccess)
            return cuda_fail(e, "memset");
        int64_t kernels = 0;
        for (int d = 0; d < n_domains; d++) {
            const int64_t q0 = offsets[d], cnt = offsets[d + 1] - offsets[d];
            if ((e = launch_plain(domains[d]->d_self, q0, cnt, src, out, S->W.counters, stream)) != cudaSuccess)
                return cuda_fail(e, "plain kernel");
            kernels += cnt > 0 ? 1 : 0;
        }
        S->last.kernels = kernels;
    } else {
        const int qpt = g_tun.tree ? std::min(g_tun.qpt, 2) : g_tun.qpt;
        // the tree sweep gives each warp its own unit, the flat sweep each CTA
        const int64_t tile = (g_tun.tree ? 32LL : 256LL) * qpt;
        const int key = (((qpt * 2 + (g_tun.tree ? 1 : 0)) * 4096 + g_tun.cell_q) * 5 +
                         (grid_tiled ? src.tile_lw - 2 : 0)) * 4096 + std::min(g_tun.flat_max, 4095);
        if (grouped) {
            // groups of consecutive domains with about n / G queries each
            const int G = n_groups;
            std::vector<int> gb(1, 0);
            for (int g = 1; g < G; g++) {
                int d = gb.back() + 1;
                while (d < n_domains && offsets[d] < (int64_t)((double)n * g / G)) d++;
                if (d < n_domains) gb.push_back(d);
            }
            gb.push_back(n_domains);
            const int ng = (int)gb.size() - 1;
            // every table, scratch and stream first: nothing below waits on the host
            std::vector<std::vector<int64_t>> og(ng);
            int64_t n_max = 0;
            double near_max = 0.0;
            for (int g = 0; g < ng; g++) {
                const int d0 = gb[g], d1 = gb[g + 1];
                og[g].resize(d1 - d0 + 1);
                for (int i = 0; i <= d1 - d0; i++) og[g][i] = offsets[d0 + i] - offsets[d0];
                PointSrc sg = src;
                if ((st = build_tables(S, S->grp[g], domains + d0, d1 - d0, og[g].data(), key, false, sg, 0, tile)) !=
                    WN_OK)
                    return st;
                n_max = std::max(n_max, og[g].back());
                near_max = std::max(near_max, near_expected_of(domains + d0, d1 - d0, og[g].data()));
            }
            if ((e = ensure_work(S->W, n_max, (int64_t)near_max)) != cudaSuccess) return cuda_fail(e, "scratch");
            if (!S->s_h2d) {
                if ((e = cudaStreamCreateWithFlags(&S->s_h2d, cudaStreamNonBlocking)) != cudaSuccess ||
                    (e = cudaStreamCreateWithFlags(&S->s_d2h, cudaStreamNonBlocking)) != cudaSuccess)
                    return cuda_fail(e, "copy streams");
                for (int i = 0; i < 2 * kMaxGroups + 2; i++)
                    if ((e = cudaEventCreateWithFlags(&S->ev[i], cudaEventDisableTiming)) != cudaSuccess)
                        return cuda_fail(e, "copy events");
            }
            cudaEvent_t ev_in = S->ev[2 * kMaxGroups], ev_out = S->ev[2 * kMaxGroups + 1];
            // the copy streams start after the caller's earlier work
            if ((e = cudaEventRecord(ev_in, stream)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(S->s_h2d, ev_in, 0)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(S->s_d2h, ev_in, 0)) != cudaSuccess)
                return cuda_fail(e, "copy streams");
            for (int g = 0; g < ng; g++) {
                const int64_t q0 = offsets[gb[g]], nq = offsets[gb[g + 1]] - q0;
                if ((e = cudaMemcpyAsync(S->st_pts + 2 * q0, points + 2 * q0, 2 * nq * sizeof(double),
                                         cudaMemcpyHostToDevice, S->s_h2d)) != cudaSuccess ||
                    (e = cudaEventRecord(S->ev[g], S->s_h2d)) != cudaSuccess)
                    return cuda_fail(e, "copy points");
            }
            int64_t kernels = 0;
            for (int g = 0; g < ng; g++) {
                const int d0 = gb[g], nd = gb[g + 1] - d0;
                const int64_t q0 = offsets[d0], nq = og[g].back();
                const Tables &T = S->grp[g];
                Work Wg = work_with(S, T);
                PointSrc sg = src;
                sg.pts = S->st_pts + 2 * q0;
                OutDst og_out = out;
                if (out.w) og_out.w = out.w + q0;
                if (out.st) og_out.st = out.st + q0;
                LaunchCfg cfg{S->n_sm, g_tun, nullptr};
                cfg.n_flat = T.n_flat;
                for (int d = d0; d < d0 + nd; d++) cfg.rational |= domains[d]->dev.w != nullptr;
                const DomDev *d_doms = nd == 1 ? domains[d0]->d_self : T.doms;
                if ((e = cudaStreamWaitEvent(stream, S->ev[g], 0)) != cudaSuccess)
                    return cuda_fail(e, "copy points");
                if ((e = launch_mixed(Wg, d_doms, nd, T.units, T.n_units, T.offsets, nq, sg, og_out, cfg, stream)) !=
                    cudaSuccess)
                    return cuda_fail(e, "mixed kernels");
                kernels += mixed_kernel_count(Wg, cfg);
                if ((e = cudaEventRecord(S->ev[kMaxGroups + g], stream)) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(S->s_d2h, S->ev[kMaxGroups + g], 0)) != cudaSuccess)
                    return cuda_fail(e, "copy results");
                if (h_w && (e = cudaMemcpyAsync(out_w + q0, S->st_w + q0, nq * sizeof(double), cudaMemcpyDeviceToHost,
                                                S->s_d2h)) != cudaSuccess)
                    return cuda_fail(e, "copy winding");
                if (h_st && (e = cudaMemcpyAsync(out_st + q0, S->st_st + q0, nq, cudaMemcpyDeviceToHost, S->s_d2h)) !=
                                cudaSuccess)
                    return cuda_fail(e, "copy states");
            }
            if ((e = cudaEventRecord(ev_out, S->s_d2h)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(stream, ev_out, 0)) != cudaSuccess ||
                (e = cudaStreamSynchronize(stream)) != cudaSuccess)
                return cuda_fail(e, "synchronize");
            S->last.queries = n;
            S->last.kernels = kernels;
            return WN_OK;
        }
        Tables &T = S->main;
        if ((st = build_tables(S, T, domains, n_domains, offsets, key, grid_tiled, src, grid.nv, tile)) != WN_OK)
            return st;
        if ((e = ensure_work(S->W, n, (int64_t)near_expected_of(domains, n_domains, offsets))) != cudaSuccess)
            return cuda_fail(e, "scratch");
        Work Wl = work_with(S, T);
        LaunchCfg cfg{S->n_sm, g_tun, S->profiling ? &S->events : nullptr};
        cfg.n_flat = T.n_flat;
        if (S->counting) cfg.work = S->d_work;
        cfg.grid_tiled = grid_tiled;
        for (int d = 0; d < n_domains; d++) cfg.rational |= domains[d]->dev.w != nullptr;
        const DomDev *d_doms = n_domains == 1 ? domains[0]->d_self : T.doms;
        // graph replay: only for device buffers on a non-default stream, not while profiling or counting
        const bool graph = g_tun.use_graph && !S->profiling && !S->counting && stream != nullptr && !h_pts &&
                           !h_w && !h_st;
        if (graph) {
            std::vector<uintptr_t> gk = {(uintptr_t)stream, (uintptr_t)src.pts, (uintptr_t)out.w,
                                         (uintptr_t)out.st, (uintptr_t)out.bits, (uintptr_t)out.nbound,
                                         (uintptr_t)n, (uintptr_t)src.nu, (uintptr_t)src.nv,
                                         (uintptr_t)T.key, (uintptr_t)g_tun.sweep_ctas_per_sm,
                                         (uintptr_t)g_tun.near_ctas_per_sm, (uintptr_t)g_tun.bucket,
                                         (uintptr_t)S->W.acc2, (uintptr_t)S->W.near_items, (uintptr_t)S->W.perm,
                                         (uintptr_t)T.units, (uintptr_t)S->W.cell_cnt, (uintptr_t)T.bchunks, (uintptr_t)S->W.run_off,
                                         (uintptr_t)g_tun.near_depth, (uintptr_t)g_tun.near_chunk,
                                         (uintptr_t)g_tun.near_refill, (uintptr_t)Wl.cap_near,
                                         (uintptr_t)Wl.cap_f64};
            for (int d = 0; d < n_domains; d++) gk.push_back((uintptr_t)domains[d]);
            cudaGraphExec_t exec = nullptr;
            for (auto &g : S->graphs)
                if (g.first == gk) {
                    exec = g.second;
                    break;
                }
            if (!exec) {
                if (S->graphs.size() >= (size_t)kMaxGraphs) {
                    cudaGraphExecDestroy(S->graphs.front().second);
                    S->graphs.erase(S->graphs.begin());
                }
                cudaGraph_t g = nullptr;
                if ((e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                    return cuda_fail(e, "begin capture");
                e = launch_mixed(Wl, d_doms, n_domains, T.units, T.n_units, T.offsets, n, src, out, cfg, stream);
                cudaError_t e2 = cudaStreamEndCapture(stream, &g);
                if (e != cudaSuccess || e2 != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return cuda_fail(e != cudaSuccess ? e : e2, "capture");
                }
                e = cudaGraphInstantiate(&exec, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
                S->graphs.push_back({gk, exec});
            }
            if ((e = cudaGraphLaunch(exec, stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
            S->graph_launches++;
        } else if ((e = launch_mixed(Wl, d_doms, n_domains, T.units, T.n_units, T.offsets, n, src, out, cfg,
                                     stream)) != cudaSuccess) {
            return cuda_fail(e, "mixed kernels");
        }
        S->last.queries = n;
        S->last.kernels = mixed_kernel_count(Wl, cfg);
    }
    if (h_w && (e = cudaMemcpyAsync(out_w, S->st_w, n * sizeof(double), cudaMemcpyDeviceToHost,
                                    stream)) != cudaSuccess)
        return cuda_fail(e, "copy winding");
    if (h_st && (e = cudaMemcpyAsync(out_st, S->st_st, n, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "copy states");
    if (h_pts || h_w || h_st) {
        if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "synchronize");
    }
    return WN_OK;
}

wn_status wn_query_batched(const wn_domain *const *domains, int32_t n_domains,
                           const int64_t *point_offsets, const double *points, double *out_winding,
                           uint8_t *out_inside, int precision, wn_stream stream)
{
    PointSrc g{};
    return query_impl(domains, n_domains, point_offsets, points, out_winding, out_inside, precision,
                      (cudaStream_t)stream, g, nullptr, nullptr);
}

wn_status wn_query(const wn_domain *domain, const double *points, int64_t n, double *out_winding,
                   uint8_t *out_inside, int precision, wn_stream stream)
{
    if (!domain) return fail(WN_ERR_ARG, "domain is NULL");
    if (n < 0) return fail(WN_ERR_ARG, "n < 0");
    int64_t off[2] = {0, n};
    PointSrc g{};
    return query_impl(&domain, 1, off, points, out_winding, out_inside, precision,
                      (cudaStream_t)stream, g, nullptr, nullptr);
}

wn_status wn_query_grid_bitmask(const wn_domain *domain, int32_t nu, int32_t nv, uint32_t *out_bits,
                                int64_t *out_boundary, int precision, wn_stream stream)
{
    if (!domain || !out_bits) return fail(WN_ERR_ARG, "domain or out_bits is NULL");
    if (nu < 1 || nv < 1 || nu > 65536 || nv > 65536) return fail(WN_ERR_LIMIT, "grid size outside 1..65536");
    const int64_t n = (int64_t)nu * nv;
    if (n > WN_MAX_QUERIES_PER_CALL) return fail(WN_ERR_LIMIT, "grid larger than 2^31-1 cells");
    if (!is_device_ptr(out_bits) || (out_boundary && !is_device_ptr(out_boundary)))
        return fail(WN_ERR_ARG, "grid outputs must be device memory");
    int64_t off[2] = {0, n};
    PointSrc g{};
    g.pts = nullptr;
    g.nu = nu;
    g.nv = nv;
    g.su = domain->dev.Pu > 0 ? domain->dev.Pu : 1.0;
    g.sv = domain->dev.Pv > 0 ? domain->dev.Pv : 1.0;
    return query_impl(&domain, 1, off, nullptr, nullptr, nullptr, precision, (cudaStream_t)stream, g,
                      out_bits, out_boundary);
}

wn_status wn_autotune(const wn_domain *const *domains, int32_t n_domains, const int64_t *point_offsets,
                      const double *points, int32_t iterations, double *best_ms, wn_stream stream)
{
    if (iterations < 1 || iterations > 100) return fail(WN_ERR_ARG, "iterations must be 1..100");
    if (!point_offsets || n_domains < 0) return fail(WN_ERR_ARG, "bad domain list");
    if (!points || !is_device_ptr(points)) return fail(WN_ERR_ARG, "autotune needs device points");
    const int64_t n = point_offsets[n_domains];
    if (n <= 0) return WN_OK;
    double *w = nullptr;
    uint8_t *st = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&w, n * sizeof(double))) != cudaSuccess) return cuda_fail(e, "autotune buffers");
    if ((e = cudaMalloc(&st, n)) != cudaSuccess) {
        cudaFree(w);
        return cuda_fail(e, "autotune buffers");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaStream_t s = (cudaStream_t)stream;
    Tuning best, saved;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        best = saved = g_tun;
    }
    auto trial = [&](const Tuning &t, double &ms) -> wn_status {
        {
            std::lock_guard<std::mutex> lk(g_mu);
            g_tun = t;
            g_tun.use_graph = 0;
        }
        PointSrc g{};
        wn_status r = query_impl(domains, n_domains, point_offsets, points, w, st, WN_PREC_MIXED, s, g,
                                 nullptr, nullptr);
        if (r != WN_OK) return r;
        cudaEventRecord(e0, s);
        for (int i = 0; i < iterations; i++) {
            r = query_impl(domains, n_domains, point_offsets, points, w, st, WN_PREC_MIXED, s, g, nullptr,
                           nullptr);
            if (r != WN_OK) return r;
        }
        cudaEventRecord(e1, s);
        cudaError_t ee = cudaEventSynchronize(e1);
        if (ee != cudaSuccess) return cuda_fail(ee, "autotune timing");
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        ms = (double)f / iterations;
        return WN_OK;
    };
    double best_t = 0.0;
    wn_status r = trial(best, best_t);
    // coordinate descent, one knob at a time from the current best
    struct Knob {
        int Tuning::*field;
        int n;
        int vals[4];
    };
    const Knob knobs[] = {{&Tuning::qpt, 2, {1, 2}},
                          {&Tuning::sweep_ctas_per_sm, 4, {2, 3, 4, 6}},
                          {&Tuning::near_ctas_per_sm, 3, {4, 8, 16}},
                          {&Tuning::cell_q, 3, {32, 64, 128}},
                          {&Tuning::bucket, 2, {1, 0}},
                          {&Tuning::near_depth, 3, {16, 22, 28}},
                          {&Tuning::near_chunk, 3, {64, 128, 256}},
                          {&Tuning::near_refill, 3, {8, 16, 24}},
                          {&Tuning::flat_max, 3, {0, 16, 32}}};
    for (const Knob &kb : knobs) {
        if (r != WN_OK) break;
        for (int i = 0; i < kb.n && r == WN_OK; i++) {
            Tuning t = best;
            int &field = t.*(kb.field);
            const int *vals = kb.vals;
            if (field == vals[i]) continue;
            field = vals[i];
            double ms = 0.0;
            r = trial(t, ms);
            if (r == WN_OK && ms < best_t) {
                best_t = ms;
                best = t;
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_tun = (r == WN_OK) ? best : saved;
        g_tun.use_graph = saved.use_graph;
        drop_graphs();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(w);
    cudaFree(st);
    if (r == WN_OK && best_ms) *best_ms = best_t;
    return r;
}

wn_status wn_get_tuning(int32_t *out, int32_t n_out)
{
    if (!out || n_out < 0) return fail(WN_ERR_ARG, "out is NULL or n_out < 0");
    std::lock_guard<std::mutex> lk(g_mu);
    const int32_t v[12] = {g_tun.qpt, g_tun.sweep_ctas_per_sm, g_tun.near_ctas_per_sm, g_tun.use_graph,
                           g_tun.tree, g_tun.cell_q, g_tun.bucket, g_tun.near_depth, g_tun.near_chunk,
                           g_tun.near_refill, g_tun.flat_max, g_tun.grid_tile_w};
    for (int i = 0; i < n_out && i < 12; i++) out[i] = v[i];
    return WN_OK;
}

wn_status wn_set_profiling(int32_t on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    wn_status st;
    DevState *S = dev_state(st);
    if (!S) return st;
    cudaDeviceSynchronize();
    for (cudaEvent_t e : S->events) cudaEventDestroy(e);
    S->events.clear();
    S->profiling = on != 0;
    return WN_OK;
}

wn_status wn_set_work_counting(int32_t on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    wn_status st;
    DevState *S = dev_state(st);
    if (!S) return st;
    cudaError_t e;
    if (on && !S->d_work) {
        if ((e = cudaMalloc(&S->d_work, WK_N * sizeof(unsigned long long))) != cudaSuccess) {
            S->d_work = nullptr;
            return cuda_fail(e, "work tallies");
        }
    }
    if (S->d_work && (e = cudaMemset(S->d_work, 0, WK_N * sizeof(unsigned long long))) != cudaSuccess)
        return cuda_fail(e, "work tallies");
    S->counting = on != 0;
    return WN_OK;
}

// Read tallies [first, first + count) of the counting builds and clear them.
static wn_status read_work(int first, int count, int64_t *out)
{
    if (!out) return fail(WN_ERR_ARG, "out is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    wn_status st;
    DevState *S = dev_state(st);
    if (!S) return st;
    unsigned long long c[WK_N] = {};
    cudaError_t e;
    if (S->d_work) {
        if ((e = cudaMemcpy(c, S->d_work + first, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost)) !=
            cudaSuccess)
            return cuda_fail(e, "read work tallies");
        if ((e = cudaMemset(S->d_work + first, 0, count * sizeof(unsigned long long))) != cudaSuccess)
            return cuda_fail(e, "work tallies");
    }
    for (int i = 0; i < count; i++) out[i] = (int64_t)c[i];
    return WN_OK;
}

wn_status wn_sweep_work(int64_t *out, int32_t n_out)
{
    if (n_out < 0) return fail(WN_ERR_ARG, "n_out < 0");
    int64_t all[WK_SWEEP_N];
    const wn_status st = read_work(0, WK_SWEEP_N, out ? all : nullptr);
    if (st != WN_OK) return st;
    for (int i = 0; i < n_out && i < WK_SWEEP_N; i++) out[i] = all[i];
    return WN_OK;
}

wn_status wn_near_work(int64_t *out4) { return read_work(WK_NEAR_NODE, WK_N - WK_NEAR_NODE, out4); }

wn_status wn_kernel_times(double *ms6, int64_t *n_calls)
{
    if (!ms6) return fail(WN_ERR_ARG, "ms6 is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    wn_status st;
    DevState *S = dev_state(st);
    if (!S) return st;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    const int ni = kProfEvents - 1;
    for (int k = 0; k < ni; k++) ms6[k] = 0.0;
    const size_t calls = S->events.size() / kProfEvents;
    for (size_t c = 0; c < calls; c++)
        for (int k = 0; k < ni; k++) {
            float ms = 0.f;
            if ((e = cudaEventElapsedTime(&ms, S->events[kProfEvents * c + k],
                                          S->events[kProfEvents * c + k + 1])) != cudaSuccess)
                return cuda_fail(e, "cudaEventElapsedTime");
            ms6[k] += ms;
        }
    if (n_calls) *n_calls = (int64_t)calls;
    for (cudaEvent_t ev : S->events) cudaEventDestroy(ev);
    S->events.clear();
    return WN_OK;
}

wn_status wn_eval_gap_angle(const float *y, const float *x, float *out, int64_t n, wn_stream stream)
{
    if (n < 0) return fail(WN_ERR_ARG, "n < 0");
    if (n == 0) return WN_OK;
    if (!y || !x || !out || !is_device_ptr(y) || !is_device_ptr(x) || !is_device_ptr(out))
        return fail(WN_ERR_ARG, "y, x and out must be device memory");
    cudaError_t e = launch_gap_angle(y, x, out, n, (cudaStream_t)stream);
    return e == cudaSuccess ? WN_OK : cuda_fail(e, "gap angle kernel");
}

wn_status wn_last_escalated(int64_t *out_idx, int64_t capacity, int64_t *n_out)
{
    if (!n_out || capacity < 0 || (capacity > 0 && !out_idx)) return fail(WN_ERR_ARG, "bad output buffer");
    std::lock_guard<std::mutex> lk(g_mu);
    wn_status st;
    DevState *S = dev_state(st);
    if (!S) return st;
    unsigned long long c[CNT_N];
    cudaError_t e = cudaMemcpy(c, S->W.counters, sizeof c, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read counters");
    const int64_t n = std::min<int64_t>((int64_t)c[CNT_ESC], S->W.cap_q);
    *n_out = n;
    const int64_t m = std::min(n, capacity);
    if (m > 0) {
        std::vector<uint2> v((size_t)m);
        if ((e = cudaMemcpy(v.data(), S->W.esc_q, m * sizeof(uint2), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "read escalated queries");
        for (int64_t i = 0; i < m; i++) out_idx[i] = (int64_t)v[i].x;
    }
    return WN_OK;
}

wn_status wn_get_stats(wn_stats *out)
{
    if (!out) return fail(WN_ERR_ARG, "out is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    wn_status st;
    DevState *S = dev_state(st);
    if (!S) return st;
    unsigned long long c[CNT_N];
    cudaError_t e = cudaMemcpy(c, S->W.counters, sizeof c, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read counters");
    out->queries = S->last.queries;
    out->near_pairs = c[CNT_NEAR];
    out->fp64_pairs = c[CNT_F64];
    out->fp64_queries = c[CNT_ESC];
    const int64_t cap_near = g_lim_near > 0 ? std::min(S->W.cap_near, g_lim_near) : S->W.cap_near;
    const int64_t cap_f64 = g_lim_f64 > 0 ? std::min(S->W.cap_f64, g_lim_f64) : S->W.cap_f64;
    out->overflow = ((c[CNT_NEAR] > (unsigned long long)cap_near) ? (int64_t)(c[CNT_NEAR] - cap_near) : 0) +
                    ((c[CNT_F64] > (unsigned long long)cap_f64) ? (int64_t)(c[CNT_F64] - cap_f64) : 0);
    out->depth_cap = c[CNT_DEPTH];
    out->kernels = S->last.kernels;
    return WN_OK;
}

}  // extern "C"
