// wn_internal.h -- host-side declarations shared by the library's translation
// units (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "wn_dev.cuh"

struct wn_domain {
    wn::DomDev dev;            // device pointers filled in
    wn::DomDev *d_self;        // device copy of dev
    std::vector<void *> allocs;  // device allocations owned by the domain
    int device;
    int64_t n_records;
    int64_t n_instances;
    int64_t sweep_records;     // sum over instances of their record counts
    double near_density;       // expected near pairs per uniform query: sum of the records'
                               // circle areas over the query area
};

namespace wn {

// Where the query points come from.
struct PointSrc {
    const double *pts;         // x,y interleaved, indexed by global query index
    int32_t nu, nv;            // grid mode when pts == nullptr
    double su, sv;             // grid scale (period or 1)
    int32_t tiles_x;           // grid mode, tree sweep: positions walk tiles of 64 cells, this many per row
    int32_t tile_lw;           // log2 of the tile width in cells (the height is 64 / width)
};

// Output of a query call.
struct OutDst {
    double *w;                 // may be null
    uint8_t *st;               // may be null
    uint32_t *bits;            // grid bitmask mode
    unsigned long long *nbound;  // grid boundary counter
};

// Per-device scratch of the mixed path, with the batch tables of the call in
// place (the tables themselves are owned and sized elsewhere: the API keeps
// one set per list of domains, the allocation-free query a fixed one).
struct Work {
    int32_t *acc2 = nullptr;   // per query: (2 * crossings + line halves) * 4 | QF_* flags
    float *theta = nullptr;    // sum of gap angles, per query
    Item *near_items = nullptr;
    SubItem *f64_items = nullptr;
    uint2 *esc_q = nullptr;    // (query, batch entry) recomputed in FP64
    unsigned long long *counters = nullptr;  // see CNT_*
    int4 *units = nullptr;     // (dom, first query, count, first position in the bucketed order)
    DomDev *doms = nullptr;
    int64_t *offsets = nullptr;  // device copy of point offsets
    // spatial bucketing of the queries (null: sweep in input order)
    int *cell_of = nullptr;    // per query
    int *perm = nullptr;       // per query
    int *cell_cnt = nullptr;   // per cell
    int *run_off = nullptr;    // per run and cell of the run's domain: the run's offset in the cell
    int4 *dcell = nullptr;     // per domain: first cell, G
    int *bin_chunk = nullptr;  // per 4096 cells: chunk sum, then its first position
    int4 *bchunks = nullptr;   // (domain, first query, count, first run_off entry): runs of one domain's queries
    int n_cells = 0;
    int n_bchunks = 0;
    int64_t cap_bin_q = 0, cap_cells = 0, cap_chunk = 0, cap_runoff = 0;
    int64_t cap_q = 0, cap_near = 0, cap_f64 = 0;
};

// Spatial bucketing: at most kBinMaxG x kBinMaxG cells per domain, so that a
// CTA can count one domain's cells in shared memory.
constexpr int kBinMaxG = 110;
constexpr int kBinSmemCells = 12288;
// A query's cell (< 2^14) and its rank among its run's queries of that cell
// share one 32-bit word: runs hold at most 2^kBinRankBits queries.
constexpr int kBinRankBits = 17;
constexpr int kBinRunMax = 1 << kBinRankBits;
constexpr int kBinRunPerCell = 2;       // a run: about this many queries per cell of its domain
                                        //   (measured on the B-Rep batch: 2 < 4 < 8 < 16 in time)
static_assert(kBinMaxG * kBinMaxG <= kBinSmemCells, "cell counters must fit shared memory");
static_assert(kBinSmemCells <= (1 << (31 - kBinRankBits)), "a cell and a rank must fit one int");

// Device counters of one mixed call.  CNT_DEPTH counts FP64 walks that
// reached the depth cap (reported BOUNDARY: the oracle's reading of a walk
// that cannot end, unreachable for d > eps by Lemma 2).
enum { CNT_NEAR = 0, CNT_F64 = 1, CNT_ESC = 2, CNT_UNIT = 3, CNT_DEPTH = 4, CNT_OVF = 5,
       CNT_FLAT_UNIT = 6, CNT_NEAR_CURSOR = 7, CNT_BIN_RUN = 8, CNT_SCAT_RUN = 9, CNT_N = 10 };

// Work tallies of the counting build of the tree sweep (per query slot):
// node tests, nodes whose crossings telescoped, expansion evaluations and
// their terms, record tests with the near check (Alg. 1's root step), record
// tests for crossings and gap angle, record tests for crossings only, exact
// FP64 recomputations, ellipse tests of records whose circle held the query,
// control-point box tests of records whose ellipse held it; then per warp
// (not per query slot): node visits and record iterations of the leaves,
// each serving the warp's 32 * QPT query slots.  Then the tallies of the
// counting build of the FP32 near walk: nodes tested (Eq. 5), nodes
// accepted as far (a chord each), evaluations of gamma(m) and the sum of
// their segments' degrees.
enum { WK_NODE = 0, WK_TELE = 1, WK_EXPANSION = 2, WK_TERMS = 3, WK_REC_NEAR = 4, WK_REC_FAR = 5,
       WK_REC_CROSS = 6, WK_EXACT = 7, WK_ELLIPSE = 8, WK_BOX = 9, WK_WARP_NODE = 10, WK_WARP_REC = 11,
       WK_SWEEP_N = 12, WK_NEAR_NODE = 12, WK_NEAR_FAR = 13, WK_NEAR_EVAL = 14, WK_NEAR_DEG = 15, WK_N = 16 };

// FP32 walk depth: the cap is a tuning knob (the stack holds kDepthCap32Max
// levels); Lemma 2 bounds the depth a pair needs by log2(B / max(eps, d)),
// and a pair that reaches the cap hands its tail to the FP64 walk.
constexpr int kDepthCap32Min = 12;
constexpr int kNearChunkMin = 32, kNearChunkMax = 1024;

struct Tuning {
    int qpt = 2;               // queries per sweep thread
    int sweep_ctas_per_sm = 4;
    int near_ctas_per_sm = 8;
    int use_graph = 0;
    int tree = 1;              // 1: cluster sweep with gap-angle expansions; 0: flat sweep
    int bucket = 1;            // 1: bucket queries spatially before the sweep
    int cell_q = 64;           // target queries per bucket cell
    int near_depth = 22;       // FP32 near-walk depth cap (kDepthCap32Min..kDepthCap32Max)
    int near_chunk = 128;      // near pairs a warp draws per atomic (32..1024, multiple of 32)
    int near_refill = 16;      // idle lanes that trigger a refill (1..32)
    int flat_max = 0;          // planar domains with at most this many records take the flat sweep (0: none)
    int grid_tile_w = 8;       // grid queries: tile width in cells (8, 16, 32 or 64; 64 cells per tile)
};

constexpr int kSweepThreads = 256;   // threads of a sweep CTA
// Queries per thread of the flat sweep when it shares a batch with the tree
// sweep (a unit is one CTA's kSweepThreads * kFlatQpt queries).
constexpr int kFlatQpt = 2;

constexpr int kProfEvents = 7;   // events per profiled mixed call (6 intervals)

struct LaunchCfg {
    int n_sm;
    Tuning tun;
    std::vector<cudaEvent_t> *events;  // non-null: record kProfEvents events per call
    unsigned long long *work = nullptr; // non-null: counting build of the tree sweep adds WK_* here
    bool grid_tiled = false;            // grid positions in 8 x 8 tiles instead of bucketing
    bool rational = false;              // some domain of the batch has rational segments
    int n_flat = 0;                     // flat-sweep units after the tree units in the unit list
};

// Kernels (wn_kernels.cu)
// App. A.1's bound of |gamma'| for a rational segment of degree n, and the
// bounds on its eighths [j/8, (j+1)/8] (each at most B) (wn_domain.cu)
double rational_segment_bound(const double *P, const double *w, int n);
void rational_eighth_bounds(const double *P, const double *w, int n, double B, double out[8]);
bool mixed_buckets(const Work &W, const LaunchCfg &cfg);        // bucketing kernels run
// CTAs of k_bin_count (0) or k_bin_scatter (1) that fit on one SM; queried
// once and cached (first called when a device's state is set up, outside
// stream capture)
int bin_blocks_per_sm(int scatter);
int mixed_kernel_count(const Work &W, const LaunchCfg &cfg);    // kernels one launch_mixed issues
cudaError_t launch_mixed(const Work &W, const DomDev *d_doms, int n_doms, const int4 *d_units,
                         int n_units, const int64_t *d_offsets, int64_t n_queries, PointSrc src,
                         OutDst out, const LaunchCfg &cfg, cudaStream_t s);
// The sweep's gap angle (gap_angle in wn_kernels.cu) on n device values.
cudaError_t launch_gap_angle(const float *y, const float *x, float *out, int64_t n, cudaStream_t s);
cudaError_t launch_plain(const DomDev *d_dom, int64_t q0, int64_t n, PointSrc src, OutDst out,
                         unsigned long long *counters, cudaStream_t s);
struct PeReq {
    int a, b;
    long long IA, JA, IB, JB;
};
cudaError_t launch_pe_eval(const DomDev *d_dom, const PeReq *d_req, int n, double *d_out,
                           cudaStream_t s);

// Domain build (wn_domain.cu)
int build_domain(const int32_t *loop_offsets, int32_t n_loops, const int32_t *degrees,
                 const double *cps, const double *weights, double Pu, double Pv, double eps,
                 wn_domain **out, std::string &err);

}  // namespace wn
