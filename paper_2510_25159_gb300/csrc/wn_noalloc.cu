// wn_noalloc.cu -- wn_query_noalloc: the mixed-precision query of one domain
// with its scratch memory in a fixed, file-scope device array instead of
// library allocations.
//
// Who needs it: callers that must not allocate device memory once they are
// running -- code inside a custom allocator or memory-pool callback (where a
// nested cudaMalloc would re-enter the allocator), real-time or
// safety-certified loops that forbid allocation after start-up, and
// processes that run with a hard device-memory budget where a first-call
// cudaMalloc of the scratch buffers could fail or evict something else.
//
// Cost: kScratchBytes of device memory on each device the process calls it
// on, held until the process exits.  The library has no relocatable device
// code and CUDA loads modules lazily, so the array is placed on a device
// when the first call there loads this module (an implicit allocation),
// and kernels load (and reserve local memory) at their first launch: the
// first call on a device places the array and launches every kernel a
// call can use once on an empty work list, so callers make it at start-up
// (n = 0 does only this set-up).
#include <cstdint>
#include <mutex>

#include "wn.h"
#include "wn_internal.h"

using namespace wn;

namespace {

constexpr int64_t kMaxQ = WN_NOALLOC_MAX_QUERIES;
constexpr int64_t kMaxUnits = (kMaxQ + 31) / 32;          // tiles of at least 32 queries
constexpr int64_t kNearCap = 4 * kMaxQ;                   // near pairs; overflow recomputes in FP64
constexpr int64_t kF64Cap = kMaxQ;

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffCounters = 0;
constexpr size_t kOffUnits = align256(kOffCounters + CNT_N * sizeof(unsigned long long));
constexpr size_t kOffOffsets = align256(kOffUnits + kMaxUnits * sizeof(int4));
constexpr size_t kOffAcc2 = align256(kOffOffsets + 2 * sizeof(int64_t));
constexpr size_t kOffTheta = align256(kOffAcc2 + kMaxQ * sizeof(int32_t));
constexpr size_t kOffEsc = align256(kOffTheta + kMaxQ * sizeof(float));
constexpr size_t kOffNear = align256(kOffEsc + kMaxQ * sizeof(uint2));
constexpr size_t kOffF64 = align256(kOffNear + kNearCap * sizeof(Item));
constexpr size_t kScratchBytes = align256(kOffF64 + kF64Cap * sizeof(SubItem));

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
bool g_ready[64];

// The scratch array's device address per device (set once per device).
unsigned char *g_base[64];

// The mixed path's scratch carved out of the array at `base`.
Work scratch_work(unsigned char *base)
{
    Work W;
    W.counters = reinterpret_cast<unsigned long long *>(base + kOffCounters);
    W.units = reinterpret_cast<int4 *>(base + kOffUnits);
    W.offsets = reinterpret_cast<int64_t *>(base + kOffOffsets);
    W.acc2 = reinterpret_cast<int32_t *>(base + kOffAcc2);
    W.theta = reinterpret_cast<float *>(base + kOffTheta);
    W.esc_q = reinterpret_cast<uint2 *>(base + kOffEsc);
    W.near_items = reinterpret_cast<Item *>(base + kOffNear);
    W.f64_items = reinterpret_cast<SubItem *>(base + kOffF64);
    W.cap_q = kMaxQ;
    W.cap_near = kNearCap;
    W.cap_f64 = kF64Cap;
    return W;
}

// The fixed launch shape: tree sweep, 2 queries per thread, no bucketing.
Tuning fixed_tuning()
{
    Tuning tun;
    tun.qpt = 2;
    tun.tree = 1;
    return tun;
}

// Work list of one domain: tiles of `tile` queries, and the offsets {0, n}.
__global__ void k_fill_units(int4 *units, int64_t *offsets, int n_units, int tile, int n)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n_units) units[u] = make_int4(0, u * tile, min(tile, n - u * tile), 0);
    if (u == 0) {
        offsets[0] = 0;
        offsets[1] = n;
    }
}

// A failed lookup leaves its error for the caller to see (the call then
// returns WN_ERR_ARG before anything else runs).
bool device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) return false;
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" wn_status wn_query_noalloc(const wn_domain *domain, const double *points, int64_t n,
                                      double *out_winding, uint8_t *out_inside, wn_stream stream)
{
    if (!domain) return WN_ERR_ARG;
    if (n < 0) return WN_ERR_ARG;
    if (n > kMaxQ) return WN_ERR_LIMIT;      // more than WN_NOALLOC_MAX_QUERIES: split the call
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return WN_ERR_CUDA;
    if (domain->device != dev) return WN_ERR_ARG;
    int n_sm = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ready[dev]) {
            // once per device, with that device current: the array's address
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) return WN_ERR_CUDA;
            g_base[dev] = static_cast<unsigned char *>(p);
            // then every kernel a call can launch, once on an empty work
            // list: each launch loads the kernel's code and reserves its
            // local memory now, so that later calls allocate nothing
            e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return WN_ERR_CUDA;
            Work W0 = scratch_work(g_base[dev]);
            cudaStream_t s0 = (cudaStream_t)stream;
            k_fill_units<<<1, 128, 0, s0>>>(W0.units, W0.offsets, 0, 64, 0);
            if ((e = cudaGetLastError()) != cudaSuccess) return WN_ERR_CUDA;
            for (int rat = 0; rat < 2; rat++) {
                LaunchCfg c0{n_sm, fixed_tuning(), nullptr};
                c0.rational = rat != 0;
                PointSrc src0{};
                OutDst out0{};
                if (launch_mixed(W0, domain->d_self, 1, W0.units, 0, W0.offsets, 0, src0, out0, c0, s0) !=
                    cudaSuccess)
                    return WN_ERR_CUDA;
            }
            g_ready[dev] = true;
        }
    }
    // n == 0 after the set-up: the start-up call that places the array
    if (n == 0) return WN_OK;
    if (!points || !device_ptr(points) || (out_winding && !device_ptr(out_winding)) ||
        (out_inside && !device_ptr(out_inside)))
        return WN_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(points) & 15) return WN_ERR_ARG;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return WN_ERR_CUDA;
    Work W = scratch_work(g_base[dev]);
    const Tuning tun = fixed_tuning();
    const int tile = 32 * tun.qpt;    // the tree sweep gives each warp one unit
    const int n_units = (int)((n + tile - 1) / tile);
    cudaStream_t s = (cudaStream_t)stream;
    k_fill_units<<<(n_units + 127) / 128, 128, 0, s>>>(W.units, W.offsets, n_units, tile, (int)n);
    if ((e = cudaGetLastError()) != cudaSuccess) return WN_ERR_CUDA;
    PointSrc src{};
    src.pts = points;
    OutDst out{};
    out.w = out_winding;
    out.st = out_inside;
    LaunchCfg cfg{n_sm, tun, nullptr};
    cfg.rational = domain->dev.w != nullptr;
    e = launch_mixed(W, domain->d_self, 1, W.units, n_units, W.offsets, n, src, out, cfg, s);
    return e == cudaSuccess ? WN_OK : WN_ERR_CUDA;
}
