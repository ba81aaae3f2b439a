// wn_tess.cu -- triangles of a trimmed cell-centre grid (the tessellation
// application of Sec. 5.4.3): the grid of cell centres classified by
// wn_query_grid_bitmask is triangulated quad by quad and a triangle is kept
// when its three vertices are inside.
//
// Vertex (i, j) has index j*nu + i.  The quad with lower-left vertex (i, j)
// has corners a = (i, j), b = (i+1, j), c = (i, j+1), d = (i+1, j+1), taken
// modulo nu / nv on a wrapped (periodic) axis, whose seam quads then exist
// too; its triangles are (a, b, d) and (a, d, c), counter-clockwise in
// (u, v).  Quads are emitted row by row, so the output order is fixed.
//
// Three launches: per-row counts (one CTA per quad row, so a thread knows
// its quad's (i, j) without a division), one scan of the row counts, and the
// writes (each row re-derives its triangles and scans them in shared
// memory).  The work is HBM-bound: the bitmask read, 12 B written per kept
// triangle.
#include <cstdint>
#include <string>

#include "wn.h"
#include "wn_internal.h"

namespace {

constexpr int kTessThreads = 256;

struct TessArgs {
    const uint32_t *bits;
    int nu, nv, qu, qv;           // vertices per row and column, quads per row and column
    int32_t *tris;
    int64_t cap;                  // triangles the output holds
    long long *row_base;          // per quad row: its count, then its first triangle
    long long *total;             // device: number of kept triangles
};

__device__ __forceinline__ bool bit_at(const uint32_t *bits, int64_t v)
{
    return (__ldg(&bits[v >> 5]) >> (v & 31)) & 1u;
}

// Kept triangles of quad (i, j): bit 0 lower (a, b, d), bit 1 upper (a, d, c);
// the four corner indices in abcd.
__device__ __forceinline__ uint32_t quad_tris(const TessArgs &A, int i, int j, int64_t abcd[4])
{
    const int i1 = (i + 1 == A.nu) ? 0 : i + 1, j1 = (j + 1 == A.nv) ? 0 : j + 1;
    abcd[0] = (int64_t)j * A.nu + i;
    abcd[1] = (int64_t)j * A.nu + i1;
    abcd[2] = (int64_t)j1 * A.nu + i;
    abcd[3] = (int64_t)j1 * A.nu + i1;
    const bool a = bit_at(A.bits, abcd[0]), b = bit_at(A.bits, abcd[1]);
    const bool c = bit_at(A.bits, abcd[2]), d = bit_at(A.bits, abcd[3]);
    return ((a && b && d) ? 1u : 0u) | ((a && d && c) ? 2u : 0u);
}

__global__ void __launch_bounds__(kTessThreads) k_tri_count(const TessArgs A)
{
    __shared__ int s_warp[kTessThreads / 32];
    const int j = blockIdx.x;
    int c = 0;
    for (int i = threadIdx.x; i < A.qu; i += kTessThreads) {
        int64_t abcd[4];
        c += __popc(quad_tris(A, i, j, abcd));
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int k = 0; k < kTessThreads / 32; k++) t += s_warp[k];
        A.row_base[j] = t;
    }
}

// Exclusive scan of the row counts in one CTA; the total goes to A.total.
__global__ void __launch_bounds__(1024) k_tri_scan(const TessArgs A)
{
    __shared__ long long s_sum[1024];
    const int t = threadIdx.x;
    const int per = (A.qv + 1023) / 1024;
    const int b = t * per, e = min(b + per, A.qv);
    long long sum = 0;
    for (int i = b; i < e; i++) sum += A.row_base[i];
    s_sum[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const long long v = t >= off ? s_sum[t - off] : 0;
        __syncthreads();
        s_sum[t] += v;
        __syncthreads();
    }
    long long run = s_sum[t] - sum;
    for (int i = b; i < e; i++) {
        const long long c = A.row_base[i];
        A.row_base[i] = run;
        run += c;
    }
    if (t == 1023) *A.total = s_sum[1023];
}

__global__ void __launch_bounds__(kTessThreads) k_tri_write(const TessArgs A)
{
    __shared__ int s_warp[kTessThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x;
    long long out = A.row_base[j];
    for (int i0 = 0; i0 < A.qu; i0 += kTessThreads) {
        const int i = i0 + threadIdx.x;
        int64_t abcd[4] = {0, 0, 0, 0};
        const uint32_t m = i < A.qu ? quad_tris(A, i, j, abcd) : 0u;
        const int c = __popc(m);
        // exclusive prefix of c over the block, in thread order
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_warp[w] = incl;
        __syncthreads();
        int before = 0, total = 0;
        for (int x = 0; x < kTessThreads / 32; x++) {
            const int sv = s_warp[x];
            before += x < w ? sv : 0;
            total += sv;
        }
        __syncthreads();
        long long pos = out + before + incl - c;
        if (m & 1u) {
            if (pos < A.cap) {
                A.tris[3 * pos] = (int32_t)abcd[0];
                A.tris[3 * pos + 1] = (int32_t)abcd[1];
                A.tris[3 * pos + 2] = (int32_t)abcd[3];
            }
            pos++;
        }
        if ((m & 2u) && pos < A.cap) {
            A.tris[3 * pos] = (int32_t)abcd[0];
            A.tris[3 * pos + 1] = (int32_t)abcd[3];
            A.tris[3 * pos + 2] = (int32_t)abcd[2];
        }
        out += total;
    }
}

bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" wn_status wn_grid_triangles(const uint32_t *bits, int32_t nu, int32_t nv, int32_t wrap_u,
                                       int32_t wrap_v, int32_t *out_tris, int64_t capacity,
                                       int64_t *out_count, wn_stream stream)
{
    if (!bits || !out_count || capacity < 0 || (capacity > 0 && !out_tris)) return WN_ERR_ARG;
    if (nu < 1 || nv < 1 || nu > 65536 || nv > 65536) return WN_ERR_LIMIT;
    if ((int64_t)nu * nv > WN_MAX_QUERIES_PER_CALL) return WN_ERR_LIMIT;
    if (!on_device(bits) || !on_device(out_count) || (capacity > 0 && !on_device(out_tris))) return WN_ERR_ARG;
    const int qu = wrap_u ? nu : nu - 1, qv = wrap_v ? nv : nv - 1;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (qu <= 0 || qv <= 0) {
        e = cudaMemsetAsync(out_count, 0, sizeof(int64_t), s);
        return e == cudaSuccess ? WN_OK : WN_ERR_CUDA;
    }
    TessArgs A;
    A.bits = bits;
    A.nu = nu;
    A.nv = nv;
    A.qu = qu;
    A.qv = qv;
    A.tris = out_tris;
    A.cap = capacity;
    A.total = reinterpret_cast<long long *>(out_count);
    // per-row counts (8 B per quad row) from the stream-ordered pool, so that
    // calls on different streams do not share them
    if ((e = cudaMallocAsync(reinterpret_cast<void **>(&A.row_base), (size_t)qv * sizeof(long long), s)) !=
        cudaSuccess)
        return e == cudaErrorMemoryAllocation ? WN_ERR_OOM : WN_ERR_CUDA;
    k_tri_count<<<qv, kTessThreads, 0, s>>>(A);
    k_tri_scan<<<1, 1024, 0, s>>>(A);
    k_tri_write<<<qv, kTessThreads, 0, s>>>(A);
    e = cudaGetLastError();
    cudaFreeAsync(A.row_base, s);
    return e == cudaSuccess ? WN_OK : WN_ERR_CUDA;
}
