// wn_multi.cu -- queries over several faces of one surface and midpoint
// filtering of curve pieces (multi-patch B-Rep processing and B-Rep
// intersection, Sec. 5.4.2):
//
//   * a point sampled on a geometric surface is inside when it lies inside
//     (or on the boundary of) ANY trimmed face that references the surface;
//   * a piece of an intersection curve, already split at the trimming
//     boundaries, is kept when its midpoint is inside the face.
//
// Both reduce to the batched mixed/plain query: the surfaces' points are
// gathered once per face that references them, classified in one batched
// call, and OR-reduced per point; the pieces' midpoints are formed on the
// device and classified.  Scratch comes from the stream-ordered pool.
#include <cstdint>
#include <vector>

#include "wn.h"
#include "wn_internal.h"

namespace {

__device__ __forceinline__ int find_le(const int64_t *off, int n, int64_t x)
{
    int lo = 0, hi = n - 1;                  // largest k with off[k] <= x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// dst[e] = src[pair_src[k] + (e - pair_off[k])] for the pair k holding e.
__global__ void k_expand_points(const double2 *__restrict__ src, double2 *__restrict__ dst,
                                const int64_t *__restrict__ pair_off, const int64_t *__restrict__ pair_src,
                                int n_pairs, int64_t E)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_le(pair_off, n_pairs, e);
        dst[e] = src[pair_src[k] + (e - pair_off[k])];
    }
}

// out[i] = 1 when any face of point i's surface has it inside or on its
// boundary, else 0.
__global__ void k_or_reduce(const uint8_t *__restrict__ st, uint8_t *__restrict__ out,
                            const int64_t *__restrict__ pt_off, const int32_t *__restrict__ surf_pair0,
                            const int64_t *__restrict__ pair_off, int n_surf, int64_t n_points)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_points;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int s = find_le(pt_off, n_surf, i);
        const int64_t local = i - pt_off[s];
        uint8_t v = 0;
        for (int k = surf_pair0[s]; k < surf_pair0[s + 1]; k++) v |= st[pair_off[k] + local] != 0 ? 1 : 0;
        out[i] = v;
    }
}

// Midpoints 0.5 (a + b) of the pieces (ax, ay, bx, by).
__global__ void k_midpoints(const double4 *__restrict__ seg, double2 *__restrict__ mid, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double4 g = seg[i];
        mid[i] = make_double2(0.5 * (g.x + g.z), 0.5 * (g.y + g.w));
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

template <typename T>
cudaError_t pool_alloc(T *&p, size_t n, cudaStream_t s)
{
    return cudaMallocAsync(reinterpret_cast<void **>(&p), (n ? n : 1) * sizeof(T), s);
}

int grid_for(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

extern "C" wn_status wn_query_surfaces(const wn_domain *const *faces, const int32_t *surface_faces,
                                       int32_t n_surfaces, const int64_t *point_offsets, const double *points,
                                       uint8_t *out_inside, int precision, wn_stream stream)
{
    if (n_surfaces < 0 || !surface_faces || !point_offsets) return WN_ERR_ARG;
    if (surface_faces[0] != 0 || point_offsets[0] != 0) return WN_ERR_ARG;
    for (int s = 0; s < n_surfaces; s++)
        if (surface_faces[s + 1] < surface_faces[s] || point_offsets[s + 1] < point_offsets[s]) return WN_ERR_ARG;
    const int32_t n_face_refs = surface_faces[n_surfaces];
    if (n_face_refs > 0 && !faces) return WN_ERR_ARG;
    for (int k = 0; k < n_face_refs; k++)
        if (!faces[k]) return WN_ERR_ARG;
    const int64_t n_points = point_offsets[n_surfaces];
    if (n_points == 0) return WN_OK;
    if (!points || !out_inside || !on_device(points) || !on_device(out_inside)) return WN_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(points) & 15) return WN_ERR_ARG;
    // one batch entry per (surface, face): the surface's points against the face
    std::vector<const wn_domain *> pd;
    std::vector<int64_t> pair_off(1, 0), pair_src;
    std::vector<int32_t> surf_pair0(1, 0);
    for (int s = 0; s < n_surfaces; s++) {
        const int64_t cnt = point_offsets[s + 1] - point_offsets[s];
        for (int k = surface_faces[s]; k < surface_faces[s + 1]; k++) {
            pd.push_back(faces[k]);
            pair_src.push_back(point_offsets[s]);
            pair_off.push_back(pair_off.back() + cnt);
        }
        surf_pair0.push_back((int32_t)pd.size());
    }
    const int n_pairs = (int)pd.size();
    const int64_t E = pair_off.back();
    if (E > WN_MAX_QUERIES_PER_CALL) return WN_ERR_LIMIT;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    double2 *xp = nullptr;
    uint8_t *xst = nullptr;
    int64_t *d_pair_off = nullptr, *d_pair_src = nullptr, *d_pt_off = nullptr;
    int32_t *d_surf_pair0 = nullptr;
    wn_status rc = WN_OK;
    if ((e = pool_alloc(xp, (size_t)E, s)) != cudaSuccess || (e = pool_alloc(xst, (size_t)E, s)) != cudaSuccess ||
        (e = pool_alloc(d_pair_off, pair_off.size(), s)) != cudaSuccess ||
        (e = pool_alloc(d_pair_src, pair_src.size(), s)) != cudaSuccess ||
        (e = pool_alloc(d_pt_off, (size_t)n_surfaces + 1, s)) != cudaSuccess ||
        (e = pool_alloc(d_surf_pair0, surf_pair0.size(), s)) != cudaSuccess) {
        rc = e == cudaErrorMemoryAllocation ? WN_ERR_OOM : WN_ERR_CUDA;
    }
    if (rc == WN_OK) {
        if ((e = cudaMemcpyAsync(d_pair_off, pair_off.data(), pair_off.size() * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (n_pairs && (e = cudaMemcpyAsync(d_pair_src, pair_src.data(), pair_src.size() * sizeof(int64_t),
                                             cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
            (e = cudaMemcpyAsync(d_pt_off, point_offsets, ((size_t)n_surfaces + 1) * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(d_surf_pair0, surf_pair0.data(), surf_pair0.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, s)) != cudaSuccess)
            rc = WN_ERR_CUDA;
    }
    if (rc == WN_OK && E > 0) {
        k_expand_points<<<grid_for(E), 256, 0, s>>>(reinterpret_cast<const double2 *>(points), xp, d_pair_off,
                                                    d_pair_src, n_pairs, E);
        if (cudaGetLastError() != cudaSuccess) rc = WN_ERR_CUDA;
        if (rc == WN_OK)
            rc = wn_query_batched(pd.data(), n_pairs, pair_off.data(), reinterpret_cast<const double *>(xp), nullptr,
                                  xst, precision, stream);
    }
    if (rc == WN_OK) {
        k_or_reduce<<<grid_for(n_points), 256, 0, s>>>(xst, out_inside, d_pt_off, d_surf_pair0, d_pair_off,
                                                       n_surfaces, n_points);
        if (cudaGetLastError() != cudaSuccess) rc = WN_ERR_CUDA;
    }
    for (void *p : {(void *)xp, (void *)xst, (void *)d_pair_off, (void *)d_pair_src, (void *)d_pt_off,
                    (void *)d_surf_pair0})
        if (p) cudaFreeAsync(p, s);
    return rc;
}

extern "C" wn_status wn_query_midpoints(const wn_domain *domain, const double *pieces, int64_t n,
                                        uint8_t *out_state, int precision, wn_stream stream)
{
    if (!domain || n < 0) return WN_ERR_ARG;
    if (n == 0) return WN_OK;
    if (n > WN_MAX_QUERIES_PER_CALL) return WN_ERR_LIMIT;
    if (!pieces || !out_state || !on_device(pieces) || !on_device(out_state)) return WN_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(pieces) & 31) return WN_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double2 *mid = nullptr;
    cudaError_t e = pool_alloc(mid, (size_t)n, s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? WN_ERR_OOM : WN_ERR_CUDA;
    k_midpoints<<<grid_for(n), 256, 0, s>>>(reinterpret_cast<const double4 *>(pieces), mid, n);
    wn_status rc = cudaGetLastError() == cudaSuccess ? WN_OK : WN_ERR_CUDA;
    if (rc == WN_OK)
        rc = wn_query(domain, reinterpret_cast<const double *>(mid), n, nullptr, out_state, precision, stream);
    cudaFreeAsync(mid, s);
    return rc;
}
