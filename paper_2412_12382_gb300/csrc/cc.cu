// Connected components of the kept subgraph (Algorithm 1, second step) with the
// lock-free union-find of uf.cuh: init parent[x] = x, hook the endpoints of
// every kept edge, then resolve every vertex to its root, which is the
// smallest id of its component, and count the roots.
#include "tec_internal.cuh"
#include "uf.cuh"

namespace tec {
namespace {

__global__ void k_cc_init(int32_t *parent, int64_t n) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x)
        parent[x] = (int32_t)x;
}

// Streams the oriented edges in tiles (rows found by binary search) and hooks
// every edge whose keep bit is set.
__global__ void __launch_bounds__(TILE_THREADS)
k_cc_hook(const int64_t *ooff, const int32_t *ocol, const uint32_t *keep, int64_t n, int64_t m,
          const int32_t *orows, const int32_t *osrc, int32_t *parent, unsigned long long *ctr) {
    if (graph_bad(ctr)) return;
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    int64_t r0, r1;
    tile_row_range(orows, ooff, n, m, r0, r1);
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (j >= m) break;
        if (!((keep[j >> 5] >> (j & 31)) & 1u)) continue;
        const int64_t u = edge_source(osrc, ooff, r0, r1, j);
        uf_link(parent, (int32_t)u, ocol[j], ctr);
    }
}

// labels must not alias parent: other threads' path compression can still
// re-point parent[x] at an intermediate ancestor after x has been resolved.
__global__ void k_cc_finish(int32_t *parent, int64_t n, int32_t *labels, unsigned long long *ctr) {
    int roots = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = uf_find(parent, (int32_t)x);
        parent[x] = r;
        if (labels) labels[x] = r;
        roots += (r == x) ? 1 : 0;
    }
    roots = warp_sum(roots);
    if (lane_id() == 0 && roots) atomicAdd(&ctr[C_NCOMP], (unsigned long long)roots);
}

inline unsigned grid_for(int64_t work) {
    int64_t g = ceil_div(work > 0 ? work : 1, 256);
    return (unsigned)(g < 65536 ? g : 65536);
}

}  // namespace

cudaError_t launch_cc_init(int32_t *parent, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_cc_init<<<grid_for(n), 256, 0, s>>>(parent, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cc_hook(const int64_t *ooff, const int32_t *ocol, const uint32_t *keep, int64_t n,
                           int64_t m, const int32_t *orows, const int32_t *osrc, int32_t *parent,
                           unsigned long long *ctr, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    k_cc_hook<<<(unsigned)ceil_div(m, TILE), TILE_THREADS, 0, s>>>(ooff, ocol, keep, n, m, orows, osrc, parent, ctr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cc_finish(int32_t *parent, int64_t n, int32_t *labels, unsigned long long *ctr,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_cc_finish<<<grid_for(n), 256, 0, s>>>(parent, n, labels, ctr);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace tec
