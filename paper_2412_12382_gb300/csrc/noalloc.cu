// Connected components of a caller-supplied edge list without any memory
// allocation (tec_components_noalloc in include/tectonic.h).
//
// Some callers cannot allocate device memory at the point where they need
// components: code that runs inside a host application which owns the GPU
// memory budget and forbids allocations behind its back, latency-sensitive
// callers for which a cudaMalloc / cudaFree (which can synchronise the whole
// device) is not acceptable, or callers that must not fail halfway for lack of
// memory.  This entry point takes its union-find scratch from one file-scope
// device array of fixed size instead.  Every GPU that loads the library holds
// that array (TEC_NOALLOC_MAX_VERTICES int32 plus a few counters, about 16 MiB)
// until the process exits.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents, so each call first re-initialises the parents and zeroes
// its counters.  Calls whose work overlaps on the GPU (different streams or
// host threads without ordering between them) race on the array and give
// wrong labels; callers must serialise them.
#include <mutex>

#include "tec_internal.cuh"
#include "uf.cuh"

namespace tec {
namespace {

constexpr int64_t NA_MAX_N = TEC_NOALLOC_MAX_VERTICES;
constexpr int NA_CTR = 64;     // int32 slots after the parents: status word and root count (as u64)

// Parents of the union-find forest, then the counters (8-byte aligned: NA_MAX_N
// is a multiple of 64).
static __device__ __align__(256) int32_t na_scratch[NA_MAX_N + NA_CTR];

constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
int32_t *na_ptr[NA_MAX_DEVICES] = {};

__global__ void k_na_init(int32_t *parent, int64_t n, unsigned long long *ctr) {
    if (blockIdx.x == 0 && threadIdx.x < 2) ctr[threadIdx.x] = 0ull;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        parent[x] = (int32_t)x;
}

// ctr[0] is the status word (ST_* bits), ctr[1] the number of roots.
__global__ void k_na_hook(const int32_t *eu, const int32_t *ev, const uint8_t *keep, int64_t n, int64_t m,
                          int32_t *parent, unsigned long long *ctr) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        if (keep && !keep[e]) continue;
        const int32_t a = eu[e], b = ev[e];
        if (a < 0 || b < 0 || (int64_t)a >= n || (int64_t)b >= n) {
            atomicOr(&ctr[0], (unsigned long long)ST_BADGRAPH);
            continue;
        }
        uf_link(parent, a, b, ctr);
    }
}

__global__ void k_na_finish(int32_t *parent, int64_t n, int32_t *labels, unsigned long long *ctr) {
    int roots = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = uf_find(parent, (int32_t)x);
        labels[x] = r;
        roots += (r == x) ? 1 : 0;
    }
    roots = warp_sum(roots);
    if (lane_id() == 0 && roots) atomicAdd(&ctr[1], (unsigned long long)roots);
}

unsigned grid_for(int64_t work) {
    const int64_t g = ceil_div(work > 0 ? work : 1, 256);
    return (unsigned)(g < 4096 ? g : 4096);
}

// Device address of na_scratch on the current device (looked up once per device).
tec_status scratch_address(int32_t **out) {
    int dev = 0;
    TEC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return set_error(TEC_EINVAL, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
        if (e != cudaSuccess || !p)
            return set_error(TEC_ECUDA, "cudaGetSymbolAddress of the component scratch failed: %s",
                             cudaGetErrorString(e));
        na_ptr[dev] = static_cast<int32_t *>(p);
    }
    *out = na_ptr[dev];
    return TEC_OK;
}

}  // namespace
}  // namespace tec

using namespace tec;

extern "C" tec_status tec_components_noalloc(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                                             const uint8_t *keep, int32_t *labels_out, int64_t *ncomp_out,
                                             void *stream) {
    clear_error();
    if (n < 0 || m < 0) return set_error(TEC_EINVAL, "negative size");
    if (n > NA_MAX_N)
        return set_error(TEC_EINVAL, "n=%lld exceeds the allocation-free maximum of %lld vertices", (long long)n,
                         (long long)NA_MAX_N);
    if (m > 0 && (!eu || !ev)) return set_error(TEC_EINVAL, "edge arrays are NULL");
    if (n > 0 && !labels_out) return set_error(TEC_EINVAL, "labels_out is NULL");
    int32_t *parent = nullptr;
    TEC_TRY(scratch_address(&parent));
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(parent + NA_MAX_N);
    cudaStream_t s = (cudaStream_t)stream;
    k_na_init<<<grid_for(n), 256, 0, s>>>(parent, n, ctr);
    if (m > 0) k_na_hook<<<grid_for(m), 256, 0, s>>>(eu, ev, keep, n, m, parent, ctr);
    if (n > 0) k_na_finish<<<grid_for(n), 256, 0, s>>>(parent, n, labels_out, ctr);
    count_launches(1 + (m > 0) + (n > 0));
    TEC_CUDA(cudaGetLastError());
    unsigned long long host_ctr[2] = {0ull, 0ull};
    TEC_CUDA(cudaMemcpyAsync(host_ctr, ctr, sizeof(host_ctr), cudaMemcpyDeviceToHost, s));
    TEC_CUDA(cudaStreamSynchronize(s));
    if (host_ctr[0] & ST_BADGRAPH) return set_error(TEC_EINVAL, "an edge endpoint is outside [0, n)");
    if (host_ctr[0] & ST_TIMEOUT) return set_error(TEC_ETIMEOUT, "a bounded union-find loop reached its cap");
    if (ncomp_out) *ncomp_out = (int64_t)host_ctr[1];
    return TEC_OK;
}
