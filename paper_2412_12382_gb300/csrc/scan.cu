// Exclusive prefix sums (int64 results) used to turn per-tile or per-row
// counts into output offsets.  Three passes: per-block totals, one block that
// scans the totals, per-block rescan with the carried-in offset.
#include "tec_internal.cuh"

namespace tec {
namespace {

constexpr int SB = 256;            // threads per block
constexpr int SI = 8;              // items per thread
constexpr int SCHUNK = SB * SI;    // 2048 items per block

template <typename T>
__device__ __forceinline__ int64_t load_or0(const T *in, int64_t i, int64_t N) {
    return i < N ? (int64_t)in[i] : 0;
}

__device__ __forceinline__ int64_t warp_incl_scan64(int64_t x) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)(threadIdx.x & 31) >= o) x += y;
    }
    return x;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ __forceinline__ int64_t block_excl_scan64(int64_t x, int64_t *total) {
    __shared__ int64_t warp_tot[SB / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan64(x);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t v = lane < SB / 32 ? warp_tot[lane] : 0;
        int64_t vi = warp_incl_scan64(v);
        if (lane < SB / 32) warp_tot[lane] = vi - v;
        if (lane == SB / 32 - 1) *total = vi;
    }
    __syncthreads();
    int64_t r = warp_tot[w] + inc - x;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void k_block_totals(const T *in, int64_t N, int64_t *bsum) {
    int64_t base = (int64_t)blockIdx.x * SCHUNK + (int64_t)threadIdx.x * SI;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SI; ++i) s += load_or0(in, base + i, N);
    __shared__ int64_t tot;
    block_excl_scan64(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One block: in-place exclusive scan of bsum[0..nb), bsum[nb] = total.
__global__ void k_scan_totals(int64_t *bsum, int64_t nb) {
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t c = 0; c < nb; c += SB) {
        int64_t i = c + threadIdx.x;
        int64_t x = i < nb ? bsum[i] : 0;
        int64_t ex = block_excl_scan64(x, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

template <typename T>
__global__ void k_block_rescan(const T *in, int64_t N, const int64_t *bsum, int64_t *out) {
    int64_t base = (int64_t)blockIdx.x * SCHUNK + (int64_t)threadIdx.x * SI;
    int64_t v[SI];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SI; ++i) { v[i] = load_or0(in, base + i, N); s += v[i]; }
    __shared__ int64_t tot;
    int64_t ex = block_excl_scan64(s, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SI; ++i) {
        if (base + i < N) out[base + i] = ex;
        ex += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[N] = bsum[gridDim.x];
}

__global__ void k_zero_total(int64_t *out) { out[0] = 0; }

template <typename T>
cudaError_t scan_impl(const T *in, int64_t N, int64_t *out, int64_t *bsum, cudaStream_t s) {
    if (N <= 0) {
        k_zero_total<<<1, 1, 0, s>>>(out);
        count_launches(1);
        return cudaGetLastError();
    }
    int64_t nb = ceil_div(N, SCHUNK);
    k_block_totals<T><<<(unsigned)nb, SB, 0, s>>>(in, N, bsum);
    k_scan_totals<<<1, SB, 0, s>>>(bsum, nb);
    k_block_rescan<T><<<(unsigned)nb, SB, 0, s>>>(in, N, bsum, out);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace

int64_t scan_bsum_size(int64_t N) { return ceil_div(N > 0 ? N : 1, SCHUNK) + 1; }

cudaError_t scan_exclusive_i64(const int64_t *in, int64_t N, int64_t *out, int64_t *bsum, cudaStream_t s) {
    return scan_impl<int64_t>(in, N, out, bsum, s);
}

cudaError_t scan_exclusive_i32(const int32_t *in, int64_t N, int64_t *out, int64_t *bsum, cudaStream_t s) {
    return scan_impl<int32_t>(in, N, out, bsum, s);
}

}  // namespace tec
