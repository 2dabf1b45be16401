// Device R-MAT sampler: the same published definition as graphgen/rmat.py
// (SplitMix64 finaliser draws keyed by (seed, sample), integer quadrant cut
// points, keyed 4-round Feistel relabelling), used to build large inputs on
// the GPU.  It is an input generator, not part of the community-detection
// method, and shares nothing with the method's library.
//
// Directed entries (src -> dst, both directions of every non-loop sample) are
// bucketed by the top `bucket_bits` bits of src, so a large graph can be
// deduplicated and sorted one bucket range at a time.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct RmatParams {
    int scale;
    uint32_t A, AB, ABC;
    uint64_t key;
    uint64_t fk[4];
    int bucket_bits;
};

__device__ __forceinline__ uint32_t feistel(uint32_t x, const RmatParams &p) {
    const int lo_bits = p.scale / 2;
    const int hi_bits = p.scale - lo_bits;
    const uint64_t mask_lo = (1ull << lo_bits) - 1ull;
    const uint64_t mask_hi = (1ull << hi_bits) - 1ull;
    uint64_t L = (uint64_t)x >> lo_bits;
    uint64_t R = (uint64_t)x & mask_lo;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if ((r & 1) == 0) L ^= mix64(p.fk[r] ^ R) & mask_hi;
        else R ^= mix64(p.fk[r] ^ L) & mask_lo;
    }
    return (uint32_t)((L << lo_bits) | R);
}

__device__ __forceinline__ void sample(uint64_t i, const RmatParams &p, uint32_t &u, uint32_t &v) {
    const uint64_t ki = mix64(p.key ^ mix64(i));
    uint32_t uu = 0, vv = 0;
    const int pairs = (p.scale + 1) / 2;
    for (int j = 0; j < pairs; ++j) {
        const uint64_t w = mix64(ki ^ (uint64_t)j);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int lvl = 2 * j + h;
            if (lvl >= p.scale) break;
            const uint32_t r = h == 0 ? (uint32_t)(w >> 32) : (uint32_t)(w & 0xFFFFFFFFull);
            const uint32_t ub = r >= p.AB ? 1u : 0u;
            const uint32_t vb = ((r >= p.A && r < p.AB) || r >= p.ABC) ? 1u : 0u;
            uu |= ub << lvl;
            vv |= vb << lvl;
        }
    }
    u = feistel(uu, p);
    v = feistel(vv, p);
}

__global__ void k_count(RmatParams p, uint64_t nsamples, unsigned long long *counts) {
    extern __shared__ unsigned int hist[];
    const int nb = 1 << p.bucket_bits;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const int shift = p.scale - p.bucket_bits;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsamples;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u, v;
        sample(i, p, u, v);
        if (u == v) continue;
        atomicAdd(&hist[u >> shift], 1u);
        atomicAdd(&hist[v >> shift], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (hist[b]) atomicAdd(&counts[b], (unsigned long long)hist[b]);
}

__global__ void k_emit(RmatParams p, uint64_t nsamples, int b0, int b1, long long *keys,
                       unsigned long long *cursor, long long cap) {
    const int shift = p.scale - p.bucket_bits;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsamples;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u, v;
        sample(i, p, u, v);
        if (u == v) continue;
        const int bu = (int)(u >> shift), bv = (int)(v >> shift);
        if (bu >= b0 && bu < b1) {
            unsigned long long at = atomicAdd(cursor, 1ull);
            if ((long long)at < cap) keys[at] = ((long long)u << 32) | (long long)v;
        }
        if (bv >= b0 && bv < b1) {
            unsigned long long at = atomicAdd(cursor, 1ull);
            if ((long long)at < cap) keys[at] = ((long long)v << 32) | (long long)u;
        }
    }
}

RmatParams make_params(int scale, uint32_t A, uint32_t AB, uint32_t ABC, uint64_t key, const uint64_t *fk,
                       int bucket_bits) {
    RmatParams p;
    p.scale = scale;
    p.A = A;
    p.AB = AB;
    p.ABC = ABC;
    p.key = key;
    for (int r = 0; r < 4; ++r) p.fk[r] = fk[r];
    p.bucket_bits = bucket_bits;
    return p;
}

// ---------------------------------------------------------------- DC-SBM

__device__ __forceinline__ uint64_t draw_word(uint64_t key, uint64_t counter) { return mix64(key ^ mix64(counter)); }

// Largest i in [0, len) with a[i] <= x (a non-decreasing, a[0] <= x).
__device__ __forceinline__ int64_t pick(const long long *a, int64_t len, long long x) {
    int64_t lo = 0, hi = len - 1;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (a[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_dcsbm(uint64_t key, int64_t samples, int n, int k, uint64_t mu_cut, const int *block,
                        const int *order, const long long *cum, const long long *bstart, long long voff,
                        long long *keys) {
    const unsigned long long W = (unsigned long long)cum[n];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < samples;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t w0 = draw_word(key, 4ull * e), w1 = draw_word(key, 4ull * e + 1);
        const uint64_t w2 = draw_word(key, 4ull * e + 2), w3 = draw_word(key, 4ull * e + 3);
        int u, v;
        if ((w0 >> 11) < mu_cut) {
            const int64_t iu = pick(cum, n + 1, (long long)__umul64hi(w1, W));
            const int bu = block[order[iu]];
            const unsigned long long vb = (unsigned long long)(bstart[bu + 1] - bstart[bu]);
            int64_t iv = iu;
            if (W - vb != 0) {
                long long pv = (long long)__umul64hi(w2, W - vb);
                if (pv >= bstart[bu]) pv += (long long)vb;
                if (pv > (long long)W - 1) pv = (long long)W - 1;
                iv = pick(cum, n + 1, pv);
            }
            u = order[iu];
            v = order[iv];
        } else {
            const int64_t b = pick(bstart, k + 1, (long long)__umul64hi(w1, W));
            const unsigned long long vb = (unsigned long long)(bstart[b + 1] - bstart[b]);
            u = order[pick(cum, n + 1, bstart[b] + (long long)__umul64hi(w2, vb))];
            v = order[pick(cum, n + 1, bstart[b] + (long long)__umul64hi(w3, vb))];
        }
        const long long gu = voff + u, gv = voff + v;
        keys[2 * e] = u == v ? -1ll : ((gu << 32) | gv);
        keys[2 * e + 1] = u == v ? -1ll : ((gv << 32) | gu);
    }
}

}  // namespace

extern "C" {

// Directed keys (src << 32 | dst, both directions, -1 for self-loops) of the
// samples of one DC-SBM graph whose vertex arrays are on the device; vertex
// ids are offset by voff.  keys needs 2 * samples entries.
int gg_dcsbm(uint64_t key, int64_t samples, int n, int k, uint64_t mu_cut, const int *block, const int *order,
             const long long *cum, const long long *bstart, long long voff, long long *keys, void *stream) {
    if (n < 1 || k < 1) return 1;
    k_dcsbm<<<2048, 256, 0, (cudaStream_t)stream>>>(key, samples, n, k, mu_cut, block, order, cum, bstart, voff, keys);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}


// counts[2^bucket_bits] (device, zeroed by the caller) += directed entries per src bucket.
int gg_rmat_count(int scale, uint64_t nsamples, uint32_t A, uint32_t AB, uint32_t ABC, uint64_t key,
                  const uint64_t *feistel_keys, int bucket_bits, unsigned long long *counts, void *stream) {
    if (scale < 2 || scale > 31 || bucket_bits < 0 || bucket_bits > scale || bucket_bits > 12) return 1;
    RmatParams p = make_params(scale, A, AB, ABC, key, feistel_keys, bucket_bits);
    const size_t smem = sizeof(unsigned int) << bucket_bits;
    k_count<<<4096, 256, smem, (cudaStream_t)stream>>>(p, nsamples, counts);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// Writes the keys (src << 32 | dst) of buckets [b0, b1) to keys[0..cap) in
// arbitrary order; *cursor (device, zeroed by the caller) ends at the count.
int gg_rmat_emit(int scale, uint64_t nsamples, uint32_t A, uint32_t AB, uint32_t ABC, uint64_t key,
                 const uint64_t *feistel_keys, int bucket_bits, int b0, int b1, long long *keys,
                 unsigned long long *cursor, long long cap, void *stream) {
    if (scale < 2 || scale > 31 || bucket_bits < 0 || bucket_bits > scale) return 1;
    RmatParams p = make_params(scale, A, AB, ABC, key, feistel_keys, bucket_bits);
    k_emit<<<8192, 256, 0, (cudaStream_t)stream>>>(p, nsamples, b0, b1, keys, cursor, cap);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
