// Per-graph features for the threshold picker and the adjusted Rand index.
//
// Features (tec_features): the 64-bin histogram of Tectonic weights on the
// grid i/128 -- bin = min(63, floor(128 t / (deg u + deg v))), the level an
// edge reaches in a sweep of thresholds i/128 -- divided by m, then
// ln(2m / n) and ln(m); one row of 66 floats per graph of a batch.
//
// ARI (tec_ari, Hubert & Arabie 1985): for component labels c and reference
// blocks b of one graph with n vertices,
//   S_ab = sum over cells (c, b) of C(n_cb, 2), S_a = sum over components of
//   C(size, 2), S_b = sum over blocks of C(size, 2), T = C(n, 2),
//   ARI = (2 T S_ab - 2 S_a S_b) / (T (S_a + S_b) - 2 S_a S_b),
// with ARI = 1 when the denominator is 0 (both partitions all singletons or
// both one cluster) or n < 2.  Cell counts come from a device hash table
// keyed by (component root, block); all sums are exact 64-bit integers and
// the ratio is formed from exact 128-bit numerator and denominator.
#include "tec_internal.cuh"

namespace tec {
namespace {

constexpr int NBINS = 64;

__device__ __forceinline__ int seg_of(const int64_t *seg_off, int nseg, int64_t x) {
    int lo = 0, hi = nseg - 1;                   // last segment starting at or before x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(TILE_THREADS)
k_feat_hist(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t, int64_t n, int64_t m,
            const int64_t *seg_off, int nseg, unsigned int *hist, unsigned long long *ctr) {
    __shared__ unsigned int s_h[NBINS];
    if (graph_bad(ctr)) return;
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    const int64_t klast = min(k0 + TILE, m) - 1;
    const int64_t r0 = row_search(ooff, 0, n - 1, k0);
    const int64_t r1 = row_search(ooff, r0, n - 1, klast);
    const int s0 = seg_off ? seg_of(seg_off, nseg, r0) : 0;
    const int s1 = seg_off ? seg_of(seg_off, nseg, r1) : 0;
    const bool one = s0 == s1;                   // the common case: aggregate in shared memory
    if (threadIdx.x < NBINS) s_h[threadIdx.x] = 0u;
    __syncthreads();
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (j >= m) break;
        const int64_t u = row_search(ooff, r0, r1, j);
        const int64_t s = (int64_t)deg[u] + deg[ocol[j]];
        int64_t b = (128 * (int64_t)t[j]) / s;
        if (b > NBINS - 1) b = NBINS - 1;
        if (one) atomicAdd(&s_h[b], 1u);
        else atomicAdd(&hist[(int64_t)seg_of(seg_off, nseg, u) * NBINS + b], 1u);
    }
    __syncthreads();
    if (one && threadIdx.x < NBINS && s_h[threadIdx.x]) atomicAdd(&hist[(int64_t)s0 * NBINS + threadIdx.x], s_h[threadIdx.x]);
}

// One warp per graph: 64 normalised bins, ln(2m/n), ln(m).
__global__ void k_feat_final(const unsigned int *hist, const int64_t *seg_off, int nseg, int64_t n_all,
                             float *feat) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (w >= nseg) return;
    const int lane = (int)lane_id();
    const unsigned int h0 = hist[(int64_t)w * NBINS + lane], h1 = hist[(int64_t)w * NBINS + 32 + lane];
    unsigned long long mm = (unsigned long long)h0 + h1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mm += __shfl_xor_sync(0xffffffffu, mm, o);
    const int64_t nv = seg_off ? seg_off[w + 1] - seg_off[w] : n_all;
    float *f = feat + (int64_t)w * (NBINS + 2);
    const float mf = (float)mm;
    f[lane] = mm ? (float)h0 / mf : 0.f;
    f[32 + lane] = mm ? (float)h1 / mf : 0.f;
    if (lane == 0) {
        f[NBINS] = (mm && nv) ? logf(2.f * mf / (float)nv) : 0.f;
        f[NBINS + 1] = mm ? logf(mf) : 0.f;
    }
}

// ---------------------------------------------------------------- ARI

constexpr unsigned long long EMPTY = ~0ull;

__device__ __forceinline__ uint64_t hkey(uint64_t key, int bits) {
    return (key * 0x9E3779B97F4A7C15ull) >> (64 - bits);
}

__global__ void k_block_sizes(const int32_t *truth, int64_t n, const int64_t *seg_off, int nseg, unsigned int *bsz,
                              unsigned long long *ctr) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int b = truth[x];
        if (b < 0 || b >= NBINS) { flag_status(ctr, ST_BADGRAPH); continue; }
        const int s = seg_off ? seg_of(seg_off, nseg, x) : 0;
        atomicAdd(&bsz[(int64_t)s * NBINS + b], 1u);
    }
}

// Component sizes and (root, block) cell counts of one level.
__global__ void k_ari_cells(const int32_t *labels, const int32_t *truth, int64_t n, const int64_t *seg_off, int nseg,
                            unsigned int *size, unsigned long long *keys, unsigned int *cnt, int bits,
                            unsigned long long *ctr) {
    const uint64_t mask = (1ull << bits) - 1ull;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int b = truth[x];
        if (b < 0 || b >= NBINS) continue;       // reported by k_block_sizes
        const int64_t base = seg_off ? seg_off[seg_of(seg_off, nseg, x)] : 0;
        const int64_t root = base + labels[x];
        if (root < 0 || root >= n) { flag_status(ctr, ST_BADGRAPH); continue; }
        atomicAdd(&size[root], 1u);
        const uint64_t key = ((uint64_t)root << 6) | (uint64_t)b;
        uint64_t h = hkey(key, bits);
        for (uint64_t probe = 0; probe <= mask; ++probe) {
            const unsigned long long old = atomicCAS(&keys[h], EMPTY, (unsigned long long)key);
            if (old == EMPTY || old == key) {
                atomicAdd(&cnt[h], 1u);
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

__device__ __forceinline__ unsigned long long c2(unsigned long long x) { return x * (x - (x > 0)) / 2; }

// sums[3 s + 0] = S_ab, sums[3 s + 1] = S_a of segment s.
__global__ void k_ari_reduce(const unsigned long long *keys, const unsigned int *cnt, int64_t tsize,
                             const unsigned int *size, int64_t n, const int64_t *seg_off, int nseg,
                             unsigned long long *sums) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tsize; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned int c = cnt[i];
        if (c > 1) {
            const int64_t root = (int64_t)(keys[i] >> 6);
            const int s = seg_off ? seg_of(seg_off, nseg, root) : 0;
            atomicAdd(&sums[3 * s], c2(c));
        }
        if (i < n && size[i] > 1) {
            const int s = seg_off ? seg_of(seg_off, nseg, i) : 0;
            atomicAdd(&sums[3 * s + 1], c2(size[i]));
        }
    }
}

__device__ double i128_to_double(__int128 v) {
    const bool neg = v < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const double d = (double)(uint64_t)(u >> 64) * 18446744073709551616.0 + (double)(uint64_t)u;
    return neg ? -d : d;
}

__global__ void k_ari_final(const unsigned long long *sums, const unsigned int *bsz, const int64_t *seg_off, int nseg,
                            int64_t n_all, double *out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const int64_t nv = seg_off ? seg_off[s + 1] - seg_off[s] : n_all;
    unsigned long long sb = 0;
    for (int b = 0; b < NBINS; ++b) sb += c2(bsz[(int64_t)s * NBINS + b]);
    const unsigned long long sab = sums[3 * s], sa = sums[3 * s + 1];
    const unsigned long long T = (unsigned long long)nv * (unsigned long long)(nv > 0 ? nv - 1 : 0) / 2;
    const __int128 num = 2 * (__int128)T * sab - 2 * (__int128)sa * sb;
    const __int128 den = (__int128)T * (sa + sb) - 2 * (__int128)sa * sb;
    out[s] = (nv < 2 || den == 0) ? 1.0 : i128_to_double(num) / i128_to_double(den);
}

// Per graph: the first level of highest ARI (ari is k x nseg).
__global__ void k_best_level(const double *ari, int k, int nseg, int32_t *best, double *best_ari) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    int bi = 0;
    double bv = ari[s];
    for (int L = 1; L < k; ++L) {
        const double v = ari[(int64_t)L * nseg + s];
        if (v > bv) { bv = v; bi = L; }
    }
    best[s] = bi;
    if (best_ari) best_ari[s] = bv;
}

inline unsigned grid_for(int64_t work) {
    const int64_t g = ceil_div(work > 0 ? work : 1, 256);
    return (unsigned)(g < 65536 ? g : 65536);
}

}  // namespace

cudaError_t launch_features(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                            int64_t n, int64_t m, const int64_t *seg_off, int nseg, unsigned int *hist, float *feat,
                            unsigned long long *ctr, cudaStream_t s) {
    const int ns = seg_off ? nseg : 1;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)ns * NBINS * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (m > 0)
        k_feat_hist<<<(unsigned)ceil_div(m, TILE), TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, seg_off, ns, hist,
                                                                         ctr);
    k_feat_final<<<(unsigned)ceil_div((int64_t)ns * 32, 256), 256, 0, s>>>(hist, seg_off, ns, n, feat);
    count_launches(m > 0 ? 2 : 1);
    return cudaGetLastError();
}

cudaError_t launch_best_level(const double *ari, int k, int nseg, int32_t *best, double *best_ari, cudaStream_t s) {
    if (nseg <= 0) return cudaSuccess;
    k_best_level<<<(unsigned)ceil_div(nseg, 128), 128, 0, s>>>(ari, k, nseg, best, best_ari);
    count_launches(1);
    return cudaGetLastError();
}

int ari_table_bits(int64_t n) {
    int bits = 6;
    while (((int64_t)1 << bits) < 2 * n) ++bits;
    return bits;
}

cudaError_t launch_ari(const int32_t *labels, int k, const int32_t *truth, int64_t n, const int64_t *seg_off, int nseg,
                       unsigned int *bsz, unsigned int *size, unsigned long long *keys, unsigned int *cnt,
                       unsigned long long *sums, double *out, unsigned long long *ctr, cudaStream_t s) {
    const int ns = seg_off ? nseg : 1;
    const int bits = ari_table_bits(n);
    const int64_t tsize = (int64_t)1 << bits;
    cudaError_t e = cudaMemsetAsync(bsz, 0, (size_t)ns * NBINS * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (n > 0) k_block_sizes<<<grid_for(n), 256, 0, s>>>(truth, n, seg_off, ns, bsz, ctr);
    int launched = n > 0 ? 1 : 0;
    for (int L = 0; L < k; ++L) {
        if ((e = cudaMemsetAsync(keys, 0xFF, (size_t)tsize * sizeof(unsigned long long), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(cnt, 0, (size_t)tsize * sizeof(unsigned int), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(size, 0, (size_t)(n > 0 ? n : 1) * sizeof(unsigned int), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(sums, 0, (size_t)3 * ns * sizeof(unsigned long long), s)) != cudaSuccess) return e;
        if (n > 0) {
            k_ari_cells<<<grid_for(n), 256, 0, s>>>(labels + (int64_t)L * n, truth, n, seg_off, ns, size, keys, cnt,
                                                    bits, ctr);
            k_ari_reduce<<<grid_for(tsize), 256, 0, s>>>(keys, cnt, tsize, size, n, seg_off, ns, sums);
            launched += 2;
        }
        k_ari_final<<<(unsigned)ceil_div(ns, 128), 128, 0, s>>>(sums, bsz, seg_off, ns, n, out + (int64_t)L * ns);
        ++launched;
    }
    count_launches(launched);
    return cudaGetLastError();
}

}  // namespace tec
