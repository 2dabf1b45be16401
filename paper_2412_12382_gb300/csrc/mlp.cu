// Learned threshold picker: a 66 -> 128 -> 128 -> 1 ReLU network on the
// per-graph features of tec_features, trained with mean squared error and
// Adam (Kingma & Ba 2015).  The paper picks thresholds by rules of thumb
// (Sec. IV-D); this network replaces them, rated against the best threshold
// of the full sweep.
//
// Parameters (float32, one device vector): W1 [128 x 66] row-major, b1 [128],
// W2 [128 x 128], b2 [128], w3 [128], b3.  A step on a batch of B samples:
//   k_forward   one 128-thread block per sample: h1 = relu(W1 x + b1),
//               h2 = relu(W2 h1 + b2), y = w3 . h2 + b3 (pre-activations kept);
//   k_backward  one block per sample: dy = 2 (y - t) / B, dz2 = dy w3 [z2 > 0],
//               dz1 = (W2^T dz2) [z1 > 0];
//   k_grad      one thread per parameter, summing its batch contributions in
//               sample order (no atomics: gradients are reproducible);
//   k_adam      one thread per parameter.
// Mini-batches of a training epoch follow a keyed Feistel permutation of the
// sample indices, computed on the fly.
#include <cmath>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "tec_internal.cuh"

namespace tec {
namespace {

constexpr int IN = TEC_PICKER_INPUTS;
constexpr int HID = TEC_PICKER_HIDDEN;
constexpr int OFF_W1 = 0, OFF_B1 = HID * IN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID;
constexpr int OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == TEC_PICKER_PARAMS, "parameter layout");

__device__ __forceinline__ float rb(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <bool BF16>
__global__ void __launch_bounds__(HID) k_forward(const float *__restrict__ P, const float *__restrict__ X, int64_t B,
                                                 float *__restrict__ Z1, float *__restrict__ Z2,
                                                 float *__restrict__ Y) {
    __shared__ float sx[IN], sxl[IN], sh[HID], sred[HID / 32];
    const int64_t b = blockIdx.x;
    if (b >= B) return;
    const int j = threadIdx.x;
    // bf16: each input is the sum of two bf16 values (x = hi + lo, hi = bf16(x),
    // lo = bf16(x - hi)), so the inputs, whose rounding would otherwise move
    // the output most, keep about 16 significant bits; weights and hidden
    // activations are single bf16 values; products accumulate in float32
    for (int i = j; i < IN; i += HID) {
        const float x = X[b * IN + i];
        sx[i] = BF16 ? rb(x) : x;
        sxl[i] = BF16 ? rb(x - rb(x)) : 0.f;
    }
    __syncthreads();
    float z = P[OFF_B1 + j];
    for (int i = 0; i < IN; ++i) {
        const float w = BF16 ? rb(P[OFF_W1 + j * IN + i]) : P[OFF_W1 + j * IN + i];
        z += w * sx[i];
        if (BF16) z += w * sxl[i];
    }
    if (Z1) Z1[b * HID + j] = z;
    sh[j] = BF16 ? rb(fmaxf(z, 0.f)) : fmaxf(z, 0.f);
    __syncthreads();
    float z2 = P[OFF_B2 + j];
    for (int k = 0; k < HID; ++k) z2 += (BF16 ? rb(P[OFF_W2 + j * HID + k]) : P[OFF_W2 + j * HID + k]) * sh[k];
    if (Z2) Z2[b * HID + j] = z2;
    const float h2 = BF16 ? rb(fmaxf(z2, 0.f)) : fmaxf(z2, 0.f);
    float c = (BF16 ? rb(P[OFF_W3 + j]) : P[OFF_W3 + j]) * h2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((j & 31) == 0) sred[j >> 5] = c;
    __syncthreads();
    if (j == 0) {
        float y = P[OFF_B3];
        for (int w = 0; w < HID / 32; ++w) y += sred[w];
        Y[b] = y;
    }
}

// With GIVEN, DY already holds dloss/dy of every sample (the soft-level
// loss); otherwise dy is the squared error's 2 (y - t) / B.
template <bool GIVEN>
__global__ void __launch_bounds__(HID) k_backward(const float *__restrict__ P, const float *__restrict__ Z1,
                                                  const float *__restrict__ Z2, const float *__restrict__ Y,
                                                  const float *__restrict__ T, int64_t B, float *__restrict__ DY,
                                                  float *__restrict__ DZ1, float *__restrict__ DZ2) {
    __shared__ float sd[HID];
    const int64_t b = blockIdx.x;
    if (b >= B) return;
    const int j = threadIdx.x;
    const float dy = GIVEN ? DY[b] : 2.f * (Y[b] - T[b]) / (float)B;
    if (!GIVEN && j == 0) DY[b] = dy;
    const float d2 = Z2[b * HID + j] > 0.f ? dy * P[OFF_W3 + j] : 0.f;
    DZ2[b * HID + j] = d2;
    sd[j] = d2;
    __syncthreads();
    float a = 0.f;                                   // (W2^T dz2)_j
    for (int r = 0; r < HID; ++r) a += P[OFF_W2 + r * HID + j] * sd[r];
    DZ1[b * HID + j] = Z1[b * HID + j] > 0.f ? a : 0.f;
}

// Gradient of parameter p summed over the batch, in sample order.
__global__ void k_grad(const float *__restrict__ X, const float *__restrict__ Z1, const float *__restrict__ Z2,
                       const float *__restrict__ DY, const float *__restrict__ DZ1, const float *__restrict__ DZ2,
                       int64_t B, float *__restrict__ G) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    float g = 0.f;
    if (p < OFF_B1) {
        const int j = p / IN, i = p % IN;
        for (int64_t b = 0; b < B; ++b) g += DZ1[b * HID + j] * X[b * IN + i];
    } else if (p < OFF_W2) {
        const int j = p - OFF_B1;
        for (int64_t b = 0; b < B; ++b) g += DZ1[b * HID + j];
    } else if (p < OFF_B2) {
        const int j = (p - OFF_W2) / HID, k = (p - OFF_W2) % HID;
        for (int64_t b = 0; b < B; ++b) g += DZ2[b * HID + j] * fmaxf(Z1[b * HID + k], 0.f);
    } else if (p < OFF_W3) {
        const int j = p - OFF_B2;
        for (int64_t b = 0; b < B; ++b) g += DZ2[b * HID + j];
    } else if (p < OFF_B3) {
        const int j = p - OFF_W3;
        for (int64_t b = 0; b < B; ++b) g += DY[b] * fmaxf(Z2[b * HID + j], 0.f);
    } else {
        for (int64_t b = 0; b < B; ++b) g += DY[b];
    }
    G[p] = g;
}

// Mean squared error of the batch (one block).
__global__ void k_loss(const float *__restrict__ Y, const float *__restrict__ T, int64_t B, float *out) {
    __shared__ double s[256];
    double a = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
        const double d = (double)Y[b] - (double)T[b];
        a += d * d;
    }
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)(s[0] / (double)(B > 0 ? B : 1));
}

// Mixed objective per sample, one warp each: mix * (y - t)^2 + (1 - mix) *
// sum_i w_i L_i, with w_i ~ exp(-(i - 64 y)^2 / (2 sigma^2)) over the grid
// levels i = 1..64 (normalised) and L_i the ARI lost at level i.  Writes
// dloss/dy / B to DY and the sample's loss to SL.
__global__ void k_soft_dy(const float *__restrict__ Y, const float *__restrict__ T, const float *__restrict__ A,
                          int64_t B, float sigma, float mix, float *__restrict__ DY, float *__restrict__ SL) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= B) return;
    const int lane = (int)lane_id();
    const float p = 64.f * Y[b];
    const float inv = 1.f / (sigma * sigma);
    float d[2], a[2], L[2];
    for (int h = 0; h < 2; ++h) {
        const int i = 1 + lane + 32 * h;
        d[h] = (float)i - p;
        a[h] = -0.5f * d[h] * d[h] * inv;
        L[h] = A[b * 64 + i - 1];
    }
    float amax = fmaxf(a[0], a[1]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    float z = 0.f, wl = 0.f, wld = 0.f, wd = 0.f;
    for (int h = 0; h < 2; ++h) {
        const float w = expf(a[h] - amax);
        z += w;
        wl += w * L[h];
        wld += w * L[h] * d[h];
        wd += w * d[h];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        z += __shfl_xor_sync(0xffffffffu, z, o);
        wl += __shfl_xor_sync(0xffffffffu, wl, o);
        wld += __shfl_xor_sync(0xffffffffu, wld, o);
        wd += __shfl_xor_sync(0xffffffffu, wd, o);
    }
    if (lane == 0) {
        const float val = wl / z;
        const float dval = 64.f * inv * (wld / z - val * (wd / z));
        const float e = Y[b] - T[b];
        DY[b] = (mix * 2.f * e + (1.f - mix) * dval) / (float)B;
        SL[b] = mix * e * e + (1.f - mix) * val;
    }
}

// Mean of the per-sample losses SL (one block).
__global__ void k_mean(const float *__restrict__ SL, int64_t B, float *out) {
    __shared__ double s[256];
    double a = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) a += (double)SL[b];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)(s[0] / (double)(B > 0 ? B : 1));
}

__global__ void k_adam(float *P, float *M, float *V, const float *G, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float g = G[p];
    const float m = b1 * M[p] + (1.f - b1) * g;
    const float v = b2 * V[p] + (1.f - b2) * g * g;
    M[p] = m;
    V[p] = v;
    P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__device__ __forceinline__ uint64_t mix64d(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Keyed bijection of [0, 2^bits), walked until it lands in [0, N).
__device__ __forceinline__ int64_t shuffle_index(int64_t i, int64_t N, int bits, uint64_t key) {
    const int lo = bits / 2, hi = bits - lo;
    const uint64_t mlo = (1ull << lo) - 1ull, mhi = (1ull << hi) - 1ull;
    uint64_t x = (uint64_t)i;
    for (int walk = 0; walk < 64; ++walk) {
        uint64_t L = x >> lo, R = x & mlo;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if ((r & 1) == 0) L ^= mix64d(key + r ^ R) & mhi;
            else R ^= mix64d(key + r ^ L) & mlo;
        }
        x = (L << lo) | R;
        if ((int64_t)x < N) return (int64_t)x;
    }
    return i;   // not reached for N > 2^(bits-1)
}

__global__ void k_gather(const float *__restrict__ F, const float *__restrict__ T, int64_t N, int64_t first,
                         int64_t B, int bits, uint64_t key, float *__restrict__ X, float *__restrict__ TB) {
    const int64_t b = blockIdx.x;
    if (b >= B) return;
    const int64_t src = key ? shuffle_index(first + b, N, bits, key) : first + b;
    for (int i = threadIdx.x; i < IN; i += blockDim.x) X[b * IN + i] = F[src * IN + i];
    if (threadIdx.x == 0) TB[b] = T[src];
}

// The ARI-loss rows (64 each) of the same samples as k_gather.
__global__ void k_gather_rows(const float *__restrict__ L, int64_t N, int64_t first, int64_t B, int bits,
                              uint64_t key, float *__restrict__ AB) {
    const int64_t b = blockIdx.x;
    if (b >= B) return;
    const int64_t src = key ? shuffle_index(first + b, N, bits, key) : first + b;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) AB[b * 64 + i] = L[src * 64 + i];
}

// Grid threshold per graph: b = clamp(round(64 y), 1, 64), theta = b / 128.
__global__ void k_pick(const float *y, int64_t N, int64_t *p, int64_t *q) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const float v = y[s] * 64.f;
    int64_t b = isfinite(v) ? (int64_t)rintf(fminf(fmaxf(v, 1.f), 64.f)) : 1;
    p[s] = b;
    q[s] = 128;
}

}  // namespace
}  // namespace tec

using namespace tec;

extern "C" tec_status tec_picker_thresholds(const float *y, int64_t N, int64_t *p_out, int64_t *q_out, void *stream) {
    clear_error();
    if (N < 0 || (N > 0 && (!y || !p_out || !q_out))) return set_error(TEC_EINVAL, "bad argument");
    if (N == 0) return TEC_OK;
    k_pick<<<(unsigned)ceil_div(N, 256), 256, 0, (cudaStream_t)stream>>>(y, N, p_out, q_out);
    count_launches(1);
    TEC_CUDA(cudaGetLastError());
    return TEC_OK;
}

struct tec_picker {
    int device = 0;
    cudaStream_t stream = nullptr;
    float *P = nullptr, *M = nullptr, *V = nullptr, *G = nullptr;
    int64_t cap = 0;                     // batch capacity of the work buffers
    float *X = nullptr, *T = nullptr, *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr;
    float *DY = nullptr, *DZ1 = nullptr, *DZ2 = nullptr, *loss = nullptr;
    float *A = nullptr, *SL = nullptr;   // soft-level loss: ARI-loss rows (64 per sample), per-sample losses
    int64_t step = 0;
};

namespace {

void picker_free_work(tec_picker *p) {
    float *bufs[] = {p->X, p->T, p->Z1, p->Z2, p->Y, p->DY, p->DZ1, p->DZ2, p->A, p->SL};
    for (float *b : bufs)
        if (b) cudaFree(b);
    p->X = p->T = p->Z1 = p->Z2 = p->Y = p->DY = p->DZ1 = p->DZ2 = p->A = p->SL = nullptr;
    p->cap = 0;
}

tec_status picker_work(tec_picker *p, int64_t B) {
    if (p->cap >= B) return TEC_OK;
    picker_free_work(p);
    const int64_t c = B < 256 ? 256 : B;
    float **bufs[] = {&p->X, &p->T, &p->Z1, &p->Z2, &p->Y, &p->DY, &p->DZ1, &p->DZ2, &p->A, &p->SL};
    const int64_t sizes[] = {c * IN, c, c * HID, c * HID, c, c, c * HID, c * HID, c * 64, c};
    for (int i = 0; i < 10; ++i) {
        cudaError_t e = cudaMalloc((void **)bufs[i], (size_t)sizes[i] * sizeof(float));
        if (e != cudaSuccess) {
            cudaGetLastError();
            picker_free_work(p);
            return set_error(TEC_ENOMEM, "picker work buffers: %s", cudaGetErrorString(e));
        }
    }
    p->cap = c;
    return TEC_OK;
}

// Forward + backward + gradient of one batch already in p->X / p->T (and,
// for the soft-level loss (soft), p->A).
tec_status picker_batch_grad(tec_picker *p, int64_t B, bool soft = false, float sigma = 1.f, float mix = 1.f) {
    cudaStream_t s = p->stream;
    k_forward<false><<<(unsigned)B, HID, 0, s>>>(p->P, p->X, B, p->Z1, p->Z2, p->Y);
    if (soft) {
        k_soft_dy<<<(unsigned)ceil_div(B * 32, 256), 256, 0, s>>>(p->Y, p->T, p->A, B, sigma, mix, p->DY, p->SL);
        k_backward<true><<<(unsigned)B, HID, 0, s>>>(p->P, p->Z1, p->Z2, p->Y, p->T, B, p->DY, p->DZ1, p->DZ2);
    } else {
        k_backward<false><<<(unsigned)B, HID, 0, s>>>(p->P, p->Z1, p->Z2, p->Y, p->T, B, p->DY, p->DZ1, p->DZ2);
    }
    k_grad<<<(unsigned)ceil_div(NPARAM, 256), 256, 0, s>>>(p->X, p->Z1, p->Z2, p->DY, p->DZ1, p->DZ2, B, p->G);
    if (soft) k_mean<<<1, 256, 0, s>>>(p->SL, B, p->loss);
    else k_loss<<<1, 256, 0, s>>>(p->Y, p->T, B, p->loss);
    count_launches(soft ? 5 : 4);
    TEC_CUDA(cudaGetLastError());
    return TEC_OK;
}

tec_status picker_adam(tec_picker *p, float lr, float b1, float b2, float eps) {
    ++p->step;
    const float c1 = 1.f - powf(b1, (float)p->step), c2 = 1.f - powf(b2, (float)p->step);
    k_adam<<<(unsigned)ceil_div(NPARAM, 256), 256, 0, p->stream>>>(p->P, p->M, p->V, p->G, lr, b1, b2, eps, c1, c2);
    count_launches(1);
    TEC_CUDA(cudaGetLastError());
    return TEC_OK;
}

}  // namespace

extern "C" {

tec_status tec_picker_create(const float *init_params, void *stream, tec_picker **out) {
    clear_error();
    if (!out) return set_error(TEC_EINVAL, "out is NULL");
    *out = nullptr;
    tec_picker *p = new (std::nothrow) tec_picker();
    if (!p) return set_error(TEC_ENOMEM, "host allocation failed");
    p->stream = (cudaStream_t)stream;
    cudaGetDevice(&p->device);
    float **bufs[] = {&p->P, &p->M, &p->V, &p->G};
    for (float **b : bufs) {
        cudaError_t e = cudaMalloc((void **)b, NPARAM * sizeof(float));
        if (e == cudaSuccess) e = cudaMemsetAsync(*b, 0, NPARAM * sizeof(float), p->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            tec_picker_free(p);
            return set_error(TEC_ENOMEM, "picker parameters: %s", cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaMalloc((void **)&p->loss, sizeof(float));
    if (e == cudaSuccess && init_params)
        e = cudaMemcpyAsync(p->P, init_params, NPARAM * sizeof(float), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        tec_picker_free(p);
        return set_error(TEC_ECUDA, "picker initialisation: %s", cudaGetErrorString(e));
    }
    *out = p;
    return TEC_OK;
}

tec_status tec_picker_free(tec_picker *p) {
    clear_error();
    if (!p) return TEC_OK;
    cudaStreamSynchronize(p->stream);
    picker_free_work(p);
    float *bufs[] = {p->P, p->M, p->V, p->G, p->loss};
    for (float *b : bufs)
        if (b) cudaFree(b);
    delete p;
    return TEC_OK;
}

tec_status tec_picker_get_params(tec_picker *p, float *params_out, float *adam_m_out, float *adam_v_out,
                                 int64_t *step_out) {
    clear_error();
    if (!p || !params_out) return set_error(TEC_EINVAL, "NULL argument");
    TEC_CUDA(cudaMemcpyAsync(params_out, p->P, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, p->stream));
    if (adam_m_out) TEC_CUDA(cudaMemcpyAsync(adam_m_out, p->M, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, p->stream));
    if (adam_v_out) TEC_CUDA(cudaMemcpyAsync(adam_v_out, p->V, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, p->stream));
    TEC_CUDA(cudaStreamSynchronize(p->stream));
    if (step_out) *step_out = p->step;
    return TEC_OK;
}

tec_status tec_picker_set_params(tec_picker *p, const float *params, const float *adam_m, const float *adam_v,
                                 int64_t step) {
    clear_error();
    if (!p || !params) return set_error(TEC_EINVAL, "NULL argument");
    TEC_CUDA(cudaMemcpyAsync(p->P, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    if (adam_m) TEC_CUDA(cudaMemcpyAsync(p->M, adam_m, NPARAM * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    else TEC_CUDA(cudaMemsetAsync(p->M, 0, NPARAM * sizeof(float), p->stream));
    if (adam_v) TEC_CUDA(cudaMemcpyAsync(p->V, adam_v, NPARAM * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    else TEC_CUDA(cudaMemsetAsync(p->V, 0, NPARAM * sizeof(float), p->stream));
    TEC_CUDA(cudaStreamSynchronize(p->stream));
    p->step = step;
    return TEC_OK;
}

tec_status tec_picker_forward(tec_picker *p, const float *feats, int64_t N, int bf16, float *out) {
    clear_error();
    if (!p || (N > 0 && (!feats || !out))) return set_error(TEC_EINVAL, "NULL argument");
    if (N <= 0) return TEC_OK;
    if (N > 2147483647) return set_error(TEC_EINVAL, "too many samples");
    if (bf16) k_forward<true><<<(unsigned)N, HID, 0, p->stream>>>(p->P, feats, N, nullptr, nullptr, out);
    else k_forward<false><<<(unsigned)N, HID, 0, p->stream>>>(p->P, feats, N, nullptr, nullptr, out);
    count_launches(1);
    TEC_CUDA(cudaGetLastError());
    return TEC_OK;
}

// Orders stream `after` behind the work queued so far on stream `before`.
static tec_status stream_after(cudaStream_t before, cudaStream_t after) {
    if (before == after) return TEC_OK;
    cudaEvent_t ev;
    TEC_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, before);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(after, ev, 0);
    cudaEventDestroy(ev);
    TEC_CUDA(e);
    return TEC_OK;
}

tec_status tec_pick_threshold(tec_graph *g, tec_picker *p, const int64_t *seg_off, int nseg, int bf16,
                              int64_t *p_out, int64_t *q_out) {
    clear_error();
    if (!g || !p || !p_out || !q_out) return set_error(TEC_EINVAL, "NULL argument");
    if (seg_off && nseg < 1) return set_error(TEC_EINVAL, "nseg must be >= 1 with a segment table");
    const int64_t ns = seg_off ? nseg : 1;
    TEC_TRY(picker_work(p, ns));
    TEC_TRY(stream_after(p->stream, g->stream));    // parameters and work buffers settled
    TEC_TRY(tec_features(g, seg_off, nseg, p->X));
    clear_error();
    if (bf16) k_forward<true><<<(unsigned)ns, HID, 0, g->stream>>>(p->P, p->X, ns, nullptr, nullptr, p->Y);
    else k_forward<false><<<(unsigned)ns, HID, 0, g->stream>>>(p->P, p->X, ns, nullptr, nullptr, p->Y);
    k_pick<<<(unsigned)ceil_div(ns, 256), 256, 0, g->stream>>>(p->Y, ns, p_out, q_out);
    count_launches(2);
    TEC_CUDA(cudaGetLastError());
    TEC_TRY(stream_after(g->stream, p->stream));    // the picker's next use waits for its buffers
    return TEC_OK;
}

tec_status tec_picker_loss_grad(tec_picker *p, const float *feats, const float *target, int64_t N, float *loss_out,
                                float *grad_out) {
    clear_error();
    if (!p || N <= 0 || !feats || !target) return set_error(TEC_EINVAL, "bad argument");
    if (N > 2147483647) return set_error(TEC_EINVAL, "too many samples");
    TEC_TRY(picker_work(p, N));
    TEC_CUDA(cudaMemcpyAsync(p->X, feats, (size_t)N * IN * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    TEC_CUDA(cudaMemcpyAsync(p->T, target, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    TEC_TRY(picker_batch_grad(p, N));
    if (grad_out)
        TEC_CUDA(cudaMemcpyAsync(grad_out, p->G, NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    if (loss_out) {
        TEC_CUDA(cudaMemcpyAsync(loss_out, p->loss, sizeof(float), cudaMemcpyDeviceToHost, p->stream));
        TEC_CUDA(cudaStreamSynchronize(p->stream));
    }
    return TEC_OK;
}

tec_status tec_picker_adam_step(tec_picker *p, const float *grad, float lr, float beta1, float beta2, float eps) {
    clear_error();
    if (!p) return set_error(TEC_EINVAL, "picker is NULL");
    if (grad) TEC_CUDA(cudaMemcpyAsync(p->G, grad, NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    return picker_adam(p, lr, beta1, beta2, eps);
}

static tec_status train_impl(tec_picker *p, const float *feats, const float *target, const float *ari_loss,
                             int64_t N, int epochs, int batch, float lr, uint64_t seed, bool soft, float sigma,
                             float mix, float *loss_out) {
    TEC_TRY(picker_work(p, batch));
    int bits = 1;
    while (((int64_t)1 << bits) < N) ++bits;
    std::vector<float> ep_loss(epochs > 0 ? epochs : 1, 0.f);
    for (int e = 0; e < epochs; ++e) {
        uint64_t key = seed * 0x9E3779B97F4A7C15ull + (uint64_t)(e + 1) * 0xD1B54A32D192ED03ull;
        if (!key) key = 1;
        double acc = 0.0;
        for (int64_t first = 0; first < N; first += batch) {
            const int64_t B = N - first < batch ? N - first : batch;
            k_gather<<<(unsigned)B, 128, 0, p->stream>>>(feats, target, N, first, B, bits, key, p->X, p->T);
            if (soft) k_gather_rows<<<(unsigned)B, 64, 0, p->stream>>>(ari_loss, N, first, B, bits, key, p->A);
            count_launches(soft ? 2 : 1);
            TEC_TRY(picker_batch_grad(p, B, soft, sigma, mix));
            TEC_TRY(picker_adam(p, lr, 0.9f, 0.999f, 1e-8f));
            if (loss_out) {
                float l = 0.f;
                TEC_CUDA(cudaMemcpyAsync(&l, p->loss, sizeof(float), cudaMemcpyDeviceToHost, p->stream));
                TEC_CUDA(cudaStreamSynchronize(p->stream));
                acc += (double)l * (double)B;
            }
        }
        ep_loss[e] = (float)(acc / (double)N);
    }
    if (loss_out)
        for (int e = 0; e < epochs; ++e) loss_out[e] = ep_loss[e];
    TEC_CUDA(cudaStreamSynchronize(p->stream));
    return TEC_OK;
}

tec_status tec_picker_train(tec_picker *p, const float *feats, const float *target, int64_t N, int epochs, int batch,
                            float lr, uint64_t seed, float *loss_out) {
    clear_error();
    if (!p || N <= 0 || !feats || !target || epochs < 0 || batch < 1) return set_error(TEC_EINVAL, "bad argument");
    return train_impl(p, feats, target, nullptr, N, epochs, batch, lr, seed, false, 1.f, 1.f, loss_out);
}

static tec_status check_soft(float sigma, float mix) {
    if (!(sigma >= 0.05f && sigma <= 64.f)) return set_error(TEC_EINVAL, "sigma must lie in [0.05, 64]");
    if (!(mix >= 0.f && mix <= 1.f)) return set_error(TEC_EINVAL, "mix must lie in [0, 1]");
    return TEC_OK;
}

tec_status tec_picker_soft_loss_grad(tec_picker *p, const float *feats, const float *target, const float *ari_loss,
                                     int64_t N, float sigma, float mix, float *loss_out, float *grad_out) {
    clear_error();
    if (!p || N <= 0 || !feats || !target || !ari_loss) return set_error(TEC_EINVAL, "bad argument");
    if (N > 2147483647) return set_error(TEC_EINVAL, "too many samples");
    TEC_TRY(check_soft(sigma, mix));
    TEC_TRY(picker_work(p, N));
    TEC_CUDA(cudaMemcpyAsync(p->X, feats, (size_t)N * IN * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    TEC_CUDA(cudaMemcpyAsync(p->T, target, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    TEC_CUDA(cudaMemcpyAsync(p->A, ari_loss, (size_t)N * 64 * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    TEC_TRY(picker_batch_grad(p, N, true, sigma, mix));
    if (grad_out)
        TEC_CUDA(cudaMemcpyAsync(grad_out, p->G, NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    if (loss_out) {
        TEC_CUDA(cudaMemcpyAsync(loss_out, p->loss, sizeof(float), cudaMemcpyDeviceToHost, p->stream));
        TEC_CUDA(cudaStreamSynchronize(p->stream));
    }
    return TEC_OK;
}

tec_status tec_picker_train_soft(tec_picker *p, const float *feats, const float *target, const float *ari_loss,
                                 int64_t N, int epochs, int batch, float lr, uint64_t seed, float sigma, float mix,
                                 float *loss_out) {
    clear_error();
    if (!p || N <= 0 || !feats || !target || !ari_loss || epochs < 0 || batch < 1)
        return set_error(TEC_EINVAL, "bad argument");
    TEC_TRY(check_soft(sigma, mix));
    return train_impl(p, feats, target, ari_loss, N, epochs, batch, lr, seed, true, sigma, mix, loss_out);
}

}  // extern "C"
