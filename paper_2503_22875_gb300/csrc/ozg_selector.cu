// Learned slice selector: the adaptive split number the paper proposes as future work
// (Sec. 4: dynamically adjusting the split number to the accuracy a region needs, since cost
// grows quadratically with the split number).
//
// Features (24, per GEMM): log2 m, log2 n, log2 k; for op(A) a 10-bin histogram (as fractions)
// of the within-row exponent gap e_i - E(a_il) (bins [0,4), [4,8), ..., [32,36), and [36, inf)
// together with zeros); the same for the columns of op(B); log10 of the requested error.
// Model: MLP 24 -> 64 -> 64 -> 11 (ReLU), BF16 weights, FP32 accumulation, classes s = 2..12.
// Decision: the smallest s whose cumulative predicted probability of "the minimal sufficient
// slice count is <= s" reaches the model's threshold.
//
// Kernels: the gap histogram (one extra read of each operand, after the split computed the row
// exponents), the inference (one warp per GEMM; its result is written to device memory where
// the slice GEMM reads it -- no host round trip), and the training step (forward, backward and
// Adam update for a batch, FP32 master weights, BF16-rounded weights in the forward pass).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "ozg_context.h"
#include "ozg_split_dev.cuh"

namespace ozg {
namespace {

__device__ __forceinline__ int exp_of_bits(uint64_t b) {  // frexp exponent of |x| != 0
  const int eb = (int)((b >> 52) & 0x7FF);
  if (eb) return eb - 1022;
  const uint64_t mant = b & 0xFFFFFFFFFFFFFull;
  return (64 - __clzll((long long)mant)) - 1074;
}

// one 32 x 64 tile of a split job: histogram of e_row - E(x) into 10 bins
__device__ void hist_tile(const SplitArgs& J, int64_t u, unsigned int* sh) {
  const int64_t ltiles = (J.k + 63) / 64;
  const int64_t r0 = (u / ltiles) * 32, l0 = (u % ltiles) * 64;
  for (int q = 0; q < 8; ++q) {
    const int idx = q * 256 + threadIdx.x;
    int64_t row, l;
    if (J.strided) {
      row = r0 + idx % 32;
      l = l0 + idx / 32;
    } else {
      row = r0 + idx / 64;
      l = l0 + idx % 64;
    }
    if (row >= J.rows || l >= J.k) continue;
    uint64_t b;
    if (!J.cplx) {
      const uint64_t* p = reinterpret_cast<const uint64_t*>(J.X);
      b = __ldg(J.strided ? p + row + l * J.ld : p + l + row * J.ld) & 0x7FFFFFFFFFFFFFFFull;
    } else {
      const ulonglong2* p = reinterpret_cast<const ulonglong2*>(J.X);
      const ulonglong2 v = __ldg(J.strided ? p + row + l * J.ld : p + l + row * J.ld);
      const uint64_t x = v.x & 0x7FFFFFFFFFFFFFFFull, y = v.y & 0x7FFFFFFFFFFFFFFFull;
      b = x > y ? x : y;
    }
    int bin = 9;
    if (b != 0) {
      const int gap = exponent_from_maxbits(J.maxbits[row]) - exp_of_bits(b);  // e_i from the row maximum
      bin = gap < 36 ? (gap < 0 ? 0 : gap / 4) : 9;
    }
    atomicAdd(&sh[bin], 1u);
  }
}

__global__ void __launch_bounds__(256) gap_hist_pair(SplitArgs a, SplitArgs b, int64_t units_a) {
  __shared__ unsigned int sh[10];
  if (threadIdx.x < 10) sh[threadIdx.x] = 0;
  __syncthreads();
  const bool first = (int64_t)blockIdx.x < units_a;
  const SplitArgs& J = first ? a : b;
  hist_tile(J, first ? blockIdx.x : blockIdx.x - units_a, sh);
  __syncthreads();
  if (threadIdx.x < 10 && sh[threadIdx.x]) atomicAdd(&J.hist[threadIdx.x], (unsigned long long)sh[threadIdx.x]);
}


// Batched features over the row-maximum units (32 rows x kRmStridedK k of a strided job, each
// thread one row and 16 of its elements; 8 rows x kRmContigK k of a contiguous job, each warp
// one row and each thread 32 of its elements), so every thread reads its row's exponent once.
// Each thread bins its elements into ten 6-bit counters packed in one 64-bit word (at most 32
// elements), the warp sums them with integer reductions, and one shared-memory add per bin and
// warp precedes one global add per bin and CTA.
__device__ __forceinline__ int gap_bin(uint64_t b, int e_row) {
  if (b == 0) return 9;
  const int gap = e_row - exp_of_bits(b);
  return gap < 36 ? (gap < 0 ? 0 : gap / 4) : 9;
}
__device__ __forceinline__ uint64_t abs_bits(const SplitArgs& J, int64_t row, int64_t l) {
  if (!J.cplx) {
    const uint64_t* X = reinterpret_cast<const uint64_t*>(J.X);
    return __ldg(J.strided ? X + row + l * J.ld : X + l + row * J.ld) & kAbsMask;
  }
  const ulonglong2* X = reinterpret_cast<const ulonglong2*>(J.X);
  const ulonglong2 v = __ldg(J.strided ? X + row + l * J.ld : X + l + row * J.ld);
  const uint64_t x = v.x & kAbsMask, y = v.y & kAbsMask;
  return x > y ? x : y;
}
__global__ void __launch_bounds__(256) gap_hist_batched(const SplitArgs* jobs, const int2* units) {
  __shared__ unsigned int sh[10];
  if (threadIdx.x < 10) sh[threadIdx.x] = 0;
  __syncthreads();
  const int2 ur = units[blockIdx.x];
  const SplitArgs J = jobs[ur.x];
  if (J.hist != nullptr) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long packed = 0;
    if (J.strided) {
      const int64_t kt = (J.k + kRmStridedK - 1) / kRmStridedK;
      const int64_t row = (ur.y / kt) * 32 + lane, l0 = (ur.y % kt) * kRmStridedK + w;
      if (row < J.rows) {
        const int e_row = exponent_from_maxbits(J.maxbits[row]);
#pragma unroll
        for (int i = 0; i < kRmStridedK / 8; ++i) {
          const int64_t l = l0 + 8 * i;
          if (l < J.k) packed += 1ull << (6 * gap_bin(abs_bits(J, row, l), e_row));
        }
      }
    } else {
      const int64_t kt = (J.k + kRmContigK - 1) / kRmContigK;
      const int64_t row = (ur.y / kt) * 8 + w, l0 = (ur.y % kt) * kRmContigK + lane;
      if (row < J.rows) {
        const int e_row = exponent_from_maxbits(J.maxbits[row]);
#pragma unroll 8
        for (int i = 0; i < kRmContigK / 32; ++i) {
          const int64_t l = l0 + 32 * i;
          if (l < J.k) packed += 1ull << (6 * gap_bin(abs_bits(J, row, l), e_row));
        }
      }
    }
    static_assert(kRmStridedK / 8 <= 63 && kRmContigK / 32 <= 63, "6-bit counters");
#pragma unroll
    for (int bin = 0; bin < 10; ++bin) {
      const unsigned v = __reduce_add_sync(0xffffffffu, (unsigned)((packed >> (6 * bin)) & 63ull));
      if (lane == 0 && v) atomicAdd(&sh[bin], v);
    }
  }
  __syncthreads();
  if (J.hist != nullptr && threadIdx.x < 10 && sh[threadIdx.x])
    atomicAdd(&J.hist[threadIdx.x], (unsigned long long)sh[threadIdx.x]);
}

// ---------------------------------------------------------------------------- inference
__device__ __forceinline__ float bf(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// One warp: features -> MLP -> decision.  feat_out / prob_out (optional) receive the raw
// features and the class probabilities.
__device__ void select_warp(const SelectorDev* M, const unsigned long long* hA, const unsigned long long* hB,
                            int64_t m, int64_t n, int64_t k, float log10_target, int s_cap, int* s_out1,
                            int* s_out2, float* feat_out, float* prob_out) {
  const int lane = threadIdx.x & 31;
  float f = 0.f;
  if (lane < 3) {
    const int64_t d = lane == 0 ? m : (lane == 1 ? n : k);
    f = log2f((float)d);
  } else if (lane < 13) {
    f = (float)((double)hA[lane - 3] / ((double)m * (double)k));
  } else if (lane < 23) {
    f = (float)((double)hB[lane - 13] / ((double)n * (double)k));
  } else if (lane == 23) {
    f = log10_target;
  }
  if (feat_out != nullptr && lane < kSelIn) feat_out[lane] = f;
  if (M == nullptr) return;  // features only
  const float x = lane < kSelIn ? (f - M->mean[lane]) * M->inv_std[lane] : 0.f;
  // layer 1: lane owns hidden units lane and lane + 32
  float h1a = M->b1[lane], h1b = M->b1[lane + 32];
  for (int j = 0; j < kSelIn; ++j) {
    const float xj = __shfl_sync(0xffffffffu, x, j);
    h1a = fmaf(bf(M->W1[lane * kSelIn + j]), xj, h1a);
    h1b = fmaf(bf(M->W1[(lane + 32) * kSelIn + j]), xj, h1b);
  }
  h1a = fmaxf(h1a, 0.f);
  h1b = fmaxf(h1b, 0.f);
  float h2a = M->b2[lane], h2b = M->b2[lane + 32];
  for (int j = 0; j < kSelH; ++j) {
    const float hj = __shfl_sync(0xffffffffu, j < 32 ? h1a : h1b, j & 31);
    h2a = fmaf(bf(M->W2[lane * kSelH + j]), hj, h2a);
    h2b = fmaf(bf(M->W2[(lane + 32) * kSelH + j]), hj, h2b);
  }
  h2a = fmaxf(h2a, 0.f);
  h2b = fmaxf(h2b, 0.f);
  float z = lane < kSelOut ? M->b3[lane] : -INFINITY;
  for (int j = 0; j < kSelH; ++j) {
    const float hj = __shfl_sync(0xffffffffu, j < 32 ? h2a : h2b, j & 31);
    if (lane < kSelOut) z = fmaf(bf(M->W3[lane * kSelH + j]), hj, z);
  }
  // softmax over the 11 classes, then the cumulative rule (lane 0, classes in order)
  float zmax = z;
  for (int o = 16; o > 0; o >>= 1) zmax = fmaxf(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
  const float ez = lane < kSelOut ? expf(z - zmax) : 0.f;
  float sum = ez;
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  const float p = ez / sum;
  if (prob_out != nullptr && lane < kSelOut) prob_out[lane] = p;
  float cum = 0.f;
  int chosen = -1;
  for (int c = 0; c < kSelOut; ++c) {
    cum += __shfl_sync(0xffffffffu, p, c);
    if (chosen < 0 && cum >= M->threshold) chosen = c;
  }
  int s = chosen < 0 ? M->fallback : M->s_lo + chosen;
  if (s < 1) s = 1;
  if (s > s_cap) s = s_cap;
  if (lane == 0) {
    if (s_out1) *s_out1 = s;
    if (s_out2) *s_out2 = s;
  }
}

__global__ void select_single(const SelectorDev* M, const unsigned long long* hA, const unsigned long long* hB,
                              int64_t m, int64_t n, int64_t k, float log10_target, int s_cap, int* s_out,
                              float* feat_out, float* prob_out) {
  select_warp(M, hA, hB, m, n, k, log10_target, s_cap, s_out, nullptr, feat_out, prob_out);
}

__global__ void select_batched(const SelectorDev* M, const SelectJob* jobs, int njobs, float log10_target) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= njobs) return;
  const SelectJob J = jobs[w];
  if (!J.active) return;
  select_warp(M, J.histA, J.histB, J.m, J.n, J.k, log10_target, J.s_cap, J.s_out1, J.s_out2, nullptr, nullptr);
}

// ---------------------------------------------------------------------------- training
// theta = [W1 (64x24), b1 (64), W2 (64x64), b2 (64), W3 (11x64), b3 (11)], FP32 master weights.
// The forward pass uses the weights rounded to BF16 (as inference does); the gradient passes
// straight through the rounding.  Loss: mean cross-entropy over the batch.
constexpr int oW1 = 0, oB1 = oW1 + kSelH * kSelIn, oW2 = oB1 + kSelH, oB2 = oW2 + kSelH * kSelH,
              oW3 = oB2 + kSelH, oB3 = oW3 + kSelOut * kSelH;
constexpr int kSamplesPerBlock = 16;

__device__ __forceinline__ float rbf(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

__global__ void __launch_bounds__(64) mlp_grads_kernel(const float* __restrict__ theta, const float* __restrict__ X,
                                                       const int* __restrict__ y, int B, float* __restrict__ grad,
                                                       float* __restrict__ loss) {
  __shared__ float g[kSelParams];
  __shared__ float x[kSelIn], h1[kSelH], h2[kSelH], z[kSelOut], dz[kSelOut], dh2[kSelH];
  __shared__ float lsum;
  const int t = threadIdx.x;
  for (int i = t; i < kSelParams; i += 64) g[i] = 0.f;
  if (t == 0) lsum = 0.f;
  __syncthreads();
  const int b0 = blockIdx.x * kSamplesPerBlock;
  for (int sidx = b0; sidx < min(B, b0 + kSamplesPerBlock); ++sidx) {
    if (t < kSelIn) x[t] = X[(size_t)sidx * kSelIn + t];
    __syncthreads();
    float a1 = theta[oB1 + t];
    for (int j = 0; j < kSelIn; ++j) a1 = fmaf(rbf(theta[oW1 + t * kSelIn + j]), x[j], a1);
    h1[t] = fmaxf(a1, 0.f);
    __syncthreads();
    float a2 = theta[oB2 + t];
    for (int j = 0; j < kSelH; ++j) a2 = fmaf(rbf(theta[oW2 + t * kSelH + j]), h1[j], a2);
    h2[t] = fmaxf(a2, 0.f);
    __syncthreads();
    if (t < kSelOut) {
      float a3 = theta[oB3 + t];
      for (int j = 0; j < kSelH; ++j) a3 = fmaf(rbf(theta[oW3 + t * kSelH + j]), h2[j], a3);
      z[t] = a3;
    }
    __syncthreads();
    if (t == 0) {
      float zm = z[0];
      for (int o = 1; o < kSelOut; ++o) zm = fmaxf(zm, z[o]);
      float se = 0.f;
      for (int o = 0; o < kSelOut; ++o) se += expf(z[o] - zm);
      const int lab = y[sidx];
      for (int o = 0; o < kSelOut; ++o) dz[o] = (expf(z[o] - zm) / se - (o == lab ? 1.f : 0.f)) / (float)B;
      lsum += (logf(se) + zm - z[lab]) / (float)B;
    }
    __syncthreads();
    // W3 / b3: thread t owns column t of W3
    for (int o = 0; o < kSelOut; ++o) g[oW3 + o * kSelH + t] += dz[o] * h2[t];
    if (t < kSelOut) g[oB3 + t] += dz[t];
    float d2 = 0.f;
    if (h2[t] > 0.f)
      for (int o = 0; o < kSelOut; ++o) d2 = fmaf(rbf(theta[oW3 + o * kSelH + t]), dz[o], d2);
    dh2[t] = d2;
    __syncthreads();
    // W2 / b2: thread t owns row t
    for (int j = 0; j < kSelH; ++j) g[oW2 + t * kSelH + j] += dh2[t] * h1[j];
    g[oB2 + t] += dh2[t];
    float d1 = 0.f;
    if (h1[t] > 0.f)
      for (int o = 0; o < kSelH; ++o) d1 = fmaf(rbf(theta[oW2 + o * kSelH + t]), dh2[o], d1);
    // W1 / b1: thread t owns row t
    for (int j = 0; j < kSelIn; ++j) g[oW1 + t * kSelIn + j] += d1 * x[j];
    g[oB1 + t] += d1;
    __syncthreads();
  }
  for (int i = t; i < kSelParams; i += 64)
    if (g[i] != 0.f) atomicAdd(&grad[i], g[i]);
  if (t == 0 && loss != nullptr) atomicAdd(loss, lsum);
}

__global__ void adam_kernel(float* theta, const float* grad, float* m1, float* m2, float lr, float b1, float b2,
                            float eps, float c1, float c2, float scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kSelParams) return;
  const float gi = grad[i] * scale;
  m1[i] = b1 * m1[i] + (1.f - b1) * gi;
  m2[i] = b2 * m2[i] + (1.f - b2) * gi * gi;
  theta[i] -= lr * (m1[i] / c1) / (sqrtf(m2[i] / c2) + eps);
}

__global__ void repair_prep_kernel(const double* err, double target, int* not_repaired, const double* saved,
                                   double* C, int64_t m, int64_t n, int64_t ldc, int w, int restore) {
  const double e = *err;
  const bool bad = !(e <= target);  // NaN counts as a failed check
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx == 0) *not_repaired = bad ? 0 : 1;
  if (!bad || !restore) return;
  if (idx >= m * n * w) return;
  const int64_t part = idx % w, ij = idx / w, i = ij % m, j = ij / m;
  C[(i + j * ldc) * w + part] = saved[(i + j * m) * w + part];
}

}  // namespace

cudaError_t launch_repair_prep(const double* err, double target, int* not_repaired, const double* saved, double* C,
                               int64_t m, int64_t n, int64_t ldc, int w, int restore, cudaStream_t st) {
  const int64_t total = restore ? m * n * w : 1;
  { repair_prep_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(err, target, not_repaired, saved, C, m, n, ldc, w,
                                                                     restore); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_mlp_grads(const float* theta, const float* X, const int* y, int B, float* grad, float* loss,
                             cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * kSelParams, st);
  if (e == cudaSuccess && loss) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return e;
  { mlp_grads_kernel<<<(B + kSamplesPerBlock - 1) / kSamplesPerBlock, 64, 0, st>>>(theta, X, y, B, grad, loss); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, const float* grad, float* m1, float* m2, int step, float lr, float b1, float b2,
                        float eps, float scale, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  { adam_kernel<<<(kSelParams + 255) / 256, 256, 0, st>>>(theta, grad, m1, m2, lr, b1, b2, eps, c1, c2, scale); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_gap_hist_pair(const SplitArgs& a, const SplitArgs& b, cudaStream_t st) {
  const int64_t ua = ((a.rows + 31) / 32) * ((a.k + 63) / 64), ub = ((b.rows + 31) / 32) * ((b.k + 63) / 64);
  if (ua + ub <= 0) return cudaSuccess;
  { gap_hist_pair<<<(unsigned)(ua + ub), 256, 0, st>>>(a, b, ua); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_gap_hist_batched(const SplitArgs* jobs_dev, const int2* rowmax_units_dev, int64_t units,
                                    cudaStream_t st) {
  if (units <= 0) return cudaSuccess;
  { gap_hist_batched<<<(unsigned)units, 256, 0, st>>>(jobs_dev, rowmax_units_dev); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_select_single(const SelectorDev* M, const unsigned long long* hA, const unsigned long long* hB,
                                 int64_t m, int64_t n, int64_t k, float log10_target, int s_cap, int* s_out,
                                 float* feat_out, float* prob_out, cudaStream_t st) {
  { select_single<<<1, 32, 0, st>>>(M, hA, hB, m, n, k, log10_target, s_cap, s_out, feat_out, prob_out); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_select_batched(const SelectorDev* M, const SelectJob* jobs_dev, int njobs, float log10_target,
                                  cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  { select_batched<<<(njobs + 3) / 4, 128, 0, st>>>(M, jobs_dev, njobs, log10_target); note_launch(); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- model file
// Little-endian: "OZGSEL01", int32 {version = 1, in = 24, h = 64, out = 11, s_lo, fallback},
// float threshold, float mean[24], float std[24], u16 W1[64x24], float b1[64], u16 W2[64x64],
// float b2[64], u16 W3[11x64], float b3[11] (weights row-major [out][in], BF16 bit patterns).
int read_selector_file(const char* path, SelectorDev* out) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return OZG_ERR_INVALID;
  char magic[8];
  int32_t hdr[6];
  float thr;
  float stdv[kSelIn];
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "OZGSEL01", 8) == 0 &&
            std::fread(hdr, 4, 6, f) == 6 && hdr[0] == 1 && hdr[1] == kSelIn && hdr[2] == kSelH &&
            hdr[3] == kSelOut && std::fread(&thr, 4, 1, f) == 1 && std::fread(out->mean, 4, kSelIn, f) == kSelIn &&
            std::fread(stdv, 4, kSelIn, f) == kSelIn &&
            std::fread(out->W1, 2, kSelH * kSelIn, f) == (size_t)kSelH * kSelIn &&
            std::fread(out->b1, 4, kSelH, f) == kSelH &&
            std::fread(out->W2, 2, kSelH * kSelH, f) == (size_t)kSelH * kSelH &&
            std::fread(out->b2, 4, kSelH, f) == kSelH &&
            std::fread(out->W3, 2, kSelOut * kSelH, f) == (size_t)kSelOut * kSelH &&
            std::fread(out->b3, 4, kSelOut, f) == kSelOut;
  std::fclose(f);
  if (!ok) return OZG_ERR_INVALID;
  out->s_lo = hdr[4];
  out->fallback = hdr[5];
  out->threshold = thr;
  for (int i = 0; i < kSelIn; ++i) out->inv_std[i] = stdv[i] > 0.f ? 1.f / stdv[i] : 0.f;
  if (out->s_lo < 1 || out->s_lo + kSelOut - 1 > OZG_MAX_SLICES || out->fallback < 1 ||
      out->fallback > OZG_MAX_SLICES || !(thr > 0.f && thr <= 1.f))
    return OZG_ERR_INVALID;
  return OZG_OK;
}

}  // namespace ozg

// ---------------------------------------------------------------------------- C ABI
using namespace ozg::host;

extern "C" int ozg_load_selector(ozg_ctx* c, const char* path) {
  if (!c || !path) return OZG_ERR_INVALID;
  ozg::SelectorDev h;
  std::memset(&h, 0, sizeof(h));
  int rc = ozg::read_selector_file(path, &h);
  if (rc) return rc;
  cudaSetDevice(c->device);
  if (!c->dsel) {
    if (cudaMalloc(&c->dsel, sizeof(ozg::SelectorDev)) != cudaSuccess) {
      cudaGetLastError();
      c->dsel = nullptr;
      return OZG_ERR_ALLOC;
    }
  }
  OZG_CUDA(cudaStreamSynchronize(c->stream));
  OZG_CUDA(cudaMemcpy(c->dsel, &h, sizeof(h), cudaMemcpyHostToDevice));
  c->sel_s_hi = h.s_lo + ozg::kSelOut - 1;
  c->fallback_slices = h.fallback;  // the model's conservative count (ozg_set_fallback_slices overrides)
  c->plan.reset();  // a captured grouped plan embeds the previous selector state
  return OZG_OK;
}

extern "C" int ozg_set_target_error(ozg_ctx* c, double target) {
  if (!c) return OZG_ERR_INVALID;
  if (!(target > 0.0) || !std::isfinite(target)) return -2;
  c->target = target;
  c->plan.reset();
  return OZG_OK;
}

extern "C" int ozg_selector_features(ozg_ctx* c, char transa, char transb, int64_t m, int64_t n, int64_t k,
                                     const double* A, int64_t lda, const double* B, int64_t ldb, float* feat_out,
                                     float* prob_out, int* s_out) {
  if (!c || !feat_out) return OZG_ERR_INVALID;
  char ta = norm_trans(transa), tb = norm_trans(transb);
  if (ta == 'C') ta = 'T';
  if (tb == 'C') tb = 'T';
  if (ta != 'N' && ta != 'T') return -2;
  if (tb != 'N' && tb != 'T') return -3;
  if (m <= 0) return -4;
  if (n <= 0) return -5;
  if (k <= 0) return -6;
  if (lda < ((ta == 'N') ? m : k)) return -9;
  if (ldb < ((tb == 'N') ? k : n)) return -11;
  cudaSetDevice(c->device);
  const int64_t Kp = (k + 7) / 8 * 8;
  Carve cv;
  const size_t oDA = cv.take((size_t)m * Kp * 2), oDB = cv.take((size_t)n * Kp * 2);
  const size_t oMA = cv.take(8 * (size_t)m), oMB = cv.take(8 * (size_t)n), oE = cv.take(4 * (size_t)m),
               oF = cv.take(4 * (size_t)n), oH = cv.take(2 * 10 * 8);
  int rc = ensure_ws(c, cv.off);
  if (rc) return rc;
  cudaStream_t st = c->stream;
  ozg::SplitArgs sa;
  sa.X = A;
  sa.ld = lda;
  sa.rows = m;
  sa.k = k;
  sa.strided = (ta == 'N');
  sa.s = 1;
  sa.Kp = Kp;
  sa.plane_rows = m;
  sa.D = at<__half>(c, oDA);
  sa.maxbits = at<unsigned long long>(c, oMA);
  sa.exps = at<int32_t>(c, oE);
  sa.nonfinite = c->dflags + 2;
  ozg::SplitArgs sb = sa;
  sb.X = B;
  sb.ld = ldb;
  sb.rows = n;
  sb.strided = (tb == 'T');
  sb.plane_rows = n;
  sb.D = at<__half>(c, oDB);
  sb.maxbits = at<unsigned long long>(c, oMB);
  sb.exps = at<int32_t>(c, oF);
  unsigned long long* hist = at<unsigned long long>(c, oH);
  OZG_CUDA(cudaMemsetAsync(hist, 0, 2 * 10 * 8, st));
  if (ozg::stats_fused(sa) && ozg::stats_fused(sb)) {  // row maxima and features in one read
    sa.hist = hist;
    sb.hist = hist + 10;
    OZG_CUDA(ozg::launch_stats_pair(sa, sb, st));
  } else {
    OZG_CUDA(ozg::launch_rowmax(sa, st));
    OZG_CUDA(ozg::launch_rowmax(sb, st));
    sa.hist = hist;
    sb.hist = hist + 10;
    OZG_CUDA(ozg::launch_gap_hist_pair(sa, sb, st));
  }
  const bool model = c->sel_s_hi > 0;
  OZG_CUDA(ozg::launch_select_single(model ? c->dsel : nullptr, hist, hist + 10, m, n, k,
                                     (float)std::log10(c->target), std::max(c->sel_s_hi, c->fallback_slices),
                                     model ? s_out : nullptr, feat_out, model ? prob_out : nullptr, st));
  OZG_CUDA(cudaStreamSynchronize(st));
  return OZG_OK;
}

static int ensure_train(ozg_ctx* c) {
  if (c->train) return OZG_OK;
  cudaSetDevice(c->device);
  if (cudaMalloc(&c->train, sizeof(float) * (4 * ozg::kSelParams + 4)) != cudaSuccess) {
    cudaGetLastError();
    c->train = nullptr;
    return OZG_ERR_ALLOC;
  }
  OZG_CUDA(cudaMemset(c->train, 0, sizeof(float) * (4 * ozg::kSelParams + 4)));
  return OZG_OK;
}

extern "C" int ozg_selector_set_params(ozg_ctx* c, const float* theta) {
  if (!c || !theta) return OZG_ERR_INVALID;
  int rc = ensure_train(c);
  if (rc) return rc;
  OZG_CUDA(cudaStreamSynchronize(c->stream));
  OZG_CUDA(cudaMemcpy(c->train, theta, sizeof(float) * ozg::kSelParams, cudaMemcpyHostToDevice));
  OZG_CUDA(cudaMemset(c->train + 2 * ozg::kSelParams, 0, sizeof(float) * 2 * ozg::kSelParams));
  c->adam_step = 0;
  return OZG_OK;
}

extern "C" int ozg_selector_get_params(ozg_ctx* c, float* theta) {
  if (!c || !theta || !c->train) return OZG_ERR_INVALID;
  OZG_CUDA(cudaStreamSynchronize(c->stream));
  OZG_CUDA(cudaMemcpy(theta, c->train, sizeof(float) * ozg::kSelParams, cudaMemcpyDeviceToHost));
  return OZG_OK;
}

extern "C" int ozg_selector_grads(ozg_ctx* c, const float* X, const int* y, int B, float* grad, float* loss) {
  if (!c || !X || !y || B <= 0 || !c->train) return OZG_ERR_INVALID;
  float* theta = c->train;
  float* g = theta + ozg::kSelParams;
  float* l = theta + 4 * ozg::kSelParams;
  OZG_CUDA(ozg::launch_mlp_grads(theta, X, y, B, g, l, c->stream));
  OZG_CUDA(cudaStreamSynchronize(c->stream));
  if (grad) OZG_CUDA(cudaMemcpy(grad, g, sizeof(float) * ozg::kSelParams, cudaMemcpyDeviceToHost));
  if (loss) OZG_CUDA(cudaMemcpy(loss, l, sizeof(float), cudaMemcpyDeviceToHost));
  return OZG_OK;
}

extern "C" int ozg_selector_train_step(ozg_ctx* c, const float* X, const int* y, int B, float lr, float* loss) {
  if (!c || !X || !y || B <= 0 || !c->train || !(lr > 0.f)) return OZG_ERR_INVALID;
  float* theta = c->train;
  float* g = theta + ozg::kSelParams;
  float* m1 = theta + 2 * ozg::kSelParams;
  float* m2 = theta + 3 * ozg::kSelParams;
  float* l = theta + 4 * ozg::kSelParams;
  OZG_CUDA(ozg::launch_mlp_grads(theta, X, y, B, g, l, c->stream));
  ++c->adam_step;
  OZG_CUDA(ozg::launch_adam(theta, g, m1, m2, c->adam_step, lr, 0.9f, 0.999f, 1e-8f, 1.0f, c->stream));
  if (loss) {
    OZG_CUDA(cudaMemcpyAsync(loss, l, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    OZG_CUDA(cudaStreamSynchronize(c->stream));
  }
  return OZG_OK;
}
