// K9: native FP64 / complex128 GEMM on the CUDA cores (the "dgemm" compute mode of Sec. 3.1 and
// the native comparison of Sec. 4).  FP64 throughput on this part (~1 TFLOP/s, DFMA and DMMA
// alike) is the bound, so the kernel is a plain register-blocked shared-memory GEMM:
// 64 x 64 output tile per 256 threads, 4 x 4 outputs per thread, k blocked by 16, each output
// accumulated with fma in ascending k.  Also used when an emulated call meets Inf/NaN inputs
// (gated by the flag the split kernel sets).
#include "ozg_internal.h"

namespace ozg {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

template <int CPLX>
struct Elem;
template <>
struct Elem<0> {
  using T = double;
};
template <>
struct Elem<1> {
  using T = double2;
};

__device__ __forceinline__ double load_op(const double* X, int64_t ld, char t, int64_t r, int64_t c) {
  return (t == 'N') ? X[r + c * ld] : X[c + r * ld];
}
__device__ __forceinline__ double2 load_op(const double2* X, int64_t ld, char t, int64_t r, int64_t c) {
  double2 v = (t == 'N') ? X[r + c * ld] : X[c + r * ld];
  if (t == 'C') v.y = -v.y;
  return v;
}
__device__ __forceinline__ void mac(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void mac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ double zero_of(double) { return 0.0; }
__device__ __forceinline__ double2 zero_of(double2) { return make_double2(0.0, 0.0); }

template <int CPLX>
__global__ void __launch_bounds__(256) native_gemm_kernel(NativeArgs P) {
  using T = typename Elem<CPLX>::T;
  if (P.gate != nullptr && *P.gate == 0) return;
  __shared__ T As[TK][TM + 1];
  __shared__ T Bs[TK][TN + 1];
  const T* A = reinterpret_cast<const T*>(P.A);
  const T* B = reinterpret_cast<const T*>(P.B);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t m0 = (int64_t)blockIdx.y * TM, n0 = (int64_t)blockIdx.x * TN;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero_of(T());
  for (int64_t k0 = 0; k0 < P.k; k0 += TK) {
    // A tile: TM rows x TK k; thread loads 4 elements
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = threadIdx.x + 256 * q;  // 0 .. 1023
      int rr, kk;
      if (P.ta == 'N') {
        rr = idx % TM;
        kk = idx / TM;
      } else {
        kk = idx % TK;
        rr = idx / TK;
      }
      int64_t gr = m0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < P.m && gk < P.k) ? load_op(A, P.lda, P.ta, gr, gk) : zero_of(T());
      int cc, kb;
      if (P.tb == 'N') {
        kb = idx % TK;
        cc = idx / TK;
      } else {
        cc = idx % TN;
        kb = idx / TN;
      }
      int64_t gc = n0 + cc, gk2 = k0 + kb;
      Bs[kb][cc] = (gc < P.n && gk2 < P.k) ? load_op(B, P.ldb, P.tb, gk2, gc) : zero_of(T());
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t r = m0 + ty + 16 * i, c = n0 + tx + 16 * j;
      if (r >= P.m || c >= P.n) continue;
      if (!CPLX) {
        double* cp = P.C + r + c * P.ldc;
        double t = reinterpret_cast<double*>(&acc[i][j])[0];
        *cp = P.beta_zero ? P.alpha[0] * t : fma(P.alpha[0], t, P.beta[0] * *cp);
      } else {
        double* cp = P.C + 2 * (r + c * P.ldc);
        double tr = reinterpret_cast<double*>(&acc[i][j])[0], ti = reinterpret_cast<double*>(&acc[i][j])[1];
        double re = fma(P.alpha[0], tr, -(P.alpha[1] * ti));
        double im = fma(P.alpha[0], ti, P.alpha[1] * tr);
        if (!P.beta_zero) {
          double cr = cp[0], ci = cp[1];
          re += fma(P.beta[0], cr, -(P.beta[1] * ci));
          im += fma(P.beta[0], ci, P.beta[1] * cr);
        }
        cp[0] = re;
        cp[1] = im;
      }
    }
}

__global__ void scale_c_kernel(double* C, int64_t m, int64_t n, int64_t ldc, double br, double bi, int cplx,
                               int zero) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * n) return;
  int64_t i = idx % m, j = idx / m;
  if (!cplx) {
    double* p = C + i + j * ldc;
    *p = zero ? 0.0 : br * *p;
  } else {
    double* p = C + 2 * (i + j * ldc);
    if (zero) {
      p[0] = 0.0;
      p[1] = 0.0;
    } else {
      double cr = p[0], ci = p[1];
      p[0] = fma(br, cr, -(bi * ci));
      p[1] = fma(br, ci, bi * cr);
    }
  }
}

}  // namespace

cudaError_t launch_native_gemm(const NativeArgs& a, cudaStream_t st) {
  if (a.m <= 0 || a.n <= 0) return cudaSuccess;
  dim3 grid((unsigned)((a.n + TN - 1) / TN), (unsigned)((a.m + TM - 1) / TM));
  if (grid.y > 65535) return cudaErrorInvalidValue;
  if (a.cplx)
    { native_gemm_kernel<1><<<grid, 256, 0, st>>>(a); note_launch(); }
  else
    { native_gemm_kernel<0><<<grid, 256, 0, st>>>(a); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_scale_c(double* C, int64_t m, int64_t n, int64_t ldc, const double* beta, int cplx,
                           cudaStream_t st) {
  int64_t total = m * n;
  if (total <= 0) return cudaSuccess;
  int zero = (beta[0] == 0.0 && (!cplx || beta[1] == 0.0));
  { scale_c_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(C, m, n, ldc, beta[0], cplx ? beta[1] : 0.0, cplx,
                                                                 zero); note_launch(); }
  return cudaGetLastError();
}

}  // namespace ozg
