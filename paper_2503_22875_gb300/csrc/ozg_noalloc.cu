// ozg_dgemm_noalloc: the emulated DGEMM for callers that cannot allocate device memory.
//
// Some callers of a BLAS-style GEMM are not allowed to call cudaMalloc: code inside an
// interposed dgemm_ of a host application that already owns all device memory through its own
// pool or a fixed budget (an allocation behind its back can fail or break its accounting), and
// latency-critical paths where cudaMalloc/cudaFree would synchronise the whole device.  This
// entry point serves them: it takes the caller's inputs and output and a stream, and keeps all
// of its scratch (digit planes, exponents, row maxima, per-CTA partial-sum tiles, flags) in one
// file-scope device array of fixed size, so it calls no cudaMalloc, cudaFree or allocating
// library routine.
//
// The array is part of this library's device image: every GPU that loads it holds
// kNoAllocScratchBytes until the process exits.  All calls share the array and it keeps the
// last call's contents; each call clears what must start at zero.  Calls whose work overlaps on
// the GPU (different streams, or different host threads without ordering) race on the array.
// The kernels, their order and their arithmetic are those of ozg_dgemm.
#include <cstring>
#include <mutex>

#include "../../include/ozg.h"
#include "ozg_internal.h"

constexpr size_t kNoAllocScratchBytes = size_t(OZG_NOALLOC_SCRATCH_BYTES);  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};  // the context the address was resolved in
int g_scratch_sms[kMaxDevices] = {};
std::mutex g_setup_mu;

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// The calling thread's current context (CUcontext as void*), through the driver entry point the
// runtime exposes; null when it cannot be queried.
void* current_context() {
  typedef CUresult (*GetCtxFn)(CUcontext*);
  static GetCtxFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<GetCtxFn>(p);
    looked = true;
  }
  CUcontext c = nullptr;
  if (fn == nullptr || fn(&c) != CUDA_SUCCESS) return nullptr;
  return static_cast<void*>(c);
}

// Set-up, once per device (that device current): resolve the device address of the array.  In
// host code the array's name is only a host-side stand-in, never a device address.  The address
// belongs to the device's context; if that context was destroyed and created anew (for example
// by cudaDeviceReset in the host application), the set-up runs again in the new one.
int device_scratch(int dev, void** addr, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return OZG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  void* ctx = current_context();
  if (!g_scratch_addr[dev] || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return OZG_ERR_CUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return OZG_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = current_context();  // the runtime call above made the context current
    g_scratch_sms[dev] = n;
  }
  *addr = g_scratch_addr[dev];
  *sms = g_scratch_sms[dev];
  return OZG_OK;
}

char upper(char t) { return (t >= 'a' && t <= 'z') ? (char)(t - 'a' + 'A') : t; }

}  // namespace

extern "C" int ozg_dgemm_noalloc(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                                 double* C, int64_t ldc, int slices, void* stream) {
  char ta = upper(transa), tb = upper(transb);
  if (ta == 'C') ta = 'T';
  if (tb == 'C') tb = 'T';
  if (ta != 'N' && ta != 'T') return -1;
  if (tb != 'N' && tb != 'T') return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  const int64_t nrowa = (ta == 'N') ? m : k, nrowb = (tb == 'N') ? k : n;
  if (lda < (nrowa > 1 ? nrowa : 1)) return -8;
  if (ldb < (nrowb > 1 ? nrowb : 1)) return -10;
  if (ldc < (m > 1 ? m : 1)) return -13;
  if (slices == 0 || slices < OZG_NATIVE || slices > OZG_MAX_SLICES) return -14;
  if (m == 0 || n == 0) return OZG_OK;
  if ((alpha == 0.0 || k == 0) && beta == 1.0) return OZG_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double be[2] = {beta, 0.0};
  if (alpha == 0.0 || k == 0) return ozg::launch_scale_c(C, m, n, ldc, be, 0, st) == cudaSuccess ? OZG_OK : OZG_ERR_CUDA;

  ozg::NativeArgs na;
  na.ta = ta;
  na.tb = tb;
  na.m = m;
  na.n = n;
  na.k = k;
  na.A = A;
  na.lda = lda;
  na.B = B;
  na.ldb = ldb;
  na.C = C;
  na.ldc = ldc;
  na.alpha[0] = alpha;
  na.beta[0] = beta;
  na.beta_zero = (beta == 0.0);
  if (slices == OZG_NATIVE) return ozg::launch_native_gemm(na, st) == cudaSuccess ? OZG_OK : OZG_ERR_CUDA;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OZG_ERR_CUDA;
  void* base = nullptr;
  int sms = 0;
  int rc = device_scratch(dev, &base, &sms);
  if (rc) return rc;

  // carve the fixed array: flags | maxima | exponents | digit planes A, B | FP64 tile sums
  const int s = slices;
  const int64_t Kp = (k + 7) / 8 * 8;
  const int BM = ozg::slice_gemm_tile_m(), BN = ozg::slice_gemm_tile_n();
  const int64_t tiles = ((m + BM - 1) / BM) * ((n + BN - 1) / BN);
  const size_t tile_bytes = (size_t)BM * BN * 16;  // per-CTA scratch tile, 16 bytes per output
  size_t off = 0;
  const size_t oFlags = off;
  off = round256(off + 4 * sizeof(int));
  const size_t oMA = off;
  off = round256(off + 8 * (size_t)m);
  const size_t oMB = off;
  off = round256(off + 8 * (size_t)n);
  const size_t oE = off;
  off = round256(off + 4 * (size_t)m);
  const size_t oF = off;
  off = round256(off + 4 * (size_t)n);
  const size_t oDA = off;
  off = round256(off + (size_t)s * m * Kp * 2);
  const size_t oDB = off;
  off = round256(off + (size_t)s * n * Kp * 2);
  const size_t oR = off;
  if (off + tile_bytes > kNoAllocScratchBytes) return OZG_ERR_UNSUPPORTED;  // problem too large
  int64_t grid = (int64_t)((kNoAllocScratchBytes - off) / tile_bytes);
  if (grid > tiles) grid = tiles;
  if (grid > sms) grid = sms;

  unsigned char* p = static_cast<unsigned char*>(base);
  int* flags = reinterpret_cast<int*>(p + oFlags);  // [0] device status, [1] non-finite flag
  if (cudaMemsetAsync(flags, 0, 4 * sizeof(int), st) != cudaSuccess) return OZG_ERR_CUDA;

  ozg::SplitArgs sa;
  sa.X = A;
  sa.ld = lda;
  sa.rows = m;
  sa.k = k;
  sa.strided = (ta == 'N');
  sa.s = s;
  sa.Kp = Kp;
  sa.plane_rows = m;
  sa.D = reinterpret_cast<__half*>(p + oDA);
  sa.maxbits = reinterpret_cast<unsigned long long*>(p + oMA);  // zeroed by launch_split
  sa.exps = reinterpret_cast<int32_t*>(p + oE);
  sa.nonfinite = flags + 1;
  if (ozg::launch_split(sa, st) != cudaSuccess) return OZG_ERR_CUDA;
  ozg::SplitArgs sb = sa;
  sb.X = B;
  sb.ld = ldb;
  sb.rows = n;
  sb.strided = (tb == 'T');
  sb.plane_rows = n;
  sb.D = reinterpret_cast<__half*>(p + oDB);
  sb.maxbits = reinterpret_cast<unsigned long long*>(p + oMB);
  sb.exps = reinterpret_cast<int32_t*>(p + oF);
  if (ozg::launch_split(sb, st) != cudaSuccess) return OZG_ERR_CUDA;

  CUtensorMap tmA, tmB;
  if (ozg::make_digit_tmap(&tmA, sa.D, k, m, Kp, s, BM) != cudaSuccess) return OZG_ERR_CUDA;
  if (ozg::make_digit_tmap(&tmB, sb.D, k, n, Kp, s, BN) != cudaSuccess) return OZG_ERR_CUDA;
  ozg::GemmArgs ga;
  ga.rows = m;
  ga.cols = n;
  ga.m = m;
  ga.n = n;
  ga.k = k;
  ga.s = s;
  ga.e = sa.exps;
  ga.f = sb.exps;
  ga.C = C;
  ga.ldc = ldc;
  ga.alpha[0] = alpha;
  ga.beta[0] = beta;
  ga.beta_zero = (beta == 0.0);
  ga.Rws = reinterpret_cast<double*>(p + oR);
  ga.status = flags;
  ga.nonfinite = flags + 1;
  ga.grid = (int)grid;
  if (ozg::launch_slice_gemm(tmA, tmB, ga, st) != cudaSuccess) return OZG_ERR_CUDA;
  na.gate = flags + 1;
  if (ozg::launch_native_gemm(na, st) != cudaSuccess) return OZG_ERR_CUDA;
  return OZG_OK;
}
