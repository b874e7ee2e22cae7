// libozg_blas.so: Fortran dgemm_ / zgemm_ that offload a host program's BLAS calls to the GPU
// emulation (the automatic-offload side of the paper, Sec. 3.1: one preloaded library that
// intercepts the BLAS call and runs it on the GPU in the mode named by an environment
// variable).  Data movement follows one of the three strategies of Sec. 2.1 (named by
// OZG_DATA_STRATEGY): explicit copies (DMA from the caller's host arrays to the device, and back),
// cache-coherent access (the kernels read and write the caller's host arrays in place over the
// CPU-GPU link), or migration on first use (the pages of an array move to GPU memory the first
// time a call uses it and stay there; the CPU keeps coherent access).  See include/ozg_blas.h
// for the contract.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <unistd.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <iterator>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/ozg.h"
#include "../../include/ozg_blas.h"

namespace {

typedef void (*gemm_fn)(const char*, const char*, const int*, const int*, const int*, const double*, const double*,
                        const int*, const double*, const int*, const double*, double*, const int*, size_t, size_t);

std::mutex g_mu;
ozg_ctx* g_ctx = nullptr;
cudaStream_t g_stream = nullptr;
int g_mode = 0;  // 0: not read yet
long long g_min_mnk = 0;
void* g_dev = nullptr;
size_t g_dev_cap = 0;
gemm_fn g_next_d = nullptr, g_next_z = nullptr;
bool g_resolved = false;
std::atomic<long long> g_offloaded{0}, g_passed{0}, g_migrated{0};

// data strategies (the values of ozg_blas_parse_strategy)
constexpr int kCopy = 0, kCoherent = 1, kMigrate = 2;
int g_strategy_req = -1;  // requested (-1: not read yet)
int g_strategy = -1;      // in effect (-1: not decided yet; decided at the first GPU use)
// migration on first use: page-aligned [start, end) ranges already moved to GPU memory
std::map<uintptr_t, uintptr_t> g_moved;
size_t g_moved_bytes = 0, g_move_limit = 0;
bool g_move_failed = false;

char upper(char c) { return (c >= 'a' && c <= 'z') ? (char)(c - 'a' + 'A') : c; }

int parse_strategy(const char* s) {
  if (!s) return -1;
  if (std::strcmp(s, "copy") == 0) return kCopy;
  if (std::strcmp(s, "coherent") == 0) return kCoherent;
  if (std::strcmp(s, "migrate") == 0) return kMigrate;
  return -1;
}

int parse_mode(const char* s) {
  if (!s) return 0;
  if (std::strcmp(s, "dgemm") == 0) return OZG_NATIVE;
  const char* pre = "fp64_int8_";
  size_t n = std::strlen(pre);
  if (std::strncmp(s, pre, n) != 0) return 0;
  const char* p = s + n;
  if (!*p) return 0;
  int v = 0;
  for (; *p; ++p) {
    if (*p < '0' || *p > '9') return 0;
    v = v * 10 + (*p - '0');
    if (v > OZG_MAX_SLICES) return 0;
  }
  return (v >= 1) ? v : 0;
}

void init_locked() {
  if (g_mode == 0) {
    const char* e = std::getenv("OZG_COMPUTE_MODE");
    int m = e ? parse_mode(e) : 7;
    if (m == 0) {
      std::fprintf(stderr, "ozg_blas: invalid OZG_COMPUTE_MODE '%s'; using fp64_int8_7\n", e);
      m = 7;
    }
    g_mode = m;
    const char* t = std::getenv("OZG_OFFLOAD_MIN_MNK");
    g_min_mnk = t ? std::atoll(t) : 0;
  }
  if (g_strategy_req < 0) {
    const char* e = std::getenv("OZG_DATA_STRATEGY");
    int v = e ? parse_strategy(e) : kCopy;
    if (v < 0) {
      std::fprintf(stderr, "ozg_blas: invalid OZG_DATA_STRATEGY '%s'; using copy\n", e);
      v = kCopy;
    }
    g_strategy_req = v;
  }
  if (!g_resolved) {
    g_next_d = reinterpret_cast<gemm_fn>(dlsym(RTLD_NEXT, "dgemm_"));
    g_next_z = reinterpret_cast<gemm_fn>(dlsym(RTLD_NEXT, "zgemm_"));
    g_resolved = true;
  }
}

// The strategy in effect on the current device: in-place access needs the GPU to reach
// pageable host memory (cudaDevAttrPageableMemoryAccess, e.g. through the CPU's page tables on
// a coherent CPU-GPU link); migration also needs concurrent managed access.  Otherwise the
// request falls back (with a message) to the next weaker strategy.
int decide_strategy_locked(int req) {
  if (req == kCopy) return kCopy;
  int dev = 0, pageable = 0, concurrent = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&concurrent, cudaDevAttrConcurrentManagedAccess, dev) != cudaSuccess) {
    cudaGetLastError();
    pageable = concurrent = 0;
  }
  if (!pageable) {
    std::fprintf(stderr, "ozg_blas: the GPU cannot access pageable host memory; data strategy copy\n");
    return kCopy;
  }
  if (req == kMigrate && !concurrent) {
    std::fprintf(stderr, "ozg_blas: no concurrent managed access; data strategy coherent\n");
    return kCoherent;
  }
  if (req == kMigrate && g_move_limit == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      tot = 0;
    }
    const char* lim = std::getenv("OZG_MIGRATE_LIMIT_MB");
    g_move_limit = lim ? (size_t)std::atoll(lim) << 20 : tot / 2;
  }
  return req;
}

// Migration on first use: move the parts of [p, p + bytes) not moved before to GPU memory
// (stream-ordered before the call's kernels).  Correctness never depends on this map -- every
// access to such memory is coherent wherever the pages are -- so an array freed and reallocated
// by the application only costs speed.  Moving stops at the limit; later arrays are accessed in
// place.
void migrate_first_use_locked(const void* p, size_t bytes, int dev) {
  if (bytes == 0 || g_move_failed) return;
  static const uintptr_t page = (uintptr_t)sysconf(_SC_PAGESIZE);
  uintptr_t a = (uintptr_t)p / page * page, b = ((uintptr_t)p + bytes + page - 1) / page * page;
  std::vector<std::pair<uintptr_t, uintptr_t>> gaps;
  uintptr_t cur = a;
  auto it = g_moved.upper_bound(a);
  if (it != g_moved.begin()) --it;
  for (; it != g_moved.end() && it->first < b; ++it) {
    if (it->second <= cur) continue;
    if (it->first > cur) gaps.push_back({cur, it->first});
    cur = it->second > cur ? it->second : cur;
  }
  if (cur < b) gaps.push_back({cur, b});
  for (auto& gp : gaps) {
    const size_t len = gp.second - gp.first;
    if (g_moved_bytes + len > g_move_limit) return;
    cudaMemLocation loc;
    loc.type = cudaMemLocationTypeDevice;
    loc.id = dev;
    if (cudaMemPrefetchAsync(reinterpret_cast<const void*>(gp.first), len, loc, 0, g_stream) != cudaSuccess) {
      cudaGetLastError();
      g_move_failed = true;
      std::fprintf(stderr, "ozg_blas: page migration failed; arrays are accessed in place\n");
      return;
    }
    g_moved_bytes += len;
    g_migrated += (long long)len;
    // insert and merge with the neighbours
    uintptr_t lo = gp.first, hi = gp.second;
    auto nx = g_moved.lower_bound(lo);
    if (nx != g_moved.begin()) {
      auto pv = std::prev(nx);
      if (pv->second >= lo) {
        lo = pv->first;
        hi = pv->second > hi ? pv->second : hi;
        g_moved.erase(pv);
      }
    }
    nx = g_moved.lower_bound(lo);
    while (nx != g_moved.end() && nx->first <= hi) {
      hi = nx->second > hi ? nx->second : hi;
      nx = g_moved.erase(nx);
    }
    g_moved[lo] = hi;
  }
}

bool ensure_gpu_locked() {
  if (g_ctx) {
    if (g_strategy < 0) g_strategy = decide_strategy_locked(g_strategy_req);
    return true;
  }
  if (ozg_create(&g_ctx, 0) != OZG_OK) {
    g_ctx = nullptr;
    return false;
  }
  if (cudaStreamCreateWithFlags(&g_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    g_stream = nullptr;
  }
  ozg_set_stream(g_ctx, g_stream);
  if (g_strategy < 0) g_strategy = decide_strategy_locked(g_strategy_req);
  return true;
}

bool grow(void** buf, size_t* cap, size_t need) {  // device buffer of at least `need` bytes
  if (need <= *cap) return true;
  if (*buf) {
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
  }
  size_t want = need + need / 4;
  if (cudaMalloc(buf, want) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return false;
  }
  *cap = want;
  return true;
}

void xerbla(const char* name, int info) {
  std::fprintf(stderr, " ** On entry to %s parameter number %2d had an illegal value\n", name, info);
}

// elements spanned by a column-major rows x cols block with leading dimension ld
size_t span(long long rows, long long cols, long long ld) {
  if (rows <= 0 || cols <= 0) return 0;
  return (size_t)((cols - 1) * ld + rows);
}

// Shared body of dgemm_ / zgemm_ (esz = 8 or 16 bytes per element).
void gemm_offload(bool cplx, const char* transa, const char* transb, const int* pm, const int* pn, const int* pk,
                  const double* alpha, const double* A, const int* plda, const double* B, const int* pldb,
                  const double* beta, double* C, const int* pldc, size_t la, size_t lb) {
  const char* name = cplx ? "ZGEMM " : "DGEMM ";
  char ta = upper(*transa), tb = upper(*transb);
  const int m = *pm, n = *pn, k = *pk, lda = *plda, ldb = *pldb, ldc = *pldc;
  auto ok_t = [&](char t) { return t == 'N' || t == 'T' || t == 'C'; };
  int info = 0;
  int nrowa = (ta == 'N') ? m : k, nrowb = (tb == 'N') ? k : n;
  if (!ok_t(ta)) info = 1;
  else if (!ok_t(tb)) info = 2;
  else if (m < 0) info = 3;
  else if (n < 0) info = 4;
  else if (k < 0) info = 5;
  else if (lda < (nrowa > 1 ? nrowa : 1)) info = 8;
  else if (ldb < (nrowb > 1 ? nrowb : 1)) info = 10;
  else if (ldc < (m > 1 ? m : 1)) info = 13;
  if (info) {
    xerbla(name, info);
    return;
  }
  const bool alpha_zero = alpha[0] == 0.0 && (!cplx || alpha[1] == 0.0);
  const bool beta_one = beta[0] == 1.0 && (!cplx || beta[1] == 0.0);
  const bool beta_zero = beta[0] == 0.0 && (!cplx || beta[1] == 0.0);
  if (m == 0 || n == 0 || ((alpha_zero || k == 0) && beta_one)) return;

  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  gemm_fn next = cplx ? g_next_z : g_next_d;
  if (next && (long long)m * n * k < g_min_mnk) {
    ++g_passed;
    next(transa, transb, pm, pn, pk, alpha, A, plda, B, pldb, beta, C, pldc, la, lb);
    return;
  }
  const size_t esz = cplx ? 16 : 8;
  const size_t sA = span(nrowa, (ta == 'N') ? k : m, lda), sB = span(nrowb, (tb == 'N') ? n : k, ldb);
  const size_t sC = span(m, n, ldc);
  const size_t oA = 0, oB = (oA + sA * esz + 255) / 256 * 256, oC = (oB + sB * esz + 255) / 256 * 256;
  const size_t total = oC + sC * esz;
  int rc = OZG_ERR_ALLOC;
  if (ensure_gpu_locked() && g_strategy != kCopy) {
    // in place: the kernels read op(A), op(B) (and C when beta != 0) from the caller's arrays and
    // write C there; with migration the arrays' pages move to GPU memory on first use
    if (g_strategy == kMigrate) {
      int dev = 0;
      cudaGetDevice(&dev);
      migrate_first_use_locked(A, sA * esz, dev);
      migrate_first_use_locked(B, sB * esz, dev);
      migrate_first_use_locked(C, sC * esz, dev);
    }
    rc = cplx ? ozg_zgemm(g_ctx, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, g_mode, nullptr)
              : ozg_dgemm(g_ctx, ta, tb, m, n, k, alpha[0], A, lda, B, ldb, beta[0], C, ldc, g_mode, nullptr);
    if (rc == OZG_OK) {
      if (cudaStreamSynchronize(g_stream) == cudaSuccess) {
        rc = ozg_sync(g_ctx);
      } else {
        cudaGetLastError();
        rc = OZG_ERR_CUDA;
      }
    }
    if (rc == OZG_OK) {
      ++g_offloaded;
      return;
    }
    // A failure inside the launch sequence may have written part of C already: the CPU BLAS
    // below recomputes C only when beta == 0 made C write-only.
    if (!beta_zero) {
      std::fprintf(stderr, "ozg_blas: GPU path failed (%s) after C may have been modified\n", ozg_strerror(rc));
      return;
    }
  }
  // copies: DMA straight from and to the caller's (pageable) arrays, no CPU staging copy
  bool gpu = g_ctx != nullptr && g_strategy == kCopy && grow(&g_dev, &g_dev_cap, total);
  if (gpu) {
    char* dp = static_cast<char*>(g_dev);
    const bool need_c = !beta_zero;
    cudaError_t e = cudaSuccess;
    if (sA) e = cudaMemcpyAsync(dp + oA, A, sA * esz, cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess && sB) e = cudaMemcpyAsync(dp + oB, B, sB * esz, cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess && need_c) e = cudaMemcpyAsync(dp + oC, C, sC * esz, cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess) {
      const double* dA = reinterpret_cast<const double*>(dp + oA);
      const double* dB = reinterpret_cast<const double*>(dp + oB);
      double* dC = reinterpret_cast<double*>(dp + oC);
      // k == 0 or alpha == 0 never reads A / B; give the library valid (unused) pointers
      rc = cplx ? ozg_zgemm(g_ctx, ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc, g_mode, nullptr)
                : ozg_dgemm(g_ctx, ta, tb, m, n, k, alpha[0], dA, lda, dB, ldb, beta[0], dC, ldc, g_mode, nullptr);
      if (rc == OZG_OK) {
        // rows 0 .. m-1 of each column only: rows m .. ldc-1 stay untouched
        e = cudaMemcpy2DAsync(C, (size_t)ldc * esz, dC, (size_t)ldc * esz, (size_t)m * esz, (size_t)n,
                              cudaMemcpyDeviceToHost, g_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
        if (e == cudaSuccess) rc = ozg_sync(g_ctx);
        else rc = OZG_ERR_CUDA;
      }
    } else {
      rc = OZG_ERR_CUDA;
    }
    if (e != cudaSuccess) cudaGetLastError();
    if (rc == OZG_OK) {
      ++g_offloaded;
      return;
    }
  }
  if (next) {
    std::fprintf(stderr, "ozg_blas: GPU path failed (%s); using the CPU BLAS\n", ozg_strerror(rc));
    ++g_passed;
    next(transa, transb, pm, pn, pk, alpha, A, plda, B, pldb, beta, C, pldc, la, lb);
  } else {
    std::fprintf(stderr, "ozg_blas: GPU path failed (%s) and no CPU BLAS is loaded; C is unchanged\n",
                 ozg_strerror(rc));
  }
}

}  // namespace

extern "C" {

void dgemm_(const char* transa, const char* transb, const int* m, const int* n, const int* k, const double* alpha,
            const double* A, const int* lda, const double* B, const int* ldb, const double* beta, double* C,
            const int* ldc, size_t la, size_t lb) {
  gemm_offload(false, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, la, lb);
}

void zgemm_(const char* transa, const char* transb, const int* m, const int* n, const int* k, const double* alpha,
            const double* A, const int* lda, const double* B, const int* ldb, const double* beta, double* C,
            const int* ldc, size_t la, size_t lb) {
  gemm_offload(true, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, la, lb);
}

int ozg_blas_parse_mode(const char* mode) { return parse_mode(mode); }

int ozg_blas_get_mode(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  return g_mode;
}

int ozg_blas_set_mode(int slices) {
  if (slices == 0 || slices < OZG_NATIVE || slices > OZG_MAX_SLICES) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  g_mode = slices;
  return 0;
}

int ozg_blas_parse_strategy(const char* strategy) { return parse_strategy(strategy); }

int ozg_blas_get_strategy(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  return g_strategy >= 0 ? g_strategy : g_strategy_req;
}

int ozg_blas_set_strategy(int strategy) {
  if (strategy < kCopy || strategy > kMigrate) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  g_strategy_req = strategy;
  g_strategy = g_ctx ? decide_strategy_locked(strategy) : -1;
  return 0;
}

long long ozg_blas_migrated_bytes(void) { return g_migrated.load(); }

long long ozg_blas_offloaded_calls(void) { return g_offloaded.load(); }
long long ozg_blas_passed_calls(void) { return g_passed.load(); }

}  // extern "C"
