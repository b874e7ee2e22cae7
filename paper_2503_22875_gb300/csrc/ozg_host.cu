// Host-side helpers shared by the C ABI translation units: CUDA error capture, workspace
// growth, per-phase event timing, and the tile-variant autotuner's cache.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>

#include "ozg_context.h"

namespace ozg {

long long& launch_counter() {
  static long long n = 0;
  return n;
}

namespace host {

namespace {
char g_last_cuda[256] = "no error";
std::mutex g_err_mu;
}  // namespace

const char* last_cuda_error_text() { return g_last_cuda; }

int cuda_fail(cudaError_t e) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  std::snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return OZG_ERR_CUDA;
}

char norm_trans(char t) {
  if (t >= 'a' && t <= 'z') t = (char)(t - 'a' + 'A');
  return t;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static int grow_buffer(ozg_ctx* c, void** buf, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return OZG_OK;
  OZG_CUDA(cudaStreamSynchronize(c->stream));
  if (*buf) {
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
  }
  size_t want = align_up(bytes + bytes / 8, 1 << 20);
  if (c->fail_allocs > 0) {  // injected failure (test hook), as if cudaMalloc had failed
    --c->fail_allocs;
    return OZG_ERR_ALLOC;
  }
  cudaError_t e = cudaMalloc(buf, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return OZG_ERR_ALLOC;
  }
  *cap = want;
  return OZG_OK;
}

int ensure_ws(ozg_ctx* c, size_t bytes) { return grow_buffer(c, &c->ws, &c->ws_cap, bytes); }
int ensure_z3ws(ozg_ctx* c, size_t bytes) { return grow_buffer(c, &c->z3ws, &c->z3ws_cap, bytes); }

int ensure_gws(ozg_ctx* c, size_t bytes) {
  if (bytes <= c->gws_cap) return OZG_OK;
  c->plan.reset();  // a captured plan points into the old buffer
  ++c->gws_epoch;
  return grow_buffer(c, &c->gws, &c->gws_cap, bytes);
}

cudaEvent_t pool_get(ozg_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

PhaseScope::PhaseScope(ozg_ctx* c_, int ph) : c(c_), phase(ph) {
  if (!c->prof) return;
  // no marks inside a graph capture (the replays are timed as a whole)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  if ((a = pool_get(c)) != nullptr) cudaEventRecord(a, c->stream);
}

PhaseScope::~PhaseScope() {
  if (!a) return;
  cudaEvent_t b = pool_get(c);
  if (!b) {
    c->pool.push_back(a);
    return;
  }
  cudaEventRecord(b, c->stream);
  c->pending.push_back({phase, a, b});
}

// Shape bucket: rounded log2 of the stacked rows, cols and k, plus the slice count.
uint64_t shape_bucket(int64_t rows, int64_t cols, int64_t k, int s) {
  auto lg = [](int64_t x) { return (uint64_t)std::lround(std::log2((double)(x > 0 ? x : 1)) * 2.0); };
  return (lg(rows) << 40) | (lg(cols) << 24) | (lg(k) << 8) | (uint64_t)s;
}

static void tune_load(ozg_ctx* c) {
  if (c->tune_loaded) return;
  c->tune_loaded = true;
  if (c->tune_path.empty()) return;
  std::ifstream in(c->tune_path);
  std::string line;
  while (std::getline(in, line)) {
    unsigned long long b = 0;
    int v = 0;
    // single-call variants: 0 .. 3 and the stacked group pairs (no CTA pairs for single calls)
    if (std::sscanf(line.c_str(), "%llx %d", &b, &v) == 2 && ((v >= 0 && v <= 3) || v == kStackedVariant))
      c->tune[b] = v;
  }
}

void tune_store(ozg_ctx* c, uint64_t bucket, int variant) {
  c->tune[bucket] = variant;
  if (c->tune_path.empty()) return;
  std::ofstream out(c->tune_path, std::ios::app);
  out << std::hex << bucket << std::dec << " " << variant << "\n";
}

// Heuristic variant: the tile width that wastes the least output area (ties -> 256 wide); for
// 256-wide tiles deferred epilogue pushes when k >= 2048 (they then overlap the next chains'
// MMAs; for short k the epilogue is the bottleneck and immediate pushes measured faster); for
// 128-wide tiles two 64-wide k sub-tiles per stage (measured faster than the deeper 6-stage
// pipeline for s = 7..12 once grouped tiles are handed out dynamically).
static int heuristic_variant(int64_t rows, int64_t cols, int64_t k, int s) {
  (void)rows;
  (void)s;
  const int64_t p256 = (cols + 255) / 256 * 256, p128 = (cols + 127) / 128 * 128;
  if (p128 < p256) return 1;
  return k >= 2048 ? 2 : 0;
}

int choose_variant(ozg_ctx* c, int64_t rows, int64_t cols, int64_t k, int s) {
  // single calls have no CTA-pair kernel: a forced pair variant runs as the 1-CTA 128-wide one
  if (c->force_variant >= 0) return c->force_variant == kPairVariant ? 1 : c->force_variant;
  tune_load(c);
  auto it = c->tune.find(shape_bucket(rows, cols, k, s));
  if (it != c->tune.end()) return it->second;
  // the stacked group pairs where they apply: on square DGEMMs of 1024 .. 8192 at s = 7 .. 10
  // they measured 0.47 - 1.06x the time of the width heuristic's choice (faster except for
  // 2048^3 and for 8192^3 at s = 10, by 6%)
  if (s <= stacked_max_slices() && !c->exact) return kStackedVariant;
  return heuristic_variant(rows, cols, k, s);
}

}  // namespace host
}  // namespace ozg

extern "C" int ozg_kernel_launches(long long* out) {
  if (!out) return OZG_ERR_INVALID;
  *out = __atomic_load_n(&ozg::launch_counter(), __ATOMIC_RELAXED);
  return OZG_OK;
}
