// The library context (opaque ozg_ctx of the C ABI) and the host-side helpers shared by the
// API translation units.  Not part of the public interface.
#pragma once
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ozg.h"
#include "ozg_internal.h"

namespace ozg {
namespace host {
struct GroupPlan;  // a captured grouped call (ozg_grouped.cu)
void destroy_plan(GroupPlan* p);
struct PlanDeleter {
  void operator()(GroupPlan* p) const { destroy_plan(p); }
};
}  // namespace host
}  // namespace ozg

struct ozg_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;  // single-call workspace
  size_t ws_cap = 0;
  int* dflags = nullptr;     // [0] status (sticky until ozg_sync), [1] non-finite flag of the last call
  double* dcheck = nullptr;  // max sampled error of the last call
  int check_samples = 0;
  uint64_t check_seed = 0x5EED;
  // per-phase timing
  bool prof = false;
  struct Mark {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Mark> pending;
  std::vector<cudaEvent_t> pool;
  double acc_ms[OZG_NUM_PHASES] = {};
  int64_t acc_n[OZG_NUM_PHASES] = {};
  // grouped calls: own workspace (kept while a captured plan refers to it)
  void* gws = nullptr;
  size_t gws_cap = 0;
  uint64_t gws_epoch = 0;
  std::unique_ptr<ozg::host::GroupPlan, ozg::host::PlanDeleter> plan;
  bool graphs = true;
  int fallback_slices = 7;
  int exact = 0;  // correctly rounded (exact-sum) epilogue for single calls
  // autotuner: shape bucket -> tile variant, optionally persisted as text
  int autotune = 0;
  int force_variant = -1;  // >= 0: every call uses this tile variant
  std::string tune_path;
  std::unordered_map<uint64_t, int> tune;
  bool tune_loaded = false;
  // learned slice selector
  ozg::SelectorDev* dsel = nullptr;  // device copy of the loaded model
  int sel_s_hi = 0;                  // largest class of the loaded model (0: no model)
  double target = 1e-12;             // requested error for automatic slice counts
  float* train = nullptr;            // [theta | grad | m1 | m2 | loss] for on-GPU training
  int adam_step = 0;
  int fail_allocs = 0;  // test hook: the next n workspace allocations fail on the host side
  // 3M complex products: the real operands and products
  void* z3ws = nullptr;
  size_t z3ws_cap = 0;
  // a grouped call whose reports are read after its work finished (host-memory batches)
  struct DeferredReports {
    std::vector<int> widx, ws;
    std::vector<char> wauto;
    int64_t n = 0;
    ozg_report* reps = nullptr;
  } deferred;
  // grouped calls on host memory: device staging, copy streams and one sub-context per part
  void* hstage = nullptr;
  size_t hstage_cap = 0;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  std::vector<ozg_ctx*> hsub;
  std::vector<cudaEvent_t> hev;  // [2 per part]: inputs staged, part computed
  int host_parts = 16;
};

namespace ozg {
namespace host {

int cuda_fail(cudaError_t e);
const char* last_cuda_error_text();
#define OZG_CUDA(x)                                         \
  do {                                                      \
    cudaError_t e_ = (x);                                   \
    if (e_ != cudaSuccess) return ::ozg::host::cuda_fail(e_); \
  } while (0)

char norm_trans(char t);
size_t align_up(size_t x, size_t a);

// Bump allocator over a workspace.
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  }
};

int ensure_ws(ozg_ctx* c, size_t bytes);
int ensure_gws(ozg_ctx* c, size_t bytes);  // grouped workspace; bumps gws_epoch when it moves
int ensure_z3ws(ozg_ctx* c, size_t bytes);  // 3M operands and products
cudaEvent_t pool_get(ozg_ctx* c);

// Records an event pair around one phase on the context stream when profiling is on.
struct PhaseScope {
  ozg_ctx* c;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseScope(ozg_ctx* c_, int ph);
  ~PhaseScope();
};

template <typename T>
T* at(ozg_ctx* c, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(c->ws) + off);
}
template <typename T>
T* gat(ozg_ctx* c, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(c->gws) + off);
}

// tile variant for one GEMM shape (bit 0: BN = 128, bit 1: deferred pushes): the autotuned
// choice if known, else the heuristic (least padding; deferral for k >= 2048)
int choose_variant(ozg_ctx* c, int64_t rows, int64_t cols, int64_t k, int s);
// grouped calls (ozg_grouped.cu): with sync_reports == false the reports are filled in by
// grouped_collect_reports once the work has finished
int grouped_call(ozg_ctx* c, int64_t count, const ozg_gemm_desc* descs, const int* slices, ozg_report* reps,
                 bool sync_reports);
int grouped_collect_reports(ozg_ctx* c);
uint64_t shape_bucket(int64_t rows, int64_t cols, int64_t k, int s);
void tune_store(ozg_ctx* c, uint64_t bucket, int variant);

}  // namespace host
}  // namespace ozg
