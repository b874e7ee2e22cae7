// ozg_dgemm_grouped_host: the grouped emulated DGEMM on matrices in host (CPU) memory, the
// offload the paper's library performs for BLAS calls (Sec. 2.1, 3.1), for a whole batch.
//
// The batch is cut into parts of about equal work.  Part p's inputs are copied into device
// staging on one copy stream, computed by a grouped call on part p's own sub-context and stream
// (its CUDA graph is replayed while the batch stays the same), and its results are copied back on
// a second copy stream, so the copies of one part overlap the computation of the others.
// Matrices whose host regions touch or overlap are staged as one region and moved by one copy;
// C is copied back only where the call writes it (rows 0..m-1 of each column).
#include <algorithm>
#include <cstring>
#include <vector>

#include "ozg_context.h"

namespace ozg {
namespace host {
namespace {

struct Region {
  const char* lo;  // host bytes [lo, hi)
  const char* hi;
  int64_t call;
  int kind;  // 0 A, 1 B
};

// Elements of a column-major operand with `rows` x `cols` storage and leading dimension ld that
// a BLAS call may read: (cols - 1) ld + rows (the padding rows after the last column are not ours).
size_t operand_bytes(int64_t rows, int64_t cols, int64_t ld) {
  if (rows <= 0 || cols <= 0) return 0;
  return (size_t)((cols - 1) * ld + rows) * sizeof(double);
}

int ensure_hstage(ozg_ctx* c, size_t bytes) {
  if (bytes <= c->hstage_cap) return OZG_OK;
  OZG_CUDA(cudaDeviceSynchronize());
  if (c->hstage) cudaFree(c->hstage);
  c->hstage = nullptr;
  c->hstage_cap = 0;
  const size_t want = align_up(bytes + bytes / 16, 1 << 20);
  if (c->fail_allocs > 0) {
    --c->fail_allocs;
    return OZG_ERR_ALLOC;
  }
  if (cudaMalloc(&c->hstage, want) != cudaSuccess) {
    cudaGetLastError();
    c->hstage = nullptr;
    return OZG_ERR_ALLOC;
  }
  c->hstage_cap = want;
  return OZG_OK;
}

// Sub-contexts, streams and events for `parts` parts; each sub-context takes the parent's
// settings (selector, target, fallback, check samples, tile variant, autotuning, graphs).
int ensure_parts(ozg_ctx* c, int parts) {
  OZG_CUDA(cudaSetDevice(c->device));
  if (!c->h2d) OZG_CUDA(cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking));
  if (!c->d2h) OZG_CUDA(cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking));
  while ((int)c->hsub.size() < parts) {
    ozg_ctx* s = nullptr;
    int rc = ozg_create(&s, 0);
    if (rc) return rc;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      ozg_destroy(s);
      return cuda_fail(cudaGetLastError());
    }
    s->stream = st;
    c->hsub.push_back(s);
    for (int e = 0; e < 2; ++e) {
      cudaEvent_t ev = nullptr;
      OZG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      c->hev.push_back(ev);
    }
  }
  for (int p = 0; p < parts; ++p) {
    ozg_ctx* s = c->hsub[p];
    if (c->dsel) {
      if (!s->dsel && cudaMalloc(&s->dsel, sizeof(SelectorDev)) != cudaSuccess) {
        cudaGetLastError();
        s->dsel = nullptr;
        return OZG_ERR_ALLOC;
      }
      OZG_CUDA(cudaMemcpy(s->dsel, c->dsel, sizeof(SelectorDev), cudaMemcpyDeviceToDevice));
    }
    const int sel_hi = c->dsel ? c->sel_s_hi : 0;
    if (s->sel_s_hi != sel_hi || s->fallback_slices != c->fallback_slices || s->target != c->target ||
        s->check_samples != c->check_samples || s->force_variant != c->force_variant ||
        s->autotune != c->autotune || s->graphs != c->graphs)
      s->plan.reset();
    s->sel_s_hi = sel_hi;
    s->fallback_slices = c->fallback_slices;
    s->target = c->target;
    s->check_samples = c->check_samples;
    s->force_variant = c->force_variant;
    s->autotune = c->autotune;
    s->graphs = c->graphs;
  }
  return OZG_OK;
}

}  // namespace
}  // namespace host
}  // namespace ozg

using namespace ozg::host;

extern "C" int ozg_dgemm_grouped_host(ozg_ctx* c, int64_t count, const ozg_gemm_desc* descs, const int* slices,
                                      ozg_report* reps) {
  if (!c || count < 0 || (count > 0 && !descs)) return OZG_ERR_INVALID;
  if (count == 0) return OZG_OK;
  if (count > (1 << 20)) return OZG_ERR_UNSUPPORTED;
  // the BLAS argument checks of the device path first (nothing is copied for an invalid batch)
  for (int64_t i = 0; i < count; ++i) {
    const ozg_gemm_desc& d = descs[i];
    const char ta = norm_trans(d.transa) == 'C' ? 'T' : norm_trans(d.transa);
    const char tb = norm_trans(d.transb) == 'C' ? 'T' : norm_trans(d.transb);
    int rc = 0;
    if (ta != 'N' && ta != 'T') rc = -1;
    else if (tb != 'N' && tb != 'T') rc = -2;
    else if (d.m < 0) rc = -3;
    else if (d.n < 0) rc = -4;
    else if (d.k < 0) rc = -5;
    else if (d.lda < std::max<int64_t>(1, ta == 'N' ? d.m : d.k)) rc = -8;
    else if (d.ldb < std::max<int64_t>(1, tb == 'N' ? d.k : d.n)) rc = -10;
    else if (d.ldc < std::max<int64_t>(1, d.m)) rc = -13;
    else if (slices && (slices[i] < 0 || slices[i] > OZG_MAX_SLICES)) rc = -14;
    if (rc) {
      if (reps) {
        std::memset(reps, 0, sizeof(ozg_report) * (size_t)count);
        for (int64_t j = 0; j < count; ++j) reps[j].est_err = reps[j].max_real = reps[j].max_imag = NAN;
        reps[i].status = rc;
      }
      return OZG_ERR_INVALID;
    }
  }
  const int parts = (int)std::max<int64_t>(1, std::min<int64_t>(c->host_parts, count));
  int rc = ensure_parts(c, parts);
  if (rc) return rc;

  // parts in call order with work (2 m n k) shares rising and then falling (1, 2, 3, .., 3, 2, 1):
  // the first part's copy-in and the last part's compute and copy-out are not overlapped, so
  // they are kept small, while the middle parts are large enough to keep the per-part launches
  // and the tail of each part's persistent launch small against its work
  std::vector<double> wsum(count + 1, 0.0);
  for (int64_t i = 0; i < count; ++i) wsum[i + 1] = wsum[i] + 2.0 * descs[i].m * descs[i].n * descs[i].k;
  std::vector<double> share(parts + 1, 0.0);
  for (int p = 0; p < parts; ++p) share[p + 1] = share[p] + (double)std::min(p + 1, parts - p);
  std::vector<int64_t> cut(parts + 1, 0);
  cut[parts] = count;
  for (int p = 1; p < parts; ++p) {
    const double want = wsum[count] * share[p] / share[parts];
    cut[p] = std::max(cut[p - 1], (int64_t)(std::lower_bound(wsum.begin(), wsum.end(), want) - wsum.begin()));
    cut[p] = std::min(cut[p], count);
  }

  // staging layout: per part, the merged input regions (A and B), then C (compact, ld = m)
  struct Run {
    const char* lo;
    const char* hi;
    size_t off;
  };
  std::vector<std::vector<Run>> runs(parts);
  struct CRun {  // C of calls first..last (one call unless compact and adjacent)
    const char* lo;
    const char* hi;
    size_t off;
    int64_t first, last;
    bool compact, beta;
  };
  std::vector<std::vector<CRun>> cruns(parts);
  std::vector<size_t> offA(count), offB(count), offC(count);
  size_t total = 0;
  for (int p = 0; p < parts; ++p) {
    std::vector<Region> regs;
    for (int64_t i = cut[p]; i < cut[p + 1]; ++i) {
      const ozg_gemm_desc& d = descs[i];
      if (d.m == 0 || d.n == 0) continue;
      const char ta = norm_trans(d.transa) == 'N' ? 'N' : 'T', tb = norm_trans(d.transb) == 'N' ? 'N' : 'T';
      const size_t ba = operand_bytes(ta == 'N' ? d.m : d.k, ta == 'N' ? d.k : d.m, d.lda);
      const size_t bb = operand_bytes(tb == 'N' ? d.k : d.n, tb == 'N' ? d.n : d.k, d.ldb);
      if (ba) regs.push_back({reinterpret_cast<const char*>(d.A), reinterpret_cast<const char*>(d.A) + ba, i, 0});
      if (bb) regs.push_back({reinterpret_cast<const char*>(d.B), reinterpret_cast<const char*>(d.B) + bb, i, 1});
    }
    std::sort(regs.begin(), regs.end(), [](const Region& a, const Region& b) { return a.lo < b.lo; });
    for (size_t r = 0; r < regs.size(); ++r) {
      if (runs[p].empty() || regs[r].lo > runs[p].back().hi) {  // a gap: a new staged region
        total = align_up(total, 256);
        runs[p].push_back({regs[r].lo, regs[r].hi, total});
        total += regs[r].hi - regs[r].lo;
      } else if (regs[r].hi > runs[p].back().hi) {  // touching or overlapping: extend
        total += regs[r].hi - runs[p].back().hi;
        runs[p].back().hi = regs[r].hi;
      }
      const Run& u = runs[p].back();
      (regs[r].kind == 0 ? offA : offB)[regs[r].call] = u.off + (size_t)(regs[r].lo - u.lo);
    }
    // C: compact (ld = m) in staging; compact host C's that follow each other in memory and in
    // call order stay adjacent in staging too and move as one run
    for (int64_t i = cut[p]; i < cut[p + 1]; ++i) {
      const ozg_gemm_desc& d = descs[i];
      const size_t bytes = (size_t)std::max<int64_t>(d.m, 0) * std::max<int64_t>(d.n, 0) * sizeof(double);
      const char* h = reinterpret_cast<const char*>(d.C);
      const bool compact = d.ldc == d.m && bytes > 0;
      if (compact && !cruns[p].empty() && cruns[p].back().compact && cruns[p].back().hi == h) {
        offC[i] = cruns[p].back().off + (size_t)(h - cruns[p].back().lo);
        cruns[p].back().hi = h + bytes;
        cruns[p].back().last = i;
        cruns[p].back().beta |= d.beta != 0.0;
        total += bytes;
        continue;
      }
      total = align_up(total, 256);
      offC[i] = total;
      if (bytes > 0) cruns[p].push_back({h, h + bytes, total, i, i, compact, d.beta != 0.0});
      total += bytes;
    }
  }
  rc = ensure_hstage(c, std::max<size_t>(total, 256));
  if (rc) return rc;
  char* stage = static_cast<char*>(c->hstage);

  std::vector<ozg_gemm_desc> dev(descs, descs + count);
  for (int64_t i = 0; i < count; ++i) {
    ozg_gemm_desc& d = dev[i];
    if (d.m == 0 || d.n == 0) continue;
    if (d.k > 0) {
      d.A = reinterpret_cast<const double*>(stage + offA[i]);
      d.B = reinterpret_cast<const double*>(stage + offB[i]);
    }
    d.C = reinterpret_cast<double*>(stage + offC[i]);
    d.ldc = d.m;
  }
  if (reps) std::memset(reps, 0, sizeof(ozg_report) * (size_t)count);
  int err = OZG_OK;
  for (int p = 0; p < parts && !err; ++p) {
    ozg_ctx* s = c->hsub[p];
    cudaEvent_t in = c->hev[2 * p], done = c->hev[2 * p + 1];
    for (const Run& u : runs[p])
      if (cudaMemcpyAsync(stage + u.off, u.lo, u.hi - u.lo, cudaMemcpyHostToDevice, c->h2d) != cudaSuccess)
        err = cuda_fail(cudaGetLastError());
    for (const CRun& u : cruns[p]) {  // C_old where a call reads it
      if (err || !u.beta) continue;
      const ozg_gemm_desc& d = descs[u.first];
      cudaError_t e = u.compact ? cudaMemcpyAsync(stage + u.off, u.lo, u.hi - u.lo, cudaMemcpyHostToDevice, c->h2d)
                                : cudaMemcpy2DAsync(stage + u.off, d.m * sizeof(double), d.C, d.ldc * sizeof(double),
                                                    d.m * sizeof(double), d.n, cudaMemcpyHostToDevice, c->h2d);
      if (e != cudaSuccess) err = cuda_fail(cudaGetLastError());
    }
    if (err) break;
    OZG_CUDA(cudaEventRecord(in, c->h2d));
    OZG_CUDA(cudaStreamWaitEvent(s->stream, in, 0));
    const int64_t n = cut[p + 1] - cut[p];
    if (n > 0) {
      err = grouped_call(s, n, dev.data() + cut[p], slices ? slices + cut[p] : nullptr, reps ? reps + cut[p] : nullptr,
                         false);
      if (err) break;
    }
    OZG_CUDA(cudaEventRecord(done, s->stream));
    OZG_CUDA(cudaStreamWaitEvent(c->d2h, done, 0));
    for (const CRun& u : cruns[p]) {  // C back to host: only the entries the calls write
      if (err) break;
      const ozg_gemm_desc& d = descs[u.first];
      cudaError_t e = u.compact ? cudaMemcpyAsync(const_cast<char*>(u.lo), stage + u.off, u.hi - u.lo,
                                                  cudaMemcpyDeviceToHost, c->d2h)
                                : cudaMemcpy2DAsync(d.C, d.ldc * sizeof(double), stage + u.off, d.m * sizeof(double),
                                                    d.m * sizeof(double), d.n, cudaMemcpyDeviceToHost, c->d2h);
      if (e != cudaSuccess) err = cuda_fail(cudaGetLastError());
    }
  }
  // wait for everything queued (also after an error), then the deferred reports
  cudaError_t se = cudaStreamSynchronize(c->d2h);
  for (int p = 0; p < parts; ++p) {
    cudaError_t pe = cudaStreamSynchronize(c->hsub[p]->stream);
    if (se == cudaSuccess) se = pe;
    if (!err && reps) err = grouped_collect_reports(c->hsub[p]);
    int dst = ozg_sync(c->hsub[p]);  // device-side status of the part (time-outs)
    if (!err && dst) err = dst;
  }
  if (!err && se != cudaSuccess) err = cuda_fail(se);
  return err;
}

extern "C" int ozg_set_host_parts(ozg_ctx* c, int parts) {
  if (!c) return OZG_ERR_INVALID;
  if (parts < 1 || parts > 64) return -2;
  c->host_parts = parts;
  return OZG_OK;
}
