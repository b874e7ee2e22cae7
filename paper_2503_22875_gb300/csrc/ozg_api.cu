// C ABI (include/ozg.h): argument checking with BLAS xerbla numbering, quick returns,
// workspace management and the launch sequence of the emulated GEMM:
//   split(op(A)) -> split(op(B)) -> fused slice-GEMM + epilogue -> native kernel gated on
//   the non-finite flag (runs only if an input held Inf/NaN).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "ozg_context.h"

namespace {
using namespace ozg::host;

int check_gemm_args(bool cplx, char& ta, char& tb, int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb,
                    int64_t ldc) {
  ta = norm_trans(ta);
  tb = norm_trans(tb);
  if (!cplx) {  // BLAS dgemm accepts 'C' as 'T'
    if (ta == 'C') ta = 'T';
    if (tb == 'C') tb = 'T';
  }
  if (ta != 'N' && ta != 'T' && ta != 'C') return -1;
  if (tb != 'N' && tb != 'T' && tb != 'C') return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  int64_t nrowa = (ta == 'N') ? m : k, nrowb = (tb == 'N') ? k : n;
  if (lda < (nrowa > 1 ? nrowa : 1)) return -8;
  if (ldb < (nrowb > 1 ? nrowb : 1)) return -10;
  if (ldc < (m > 1 ? m : 1)) return -13;
  return 0;
}

// Emulated real or complex GEMM.  alpha/beta: {re, im} (im ignored for real).  When Gdbg is
// set, exports the int64 group products instead of computing C.
int emu_gemm(ozg_ctx* c, bool cplx, char ta, char tb, int64_t m, int64_t n, int64_t k, const double* alpha,
             const double* A, int64_t lda, const double* B, int64_t ldb, const double* beta, double* C, int64_t ldc,
             int s, ozg_report* rep, int64_t* Gdbg) {
  // automatic slice count: the selector chooses s on the device; digit planes are written for
  // its largest class (by the prefix property the GEMM uses the first s), the sampled check is
  // always on, and a failed check re-runs the call at the fallback count
  const bool autos = (s == 0) && c->sel_s_hi > 0 && !Gdbg;
  if (s == 0 && !autos) s = c->fallback_slices;
  const int s_fb = c->fallback_slices;
  if (autos) s = std::max(c->sel_s_hi, s_fb);
  const int nsamp = autos ? std::max(c->check_samples, 64) : c->check_samples;
  const bool beta_zero0 = (beta[0] == 0.0 && (!cplx || beta[1] == 0.0));
  const int64_t Kp = (int64_t)align_up((size_t)k, 8);
  const int64_t prA = cplx ? 2 * m : m, prB = cplx ? 2 * n : n;
  const int BM = ozg::slice_gemm_tile_m();
  auto grid_of = [&](int variant) {
    const int BN = ozg::slice_gemm_tile_n_of(variant);
    const int64_t tiles = ((prA + BM - 1) / BM) * ((prB + BN - 1) / BN);
    return (int)(tiles < c->num_sms ? tiles : c->num_sms);
  };  // depends on the tile width (bit 0) only
  const int grid = grid_of(0) > grid_of(1) ? grid_of(0) : grid_of(1);  // R scratch for either width
  Carve cv;
  size_t oDA = cv.take((size_t)s * prA * Kp * 2), oDB = cv.take((size_t)s * prB * Kp * 2);
  size_t oE = cv.take(4 * (size_t)m), oF = cv.take(4 * (size_t)n);
  size_t oMA = cv.take(8 * (size_t)m), oMB = cv.take(8 * (size_t)n);
  size_t oR = cv.take((size_t)grid * BM * 256 * 16);  // 16 bytes per output (128-bit Horner sum)
  size_t oCold = cv.take((size_t)(nsamp > 0 ? nsamp : 1) * 16);
  size_t oHist = cv.take(2 * 10 * 8), oSd = cv.take(4 * sizeof(int)), oErr2 = cv.take(sizeof(double));
  size_t oSaved = cv.take((autos && !beta_zero0) ? (size_t)m * n * (cplx ? 16 : 8) : 8);
  int rc = ensure_ws(c, cv.off);
  if (rc) return rc;
  cudaStream_t st = c->stream;
  int* nonfinite = c->dflags + 1;
  OZG_CUDA(cudaMemsetAsync(nonfinite, 0, sizeof(int), st));

  PhaseScope* split_scope = new PhaseScope(c, OZG_PHASE_SPLIT);
  ozg::SplitArgs sa;
  sa.X = A;
  sa.ld = lda;
  sa.rows = m;
  sa.k = k;
  sa.strided = (ta == 'N');
  sa.conj = (ta == 'C');
  sa.cplx = cplx;
  sa.s = s;
  sa.Kp = Kp;
  sa.plane_rows = prA;
  sa.D = at<__half>(c, oDA);
  sa.maxbits = at<unsigned long long>(c, oMA);
  sa.exps = at<int32_t>(c, oE);
  sa.nonfinite = nonfinite;
  // learned count: row maxima -> features -> selection -> digits up to the selected count only
  int* s_dev = at<int>(c, oSd);  // [0] chosen s, [1] 1 unless the check forced a re-run
  if (autos) sa.plane_to = s_dev;
  ozg::SplitArgs sb = sa;
  sb.X = B;
  sb.ld = ldb;
  sb.rows = n;
  sb.strided = (tb != 'N');
  sb.conj = (tb == 'C');
  sb.plane_rows = prB;
  sb.D = at<__half>(c, oDB);
  sb.maxbits = at<unsigned long long>(c, oMB);
  sb.exps = at<int32_t>(c, oF);
  // learned count with rows that fit a fused statistics unit: row maxima and features in one read
  const bool fused = autos && ozg::stats_fused(sa) && ozg::stats_fused(sb);
  unsigned long long* hist = at<unsigned long long>(c, oHist);
  {
    cudaError_t e = cudaSuccess;
    if (fused) {
      e = cudaMemsetAsync(hist, 0, 2 * 10 * 8, st);
      ozg::SplitArgs ha = sa, hb = sb;
      ha.hist = hist;
      hb.hist = hist + 10;
      if (e == cudaSuccess) e = ozg::launch_stats_pair(ha, hb, st);
    } else {
      e = autos ? ozg::launch_rowmax(sa, st) : ozg::launch_split(sa, st);
      if (e == cudaSuccess) e = autos ? ozg::launch_rowmax(sb, st) : ozg::launch_split(sb, st);
    }
    delete split_scope;
    OZG_CUDA(e);
  }
  if (autos) {
    PhaseScope ps(c, OZG_PHASE_SELECT);
    if (!fused) {
      OZG_CUDA(cudaMemsetAsync(hist, 0, 2 * 10 * 8, st));
      ozg::SplitArgs ha = sa, hb = sb;
      ha.hist = hist;
      hb.hist = hist + 10;
      OZG_CUDA(ozg::launch_gap_hist_pair(ha, hb, st));
    }
    OZG_CUDA(ozg::launch_select_single(c->dsel, hist, hist + 10, m, n, k, (float)std::log10(c->target), s, s_dev,
                                       nullptr, nullptr, st));
  }
  if (autos) {
    PhaseScope ps(c, OZG_PHASE_SPLIT);
    OZG_CUDA(ozg::launch_digits(sa, st));
    OZG_CUDA(ozg::launch_digits(sb, st));
  }

  CUtensorMap tmA, tmB[2];
  OZG_CUDA(ozg::make_digit_tmap(&tmA, sa.D, k, prA, Kp, s, BM));
  OZG_CUDA(ozg::make_digit_tmap(&tmB[0], sb.D, k, prB, Kp, s, ozg::slice_gemm_tile_n_of(0)));
  OZG_CUDA(ozg::make_digit_tmap(&tmB[1], sb.D, k, prB, Kp, s, ozg::slice_gemm_tile_n_of(1)));
  // tmB[v & 1] serves variant v
  int variant = choose_variant(c, prA, prB, k, s);
  ozg::GemmArgs ga;
  ga.rows = prA;
  ga.cols = prB;
  ga.m = m;
  ga.n = n;
  ga.k = k;
  ga.s = s;
  ga.cplx = cplx;
  ga.e = sa.exps;
  ga.f = sb.exps;
  ga.C = C;
  ga.ldc = ldc;
  ga.alpha[0] = alpha[0];
  ga.alpha[1] = cplx ? alpha[1] : 0.0;
  ga.beta[0] = beta[0];
  ga.beta[1] = cplx ? beta[1] : 0.0;
  ga.beta_zero = (beta[0] == 0.0 && (!cplx || beta[1] == 0.0));
  ga.Rws = at<double>(c, oR);
  ga.Gdbg = Gdbg;
  ga.status = c->dflags;
  ga.nonfinite = Gdbg ? nullptr : nonfinite;
  ga.variant = variant;
  ga.defer = ozg::variant_defers(variant);
  ga.grid = grid_of(variant);
  ga.s_dev = autos ? s_dev : nullptr;
  ga.exact = c->exact;
  if (c->autotune && c->force_variant < 0 && !Gdbg && ga.beta_zero && !autos) {
    const uint64_t bucket = shape_bucket(prA, prB, k, s);
    if (c->tune.find(bucket) == c->tune.end()) {
      // time the 1-CTA variants (two widths x stage shape or deferred pushes, and the stacked
      // group pairs) on this call (C is write-only here and every variant gives the same bits)
      float best = 1e30f;
      for (int v : {0, 1, 2, 3, ozg::kStackedVariant}) {
        if (v == ozg::kStackedVariant && (s > ozg::stacked_max_slices() || c->exact)) continue;
        ozg::GemmArgs gt = ga;
        gt.variant = v;
        gt.defer = ozg::variant_defers(v);
        gt.grid = grid_of(v);
        cudaEvent_t e0 = pool_get(c), e1 = pool_get(c);
        if (!e0 || !e1) return OZG_ERR_CUDA;
        OZG_CUDA(cudaEventRecord(e0, st));
        cudaError_t le = ozg::launch_slice_gemm(tmA, tmB[v & 1], gt, st);
        OZG_CUDA(cudaEventRecord(e1, st));
        float ms = 1e30f;
        if (le == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        c->pool.push_back(e0);
        c->pool.push_back(e1);
        OZG_CUDA(le);
        if (ms < best) {
          best = ms;
          variant = v;
        }
      }
      tune_store(c, bucket, variant);
      ga.variant = variant;
      ga.defer = ozg::variant_defers(variant);
      ga.grid = grid_of(variant);
    }
  }
  ozg::CheckArgs ck;
  if (autos && !beta_zero0)
    OZG_CUDA(cudaMemcpy2DAsync(at<double>(c, oSaved), (size_t)m * (cplx ? 16 : 8), C, (size_t)ldc * (cplx ? 16 : 8),
                               (size_t)m * (cplx ? 16 : 8), (size_t)n, cudaMemcpyDeviceToDevice, st));
  if (nsamp > 0 && !Gdbg) {
    ck.ta = ta;
    ck.tb = tb;
    ck.m = m;
    ck.n = n;
    ck.k = k;
    ck.A = A;
    ck.lda = lda;
    ck.B = B;
    ck.ldb = ldb;
    ck.C = C;
    ck.ldc = ldc;
    ck.alpha[0] = ga.alpha[0];
    ck.alpha[1] = ga.alpha[1];
    ck.beta[0] = ga.beta[0];
    ck.beta[1] = ga.beta[1];
    ck.beta_zero = ga.beta_zero;
    ck.cplx = cplx;
    ck.nsamp = nsamp;
    ck.seed = c->check_seed++;
    ck.cold = at<double>(c, oCold);
    ck.err_out = c->dcheck;
    ck.part_err = cplx ? c->dcheck + 1 : nullptr;
    ck.gate = nonfinite;
    if (!cplx) {  // the split's exponents bound every product: exact integer reference
      ck.ea = sa.exps;
      ck.fb = sb.exps;
    }
    PhaseScope ps(c, OZG_PHASE_CHECK);
    OZG_CUDA(ozg::launch_check_pre(ck, st));
  }
  {
    PhaseScope ps(c, OZG_PHASE_GEMM);
    OZG_CUDA(ozg::launch_slice_gemm(tmA, tmB[ga.variant & 1], ga, st));
  }
  if (Gdbg) return OZG_OK;

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
  na.alpha[0] = ga.alpha[0];
  na.alpha[1] = ga.alpha[1];
  na.beta[0] = ga.beta[0];
  na.beta[1] = ga.beta[1];
  na.beta_zero = ga.beta_zero;
  na.cplx = cplx;
  na.gate = nonfinite;
  {
    PhaseScope ps(c, OZG_PHASE_NATIVE);
    OZG_CUDA(ozg::launch_native_gemm(na, st));
  }
  if (nsamp > 0) {
    PhaseScope ps(c, OZG_PHASE_CHECK);
    OZG_CUDA(ozg::launch_check_post(ck, st));
  }
  const int s_rep = std::min(s_fb, s);
  if (autos) {  // judged by the check: re-run at the fallback count when the error is too large
    OZG_CUDA(ozg::launch_repair_prep(c->dcheck, c->target, s_dev + 1, at<double>(c, oSaved), C, m, n, ldc,
                                     cplx ? 2 : 1, beta_zero0 ? 0 : 1, st));
    // the planes above the selected count, for the re-run only
    ozg::SplitArgs ca = sa, cb = sb;
    ca.plane_from = cb.plane_from = s_dev;
    ca.plane_to = cb.plane_to = nullptr;
    ca.gate = cb.gate = s_dev + 1;
    OZG_CUDA(ozg::launch_digits(ca, st));
    OZG_CUDA(ozg::launch_digits(cb, st));
    ozg::GemmArgs g2 = ga;
    g2.s = s_rep;
    g2.s_dev = nullptr;
    g2.nonfinite = s_dev + 1;  // the kernel exits unless the repair is needed
    OZG_CUDA(ozg::launch_slice_gemm(tmA, tmB[g2.variant & 1], g2, st));
    ozg::CheckArgs ck2 = ck;
    ck2.err_out = at<double>(c, oErr2);
    ck2.part_err = nullptr;
    ck2.gate = s_dev + 1;
    OZG_CUDA(ozg::launch_check_post(ck2, st));
  }
  if (rep) {
    int h = 0, sd[2] = {s, 1};
    double err = 0.0, err2 = 0.0, parts[2] = {NAN, NAN};
    OZG_CUDA(cudaMemcpyAsync(&h, nonfinite, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (nsamp > 0) OZG_CUDA(cudaMemcpyAsync(&err, c->dcheck, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (nsamp > 0 && cplx) OZG_CUDA(cudaMemcpyAsync(parts, c->dcheck + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (autos) {
      OZG_CUDA(cudaMemcpyAsync(sd, s_dev, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
      OZG_CUDA(cudaMemcpyAsync(&err2, at<double>(c, oErr2), sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    OZG_CUDA(cudaStreamSynchronize(st));
    rep->nonfinite = h;
    rep->slices_used = h ? -1 : (autos ? (sd[1] ? sd[0] : s_rep) : s);
    rep->samples = (nsamp > 0 && !h) ? nsamp : 0;
    rep->est_err = rep->samples ? ((autos && !sd[1]) ? err2 : err) : NAN;
    rep->max_real = (rep->samples && cplx && !(autos && !sd[1])) ? parts[0] : NAN;
    rep->max_imag = (rep->samples && cplx && !(autos && !sd[1])) ? parts[1] : NAN;
    rep->selected = autos ? sd[0] : 0;
    rep->repaired = (autos && !h && !sd[1]) ? 1 : 0;
  }
  return OZG_OK;
}

int gemm_entry(ozg_ctx* c, bool cplx, char ta, char tb, int64_t m, int64_t n, int64_t k, const double* alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb, const double* beta, double* C,
               int64_t ldc, int slices, ozg_report* rep, bool native) {
  // BLAS order: argument errors are reported before anything else (no device work, no context use)
  int rc = check_gemm_args(cplx, ta, tb, m, n, k, lda, ldb, ldc);
  if (rc) return rc;
  if (!native && (slices < OZG_NATIVE || slices > OZG_MAX_SLICES)) return -14;
  if (!c) return OZG_ERR_INVALID;
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->slices_used = native ? -1 : slices;
    rep->est_err = NAN;
    rep->max_real = NAN;
    rep->max_imag = NAN;
  }
  if (m == 0 || n == 0) return OZG_OK;
  const bool alpha_zero = alpha[0] == 0.0 && (!cplx || alpha[1] == 0.0);
  const bool beta_one = beta[0] == 1.0 && (!cplx || beta[1] == 0.0);
  if ((alpha_zero || k == 0) && beta_one) return OZG_OK;
  cudaSetDevice(c->device);
  if (alpha_zero || k == 0) {
    OZG_CUDA(ozg::launch_scale_c(C, m, n, ldc, beta, cplx, c->stream));
    return OZG_OK;
  }
  if (native || slices == OZG_NATIVE) {
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
    na.alpha[0] = alpha[0];
    na.alpha[1] = cplx ? alpha[1] : 0.0;
    na.beta[0] = beta[0];
    na.beta[1] = cplx ? beta[1] : 0.0;
    na.beta_zero = beta[0] == 0.0 && (!cplx || beta[1] == 0.0);
    na.cplx = cplx;
    {
      PhaseScope ps(c, OZG_PHASE_NATIVE);
      OZG_CUDA(ozg::launch_native_gemm(na, c->stream));
    }
    if (rep) rep->slices_used = -1;
    return OZG_OK;
  }
  return emu_gemm(c, cplx, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, rep, nullptr);
}

}  // namespace

extern "C" {

int ozg_create(ozg_ctx** out, size_t workspace_bytes) {
  if (!out) return OZG_ERR_INVALID;
  *out = nullptr;
  ozg_ctx* c = new ozg_ctx();
  OZG_CUDA(cudaGetDevice(&c->device));
  OZG_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  OZG_CUDA(ozg::prepare_kernels());
  if (cudaMalloc(&c->dcheck, 4 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return OZG_ERR_ALLOC;
  }
  if (cudaMalloc(&c->dflags, 4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return OZG_ERR_ALLOC;
  }
  OZG_CUDA(cudaMemset(c->dflags, 0, 4 * sizeof(int)));
  if (workspace_bytes) {
    int rc = ensure_ws(c, workspace_bytes);
    if (rc) {
      cudaFree(c->dflags);
      delete c;
      return rc;
    }
  }
  *out = c;
  return OZG_OK;
}

int ozg_destroy(ozg_ctx* c) {
  if (!c) return OZG_OK;
  cudaStreamSynchronize(c->stream);
  for (auto& mk : c->pending) {
    cudaEventDestroy(mk.a);
    cudaEventDestroy(mk.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->ws) cudaFree(c->ws);
  if (c->dflags) cudaFree(c->dflags);
  if (c->dcheck) cudaFree(c->dcheck);
  if (c->dsel) cudaFree(c->dsel);
  if (c->train) cudaFree(c->train);
  c->plan.reset();
  if (c->gws) cudaFree(c->gws);
  if (c->z3ws) cudaFree(c->z3ws);
  for (ozg_ctx* s : c->hsub) {  // host-memory batch parts
    cudaStream_t st = s->stream;
    ozg_destroy(s);
    if (st) cudaStreamDestroy(st);
  }
  for (cudaEvent_t e : c->hev) cudaEventDestroy(e);
  if (c->h2d) cudaStreamDestroy(c->h2d);
  if (c->d2h) cudaStreamDestroy(c->d2h);
  if (c->hstage) cudaFree(c->hstage);
  delete c;
  return OZG_OK;
}

int ozg_set_exact_epilogue(ozg_ctx* c, int enable) {
  if (!c) return OZG_ERR_INVALID;
  c->exact = enable != 0;
  return OZG_OK;
}

int ozg_set_check_samples(ozg_ctx* c, int samples) {
  if (!c) return OZG_ERR_INVALID;
  if (samples < 0 || samples > (1 << 20)) return -2;
  c->check_samples = samples;
  return OZG_OK;
}

int ozg_set_stream(ozg_ctx* c, void* stream) {
  if (!c) return OZG_ERR_INVALID;
  c->stream = static_cast<cudaStream_t>(stream);
  return OZG_OK;
}

int ozg_sync(ozg_ctx* c) {
  if (!c) return OZG_ERR_INVALID;
  OZG_CUDA(cudaStreamSynchronize(c->stream));
  int h = 0;
  OZG_CUDA(cudaMemcpy(&h, c->dflags, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) OZG_CUDA(cudaMemset(c->dflags, 0, sizeof(int)));
  return h ? (h == 3 ? OZG_ERR_TIMEOUT : OZG_ERR_CUDA) : OZG_OK;
}

const char* ozg_strerror(int code) {
  if (code < 0) return "invalid argument (BLAS argument position = -code)";
  switch (code) {
    case OZG_OK: return "success";
    case OZG_ERR_CUDA: return "CUDA runtime error";
    case OZG_ERR_ALLOC: return "device workspace allocation failed";
    case OZG_ERR_TIMEOUT: return "a bounded device-side wait expired";
    case OZG_ERR_UNSUPPORTED: return "unsupported request";
    case OZG_ERR_INVALID: return "invalid context or argument";
    default: return "unknown error";
  }
}

const char* ozg_last_cuda_error(void) { return ozg::host::last_cuda_error_text(); }

int ozg_set_profiling(ozg_ctx* c, int enable) {
  if (!c) return OZG_ERR_INVALID;
  c->prof = enable != 0;
  return OZG_OK;
}

int ozg_phase_times(ozg_ctx* c, double* ms, int64_t* counts) {
  if (!c) return OZG_ERR_INVALID;
  OZG_CUDA(cudaStreamSynchronize(c->stream));
  for (auto& mk : c->pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, mk.a, mk.b) == cudaSuccess) {
      c->acc_ms[mk.phase] += t;
      c->acc_n[mk.phase] += 1;
    } else {
      cudaGetLastError();
    }
    c->pool.push_back(mk.a);
    c->pool.push_back(mk.b);
  }
  c->pending.clear();
  for (int i = 0; i < OZG_NUM_PHASES; ++i) {
    if (ms) ms[i] = c->acc_ms[i];
    if (counts) counts[i] = c->acc_n[i];
    c->acc_ms[i] = 0.0;
    c->acc_n[i] = 0;
  }
  return OZG_OK;
}

int ozg_dgemm(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
              const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
              int slices, ozg_report* rep) {
  double al[2] = {alpha, 0.0}, be[2] = {beta, 0.0};
  return gemm_entry(ctx, false, transa, transb, m, n, k, al, A, lda, B, ldb, be, C, ldc, slices, rep, false);
}

int ozg_zgemm(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k, const double* alpha,
              const double* A, int64_t lda, const double* B, int64_t ldb, const double* beta, double* C,
              int64_t ldc, int slices, ozg_report* rep) {
  if (!alpha || !beta) return OZG_ERR_INVALID;
  return gemm_entry(ctx, true, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, rep, false);
}

int ozg_native_dgemm(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                     int64_t ldc) {
  double al[2] = {alpha, 0.0}, be[2] = {beta, 0.0};
  return gemm_entry(ctx, false, transa, transb, m, n, k, al, A, lda, B, ldb, be, C, ldc, OZG_NATIVE, nullptr, true);
}

int ozg_native_zgemm(ozg_ctx* ctx, char transa, char transb, int64_t m, int64_t n, int64_t k, const double* alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, const double* beta, double* C,
                     int64_t ldc) {
  if (!alpha || !beta) return OZG_ERR_INVALID;
  return gemm_entry(ctx, true, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, OZG_NATIVE, nullptr,
                    true);
}

static int debug_split_impl(ozg_ctx* c, bool cplx, char trans, int64_t rows, int64_t k, const double* X, int64_t ld,
                            int s, int32_t* e_out, int8_t* digits_out) {
  if (!c) return OZG_ERR_INVALID;
  trans = norm_trans(trans);
  if (!cplx && trans == 'C') trans = 'T';
  if (trans != 'N' && trans != 'T' && trans != 'C') return -1;
  if (rows < 0) return -2;
  if (k <= 0) return -3;
  int64_t nrow = (trans == 'N') ? rows : k;
  if (ld < (nrow > 1 ? nrow : 1)) return -5;
  if (s < 1 || s > OZG_MAX_SLICES) return -6;
  if (rows == 0) return OZG_OK;
  cudaSetDevice(c->device);
  const int64_t Kp = (int64_t)align_up((size_t)k, 8);
  const int64_t pr = cplx ? 2 * rows : rows;
  Carve cv;
  size_t oD = cv.take((size_t)s * pr * Kp * 2), oM = cv.take(8 * (size_t)rows), oE = cv.take(4 * (size_t)rows);
  int rc = ensure_ws(c, cv.off);
  if (rc) return rc;
  ozg::SplitArgs sa;
  sa.X = X;
  sa.ld = ld;
  sa.rows = rows;
  sa.k = k;
  sa.strided = (trans == 'N');
  sa.conj = (trans == 'C');
  sa.cplx = cplx;
  sa.s = s;
  sa.Kp = Kp;
  sa.plane_rows = pr;
  sa.D = at<__half>(c, oD);
  sa.maxbits = at<unsigned long long>(c, oM);
  sa.exps = at<int32_t>(c, oE);
  sa.nonfinite = c->dflags + 1;
  OZG_CUDA(ozg::launch_split(sa, c->stream));
  OZG_CUDA(ozg::launch_digits_to_i8(sa.D, s, pr, k, Kp, digits_out, c->stream));
  OZG_CUDA(cudaMemcpyAsync(e_out, sa.exps, 4 * (size_t)rows, cudaMemcpyDeviceToDevice, c->stream));
  OZG_CUDA(cudaStreamSynchronize(c->stream));
  return OZG_OK;
}

int ozg_debug_split(ozg_ctx* ctx, char trans, int64_t rows, int64_t k, const double* X, int64_t ld, int slices,
                    int32_t* e_out, int8_t* digits_out) {
  return debug_split_impl(ctx, false, trans, rows, k, X, ld, slices, e_out, digits_out);
}

int ozg_debug_zsplit(ozg_ctx* ctx, char trans, int64_t rows, int64_t k, const double* X, int64_t ld, int slices,
                     int32_t* e_out, int8_t* digits_out) {
  return debug_split_impl(ctx, true, trans, rows, k, X, ld, slices, e_out, digits_out);
}

int ozg_debug_group_products(ozg_ctx* c, char transa, char transb, int64_t m, int64_t n, int64_t k,
                             const double* A, int64_t lda, const double* B, int64_t ldb, int slices,
                             int64_t* G_out) {
  if (!c) return OZG_ERR_INVALID;
  int rc = check_gemm_args(false, transa, transb, m, n, k, lda, ldb, m > 0 ? m : 1);
  if (rc) return rc;
  if (slices < 1 || slices > OZG_MAX_SLICES) return -14;
  if (m == 0 || n == 0 || k == 0) return OZG_OK;
  // the export sums the int32 pushes of a group in int64: |G_g| <= s k 127^2 fits for any k
  // that fits in memory
  cudaSetDevice(c->device);
  double one[2] = {1.0, 0.0}, zero[2] = {0.0, 0.0};
  rc = emu_gemm(c, false, transa, transb, m, n, k, one, A, lda, B, ldb, zero, nullptr, m, slices, nullptr, G_out);
  if (rc) return rc;
  OZG_CUDA(cudaStreamSynchronize(c->stream));
  return ozg_sync(c);
}

}  // extern "C"
