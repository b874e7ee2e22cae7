// ozg_dgemm_grouped: many independent, uneven emulated DGEMMs with per-call slice counts in a
// fixed, short launch sequence (batched split, one persistent grouped slice-GEMM launch, batched
// native fallback, batched error check), captured once into a CUDA graph and replayed while the
// same batch (pointers, shapes, slice counts) is submitted again.
//
// Load balance: the tiles of all calls are sorted by cost (slice pairs x k-blocks) and assigned
// longest-first to the least-loaded CTA; the persistent kernel's CTA b then walks slots
// b, b + grid, ... of the interleaved list (empty slots are skipped).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <vector>

#include "ozg_context.h"

namespace ozg {
namespace host {

struct GroupPlan {
  uint64_t key = 0, epoch = 0;
  int ncalls = 0, nsamp = 0, variant = 0, grid = 0, njobs = 0, ntiles = 0;
  long long nkernels = 0;  // kernels one replay of the captured graph launches
  int64_t rowmax_units = 0, digit_units = 0, stats_units = 0;
  cudaGraphExec_t exec = nullptr;
  size_t oFlags = 0, flags_bytes = 0, oMax = 0, max_bytes = 0;
  size_t oJobs = 0, oRmTab = 0, oDgTab = 0, oStTab = 0, oCalls = 0, oTiles = 0, oNative = 0, oFlagPtrs = 0;
  size_t oNList = 0, oNPre = 0, oNTot = 0, oChecks = 0, oErrs = 0, oCold = 0, oR = 0;
  std::vector<int> s_used;
  // automatic (selector) calls
  int any_auto = 0, s_fb = 0;
  int64_t save_units = 0;
  size_t oHist = 0, hist_bytes = 0, oSel = 0, oSused = 0, oRep = 0, oSavePre = 0, oSaved = 0;
  // escalation stages 2 (min(s + 2, fallback)) and 3 (the fallback) of rejected learned calls
  size_t oCalls2 = 0, oChecks2 = 0, oErrs2 = 0, oSkip2 = 0, oJobs2 = 0, oCounter = 0;
  size_t oCalls3 = 0, oChecks3 = 0, oErrs3 = 0, oSkip3 = 0, oJobs3 = 0, oRep2 = 0, oS2 = 0;
  // gated digit passes: per-job starts in the digit unit table, and the device-built job list
  size_t oDgStart = 0, oDgList = 0, oDgPre = 0, oDgTot = 0;
  std::vector<char> autom;
};

void destroy_plan(GroupPlan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  delete p;
}

namespace {

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

int tile_n_of(int variant) { return slice_gemm_tile_n_of(variant); }

// All tiles in decreasing estimated cost (tiles of one call stay together, so tiles that share
// digit panels run at about the same time).  The kernel hands them out dynamically -- each CTA
// claims the next tile when it starts one -- so the order gives the longest-first balance and
// costs that are only known on the device (selected slice counts) cannot unbalance the launch.
std::vector<GroupTile> ordered_tiles(const ozg_gemm_desc* d, const std::vector<int>& s, int64_t count, int variant) {
  struct T {
    double cost;
    GroupTile t;
  };
  const int BN = tile_n_of(variant), BMv = slice_gemm_tile_m_of(variant);
  std::vector<T> all;
  for (int64_t c = 0; c < count; ++c) {
    const int64_t tm = (d[c].m + BMv - 1) / BMv, tn = (d[c].n + BN - 1) / BN;
    // per tile, the same for all tiles of a call (they stay together): slice products x k
    // (in 16-wide steps) plus the epilogue's per-group work, times the call's mean valid tile
    // width (16-column steps) -- an estimate that orders measurably better than the padded width
    const double kb = (double)((d[c].k + 15) / 16) / 4.0;
    const double w = (double)((d[c].n + 15) / 16 * 16) / (double)tn;
    const double cost = ((double)(s[c] * (s[c] + 1) / 2) * kb + 2 * s[c]) * w;
    for (int64_t i = 0; i < tm; ++i)
      for (int64_t j = 0; j < tn; ++j) all.push_back({cost, {(int)c, (int)i, (int)j, 0}});
  }
  std::stable_sort(all.begin(), all.end(), [](const T& a, const T& b) { return a.cost > b.cost; });
  std::vector<GroupTile> out;
  out.reserve(all.size());
  for (const T& x : all) out.push_back(x.t);
  return out;
}

int enqueue(ozg_ctx* c, const GroupPlan& P) {
  cudaStream_t st = c->stream;
  OZG_CUDA(cudaMemsetAsync(gat<char>(c, P.oFlags), 0, P.flags_bytes, st));
  OZG_CUDA(cudaMemsetAsync(gat<char>(c, P.oMax), 0, P.max_bytes, st));
  // [0]: tile counter of the main launch; [1], [2]: tile counter and "some call is re-run" of
  // escalation stage 2; [3], [4]: the same for stage 3
  OZG_CUDA(cudaMemsetAsync(gat<char>(c, P.oCounter), 0, sizeof(int) * 5, st));
  // row maxima (and, for learned calls, the selector's features in the same read): jobs whose
  // whole rows fit a fused statistics unit take one pass; longer ones the two-pass units
  if (P.any_auto) OZG_CUDA(cudaMemsetAsync(gat<char>(c, P.oHist), 0, P.hist_bytes, st));
  OZG_CUDA(launch_stats_batched(gat<SplitArgs>(c, P.oJobs), gat<int2>(c, P.oStTab), P.stats_units, P.any_auto, st));
  OZG_CUDA(launch_rowmax_batched(gat<SplitArgs>(c, P.oJobs), gat<int2>(c, P.oRmTab), P.rowmax_units, st));
  if (!P.any_auto) {
    OZG_CUDA(launch_digits_batched(gat<SplitArgs>(c, P.oJobs), gat<int2>(c, P.oDgTab), P.digit_units, nullptr, 0,
                                   st));
  } else {
    // features -> selection -> digits up to each call's selected count
    if (P.rowmax_units > 0)
      OZG_CUDA(launch_gap_hist_batched(gat<SplitArgs>(c, P.oJobs), gat<int2>(c, P.oRmTab), P.rowmax_units, st));
    OZG_CUDA(launch_select_batched(c->dsel, gat<SelectJob>(c, P.oSel), P.ncalls, (float)std::log10(c->target), st));
    OZG_CUDA(launch_digits_batched(gat<SplitArgs>(c, P.oJobs), gat<int2>(c, P.oDgTab), P.digit_units, nullptr, 0,
                                   st));
    OZG_CUDA(launch_save_restore_batched(gat<RepairJob>(c, P.oRep), gat<int64_t>(c, P.oSavePre), P.save_units,
                                         P.ncalls, 0, st));
  }
  if (P.nsamp > 0) OZG_CUDA(launch_check_batched_pre(gat<CheckArgs>(c, P.oChecks), P.ncalls, P.nsamp, st));
  GroupArgs g;
  g.tiles = gat<GroupTile>(c, P.oTiles);
  g.ntiles = P.ntiles;
  g.calls = gat<GroupCall>(c, P.oCalls);
  g.status = c->dflags;
  g.Rws = gat<double>(c, P.oR);
  g.defer = variant_defers(P.variant);
  g.tile_counter = gat<int>(c, P.oCounter);
  {
    PhaseScope ps(c, OZG_PHASE_GEMM);
    OZG_CUDA(launch_slice_gemm_grouped(g, P.variant, P.grid, st));
  }
  OZG_CUDA(launch_native_batched(gat<NativeArgs>(c, P.oNative), P.ncalls, gat<const int*>(c, P.oFlagPtrs),
                                 gat<int>(c, P.oNList), gat<int64_t>(c, P.oNPre), gat<int64_t>(c, P.oNTot),
                                 2 * c->num_sms, st));
  if (P.nsamp > 0)
    OZG_CUDA(launch_check_batched_post(gat<CheckArgs>(c, P.oChecks), P.ncalls, P.nsamp, gat<double>(c, P.oErrs), st));
  if (P.any_auto) {
    // the check judges the selector: a rejected call is re-run at min(s + 2, fallback) (stage 2),
    // and one rejected again at the fallback count (stage 3).  Each stage's launches are gated on
    // a device flag, so they return at once when no call needs them.
    struct Stage {
      size_t rep, jobs, calls, checks, errs;
      int ctr;
    };
    const Stage stages[2] = {{P.oRep, P.oJobs2, P.oCalls2, P.oChecks2, P.oErrs2, 1},
                             {P.oRep2, P.oJobs3, P.oCalls3, P.oChecks3, P.oErrs3, 3}};
    int* ctr = gat<int>(c, P.oCounter);
    for (const Stage& S : stages) {
      OZG_CUDA(launch_repair_prep_batched(gat<RepairJob>(c, S.rep), P.ncalls, c->target, ctr + S.ctr + 1, st));
      OZG_CUDA(launch_save_restore_batched(gat<RepairJob>(c, S.rep), gat<int64_t>(c, P.oSavePre), P.save_units,
                                           P.ncalls, 1, st));
      OZG_CUDA(launch_digits_gated(gat<SplitArgs>(c, S.jobs), P.njobs, gat<int64_t>(c, P.oDgStart), ctr + S.ctr + 1,
                                   gat<int>(c, P.oDgList), gat<int64_t>(c, P.oDgPre), gat<int64_t>(c, P.oDgTot),
                                   8 * c->num_sms, st));
      GroupArgs gs = g;
      gs.calls = gat<GroupCall>(c, S.calls);
      gs.tile_counter = ctr + S.ctr;
      gs.run = ctr + S.ctr + 1;
      {
        PhaseScope ps(c, OZG_PHASE_GEMM);
        OZG_CUDA(launch_slice_gemm_grouped(gs, P.variant, P.grid, st));
      }
      OZG_CUDA(launch_check_batched_post(gat<CheckArgs>(c, S.checks), P.ncalls, P.nsamp, gat<double>(c, S.errs),
                                         st));
    }
  }
  return OZG_OK;
}

int check_desc(const ozg_gemm_desc& d, char& ta, char& tb) {
  ta = norm_trans(d.transa);
  tb = norm_trans(d.transb);
  if (ta == 'C') ta = 'T';
  if (tb == 'C') tb = 'T';
  if (ta != 'N' && ta != 'T') return -1;
  if (tb != 'N' && tb != 'T') return -2;
  if (d.m < 0) return -3;
  if (d.n < 0) return -4;
  if (d.k < 0) return -5;
  const int64_t nrowa = (ta == 'N') ? d.m : d.k, nrowb = (tb == 'N') ? d.k : d.n;
  if (d.lda < (nrowa > 1 ? nrowa : 1)) return -8;
  if (d.ldb < (nrowb > 1 ? nrowb : 1)) return -10;
  if (d.ldc < (d.m > 1 ? d.m : 1)) return -13;
  return 0;
}

// Build (upload) the plan's tables for `variant` into the grouped workspace.
int build_plan(ozg_ctx* c, int64_t count, const ozg_gemm_desc* d, const std::vector<int>& s,
               const std::vector<char>& TA, const std::vector<char>& TB, const std::vector<char>& autom, int variant,
               GroupPlan* P) {
  // s[i]: slice count of fixed calls; for automatic calls the fallback count (a cost estimate
  // and the re-run count), while their digit planes are written for the selector's top class
  int any_auto = 0;
  for (int64_t i = 0; i < count; ++i) any_auto |= autom[i];
  const int s_hi = std::max(c->sel_s_hi, c->fallback_slices);
  std::vector<int> planes(count);
  for (int64_t i = 0; i < count; ++i) planes[i] = autom[i] ? s_hi : s[i];
  const int nsamp = any_auto ? std::max(c->check_samples, 64) : c->check_samples;
  P->any_auto = any_auto;
  P->autom = autom;
  P->s_fb = c->fallback_slices;
  P->ncalls = (int)count;
  P->nsamp = nsamp;
  P->variant = variant;
  P->s_used = s;
  int64_t total_tiles = 0;
  const int BN = tile_n_of(variant), BMv = slice_gemm_tile_m_of(variant);
  for (int64_t i = 0; i < count; ++i) total_tiles += ((d[i].m + BMv - 1) / BMv) * ((d[i].n + BN - 1) / BN);
  if (variant == kPairVariant)  // whole 2-CTA clusters, as many as can be resident, one per pair tile
    P->grid = (int)(2 * std::max<int64_t>(1, std::min<int64_t>(pair_max_ctas() / 2, total_tiles)));
  else
    P->grid = (int)std::max<int64_t>(1, std::min<int64_t>(c->num_sms, total_tiles));
  std::vector<GroupTile> tiles = ordered_tiles(d, s, count, variant);
  P->ntiles = (int)tiles.size();

  Carve cv;
  P->oFlags = cv.take(sizeof(int) * count);
  P->flags_bytes = sizeof(int) * count;
  std::vector<size_t> oMA(count), oMB(count), oEA(count), oEB(count), oDA(count), oDB(count);
  size_t max0 = cv.off;
  for (int64_t i = 0; i < count; ++i) {
    oMA[i] = cv.take(8 * (size_t)d[i].m);
    oMB[i] = cv.take(8 * (size_t)d[i].n);
  }
  P->oMax = max0;
  P->max_bytes = cv.off - max0;
  for (int64_t i = 0; i < count; ++i) {
    const int64_t Kp = (d[i].k + 7) / 8 * 8;
    oEA[i] = cv.take(4 * (size_t)d[i].m);
    oEB[i] = cv.take(4 * (size_t)d[i].n);
    oDA[i] = cv.take((size_t)planes[i] * d[i].m * Kp * 2);
    oDB[i] = cv.take((size_t)planes[i] * d[i].n * Kp * 2);
  }
  P->njobs = (int)(2 * count);
  P->oJobs = cv.take(sizeof(SplitArgs) * 2 * count);
  // work-unit tables of the batched split (job j = 2i for A, 2i + 1 for B of call i): fused
  // statistics units for jobs whose rows fit one, two-pass row-maximum units for the others
  std::vector<int2> rmtab, dgtab, sttab;
  std::vector<int64_t> dgstart(2 * count + 1, 0);  // job j's digit units: [dgstart[j], dgstart[j + 1])
  for (int64_t i = 0; i < count; ++i)
    for (int side = 0; side < 2; ++side) {
      SplitArgs x;
      x.rows = side ? d[i].n : d[i].m;
      x.k = d[i].k;
      x.strided = side ? (TB[i] == 'T') : (TA[i] == 'N');
      const int job = (int)(2 * i + side);
      if (stats_fused(x)) {
        for (int64_t u = 0, nu = stats_units_of(x); u < nu; ++u) sttab.push_back(make_int2(job, (int)u));
      } else {
        for (int64_t u = 0, nu = rowmax_units_of(x); u < nu; ++u) rmtab.push_back(make_int2(job, (int)u));
      }
      for (int64_t u = 0, nu = digit_units_of(x); u < nu; ++u) dgtab.push_back(make_int2(job, (int)u));
      dgstart[job + 1] = (int64_t)dgtab.size();
    }
  P->oRmTab = cv.take(sizeof(int2) * std::max<size_t>(rmtab.size(), 1));
  P->oDgTab = cv.take(sizeof(int2) * std::max<size_t>(dgtab.size(), 1));
  P->oStTab = cv.take(sizeof(int2) * std::max<size_t>(sttab.size(), 1));
  P->oCalls = cv.take(sizeof(GroupCall) * count + 64);
  P->oTiles = cv.take(sizeof(GroupTile) * tiles.size());
  P->oNative = cv.take(sizeof(NativeArgs) * count);
  P->oFlagPtrs = cv.take(sizeof(int*) * count);
  P->oNList = cv.take(sizeof(int) * count);
  P->oNPre = cv.take(sizeof(int64_t) * (count + 1));
  P->oNTot = cv.take(sizeof(int64_t) * 2);
  P->oChecks = cv.take(sizeof(CheckArgs) * count);
  P->oErrs = cv.take(sizeof(double) * count);
  P->oCold = cv.take(sizeof(double) * 2 * (size_t)std::max(nsamp, 1) * count);
  P->oR = cv.take((size_t)P->grid * 128 * 256 * 16);
  P->oCounter = cv.take(sizeof(int) * 5);  // tile counters and re-run flags of the stages
  std::vector<int64_t> sp(count + 1, 0);
  std::vector<size_t> oSv(count, 0);
  if (any_auto) {
    P->oHist = cv.take(sizeof(unsigned long long) * 20 * count);
    P->hist_bytes = sizeof(unsigned long long) * 20 * count;
    P->oSel = cv.take(sizeof(SelectJob) * count);
    P->oSused = cv.take(sizeof(int) * count);
    P->oRep = cv.take(sizeof(RepairJob) * count);
    P->oSavePre = cv.take(sizeof(int64_t) * (count + 1));
    P->oCalls2 = cv.take(sizeof(GroupCall) * count + 64);
    P->oChecks2 = cv.take(sizeof(CheckArgs) * count);
    P->oErrs2 = cv.take(sizeof(double) * count);
    P->oSkip2 = cv.take(sizeof(int) * count);
    P->oJobs2 = cv.take(sizeof(SplitArgs) * 2 * count);
    P->oCalls3 = cv.take(sizeof(GroupCall) * count + 64);
    P->oChecks3 = cv.take(sizeof(CheckArgs) * count);
    P->oErrs3 = cv.take(sizeof(double) * count);
    P->oSkip3 = cv.take(sizeof(int) * count);
    P->oJobs3 = cv.take(sizeof(SplitArgs) * 2 * count);
    P->oRep2 = cv.take(sizeof(RepairJob) * count);
    P->oS2 = cv.take(sizeof(int) * count);
    P->oDgStart = cv.take(sizeof(int64_t) * (2 * count + 1));
    P->oDgList = cv.take(sizeof(int) * 2 * count);
    P->oDgPre = cv.take(sizeof(int64_t) * (2 * count + 1));
    P->oDgTot = cv.take(sizeof(int64_t) * 2);
    for (int64_t i = 0; i < count; ++i) {
      const bool sv = autom[i] && d[i].beta != 0.0;
      sp[i + 1] = sp[i] + (sv ? (d[i].m * d[i].n + 255) / 256 : 0);
      if (sv) oSv[i] = cv.take(sizeof(double) * d[i].m * d[i].n);
    }
    P->save_units = sp[count];
  }
  int rc = ensure_gws(c, cv.off);
  if (rc) return rc;
  P->epoch = c->gws_epoch;

  std::vector<SplitArgs> jobs(2 * count);
  std::vector<GroupCall> calls(count);
  std::vector<NativeArgs> nat(count);
  std::vector<const int*> fptr(count);
  std::vector<CheckArgs> chk(count);
  int* flags = gat<int>(c, P->oFlags);
  for (int64_t i = 0; i < count; ++i) {
    const int64_t Kp = (d[i].k + 7) / 8 * 8;
    SplitArgs a;
    a.X = d[i].A;
    a.ld = d[i].lda;
    a.rows = d[i].m;
    a.k = d[i].k;
    a.strided = (TA[i] == 'N');
    a.s = planes[i];
    a.Kp = Kp;
    a.plane_rows = d[i].m;
    a.D = gat<__half>(c, oDA[i]);
    a.maxbits = gat<unsigned long long>(c, oMA[i]);
    a.exps = gat<int32_t>(c, oEA[i]);
    a.nonfinite = flags + i;
    a.hist = autom[i] ? gat<unsigned long long>(c, P->oHist) + 20 * i : nullptr;
    SplitArgs b = a;
    b.X = d[i].B;
    b.ld = d[i].ldb;
    b.rows = d[i].n;
    b.strided = (TB[i] == 'T');
    b.plane_rows = d[i].n;
    b.D = gat<__half>(c, oDB[i]);
    b.maxbits = gat<unsigned long long>(c, oMB[i]);
    b.exps = gat<int32_t>(c, oEB[i]);
    b.hist = autom[i] ? gat<unsigned long long>(c, P->oHist) + 20 * i + 10 : nullptr;
    if (autom[i]) {  // digits only up to the count the selector writes into the call's slot
      const int* sel = &gat<GroupCall>(c, P->oCalls)[i].s;
      a.plane_to = sel;
      b.plane_to = sel;
    }
    jobs[2 * i] = a;
    jobs[2 * i + 1] = b;

    GroupCall& g = calls[i];
    OZG_CUDA(make_digit_tmap(&g.tmA, a.D, d[i].k, d[i].m, Kp, planes[i], 128));
    OZG_CUDA(make_digit_tmap(&g.tmB, b.D, d[i].k, d[i].n, Kp, planes[i], BN));
    OZG_CUDA(make_digit_tmap(&g.tmBh, b.D, d[i].k, d[i].n, Kp, planes[i], BN / 2));
    g.rows = d[i].m;
    g.cols = d[i].n;
    g.m = d[i].m;
    g.n = d[i].n;
    g.k = d[i].k;
    g.s = s[i];
    g.cplx = 0;
    g.beta_zero = d[i].beta == 0.0;
    g.e = a.exps;
    g.f = b.exps;
    g.C = d[i].C;
    g.ldc = d[i].ldc;
    g.alpha[0] = d[i].alpha;
    g.beta[0] = d[i].beta;
    g.nonfinite = flags + i;

    NativeArgs& na = nat[i];
    na.ta = TA[i];
    na.tb = TB[i];
    na.m = d[i].m;
    na.n = d[i].n;
    na.k = d[i].k;
    na.A = d[i].A;
    na.lda = d[i].lda;
    na.B = d[i].B;
    na.ldb = d[i].ldb;
    na.C = d[i].C;
    na.ldc = d[i].ldc;
    na.alpha[0] = d[i].alpha;
    na.beta[0] = d[i].beta;
    na.beta_zero = d[i].beta == 0.0;
    fptr[i] = flags + i;

    CheckArgs& ck = chk[i];
    ck.ta = TA[i];
    ck.tb = TB[i];
    ck.m = d[i].m;
    ck.n = d[i].n;
    ck.k = d[i].k;
    ck.A = d[i].A;
    ck.lda = d[i].lda;
    ck.B = d[i].B;
    ck.ldb = d[i].ldb;
    ck.C = d[i].C;
    ck.ldc = d[i].ldc;
    ck.alpha[0] = d[i].alpha;
    ck.beta[0] = d[i].beta;
    ck.beta_zero = d[i].beta == 0.0;
    ck.nsamp = nsamp;
    ck.seed = c->check_seed + (uint64_t)i * 0x9E3779B9ull;
    ck.cold = gat<double>(c, P->oCold) + 2 * (size_t)std::max(nsamp, 1) * i;
    ck.err_out = gat<double>(c, P->oErrs) + i;
    ck.gate = flags + i;
    ck.ea = gat<int32_t>(c, oEA[i]);  // the split's exponents: exact integer reference
    ck.fb = gat<int32_t>(c, oEB[i]);
  }
  c->check_seed += 1;
  std::vector<SelectJob> sel;
  std::vector<RepairJob> rep, rep2;
  std::vector<GroupCall> calls2, calls3;
  std::vector<CheckArgs> chk2, chk3;
  if (any_auto) {
    sel.resize(count);
    rep.resize(count);
    calls2 = calls;
    calls3 = calls;
    chk2 = chk;
    chk3 = chk;
    GroupCall* calls_dev = gat<GroupCall>(c, P->oCalls);
    GroupCall* calls2_dev = gat<GroupCall>(c, P->oCalls2);
    GroupCall* calls3_dev = gat<GroupCall>(c, P->oCalls3);
    for (int64_t i = 0; i < count; ++i) {
      SelectJob& J = sel[i];
      J.histA = gat<unsigned long long>(c, P->oHist) + 20 * i;
      J.histB = J.histA + 10;
      J.m = d[i].m;
      J.n = d[i].n;
      J.k = d[i].k;
      J.s_out1 = &calls_dev[i].s;  // the grouped kernel reads the call's slice count here
      J.s_out2 = gat<int>(c, P->oSused) + i;
      J.s_cap = planes[i];
      J.active = autom[i];
      // stage 1 -> 2: the selected count, then min(selected + 2, fallback)
      RepairJob& R = rep[i];
      R.auto_mode = autom[i];
      R.beta_nz = d[i].beta != 0.0;
      R.err = gat<double>(c, P->oErrs) + i;
      R.ran = nullptr;
      R.s_cur = &calls_dev[i].s;
      R.s_next = &calls2_dev[i].s;
      R.s_copy = gat<int>(c, P->oS2) + i;
      R.s_add = 2;
      R.s_fb = std::min(s[i], planes[i]);
      R.skip_next = gat<int>(c, P->oSkip2) + i;
      R.nonfinite = flags + i;
      R.C = d[i].C;
      R.saved = (autom[i] && d[i].beta != 0.0) ? gat<double>(c, oSv[i]) : nullptr;
      R.m = d[i].m;
      R.n = d[i].n;
      R.ldc = d[i].ldc;
      // stage 2 -> 3: the fallback count
      RepairJob R2 = R;
      R2.err = gat<double>(c, P->oErrs2) + i;
      R2.ran = R.skip_next;
      R2.s_cur = &calls2_dev[i].s;
      R2.s_next = &calls3_dev[i].s;
      R2.s_copy = nullptr;
      R2.s_add = 0;
      R2.skip_next = gat<int>(c, P->oSkip3) + i;
      rep2.push_back(R2);
      calls2[i].s = R.s_fb;  // rewritten on the device for the calls that are re-run
      calls2[i].nonfinite = R.skip_next;  // a stage's launch skips every call it does not re-run
      calls3[i].s = R.s_fb;
      calls3[i].nonfinite = R2.skip_next;
      chk2[i].err_out = gat<double>(c, P->oErrs2) + i;
      chk2[i].gate = R.skip_next;
      chk3[i].err_out = gat<double>(c, P->oErrs3) + i;
      chk3[i].gate = R2.skip_next;
    }
  }
  P->rowmax_units = (int64_t)rmtab.size();
  P->digit_units = (int64_t)dgtab.size();
  P->stats_units = (int64_t)sttab.size();
  cudaStream_t st = c->stream;
  OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oJobs), jobs.data(), sizeof(SplitArgs) * jobs.size(), cudaMemcpyHostToDevice, st));
  std::vector<SplitArgs> jobs2, jobs3;
  if (any_auto) {
    // completion of the digit planes for calls the check rejects: planes (s1, s2] for stage 2
    // and (s2, fallback] for stage 3
    jobs2 = jobs;
    jobs3 = jobs;
    for (int64_t i = 0; i < count; ++i)
      for (int side = 0; side < 2; ++side) {
        SplitArgs& x = jobs2[2 * i + side];
        x.plane_from = &gat<GroupCall>(c, P->oCalls)[i].s;
        x.plane_to = &gat<GroupCall>(c, P->oCalls2)[i].s;
        x.gate = gat<int>(c, P->oSkip2) + i;  // 1 unless the call is re-run
        x.hist = nullptr;
        SplitArgs& y = jobs3[2 * i + side];
        y.plane_from = &gat<GroupCall>(c, P->oCalls2)[i].s;
        y.plane_to = &gat<GroupCall>(c, P->oCalls3)[i].s;
        y.gate = gat<int>(c, P->oSkip3) + i;
        y.hist = nullptr;
      }
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oJobs2), jobs2.data(), sizeof(SplitArgs) * jobs2.size(),
                             cudaMemcpyHostToDevice, st));
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oJobs3), jobs3.data(), sizeof(SplitArgs) * jobs3.size(),
                             cudaMemcpyHostToDevice, st));
  }
  if (!rmtab.empty())
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oRmTab), rmtab.data(), sizeof(int2) * rmtab.size(), cudaMemcpyHostToDevice,
                             st));
  if (!dgtab.empty())
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oDgTab), dgtab.data(), sizeof(int2) * dgtab.size(), cudaMemcpyHostToDevice,
                             st));
  if (!sttab.empty())
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oStTab), sttab.data(), sizeof(int2) * sttab.size(), cudaMemcpyHostToDevice,
                             st));
  OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oCalls), calls.data(), sizeof(GroupCall) * calls.size(), cudaMemcpyHostToDevice, st));
  OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oTiles), tiles.data(), sizeof(GroupTile) * tiles.size(), cudaMemcpyHostToDevice, st));
  OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oNative), nat.data(), sizeof(NativeArgs) * nat.size(), cudaMemcpyHostToDevice, st));
  OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oFlagPtrs), fptr.data(), sizeof(int*) * fptr.size(), cudaMemcpyHostToDevice, st));
  OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oChecks), chk.data(), sizeof(CheckArgs) * chk.size(), cudaMemcpyHostToDevice, st));
  if (any_auto) {
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oSel), sel.data(), sizeof(SelectJob) * count, cudaMemcpyHostToDevice, st));
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oRep), rep.data(), sizeof(RepairJob) * count, cudaMemcpyHostToDevice, st));
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oSavePre), sp.data(), sizeof(int64_t) * (count + 1),
                             cudaMemcpyHostToDevice, st));
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oCalls2), calls2.data(), sizeof(GroupCall) * count,
                             cudaMemcpyHostToDevice, st));
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oChecks2), chk2.data(), sizeof(CheckArgs) * count,
                             cudaMemcpyHostToDevice, st));
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oRep2), rep2.data(), sizeof(RepairJob) * count, cudaMemcpyHostToDevice,
                             st));
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oDgStart), dgstart.data(), sizeof(int64_t) * dgstart.size(),
                             cudaMemcpyHostToDevice, st));
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oCalls3), calls3.data(), sizeof(GroupCall) * count,
                             cudaMemcpyHostToDevice, st));
    OZG_CUDA(cudaMemcpyAsync(gat<void>(c, P->oChecks3), chk3.data(), sizeof(CheckArgs) * count,
                             cudaMemcpyHostToDevice, st));
  }
  OZG_CUDA(cudaStreamSynchronize(st));  // host tables are stack-owned
  return OZG_OK;
}

}  // namespace
}  // namespace host
}  // namespace ozg

using namespace ozg::host;

namespace ozg {
namespace host {
namespace {

// Per-call reports of the context's current plan: read the flags, selections, escalation skips
// and sampled errors back from the device (synchronises the stream).
int read_reports(ozg_ctx* c, int64_t n, const std::vector<int>& widx, const std::vector<int>& ws,
                 const std::vector<char>& wauto, ozg_report* reps) {
  GroupPlan* P = c->plan.get();
  std::vector<int> fl(n), su(n, 0), sk2(n, 1), sk3(n, 1), s2(n, 0);
  std::vector<double> er(n, NAN), er2(n, NAN), er3(n, NAN);
  cudaStream_t st = c->stream;
  OZG_CUDA(cudaMemcpyAsync(fl.data(), gat<int>(c, P->oFlags), sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  if (P->nsamp > 0)
    OZG_CUDA(cudaMemcpyAsync(er.data(), gat<double>(c, P->oErrs), sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  if (P->any_auto) {
    OZG_CUDA(cudaMemcpyAsync(su.data(), gat<int>(c, P->oSused), sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    OZG_CUDA(cudaMemcpyAsync(sk2.data(), gat<int>(c, P->oSkip2), sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    OZG_CUDA(cudaMemcpyAsync(sk3.data(), gat<int>(c, P->oSkip3), sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    OZG_CUDA(cudaMemcpyAsync(s2.data(), gat<int>(c, P->oS2), sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    OZG_CUDA(cudaMemcpyAsync(er2.data(), gat<double>(c, P->oErrs2), sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    OZG_CUDA(cudaMemcpyAsync(er3.data(), gat<double>(c, P->oErrs3), sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  }
  OZG_CUDA(cudaStreamSynchronize(st));
  for (int64_t i = 0; i < n; ++i) {
    ozg_report& r = reps[widx[i]];
    const bool au = P->any_auto && wauto[i];
    const int runs = (au && !fl[i]) ? (sk2[i] ? 0 : (sk3[i] ? 1 : 2)) : 0;  // escalations
    r.nonfinite = fl[i];
    r.selected = au ? su[i] : 0;
    r.repaired = runs;
    r.slices_used = fl[i] ? -1 : (au ? (runs == 0 ? su[i] : (runs == 1 ? s2[i] : ws[i])) : ws[i]);
    r.samples = (P->nsamp > 0 && !fl[i]) ? P->nsamp : 0;
    r.est_err = r.samples ? (runs == 0 ? er[i] : (runs == 1 ? er2[i] : er3[i])) : NAN;
  }
  return OZG_OK;
}

}  // namespace

// The grouped call.  With sync_reports == false and reps set, the reports are initialised and the
// call returns once its work is queued; grouped_collect_reports fills them in later.
int grouped_call(ozg_ctx* c, int64_t count, const ozg_gemm_desc* descs, const int* slices, ozg_report* reps,
                 bool sync_reports) {
  if (!c || count < 0 || (count > 0 && !descs)) return OZG_ERR_INVALID;
  c->deferred.reps = nullptr;
  if (count == 0) return OZG_OK;
  if (count > (1 << 20)) return OZG_ERR_UNSUPPORTED;
  std::vector<char> TA(count), TB(count), autom_all(count, 0);
  std::vector<int> s(count);
  bool bad = false;
  for (int64_t i = 0; i < count; ++i) {
    int rc = check_desc(descs[i], TA[i], TB[i]);
    const int si = slices ? slices[i] : 0;
    if (!rc && (si < 0 || si > OZG_MAX_SLICES)) rc = -14;
    s[i] = si == 0 ? c->fallback_slices : si;
    autom_all[i] = (si == 0 && c->sel_s_hi > 0) ? 1 : 0;
    if (reps) {
      std::memset(&reps[i], 0, sizeof(ozg_report));
      reps[i].status = rc;
      reps[i].slices_used = s[i];
      reps[i].est_err = NAN;
      reps[i].max_real = NAN;
      reps[i].max_imag = NAN;
    }
    if (rc) bad = true;
  }
  if (bad) return OZG_ERR_INVALID;
  // calls the emulated kernels cannot take (empty, k == 0, alpha == 0) go through ozg_dgemm
  std::vector<ozg_gemm_desc> work;
  std::vector<int> ws, widx;
  for (int64_t i = 0; i < count; ++i) {
    const ozg_gemm_desc& d = descs[i];
    if (d.m == 0 || d.n == 0 || d.k == 0 || d.alpha == 0.0) {
      int rc = ozg_dgemm(c, d.transa, d.transb, d.m, d.n, d.k, d.alpha, d.A, d.lda, d.B, d.ldb, d.beta, d.C, d.ldc,
                         slices ? slices[i] : 0, nullptr);
      if (rc) return rc;
      if (reps) reps[i].samples = 0;
      continue;
    }
    work.push_back(d);
    ws.push_back(s[i]);
    widx.push_back((int)i);
  }
  if (work.empty()) return OZG_OK;
  cudaSetDevice(c->device);
  const int64_t n = (int64_t)work.size();
  std::vector<char> wa(n), wb(n), wauto(n);
  for (int64_t i = 0; i < n; ++i) {
    wa[i] = TA[widx[i]];
    wb[i] = TB[widx[i]];
    wauto[i] = autom_all[widx[i]];
  }
  uint64_t key = 1469598103934665603ull;
  key = fnv(key, work.data(), sizeof(ozg_gemm_desc) * n);
  key = fnv(key, ws.data(), sizeof(int) * n);
  key = fnv(key, &c->check_samples, sizeof(int));
  key = fnv(key, &c->autotune, sizeof(int));
  key = fnv(key, wauto.data(), n);

  GroupPlan* P = c->plan.get();
  const bool reuse = P && P->key == key && P->epoch == c->gws_epoch;
  PhaseScope ps(c, OZG_PHASE_GROUPED);
  if (!reuse) {
    c->plan.reset();
    // tile variant: autotuned per batch when every call writes C without reading it (all
    // variants give bit-identical results), else the padding heuristic summed over the batch;
    // for 256-wide tiles, deferred pushes when the work-weighted mean k is long
    int variant;
    double pad0 = 0, pad1 = 0, wk = 0, wsum = 0, w = 0;
    bool all_beta_zero = true;
    for (int64_t i = 0; i < n; ++i) {
      pad0 += (double)((work[i].m + 127) / 128) * ((work[i].n + 255) / 256) * 256 * ws[i] * ws[i];
      pad1 += (double)((work[i].m + 127) / 128) * ((work[i].n + 127) / 128) * 128 * ws[i] * ws[i];
      const double wi = (double)work[i].m * work[i].n * ws[i] * ws[i];
      wk += wi * work[i].k;
      wsum += wi * ws[i];
      w += wi;
      all_beta_zero = all_beta_zero && work[i].beta == 0.0;
    }
    (void)wsum;
    // the stacked kernel takes batches whose largest slice count (automatic calls: up to the
    // selector's top class or the fallback) is within its limit
    int smax = 0;
    const int s_hi = std::max(c->sel_s_hi, c->fallback_slices);
    for (int64_t i = 0; i < n; ++i) smax = std::max(smax, wauto[i] ? s_hi : ws[i]);
    const bool stacked_ok = smax <= ozg::stacked_max_slices();
    // 128-wide tiles take the stacked group pairs when the batch's slice counts allow them
    // (measured faster than the one-group kernel on grouped batches of short and medium k)
    if (pad1 < pad0)
      variant = stacked_ok ? ozg::kStackedVariant : 1;
    else
      variant = (w > 0 && wk >= 2048.0 * w) ? 2 : 0;
    auto tuned = c->tune.find(key);
    if (c->force_variant >= 0) {
      variant = (c->force_variant == ozg::kStackedVariant && !stacked_ok) ? 1 : c->force_variant;
    } else if (tuned != c->tune.end()) {
      variant = tuned->second;
    } else if (c->autotune && all_beta_zero) {
      float best = 1e30f;
      const bool pair_ok = ozg::pair_max_ctas() >= 2;
      for (int v = 0; v < OZG_NUM_TILE_VARIANTS; ++v) {
        if ((v == ozg::kPairVariant && !pair_ok) || (v == ozg::kStackedVariant && !stacked_ok)) continue;
        std::unique_ptr<GroupPlan, PlanDeleter> T(new GroupPlan());
        int rc = build_plan(c, n, work.data(), ws, wa, wb, wauto, v, T.get());
        if (rc) return rc;
        cudaEvent_t e0 = pool_get(c), e1 = pool_get(c);
        if (!e0 || !e1) return OZG_ERR_CUDA;
        rc = enqueue(c, *T);  // warm-up (also fills the digit planes)
        if (!rc) {
          cudaEventRecord(e0, c->stream);
          rc = enqueue(c, *T);
          cudaEventRecord(e1, c->stream);
        }
        float ms = 1e30f;
        if (!rc && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        c->pool.push_back(e0);
        c->pool.push_back(e1);
        if (rc) return rc;
        if (ms < best) {
          best = ms;
          variant = v;
        }
      }
      c->tune[key] = variant;
    }
    std::unique_ptr<GroupPlan, PlanDeleter> NP(new GroupPlan());
    int rc = build_plan(c, n, work.data(), ws, wa, wb, wauto, variant, NP.get());
    if (rc) return rc;
    NP->key = key;
    if (c->graphs && c->stream != nullptr) {
      cudaGraph_t graph = nullptr;
      OZG_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      const long long before = ozg::launch_counter();
      rc = enqueue(c, *NP);
      NP->nkernels = ozg::launch_counter() - before;
      __atomic_fetch_sub(&ozg::launch_counter(), NP->nkernels, __ATOMIC_RELAXED);  // counted per replay
      cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      OZG_CUDA(ce);
      cudaError_t ie = cudaGraphInstantiate(&NP->exec, graph, 0);
      cudaGraphDestroy(graph);
      OZG_CUDA(ie);
    }
    c->plan.reset(NP.release());
    P = c->plan.get();
  }
  if (P->exec) {
    OZG_CUDA(cudaGraphLaunch(P->exec, c->stream));
    __atomic_fetch_add(&ozg::launch_counter(), P->nkernels, __ATOMIC_RELAXED);
  } else {
    int rc = enqueue(c, *P);
    if (rc) return rc;
  }
  if (reps) {
    if (sync_reports) return read_reports(c, n, widx, ws, wauto, reps);
    c->deferred.widx = widx;
    c->deferred.ws = ws;
    c->deferred.wauto = wauto;
    c->deferred.n = n;
    c->deferred.reps = reps;
  }
  return OZG_OK;
}

int grouped_collect_reports(ozg_ctx* c) {
  if (c->deferred.reps == nullptr) return OZG_OK;
  ozg_report* reps = c->deferred.reps;
  c->deferred.reps = nullptr;
  return read_reports(c, c->deferred.n, c->deferred.widx, c->deferred.ws, c->deferred.wauto, reps);
}

}  // namespace host
}  // namespace ozg

extern "C" int ozg_dgemm_grouped(ozg_ctx* c, int64_t count, const ozg_gemm_desc* descs, const int* slices,
                                 ozg_report* reps) {
  if (!c) return OZG_ERR_INVALID;
  return grouped_call(c, count, descs, slices, reps, true);
}

extern "C" int ozg_set_graphs(ozg_ctx* c, int enable) {
  if (!c) return OZG_ERR_INVALID;
  c->graphs = enable != 0;
  c->plan.reset();
  return OZG_OK;
}

extern "C" int ozg_set_fallback_slices(ozg_ctx* c, int s) {
  if (!c) return OZG_ERR_INVALID;
  if (s < 1 || s > OZG_MAX_SLICES) return -2;
  c->fallback_slices = s;
  return OZG_OK;
}

// Region-adaptive slice counts: one GEMM cut into row_blocks x col_blocks regions of C, each a
// call of one grouped launch over the full k with slice count 0, so that (with a selector
// loaded) every region gets the count its own rows of op(A) and columns of op(B) need.  The
// regions' row and column bands differ by at most one in size; an empty band (more blocks than
// rows or columns) is a quick return.
extern "C" int ozg_dgemm_regions(ozg_ctx* c, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                                 int64_t ldc, int row_blocks, int col_blocks, ozg_report* reps) {
  ozg_gemm_desc whole{};
  whole.transa = transa;
  whole.transb = transb;
  whole.m = m;
  whole.n = n;
  whole.k = k;
  whole.lda = lda;
  whole.ldb = ldb;
  whole.ldc = ldc;
  char ta, tb;
  int rc = check_desc(whole, ta, tb);
  if (!rc && row_blocks < 1) rc = -14;
  if (!rc && col_blocks < 1) rc = -15;
  if (!rc && !c) return OZG_ERR_INVALID;  // BLAS argument errors are reported first
  if (!rc && (int64_t)row_blocks * col_blocks > (1 << 20)) return OZG_ERR_UNSUPPORTED;
  const int64_t count = rc ? 0 : (int64_t)row_blocks * col_blocks;
  if (reps && !rc) std::memset(reps, 0, sizeof(ozg_report) * (size_t)count);
  if (rc) return rc;
  if (m == 0 || n == 0) return OZG_OK;
  std::vector<ozg_gemm_desc> d((size_t)count);
  for (int i = 0; i < row_blocks; ++i) {
    const int64_t r0 = m * i / row_blocks, r1 = m * (i + 1) / row_blocks;
    for (int j = 0; j < col_blocks; ++j) {
      const int64_t c0 = n * j / col_blocks, c1 = n * (j + 1) / col_blocks;
      ozg_gemm_desc& x = d[(size_t)i * col_blocks + j];
      x = whole;
      x.m = r1 - r0;
      x.n = c1 - c0;
      x.alpha = alpha;
      x.beta = beta;
      x.A = ta == 'N' ? A + r0 : A + r0 * lda;  // rows r0 .. r1-1 of op(A)
      x.B = tb == 'N' ? B + c0 * ldb : B + c0;  // columns c0 .. c1-1 of op(B)
      x.C = C + r0 + c0 * ldc;
    }
  }
  std::vector<int> zero((size_t)count, 0);
  return ozg_dgemm_grouped(c, count, d.data(), zero.data(), reps);
}

extern "C" int ozg_set_tile_variant(ozg_ctx* c, int variant) {
  if (!c || variant < -1 || variant >= OZG_NUM_TILE_VARIANTS) return OZG_ERR_INVALID;
  if (variant == ozg::kPairVariant && ozg::pair_max_ctas() < 2) return OZG_ERR_UNSUPPORTED;  // no 2-CTA cluster fits
  c->force_variant = variant;
  c->plan.reset();  // a cached grouped plan may hold another variant
  return OZG_OK;
}

extern "C" int ozg_get_tile_variant(ozg_ctx* c, int* variant) {
  if (!c || !variant) return OZG_ERR_INVALID;
  *variant = c->plan ? c->plan->variant : -1;
  return OZG_OK;
}

extern "C" int ozg_set_autotune(ozg_ctx* c, int enable, const char* cache_path) {
  if (!c) return OZG_ERR_INVALID;
  c->autotune = enable != 0;
  c->tune_path = cache_path ? cache_path : "";
  c->tune_loaded = false;
  return OZG_OK;
}
