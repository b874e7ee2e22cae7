// K2 + K3: the slice products of the Ozaki scheme (Sec. 2.2) on the sm_103a tensor cores,
// fused with the FP64 scale-and-accumulate epilogue.
//
// The INT8-range digits (|d| <= 127) are held in FP16, which represents them exactly, and
// multiplied by tcgen05.mma kind::f16 with FP32 accumulation in TMEM.  Every product is an
// integer below 2^14 and an accumulation chain holds at most 1024 products per entry, so every
// partial sum is an integer below 1024 * 127^2 < 2^24 and the FP32 accumulator is exact: the
// chain result IS the integer slice product.  (tcgen05.mma kind::i8 does not exist for
// sm_103a, and the legacy warp-level integer MMA runs ~15x below the FP16 tensor rate.)
//
// Per output tile (BM x BN of the (stacked) product) the schedule is group-major:
//   for g = 2 .. s+1:  for kb in k-blocks:  for p = 1 .. g-1:  D[buf] += A_p[kb] * B_{g-p}[kb]^T
// cut into chains of at most 1024 products (k-blocks x pairs).  Each finished chain is drained by the epilogue
// warps (TMEM -> registers, exact FP32 -> int32) into an int32 group sum G_g while the MMA
// warp fills the other TMEM buffer.  At the end of group g the epilogue folds G_g into
// R <- 128 R + G_g (Horner in the group index), kept per CTA in L2-resident scratch, in exact
// int64 windows of as many groups as cannot overflow (5 or 6 in practice); two windows make an
// exact 128-bit sum, later windows continue in FP64.  After the last group it writes
// C = alpha * RN(R 2^{e_i + f_j - 7(s+1)}) (+ beta C): for up to two windows (s <= 10 at any k
// that fits in memory) one rounding of the exact value, done with integer instructions, so
// with alpha = 1, beta = 0 the epilogue issues no FP64 instruction at all -- FP64 is the
// slowest pipe of this GPU.  The opt-in exact mode keeps a 128-bit Horner sum (s <= 13).
// Complex (stacked rows 2i = Re, 2i+1 = Im; columns likewise) combines the four real
// sub-products exactly in int32 before the Horner step: Re = P_rr - P_ii, Im = P_ri + P_ir.
//
// Warp roles (384 threads = 3 warpgroups, one CTA per SM, persistent over tiles):
//   warpgroup 0: warp 0 TMA producer (one lane), warp 1 TMEM allocator + MMA issuer (one lane),
//                warps 2-3 idle; the group shrinks its registers to 56 (setmaxnreg.dec)
//   warpgroups 1-2 (warps 4..11): epilogue, grown to 224 registers (setmaxnreg.inc) to hold the
//                int32 group sums; warp w reads TMEM lanes 32 (w % 4) .. +31 and half
//                (w - 4) / 4 of the BN columns.
// Register budget: 384 threads x 168 at launch = 64512 = 128 x 56 + 256 x 224.
//
// Two tile widths (BN = 256 or 128; the autotuner picks per shape) and two work sources: one
// GEMM (tiles rastered in GROUP_M row bands), or a grouped list of tiles drawn from many GEMMs,
// each with its own tensor maps, slice count and epilogue parameters (one persistent launch
// for a whole batch of uneven problems).
#include <climits>

#include "ozg_device.cuh"
#include "ozg_internal.h"
#include "ozg_round.cuh"

namespace ozg {
namespace {

constexpr int BM = 128, BK = 64;  // BK: k width of one 128-byte swizzle atom (one TMA box)
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 128 + EPI_WARPS * 32;
constexpr int REG_PRODUCER = 56, REG_EPILOGUE = 224;
static_assert(128 * REG_PRODUCER + EPI_WARPS * 32 * REG_EPILOGUE <= THREADS * 168, "register split");
constexpr int TRING = 4;       // tile-index ring depth (grouped launches)
constexpr int CHAIN_K = 1024;  // products per accumulation chain: 1024 * 127^2 = 16516096 < 2^24
constexpr int GROUP_M = 8;     // tile raster: GROUP_M row-tiles share a sweep over the column tiles
static_assert(CHAIN_K * 127 * 127 < (1 << 24), "FP32 chain must stay exact");

// One pipeline stage holds SUB 64-wide k sub-tiles of A and of B (SK = 64 SUB k).  With
// 128-wide tiles, two per stage (3 stages) give eight MMAs per barrier round trip instead of
// four -- one lane issuing a 128 x 128 x 64 block is slower than the tensor core executing it
// -- while one per stage (6 stages) hides more load latency (large s: bigger working sets).
//
// CTA pairs (PAIR, grouped launches, 128-wide): a 2-CTA cluster computes a 256 x BN tile with
// tcgen05.mma.cta_group::2 (M = 256) issued by the even-rank CTA.  Each CTA stages its own 128
// rows of A and BN / 2 of the B columns (the MMA reads the other half from the peer), so a stage
// is 48 KB instead of 64 KB and four stages fit; each CTA's TMEM holds its own 128 rows of the
// accumulator, drained by its own epilogue exactly as in a 1-CTA tile.
template <int BN_, int SUB_, bool PAIR_ = false>
struct Cfg {
  static constexpr int SUB = SUB_;
  static constexpr int SK = SUB * BK;
  static constexpr int SEG = CHAIN_K / SK;  // stages per chain
  static constexpr int STAGES = PAIR_ ? 4 : (BN_ == 256 ? 4 : (SUB_ == 2 ? 3 : 6));
  static constexpr uint32_t SUBA_BYTES = BM * BK * 2, SUBB_BYTES = (PAIR_ ? BN_ / 2 : BN_) * BK * 2;
  static constexpr uint32_t A_BYTES = SUB * SUBA_BYTES, B_BYTES = SUB * SUBB_BYTES, STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr uint32_t IDESC = umma_idesc_f16_f32(PAIR_ ? 2 * BM : BM, BN_);
  // two BN-column FP32 accumulators; 128-wide tiles also keep the int64 window words (two
  // columns per output) in the other half
  static constexpr uint32_t TMEM_COLS = 512;
  static constexpr int CPT = BN_ / 2;             // columns per epilogue thread
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
};

// Everything one output tile needs, from either work source.
struct TileJob {
  const CUtensorMap* tmA;
  const CUtensorMap* tmB;
  int tm, tn, KB, s, cplx, skip;
  int klast;  // 64-wide sub-tiles holding valid k in the last stage (1 .. SUB)
  int64_t rows, cols, n;  // stacked product rows / cols, output columns (complex: n)
  const int32_t* e;
  const int32_t* f;
  double* C;
  int64_t ldc;
  double a0, a1, b0, b1;
  int beta_zero;
};

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int& tm, int& tn) {
  int per_group = GROUP_M * tiles_n;
  int grp = t / per_group;
  int first = grp * GROUP_M;
  int gsz = min(tiles_m - first, GROUP_M);
  int r = t % per_group;
  tm = first + r % gsz;
  tn = r / gsz;
}

template <int BN_, int SUB_, bool GROUPED, bool PAIR = false>
__device__ __forceinline__ TileJob get_job(int t, const CUtensorMap* tmA, const CUtensorMap* tmB, const GemmArgs* P,
                                           const GroupArgs* G) {
  TileJob j;
  if (!GROUPED) {
    const int tiles_m = (int)((P->rows + BM - 1) / BM), tiles_n = (int)((P->cols + BN_ - 1) / BN_);
    tile_coords(t, tiles_m, tiles_n, j.tm, j.tn);
    j.tmA = tmA;
    j.tmB = tmB;
    j.KB = (int)((P->k + Cfg<BN_, SUB_>::SK - 1) / Cfg<BN_, SUB_>::SK);
    j.klast = (int)((P->k - (int64_t)(j.KB - 1) * Cfg<BN_, SUB_>::SK + BK - 1) / BK);
    j.s = P->s_dev != nullptr ? *P->s_dev : P->s;
    j.cplx = P->cplx;
    j.skip = 0;
    j.rows = P->rows;
    j.cols = P->cols;
    j.n = P->n;
    j.e = P->e;
    j.f = P->f;
    j.C = P->C;
    j.ldc = P->ldc;
    j.a0 = P->alpha[0];
    j.a1 = P->alpha[1];
    j.b0 = P->beta[0];
    j.b1 = P->beta[1];
    j.beta_zero = P->beta_zero;
  } else {
    const GroupTile gt = G->tiles[t];
    if (gt.call < 0) {  // padding slot of the load-balanced tile list
      j.skip = 1;
      return j;
    }
    const GroupCall* c = G->calls + gt.call;
    j.tm = gt.tm;
    j.tn = gt.tn;
    j.tmA = &c->tmA;
    j.tmB = PAIR ? &c->tmBh : &c->tmB;  // CTA pairs load half of the B columns each
    j.KB = (int)((c->k + Cfg<BN_, SUB_>::SK - 1) / Cfg<BN_, SUB_>::SK);
    j.klast = (int)((c->k - (int64_t)(j.KB - 1) * Cfg<BN_, SUB_>::SK + BK - 1) / BK);
    j.s = c->s;
    j.cplx = c->cplx;
    j.skip = (c->nonfinite != nullptr && *c->nonfinite) ? 1 : 0;
    j.rows = c->rows;
    j.cols = c->cols;
    j.n = c->n;
    j.e = c->e;
    j.f = c->f;
    j.C = c->C;
    j.ldc = c->ldc;
    j.a0 = c->alpha[0];
    j.a1 = c->alpha[1];
    j.b0 = c->beta[0];
    j.b1 = c->beta[1];
    j.beta_zero = c->beta_zero;
  }
  return j;
}

__device__ __forceinline__ int nseg_of(int g, int KB, int seg) { return ((g - 1) * KB + seg - 1) / seg; }

__device__ __noinline__ double ldexp_slow(double x, int E) { return ldexp(x, E); }
// x * 2^E with one rounding (the same result as ldexp); fast path when 2^E is a normal double
__device__ __forceinline__ double scale_pow2(double x, int E) {
  if (E >= -1022 && E <= 1023) return x * __longlong_as_double((long long)(E + 1023) << 52);
  return ldexp_slow(x, E);
}

// Exact epilogue (s <= kExactMaxS): R is a 128-bit integer per output, kept as (lo, hi) in 16
// bytes of the CTA's scratch tile; the group sums enter by Horner's rule R <- 128 R + G_g, and
// the final R is rounded to FP64 once.  |R| < 2^(log2 max|G_g| + 7 (s - 1) + 1), within 127 bits
// for s <= 13 and k < 2^20.  Larger s keeps an FP64 R (one rounding per Horner step).
constexpr int kExactMaxS = 13;

__device__ __forceinline__ void horner128(const void* Rp, int g, bool first, bool group2, int64_t& hi,
                                          uint64_t& lo) {
  if (first && group2) {
    lo = (uint64_t)(int64_t)g;
    hi = g < 0 ? -1 : 0;
    return;
  }
  const longlong2 v = *reinterpret_cast<const longlong2*>(Rp);
  lo = (uint64_t)v.x;
  hi = v.y;
  if (first) {  // R <- 128 R (two's complement 128-bit shift)
    hi = (int64_t)(((uint64_t)hi << 7) | (lo >> 57));
    lo <<= 7;
  }
  const uint64_t gl = (uint64_t)(int64_t)g, nl = lo + gl;
  hi = hi + (g < 0 ? -1 : 0) + (nl < lo ? 1 : 0);
  lo = nl;
}


// One output's Horner step in either mode; returns the final value (scaled) on the last push.
__device__ __forceinline__ double horner_step(void* Rp, int g, bool exact, bool first, bool group2, bool final_push,
                                              int E) {
  if (exact) {
    int64_t hi;
    uint64_t lo;
    horner128(Rp, g, first, group2, hi, lo);
    if (final_push) return round_i128(hi, lo, E);
    *reinterpret_cast<longlong2*>(Rp) = make_longlong2((long long)lo, (long long)hi);
    return 0.0;
  }
  double* Rd = reinterpret_cast<double*>(Rp);
  const double gv = (double)g;
  const double Rv = first ? (group2 ? gv : fma(*Rd, 128.0, gv)) : (*Rd + gv);
  if (final_push) return scale_pow2(Rv, E);
  *Rd = Rv;
  return 0.0;
}

// Window-closing or final step of one output, given the first slot's word s0 (int64 W0 while
// widx == 1, FP64 bits from the second window's close on) and the active window Rw after this
// push.  Final: returns RN(N 2^E).  Closing: returns the new s0 word.
__device__ __forceinline__ double final_val(long long s0, long long Rw, int widx, int wlen, int E) {
  if (widx == 0) return rn_i128_pow2(Rw < 0 ? -1 : 0, (unsigned long long)Rw, E);
  if (widx == 1) {
    long long hi;
    unsigned long long lo;
    i128_shl_add(s0, 7 * wlen, Rw, hi, lo);
    return rn_i128_pow2(hi, lo, E);
  }
  return scale_pow2(fma(__longlong_as_double(s0), scale_pow2(1.0, 7 * wlen), (double)Rw), E);
}
__device__ __forceinline__ long long close_val(long long s0, long long Rw, int widx, int wlen) {
  if (widx == 1) {
    long long hi;
    unsigned long long lo;
    i128_shl_add(s0, 7 * wlen, Rw, hi, lo);
    return __double_as_longlong(rn_i128_pow2(hi, lo, 0));
  }
  return __double_as_longlong(fma(__longlong_as_double(s0), scale_pow2(1.0, 7 * wlen), (double)Rw));
}

enum PushKind { kPlain = 0, kSpill = 1, kClose = 2, kFinal = 3 };

// Everything a push needs besides the group sums.
struct PushArgs {
  int kind, widx, wlen;
  bool first, wstart;     // first push of its group; first push of its window
  uint32_t rtm;           // TMEM address of this thread's window words (TMEM-resident mode)
  long long* Ra;          // the active window's scratch slot (L2-resident mode)
  long long* S0;          // the first window's scratch slot
  int64_t gcol0, orow;
  bool row_ok, unit_ab, odd;
  int ebase;
};

// One push for NCH consecutive outputs o0 .. o0+NCH-1 of this thread; vals holds the chunk's
// group sums (vals[i], complex: the pair vals[2i], vals[2i+1]).  The active window lives
// in TMEM (TMR: two 32-bit columns per output, one 32x32b.x32 load and store per 16 outputs) or
// in the CTA's L2-resident scratch (loads batched NCH deep before any use, to keep that many in
// flight).  Complex: the (Re, Im) column pairs are combined exactly across the lane pair first.
// The scratch words S0 and the column exponents a closing or final push of outputs
// o0 .. o0+NCH-1 needs, loaded ahead of the push (software pipelining across chunks).
template <int NCH>
__device__ __forceinline__ void prefetch_close(const PushArgs& a, const TileJob& j, int o0, long long (&s0)[NCH],
                                               int (&fe)[NCH]) {
  if (a.widx >= 1) {
#pragma unroll
    for (int i = 0; i < NCH; ++i) s0[i] = a.S0[(size_t)(o0 + i) * BM];
  } else {
#pragma unroll
    for (int i = 0; i < NCH; ++i) s0[i] = 0;
  }
  const int64_t c0 = j.cplx ? (a.gcol0 >> 1) + o0 : a.gcol0 + o0;
  const int64_t climit = j.cplx ? j.n : j.cols;
#pragma unroll
  for (int i = 0; i < NCH; ++i) fe[i] = (a.kind == kFinal && c0 + i < climit) ? __ldg(j.f + c0 + i) : 0;
}

// RN(W 2^E) for one int64 window: one correctly rounded conversion, the power of two added to
// the exponent field.  `ok` is false when the result is not a normal double (the caller then
// takes final_val).  The same value as rn_windows(0, W, S, E) with fewer instructions.
__device__ __forceinline__ double rn_single(long long W, int E, bool& ok) {
  const long long bits = __double_as_longlong(__ll2double_rn(W));
  const int ex = (int)((bits >> 52) & 0x7ff) + E;
  ok = W == 0 || (ex >= 1 && ex <= 2046);
  return W == 0 ? 0.0 : __longlong_as_double(bits + ((long long)E << 52));
}

template <int NCH, bool TMR, bool PRE = false>
__device__ __forceinline__ void window_out(const long long* rw, int o0, const PushArgs& a, const TileJob& j,
                                           const long long* s0_pre, const int* fe_pre);

template <int NCH, bool TMR, bool PRE = false>
__device__ __forceinline__ void push_chunk(const int* vals, int o0, const PushArgs& a, const TileJob& j,
                                           const long long* s0_pre = nullptr, const int* fe_pre = nullptr) {
  static_assert(!TMR || NCH == 16, "TMEM chunks are 32 columns");
  int vv[NCH];
  if (!j.cplx) {
#pragma unroll
    for (int i = 0; i < NCH; ++i) vv[i] = vals[i];
  } else {
#pragma unroll
    for (int i = 0; i < NCH; ++i) {
      const int other = __shfl_xor_sync(0xffffffffu, vals[2 * i + 1], 1);
      vv[i] = a.odd ? (vals[2 * i] + other) : (vals[2 * i] - other);
    }
  }
  long long rw[NCH];
  if (!(a.first && a.wstart)) {
    long long ro[NCH];
    if (TMR) {
      uint32_t t[32];
      tmem_ld32(a.rtm + 2 * o0, t);
      tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < NCH; ++i) ro[i] = (long long)(((unsigned long long)t[2 * i + 1] << 32) | t[2 * i]);
    } else {
#pragma unroll
      for (int i = 0; i < NCH; ++i) ro[i] = a.Ra[(size_t)(o0 + i) * BM];
    }
#pragma unroll
    for (int i = 0; i < NCH; ++i) rw[i] = a.first ? (long long)((unsigned long long)ro[i] << 7) + vv[i] : ro[i] + vv[i];
  } else {
#pragma unroll
    for (int i = 0; i < NCH; ++i) rw[i] = vv[i];
  }
  window_out<NCH, TMR, PRE>(rw, o0, a, j, s0_pre, fe_pre);
}

// The part of a push after the window value: store the active window (plain), spill the first
// window (spill), close a later window into the FP64 partial (close), or round and write C
// (final), for outputs o0 .. o0+NCH-1 whose window values are rw.
template <int NCH, bool TMR, bool PRE>
__device__ __forceinline__ void window_out(const long long* rw, int o0, const PushArgs& a, const TileJob& j,
                                           const long long* s0_pre, const int* fe_pre) {
  if (a.kind == kPlain) {
    if (TMR) {
      uint32_t t[32];
#pragma unroll
      for (int i = 0; i < NCH; ++i) {
        t[2 * i] = (uint32_t)(unsigned long long)rw[i];
        t[2 * i + 1] = (uint32_t)((unsigned long long)rw[i] >> 32);
      }
      tmem_st32(a.rtm + 2 * o0, t);
      tmem_st_wait();
    } else {
#pragma unroll
      for (int i = 0; i < NCH; ++i) a.Ra[(size_t)(o0 + i) * BM] = rw[i];
    }
    return;
  }
  if (a.kind == kSpill) {
#pragma unroll
    for (int i = 0; i < NCH; ++i) a.S0[(size_t)(o0 + i) * BM] = rw[i];
    return;
  }
  long long s0[NCH];
  int fe[NCH];
  if (PRE) {
#pragma unroll
    for (int i = 0; i < NCH; ++i) {
      s0[i] = s0_pre[i];
      fe[i] = fe_pre[i];
    }
  } else {
    prefetch_close<NCH>(a, j, o0, s0, fe);
  }
  // C is written with evict-first (streaming) stores: it is not read again by this launch, and
  // normal stores would displace digit-plane lines that the next groups read again from L2.
  // RN of the exact sum: for one or two windows all NCH outputs go through the branch-free
  // rounding together, and only results outside the normal range take the general path
  // (in batches of RB outputs, to bound the registers live at once)
  constexpr int RB = NCH < 8 ? NCH : 8;
  const int64_t c0 = j.cplx ? (a.gcol0 >> 1) + o0 : a.gcol0 + o0;
#pragma unroll
  for (int i0 = 0; i0 < NCH; i0 += RB) {
    double tv[RB];
    if (a.widx == 0 && a.kind == kFinal) {
      // a single window: one conversion per output
      unsigned bad = 0;
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        bool ok;
        tv[i] = rn_single(rw[i0 + i], a.ebase + fe[i0 + i], ok);
        bad |= ok ? 0u : 1u << i;
      }
      if (bad != 0) {
#pragma unroll
        for (int i = 0; i < RB; ++i)
          if ((bad >> i) & 1u) tv[i] = final_val(0, rw[i0 + i], 0, a.wlen, a.ebase + fe[i0 + i]);
      }
    } else if (a.widx <= 1) {
      const bool close = a.kind == kClose;
      unsigned bad = 0;
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        bool ok;
        tv[i] = rn_windows(a.widx == 0 ? 0ll : s0[i0 + i], rw[i0 + i], 7 * a.wlen, close ? 0 : a.ebase + fe[i0 + i], ok);
        bad |= ok ? 0u : 1u << i;
      }
      if (bad != 0) {
#pragma unroll
        for (int i = 0; i < RB; ++i)
          if ((bad >> i) & 1u)
            tv[i] = close ? __longlong_as_double(close_val(s0[i0 + i], rw[i0 + i], a.widx, a.wlen))
                          : final_val(s0[i0 + i], rw[i0 + i], a.widx, a.wlen, a.ebase + fe[i0 + i]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < RB; ++i)
        tv[i] = a.kind == kClose ? __longlong_as_double(close_val(s0[i0 + i], rw[i0 + i], a.widx, a.wlen))
                                 : final_val(s0[i0 + i], rw[i0 + i], a.widx, a.wlen, a.ebase + fe[i0 + i]);
    }
    if (a.kind == kClose) {
#pragma unroll
      for (int i = 0; i < RB; ++i) a.S0[(size_t)(o0 + i0 + i) * BM] = __double_as_longlong(tv[i]);
      continue;
    }
    if (!j.cplx) {
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const int64_t col = c0 + i0 + i;
        if (a.row_ok && col < j.cols) {
          double* cp = j.C + a.orow + col * j.ldc;
          __stcs(cp, a.unit_ab ? tv[i] : (j.beta_zero ? j.a0 * tv[i] : fma(j.a0, tv[i], j.b0 * *cp)));
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const int64_t jc = c0 + i0 + i;
        const bool ok = a.row_ok && jc < j.n;
        const double part = ok ? tv[i] : 0.0;
        const double partner = __shfl_xor_sync(0xffffffffu, part, 1);
        if (ok) {
          double* cp = j.C + 2 * (a.orow + jc * j.ldc);
          if (a.unit_ab) {
            __stcs(cp + (a.odd ? 1 : 0), part);
          } else {
            const double tr = a.odd ? partner : part, ti = a.odd ? part : partner;
            double re = fma(j.a0, tr, -(j.a1 * ti));
            double im = fma(j.a0, ti, j.a1 * tr);
            if (!j.beta_zero) {
              const double cr = cp[0], ci = cp[1];
              re += fma(j.b0, cr, -(j.b1 * ci));
              im += fma(j.b0, ci, j.b1 * cr);
            }
            __stcs(cp + (a.odd ? 1 : 0), a.odd ? im : re);
          }
        }
      }
    }
  }
}

// Bounded wait used during teardown after an abort (ignores the abort flag).
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > OZG_WAIT_CYCLES) return;
  }
}

template <int BN_, int SUB_, bool GROUPED, bool PAIR = false>
__device__ __forceinline__ void gemm_body(const CUtensorMap* tmA0, const CUtensorMap* tmB0, const GemmArgs* P,
                                          const GroupArgs* G) {
  static_assert(!PAIR || (GROUPED && BN_ == 128), "CTA pairs: grouped 128-wide tiles");
  using K = Cfg<BN_, SUB_, PAIR>;
  constexpr int BN = BN_, STAGES = K::STAGES, CPT = K::CPT;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES], bar_accf[2], bar_acce[2], bar_done;
  // grouped launches hand out tiles dynamically: the producer claims a tile index (atomic
  // counter) and passes it to the MMA lane and the epilogue warps through this ring
  __shared__ __align__(8) uint64_t bar_tfull[TRING], bar_tempty[TRING];
  __shared__ int tile_ring[TRING];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  int* status = GROUPED ? G->status : P->status;
  double* Rws = GROUPED ? G->Rws : P->Rws;
  int64_t* Gdbg = GROUPED ? nullptr : P->Gdbg;
  const int ntiles = GROUPED ? G->ntiles : (int)(((P->rows + BM - 1) / BM) * ((P->cols + BN - 1) / BN));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // CTA pairs: rank 0 (the leader) claims tiles, owns the stage-full, accumulator-empty and
  // tile-ring-empty barriers both CTAs arrive at, and issues the pair MMAs
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&bar_full[i], PAIR ? 2 : 1);  // pairs: each CTA's producer announces its bytes
      mbar_init(&bar_empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_accf[b], 1);
      mbar_init(&bar_acce[b], PAIR ? 2 * EPI_WARPS : EPI_WARPS);
    }
    mbar_init(&bar_done, 1);
    for (int i = 0; i < TRING; ++i) {
      mbar_init(&bar_tfull[i], 1);
      // consumers of a ring slot: the MMA lane and the epilogue warps; pairs add the peer's
      // producer and epilogue warps
      mbar_init(&bar_tempty[i], PAIR ? 2 + 2 * EPI_WARPS : 1 + EPI_WARPS);
    }
    abort_flag = 0;
    mbar_fence_init();
  }
  if (!GROUPED && warp == 0 && lane == 0) {
    tma_prefetch_desc(tmA0);
    tma_prefetch_desc(tmB0);
  }
  if (warp == 1) {
    if (PAIR)
      tmem_alloc_pair(&tmem_slot, K::TMEM_COLS);  // both CTAs of the pair, the same columns
    else
      tmem_alloc(&tmem_slot, K::TMEM_COLS);
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) {  // the peer's barriers are initialised before any remote arrival
    __syncwarp();
    cluster_sync_all();
  }
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* abort_p = &abort_flag;

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_PRODUCER));
    if (warp == 0) {
      // ---------------------------------------------------------------- TMA producer
      if (lane == 0) {
        uint32_t stage = 0, phase = 0;
        long long issued = 0;
        const CUtensorMap* last_map = nullptr;
        uint32_t tslot = 0, tphase = 0;
        // pairs: cluster c takes pair tile c first, then claims the next from the counter
        const int nunits = PAIR ? (int)(gridDim.x / 2) : (int)gridDim.x;
        int tnext = PAIR ? (int)(blockIdx.x / 2) : (int)blockIdx.x;
        for (;;) {
          int t;
          if (GROUPED && (!PAIR || leader)) {
            // claim the next tile and pass it to this CTA's consumers (and the peer's, for pairs)
            const bool ok = PAIR ? mbar_wait_cluster(&bar_tempty[tslot], tphase ^ 1, abort_p, status)
                                 : mbar_wait(&bar_tempty[tslot], tphase ^ 1, abort_p, status);
            if (!ok) goto producer_done;
            t = tnext < ntiles ? tnext : -1;
            tile_ring[tslot] = t;
            mbar_arrive(&bar_tfull[tslot]);
            if (PAIR) {
              st_shared_cluster(mapa_shared(&tile_ring[tslot], 1), t);
              mbar_arrive_cluster(mapa_shared(&bar_tfull[tslot], 1));  // release: the slot write first
            }
            if (++tslot == TRING) {
              tslot = 0;
              tphase ^= 1;
            }
            if (t >= 0) tnext = nunits + atomicAdd(G->tile_counter, 1);
          } else if (GROUPED) {
            // pair follower: the leader's tile, from this CTA's ring slot
            if (!mbar_wait_cluster(&bar_tfull[tslot], tphase, abort_p, status)) goto producer_done;
            t = tile_ring[tslot];
            // the release of the slot depends on the value read, so it cannot overtake the load
            if (t != INT_MIN) mbar_arrive_remote(mapa_shared(&bar_tempty[tslot], 0));
            if (++tslot == TRING) {
              tslot = 0;
              tphase ^= 1;
            }
          } else {
            t = tnext < ntiles ? tnext : -1;
            tnext += gridDim.x;
          }
          if (t < 0) break;
          const TileJob j = get_job<BN_, SUB_, GROUPED, PAIR>(t, tmA0, tmB0, P, G);
          if (j.skip) continue;
          if (GROUPED && j.tmA != last_map) {
            tensormap_acquire(j.tmA);
            tensormap_acquire(j.tmB);
            last_map = j.tmA;
          }
          // pairs: this CTA's 128 rows of the 256-row tile, and its half of the B columns
          const int arow = PAIR ? (j.tm * 2 + (int)rank) * BM : j.tm * BM;
          const int brow = PAIR ? j.tn * BN + (int)rank * (BN / 2) : j.tn * BN;
          for (int g = 2; g <= j.s + 1; ++g)
            for (int kbi = 0; kbi < j.KB; ++kbi)
              for (int p = 1; p < g; ++p) {
                const int kb = (g & 1) ? j.KB - 1 - kbi : kbi;  // snake: each group starts where the last ended
                if (!mbar_wait(&bar_empty[stage], phase ^ 1, abort_p, status)) goto producer_done;
                uint8_t* sA = smem + stage * K::STAGE_BYTES;
                const int nsub = kb == j.KB - 1 ? j.klast : K::SUB;  // an all-zero tail sub-tile is skipped
                const uint32_t bytes = (uint32_t)nsub * (K::SUBA_BYTES + K::SUBB_BYTES);
                if (PAIR) {
                  // both CTAs' copies complete on the leader's stage barrier, which each producer
                  // first arms with its own byte count
                  const uint32_t fbar = mapa_shared(&bar_full[stage], 0);
                  mbar_arrive_expect_tx_remote(fbar, bytes);
#pragma unroll
                  for (int h = 0; h < K::SUB; ++h)
                    if (h < nsub) {
                      tma_load_3d_pair(j.tmA, fbar, sA + h * K::SUBA_BYTES, kb * K::SK + h * BK, arow, p - 1);
                      tma_load_3d_pair(j.tmB, fbar, sA + K::A_BYTES + h * K::SUBB_BYTES, kb * K::SK + h * BK, brow,
                                       g - p - 1);
                    }
                } else {
                  mbar_arrive_expect_tx(&bar_full[stage], bytes);
#pragma unroll
                  for (int h = 0; h < K::SUB; ++h)
                    if (h < nsub) {
                      tma_load_3d(j.tmA, &bar_full[stage], sA + h * K::SUBA_BYTES, kb * K::SK + h * BK, arow, p - 1);
                      tma_load_3d(j.tmB, &bar_full[stage], sA + K::A_BYTES + h * K::SUBB_BYTES, kb * K::SK + h * BK,
                                  brow, g - p - 1);
                    }
                }
                ++issued;
                if (++stage == STAGES) {
                  stage = 0;
                  phase ^= 1;
                }
              }
        }
      producer_done:
        if (*abort_p) {
          if (!PAIR || leader) {
            // wait (bounded) for the copies still in flight into this CTA's shared memory
            uint32_t st = stage, ph = phase;
            for (long long i = 0; i < STAGES && i < issued; ++i) {
              if (st == 0) {
                st = STAGES - 1;
                ph ^= 1;
              } else {
                --st;
              }
              drain_wait(&bar_full[st], ph);
            }
          } else {
            // the follower's copies complete on the leader's barriers: give them time to land
            const long long t0 = clock64();
            while (clock64() - t0 < 2000000ll) {
            }
          }
        }
      }
    } else if (warp == 1) {
      // ---------------------------------------------------------------- MMA issuer
      // (pairs: the leader's lane issues for both CTAs; the follower's lane has no work)
      if (lane == 0 && (!PAIR || leader)) {
        uint32_t stage = 0, phase = 0;
        uint32_t acc_par = 0;  // bit b: parity of the next use of TMEM buffer b
        int buf = 0;
        uint32_t tslot = 0, tphase = 0;
        int tnext = blockIdx.x;
        for (;;) {
          int t;
          if (GROUPED) {
            if (!mbar_wait(&bar_tfull[tslot], tphase, abort_p, status)) goto mma_done;
            t = tile_ring[tslot];
            mbar_arrive(&bar_tempty[tslot]);
            if (++tslot == TRING) {
              tslot = 0;
              tphase ^= 1;
            }
          } else {
            t = tnext < ntiles ? tnext : -1;
            tnext += gridDim.x;
          }
          if (t < 0) break;
          const TileJob j = get_job<BN_, SUB_, GROUPED, PAIR>(t, tmA0, tmB0, P, G);
          if (j.skip) continue;
          for (int g = 2; g <= j.s + 1; ++g) {
            const int nblk = (g - 1) * j.KB;
            int b = 0;
            for (int kbi = 0; kbi < j.KB; ++kbi)
              for (int p = 1; p < g; ++p) {
                const int kb = (g & 1) ? j.KB - 1 - kbi : kbi;  // snake: each group starts where the last ended
                const bool chain_start = (b % K::SEG) == 0;
                if (chain_start) {
                  // pairs: both CTAs' epilogues release the buffer
                  if (!mbar_wait(&bar_acce[buf], ((acc_par >> buf) & 1) ^ 1, abort_p, status)) goto mma_done;
                  tc_fence_after();
                }
                if (!mbar_wait(&bar_full[stage], phase, abort_p, status)) goto mma_done;
                tc_fence_after();
                {
                  uint8_t* sA = smem + stage * K::STAGE_BYTES;
                  const int nsub = kb == j.KB - 1 ? j.klast : K::SUB;
                  const uint32_t dt = tmem + (uint32_t)(buf * BN);
#pragma unroll
                  for (int h = 0; h < K::SUB; ++h)
                    if (h < nsub) {
                      // pairs: the descriptors name this CTA's tiles; the MMA takes the peer's
                      // halves at the same shared-memory offsets
                      const uint64_t da = umma_desc_sw128(sA + h * K::SUBA_BYTES);
                      const uint64_t db = umma_desc_sw128(sA + K::A_BYTES + h * K::SUBB_BYTES);
#pragma unroll
                      for (int q = 0; q < BK / 16; ++q) {
                        const uint32_t acc = (!chain_start || h != 0 || q != 0) ? 1u : 0u;
                        if (PAIR)
                          umma_f16_pair(dt, da + (uint64_t)(2 * q), db + (uint64_t)(2 * q), K::IDESC, acc);
                        else
                          umma_f16(dt, da + (uint64_t)(2 * q), db + (uint64_t)(2 * q), K::IDESC, acc);
                      }
                    }
                }
                if (PAIR)
                  umma_commit_pair_mc(&bar_empty[stage], 3);  // the stage is free in both CTAs
                else
                  umma_commit(&bar_empty[stage]);
                if (++stage == STAGES) {
                  stage = 0;
                  phase ^= 1;
                }
                ++b;
                if (b % K::SEG == 0 || b == nblk) {
                  if (PAIR)
                    umma_commit_pair_mc(&bar_accf[buf], 3);  // the chain is ready in both CTAs' TMEM
                  else
                    umma_commit(&bar_accf[buf]);
                  acc_par ^= 1u << buf;
                  buf ^= 1;
                }
              }
          }
        }
      mma_done:
        // all MMAs issued by this thread must finish before TMEM is released
        if (PAIR)
          umma_commit_pair_mc(&bar_done, 1);
        else
          umma_commit(&bar_done);
        drain_wait(&bar_done, 0);
      }
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_EPILOGUE));
    const int ew = warp - 4;
    const int quad = warp & 3;
    const int chalf = ew >> 2;
    const int r = quad * 32 + lane;
    uint32_t acc_par = 0;
    int buf = 0;
    double* Rbase = Rws + (size_t)blockIdx.x * BM * BN * 2;  // room for 16 bytes per output
    const bool exact_mode = GROUPED ? false : (P->exact != 0);
    const bool defer_ok = GROUPED ? (G->defer != 0) : (P->defer != 0);
    // Active window words: in TMEM columns 2 BN .. 4 BN for 128-wide tiles (the accumulators
    // use 0 .. 2 BN; two 32-bit columns per output), else in the CTA's scratch tile.
    constexpr bool TMR = (BN == 128);
    constexpr int NCH = TMR ? 16 : 8;  // outputs per push chunk
    const uint32_t rtm = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(2 * BN + chalf * CPT * 2);
    // A plain push can be spread over the drains that precede the next push, so that it
    // overlaps the MMA warp's next chains instead of stalling them (the MMA runs at most one
    // chain ahead of the drains).  Other pushes run at once.
    int Gs[CPT];
    int pend_o = CPT, pend_chunk = CPT, pend_nout = CPT;
    PushArgs pend;
    const bool odd = (lane & 1) != 0;
    uint32_t tslot = 0, tphase = 0;
    int tnext = blockIdx.x;
    for (;;) {
      int t;
      if (GROUPED) {
        const bool ok = PAIR ? mbar_wait_cluster(&bar_tfull[tslot], tphase, abort_p, status)
                             : mbar_wait(&bar_tfull[tslot], tphase, abort_p, status);
        if (!ok) goto epi_done;
        t = tile_ring[tslot];
        __syncwarp();
        if (lane == 0) {
          if (PAIR) {
            // the leader's ring slot; the release depends on the value read (see the producer)
            if (t != INT_MIN) mbar_arrive_remote(mapa_shared(&bar_tempty[tslot], 0));
          } else {
            mbar_arrive(&bar_tempty[tslot]);
          }
        }
        if (++tslot == TRING) {
          tslot = 0;
          tphase ^= 1;
        }
      } else {
        t = tnext < ntiles ? tnext : -1;
        tnext += gridDim.x;
      }
      if (t < 0) break;
      const TileJob j = get_job<BN_, SUB_, GROUPED, PAIR>(t, tmA0, tmB0, P, G);
      if (j.skip) continue;
      const int s = j.s;
      const int push_segs = j.cplx ? 32 : 64;  // int32 group sums stay below 2^31
      // row of the (stacked) product; pairs: this CTA's 128 rows of the 256-row tile
      const int64_t grow = (int64_t)(PAIR ? j.tm * 2 + (int)rank : j.tm) * BM + r;
      const bool row_ok = grow < j.rows;
      const int64_t orow = j.cplx ? (grow >> 1) : grow;
      const int e_row = (row_ok && j.e != nullptr) ? j.e[orow] : 0;
      const int64_t gcol0 = (int64_t)j.tn * BN + chalf * CPT;
      const int win = window_len(s, (int64_t)j.KB * K::SK, j.cplx);
      const int nout = j.cplx ? CPT / 2 : CPT;  // outputs of this thread
      // scratch slots: S0 (first window, later the FP64 partial), S1 (windows 1, 2, ... when the
      // active window is not in TMEM)
      long long* S0t = reinterpret_cast<long long*>(Rbase) + (size_t)(j.cplx ? chalf * CPT / 2 : chalf * CPT) * BM + r;
      long long* S1t = S0t + (size_t)BM * BN;
      PushArgs pa;
      pa.rtm = rtm;
      pa.S0 = S0t;
      pa.gcol0 = gcol0;
      pa.orow = orow;
      pa.row_ok = row_ok;
      pa.unit_ab = j.beta_zero && j.a0 == 1.0 && j.a1 == 0.0;  // C = RN(T): no FP64 work
      pa.odd = odd;
      pa.ebase = e_row - 7 * (s + 1);
      for (int g = 2; g <= s + 1; ++g) {
        const int widx = (g - 2) / win, pos = (g - 2) % win;
        const int wlen = min(win, s - widx * win);
        pa.widx = widx;
        pa.wlen = wlen;
        pa.Ra = widx == 0 ? S0t : S1t;
        int Gr[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) Gr[c] = 0;
        const int nseg = nseg_of(g, j.KB, K::SEG);
        bool first_push = true;
        for (int seg = 0; seg < nseg; ++seg) {
          if (!mbar_wait(&bar_accf[buf], (acc_par >> buf) & 1, abort_p, status)) goto epi_done;
          tc_fence_after();
          {
            const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * BN + chalf * CPT);
#pragma unroll
            for (int cc = 0; cc < CPT / 32; ++cc) {
              uint32_t v[32];
              tmem_ld32(taddr + cc * 32, v);
              tmem_ld_wait();
#pragma unroll
              for (int i = 0; i < 32; ++i) Gr[cc * 32 + i] += __float2int_rn(__uint_as_float(v[i]));
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            if (PAIR)
              mbar_arrive_remote(mapa_shared(&bar_acce[buf], 0));  // the leader's MMA lane waits on it
            else
              mbar_arrive(&bar_acce[buf]);
          }
          acc_par ^= 1u << buf;
          buf ^= 1;
          const bool group_end = (seg == nseg - 1);
          const bool push_now = group_end || ((seg + 1) % push_segs) == 0;
          if (pend_o < pend_nout) {  // advance the pending push; complete it before the next one
            const int o1 = push_now ? pend_nout : min(pend_nout, pend_o + pend_chunk);
#pragma unroll 1
            for (int o = pend_o; o < o1; o += NCH) push_chunk<NCH, TMR>(Gs + (j.cplx ? 2 * o : o), o, pend, j);
            pend_o = o1;
          }
          if (!push_now) continue;
          const bool final_push = group_end && g == s + 1;
          const bool exact_now = exact_mode && s <= kExactMaxS;
          pa.first = first_push;
          pa.wstart = first_push && pos == 0;
          const bool win_end = group_end && pos == wlen - 1;
          pa.kind = final_push ? kFinal : !win_end ? kPlain : widx >= 1 ? kClose : TMR ? kSpill : kPlain;
          if (TMR && !exact_now && Gdbg == nullptr) {
            // TMEM-resident windows: every push goes straight from the registers.  The chunk
            // loop stays rolled (small code); after each chunk the array is rotated by one
            // chunk, so the chunk is always Gr[0 ..] and every index is a compile-time constant.
            const int W = j.cplx ? 2 : 1;  // group sums per output
#pragma unroll 1
            for (int o = 0; o < nout; o += NCH) {
              push_chunk<NCH, TMR>(Gr, o, pa, j);
#pragma unroll
              for (int c = 0; c < CPT - NCH; ++c) Gr[c] = Gr[c + NCH];
              if (W == 2) {
#pragma unroll
                for (int c = 0; c < CPT - NCH; ++c) Gr[c] = Gr[c + NCH];
              }
            }
#pragma unroll
            for (int c = 0; c < CPT; ++c) Gr[c] = 0;
            first_push = false;
            continue;
          }
          // ---- push the group sums into R (or, for inspection, export them) ----
          // Pushes happen once per group (per 64 chains at most): the sums move to a
          // thread-local array indexed at run time, so the FP64 work below runs in a rolled
          // loop with few live registers while Gr stays in registers for the drains above.
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            Gs[c] = Gr[c];
            Gr[c] = 0;
          }
          if (pa.kind == kPlain && !exact_now && Gdbg == nullptr) {
            // drains before the next push: the rest of this group, or the next group's chains
            const int left = group_end ? nseg_of(g + 1, j.KB, K::SEG) : nseg - (seg + 1);
            const int drains = min(left, push_segs);
            if (defer_ok && drains >= 2) {
              pend = pa;
              pend_o = 0;
              pend_nout = nout;
              pend_chunk = (nout + drains - 2) / (drains - 1);
              pend_chunk = (pend_chunk + NCH - 1) / NCH * NCH;
              first_push = false;
              continue;
            }
          }
          if (Gdbg != nullptr) {
            // a group longer than the int32 fold interval arrives in several pushes: the export
            // sums them in int64 (each output is written by this thread only)
#pragma unroll 1
            for (int c = 0; c < CPT; ++c) {
              const int64_t gc = gcol0 + c;
              if (row_ok && gc < j.cols) {
                int64_t* gp = Gdbg + ((int64_t)(g - 2) * j.rows + grow) * j.cols + gc;
                *gp = first_push ? (int64_t)Gs[c] : *gp + (int64_t)Gs[c];
              }
            }
          } else if (exact_now) {
            // correctly rounded mode: exact 128-bit Horner sum, one rounding at the end
            char* Rt = reinterpret_cast<char*>(Rbase) + ((size_t)(j.cplx ? chalf * CPT / 2 : chalf * CPT) * BM + r) * 16;
            const int ebase = e_row - 7 * (s + 1);
            if (!j.cplx) {
#pragma unroll 2
              for (int c = 0; c < CPT; ++c) {
                const int64_t col = gcol0 + c;
                const bool ok = row_ok && col < j.cols;
                const int E = final_push && ok ? ebase + __ldg(j.f + col) : 0;
                const double tv = horner_step(Rt + (size_t)c * BM * 16, Gs[c], true, first_push, g == 2, final_push, E);
                if (final_push && ok) {
                  double* cp = j.C + orow + col * j.ldc;
                  __stcs(cp, j.beta_zero ? j.a0 * tv : fma(j.a0, tv, j.b0 * *cp));
                }
              }
            } else {
#pragma unroll 2
              for (int c = 0; c < CPT / 2; ++c) {
                const int other = __shfl_xor_sync(0xffffffffu, Gs[2 * c + 1], 1);
                const int comb = odd ? (Gs[2 * c] + other) : (Gs[2 * c] - other);
                const int64_t jc = (gcol0 >> 1) + c;
                const bool ok = row_ok && jc < j.n;
                const int E = final_push && ok ? ebase + __ldg(j.f + jc) : 0;
                const double v = horner_step(Rt + (size_t)c * BM * 16, comb, true, first_push, g == 2, final_push, E);
                if (final_push) {
                  const double part = ok ? v : 0.0;
                  const double partner = __shfl_xor_sync(0xffffffffu, part, 1);
                  const double tr = odd ? partner : part, ti = odd ? part : partner;
                  if (ok) {
                    double* cp = j.C + 2 * (orow + jc * j.ldc);
                    double re = fma(j.a0, tr, -(j.a1 * ti));
                    double im = fma(j.a0, ti, j.a1 * tr);
                    if (!j.beta_zero) {
                      const double cr = cp[0], ci = cp[1];
                      re += fma(j.b0, cr, -(j.b1 * ci));
                      im += fma(j.b0, ci, j.b1 * cr);
                    }
                    __stcs(cp + (odd ? 1 : 0), odd ? im : re);
                  }
                }
              }
            }
          } else {
#pragma unroll 1
            for (int o = 0; o < nout; o += NCH) push_chunk<NCH, TMR>(Gs + (j.cplx ? 2 * o : o), o, pa, j);
          }
          first_push = false;
        }
      }
    }
  epi_done:;
  }

  tc_fence_before();
  __syncthreads();
  // pairs: neither CTA leaves (or frees TMEM) while the peer may still reach its shared memory
  // or the leader's MMAs its TMEM
  if (PAIR) {
    __syncwarp();
    cluster_sync_all();
  }
  if (warp == 1) {
    tc_fence_after();
    if (PAIR)
      tmem_dealloc_pair(tmem, K::TMEM_COLS);
    else
      tmem_dealloc(tmem, K::TMEM_COLS);
  }
}

// ------------------------------------------------------------------------ stacked group pairs
// Variant 5 (128 x 128 output tiles): the groups are taken two at a time.  For groups g and
// g + 1 every plane pair shares a plane with a neighbour: A_p meets B_{g-p} (group g) and
// B_{g+1-p} (group g + 1).  So one k sub-tile of a pass loads A_1 .. A_g and B_g .. B_1 once
// each and issues, for p = 1 .. g - 1, one N = 256 MMA whose B operand is the two consecutive
// B tiles [B_{g+1-p}; B_{g-p}] -- accumulator columns 0 .. 127 collect group g + 1, columns
// 128 .. 255 group g -- and, for p = g, an N = 128 MMA (A_g B_1, group g + 1); that last stage
// also loads the next k sub-tile's B_g, so only a pass's first stage issues no MMA.  Against the
// one-group schedule this halves the shared-memory fill (L2 -> SM bytes) and the MMA
// instructions per product.  The stage ring holds one A and one B sub-tile (64 k) per entry;
// a B tile is used by its own stage and the next, so the commit after a stage frees the entry
// of the stage before it.  Entry 0's B tile is also written to a mirror slot behind the last
// entry, so the two B tiles of a stage are adjacent across the end of the ring too.  A window
// with an odd number of groups ends with its first group alone (one N = 128 MMA per plane pair,
// into columns 128 .. 255): a tile then starts with a pass of two groups, whose chains are twice
// as long as a lone group's, so the two accumulators keep the tensor pipe busy longer while the
// epilogue rounds the previous tile.
//
// The two 256-column accumulators fill TMEM, so the int64 windows live in the epilogue's
// registers, and every drained chain is added into them directly: the window is linear in the
// group sums, W = sum_g 128^(gend - g) G_g, and a chain of groups g, g + 1 adds
// 128^(gend - g - 1) (128 c_g + c_{g+1}) exactly.  A chain covers whole k sweeps, at most
// 1024 products in each accumulator column.
namespace stk {
constexpr int NE = 6;                      // stage ring entries
constexpr uint32_t SLOT = BM * BK * 2;     // one 128-row x 64-k fp16 sub-tile (16 KB, one TMA box)
constexpr uint32_t A_OFF = 0, B_OFF = NE * SLOT;
// B slots: one per entry and a mirror of entry 0's behind the last, so that the B tiles of
// every two consecutive stages are adjacent (one N = 256 operand) also across the ring's end;
// behind them the epilogue's staging of the spilled first-window words (8 per thread)
constexpr uint32_t S0_OFF = (2 * NE + 1) * SLOT;
constexpr size_t SMEM = (size_t)S0_OFF + 8 * EPI_WARPS * 32 * sizeof(long long) + 1024;
constexpr uint32_t IDESC2 = umma_idesc_f16_f32(BM, 256), IDESC1 = umma_idesc_f16_f32(BM, 128);
constexpr int CHAIN_STAGES = CHAIN_K / BK;  // 64-k MMA stages per accumulator column and chain
constexpr int MAX_S = CHAIN_STAGES;          // a two-group sweep of g stages must fit one chain
constexpr int NOUT = 64;                     // outputs per epilogue thread (real; complex: 32)
constexpr uint64_t DSLOT = SLOT >> 4;         // descriptor start-address units per ring entry
static_assert(SMEM <= 227 * 1024, "stage ring");
static_assert(SMEM < (1u << 18), "descriptor start addresses stay within their 14-bit field");
}  // namespace stk

// The four K = 16 MMAs of one 64-wide k sub-tile; the first overwrites the accumulator when it
// starts a chain.
__device__ __forceinline__ void stk_mma4(uint32_t dt, uint64_t da, uint64_t db, uint32_t idesc, bool fresh) {
  umma_f16(dt, da, db, idesc, fresh ? 0u : 1u);
#pragma unroll
  for (int k16 = 1; k16 < BK / 16; ++k16) umma_f16(dt, da + (uint64_t)(2 * k16), db + (uint64_t)(2 * k16), idesc, 1u);
}

// Pass q of the window [wstart, wstart + wlen): the groups ga, ga + 1, or the lone group ga =
// wstart (last pass of a window with an odd count).
__device__ __forceinline__ void stk_pass(int wstart, int wlen, int q, int& ga, bool& two) {
  if (wlen & 1) {
    two = q < (wlen - 1) / 2;
    ga = two ? wstart + 1 + 2 * q : wstart;
  } else {
    two = true;
    ga = wstart + 2 * q;
  }
}
// Length of the first window.  With three or more windows every window but the last holds win
// groups, as in the one-group kernels (their FP64 continuation rounds per window, so the split
// must be the same for the same bits).  With two windows the exact sum is rounded once and any
// split into windows of at most win groups gives the same bits: the first takes one group
// less when that makes the second window's count even (a lone group of a later window pairs
// far more planes than the lone group 2 of the first).
__device__ __forceinline__ int stk_len0(int s, int win) {
  if (s <= win || s > 2 * win) return min(s, win);
  return (((win - s) & 1) && s - (win - 1) <= win) ? win - 1 : win;
}
// k sweeps per chain: a sweep adds ga (two groups) or ga - 1 (lone group) 64-k MMA stages to
// the accumulator columns that collect the most
__device__ __forceinline__ int stk_sweeps(int ga, bool two) { return stk::CHAIN_STAGES / (two ? ga : ga - 1); }

template <bool GROUPED>
__device__ __forceinline__ void stacked_body(const CUtensorMap* tmA0, const CUtensorMap* tmB0, const GemmArgs* P,
                                             const GroupArgs* G) {
  using namespace stk;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bar_full[NE], bar_empty[NE], bar_accf[2], bar_acce[2], bar_done;
  __shared__ __align__(8) uint64_t bar_tfull[TRING], bar_tempty[TRING];
  __shared__ int tile_ring[TRING];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  int* status = GROUPED ? G->status : P->status;
  double* Rws = GROUPED ? G->Rws : P->Rws;
  const int ntiles = GROUPED ? G->ntiles : (int)(((P->rows + BM - 1) / BM) * ((P->cols + 127) / 128));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NE; ++i) {
      mbar_init(&bar_full[i], 1);
      mbar_init(&bar_empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_accf[b], 1);
      mbar_init(&bar_acce[b], EPI_WARPS);
    }
    mbar_init(&bar_done, 1);
    for (int i = 0; i < TRING; ++i) {
      mbar_init(&bar_tfull[i], 1);
      mbar_init(&bar_tempty[i], 1 + EPI_WARPS);
    }
    abort_flag = 0;
    mbar_fence_init();
  }
  if (!GROUPED && warp == 0 && lane == 0) {
    tma_prefetch_desc(tmA0);
    tma_prefetch_desc(tmB0);
  }
  if (warp == 1) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* abort_p = &abort_flag;

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_PRODUCER));
    if (warp == 0) {
      // ---------------------------------------------------------------- TMA producer
      if (lane == 0) {
        uint32_t e = 0, eph = 0;
        long long issued = 0;
        const CUtensorMap* last_map = nullptr;
        uint32_t tslot = 0, tphase = 0;
        int tnext = blockIdx.x;
        for (;;) {
          int t;
          if (GROUPED) {
            if (!mbar_wait(&bar_tempty[tslot], tphase ^ 1, abort_p, status)) goto producer_done;
            t = tnext < ntiles ? tnext : -1;
            tile_ring[tslot] = t;
            mbar_arrive(&bar_tfull[tslot]);
            if (++tslot == TRING) {
              tslot = 0;
              tphase ^= 1;
            }
            if (t >= 0) tnext = (int)gridDim.x + atomicAdd(G->tile_counter, 1);
          } else {
            t = tnext < ntiles ? tnext : -1;
            tnext += gridDim.x;
          }
          if (t < 0) break;
          const TileJob j = get_job<128, 2, GROUPED>(t, tmA0, tmB0, P, G);
          if (j.skip) continue;
          if (GROUPED && j.tmA != last_map) {
            tensormap_acquire(j.tmA);
            tensormap_acquire(j.tmB);
            last_map = j.tmA;
          }
          const int KB = (j.KB - 1) * 2 + j.klast;  // 64-wide k sub-tiles
          const int arow = j.tm * BM, brow = j.tn * 128;
          const int win = window_len(j.s, (int64_t)j.KB * 128, j.cplx);
          int pc = 0;
          for (int wstart = 2, wlen = stk_len0(j.s, win); wstart <= j.s + 1;
               wstart += wlen, wlen = min(win, j.s + 2 - wstart)) {
            for (int q = 0; q < (wlen + 1) / 2; ++q, ++pc) {
              int ga;
              bool two;
              stk_pass(wstart, wlen, q, ga, two);
              for (int kbi = 0; kbi < KB; ++kbi) {
                const int kb = (pc & 1) ? KB - 1 - kbi : kbi;  // snake: a pass starts where the last ended
                const int kbn = (pc & 1) ? kb - 1 : kb + 1;    // the sweep's next k block
                // stage i: A_i (i >= 1) and B_{ga-i} (i <= ga - 1); with two groups, stage ga also
                // carries B_ga of the next k block, so only the pass's first sweep has a stage 0;
                // a lone group has none
                for (int i = (two && kbi == 0) ? 0 : 1; i <= (two ? ga : ga - 1); ++i) {
                  if (!mbar_wait(&bar_empty[e], eph ^ 1, abort_p, status)) goto producer_done;
                  const bool last = i == ga;  // two groups only
                  const bool hasA = i >= 1, hasB = last ? kbi + 1 < KB : true;
                  const bool mirror = hasB && e == 0;
                  mbar_arrive_expect_tx(&bar_full[e], (hasA ? SLOT : 0u) + (hasB ? SLOT : 0u) + (mirror ? SLOT : 0u));
                  if (hasA) tma_load_3d(j.tmA, &bar_full[e], smem + A_OFF + e * SLOT, kb * BK, arow, i - 1);
                  if (hasB) {
                    const int bk = (last ? kbn : kb) * BK, bz = last ? ga - 1 : ga - i - 1;
                    tma_load_3d(j.tmB, &bar_full[e], smem + B_OFF + e * SLOT, bk, brow, bz);
                    if (mirror) tma_load_3d(j.tmB, &bar_full[e], smem + B_OFF + NE * SLOT, bk, brow, bz);
                  }
                  ++issued;
                  if (++e == NE) {
                    e = 0;
                    eph ^= 1;
                  }
                }
              }
            }
          }
        }
      producer_done:
        if (*abort_p) {
          uint32_t st = e, ph = eph;
          for (long long i = 0; i < NE && i < issued; ++i) {
            if (st == 0) {
              st = NE - 1;
              ph ^= 1;
            } else {
              --st;
            }
            drain_wait(&bar_full[st], ph);
          }
        }
      }
    } else if (warp == 1) {
      // ---------------------------------------------------------------- MMA issuer
      if (lane == 0) {
        uint32_t e = 0, eph = 0;
        int eprev = -1;  // ring entry of the previous stage (freed by the next commit)
        const uint64_t dA0 = umma_desc_sw128(smem + A_OFF), dB0 = umma_desc_sw128(smem + B_OFF);
        uint32_t acc_par = 0;
        int buf = 0;
        uint32_t tslot = 0, tphase = 0;
        int tnext = blockIdx.x;
        for (;;) {
          int t;
          if (GROUPED) {
            if (!mbar_wait(&bar_tfull[tslot], tphase, abort_p, status)) goto mma_done;
            t = tile_ring[tslot];
            mbar_arrive(&bar_tempty[tslot]);
            if (++tslot == TRING) {
              tslot = 0;
              tphase ^= 1;
            }
          } else {
            t = tnext < ntiles ? tnext : -1;
            tnext += gridDim.x;
          }
          if (t < 0) break;
          const TileJob j = get_job<128, 2, GROUPED>(t, tmA0, tmB0, P, G);
          if (j.skip) continue;
          const int KB = (j.KB - 1) * 2 + j.klast;
          const int win = window_len(j.s, (int64_t)j.KB * 128, j.cplx);
          for (int wstart = 2, wlen = stk_len0(j.s, win); wstart <= j.s + 1;
               wstart += wlen, wlen = min(win, j.s + 2 - wstart)) {
            for (int q = 0; q < (wlen + 1) / 2; ++q) {
              int ga;
              bool two;
              stk_pass(wstart, wlen, q, ga, two);
              const int spc = stk_sweeps(ga, two);
              bool fresh = false;  // the next MMA starts a chain (overwrites the accumulator)
              int left = 0;        // k sweeps left in the current chain
              for (int kbi = 0; kbi < KB; ++kbi) {
                if (left == 0) {
                  if (!mbar_wait(&bar_acce[buf], ((acc_par >> buf) & 1) ^ 1, abort_p, status)) goto mma_done;
                  tc_fence_after();
                  fresh = true;
                  left = spc;
                }
                const uint32_t dt = tmem + (uint32_t)(buf * 256);
                // descriptors advance by SLOT >> 4 per ring entry (the start-address field)
                if (!two) {
                  // lone group: A_i B_{ga-i} into columns 128 .. 255
                  for (int i = 1; i < ga; ++i) {
                    if (!mbar_wait(&bar_full[e], eph, abort_p, status)) goto mma_done;
                    tc_fence_after();
                    stk_mma4(dt + 128, dA0 + e * DSLOT, dB0 + e * DSLOT, IDESC1, fresh);
                    fresh = false;
                    if (eprev >= 0) umma_commit(&bar_empty[eprev]);
                    eprev = (int)e;
                    if (++e == NE) {
                      e = 0;
                      eph ^= 1;
                    }
                  }
                } else {
                  if (kbi == 0) {
                    // the pass's stage 0: B_ga only, no MMA; it frees the previous stage's entry
                    if (!mbar_wait(&bar_full[e], eph, abort_p, status)) goto mma_done;
                    tc_fence_after();
                    if (eprev >= 0) umma_commit(&bar_empty[eprev]);
                    eprev = (int)e;
                    if (++e == NE) {
                      e = 0;
                      eph ^= 1;
                    }
                  }
                  for (int i = 1; i < ga; ++i) {
                    if (!mbar_wait(&bar_full[e], eph, abort_p, status)) goto mma_done;
                    tc_fence_after();
                    // [B_{ga+1-i}; B_{ga-i}] are adjacent slots (at the ring's end, the last slot
                    // and entry 0's mirror): one N = 256 operand
                    stk_mma4(dt, dA0 + e * DSLOT, dB0 + (uint32_t)eprev * DSLOT, IDESC2, fresh);
                    fresh = false;
                    umma_commit(&bar_empty[eprev]);  // the previous entry's B was last used here
                    eprev = (int)e;
                    if (++e == NE) {
                      e = 0;
                      eph ^= 1;
                    }
                  }
                  // stage ga: A_ga B_1 (group ga + 1 only) into columns 0 .. 127; its B slot holds
                  // the next sweep's B_ga
                  if (!mbar_wait(&bar_full[e], eph, abort_p, status)) goto mma_done;
                  tc_fence_after();
                  stk_mma4(dt, dA0 + e * DSLOT, dB0 + (uint32_t)eprev * DSLOT, IDESC1, false);
                  umma_commit(&bar_empty[eprev]);
                  eprev = (int)e;
                  if (++e == NE) {
                    e = 0;
                    eph ^= 1;
                  }
                }
                if (--left == 0 || kbi == KB - 1) {
                  umma_commit(&bar_accf[buf]);
                  acc_par ^= 1u << buf;
                  buf ^= 1;
                  left = 0;
                }
              }
            }
          }
        }
      mma_done:
        umma_commit(&bar_done);
        drain_wait(&bar_done, 0);
      }
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_EPILOGUE));
    const int ew = warp - 4;
    const int quad = warp & 3;
    const int chalf = ew >> 2;
    const int r = quad * 32 + lane;
    uint32_t acc_par = 0;
    int buf = 0;
    double* Rbase = Rws + (size_t)blockIdx.x * BM * 128 * 2;
    const bool odd = (lane & 1) != 0;
    uint32_t tslot = 0, tphase = 0;
    int tnext = blockIdx.x;
    for (;;) {
      int t;
      if (GROUPED) {
        if (!mbar_wait(&bar_tfull[tslot], tphase, abort_p, status)) goto epi_done;
        t = tile_ring[tslot];
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_tempty[tslot]);
        if (++tslot == TRING) {
          tslot = 0;
          tphase ^= 1;
        }
      } else {
        t = tnext < ntiles ? tnext : -1;
        tnext += gridDim.x;
      }
      if (t < 0) break;
      const TileJob j = get_job<128, 2, GROUPED>(t, tmA0, tmB0, P, G);
      if (j.skip) continue;
      const int s = j.s;
      const int KB = (j.KB - 1) * 2 + j.klast;
      const int64_t grow = (int64_t)j.tm * BM + r;
      const bool row_ok = grow < j.rows;
      const int64_t orow = j.cplx ? (grow >> 1) : grow;
      const int e_row = (row_ok && j.e != nullptr) ? j.e[orow] : 0;
      const int win = window_len(s, (int64_t)j.KB * 128, j.cplx);
      const int nout = j.cplx ? NOUT / 2 : NOUT;
      PushArgs pa;
      pa.S0 = reinterpret_cast<long long*>(Rbase) + (size_t)(j.cplx ? chalf * NOUT / 2 : chalf * NOUT) * BM + r;
      pa.gcol0 = (int64_t)j.tn * 128 + chalf * NOUT;
      pa.orow = orow;
      pa.row_ok = row_ok;
      pa.unit_ab = j.beta_zero && j.a0 == 1.0 && j.a1 == 0.0;
      pa.odd = odd;
      pa.ebase = e_row - 7 * (s + 1);
      const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(chalf * NOUT);
      // the column exponents of this warp's outputs, loaded now (their latency hides behind the
      // drains) one or two per lane and handed out by shuffles when C is written
      int fcol[2];
      {
        const int64_t c0 = j.cplx ? (pa.gcol0 >> 1) : pa.gcol0;
        const int64_t climit = j.cplx ? j.n : j.cols;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t c = c0 + h * 32 + lane;
          fcol[h] = (c < climit && (h == 0 || !j.cplx)) ? __ldg(j.f + c) : 0;
        }
      }
      // real tiles: the warp finishes only the 8-output chunks that reach into C, and none when
      // its 32 rows all lie past C's last row (warp-uniform; the padding's sums are never written)
      int nfin = nout;
      if (!j.cplx) {
        int nvalid = (int)max((int64_t)0, min((int64_t)NOUT, j.cols - pa.gcol0));
        if ((int64_t)j.tm * BM + quad * 32 >= j.rows) nvalid = 0;
        nfin = (nvalid + 7) & ~7;
      }
      int widx = 0;
      for (int wstart = 2, wlen = stk_len0(s, win); wstart <= s + 1;
           wstart += wlen, wlen = min(win, s + 2 - wstart), ++widx) {
        const int gend = wstart + wlen - 1;
        long long W[NOUT];
#pragma unroll
        for (int c = 0; c < NOUT; ++c) W[c] = 0;
        long long* sbuf = reinterpret_cast<long long*>(smem + S0_OFF) + ew * 32 + lane;
        if (widx >= 1 && nfin > 0) {  // the first chunk's spilled words, staged while this window drains
#pragma unroll
          for (int i = 0; i < 8; ++i) cp_async8(sbuf + i * EPI_WARPS * 32, pa.S0 + (size_t)i * BM);
          cp_async_commit();
        }
        for (int q = 0; q < (wlen + 1) / 2; ++q) {
          int ga;
          bool two;
          stk_pass(wstart, wlen, q, ga, two);
          const int spc = stk_sweeps(ga, two);
          const int nch = (KB + spc - 1) / spc;
          // real pair passes run in increasing ga and close the window (a lone group runs last),
          // so they accumulate by Horner's rule: W <- 128^2 W before the pass, chains added
          // unshifted; the lone group and complex data add their chains shifted to their weight
          const bool horner = two && !j.cplx;
          const int sh = horner ? 0 : 7 * (gend - ga - (two ? 1 : 0));
          if (horner) {
#pragma unroll
            for (int c = 0; c < NOUT; ++c) W[c] = (long long)((unsigned long long)W[c] << 14);
          }
          for (int ch = 0; ch < nch; ++ch) {
            if (!mbar_wait(&bar_accf[buf], (acc_par >> buf) & 1, abort_p, status)) goto epi_done;
            tc_fence_after();
            const uint32_t ta = tl + (uint32_t)(buf * 256);
#pragma unroll
            for (int cc = 0; cc < NOUT / 16; ++cc) {
              uint32_t h1[16], h0[16];
              tmem_ld16(ta + 128 + cc * 16, h1);  // group ga
              if (two) tmem_ld16(ta + cc * 16, h0);  // group ga + 1
              tmem_ld_wait();
              if (cc == NOUT / 16 - 1) {
                // the accumulator is read: the MMA lane may refill it while this chunk converts
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_acce[buf]);
              }
              if (horner) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  // a chain sums at most 1024 products of digits |d| <= 127 (< 2^24), so
                  // 128 c_ga + c_{ga+1} stays below 2^31 and combines in 32 bits
                  const int v = __float2int_rn(__uint_as_float(h1[i])) * 128 + __float2int_rn(__uint_as_float(h0[i]));
                  W[cc * 16 + i] += (long long)v;
                }
              } else if (!j.cplx) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  const long long v = __float2int_rn(__uint_as_float(h1[i]));
                  W[cc * 16 + i] += (long long)((unsigned long long)v << sh);
                }
              } else {
                // (Re, Im) of 8 outputs: even lanes Re = P_rr - P_ii, odd lanes Im = P_ir + P_ri
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  const int a1 = __float2int_rn(__uint_as_float(h1[2 * i]));
                  const int b1 = __shfl_xor_sync(0xffffffffu, __float2int_rn(__uint_as_float(h1[2 * i + 1])), 1);
                  const long long v1 = odd ? (long long)a1 + b1 : (long long)a1 - b1;
                  long long v = v1;
                  if (two) {
                    const int a0 = __float2int_rn(__uint_as_float(h0[2 * i]));
                    const int b0 = __shfl_xor_sync(0xffffffffu, __float2int_rn(__uint_as_float(h0[2 * i + 1])), 1);
                    v = v1 * 128 + (odd ? (long long)a0 + b0 : (long long)a0 - b0);
                  }
                  W[cc * 8 + i] += (long long)((unsigned long long)v << sh);
                }
              }
            }
            acc_par ^= 1u << buf;
            buf ^= 1;
          }
        }
        // the window is complete: spill the first one, close a later one into the FP64
        // partial, or round the last one and write C (chunks of 8 outputs, the array rotated
        // after each so every index stays a compile-time constant)
        pa.widx = widx;
        pa.wlen = wlen;
        pa.kind = gend == s + 1 ? kFinal : widx == 0 ? kSpill : kClose;
        // from the second window on, the spilled first-window words of the next chunk are
        // copied into shared memory while this chunk is rounded (cp.async: no registers held);
        // the first chunk's copies were issued when the window started
#pragma unroll 1
        for (int o = 0; o < nfin; o += 8) {
          long long s0c[8];
          int fe[8];
          const int fsrc = o < 32 ? fcol[0] : fcol[1];
          if (widx >= 1) {
            cp_async_wait_all();
#pragma unroll
            for (int i = 0; i < 8; ++i) s0c[i] = sbuf[i * EPI_WARPS * 32];
            if (o + 8 < nfin) {
              // the next copies overwrite these slots: their addresses depend on the last word
              // read, so they issue only once the reads have returned
              uint32_t dep = (uint32_t)s0c[7];
              asm volatile("and.b32 %0, %0, 0;" : "+r"(dep));
#pragma unroll
              for (int i = 0; i < 8; ++i)
                cp_async8(sbuf + dep + i * EPI_WARPS * 32, pa.S0 + (size_t)(o + 8 + i) * BM);
              cp_async_commit();
            }
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) s0c[i] = 0ll;
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) fe[i] = __shfl_sync(0xffffffffu, fsrc, (o + i) & 31);
          window_out<8, false, true>(W, o, pa, j, s0c, fe);
#pragma unroll
          for (int c = 0; c < NOUT - 8; ++c) W[c] = W[c + 8];
        }
      }
    }
  epi_done:
    cp_async_wait_all();  // no staging copy is left in flight (an aborted tile may leave one)
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

template <int BN_, int SUB_>
__global__ void __launch_bounds__(THREADS, 1)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const GemmArgs P) {
  if (P.nonfinite != nullptr && *P.nonfinite) return;  // the native FP64 kernel handles this call
  gemm_body<BN_, SUB_, false>(&tmA, &tmB, &P, nullptr);
}

template <int BN_, int SUB_>
__global__ void __launch_bounds__(THREADS, 1) slice_gemm_grouped_kernel(const GroupArgs G) {
  if (G.run != nullptr && *G.run == 0) return;  // a re-run launch with nothing to re-run
  gemm_body<BN_, SUB_, true>(nullptr, nullptr, nullptr, &G);
}

// CTA pairs: 2-CTA clusters over 256 x 128 pair tiles.  Both CTAs read the same run flag, so a
// gated launch returns from both before either touches the other.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1) slice_gemm_pair_kernel(const GroupArgs G) {
  if (G.run != nullptr && *G.run == 0) return;
  gemm_body<128, 2, true, true>(nullptr, nullptr, nullptr, &G);
}

// Stacked group pairs (variant 5), one GEMM or a grouped list of tiles.
__global__ void __launch_bounds__(THREADS, 1)
    slice_gemm_stacked_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                              const GemmArgs P) {
  if (P.nonfinite != nullptr && *P.nonfinite) return;
  stacked_body<false>(&tmA, &tmB, &P, nullptr);
}
__global__ void __launch_bounds__(THREADS, 1) slice_gemm_grouped_stacked_kernel(const GroupArgs G) {
  if (G.run != nullptr && *G.run == 0) return;
  stacked_body<true>(nullptr, nullptr, nullptr, &G);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

template <typename Kern>
cudaError_t set_smem_once(Kern k, size_t bytes, bool& done) {
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

}  // namespace

int slice_gemm_tile_m() { return BM; }
int slice_gemm_tile_n() { return 256; }
int slice_gemm_tile_n_of(int variant) { return ((variant & 1) || variant == kPairVariant) ? 128 : 256; }
int slice_gemm_tile_m_of(int variant) { return variant == kPairVariant ? 2 * BM : BM; }
int stacked_max_slices() { return stk::MAX_S; }

// CTAs of the pair variant that can be resident at once (2 per cluster), queried once per process.
int pair_max_ctas() {
  static int n = -1;
  if (n < 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = Cfg<128, 2, true>::SMEM;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, slice_gemm_pair_kernel, &cfg) != cudaSuccess || clusters <= 0) {
      cudaGetLastError();
      clusters = 0;
    }
    n = 2 * clusters;
  }
  return n;
}
size_t slice_gemm_smem_bytes() { return Cfg<256, 1>::SMEM; }

// Tensor map of a digit-plane set.  Half of the groups sweep k backwards, so a promotion wider
// than one 128-byte row segment of a 64-wide box fetches k that the sweep has already passed.
// That costs on short k (256-byte promotion: the learned step over 2048 GEMMs with k <= 2048 is
// 1 ms slower) and pays on long k, where it halves the L2 requests of a long sweep (256-byte
// promotion: the 8192^3 launch is 19.5 -> 18.9 ms).
constexpr int64_t kWidePromotionMinK = 2049;
cudaError_t make_digit_tmap(CUtensorMap* map, const __half* D, int64_t k, int64_t rows, int64_t Kp, int s,
                            int box_rows) {
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const CUtensorMapL2promotion promo =
      k >= kWidePromotionMinK ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
  cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)s};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)(rows * Kp * 2)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<__half*>(D), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, promo,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {
// Kernel instance of a variant: bit 0 -> 128-wide tiles; bit 1 -> deferred pushes (256-wide,
// a kernel argument) or one 64-wide k sub-tile per stage with a deeper pipeline (128-wide).
template <bool GROUPED, int BN_, int SUB_>
cudaError_t launch_one(const CUtensorMap* tmA, const CUtensorMap* tmB, const GemmArgs* a, const GroupArgs* g,
                       int grid, cudaStream_t st) {
  using K = Cfg<BN_, SUB_>;
  static bool done = false;
  cudaError_t e;
  if (GROUPED) {
    if ((e = set_smem_once(slice_gemm_grouped_kernel<BN_, SUB_>, K::SMEM, done)) != cudaSuccess) return e;
    { slice_gemm_grouped_kernel<BN_, SUB_><<<grid, THREADS, K::SMEM, st>>>(*g); note_launch(); }
  } else {
    if ((e = set_smem_once(slice_gemm_kernel<BN_, SUB_>, K::SMEM, done)) != cudaSuccess) return e;
    { slice_gemm_kernel<BN_, SUB_><<<grid, THREADS, K::SMEM, st>>>(*tmA, *tmB, *a); note_launch(); }
  }
  return cudaGetLastError();
}
template <bool GROUPED>
cudaError_t launch_stacked(const CUtensorMap* tmA, const CUtensorMap* tmB, const GemmArgs* a, const GroupArgs* g,
                           int grid, cudaStream_t st) {
  static bool done = false;
  cudaError_t e;
  if (GROUPED) {
    if ((e = set_smem_once(slice_gemm_grouped_stacked_kernel, stk::SMEM, done)) != cudaSuccess) return e;
    slice_gemm_grouped_stacked_kernel<<<grid, THREADS, stk::SMEM, st>>>(*g);
  } else {
    if ((e = set_smem_once(slice_gemm_stacked_kernel, stk::SMEM, done)) != cudaSuccess) return e;
    slice_gemm_stacked_kernel<<<grid, THREADS, stk::SMEM, st>>>(*tmA, *tmB, *a);
  }
  note_launch();
  return cudaGetLastError();
}
template <bool GROUPED>
cudaError_t launch_variant(int variant, const CUtensorMap* tmA, const CUtensorMap* tmB, const GemmArgs* a,
                           const GroupArgs* g, int grid, cudaStream_t st) {
  if (variant == kStackedVariant) return launch_stacked<GROUPED>(tmA, tmB, a, g, grid, st);
  if (!(variant & 1)) return launch_one<GROUPED, 256, 1>(tmA, tmB, a, g, grid, st);
  if (variant & 2) return launch_one<GROUPED, 128, 1>(tmA, tmB, a, g, grid, st);
  return launch_one<GROUPED, 128, 2>(tmA, tmB, a, g, grid, st);
}
}  // namespace

// Shared-memory opt-in for every kernel instance, once per process (outside any graph capture).
cudaError_t prepare_kernels() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(slice_gemm_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg<128, 2, true>::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(slice_gemm_stacked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stk::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(slice_gemm_grouped_stacked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stk::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(slice_gemm_kernel<256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg<256, 1>::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(slice_gemm_kernel<128, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg<128, 1>::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(slice_gemm_kernel<128, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg<128, 2>::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(slice_gemm_grouped_kernel<256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg<256, 1>::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(slice_gemm_grouped_kernel<128, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg<128, 1>::SMEM)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(slice_gemm_grouped_kernel<128, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Cfg<128, 2>::SMEM);
}

cudaError_t launch_slice_gemm(const CUtensorMap& tmA, const CUtensorMap& tmB, const GemmArgs& a, cudaStream_t st) {
  if (a.grid <= 0) return cudaSuccess;
  // the stacked kernel has no exact 128-bit mode and no group-product export; both, and slice
  // counts above its limit, run on the 128-wide one-group kernel (same tiles, same bits)
  const int v = (a.variant == kStackedVariant && (a.exact || a.Gdbg != nullptr || a.s > stacked_max_slices()))
                    ? 1 : a.variant;
  return launch_variant<false>(v, &tmA, &tmB, &a, nullptr, a.grid, st);
}

cudaError_t launch_slice_gemm_grouped(const GroupArgs& g, int variant, int grid, cudaStream_t st) {
  if (grid <= 0 || g.ntiles <= 0) return cudaSuccess;
  if (variant == kPairVariant) {
    if (grid % 2) return cudaErrorInvalidValue;  // whole clusters
    static bool done = false;
    cudaError_t e = set_smem_once(slice_gemm_pair_kernel, Cfg<128, 2, true>::SMEM, done);
    if (e != cudaSuccess) return e;
    slice_gemm_pair_kernel<<<grid, THREADS, Cfg<128, 2, true>::SMEM, st>>>(g);
    note_launch();
    return cudaGetLastError();
  }
  return launch_variant<true>(variant, nullptr, nullptr, nullptr, &g, grid, st);
}

}  // namespace ozg
