// Batched companions of the split, native and check kernels for the grouped GEMM: one launch
// covers every call of a batch (a device-side job table plus a prefix sum of work units per job;
// each CTA finds its job by binary search), so a batch of thousands of uneven GEMMs costs a
// handful of launches and captures into a short CUDA graph.
//   * split: the same exponents and digits as the single-call kernels (Sec. 2.2's split), one
//     job per operand;
//   * native: FP64 GEMM (real) for the calls whose inputs held Inf/NaN, on a device-compacted list;
//   * check: the sampled double-double error of every call (one warp per sample).
#include "ozg_internal.h"
#include "ozg_split_dev.cuh"

namespace ozg {
namespace {

// largest j with prefix[j] <= unit (prefix[0] = 0, prefix[njobs] = total)
__device__ __forceinline__ int find_job(const int64_t* prefix, int njobs, int64_t unit) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= unit)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// element (i, l) of the job's op(X) as raw bits; complex gives (re, im) with conjugation applied
__device__ __forceinline__ void load_elem(const SplitArgs& J, int64_t i, int64_t l, uint64_t& re, uint64_t& im) {
  if (!J.cplx) {
    const uint64_t* p = reinterpret_cast<const uint64_t*>(J.X);
    re = __ldg(J.strided ? p + i + l * J.ld : p + l + i * J.ld);
    im = 0;
  } else {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(J.X);
    ulonglong2 v = __ldg(J.strided ? p + i + l * J.ld : p + l + i * J.ld);
    re = v.x;
    im = J.conj ? (v.y ^ 0x8000000000000000ull) : v.y;
  }
}

// Row maxima.  A unit is 32 rows x 128 k of a strided job (lanes = consecutive rows, the eight
// warps interleave along k, 16 loads in flight per thread) or 8 rows x 1024 k of a contiguous
// job (a warp per row, lanes along k).  Partial maxima merge by atomicMax into the zeroed maxbits.
__global__ void __launch_bounds__(256) rowmax_batched(const SplitArgs* jobs, const int2* units) {
  const int2 ur = units[blockIdx.x];
  const SplitArgs J = jobs[ur.x];
  const int64_t u = ur.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long mx = 0;
  if (J.strided) {
    __shared__ unsigned long long red[8][32];
    const int64_t kt = (J.k + kRmStridedK - 1) / kRmStridedK;
    const int64_t row = (u / kt) * 32 + lane, l0 = (u % kt) * kRmStridedK + w;
    if (row < J.rows) {
#pragma unroll
      for (int i = 0; i < kRmStridedK / 8; ++i) {
        const int64_t l = l0 + 8 * i;
        if (l < J.k) {
          uint64_t re, im;
          load_elem(J, row, l, re, im);
          re &= kAbsMask;
          im &= kAbsMask;
          re = re > im ? re : im;
          mx = re > mx ? re : mx;
        }
      }
    }
    red[w][lane] = mx;
    __syncthreads();
    if (w == 0 && row < J.rows) {
#pragma unroll
      for (int i = 1; i < 8; ++i) mx = red[i][lane] > mx ? red[i][lane] : mx;
      if (mx) {
        atomicMax(&J.maxbits[row], mx);
        if (mx >= kInfBits) atomicExch(J.nonfinite, 1);
      }
    }
  } else {
    const int64_t kt = (J.k + kRmContigK - 1) / kRmContigK;
    const int64_t row = (u / kt) * 8 + w, l0 = (u % kt) * kRmContigK + lane;
    if (row >= J.rows) return;
#pragma unroll 8
    for (int i = 0; i < kRmContigK / 32; ++i) {
      const int64_t l = l0 + 32 * i;
      if (l < J.k) {
        uint64_t re, im;
        load_elem(J, row, l, re, im);
        re &= kAbsMask;
        im &= kAbsMask;
        re = re > im ? re : im;
        mx = re > mx ? re : mx;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = t > mx ? t : mx;
    }
    if (lane == 0 && mx) {
      atomicMax(&J.maxbits[row], mx);
      if (mx >= kInfBits) atomicExch(J.nonfinite, 1);
    }
  }
}

// Fused statistics of whole rows (real jobs with k <= kStatsK).  A unit is a block of rows of
// one job; its CTA reads them once and writes their maxima (from which the split's exponents
// come) and, for a learned call, adds the rows' within-row exponent gaps e_i - E(x_il) to the
// selector's 10-bin histogram (bins of 4, the last holding gaps >= 36 and zeros) -- the same
// counts as the two-pass form (row maxima, then a histogram pass over the operand again).
// The gap needs e_i, known only once the whole row has been read.  So each element's exponent is
// kept in shared memory as one byte, E(chunk max) - E(x) capped at 63 (plus 128 for a slot past
// the row's end), beside the exponent of its 16-element chunk's maximum; then gap = (e_i -
// E(chunk max)) + byte, exactly while it is below 36 and >= 36 whenever the byte was capped.
// With e_i - E(chunk max) also capped at 63, four bytes add without carries in one 32-bit add,
// and gap / 4 indexes a 64-entry table (bins 0 .. 8, bin 9 for 9 .. 31, nothing for the slots
// past the row's end at 32 .. 63).
// Only the high 32-bit word of each element is loaded: it holds the exponent field.  When the
// chunk's maximum has a biased exponent >= 36, the biased exponents give every byte exactly
// (a subnormal or zero element then gets a byte >= 36, its true gap being larger), and that
// maximum's high word has the same frexp exponent as the full value.  Chunks with a smaller
// maximum (below 2^-987) reload their full words and take the exact path.
// Thread layout: strided jobs (adjacent rows adjacent in memory) 16 rows x 16 column phases, so
// a warp's load covers two 128-byte column segments; contiguous jobs 8 rows (a warp each) x 32
// phases along k.  Thread (r, ph) takes elements l = ph + P i of its row, 16 loads in flight.
constexpr int kStatsThreads = 256, kStatsChunk = 16;
constexpr int kStatsChunks = kStatsK / 16 / kStatsChunk;  // chunks per thread at most (strided)
constexpr size_t kStatsHistSmem = (size_t)kStatsChunks * kStatsThreads * (sizeof(short) + kStatsChunk);
constexpr uint32_t kFastMaxHi = 36u << 20;  // high word of 2^(36 - 1023): smallest fast-path chunk maximum
static_assert(kStatsK % (16 * kStatsChunk) == 0, "whole chunks");
// a thread counts at most ceil(k / 16) elements in each of stats_blocks_per_unit(k) blocks of a
// unit: at most 128 for k <= kStatsK, and 1024 / k * ceil(k / 16) <= 128 below
static_assert(kStatsK / 16 < 256 && 2 * kStatsBlockElems / 16 < 256, "per-thread bin counts fit 8-bit fields");

extern __shared__ __align__(16) uint8_t stats_smem[];

// 0x80 in the bytes of a four-byte word whose slots lie past the row's end (valid = slots of the
// word before the end; <= 0: all four past it)
__device__ __forceinline__ uint32_t past_end_bytes(int valid) {
  return valid >= 4 ? 0u : (valid <= 0 ? 0x80808080u : 0x80808080u << (8 * valid));
}

// Exact path of one chunk (its maximum is subnormal, zero or below 2^-987): the full words, the
// frexp exponents, and the chunk's bytes when hist is set.  Returns the chunk maximum's bits.
__device__ __noinline__ uint64_t stats_chunk_exact(const uint64_t* p, int64_t step, int i0, int n_t, bool hist,
                                                   short* cmx, uint32_t* bytes, int c, int tid) {
  uint64_t v[kStatsChunk];
  uint64_t cm = 0;
#pragma unroll
  for (int q = 0; q < kStatsChunk; ++q) {
    v[q] = i0 + q < n_t ? (__ldg(p + (int64_t)(i0 + q) * step) & kAbsMask) : 0ull;
    cm = v[q] > cm ? v[q] : cm;
  }
  if (hist) {
    const int ecm = exponent_from_maxbits(cm);
    cmx[c * kStatsThreads + tid] = cm ? (short)ecm : (short)-32768;  // all-zero chunk: every gap huge
#pragma unroll
    for (int w4 = 0; w4 < kStatsChunk / 4; ++w4) {
      uint32_t word = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint64_t x = v[4 * w4 + b];
        const int d = x ? min(63, ecm - exponent_from_maxbits(x)) : 63;
        word |= (uint32_t)d << (8 * b);
      }
      bytes[(4 * c + w4) * kStatsThreads + tid] = word | past_end_bytes(n_t - i0 - 4 * w4);
    }
  }
  return cm;
}

template <bool HIST>
__device__ __forceinline__ void stats_unit(const SplitArgs& J, int64_t unit) {
  __shared__ unsigned long long red[8][16];
  __shared__ unsigned int sh[10];
  __shared__ uint4 onehot[64];  // gap / 4 -> +1 in its bin's 8-bit field of (bins 0-3, 4-7, 8-9)
  short* cmx = reinterpret_cast<short*>(stats_smem);  // [chunk][tid]: frexp exponent of the chunk max
  uint32_t* bytes = reinterpret_cast<uint32_t*>(stats_smem + kStatsChunks * kStatsThreads * sizeof(short));  // [word][tid]
  const int tid = threadIdx.x;
  if (HIST && tid < 10) sh[tid] = 0;
  if (HIST && tid < 64) {
    const int bin = tid < 9 ? tid : (tid < 32 ? 9 : -1);  // -1: a slot past the row's end
    uint4 o = make_uint4(0, 0, 0, 0);
    if (bin >= 0 && bin < 4) o.x = 1u << (8 * bin);
    else if (bin >= 4 && bin < 8) o.y = 1u << (8 * (bin - 4));
    else if (bin >= 8) o.z = 1u << (8 * (bin - 8));
    onehot[tid] = o;
  }
  const bool hist = HIST && J.hist != nullptr;
  const bool strided = J.strided != 0;
  const int P = strided ? 16 : 32;
  const int R = kStatsThreads / P;  // rows per block
  const int r = strided ? (tid & 15) : (tid >> 5);
  const int ph = strided ? (tid >> 4) : (tid & 31);
  const int lane = tid & 31, warp = tid >> 5;
  const int n_t = ph < J.k ? (int)((J.k - 1 - ph) / P + 1) : 0;  // elements of a full row per thread
  const int nch = (n_t + kStatsChunk - 1) / kStatsChunk;
  const int64_t step = strided ? (int64_t)P * J.ld : (int64_t)P;
  const int64_t nrb = (J.rows + R - 1) / R, G = stats_blocks_per_unit(J.k);
  const int64_t rb_end = min(nrb, (unit + 1) * G);
  uint32_t c0 = 0, c1 = 0, c2 = 0;  // this thread's 8-bit counts of bins 0-3, 4-7, 8-9 over the unit
  if (HIST) __syncthreads();  // the shared counters and table are ready before their first use
  for (int64_t rb = unit * G; rb < rb_end; ++rb) {
    const int64_t row = rb * R + r;
    const bool row_ok = row < J.rows;
    const int nt = row_ok ? n_t : 0;
    const int nc = row_ok ? nch : 0;
    const uint64_t* X = reinterpret_cast<const uint64_t*>(J.X);
    const uint64_t* p = strided ? X + row + (int64_t)ph * J.ld : X + row * J.ld + ph;
    const uint32_t* phi = reinterpret_cast<const uint32_t*>(p) + 1;  // high words (little-endian)
    uint32_t nx[kStatsChunk];
    auto load = [&](int c) {
      const uint32_t* a = phi + 2 * (int64_t)(kStatsChunk * c) * step;
#pragma unroll
      for (int q = 0; q < kStatsChunk; ++q) {
        nx[q] = kStatsChunk * c + q < nt ? __ldg(a) : 0u;
        a += 2 * step;
      }
    };
    if (nc > 0) load(0);
    uint64_t mx = 0;
    for (int c = 0; c < nc; ++c) {
      uint32_t h[kStatsChunk];
#pragma unroll
      for (int q = 0; q < kStatsChunk; ++q) h[q] = nx[q] & 0x7FFFFFFFu;
      if (c + 1 < nc) load(c + 1);  // the next chunk's loads fly while this one is processed
      uint32_t cmh = 0;
#pragma unroll
      for (int q = 0; q < kStatsChunk; ++q) cmh = max(cmh, h[q]);
      if (cmh >= kFastMaxHi) {
        const uint64_t cm = (uint64_t)cmh << 32;  // same frexp exponent as the chunk maximum
        mx = cm > mx ? cm : mx;
        if (hist) {
          const int ebm = (int)(cmh >> 20);
          cmx[c * kStatsThreads + tid] = (short)(ebm - 1022);
#pragma unroll
          for (int w4 = 0; w4 < kStatsChunk / 4; ++w4) {
            uint32_t word = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) word |= (uint32_t)min(63, ebm - (int)(h[4 * w4 + b] >> 20)) << (8 * b);
            word |= past_end_bytes(nt - kStatsChunk * c - 4 * w4);
            bytes[(4 * c + w4) * kStatsThreads + tid] = word;
          }
        }
      } else {
        const uint64_t cm = stats_chunk_exact(p, step, kStatsChunk * c, nt, hist, cmx, bytes, c, tid);
        mx = cm > mx ? cm : mx;
      }
    }
    // row maximum over the P threads of the row
    uint64_t rmax;
    if (strided) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, mx, 16);  // the warp's two phases of the row
      mx = o > mx ? o : mx;
      if (lane < 16) red[warp][lane] = mx;
      __syncthreads();
      rmax = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) rmax = red[w][r] > rmax ? red[w][r] : rmax;
      __syncthreads();  // every thread has read red before the next block writes it
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint64_t t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
      }
      rmax = mx;
    }
    if (row_ok && ph == 0) {
      J.maxbits[row] = rmax;  // the unit holds the whole row: no merge needed
      if (rmax >= kInfBits) atomicExch(J.nonfinite, 1);
    }
    if (hist) {
      // per byte: table index (delta + byte) / 4 with delta capped at 63; four bytes per add
      const int e_row = exponent_from_maxbits(rmax);
      for (int c = 0; c < nc; ++c) {
        const int delta = min(63, max(0, e_row - (int)cmx[c * kStatsThreads + tid]));
        const uint32_t d4 = (uint32_t)delta * 0x01010101u;
#pragma unroll
        for (int w4 = 0; w4 < kStatsChunk / 4; ++w4) {
          const uint32_t q4 = ((bytes[(4 * c + w4) * kStatsThreads + tid] + d4) >> 2) & 0x3F3F3F3Fu;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const uint4 o = onehot[(q4 >> (8 * b)) & 63u];
            c0 += o.x;
            c1 += o.y;
            c2 += o.z;
          }
        }
      }
    }
  }
  if (!HIST) return;
  if (hist) {
#pragma unroll
    for (int bin = 0; bin < 10; ++bin) {
      const uint32_t w = bin < 4 ? c0 : (bin < 8 ? c1 : c2);
      const unsigned v = __reduce_add_sync(0xffffffffu, (w >> (8 * (bin & 3))) & 255u);
      if (lane == 0 && v) atomicAdd(&sh[bin], v);
    }
  }
  __syncthreads();
  if (hist && tid < 10 && sh[tid]) atomicAdd(&J.hist[tid], (unsigned long long)sh[tid]);
}

template <bool HIST>
__global__ void __launch_bounds__(kStatsThreads, 3) stats_batched(const SplitArgs* jobs, const int2* units) {
  const int2 ur = units[blockIdx.x];
  const SplitArgs J = jobs[ur.x];
  stats_unit<HIST>(J, ur.y);
}

// The two operands of one call, passed by value (single calls need no device job table).
template <bool HIST>
__global__ void __launch_bounds__(kStatsThreads, 3) stats_pair(const SplitArgs a, const SplitArgs b, int64_t units_a) {
  const bool first = (int64_t)blockIdx.x < units_a;
  stats_unit<HIST>(first ? a : b, first ? (int64_t)blockIdx.x : (int64_t)blockIdx.x - units_a);
}

// Digits (real jobs: the grouped GEMM is real).  A unit is 32 rows x kDgK k, walked as 64-wide
// sub-tiles.  Thread t computes row t/8 and the 8 consecutive k at (t%8)*8 of a sub-tile;
// strided jobs are staged (transposed) through shared memory so that global loads stay
// coalesced.  The loads of the next sub-tile are issued before the current one is processed.
__device__ __forceinline__ void digits_unit(const SplitArgs* jobs, int2 ur) {
  __shared__ uint64_t tile[64][33];
  {
    const int* gate = jobs[ur.x].gate;
    if (gate != nullptr && *gate) return;
  }
  const SplitArgs J = jobs[ur.x];
  const int t_lo = J.plane_from != nullptr ? *J.plane_from + 1 : 1;
  const int t_hi = J.plane_to != nullptr ? *J.plane_to : J.s;
  if (t_lo > t_hi) return;
  const int64_t u = ur.y;
  const int64_t ktiles = (J.k + kDgK - 1) / kDgK;
  const int64_t r0 = (u / ktiles) * 32, lbase = (u % ktiles) * kDgK;
  const int tid = threadIdx.x;
  const int r = tid / 8, lg = (tid % 8) * 8;
  const int64_t row = r0 + r;
  const bool row_ok = row < J.rows;
  const uint64_t* X = reinterpret_cast<const uint64_t*>(J.X);
  const int e = row_ok ? exponent_from_maxbits(J.maxbits[row]) : 0;
  if (row_ok && lbase == 0 && lg == 0 && t_lo == 1) J.exps[row] = e;
  const int64_t plane = J.plane_rows * J.Kp;
  const int rr = tid % 32;
  const bool rrok = r0 + rr < J.rows;
  uint64_t nx[8];
  // contiguous rows whose elements sit on 16-byte boundaries in pairs (even ld, aligned base)
  // take their eight elements as four 16-byte loads where all eight lie inside the row
  const bool pairs = !J.strided && (J.ld & 1) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  auto load = [&](int64_t l0) {
    if (pairs && row_ok && l0 + lg + 8 <= J.k) {
      const ulonglong2* p = reinterpret_cast<const ulonglong2*>(X + row * J.ld + l0 + lg);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const ulonglong2 v = __ldg(p + h);
        nx[2 * h] = v.x;
        nx[2 * h + 1] = v.y;
      }
      return;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (J.strided) {
        const int64_t l = l0 + tid / 32 + 8 * q;
        nx[q] = (rrok && l < J.k) ? __ldg(X + (r0 + rr) + l * J.ld) : 0ull;
      } else {
        const int64_t l = l0 + lg + q;
        nx[q] = (row_ok && l < J.k) ? __ldg(X + row * J.ld + l) : 0ull;
      }
    }
  };
  load(lbase);
  for (int sub = 0; sub < kDgK / 64; ++sub) {
    const int64_t l0 = lbase + 64 * sub;
    if (l0 >= J.k) break;
    uint64_t b[8];
    if (J.strided) {
      __syncthreads();  // the previous sub-tile's reads of the tile are done
#pragma unroll
      for (int q = 0; q < 8; ++q) tile[tid / 32 + 8 * q][rr] = nx[q];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 8; ++q) b[q] = tile[lg + q][r];
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) b[q] = nx[q];
    }
    if (sub + 1 < kDgK / 64 && l0 + 64 < J.k) load(l0 + 64);
    if (!row_ok || l0 + lg >= J.k) continue;
    __half* out = J.D + row * J.Kp + l0 + lg;
    if (t_hi <= 9) {
      // planes 1 .. 9 only need the first fixed-point word (fewer registers and instructions)
      DigitSrc ds[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) ds[q] = digit_src_first(b[q], e);
      store_digit_planes<9>(ds, t_lo, t_hi, out, plane);
    } else {
      DigitSrc ds[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) ds[q] = digit_src(b[q], e);
      store_digit_planes<kMaxPlanes>(ds, t_lo, t_hi, out, plane);
    }
  }
}

// Grid-stride over the units; a gated pass (re-run completion) first reads one step-wide flag.
// five CTAs per SM (48 registers): the planes 1 .. 9 path fits; the rare longer one spills a little
__global__ void __launch_bounds__(256, 5) digits_batched(const SplitArgs* jobs, const int2* units, int64_t nunits,
                                                      const int* run) {
  if (run != nullptr && *run == 0) return;  // nothing to do in this pass
  for (int64_t unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
    digits_unit(jobs, units[unit]);
    __syncthreads();  // the next unit reuses the staging tile
  }
}

// Gated digit passes (escalation stages): usually few jobs are re-run, so one CTA first lists
// the jobs whose gate is open (their unit ranges in the batch's job-major unit table), then the
// pass walks only those units instead of testing the gate of every unit of the batch.
__global__ void __launch_bounds__(1024) digits_compact(const SplitArgs* jobs, int njobs, const int64_t* unit_start,
                                                       const int* run, int* list, int64_t* prefix, int64_t* total) {
  __shared__ int n_sh;
  if (threadIdx.x == 0) n_sh = 0;
  __syncthreads();
  const bool go = run == nullptr || *run != 0;
  if (go)
    for (int j = threadIdx.x; j < njobs; j += blockDim.x) {
      const int* gate = jobs[j].gate;
      if ((gate == nullptr || *gate == 0) && unit_start[j + 1] > unit_start[j]) list[atomicAdd(&n_sh, 1)] = j;
    }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int n = n_sh;
  int64_t acc = 0;
  for (int i = 0; i < n; ++i) {
    prefix[i] = acc;
    acc += unit_start[list[i] + 1] - unit_start[list[i]];
  }
  prefix[n] = acc;
  total[0] = acc;
  total[1] = n;
}

__global__ void __launch_bounds__(256) digits_listed(const SplitArgs* jobs, const int* list, const int64_t* prefix,
                                                     const int64_t* total) {
  const int64_t nunits = total[0];
  const int n = (int)total[1];
  for (int64_t w = blockIdx.x; w < nunits; w += gridDim.x) {
    const int li = find_job(prefix, n, w);
    digits_unit(jobs, make_int2(list[li], (int)(w - prefix[li])));
    __syncthreads();  // the next unit reuses the staging tile
  }
}

// ---------------------------------------------------------------------------- native fallback
// Device-side compaction of the calls whose non-finite flag is set, then a persistent FP64
// kernel over their 64 x 64 output tiles.
// One CTA: the flags are scanned in parallel (list order does not matter), then one thread
// forms the tile prefix over the flagged calls only (usually none).
__global__ void __launch_bounds__(1024) native_compact(const NativeArgs* calls, int ncalls, const int* const* flags,
                                                       int* list, int64_t* tile_prefix, int64_t* total) {
  __shared__ int n_sh;
  if (threadIdx.x == 0) n_sh = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < ncalls; c += blockDim.x)
    if (*flags[c] != 0) list[atomicAdd(&n_sh, 1)] = c;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int n = n_sh;
  int64_t acc = 0;
  for (int i = 0; i < n; ++i) {
    const int c = list[i];
    tile_prefix[i] = acc;
    acc += ((calls[c].m + 63) / 64) * ((calls[c].n + 63) / 64);
  }
  tile_prefix[n] = acc;
  total[0] = acc;
  total[1] = n;
}

__global__ void __launch_bounds__(256) native_batched(const NativeArgs* calls, const int* list,
                                                      const int64_t* tile_prefix, const int64_t* total) {
  __shared__ double As[16][65];
  __shared__ double Bs[16][65];
  const int64_t ntiles = total[0];
  const int ncl = (int)total[1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int64_t w = blockIdx.x; w < ntiles; w += gridDim.x) {
    const int li = find_job(tile_prefix, ncl, w);
    const NativeArgs P = calls[list[li]];
    const int64_t t = w - tile_prefix[li];
    const int64_t tn_count = (P.n + 63) / 64;
    const int64_t m0 = (t / tn_count) * 64, n0 = (t % tn_count) * 64;
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < P.k; k0 += 16) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = threadIdx.x + 256 * q;
        const int rr = idx % 64, kk = idx / 64;
        const int64_t gr = m0 + rr, gk = k0 + kk, gc = n0 + rr;
        double va = 0, vb = 0;
        if (gr < P.m && gk < P.k) va = (P.ta == 'N') ? P.A[gr + gk * P.lda] : P.A[gk + gr * P.lda];
        if (gc < P.n && gk < P.k) vb = (P.tb == 'N') ? P.B[gk + gc * P.ldb] : P.B[gc + gk * P.ldb];
        As[kk][rr] = va;
        Bs[kk][rr] = vb;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jn = 0; jn < 4; ++jn) acc[i][jn] = fma(As[kk][ty + 16 * i], Bs[kk][tx + 16 * jn], acc[i][jn]);
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jn = 0; jn < 4; ++jn) {
        const int64_t r = m0 + ty + 16 * i, c = n0 + tx + 16 * jn;
        if (r >= P.m || c >= P.n) continue;
        double* cp = P.C + r + c * P.ldc;
        *cp = P.beta_zero ? P.alpha[0] * acc[i][jn] : fma(P.alpha[0], acc[i][jn], P.beta[0] * *cp);
      }
  }
}

__global__ void repair_prep_batched(const RepairJob* jobs, int njobs, double target, int* any_rerun) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= njobs) return;
  const RepairJob J = jobs[i];
  const bool ran = J.ran == nullptr || *J.ran == 0;
  const double e = J.err ? *J.err : 0.0;
  const int sc = J.s_cur ? *J.s_cur : 0;
  const bool bad = J.auto_mode && ran && !(J.nonfinite && *J.nonfinite) && !(e <= target) && sc < J.s_fb;
  if (bad) {
    const int sn = J.s_add > 0 ? min(sc + J.s_add, J.s_fb) : J.s_fb;
    if (J.s_next) *J.s_next = sn;
    if (J.s_copy) *J.s_copy = sn;
  }
  *J.skip_next = bad ? 0 : 1;
  if (bad && any_rerun != nullptr) atomicOr(any_rerun, 1);
}

// unit = 256 elements of one automatic, beta != 0 call
__global__ void save_restore_batched(const RepairJob* jobs, const int64_t* prefix, int njobs, int restore) {
  const int64_t unit = blockIdx.x;
  const int jb = find_job(prefix, njobs, unit);
  const RepairJob J = jobs[jb];
  if (restore && *J.skip_next) return;
  const int64_t e = (unit - prefix[jb]) * 256 + threadIdx.x;
  if (e >= J.m * J.n) return;
  const int64_t i = e % J.m, j = e / J.m;
  if (restore)
    J.C[i + j * J.ldc] = J.saved[e];
  else
    J.saved[e] = J.C[i + j * J.ldc];
}

}  // namespace

cudaError_t launch_repair_prep_batched(const RepairJob* jobs_dev, int njobs, double target, int* any_rerun,
                                       cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  { repair_prep_batched<<<(njobs + 127) / 128, 128, 0, st>>>(jobs_dev, njobs, target, any_rerun); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_save_restore_batched(const RepairJob* jobs_dev, const int64_t* prefix_dev, int64_t units,
                                        int njobs, int restore, cudaStream_t st) {
  if (units <= 0 || njobs <= 0) return cudaSuccess;
  { save_restore_batched<<<(unsigned)units, 256, 0, st>>>(jobs_dev, prefix_dev, njobs, restore); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_stats_batched(const SplitArgs* jobs_dev, const int2* units_dev, int64_t units, int hist,
                                 cudaStream_t st) {
  if (units <= 0) return cudaSuccess;
  static_assert(kStatsHistSmem <= 48 * 1024, "within the default dynamic shared-memory limit");
  if (hist) {
    stats_batched<true><<<(unsigned)units, kStatsThreads, kStatsHistSmem, st>>>(jobs_dev, units_dev);
  } else {
    stats_batched<false><<<(unsigned)units, kStatsThreads, 0, st>>>(jobs_dev, units_dev);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_stats_pair(const SplitArgs& a, const SplitArgs& b, cudaStream_t st) {
  const int64_t ua = stats_units_of(a), ub = stats_units_of(b);
  if (ua + ub <= 0) return cudaSuccess;
  if (a.hist != nullptr || b.hist != nullptr)
    stats_pair<true><<<(unsigned)(ua + ub), kStatsThreads, kStatsHistSmem, st>>>(a, b, ua);
  else
    stats_pair<false><<<(unsigned)(ua + ub), kStatsThreads, 0, st>>>(a, b, ua);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_rowmax_batched(const SplitArgs* jobs_dev, const int2* units_dev, int64_t units, cudaStream_t st) {
  if (units > 0) { rowmax_batched<<<(unsigned)units, 256, 0, st>>>(jobs_dev, units_dev); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_digits_batched(const SplitArgs* jobs_dev, const int2* units_dev, int64_t units, const int* run,
                                  int grid_cap, cudaStream_t st) {
  if (units <= 0) return cudaSuccess;
  const int64_t grid = grid_cap > 0 && units > grid_cap ? grid_cap : units;
  { digits_batched<<<(unsigned)grid, 256, 0, st>>>(jobs_dev, units_dev, units, run); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_digits_gated(const SplitArgs* jobs_dev, int njobs, const int64_t* unit_start_dev, const int* run,
                                int* list_dev, int64_t* prefix_dev, int64_t* total_dev, int grid, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  { digits_compact<<<1, 1024, 0, st>>>(jobs_dev, njobs, unit_start_dev, run, list_dev, prefix_dev, total_dev); note_launch(); }
  { digits_listed<<<grid, 256, 0, st>>>(jobs_dev, list_dev, prefix_dev, total_dev); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_native_batched(const NativeArgs* calls_dev, int ncalls, const int* const* flags_dev, int* list_dev,
                                  int64_t* prefix_dev, int64_t* total_dev, int grid, cudaStream_t st) {
  if (ncalls <= 0) return cudaSuccess;
  { native_compact<<<1, 1024, 0, st>>>(calls_dev, ncalls, flags_dev, list_dev, prefix_dev, total_dev); note_launch(); }
  { native_batched<<<grid, 256, 0, st>>>(calls_dev, list_dev, prefix_dev, total_dev); note_launch(); }
  return cudaGetLastError();
}

}  // namespace ozg
