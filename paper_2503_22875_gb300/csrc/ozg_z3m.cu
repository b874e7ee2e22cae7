// 3M (Karatsuba) complex product on the real emulation: three real emulated products instead of
// the four real sub-products of the stacked form (Sec. 2.2's scheme applied to the real and
// imaginary parts separately).  With Ar, Ai the real and imaginary parts of op(A) (conjugated
// for 'C'), Sa = RN(Ar + Ai), and the same for op(B):
//   P1 = emu(Ar, Br),  P2 = emu(Ai, Bi),  P3 = emu(Sa, Sb)
//   Re = RN(P1 - P2),  Im = RN(RN(P3 - P1) - P2)
// then alpha and beta as the stacked complex path applies them.  The three real products run as
// one grouped launch (each with its own row and column exponents); 3 m n k multiply-adds per
// slice pair instead of 4 m n k, at the price of the weaker error bound of the 3M form (the
// imaginary part's error scales with (|Ar| + |Ai|)(|Br| + |Bi|)).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ozg_context.h"

using namespace ozg::host;

namespace ozg {
namespace {

// X: complex rows x cols (column-major, ld, interleaved) -> Xr, Xi, Xs = RN(Xr + Xi), packed
// (ld = rows); the imaginary part negated when conj.
__global__ void __launch_bounds__(256) z3m_split_kernel(const double* __restrict__ X, int64_t rows, int64_t cols,
                                                        int64_t ld, int conj, double* __restrict__ Xr,
                                                        double* __restrict__ Xi, double* __restrict__ Xs) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % rows, j = t / rows;
    const double re = X[2 * (i + j * ld)];
    const double im = conj ? -X[2 * (i + j * ld) + 1] : X[2 * (i + j * ld) + 1];
    Xr[t] = re;
    Xi[t] = im;
    Xs[t] = re + im;
  }
}

__global__ void __launch_bounds__(256) z3m_combine_kernel(const double* __restrict__ P1, const double* __restrict__ P2,
                                                          const double* __restrict__ P3, int64_t m, int64_t n,
                                                          double a0, double a1, double b0, double b1, int beta_zero,
                                                          double* C, int64_t ldc) {
  const int64_t total = m * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % m, j = t / m;
    const double p1 = P1[t], p2 = P2[t], p3 = P3[t];
    const double tr = __dsub_rn(p1, p2);
    const double ti = __dsub_rn(__dsub_rn(p3, p1), p2);
    double* c = C + 2 * (i + j * ldc);
    double re = fma(a0, tr, -__dmul_rn(a1, ti));
    double im = fma(a0, ti, __dmul_rn(a1, tr));
    if (!beta_zero) {
      const double cr = c[0], ci = c[1];
      re = __dadd_rn(re, fma(b0, cr, -__dmul_rn(b1, ci)));
      im = __dadd_rn(im, fma(b0, ci, __dmul_rn(b1, cr)));
    }
    c[0] = re;
    c[1] = im;
  }
}

int grid_for(const ozg_ctx* c, int64_t total) {
  const int64_t want = (total + 255) / 256, cap = (int64_t)std::max(c->num_sms, 1) * 8;
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

}  // namespace
}  // namespace ozg

extern "C" int ozg_zgemm3m(ozg_ctx* c, char transa, char transb, int64_t m, int64_t n, int64_t k,
                           const double* alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                           const double* beta, double* C, int64_t ldc, int slices, ozg_report* rep) {
  if (!alpha || !beta) return OZG_ERR_INVALID;
  const char ta = norm_trans(transa), tb = norm_trans(transb);
  const int64_t nrowa = ta == 'N' ? m : k, nrowb = tb == 'N' ? k : n;
  int info = 0;
  if (ta != 'N' && ta != 'T' && ta != 'C') info = -1;
  else if (tb != 'N' && tb != 'T' && tb != 'C') info = -2;
  else if (m < 0) info = -3;
  else if (n < 0) info = -4;
  else if (k < 0) info = -5;
  else if (lda < std::max<int64_t>(1, nrowa)) info = -8;
  else if (ldb < std::max<int64_t>(1, nrowb)) info = -10;
  else if (ldc < std::max<int64_t>(1, m)) info = -13;
  else if (slices != OZG_NATIVE && (slices < 1 || slices > OZG_MAX_SLICES)) info = -14;
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->status = info;
    rep->est_err = rep->max_real = rep->max_imag = NAN;
  }
  if (info) return info;
  if (!c) return OZG_ERR_INVALID;  // BLAS argument errors are reported first
  if (m == 0 || n == 0) return OZG_OK;
  // native mode, k == 0 and alpha == 0 need no products: the stacked path handles them
  if (slices == OZG_NATIVE || k == 0 || (alpha[0] == 0.0 && alpha[1] == 0.0))
    return ozg_zgemm(c, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, rep);
  cudaSetDevice(c->device);
  cudaStream_t st = c->stream;
  // storage shapes of A and B (the real operands keep them; the products take 'N' / 'T')
  const int64_t ra = nrowa, ca = ta == 'N' ? k : m, rb = nrowb, cb = tb == 'N' ? n : k;
  const int nsamp = c->check_samples;
  ozg::host::Carve cv;
  const size_t oA = cv.take(sizeof(double) * 3 * ra * ca), oB = cv.take(sizeof(double) * 3 * rb * cb);
  const size_t oP = cv.take(sizeof(double) * 3 * m * n), oCold = cv.take(sizeof(double) * 2 * std::max(nsamp, 1));
  int rc = ensure_z3ws(c, cv.off);
  if (rc) return rc;
  char* base = static_cast<char*>(c->z3ws);
  double* Ar = reinterpret_cast<double*>(base + oA);
  double *Ai = Ar + ra * ca, *As = Ai + ra * ca;
  double* Br = reinterpret_cast<double*>(base + oB);
  double *Bi = Br + rb * cb, *Bs = Bi + rb * cb;
  double* P1 = reinterpret_cast<double*>(base + oP);
  double *P2 = P1 + m * n, *P3 = P2 + m * n;
  {
    PhaseScope ps(c, OZG_PHASE_SPLIT);
    { ozg::z3m_split_kernel<<<ozg::grid_for(c, ra * ca), 256, 0, st>>>(A, ra, ca, lda, ta == 'C', Ar, Ai, As); ozg::note_launch(); }
    { ozg::z3m_split_kernel<<<ozg::grid_for(c, rb * cb), 256, 0, st>>>(B, rb, cb, ldb, tb == 'C', Br, Bi, Bs); ozg::note_launch(); }
    OZG_CUDA(cudaGetLastError());
  }
  const char rta = ta == 'N' ? 'N' : 'T', rtb = tb == 'N' ? 'N' : 'T';
  ozg_gemm_desc d[3];
  const double* xa[3] = {Ar, Ai, As};
  const double* xb[3] = {Br, Bi, Bs};
  double* xp[3] = {P1, P2, P3};
  for (int i = 0; i < 3; ++i) {
    std::memset(&d[i], 0, sizeof(d[i]));
    d[i].transa = rta;
    d[i].transb = rtb;
    d[i].m = m;
    d[i].n = n;
    d[i].k = k;
    d[i].alpha = 1.0;
    d[i].beta = 0.0;
    d[i].A = xa[i];
    d[i].lda = std::max<int64_t>(1, ra);
    d[i].B = xb[i];
    d[i].ldb = std::max<int64_t>(1, rb);
    d[i].C = xp[i];
    d[i].ldc = m;
  }
  const int sl[3] = {slices, slices, slices};
  c->check_samples = 0;  // the sampled check judges the complex result below, not the real products
  rc = ozg_dgemm_grouped(c, 3, d, sl, nullptr);
  c->check_samples = nsamp;
  if (rc) return rc;
  ozg::CheckArgs ck;
  if (nsamp > 0) {
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
    ck.alpha[0] = alpha[0];
    ck.alpha[1] = alpha[1];
    ck.beta[0] = beta[0];
    ck.beta[1] = beta[1];
    ck.beta_zero = (beta[0] == 0.0 && beta[1] == 0.0) ? 1 : 0;
    ck.cplx = 1;
    ck.nsamp = nsamp;
    ck.seed = c->check_seed++;
    ck.cold = reinterpret_cast<double*>(base + oCold);
    ck.err_out = c->dcheck;
    ck.part_err = c->dcheck + 1;
    PhaseScope ps(c, OZG_PHASE_CHECK);
    OZG_CUDA(ozg::launch_check_pre(ck, st));
  }
  {
    PhaseScope ps(c, OZG_PHASE_SPLIT);
    const int beta_zero = (beta[0] == 0.0 && beta[1] == 0.0) ? 1 : 0;
    { ozg::z3m_combine_kernel<<<ozg::grid_for(c, m * n), 256, 0, st>>>(P1, P2, P3, m, n, alpha[0], alpha[1], beta[0],
                                                                       beta[1], beta_zero, C, ldc); ozg::note_launch(); }
    OZG_CUDA(cudaGetLastError());
  }
  if (nsamp > 0) {
    PhaseScope ps(c, OZG_PHASE_CHECK);
    OZG_CUDA(ozg::launch_check_post(ck, st));
  }
  if (rep) {
    double e[3] = {NAN, NAN, NAN};
    if (nsamp > 0) OZG_CUDA(cudaMemcpyAsync(e, c->dcheck, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    OZG_CUDA(cudaStreamSynchronize(st));
    rep->slices_used = slices;
    rep->samples = nsamp;
    rep->est_err = e[0];
    rep->max_real = e[1];
    rep->max_imag = e[2];
  }
  return OZG_OK;
}
