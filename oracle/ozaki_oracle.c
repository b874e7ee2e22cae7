/*
 * CPU oracle for FP64 / complex128 GEMM emulated with INT8-range integer slices
 * (the Ozaki scheme on an integer matrix-multiply unit, Sec. 2.2 of "A Pilot Study on
 * Tunable Precision Emulation via Automatic BLAS Offloading"; the tunable split number is
 * the compute mode fp64_int8_<s> of Sec. 3.1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct reference that
 * the CUDA path is checked against.  It shares no code with the CUDA library; nothing in the
 * product path may call it.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.
 *
 * Conventions (BLAS ?gemm): matrices are column-major; op(A) is m x k, op(B) is k x n;
 * op(X) = X ('N'), X^T ('T'), X^H ('C', complex only).  u = 2^-53.
 *
 * Method, as restated here (the paper names the method but does not print its arithmetic;
 * each reading below is listed with its justification in the design notes):
 *   - Row i of op(A) gets the power-of-two scale 2^e_i, e_i = frexp exponent of
 *     max_l |op(A)_il| (so every scaled entry a' = a * 2^-e_i has |a'| < 1); a zero row
 *     gets e_i = 0.  Column j of op(B) likewise gets f_j.
 *   - Digits (slices) by truncation, 7 bits each: r_0 = a'; d_t = trunc(2^7 r_{t-1});
 *     r_t = 2^7 r_{t-1} - d_t, t = 1..s.  |d_t| <= 127, all of a's sign.
 *   - Slice products: the s(s+1)/2 pairs (p,q) with p+q <= s+1, summed per group g = p+q:
 *     G_g = sum_{p+q=g} D^A_p (D^B_q)^T  (exact integers).
 *   - N_ij = sum_g G_g,ij 2^{7(s+1-g)} (exact), T_ij = N_ij 2^{e_i + f_j - 7(s+1)},
 *     t = RN(T) (one rounding), C = alpha*t + beta*C_old evaluated as fma(alpha, t, beta*C_old)
 *     (beta == 0: C = alpha*t, C_old not read).
 *   - Complex: the real and imaginary parts of a row (column) share one exponent taken from
 *     max(|Re|, |Im|); conjugation negates the imaginary digits; the four real products are
 *     combined exactly in integers: N_re = N_rr - N_ii, N_im = N_ri + N_ir.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fno-fast-math -shared -fPIC.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

static int orc_threads_req = 0;
ORC_EXPORT void orc_set_threads(int n) { orc_threads_req = n; }
ORC_EXPORT int orc_get_threads(void) {
#ifdef _OPENMP
  return orc_threads_req > 0 ? orc_threads_req : omp_get_max_threads();
#else
  return 1;
#endif
}

/* element (r, c) of op(X) where X is column-major with leading dimension ld */
static inline double op_r(char t, const double* X, int64_t ld, int64_t r, int64_t c) {
  return (t == 'N' || t == 'n') ? X[r + c * ld] : X[c + r * ld];
}

/* ---------------------------------------------------------------- O-naive: plain FP64 GEMM */
ORC_EXPORT void orc_dgemm_naive(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha,
                                const double* A, int64_t lda, const double* B, int64_t ldb,
                                double beta, double* C, int64_t ldc) {
  int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < m; ++i) {
      double acc = 0.0;
      for (int64_t l = 0; l < k; ++l) acc += op_r(ta, A, lda, i, l) * op_r(tb, B, ldb, l, j);
      double* c = &C[i + j * ldc];
      *c = (beta == 0.0) ? alpha * acc : alpha * acc + beta * (*c);
    }
  }
}

/* ------------------------------------------------------- double-double arithmetic (Sec. 2.2) */
typedef struct { double hi, lo; } dd_t;
static inline dd_t two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  dd_t r = {s, (a - (s - bb)) + (b - bb)};
  return r;
}
static inline dd_t quick_two_sum(double a, double b) {
  double s = a + b;
  dd_t r = {s, b - (s - a)};
  return r;
}
static inline dd_t two_prod(double a, double b) {
  double p = a * b;
  dd_t r = {p, fma(a, b, -p)};
  return r;
}
static inline dd_t dd_add(dd_t a, dd_t b) { /* accurate (IEEE-style) double-double addition */
  dd_t s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
static inline dd_t dd_mul_d(dd_t a, double b) {
  dd_t p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return quick_two_sum(p.hi, p.lo);
}

/* O-dd: P = op(A) op(B) accumulated in double-double, then out = alpha*P + beta*C_old in
 * double-double; the result is returned as the pair (hi, lo) (either pointer may be NULL)
 * and C receives RN(hi + lo) = hi.  Error <= ~2k u^2 (|A||B|)_ij. */
ORC_EXPORT void orc_dgemm_dd(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha,
                             const double* A, int64_t lda, const double* B, int64_t ldb,
                             double beta, double* C, int64_t ldc, double* out_hi, double* out_lo) {
  int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < m; ++i) {
      dd_t acc = {0.0, 0.0};
      for (int64_t l = 0; l < k; ++l) acc = dd_add(acc, two_prod(op_r(ta, A, lda, i, l), op_r(tb, B, ldb, l, j)));
      dd_t r = dd_mul_d(acc, alpha);
      if (beta != 0.0) r = dd_add(r, two_prod(beta, C[i + j * ldc]));
      if (C) C[i + j * ldc] = r.hi;
      if (out_hi) out_hi[i + j * m] = r.hi;
      if (out_lo) out_lo[i + j * m] = r.lo;
    }
  }
}

/* Complex double-double product P = op(A) op(B) (interleaved complex128, column-major),
 * no alpha/beta: out_* are m x n, column-major, ld = m.  Used as the error reference. */
static inline void cplx_op(char t, const double* X, int64_t ld, int64_t r, int64_t c, double* re, double* im) {
  const double* p = (t == 'N' || t == 'n') ? &X[2 * (r + c * ld)] : &X[2 * (c + r * ld)];
  *re = p[0];
  *im = (t == 'C' || t == 'c') ? -p[1] : p[1];
}
ORC_EXPORT void orc_zgemm_dd(char ta, char tb, int64_t m, int64_t n, int64_t k,
                             const double* A, int64_t lda, const double* B, int64_t ldb,
                             double* re_hi, double* re_lo, double* im_hi, double* im_lo) {
  int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < m; ++i) {
      dd_t sr = {0, 0}, si = {0, 0};
      for (int64_t l = 0; l < k; ++l) {
        double ar, ai, br, bi;
        cplx_op(ta, A, lda, i, l, &ar, &ai);
        cplx_op(tb, B, ldb, l, j, &br, &bi);
        sr = dd_add(sr, two_prod(ar, br));
        sr = dd_add(sr, two_prod(-ai, bi));
        si = dd_add(si, two_prod(ar, bi));
        si = dd_add(si, two_prod(ai, br));
      }
      re_hi[i + j * m] = sr.hi; re_lo[i + j * m] = sr.lo;
      im_hi[i + j * m] = si.hi; im_lo[i + j * m] = si.lo;
    }
  }
}

/* Plain complex FP64 GEMM (naive), C = alpha*op(A)op(B) + beta*C. */
ORC_EXPORT void orc_zgemm_naive(char ta, char tb, int64_t m, int64_t n, int64_t k, const double* alpha,
                                const double* A, int64_t lda, const double* B, int64_t ldb,
                                const double* beta, double* C, int64_t ldc) {
  int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < m; ++i) {
      double sr = 0, si = 0;
      for (int64_t l = 0; l < k; ++l) {
        double ar, ai, br, bi;
        cplx_op(ta, A, lda, i, l, &ar, &ai);
        cplx_op(tb, B, ldb, l, j, &br, &bi);
        sr += ar * br - ai * bi;
        si += ar * bi + ai * br;
      }
      double* c = &C[2 * (i + j * ldc)];
      double tr = alpha[0] * sr - alpha[1] * si, ti = alpha[0] * si + alpha[1] * sr;
      if (beta[0] != 0.0 || beta[1] != 0.0) {
        tr += beta[0] * c[0] - beta[1] * c[1];
        ti += beta[0] * c[1] + beta[1] * c[0];
      }
      c[0] = tr; c[1] = ti;
    }
  }
}

/* ------------------------------------------------------------------ O-slice: the splitter */
/* Digits of one scaled value x (|x| < 1) by truncation: d_t = trunc(2^7 r), r <- 2^7 r - d_t.
 * Every step is exact in FP64 (multiplication by 2^7, subtraction of the integer part). */
static inline void digits_of(double x, int s, int8_t* d, int64_t stride) {
  double r = x;
  for (int t = 0; t < s; ++t) {
    double y = r * 128.0;
    double q = trunc(y);
    d[t * stride] = (int8_t)q;
    r = y - q;
  }
}

/* Split the rows of op(X) (rows x k; X real, column-major, ld) into exponents e[rows] and
 * digits D[s][rows][k] (row-major inside a slice, k contiguous).  For the B operand call it
 * with trans flipped ('N' <-> 'T') so that "rows" are the columns of op(B). */
ORC_EXPORT void orc_split(char trans, int64_t rows, int64_t k, const double* X, int64_t ld, int s,
                          int32_t* e, int8_t* D) {
  for (int64_t i = 0; i < rows; ++i) {
    double amax = 0.0;
    for (int64_t l = 0; l < k; ++l) {
      double a = fabs(op_r(trans, X, ld, i, l));
      if (a > amax) amax = a;
    }
    int ex = 0;
    if (amax != 0.0) frexp(amax, &ex);
    e[i] = ex;
    for (int64_t l = 0; l < k; ++l) {
      double a = ldexp(op_r(trans, X, ld, i, l), -ex);
      digits_of(a, s, &D[i * k + l], rows * k);
    }
  }
}

/* Complex split: op(X) is rows x k complex (interleaved complex128).  Output rows are
 * interleaved: output row 2i holds Re of row i, row 2i+1 holds Im; one shared exponent
 * e[i] per complex row from max(|Re|, |Im|); trans 'C' conjugates (negates Im digits). */
ORC_EXPORT void orc_zsplit(char trans, int64_t rows, int64_t k, const double* X, int64_t ld, int s,
                           int32_t* e, int8_t* D) {
  int64_t R2 = 2 * rows;
  for (int64_t i = 0; i < rows; ++i) {
    double amax = 0.0;
    for (int64_t l = 0; l < k; ++l) {
      double re, im;
      cplx_op(trans, X, ld, i, l, &re, &im);
      if (fabs(re) > amax) amax = fabs(re);
      if (fabs(im) > amax) amax = fabs(im);
    }
    int ex = 0;
    if (amax != 0.0) frexp(amax, &ex);
    e[i] = ex;
    for (int64_t l = 0; l < k; ++l) {
      double re, im;
      cplx_op(trans, X, ld, i, l, &re, &im);
      digits_of(ldexp(re, -ex), s, &D[(2 * i) * k + l], R2 * k);
      digits_of(ldexp(im, -ex), s, &D[(2 * i + 1) * k + l], R2 * k);
    }
  }
}

/* ------------------------------------------------------------- O-int: exact slice products */
/* G[g-2][i][j] = sum_{p+q=g, (p,q) in set} sum_l DA[p-1][i][l] * DB[q-1][j][l], g = 2..2s
 * (triangle set: g <= s+1 only; square set (square != 0): all s^2 pairs, g up to 2s).
 * DA: [s][m][k], DB: [s][n][k] (row-major, k contiguous).  G: [ngroups][m][n], int64. */
ORC_EXPORT int orc_group_products(int64_t m, int64_t n, int64_t k, int s, const int8_t* DA, const int8_t* DB,
                                  int square, int64_t* G) {
  int ng = square ? 2 * s - 1 : s;
  memset(G, 0, sizeof(int64_t) * (size_t)ng * m * n);
  int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t i = 0; i < m; ++i) {
    for (int p = 1; p <= s; ++p) {
      for (int q = 1; q <= s; ++q) {
        if (!square && p + q > s + 1) continue;
        int gi = p + q - 2;
        const int8_t* a = &DA[((int64_t)(p - 1) * m + i) * k];
        for (int64_t j = 0; j < n; ++j) {
          const int8_t* b = &DB[((int64_t)(q - 1) * n + j) * k];
          int64_t acc = 0;
          for (int64_t l = 0; l < k; ++l) acc += (int64_t)a[l] * (int64_t)b[l];
          G[((int64_t)gi * m + i) * n + j] += acc;
        }
      }
    }
  }
  return ng;
}

/* ------------------------------------------------ exact wide integers and correct rounding */
/* A 256-bit two's-complement integer in four 64-bit limbs (little-endian).  N_ij needs at most
 * 31 + log2(k s) + 7(2s - 2) bits, well inside 255 bits for s <= 18 and k < 2^40. */
typedef struct { uint64_t w[4]; } i256;
static inline void i256_zero(i256* x) { memset(x, 0, sizeof(*x)); }
static inline void i256_add(i256* x, const i256* y) {
  unsigned __int128 c = 0;
  for (int t = 0; t < 4; ++t) {
    c += (unsigned __int128)x->w[t] + y->w[t];
    x->w[t] = (uint64_t)c;
    c >>= 64;
  }
}
static inline void i256_from_i64_shl(i256* x, int64_t v, int sh) { /* x = v * 2^sh, 0 <= sh < 192 */
  uint64_t fill = v < 0 ? ~0ull : 0ull;
  uint64_t src[5] = {(uint64_t)v, fill, fill, fill, fill};
  i256_zero(x);
  int ws = sh / 64, bs = sh % 64;
  for (int t = 0; t < 4; ++t) {
    int s0 = t - ws;
    uint64_t lo = (s0 >= 0) ? src[s0] : 0ull;
    uint64_t below = (s0 - 1 >= 0) ? src[s0 - 1] : 0ull;
    x->w[t] = bs ? ((lo << bs) | (below >> (64 - bs))) : lo;
  }
}
static inline int i256_neg_sign(const i256* x) { return (int)(x->w[3] >> 63); }
static inline void i256_negate(i256* x) {
  for (int t = 0; t < 4; ++t) x->w[t] = ~x->w[t];
  i256 one; i256_zero(&one); one.w[0] = 1;
  i256_add(x, &one);
}
static inline int i256_bitlen(const i256* x) { /* of a non-negative value */
  for (int t = 3; t >= 0; --t)
    if (x->w[t]) return 64 * t + 64 - __builtin_clzll(x->w[t]);
  return 0;
}
static inline int i256_bit(const i256* x, int b) { return (int)((x->w[b / 64] >> (b % 64)) & 1ull); }

/* RN(N * 2^E): the exact value rounded once to FP64 (ties to even), including the subnormal
 * range and overflow to +-Inf. */
static double round_scaled(i256 N, int64_t E) {
  int neg = i256_neg_sign(&N);
  if (neg) i256_negate(&N);
  int p = i256_bitlen(&N);
  if (p == 0) return 0.0;
  int64_t top = (int64_t)p - 1 + E;               /* exponent of the leading bit */
  if (top > 1023) return neg ? -INFINITY : INFINITY;
  int64_t q = top - 52;                            /* exponent of the ulp */
  if (q < -1074) q = -1074;
  int64_t r = q - E;                               /* bits of N below the ulp */
  double mag;
  if (r <= 0) {
    /* exact: N < 2^53 here */
    mag = ldexp((double)N.w[0], (int)E);
  } else {
    if (r > 255) { /* everything is below half an ulp of the smallest subnormal */
      return neg ? -0.0 : 0.0;
    }
    /* Q = N >> r ; rem = N mod 2^r ; half = 2^(r-1) */
    uint64_t Q = 0;
    for (int b = 0; b < 54 && (int64_t)b + r < 256; ++b) Q |= (uint64_t)i256_bit(&N, (int)(b + r)) << b;
    int rbit = i256_bit(&N, (int)(r - 1));
    int sticky = 0;
    for (int b = 0; b < r - 1; ++b) if (i256_bit(&N, b)) { sticky = 1; break; }
    if (rbit && (sticky || (Q & 1ull))) Q += 1;
    mag = ldexp((double)Q, (int)q);                /* Q <= 2^53: exact */
  }
  return neg ? -mag : mag;
}

/* O-emu core: from exponents and exact group products to RN(T).  G: [s][m][n] (groups
 * g = 2..s+1 at index g-2), or the square set with 2s-1 groups.  out: m x n, ld m. */
static double emu_entry(const int64_t* G, int ng, int s, int square, int64_t m, int64_t n, int64_t i,
                        int64_t j, int32_t ei, int32_t fj) {
  /* N = sum_g G_g 2^{7(top-g)} exactly, top = s+1 (triangle) or 2s (square set), then
   * RN(N 2^{e_i + f_j - 7 top}). */
  int top = square ? 2 * s : s + 1;
  i256 N, t;
  i256_zero(&N);
  for (int gi = 0; gi < ng; ++gi) {
    int g = gi + 2;
    i256_from_i64_shl(&t, G[((int64_t)gi * m + i) * n + j], 7 * (top - g));
    i256_add(&N, &t);
  }
  int64_t E = (int64_t)ei + fj - 7 * top;
  return round_scaled(N, E);
}

/* Full O-emu DGEMM: C = alpha*RN(T) + beta*C_old, T as in the header. square=1 uses all
 * s^2 slice pairs (test-only variant). */
ORC_EXPORT void orc_dgemm_emu(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha,
                              const double* A, int64_t lda, const double* B, int64_t ldb,
                              double beta, double* C, int64_t ldc, int s, int square) {
  if (m <= 0 || n <= 0) return;
  int32_t* e = (int32_t*)malloc(sizeof(int32_t) * m);
  int32_t* f = (int32_t*)malloc(sizeof(int32_t) * n);
  int8_t* DA = (int8_t*)malloc((size_t)s * m * (k > 0 ? k : 1));
  int8_t* DB = (int8_t*)malloc((size_t)s * n * (k > 0 ? k : 1));
  int ng = square ? 2 * s - 1 : s;
  int64_t* G = (int64_t*)malloc(sizeof(int64_t) * (size_t)ng * m * n);
  char tbf = (tb == 'N' || tb == 'n') ? 'T' : 'N'; /* columns of op(B) = rows of op(B)^T */
  orc_split(ta, m, k, A, lda, s, e, DA);
  orc_split(tbf, n, k, B, ldb, s, f, DB);
  orc_group_products(m, n, k, s, DA, DB, square, G);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double t = emu_entry(G, ng, s, square, m, n, i, j, e[i], f[j]);
      double* c = &C[i + j * ldc];
      *c = (beta == 0.0) ? alpha * t : fma(alpha, t, beta * (*c));
    }
  free(e); free(f); free(DA); free(DB); free(G);
}

/* Full O-emu ZGEMM.  Stacked split (rows 2i / 2i+1 = Re / Im), one real emulated product of
 * the stacked operands, exact integer combine, one rounding per part, then
 *   re = (alpha_r t_r - alpha_i t_i) + (beta_r c_r - beta_i c_i)
 *   im = (alpha_r t_i + alpha_i t_r) + (beta_r c_i + beta_i c_r)
 * each product pair formed as fma(x, y, -(z*w)) / fma(x, y, z*w) in that order. */
ORC_EXPORT void orc_zgemm_emu(char ta, char tb, int64_t m, int64_t n, int64_t k, const double* alpha,
                              const double* A, int64_t lda, const double* B, int64_t ldb,
                              const double* beta, double* C, int64_t ldc, int s) {
  if (m <= 0 || n <= 0) return;
  int32_t* e = (int32_t*)malloc(sizeof(int32_t) * m);
  int32_t* f = (int32_t*)malloc(sizeof(int32_t) * n);
  int64_t kk = k > 0 ? k : 1;
  int8_t* DA = (int8_t*)malloc((size_t)s * 2 * m * kk);
  int8_t* DB = (int8_t*)malloc((size_t)s * 2 * n * kk);
  int64_t M2 = 2 * m, N2 = 2 * n;
  int64_t* G = (int64_t*)malloc(sizeof(int64_t) * (size_t)s * M2 * N2);
  /* columns of op(B) as rows: op(B)^T has the same conjugation as op(B) */
  char tbf = (tb == 'N' || tb == 'n') ? 'T' : ((tb == 'T' || tb == 't') ? 'N' : 'H');
  orc_zsplit(ta, m, k, A, lda, s, e, DA);
  if (tbf == 'H') {
    /* rows of op(B) = B^H columns: row j of (B^H)^T = conj(column j of B) -> handled by a
     * local conjugating split of B with 'N' access pattern on columns */
    int64_t R2 = 2 * n;
    for (int64_t j = 0; j < n; ++j) {
      double amax = 0.0;
      for (int64_t l = 0; l < k; ++l) {
        const double* p = &B[2 * (j + l * ldb)];  /* op(B)_{l,j} = conj(B_{j,l}) */
        if (fabs(p[0]) > amax) amax = fabs(p[0]);
        if (fabs(p[1]) > amax) amax = fabs(p[1]);
      }
      int ex = 0;
      if (amax != 0.0) frexp(amax, &ex);
      f[j] = ex;
      for (int64_t l = 0; l < k; ++l) {
        const double* p = &B[2 * (j + l * ldb)];
        digits_of(ldexp(p[0], -ex), s, &DB[(2 * j) * k + l], R2 * k);
        digits_of(ldexp(-p[1], -ex), s, &DB[(2 * j + 1) * k + l], R2 * k);
      }
    }
  } else {
    orc_zsplit(tbf, n, k, B, ldb, s, f, DB);
  }
  orc_group_products(M2, N2, k, s, DA, DB, 0, G);
  /* combine: re = rr - ii, im = ri + ir, exactly, per group */
  int64_t* Gc = (int64_t*)malloc(sizeof(int64_t) * (size_t)s * m * n * 2);
  for (int gi = 0; gi < s; ++gi)
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        const int64_t* Gg = &G[(int64_t)gi * M2 * N2];
        int64_t rr = Gg[(2 * i) * N2 + 2 * j], ri = Gg[(2 * i) * N2 + 2 * j + 1];
        int64_t ir = Gg[(2 * i + 1) * N2 + 2 * j], ii = Gg[(2 * i + 1) * N2 + 2 * j + 1];
        Gc[((int64_t)gi * m + i) * n + j] = rr - ii;
        Gc[((int64_t)(s + gi) * m + i) * n + j] = ri + ir;
      }
  int do_beta = (beta[0] != 0.0 || beta[1] != 0.0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double tr = emu_entry(Gc, s, s, 0, m, n, i, j, e[i], f[j]);
      double ti = emu_entry(Gc + (int64_t)s * m * n, s, s, 0, m, n, i, j, e[i], f[j]);
      double* c = &C[2 * (i + j * ldc)];
      double re = fma(alpha[0], tr, -(alpha[1] * ti));
      double im = fma(alpha[0], ti, alpha[1] * tr);
      if (do_beta) {
        double br = fma(beta[0], c[0], -(beta[1] * c[1]));
        double bi = fma(beta[0], c[1], beta[1] * c[0]);
        re += br; im += bi;
      }
      c[0] = re; c[1] = im;
    }
  free(e); free(f); free(DA); free(DB); free(G); free(Gc);
}

/* 3M (Karatsuba) combine of three real emulated products into complex C (column-major m x n,
 * interleaved, ld ldc), given P1 = emu(Ar, Br), P2 = emu(Ai, Bi), P3 = emu(Sa, Sb) with
 * Sa = RN(Ar + Ai), Sb = RN(Br + Bi) (each m x n, ld m):
 *   t_r = RN(P1 - P2),  t_i = RN(RN(P3 - P1) - P2)
 * then alpha and beta exactly as orc_zgemm_emu applies them. */
ORC_EXPORT void orc_zgemm3m_combine(int64_t m, int64_t n, const double* P1, const double* P2, const double* P3,
                                    const double* alpha, const double* beta, double* C, int64_t ldc) {
  int do_beta = (beta[0] != 0.0 || beta[1] != 0.0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double p1 = P1[i + j * m], p2 = P2[i + j * m], p3 = P3[i + j * m];
      double tr = p1 - p2;
      double d = p3 - p1;
      double ti = d - p2;
      double* c = &C[2 * (i + j * ldc)];
      double re = fma(alpha[0], tr, -(alpha[1] * ti));
      double im = fma(alpha[0], ti, alpha[1] * tr);
      if (do_beta) {
        double br = fma(beta[0], c[0], -(beta[1] * c[1]));
        double bi = fma(beta[0], c[1], beta[1] * c[0]);
        re += br; im += bi;
      }
      c[0] = re; c[1] = im;
    }
}

/* ------------------------------------------------------------------------ O-bound */
/* A priori bound on |(op(A)op(B))_ij - T_ij| for the triangle set (exact arithmetic before
 * the final rounding).  With truncated digits every partial digit sum has the sign of a' and
 * |a' - sum_{t<=p} d_t 2^-7t| < 2^-7p.  Writing a' = A_s + rA (|rA| < 2^-7s), b' likewise,
 * a'b' - sum_{p+q<=s+1} = A_s rB + rA B_s + rA rB + (dropped pairs with p+q > s+1, p,q <= s),
 * and |dropped| <= sum_{p=2..s} |d_p| 2^-7p * |sum_{q>s+1-p} d_q 2^-7q| < sum_p 2^-7(p-1) 2^-7(s+1-p)
 * = (s-1) 2^-7s.  Hence per term: |a'||rB| + |rA||b'| + |rA||rB| + (s-1) 2^-7s [both nonzero],
 * bounded by 2^-7s (|a'| + |b'| + 2^-7s + (s-1)).  The bound returned is
 *   2^{e_i+f_j-7s} sum_l (|a'_il| + |b'_lj| + s) [a_il != 0 and b_lj != 0]
 * plus the final rounding u |T_ij| is NOT included (callers add it).  out: m x n, ld m. */
ORC_EXPORT void orc_emu_bound(char ta, char tb, int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                              const double* B, int64_t ldb, int s, double* out) {
  int32_t* e = (int32_t*)malloc(sizeof(int32_t) * m);
  int32_t* f = (int32_t*)malloc(sizeof(int32_t) * n);
  for (int64_t i = 0; i < m; ++i) {
    double amax = 0; for (int64_t l = 0; l < k; ++l) { double a = fabs(op_r(ta, A, lda, i, l)); if (a > amax) amax = a; }
    int ex = 0; if (amax != 0) frexp(amax, &ex); e[i] = ex;
  }
  char tbf = (tb == 'N' || tb == 'n') ? 'T' : 'N';
  for (int64_t j = 0; j < n; ++j) {
    double amax = 0; for (int64_t l = 0; l < k; ++l) { double a = fabs(op_r(tbf, B, ldb, j, l)); if (a > amax) amax = a; }
    int ex = 0; if (amax != 0) frexp(amax, &ex); f[j] = ex;
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double acc = 0;
      for (int64_t l = 0; l < k; ++l) {
        double a = op_r(ta, A, lda, i, l), b = op_r(tb, B, ldb, l, j);
        if (a == 0.0 || b == 0.0) continue;
        acc += fabs(ldexp(a, -e[i])) + fabs(ldexp(b, -f[j])) + (double)s;
      }
      out[i + j * m] = ldexp(acc * (1.0 + 4.0 * k * ldexp(1.0, -53)), e[i] + f[j] - 7 * s);
    }
  free(e); free(f);
}

/* ===================================================================== selector (adaptive s)
 * The adaptive split number the paper proposes (Sec. 4), as restated for this project: an MLP
 * 24 -> 64 -> 64 -> 11 over per-GEMM features predicts the minimal sufficient slice count.
 * theta = [W1 (64x24), b1 (64), W2 (64x64), b2 (64), W3 (11x64), b3 (11)], row-major [out][in].
 */
#define SEL_IN 24
#define SEL_H 64
#define SEL_OUT 11
#define O_W1 0
#define O_B1 (O_W1 + SEL_H * SEL_IN)
#define O_W2 (O_B1 + SEL_H)
#define O_B2 (O_W2 + SEL_H * SEL_H)
#define O_W3 (O_B2 + SEL_H)
#define O_B3 (O_W3 + SEL_OUT * SEL_H)
#define SEL_PARAMS (O_B3 + SEL_OUT)

/* BF16 rounding of a float: keep the top 16 bits of the IEEE single, rounding the dropped 16
 * bits to nearest with ties to even (finite inputs). */
static float bf16_round(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}
ORC_EXPORT float orc_bf16_round(float x) { return bf16_round(x); }

/* Mean cross-entropy of the MLP on a batch and its gradient, in FP64, with the weights rounded
 * to BF16 in the forward pass and the gradient passed straight through that rounding.
 * X: [B][24] normalised features (float); y: [B] classes 0..10; grad: [SEL_PARAMS] or NULL. */
ORC_EXPORT double orc_mlp_loss_grad(const float* theta, const float* X, const int* y, int B, double* grad) {
  double W1[SEL_H * SEL_IN], W2[SEL_H * SEL_H], W3[SEL_OUT * SEL_H];
  for (int i = 0; i < SEL_H * SEL_IN; ++i) W1[i] = bf16_round(theta[O_W1 + i]);
  for (int i = 0; i < SEL_H * SEL_H; ++i) W2[i] = bf16_round(theta[O_W2 + i]);
  for (int i = 0; i < SEL_OUT * SEL_H; ++i) W3[i] = bf16_round(theta[O_W3 + i]);
  if (grad) memset(grad, 0, sizeof(double) * SEL_PARAMS);
  double loss = 0.0;
  for (int b = 0; b < B; ++b) {
    const float* x = X + (size_t)b * SEL_IN;
    double h1[SEL_H], h2[SEL_H], z[SEL_OUT], p[SEL_OUT];
    for (int o = 0; o < SEL_H; ++o) {
      double a = theta[O_B1 + o];
      for (int j = 0; j < SEL_IN; ++j) a += W1[o * SEL_IN + j] * (double)x[j];
      h1[o] = a > 0 ? a : 0;
    }
    for (int o = 0; o < SEL_H; ++o) {
      double a = theta[O_B2 + o];
      for (int j = 0; j < SEL_H; ++j) a += W2[o * SEL_H + j] * h1[j];
      h2[o] = a > 0 ? a : 0;
    }
    double zm = -INFINITY;
    for (int o = 0; o < SEL_OUT; ++o) {
      double a = theta[O_B3 + o];
      for (int j = 0; j < SEL_H; ++j) a += W3[o * SEL_H + j] * h2[j];
      z[o] = a;
      if (a > zm) zm = a;
    }
    double se = 0;
    for (int o = 0; o < SEL_OUT; ++o) se += exp(z[o] - zm);
    for (int o = 0; o < SEL_OUT; ++o) p[o] = exp(z[o] - zm) / se;
    loss += (log(se) + zm - z[y[b]]) / B;
    if (!grad) continue;
    double dz[SEL_OUT], dh2[SEL_H], dh1[SEL_H];
    for (int o = 0; o < SEL_OUT; ++o) dz[o] = (p[o] - (o == y[b] ? 1.0 : 0.0)) / B;
    for (int o = 0; o < SEL_OUT; ++o) {
      grad[O_B3 + o] += dz[o];
      for (int j = 0; j < SEL_H; ++j) grad[O_W3 + o * SEL_H + j] += dz[o] * h2[j];
    }
    for (int j = 0; j < SEL_H; ++j) {
      double a = 0;
      for (int o = 0; o < SEL_OUT; ++o) a += W3[o * SEL_H + j] * dz[o];
      dh2[j] = h2[j] > 0 ? a : 0;
    }
    for (int o = 0; o < SEL_H; ++o) {
      grad[O_B2 + o] += dh2[o];
      for (int j = 0; j < SEL_H; ++j) grad[O_W2 + o * SEL_H + j] += dh2[o] * h1[j];
    }
    for (int j = 0; j < SEL_H; ++j) {
      double a = 0;
      for (int o = 0; o < SEL_H; ++o) a += W2[o * SEL_H + j] * dh2[o];
      dh1[j] = h1[j] > 0 ? a : 0;
    }
    for (int o = 0; o < SEL_H; ++o) {
      grad[O_B1 + o] += dh1[o];
      for (int j = 0; j < SEL_IN; ++j) grad[O_W1 + o * SEL_IN + j] += dh1[o] * x[j];
    }
  }
  return loss;
}

/* Inference as the GPU performs it, emulated in FP32 on the CPU: weights are BF16 bit patterns
 * (row-major [out][in]), biases FP32; each dot product is a chain of fmaf in ascending input
 * order starting from the bias; softmax with expf; the decision is the smallest class whose
 * cumulative probability reaches thr (else `fallback`), as s = s_lo + class, capped to s_cap.
 * feat: raw features [24]; probs_out: [11] or NULL.  Returns s. */
static float bf16_to_f(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float r;
  memcpy(&r, &u, 4);
  return r;
}
ORC_EXPORT int orc_mlp_select(const float* mean, const float* inv_std, const uint16_t* W1, const float* b1,
                              const uint16_t* W2, const float* b2, const uint16_t* W3, const float* b3, float thr,
                              int s_lo, int fallback, const float* feat, int s_cap, float* probs_out) {
  float x[SEL_IN], h1[SEL_H], h2[SEL_H], z[SEL_OUT];
  for (int j = 0; j < SEL_IN; ++j) x[j] = (feat[j] - mean[j]) * inv_std[j];
  for (int o = 0; o < SEL_H; ++o) {
    float a = b1[o];
    for (int j = 0; j < SEL_IN; ++j) a = fmaf(bf16_to_f(W1[o * SEL_IN + j]), x[j], a);
    h1[o] = a > 0.f ? a : 0.f;
  }
  for (int o = 0; o < SEL_H; ++o) {
    float a = b2[o];
    for (int j = 0; j < SEL_H; ++j) a = fmaf(bf16_to_f(W2[o * SEL_H + j]), h1[j], a);
    h2[o] = a > 0.f ? a : 0.f;
  }
  float zm = -INFINITY;
  for (int o = 0; o < SEL_OUT; ++o) {
    float a = b3[o];
    for (int j = 0; j < SEL_H; ++j) a = fmaf(bf16_to_f(W3[o * SEL_H + j]), h2[j], a);
    z[o] = a;
    if (a > zm) zm = a;
  }
  float ez[SEL_OUT], sum = 0.f;
  for (int o = 0; o < SEL_OUT; ++o) {
    ez[o] = expf(z[o] - zm);
    sum += ez[o];
  }
  float cum = 0.f;
  int chosen = -1;
  for (int o = 0; o < SEL_OUT; ++o) {
    const float p = ez[o] / sum;
    if (probs_out) probs_out[o] = p;
    cum += p;
    if (chosen < 0 && cum >= thr) chosen = o;
  }
  int s = chosen < 0 ? fallback : s_lo + chosen;
  if (s < 1) s = 1;
  if (s > s_cap) s = s_cap;
  return s;
}

/* The selector's features of one GEMM from their definition: log2 m, log2 n, log2 k; for the
 * rows of op(A) the fractions of entries whose exponent gap e_i - E(a) (E: frexp exponent) falls
 * in [0,4), [4,8), ..., [32,36), and the fraction that is >= 36 or zero; the same for the
 * columns of op(B); log10(target).  out: [24] floats. */
ORC_EXPORT void orc_features(char ta, char tb, int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                             const double* B, int64_t ldb, double target, float* out) {
  double hist[2][10];
  memset(hist, 0, sizeof(hist));
  for (int side = 0; side < 2; ++side) {
    const int64_t rows = side ? n : m;
    for (int64_t i = 0; i < rows; ++i) {
      double amax = 0;
      for (int64_t l = 0; l < k; ++l) {
        double v = side ? op_r(tb, B, ldb, l, i) : op_r(ta, A, lda, i, l);
        if (fabs(v) > amax) amax = fabs(v);
      }
      int e = 0;
      if (amax != 0) frexp(amax, &e);
      for (int64_t l = 0; l < k; ++l) {
        double v = side ? op_r(tb, B, ldb, l, i) : op_r(ta, A, lda, i, l);
        int bin = 9;
        if (v != 0) {
          int ev;
          frexp(v, &ev);
          int gap = e - ev;
          bin = gap < 36 ? (gap < 0 ? 0 : gap / 4) : 9;
        }
        hist[side][bin] += 1;
      }
    }
  }
  out[0] = log2f((float)m);
  out[1] = log2f((float)n);
  out[2] = log2f((float)k);
  for (int b = 0; b < 10; ++b) {
    out[3 + b] = (float)(hist[0][b] / ((double)m * (double)k));
    out[13 + b] = (float)(hist[1][b] / ((double)n * (double)k));
  }
  out[23] = (float)log10(target);
}
