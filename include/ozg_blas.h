/*
 * ozg_blas.h -- drop-in Fortran BLAS entry points of libozg_blas.so.
 *
 * The paper reaches the emulation without code changes by intercepting the application's BLAS
 * calls and offloading them to the GPU (Sec. 3.1: one LD_PRELOAD carrying the interception and
 * the emulation; the mode chosen by an environment variable).  libozg_blas.so is that
 * interposition layer for this library: preloaded (LD_PRELOAD=.../libozg_blas.so) or linked
 * before the CPU BLAS, its dgemm_ / zgemm_ replace the BLAS symbols of the same name.
 *
 * Each call runs ozg_dgemm / ozg_zgemm on the current device on the caller's HOST arrays and
 * returns when C is final (synchronous, like BLAS).  Rows m..ldc-1 of C are never written.
 * Argument errors print the BLAS xerbla message on stderr and return with C untouched.  Calls
 * from several host threads are serialised.
 *
 * Data strategy (read once, at the first call; the three strategies of the paper's Sec. 2.1):
 * OZG_DATA_STRATEGY =
 *   "copy"      (default) op(A), op(B) (and C when beta != 0) are copied to GPU memory by DMA
 *               straight from the caller's arrays (cudaMemcpyAsync on pageable memory), and the
 *               m x n block of C back the same way; no CPU staging copy is made.
 *   "coherent"  the kernels read op(A), op(B), C and write C in place, in host memory, through
 *               the coherent CPU-GPU link.  No staging copy is made.
 *   "migrate"   as "coherent", but the first call that uses an array moves its pages to GPU
 *               memory (cudaMemPrefetchAsync on the page-aligned span), where later calls find
 *               it.  The CPU keeps coherent access to moved pages.  At most OZG_MIGRATE_LIMIT_MB
 *               (default: half the GPU's memory) is moved; later arrays are accessed in place.
 * "coherent" and "migrate" need a GPU that can access pageable host memory
 * (cudaDevAttrPageableMemoryAccess), and "migrate" also cudaDevAttrConcurrentManagedAccess.
 * Without them the shim prints a message and falls back to "copy" (or from "migrate" to
 * "coherent").  Results are the same bits in every strategy.  If an in-place call fails on the
 * GPU, it is redone by the next BLAS in the link chain when beta == 0.  With beta != 0 an
 * in-place failure is only reported on stderr, because C may already have been modified.
 *
 * Mode (read once, at the first call): OZG_COMPUTE_MODE, mirroring the paper's
 * OZIMMU_COMPUTE_MODE (Sec. 3.1):
 *   "dgemm"            native FP64 on the GPU
 *   "fp64_int8_<s>"    emulation with s slices, 1 <= s <= 18 (default: fp64_int8_7)
 * OZG_OFFLOAD_MIN_MNK (default 0): calls with m*n*k below it go to the next dgemm_/zgemm_ in
 * the link chain (the CPU BLAS) when one exists.
 * Integers are the LP64 BLAS interface (32-bit); the hidden trailing arguments are the Fortran
 * lengths of the two character arguments.
 */
#ifndef OZG_BLAS_H
#define OZG_BLAS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* BLAS DGEMM: C = alpha op(A) op(B) + beta C, all arguments by reference (Fortran ABI). */
void dgemm_(const char* transa, const char* transb, const int* m, const int* n, const int* k,
            const double* alpha, const double* A, const int* lda, const double* B, const int* ldb,
            const double* beta, double* C, const int* ldc, size_t transa_len, size_t transb_len);

/* BLAS ZGEMM (complex128 as interleaved double pairs; alpha, beta point to {re, im}). */
void zgemm_(const char* transa, const char* transb, const int* m, const int* n, const int* k,
            const double* alpha, const double* A, const int* lda, const double* B, const int* ldb,
            const double* beta, double* C, const int* ldc, size_t transa_len, size_t transb_len);

/* Parse a compute-mode string as OZG_COMPUTE_MODE is parsed: returns the slice count
 * (1..18), -1 for "dgemm", or 0 if the string is not a valid mode. */
int ozg_blas_parse_mode(const char* mode);

/* The mode in effect (after the first call or an explicit ozg_blas_set_mode), same encoding. */
int ozg_blas_get_mode(void);

/* Override the mode for later calls (slices 1..18 or -1); returns 0, or -1 if invalid. */
int ozg_blas_set_mode(int slices);

/* Parse a data-strategy string as OZG_DATA_STRATEGY is parsed: 0 = "copy", 1 = "coherent",
 * 2 = "migrate", or -1 if the string is not a valid strategy. */
int ozg_blas_parse_strategy(const char* strategy);

/* The data strategy in effect (same encoding).  Before the first GPU use this is the requested
 * strategy; from then on it is the one the device supports. */
int ozg_blas_get_strategy(void);

/* Request a data strategy (0, 1 or 2) for later calls; returns 0, or -1 if invalid.  The device
 * check above applies. */
int ozg_blas_set_strategy(int strategy);

/* Bytes of host arrays moved to GPU memory by the "migrate" strategy since the process started. */
long long ozg_blas_migrated_bytes(void);

/* Number of calls offloaded to the GPU / passed to the next BLAS since the process started. */
long long ozg_blas_offloaded_calls(void);
long long ozg_blas_passed_calls(void);

#ifdef __cplusplus
}
#endif

#endif /* OZG_BLAS_H */
