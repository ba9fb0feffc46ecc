/*
 * hpmxp_testing.h -- test hooks of libhpmxp.so.
 *
 * These entry points expose single stages of the solver so the parity tests
 * can check each one against the CPU oracle.  They follow the conventions of
 * hpmxp.h (caller-owned device memory, stream ordered, status codes, no
 * traps) and are not needed to solve a system.
 */
#ifndef HPMXP_TESTING_H_
#define HPMXP_TESTING_H_

#include "hpmxp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One product of the LU's GEMM engine (section "Algorithmic Framework",
 * Fig. 1: low-precision operands, fp32 accumulation).
 *   A      M x K, K-major 16-bit (A(i,k) at A[i*lda + k]); 8-bit E4M3 when fp8
 *   B      N x K, K-major (B(j,k) at B[j*ldb + k])
 *   C      M x N column major 16-bit: mode 0 C = st(C - A B^T); mode 1 C = st(sign * A B^T);
 *          mode 2: C fp32 (ldc in floats), C = fl32(C - A B^T) (16-bit operands only, R NULL)
 *   R      optional row-major copy of the mode-1 result (may be NULL)
 *   fmt    0 BF16, 1 FP16 (operands of the 16-bit kinds, and C / R)
 *   fp8    1: E4M3 operands with fp32 scales sA[(i/128)*sa_ld + g], sB[(j/128)*sb_ld + g]
 *          per 128-deep slice g, folded as acc = fma(acc_g, fl32(sA*sB), acc)
 *   engine 0 tcgen05 tensor cores, 1 SIMT fp32 reference engine
 *   status device, one uint32 status word (zeroed by the caller)
 * K must be a multiple of 128; A, B 16-byte aligned; lda, ldb multiples of 16 bytes. */
hpmxp_status hpmxp_test_gemm(int M, int N, int K, const void* A, int64_t lda, const void* B, int64_t ldb,
                             void* C, int64_t ldc, void* R, int64_t ldr, int mode, float sign, int fmt,
                             int fp8, const float* sA, int sa_ld, const float* sB, int sb_ld, int engine,
                             uint32_t* status, void* stream);

/* fp64 -> 16-bit cast of the factorization input (round to nearest even).
 *   A in, n x n fp64 (lda); out, n x n 16-bit column major (ldo, even, 16-byte aligned). */
hpmxp_status hpmxp_test_cast(int64_t n, const double* A, int64_t lda, int prec, void* out, int64_t ldo,
                             void* stream);

/* Preconditioner application z = U^{-1} L^{-1} v with the 16-bit factors
 * (section "Algorithmic Framework": the factors as a left preconditioner).
 *   v, z  n x nrhs fp64 (ldv, ldz), nrhs 1..8; fp32: arithmetic in fp32
 *   ws    scratch of hpmxp_solve_workspace(n, nrhs, 1) bytes */
hpmxp_status hpmxp_test_precond(int64_t n, const void* LU, int64_t ldlu, int prec, const double* v,
                                int64_t ldv, double* z, int64_t ldz, int64_t nrhs, int fp32, void* ws,
                                size_t ws_bytes, void* stream);

/* Bound of the library's device-side waits whose running out is an error
 * (a CTA of the preconditioner polling for a block that another CTA has not
 * published yet; a stage of the tensor-core GEMM's operand, accumulator or C
 * pipeline that has not filled yet): at most `polls` polls and `ns`
 * nanoseconds of the GPU's global timer.  Kernels launched afterwards, by any
 * host thread, use it; a wait that runs out makes the call return
 * HPMXP_ETIMEOUT after the kernel has drained its own copies and tensor-core
 * work, which always keep the default bound.  A short budget is a way to make
 * those waits run out on purpose, with no peer missing and no GPU fault.
 *   polls 1 .. 2^28, ns <= 2e9; (0, 0) restores the defaults (2^28 polls, 2 s)
 * Returns HPMXP_EINVAL for other values. */
hpmxp_status hpmxp_test_set_wait_budget(long long polls, unsigned long long ns);

/* Fills the shared memory of every SM with `pattern` (one kernel on
 * `stream`), so that the next kernel starts on nonzero leftovers: a check
 * that kernels initialise every shared variable they read. */
hpmxp_status hpmxp_test_fill_smem(uint32_t pattern, void* stream);

/* The fp64 value of each 16-bit factor entry as the fp64 preconditioner
 * decodes it (section "Algorithmic Framework": the low-precision factors
 * applied in 64-bit arithmetic).  The decoding is exact and assembles the
 * fp64 bit pattern from the 16-bit fields with integer operations.
 *   codes  device, count 16-bit codes (BF16 or FP16 bit patterns)
 *   out    device, count doubles
 *   fmt    HPMXP_BF16 or HPMXP_FP16; anything else HPMXP_EINVAL
 * One kernel on `stream`; count == 0 launches nothing. */
hpmxp_status hpmxp_test_decode16(const uint16_t* codes, double* out, int64_t count, int fmt, void* stream);

/* Host-only check of the request executor's arena allocator (no device
 * memory is touched).  ops[i] > 0: allocate that many bytes, result[i] = the
 * 256-byte aligned offset or -1 when no free block fits (first fit);
 * ops[i] = -(k + 1): release the block allocated by op k, result[i] = free
 * bytes afterwards (freed blocks coalesce with their neighbours). */
int hpmxp_test_arena(size_t arena_bytes, const int64_t* ops, int nops, int64_t* result);

#ifdef __cplusplus
}
#endif
#endif /* HPMXP_TESTING_H_ */
