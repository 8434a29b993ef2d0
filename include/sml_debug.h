/*
 * sml_debug.h -- diagnostic entry point of the GB300 localization library (not needed by
 * users of the localization API in sml.h).
 *
 * sml_debug_umma: one tensor-core product D[128][n] = A[128][k] * B[n][k]^T computed by a
 * single tcgen05.mma chain through the same shared-memory descriptors, instruction
 * descriptor and TMEM read-out that the dilated-conv kernel uses (the GEMM inside the
 * implicit-GEMM convolution of Sec. 3.2.1).  All pointers are device memory:
 *   d_a: k/e planes of [128 rows][16 bytes] (e = 8 bf16, 16 e4m3 or 4 tf32 elements per
 *        plane): element (m, kk) at byte (kk/e)*2048 + m*16 + (kk%e)*size;
 *   d_b: k/s blocks (s = 2e elements: one MMA's K) of (n/8)*256 bytes: element (nn, kk) of
 *        block kk/s at byte (nn/8)*256 + ((kk%s)/e)*128 + (nn%8)*16 + (kk%e)*size;
 *   d_d: float32 [128][n] output (row-major).
 * n in 16..256 (multiple of 16); k a positive multiple of 32; kind 0 = bf16 (kind::f16),
 * 1 = e4m3 (kind::f8f6f4), 2 = tf32 (kind::tf32, fp32 storage of which the MMA uses 19 bits);
 * d_col: first TMEM column of the accumulator (multiple of 16, d_col + n <= 512).
 * Synchronises the stream.  Returns SML_OK, SML_ERR_BAD_ARG or SML_ERR_CUDA (also when the
 * kernel's bounded wait for the MMA gave up).
 */
#ifndef SML_DEBUG_H
#define SML_DEBUG_H

#ifdef __cplusplus
extern "C" {
#endif

int sml_debug_umma(const void* d_a, const void* d_b, float* d_d, int n, int k, int kind, int d_col, void* stream);

/*
 * sml_debug_umma_mn: one tensor-core product D = A B^T with both operands MN-major, the
 * operand layout of the weight-gradient contraction (its K runs over pixels): A is M x K,
 * B is N x K, bf16.  d_a / d_b hold shared-memory images (a_bytes / b_bytes, multiples of
 * 1024) of 32-byte-swizzled planes: plane g of A covers rows 16g..16g+15 of A, one 32-byte
 * line per k (element (m, k) at logical byte g*a_plane + k*32 + (m%16)*2, then bit 4 of
 * the byte offset XOR bit 7: the 32-byte swizzle); B likewise with b_plane, its k-th line
 * at line b_shift + k (the descriptor starts b_shift lines into the planes).  M 64 or 128,
 * N 16..256 (multiple of 16), K a positive multiple of 16; a_plane, b_plane multiples of
 * 256.  d_d: float32 [128][n], TMEM lane l in row l (lanes the MMA does not write read 0).
 * Synchronises the stream.  Returns SML_OK, SML_ERR_BAD_ARG or SML_ERR_CUDA.
 */
int sml_debug_umma_mn(const void* d_a, const void* d_b, float* d_d, int m, int n, int k, int a_bytes, int b_bytes,
                      int a_plane, int b_plane, int b_shift, void* stream);

/*
 * sml_debug_set_error_word: host-side fault injection for tests of the error paths.  Writes
 * value into the context's device error word (synchronously, with no kernel involved), as
 * a tensor-core kernel does when one of its bounded waits gives up.  The next synchronous
 * call then fails with SML_ERR_CUDA, and sml_error_word reports it to asynchronous callers.
 * Returns SML_OK, SML_ERR_BAD_ARG or SML_ERR_CUDA.
 */
struct sml_ctx;
int sml_debug_set_error_word(struct sml_ctx* ctx, int value);

#ifdef __cplusplus
}
#endif

#endif
