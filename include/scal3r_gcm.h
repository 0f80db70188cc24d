/*
 * scal3r_gcm.h -- C ABI of the steps around the test-time-training layer in
 * Scal3R's Global Context Memory (GCM) module (arXiv 2604.08542), and the
 * GEMM they run on.
 *
 * The GCM module (Sec. 4.1, Eq. 5; Supp. "Global Context Memory module") maps
 * a chunk's tokens x [T, d] (d = H * D) to
 *     [q | k | v] = x Wqkv^T + bqkv                  (query-key-value projection)
 *     q, k scaled to unit L2 norm per head            (reading: not stated in the paper)
 *     lr = base * sigmoid(x w_eta^T + b_eta)          (token-wise learning rate, Sec. 4.2;
 *                                                      the predictor's form is a reading)
 *     o  = TTT layer (scal3r_ttt.h) on q, k, v, lr
 *     out = alpha o (o Wo^T) + x                      (gated residual, Eq. 5)
 * The caller runs, on one stream: scal3r_gcm_qkv, the TTT layer
 * (scal3r_ttt_forward), scal3r_gcm_out; backward scal3r_gcm_out_backward, the
 * layer's scal3r_ttt_backward, scal3r_gcm_qkv_backward.  Each projection is
 * one tcgen05 GEMM whose epilogue does the row work (bias, the sums of squares
 * for the per-head norms, the gate and residual), so no float32 [T, 3d] or
 * [T, d] plane exists; the small row steps left (the per-head rescale with the
 * learning-rate predictor, their backward, column sums) are 16-byte-wide
 * kernels.
 *
 * Conventions: as in scal3r_ttt.h.  x, out, q, k, v, the bf16 gradients:
 * token-major, 16-byte aligned device memory.  The handle gives H and D (its
 * head_dim); a bfloat16 handle with H <= 16 and d = H * D a multiple of 256
 * (SCAL3R_ERR_UNSUPPORTED otherwise).  Parameters: wqkv [3d, d] and wo [d, d]
 * bf16 (y = x W^T), bqkv [3d], w_eta [H, d], b_eta [H], alpha [d] float32.
 * Every entry point returns SCAL3R_OK or an error code.
 */
#ifndef SCAL3R_GCM_H
#define SCAL3R_GCM_H

#include <stddef.h>
#include <stdint.h>

#include "scal3r_ttt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C = A B^T on the tcgen05 GEMM kernel: bf16 operands, float32 accumulation.
 *   A is M x K: row-major [M][K] with a_kmajor = 1, or given as its transpose,
 *     row-major [K][M], with a_kmajor = 0; rows lda elements apart.
 *   B is N x K: row-major [N][K] with b_kmajor = 1, or as [K][N] with
 *     b_kmajor = 0; rows ldb elements apart.
 *   C is row-major [M][N], rows ldc elements apart: float32 (out_fp32 = 1;
 *     accumulate = 1 adds to C) or bf16 (out_fp32 = 0).
 * N must be a multiple of 256; M, K >= 1 (ragged edges read zeros); lda, ldb
 * multiples of 8; every pointer 16-byte aligned.  SCAL3R_ERR_UNSUPPORTED
 * otherwise.  The handle carries the status word and the profiler.
 * A float32-output product whose output tiles would leave SMs idle through a
 * long K loop (a weight gradient: small M and N, long K) runs in K ranges into
 * float32 partial planes in `workspace`, then sums them in a fixed order (the
 * number of ranges is the one with the least estimated time, counting the
 * rounds of work over the SMs and the planes' extra traffic):
 * give scal3r_ttt_gemm_workspace_size bytes (device memory, 16-byte aligned,
 * owned by the caller, not touched after the stream reaches the end of the
 * call).  With a smaller or NULL workspace the product runs unsplit; the
 * result is the same up to float32 rounding order, and bitwise reproducible
 * either way. */
int scal3r_ttt_gemm(scal3r_ttt_handle* handle, const void* a, int64_t lda, int32_t a_kmajor, const void* b,
                    int64_t ldb, int32_t b_kmajor, void* c, int64_t ldc, int32_t out_fp32, int32_t accumulate,
                    int64_t M, int64_t N, int64_t K, void* workspace, size_t workspace_bytes, void* stream);

/* Test of failure detection without a GPU fault.  With enable = 1, every
 * later scal3r_ttt_gemm on this handle stores its product as usual and then
 * has its epilogue warps wait on a shared-memory barrier that no thread
 * completes.  The wait gives up after 50 ms, and the kernel frees its tensor
 * memory and returns; scal3r_ttt_get_status then reports SCAL3R_ERR_TIMEOUT.
 * No copy or MMA is in flight at that point, so the context stays usable.
 * enable = 0 turns it off. */
int scal3r_ttt_gemm_timeout_test(scal3r_ttt_handle* handle, int32_t enable);

/* Bytes of workspace scal3r_ttt_gemm uses for an M x N x K product (0: none). */
int scal3r_ttt_gemm_workspace_size(scal3r_ttt_handle* handle, int64_t M, int64_t N, int64_t K, int32_t out_fp32,
                                   size_t* bytes);

/* Bytes of device scratch (16-byte aligned, caller-owned) that each of the
 * four calls below needs for T tokens; one buffer serves all four. */
int scal3r_gcm_workspace_size(scal3r_ttt_handle* handle, int64_t T, size_t* bytes);

/* [q | k | v] = x Wqkv^T + bqkv, q and k scaled to unit L2 norm per head,
 * lr = base_lr * sigmoid(x w_eta^T + b_eta).
 *   x [T, d] bf16; base_lr > 0.
 * Writes q, k, v [T, H, D] bf16, lr [T, H], and for the backward qn, kn
 * [T, H] (the norms before scaling, from the float32 projection) and sig
 * [T, H] (the predictor's sigmoid).  The projection's epilogue writes bf16
 * q, k, v and per-64-column sums of squares; a row kernel then scales q and k
 * (so they are rounded to bf16 twice) and evaluates the predictor. */
int scal3r_gcm_qkv(scal3r_ttt_handle* handle, const void* x, const void* wqkv, const float* bqkv, const float* w_eta,
                   const float* b_eta, float base_lr, int64_t T, void* q, void* k, void* v, float* lr, float* qn,
                   float* kn, float* sig, void* workspace, size_t workspace_bytes, void* stream);

/* out = alpha o (o Wo^T) + x (Eq. 5) in the epilogue of the output product.
 *   o [T, d] bf16 (the layer's output), x [T, d] bf16.
 * Writes out [T, d] bf16 and y = o Wo^T [T, d] bf16 (kept for dalpha). */
int scal3r_gcm_out(scal3r_ttt_handle* handle, const void* o, const void* wo, const void* x, const float* alpha,
                   int64_t T, void* out, void* y, void* stream);

/* Backward of scal3r_gcm_out for d_out [T, d] bf16 (o, wo, y, alpha of the
 * forward).  The gate is folded into the weights, so no gated copy of d_out
 * is formed:  d_o = d_out diag(alpha) Wo  [T, d] bf16 (the layer's upstream
 * gradient),  dwo = diag(alpha) d_out^T o  [d, d] float32,  dalpha [d] = the
 * sums over tokens of y o d_out (fixed order).  The residual's gradient
 * (d_out itself) is added to dx by scal3r_gcm_qkv_backward. */
int scal3r_gcm_out_backward(scal3r_ttt_handle* handle, const void* d_out, const void* o, const void* wo, const void* y,
                            const float* alpha, int64_t T, void* d_o, float* dwo, float* dalpha, void* workspace,
                            size_t workspace_bytes, void* stream);

/* Backward of scal3r_gcm_qkv and the residual: from the layer's dq, dk, dv
 * [T, H, D] bf16 and dlr [T, H], with q, k, qn, kn, sig of the forward, x,
 * wqkv, w_eta, and d_out (the module's upstream gradient):
 *   dx [T, d] float32 = d_out + dqkv Wqkv + dlogit w_eta (one GEMM over the
 *     concatenated 3d + 64 columns; the residual added in its epilogue),
 *   dwqkv [3d, d], dbqkv [3d], dw_eta [H, d], db_eta [H] float32,
 * where dqkv is the gradient of the projection before the rescale and dlogit
 * the predictor's pre-sigmoid gradient (column sums in a fixed order). */
int scal3r_gcm_qkv_backward(scal3r_ttt_handle* handle, const void* dq, const void* dk, const void* dv,
                            const float* dlr, const void* q, const void* k, const float* qn, const float* kn,
                            const float* sig, float base_lr, const void* x, const void* wqkv, const float* w_eta,
                            const void* d_out, int64_t T, float* dx, float* dwqkv, float* dbqkv, float* dw_eta,
                            float* db_eta, void* workspace, size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SCAL3R_GCM_H */
