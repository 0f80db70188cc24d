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
 * The caller runs the two projections with scal3r_ttt_gemm, the TTT layer with
 * scal3r_ttt_forward / _backward, and the row steps below, all on one stream.
 *
 * Conventions: as in scal3r_ttt.h.  x, out, q, k, v, the bf16 gradients:
 * token-major, 16-byte aligned device memory.  The handle gives H and D (its
 * head_dim); H <= 16.  Every entry point returns SCAL3R_OK or an error code.
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
 * A float32-output product with fewer 128 x 256 output tiles than half the
 * SMs (a weight gradient: small M and N, long K) runs in K ranges into
 * float32 partial planes in `workspace`, then sums them in a fixed order:
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

/* Bytes of device scratch the two backward row steps need for T tokens. */
int scal3r_gcm_workspace_size(scal3r_ttt_handle* handle, int64_t T, size_t* bytes);

/* Forward row steps after the projection.
 *   qkv_raw [T, 3d] float32 (x Wqkv^T), bqkv [3d], x [T, d] bf16,
 *   w_eta [H, d] and b_eta [H] float32, base_lr > 0.
 * Writes q, k, v [T, H, D] bf16 (q and k unit-norm per head), lr [T, H], and
 * for the backward qn, kn [T, H] (the norms before scaling) and sig [T, H]
 * (the predictor's sigmoid). */
int scal3r_gcm_prep(scal3r_ttt_handle* handle, const float* qkv_raw, const float* bqkv, const void* x,
                    const float* w_eta, const float* b_eta, float base_lr, int64_t T, void* q, void* k, void* v,
                    float* lr, float* qn, float* kn, float* sig, void* stream);

/* out = alpha o y + x (Eq. 5): y [T, d] float32 (o Wo^T), x [T, d] bf16,
 * alpha [d]; out [T, d] bf16. */
int scal3r_gcm_gate(scal3r_ttt_handle* handle, const float* y, const void* x, const float* alpha, int64_t T,
                    void* out, void* stream);

/* Backward of the gate: d_out [T, d] bf16 -> dy = alpha o d_out [T, d] bf16,
 * dx = d_out [T, d] float32 (the residual path; later GEMMs add to it), and
 * dalpha [d] = sum over tokens of y o d_out (fixed order). */
int scal3r_gcm_gate_backward(scal3r_ttt_handle* handle, const void* d_out, const float* y, const float* alpha,
                             int64_t T, void* dy, float* dx, float* dalpha, void* workspace, size_t workspace_bytes,
                             void* stream);

/* Backward of the row steps after the projection: from the TTT layer's dq,
 * dk, dv [T, H, D] bf16 and dlr [T, H], with q, k, qn, kn, sig of the forward:
 *   dqkv [T, 3d] bf16 (the gradient of qkv_raw; bias gradient dbqkv [3d]),
 *   dlogit [T, 64] bf16 (the predictor's pre-sigmoid gradient, columns >= H
 *   zero; d b_eta [H] = its column sums).
 * The remaining gradients are GEMMs: dx += dqkv Wqkv, dWqkv = dqkv^T x,
 * dx += dlogit w_eta (w_eta zero-padded to [64, d]), dw_eta = dlogit^T x. */
int scal3r_gcm_prep_backward(scal3r_ttt_handle* handle, const void* dq, const void* dk, const void* dv,
                             const float* dlr, const void* q, const void* k, const float* qn, const float* kn,
                             const float* sig, float base_lr, int64_t T, void* dqkv, void* dlogit, float* dbqkv,
                             float* db_eta, void* workspace, size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SCAL3R_GCM_H */
