/*
 * scal3r_ttt.h -- C ABI of the GB300 (sm_103a) test-time-training layer of
 * Scal3R (arXiv 2604.08542), the "Global Context Memory" hot path.
 *
 * What the layer computes (per sequence s and head h, a "chain"):
 *   fast weights W = (W1 [F,D], W3 [F,D], W2 [D,F]) of the SwiGLU network
 *       f_W(x) = W2 ( SiLU(W1 x) o (W3 x) )                (Supp. Sec. A)
 *   start at w0; the sequence's tokens are cut into chunks (Sec. 4.1, 4.2);
 *   for every chunk, in order:
 *     1. one gradient step on the whole chunk at the pre-chunk weights,
 *          W <- W - grad_W sum_i lr_i L(f_W(k_i), v_i)      (Eq. 8)
 *        with the dot-product loss L = -f_W(k)^T v           (Eq. 9)
 *        or the squared error 1/2 ||f_W(k) - v||^2;
 *     2. every row of W1, W3, W2 is rescaled to a target L2 norm (its norm
 *        in w0 by default) with the clamp max(||row||, eps);
 *     3. the chunk's queries are transformed by the updated weights,
 *          o_i = f_W(q_i)                                    (Eq. 4, Sec. 4.2)
 *   The weights carry over from chunk to chunk of the same sequence (one GPU
 *   processes the chunks sequentially, Sec. 4.4).
 * The backward entry point differentiates sum(d_o * o) through the whole
 * chain of updates (gradients to q, k, v, lr and w0).
 *
 * Two BF16 implementations sit behind the same entry points, chosen by the
 * config's shape: head_dim 64 / hidden 128 runs fused per-head sweep kernels
 * (the weights of a head stay on chip for a chunk); head_dim and hidden that
 * are multiples of 256 (the paper's own AMU: one head, hd 1024, hidden
 * 4 * hd, Supp. "Global Context Memory module") run every product of a chunk
 * step as a large tcgen05 GEMM, forward and backward.  Both losses,
 * per-matrix learning rates (lr_per_matrix) and sparse checkpoints
 * (ckpt_every > 1) run on every SwiGLU path.  The head_dim-64 kernels take
 * the squared-error loss by composition: residual pieces write
 * r = v - f_W(k), the dot-loss gradient pieces take r as their values, and
 * the backward adds the apply VJP over the keys with upstream -dr.  The
 * autotuner is for the head_dim-64 path (SCAL3R_ERR_UNSUPPORTED otherwise).
 *
 * Conventions common to every entry point
 *  - T tokens, H heads, head dim D, hidden F, S sequences, C chunks.
 *  - q, k, v, o, d_o, dq, dk, dv: [T, H, D] contiguous, element type given by
 *    the config's dtype (float32 or bfloat16), 16-byte aligned device memory.
 *  - lr, dlr: [T, H] float32 device memory ([T, H, 3] with lr_per_matrix).
 *  - Fast weights of one head are P = 3*F*D float32 values packed W1, W3, W2,
 *    each row-major (the linear model: P = D*D, W row-major).  Row norms
 *    per chunk and head: R = 2*F + D (linear: D).
 *    w0 is [H, P] shared by all sequences (w0_seq_stride = 0)
 *    or one [H, P] block per sequence, w0_seq_stride floats apart.
 *  - chunk_offsets [C+1] int64 and seq_chunk_ptr [S+1] int32 are HOST arrays:
 *    chunk c covers tokens [chunk_offsets[c], chunk_offsets[c+1]) of the
 *    concatenated sequences; the chunks of sequence s are
 *    seq_chunk_ptr[s] .. seq_chunk_ptr[s+1]-1.  chunk_offsets[0] = 0, chunks
 *    are non-empty, seq_chunk_ptr is non-decreasing from 0 to C.  A sequence
 *    with no chunk is allowed (its w_final is its w0).
 *  - Every tensor is caller-owned device memory; the library owns only the
 *    handle and the schedule tables it builds for a chunk layout.  Scratch
 *    memory comes from the caller's workspace (scal3r_ttt_workspace_size).
 *  - All work is ordered on the caller's stream (a cudaStream_t passed as
 *    void*; NULL = legacy default stream).  One handle per stream at a time.
 *  - Return value: SCAL3R_OK or an error code; no exception or abort crosses
 *    the ABI.  Argument errors are found before any work is enqueued.
 *  - The first call with a new chunk layout builds and uploads a schedule
 *    (synchronous host work and one cudaMemcpy); make that call, or
 *    scal3r_ttt_plan, before capturing the stream into a CUDA graph.
 */
#ifndef SCAL3R_TTT_H
#define SCAL3R_TTT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SCAL3R_OK                 0
#define SCAL3R_ERR_INVALID_ARG    1  /* null pointer, bad offsets, bad config value */
#define SCAL3R_ERR_UNSUPPORTED    2  /* shape/dtype/loss combination not built */
#define SCAL3R_ERR_MISALIGNED     3  /* a tensor is not 16-byte aligned */
#define SCAL3R_ERR_CUDA           4  /* a CUDA runtime/driver call failed */
#define SCAL3R_ERR_TIMEOUT        5  /* a bounded device-side wait gave up */
#define SCAL3R_ERR_WORKSPACE      6  /* workspace missing or too small */
#define SCAL3R_ERR_NO_DEVICE      7  /* no sm_103 device current */
#define SCAL3R_ERR_NONFINITE      8  /* a NaN or infinity in an input or output (finite checking on;
                                        reported through scal3r_ttt_get_status) */
#define SCAL3R_ERR_BOUNDS         9  /* bounds-checking build: a kernel access left every byte range
                                        the call registered (reported through scal3r_ttt_get_status) */

/* config values */
#define SCAL3R_FP32         0   /* q,k,v,o float32: plain SIMT path */
#define SCAL3R_BF16         1   /* q,k,v,o bfloat16: tcgen05 tensor-core path */
#define SCAL3R_LOSS_DOT     0   /* L = -f(k)^T v  (Eq. 9) */
#define SCAL3R_LOSS_MSE     1   /* L = 1/2 ||f(k) - v||^2 */
#define SCAL3R_NORM_ROW_W0  0   /* rescale rows to their norm in w0 */
#define SCAL3R_NORM_NONE    1   /* no rescaling */
#define SCAL3R_NORM_UNIT    2   /* rescale rows to unit norm */

/* scal3r_ttt_config.model: the fast-weight network f_W */
#define SCAL3R_MODEL_SWIGLU 0   /* f_W(x) = W2 (SiLU(W1 x) * W3 x), Supp. Sec. A (the default) */
#define SCAL3R_MODEL_LINEAR 1   /* f_W(x) = W x, one D x D matrix (Sec. 3.2, Eq. 3-4 with a linear
                                   map): with the dot loss and no normalisation the forward is
                                   chunk-causal linear attention, a closed form for testing */

typedef struct scal3r_ttt_config {
  int32_t num_heads;    /* H >= 1 */
  int32_t head_dim;     /* D; BF16: 64 (fused per-head kernels) or a multiple of 256 up to 4096
                           (wide-weight GEMM path, e.g. the paper's AMU with hd = 1024);
                           FP32: 16 or 64 */
  int32_t hidden_dim;   /* F; BF16: 128 with D = 64, else a multiple of 256 up to 4096 (k * hd);
                           FP32: 32 or 128 */
  int32_t dtype;        /* SCAL3R_FP32 | SCAL3R_BF16 */
  int32_t loss;         /* SCAL3R_LOSS_DOT | SCAL3R_LOSS_MSE */
  int32_t weight_norm;  /* SCAL3R_NORM_ROW_W0 | SCAL3R_NORM_NONE | SCAL3R_NORM_UNIT */
  float   norm_eps;     /* clamp of the row norm; <= 0 selects 1e-6 */
  int32_t ckpt_every;   /* chunks between stored checkpoints: 0 or 1 = every chunk.  n > 1 (not
                           the linear model) stores the weights after local chunks n-1, 2n-1,
                           ... of each sequence; the backward recomputes the weights in between
                           with the forward's own gradient steps (bitwise the same), holding
                           n-1 weight sets per chain in its workspace */
  int32_t lr_per_matrix; /* 0: lr [T, H], one rate per token and head for all three matrices.
                           1 (every path): lr [T, H, 3], the rates of W1, W3, W2 in that
                           order, each matrix's gradient (Eq. 8) weighted by its own rate;
                           dlr then has the same [T, H, 3] layout */
  int32_t model;        /* SCAL3R_MODEL_SWIGLU (0) | SCAL3R_MODEL_LINEAR.  LINEAR: float32 only,
                           hidden_dim = head_dim in {16, 32, 64}, lr_per_matrix 0, ckpt_every
                           0 or 1; P = D*D (W row-major [D][D]) and wnorm keeps D row norms per
                           chunk and head.  Every loss and normalisation; forward and backward
                           only (the other entry points return SCAL3R_ERR_UNSUPPORTED) */
  int32_t deterministic; /* 0 or 1.  Every reduction of every path (partial sums over pieces,
                           sums over sequences of dw0) runs in a fixed order, so repeated calls
                           with the same inputs and layout give bitwise the same results for
                           either value; no faster non-deterministic variant exists */
} scal3r_ttt_config;

typedef struct scal3r_ttt_handle scal3r_ttt_handle;

/* Create a handle for one layer configuration on the current CUDA device.
 * Fails with SCAL3R_ERR_NO_DEVICE unless the device is compute capability
 * 10.3 (the library is built for sm_103a only). */
int scal3r_ttt_init(const scal3r_ttt_config* cfg, scal3r_ttt_handle** out);

/* Free the handle and its schedule tables.  NULL is ignored. */
void scal3r_ttt_destroy(scal3r_ttt_handle* handle);

/* Static string for a status code. */
const char* scal3r_ttt_error_string(int status);

/* Validate a chunk layout and build its schedule (work items per chunk step,
 * token split per chain).  Forward/backward calls with the same layout reuse
 * it.  Synchronous; not allowed during stream capture. */
int scal3r_ttt_plan(scal3r_ttt_handle* handle,
                    const int64_t* chunk_offsets, int32_t num_chunks,
                    const int32_t* seq_chunk_ptr, int32_t num_seqs);

/* Bytes of workspace the forward (with_backward = 0) or the backward
 * (with_backward = 1) needs for this layout.  Plans the layout if needed. */
int scal3r_ttt_workspace_size(scal3r_ttt_handle* handle,
                              const int64_t* chunk_offsets, int32_t num_chunks,
                              const int32_t* seq_chunk_ptr, int32_t num_seqs,
                              int32_t with_backward, size_t* bytes);

/* Checkpoint slots the forward writes for this layout: the number of chunks
 * C, or with ckpt_every = n > 1 the sum over sequences of floor(chunks / n). */
int scal3r_ttt_ckpt_slots(const scal3r_ttt_handle* handle, const int32_t* seq_chunk_ptr, int32_t num_seqs,
                          int64_t* slots);

/* Forward pass (Eq. 8, Eq. 9, Eq. 4 chunk by chunk; see the file comment).
 *   o        [T,H,D] out, dtype of q.
 *   w_ckpt   [C,H,P] float32 out or NULL: the weights after each chunk's
 *            update (needed by the backward).  With ckpt_every = n > 1:
 *            [scal3r_ttt_ckpt_slots, H, P], the weights after local chunks
 *            n-1, 2n-1, ... of sequence 0, then of sequence 1, ...
 *   wnorm    [C,H,R] float32 out or NULL: each row's L2 norm after the
 *            gradient step and before rescaling (needed by the backward).
 *   w_final  [S,H,P] float32 out or NULL: the weights after the last chunk
 *            of each sequence (w0 for a sequence with no chunk); pass it as
 *            the w0 of a following call to continue a stream.
 *   workspace: device scratch of at least scal3r_ttt_workspace_size(.., 0) bytes. */
int scal3r_ttt_forward(scal3r_ttt_handle* handle,
                       const void* q, const void* k, const void* v,
                       const float* lr, const float* w0, int64_t w0_seq_stride,
                       const int64_t* chunk_offsets, int32_t num_chunks,
                       const int32_t* seq_chunk_ptr, int32_t num_seqs,
                       void* o, float* w_ckpt, float* wnorm, float* w_final,
                       void* workspace, size_t workspace_bytes, void* stream);

/* The forward pass for callers that cannot allocate device memory.  The
 * paper has no counterpart of this entry point; it exists for code that may
 * not call cudaMalloc: code that runs while another thread holds a stream in
 * global-mode graph capture (cudaMalloc is refused then), plugins inside a
 * host framework that owns all device memory through its own allocator, and
 * latency-critical paths that must not enter the driver's allocator.
 *   It takes the configuration instead of a handle and no workspace; every
 * other argument means what it means for scal3r_ttt_forward, and the results
 * are those of scal3r_ttt_forward under the schedule this call uses: waves 1,
 * cost ratios 1.85 / 2.25, no tail fill (a bfloat16 handle's default
 * schedule sums a chunk's tokens over other pieces, so its results differ
 * in rounding only).  Its scratch (schedule, master weights,
 * partial sums, status word) is one fixed 32 MiB device array inside the
 * library, held by every GPU that loads the library until the process exits.
 *  - Configurations: the float32 path at any shape it takes, either loss;
 *    the bfloat16 path at head_dim 64, hidden 128 with the dot loss.  Every
 *    normalisation, a shared or per-sequence w0, one rate or per-matrix
 *    rates.  Not: the wide-weight bfloat16 shapes, the squared-error loss in
 *    bfloat16, ckpt_every > 1 (each returns SCAL3R_ERR_UNSUPPORTED or, for a
 *    ckpt_every below 0 or above 1, SCAL3R_ERR_INVALID_ARG).
 *  - The scratch needs 2 x 4P bytes of master weights per chain (sequence x
 *    head; P = 3*F*D) plus 4P bytes per piece of the busiest chunk step (the
 *    schedule cuts a step into about one piece per SM): at D=64, F=128 about
 *    90 chains fit.  A layout whose scratch does not fit returns
 *    SCAL3R_ERR_WORKSPACE before any work is enqueued.
 *  - The first call in a CUDA context sets up the array's device address;
 *    make it before any stream capture.  The schedule reaches the array
 *    through the parameters of copy kernels on `stream`: nothing is read
 *    from host memory after the call returns, and no memory copy is issued.
 *  - All calls on a device share the array and it keeps the last call's
 *    contents: calls whose GPU work overlaps race.  Order them on one stream.
 *  - A device-side wait that gives up sets the array's status word, which
 *    each call clears when it starts; scal3r_ttt_noalloc_status reads it. */
int scal3r_ttt_forward_noalloc(const scal3r_ttt_config* cfg,
                               const void* q, const void* k, const void* v,
                               const float* lr, const float* w0, int64_t w0_seq_stride,
                               const int64_t* chunk_offsets, int32_t num_chunks,
                               const int32_t* seq_chunk_ptr, int32_t num_seqs,
                               void* o, float* w_ckpt, float* wnorm, float* w_final,
                               void* stream);

/* The status word of scal3r_ttt_forward_noalloc's array (the paper has no
 * counterpart): waits for the work on `stream` to finish, returns
 * SCAL3R_OK, or SCAL3R_ERR_TIMEOUT if a kernel of an earlier call on the
 * device gave up a wait (its outputs are then undefined), and clears the
 * word.  It copies four bytes to host memory and synchronises the stream, so
 * call it outside any stream capture.  Returns SCAL3R_ERR_CUDA or
 * SCAL3R_ERR_NO_DEVICE if the runtime fails. */
int scal3r_ttt_noalloc_status(void* stream);

/* ---- Global Context Synchronisation (Sec. 4.2, Eq. 10) -------------------
 * When one chunk's tokens are spread over several processes (GPUs), the
 * chunk gradient is the sum of the per-process gradients over their token
 * shards, all taken at the same weights (Eq. 10).  These three calls split a
 * chunk step into its local parts, so that a caller can sum the gradients
 * with any collective (an all-reduce over NCCL, MPI, ...) in between:
 *   partial_grad (each process, its shard) -> all-reduce(sum) ->
 *   apply_update (each process, identical result) -> apply (its queries).
 * With one process this is exactly scal3r_ttt_forward on a layout with one
 * chunk per sequence.  The layouts passed to partial_grad and apply give
 * every sequence at most one chunk (the process's shard); otherwise
 * SCAL3R_ERR_INVALID_ARG.  The token tensors, lr, workspace and stream mean
 * what they mean for scal3r_ttt_forward.  Not available on the
 * allocation-free entry point. */

/* The gradient G = d/dW sum_i lr_i L(f_W(k_i), v_i) of Eq. 8 over the tokens
 * of each sequence's chunk, at the weights w (no update is made).
 *   w     float32 weights per sequence, [H,P] at w_seq_stride floats (0 = the
 *         same weights for every sequence), P = 3*F*D, packed W1, W3, W2.
 *   grad  [S,H,P] float32 out; a sequence without a chunk gets zeros.
 *   workspace: at least scal3r_ttt_workspace_size(.., 0) bytes for this layout. */
int scal3r_ttt_partial_grad(scal3r_ttt_handle* handle,
                            const void* k, const void* v, const float* lr,
                            const float* w, int64_t w_seq_stride,
                            const int64_t* chunk_offsets, int32_t num_chunks,
                            const int32_t* seq_chunk_ptr, int32_t num_seqs,
                            float* grad, void* workspace, size_t workspace_bytes, void* stream);

/* The update of Eq. 8 with a gradient summed outside: w_out = W - grad, with
 * every row rescaled by the handle's weight_norm (targets from w0, as in the
 * forward).  Per sequence s and head h.
 *   w     [H,P] per sequence at w_seq_stride (0 = shared); grad [S,H,P].
 *   w0    the sequence's starting weights, for the row targets, at w0_seq_stride.
 *   w_out [S,H,P] out; wnorm [S,H,2F+D] out or NULL: each row's L2 norm before
 *         rescaling (the forward's wnorm).  No workspace. */
int scal3r_ttt_apply_update(scal3r_ttt_handle* handle,
                            const float* w, int64_t w_seq_stride, const float* grad,
                            const float* w0, int64_t w0_seq_stride, int32_t num_seqs,
                            float* w_out, float* wnorm, void* stream);

/* The apply of Eq. 4, o = f_W(q), for the tokens of each sequence's chunk
 * with that sequence's weights w ([H,P] at w_seq_stride).  o [T,H,D] out in
 * the dtype of q. */
int scal3r_ttt_apply(scal3r_ttt_handle* handle, const void* q,
                     const float* w, int64_t w_seq_stride,
                     const int64_t* chunk_offsets, int32_t num_chunks,
                     const int32_t* seq_chunk_ptr, int32_t num_seqs,
                     void* o, void* workspace, size_t workspace_bytes, void* stream);

/* Backward pass: gradients of sum(d_o * o) through every chunk update.
 *   d_o      [T,H,D] upstream gradient, dtype of q.
 *   w_ckpt, wnorm: as written by the forward on the same inputs.
 *   dq, dk, dv [T,H,D] out (dtype of q); dlr [T,H] float32 out.
 *   dw0      float32 out with the shape of w0: [H,P] summed over sequences
 *            when w0_seq_stride = 0, else one block per sequence at the same
 *            stride.
 *   workspace: at least scal3r_ttt_workspace_size(.., 1) bytes. */
int scal3r_ttt_backward(scal3r_ttt_handle* handle,
                        const void* q, const void* k, const void* v,
                        const float* lr, const float* w0, int64_t w0_seq_stride,
                        const int64_t* chunk_offsets, int32_t num_chunks,
                        const int32_t* seq_chunk_ptr, int32_t num_seqs,
                        const void* d_o, const float* w_ckpt, const float* wnorm,
                        void* dq, void* dk, void* dv, float* dlr, float* dw0,
                        void* workspace, size_t workspace_bytes, void* stream);

/* How each chunk step is cut into per-CTA pieces (the autotuner's search
 * space).  Chunk lengths are part of the method and are never tuned. */
typedef struct scal3r_ttt_schedule {
  int32_t fwd_waves;        /* forward: at most fwd_waves x SM count pieces per chunk step (1..8);
                               pieces are cut so that the costliest one is as cheap as possible */
  int32_t bwd_waves;        /* backward: same for the backward steps (1..8) */
  int32_t min_piece_tokens; /* smallest piece, tokens (>= 128); the bfloat16 path.  The float32
                               path cuts pieces on its 16-token tiles with no other minimum */
  float   fwd_key_cost;     /* cost of a gradient token relative to an applied token (> 0);
                               default 2.45 for a BF16 head_dim-64 handle, else 1.85 */
  float   bwd_key_cost;     /* backward: cost of an update-VJP token vs an apply-VJP token (> 0) */
  int32_t tail_fill;        /* 0..3.  Bit 0: forward steps, bit 1: backward steps (each with one
                               wave).  The pieces modelled to end first take extra pieces cut off
                               the longest ones, launched behind the first wave; kept for a step
                               only where the library's piece-time model shortens it.  BF16
                               head_dim-64 path with the dot loss only; ignored elsewhere.
                               Default 3 for a BF16 head_dim-64 handle, else 0; the autotuner
                               tries it on and off.  Results match to rounding: a chunk's
                               token sum is split at other boundaries */
} scal3r_ttt_schedule;

/* Replace / read the handle's schedule.  Setting it drops the cached plan
 * (the next call re-plans; do it outside stream capture). */
int scal3r_ttt_set_schedule(scal3r_ttt_handle* handle, const scal3r_ttt_schedule* sch);
int scal3r_ttt_get_schedule(const scal3r_ttt_handle* handle, scal3r_ttt_schedule* sch);

/* Graph mode (default off).  When on, scal3r_ttt_forward / scal3r_ttt_backward
 * record their launch sequence into a CUDA graph the first time they see a
 * given layout and argument set, and afterwards replay it with one
 * cudaGraphLaunch on the caller's stream; a new argument set with the same
 * layout updates the executable graph in place.  The recording itself is
 * done on an internal stream, so the caller's stream may be the legacy
 * default stream.  Profiling (scal3r_ttt_profile_enable) bypasses the graph. */
int scal3r_ttt_set_graph_mode(scal3r_ttt_handle* handle, int32_t enable);

/* Autotuner: time candidate schedules on the given inputs and keep the
 * fastest in the handle (and return it in *best, with its time in *best_ms).
 * with_backward = 0 tunes the forward alone; 1 tunes forward + backward
 * (then d_o, dq, dk, dv, dlr, dw0 must be given and are overwritten).  The
 * forward outputs o, w_ckpt, wnorm are overwritten.  The tuner allocates and
 * frees its own workspace; it synchronises the stream. */
int scal3r_ttt_autotune(scal3r_ttt_handle* handle,
                        const void* q, const void* k, const void* v,
                        const float* lr, const float* w0, int64_t w0_seq_stride,
                        const int64_t* chunk_offsets, int32_t num_chunks,
                        const int32_t* seq_chunk_ptr, int32_t num_seqs,
                        void* o, float* w_ckpt, float* wnorm,
                        const void* d_o, void* dq, void* dk, void* dv, float* dlr, float* dw0,
                        int32_t with_backward, void* stream,
                        scal3r_ttt_schedule* best, float* best_ms);

/* Optional per-kernel timing.  While enabled, every kernel launch of
 * forward/backward calls on this handle is bracketed by two CUDA events
 * recorded on the call's stream (do not enable it while capturing a graph).
 * Enabling (1) clears the counters; 0 stops recording. */
int scal3r_ttt_profile_enable(scal3r_ttt_handle* handle, int32_t enable);

/* Kernel kinds of scal3r_ttt_profile_read. */
#define SCAL3R_KERNEL_FWD_SWEEP   0  /* forward token sweeps (gradient + apply pieces) */
#define SCAL3R_KERNEL_FWD_UPDATE  1  /* forward weight update + row normalisation */
#define SCAL3R_KERNEL_BWD_SWEEP   2  /* backward token sweeps */
#define SCAL3R_KERNEL_BWD_UPDATE  3  /* backward normalisation adjoint */
#define SCAL3R_KERNEL_OTHER       4  /* prologue / epilogue kernels */

/* Synchronise on the recorded events and report, for one kernel kind, the
 * number of launches, their summed device time (ms), and the summed
 * algorithmic FLOPs and HBM bytes of those launches (token-level model:
 * forward 12*D*F FLOPs per gradient token-head and 6*D*F per applied
 * token-head; backward 24*D*F per key token-head and 12*D*F per query
 * token-head, recomputation excluded). */
int scal3r_ttt_profile_read(scal3r_ttt_handle* handle, int32_t kind, int64_t* launches,
                            double* total_ms, double* flops, double* bytes);

/* Synchronise the stream and return the device status word of the last
 * calls on this handle (SCAL3R_ERR_TIMEOUT if a bounded device wait gave
 * up, SCAL3R_ERR_NONFINITE if finite checking found a NaN or infinity), then
 * clear it. */
int scal3r_ttt_get_status(scal3r_ttt_handle* handle, void* stream);

/* Finite checking (off by default).  With enable = 1, scal3r_ttt_forward and
 * scal3r_ttt_backward then scan, on the same stream and after their work, every
 * tensor they were given or wrote (forward: q, k, v, lr, w0, o, w_final;
 * backward: d_o, dq, dk, dv, dlr, dw0).  A NaN or an infinity sets the status
 * word to SCAL3R_ERR_NONFINITE, read by scal3r_ttt_get_status.  The scans are
 * memory-bound reads of those tensors; the call's own results are unchanged. */
int scal3r_ttt_set_finite_check(scal3r_ttt_handle* handle, int32_t enable);

/* Bounds checking.  A library built with SCAL3R_DEBUG_BOUNDS (the build
 * script's "bounds" variant) registers, for each scal3r_ttt_forward and
 * scal3r_ttt_backward call on a bfloat16 handle (the wide-weight path, or the
 * fused head_dim-64 kernels), the byte range of every tensor the call was
 * given and of its workspace.  Every plain global load and store of those
 * kernels and of the update kernels between them must then fall inside one
 * of them; one that does not is skipped (a load reads zeros) and the status
 * word becomes SCAL3R_ERR_BOUNDS.  TMA copies are bounded by their tensor
 * maps and are not checked here; nor are the float32 and linear paths.  The
 * extents registered are:
 *   q, k, v, o, d_o, dq, dk, dv: T*H*D elements of the dtype;
 *   lr, dlr: T*H (or T*H*3) floats;  w0, dw0: H*P floats, or
 *   (S-1)*w0_seq_stride + H*P;  w_ckpt: slots*H*P;  wnorm: C*H*(2F+D);
 *   w_final: S*H*P floats;  workspace: the bytes passed.
 * scal3r_ttt_debug_bounds(handle, tensor, shrink_bytes) registers tensor
 * number `tensor` (0 q, 1 k, 2 v, 3 lr, 4 w0, 5 o, 6 w_ckpt, 7 wnorm,
 * 8 w_final, 9 d_o, 10 dq, 11 dk, 12 dv, 13 dlr, 14 dw0, 15 workspace)
 * shrink_bytes shorter on the handle's following calls (0 restores it): a
 * test sees a violation reported while every access stays inside the real
 * buffer.  tensor = -1 only reports the build.  Returns SCAL3R_OK in a
 * bounds-checking build, SCAL3R_ERR_UNSUPPORTED otherwise,
 * SCAL3R_ERR_INVALID_ARG for a bad index or a negative shrink. */
int scal3r_ttt_debug_bounds(scal3r_ttt_handle* handle, int32_t tensor, int64_t shrink_bytes);

#ifdef __cplusplus
}
#endif

#endif /* SCAL3R_TTT_H */
