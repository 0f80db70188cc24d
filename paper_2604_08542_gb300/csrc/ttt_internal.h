// Internal types shared by the host planner and the kernels of the
// test-time-training layer.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/scal3r_ttt.h"

namespace scal3r {

// Roles of one CTA-sized piece of work inside a chunk step.
enum Role : int32_t {
  ROLE_KEY = 0,     // forward: gradient partial of chunk j at W_j (Eq. 8)
  ROLE_APPLY = 1,   // forward: o = f_{W_j}(q) for chunk j-1 (Eq. 4)
  ROLE_BKEY = 2,    // backward: VJP of chunk j's update at W_j
  ROLE_BAPPLY = 3,  // backward: VJP of chunk j-1's apply at W_j
  ROLE_BAPPLY_K = 4,  // backward, squared-error loss by composition (BF16, head_dim 64): the apply
                      // VJP over chunk j's keys at W_j with the upstream gradient -dr, where
                      // r = v - f_W(k) is what the chunk's dot-loss gradient pieces saw as values
};

// One piece of a chunk step: a token range of one chain (sequence, head).
struct WorkItem {
  int64_t t0, t1;   // tokens [t0, t1) (global token index)
  int32_t chain;    // s * H + h
  int32_t role;
  int32_t slot;     // partial-sum slot written by this piece (-1: none)
  int32_t seq;
  int32_t wchunk;   // backward: checkpoint holding the weights (-1: w0)
  int32_t aux;      // backward: first scratch tile of this piece within its step
};

// The update of one chain that closes a chunk step: reduce the partial sums
// of its pieces (fixed order), step, normalise, checkpoint.
struct UpdateItem {
  int32_t chain;
  int32_t chunk;    // global index of the chunk whose update this is, or -1
  int32_t slot0;    // first partial slot of this chain at this step
  int32_t nslots;   // number of slots (0: no key pieces, e.g. an empty range)
  int32_t last;     // forward: 1 if chunk is the last of its sequence
  int32_t seq;
  int32_t first;    // backward: 1 if this closes chunk 0 (produces dW0)
  int32_t wslot;    // forward: checkpoint slot the new weights go to (-1: none);
                    // backward: index of the weights after `chunk` in the call's
                    // weight source (checkpoints, or the recompute buffer by chain)
};

struct Step {
  int32_t item0, nitems;  // sweep pieces
  int32_t upd0, nupd;     // updates after the sweep
  int32_t nslots;         // partial slots used in this step
  int32_t scratch_tiles;  // backward: 128-token scratch tiles of all pieces
  // backward with sparse checkpoints (every n-th chunk stored):
  int32_t wseg = 0;       // 0: the step's weights are checkpoints or w0; i > 0: recompute buffer i
  int32_t rec0 = 0;       // before the step, rerun forward steps rec0 .. rec0 + nrec - 1
  int32_t nrec = 0;       //   (their gradient pieces and updates) from the segment's first weights
  int32_t segk = 0;       //   whose sources are row segk of the plan's segment table
  int32_t npost = 0;      // backward, composed squared-error loss: the last npost pieces are
                          // ROLE_BAPPLY_K, launched after the others
  int32_t nfill = 0;      // tail fill: the last nfill pieces (before any npost) start behind
                          // the first wave, in the order their SMs are modelled to free
};

struct Plan {
  std::vector<int64_t> chunk_offsets;
  std::vector<int32_t> seq_chunk_ptr;
  int32_t H = 0, S = 0, C = 0;
  int64_t T = 0;
  int32_t max_chunks = 0;
  // forward
  std::vector<WorkItem> items;
  std::vector<UpdateItem> updates;
  std::vector<Step> steps;
  int32_t max_slots = 0;
  // backward
  std::vector<WorkItem> bitems;
  std::vector<UpdateItem> bupdates;
  std::vector<Step> bsteps;
  int32_t bmax_slots = 0;
  int64_t bscratch_tiles = 0;   // max over backward steps of the 128-token tiles of all pieces
  // sparse checkpoints (ckpt_every = n > 1): the backward recomputes W_j for j
  // not a multiple of n from the segment's first weights W_{kn}
  int32_t ckpt_every = 1;
  int64_t ckpt_slots = 0;           // stored weight sets (C with a checkpoint per chunk)
  std::vector<WorkItem> ritems;     // forward step j's gradient pieces (same slots)
  std::vector<UpdateItem> rupdates; // forward step j's updates, wslot = sequence
  std::vector<Step> rsteps;         // one per forward step j < max_chunks
  std::vector<int32_t> segsrc;      // [segment][S]: checkpoint slot of W_{kn} (-1: w0; -2: not needed)
  // composed squared-error loss (BF16, head_dim 64): per forward step, the
  // residual pieces r = v - f_{W_j}(k) over chunk j (the gradient pieces'
  // token ranges, as apply pieces)
  bool mse_compose = false;
  std::vector<WorkItem> yitems;
  std::vector<Step> ysteps;
  // device copies (owned by the handle)
  WorkItem* d_items = nullptr;
  UpdateItem* d_updates = nullptr;
  WorkItem* d_bitems = nullptr;
  UpdateItem* d_bupdates = nullptr;
  WorkItem* d_ritems = nullptr;
  WorkItem* d_yitems = nullptr;
  UpdateItem* d_rupdates = nullptr;
  int32_t* d_segsrc = nullptr;
  int64_t* d_off = nullptr;     // chunk_offsets and seq_chunk_ptr (the linear model's kernels)
  int32_t* d_ptr = nullptr;
  bool valid = false;
};

// BF16 backward: 128-token tiles per sub-piece of an update-VJP piece (pass A
// then pass B); each such piece's scratch holds one sub-piece and a copy of
// the piece's bf16 weights.
constexpr int kBwdSubTiles = 4;
constexpr int kBwdScratchTiles = kBwdSubTiles + 1;

// Scheduling knobs (the autotuner's search space).
struct Schedule {
  int32_t ctas_per_wave = 0;   // 0: number of SMs
  int32_t fwd_waves = 1;       // forward: target CTAs per step = fwd_waves * ctas_per_wave
  int32_t bwd_waves = 1;       // backward: same for the backward steps
  int32_t min_tokens = 256;    // smallest piece (tokens)
  int32_t align = 128;         // piece boundaries: multiples of the kernels' token tile from the range start
                               // (128 on the BF16 path; the float32 path's tiles are 16 tokens)
  float key_cost = 1.85f;      // forward: gradient token vs applied token (measured on GB300)
  float bkey_cost = 2.25f;     // backward: update-VJP token vs apply-VJP token (measured on GB300)
  // Tail fill (bit 0: forward steps, bit 1: backward steps; one wave only).
  // The pieces that end first take extra pieces cut off the longest ones,
  // launched behind the first wave.  Its piece-time model is in units of the
  // step's cheaper token (an applied token forward, an apply-VJP token
  // backward): a fixed cost per piece plus a cost per token (and, for an
  // update-VJP piece, per sub-piece).  Fitted to per-CTA timelines of the
  // BF16 head_dim-64 kernels on GB300 (forward: a gradient tile 2.9 us and an
  // apply tile 1.2 us, plus 5.1 and 4.0 us a piece; backward: an update-VJP
  // piece of 1 / 2 / 22 tiles 22.5 / 29.3 / 175 us, an apply-VJP tile 3.3 us).
  int32_t fill = 0;
  float fill_ovh[4] = {544.f, 427.f, 568.f, 60.f};   // per piece: KEY, APPLY, BKEY, BAPPLY
  float fill_key_tok = 2.42f;    // gradient token
  float fill_bkey_tok = 2.15f;   // update-VJP token, its sub-piece costs apart
  float fill_bkey_sub = 30.f;    // per sub-piece of kBwdSubTiles tiles
  float fill_start = 32.f;       // a CTA's start on an SM another CTA has just left
  float fill_margin = 0.02f;     // kept only if the modelled step gets this much shorter
};

struct Shape {
  int32_t H, D, F;
  int32_t lin = 0;   // 1: the linear model, one D x D matrix per chain
  int32_t P() const { return lin ? D * D : 3 * F * D; }
  int32_t R() const { return lin ? D : 2 * F + D; }
};

// Device-side parameter block of one forward/backward call.
struct Params {
  // inputs
  const void* q;
  const void* k;
  const void* v;
  const float* lr;
  const float* w0;
  int64_t w0_seq_stride;
  const void* d_o;
  const float* w_ckpt_in;
  const float* wnorm_in;
  const int64_t* off;    // linear model: device copies of chunk_offsets and seq_chunk_ptr
  const int32_t* sptr;
  // outputs
  void* o;
  float* w_ckpt;
  float* wnorm;
  float* w_final;
  void* dq;
  void* dk;
  void* dv;
  float* dlr;
  float* dw0;
  // workspace regions
  float* wm;        // [2][chains][P] master weights (double buffer by step parity)
  float* rho;       // [chains][R] row-norm targets
  float* part;      // [max_slots][P] partial sums
  float* rbuf;      // backward: [chains][P] adjoint R of the next update
  float* drho;      // backward: [chains][R]
  float* dw0_chain; // backward: [chains][P] per-chain dW0 (shared w0 only)
  float* wseg;      // backward, sparse checkpoints: [n-1][chains][P] recomputed weights
  void* rtok;       // composed squared-error loss: [T][H][D] bf16 residuals r = v - f_W(k), then -dr
  void* dk2;        //   backward: [T][H][D] bf16 dk of the apply VJP over the keys
  const void* resid_v;   // apply pieces write v - f_W(x) instead of f_W(x) (values v)
  int32_t w_items;  // 1: forward pieces read their weights as the backward does (wchunk)
  void* scratch;    // backward, BF16 path: per-piece factors of the weight adjoints
  int64_t scratch_tiles;   // its size in 96 KB tiles
  int* status;      // handle-owned status word
  // shape and options
  int32_t H, D, F, S;
  int64_t T;
  int32_t loss, norm;
  int32_t lr_mat;   // 1: lr [T, H, 3], one rate per matrix (W1, W3, W2); 0: lr [T, H]
  float eps;
};

size_t workspace_bytes(const Plan& p, const Shape& s, bool with_backward);
void carve_workspace(const Plan& p, const Shape& s, bool with_backward, void* ws, Params& prm);
int build_plan(Plan& plan, const Shape& s, const Schedule& sch, int num_sms,
               const int64_t* chunk_offsets, int32_t num_chunks,
               const int32_t* seq_chunk_ptr, int32_t num_seqs, int32_t ckpt_every = 1,
               bool mse_compose = false);

// launchers (return cudaError_t of the launch)
cudaError_t launch_prep(const Params& prm, int chains, cudaStream_t st);
cudaError_t launch_update(const Params& prm, const UpdateItem* upd, int nupd, int step, cudaStream_t st);
cudaError_t launch_bupdate(const Params& prm, const UpdateItem* upd, int nupd, int step, cudaStream_t st);
cudaError_t launch_bfinal(const Params& prm, cudaStream_t st);
cudaError_t launch_gsum(const Params& prm, const UpdateItem* upd, int nupd, float* grad, cudaStream_t st);
cudaError_t launch_loadw(const Params& prm, int chains, int buf, cudaStream_t st);
cudaError_t launch_tok_negate(const Params& prm, const WorkItem* items, int nitems, const void* src, void* dst,
                              cudaStream_t st);
cudaError_t launch_tok_add(const Params& prm, const WorkItem* items, int nitems, void* acc, const void* add,
                           cudaStream_t st);
cudaError_t launch_loadw_seg(const Params& prm, int chains, int buf, const int32_t* src, cudaStream_t st);
cudaError_t launch_gcs_update(const Params& prm, int chains, const float* w, int64_t w_stride, const float* g,
                              float* w_out, float* wnorm, cudaStream_t st);
cudaError_t launch_fp32_sweep(const Params& prm, const WorkItem* items, int nitems, int step, cudaStream_t st);
cudaError_t launch_fp32_bsweep(const Params& prm, const WorkItem* items, int nitems, int step, cudaStream_t st);
cudaError_t launch_bf16_sweep(const Params& prm, const WorkItem* items, int nitems, int step,
                              const void* tmaps, cudaStream_t st);
cudaError_t launch_bf16_bsweep(const Params& prm, const WorkItem* items, int nitems, int step,
                               const void* tmaps, cudaStream_t st);
// linear model (float32): one CTA per chain runs its whole chunk loop
bool linear_shape_supported(int D, int F);
cudaError_t prepare_linear_kernels();
cudaError_t launch_linear_forward(const Params& prm, cudaStream_t st);
cudaError_t launch_linear_backward(const Params& prm, cudaStream_t st);
// Set kernel attributes once (outside any stream capture).
cudaError_t prepare_kernels();

#ifdef __CUDACC__
// Programmatic dependent launch on the chunk-step sequence (sweep, update,
// sweep, ...).  A kernel launched with launch_pdl may be scheduled on SMs
// that the kernel ahead of it in the stream has left, before that kernel has
// finished: it does its set-up (barriers, TMEM, tensor-map prefetch), then
// pdl_wait() blocks until that kernel has completed and its writes are
// visible, before the first global access.  No kernel signals its dependents
// early (griddepcontrol.launch_dependents): a sweep's successors would then
// hold SMs while the sweep's longest pieces still run, which measured 3 %
// slower.  pdl_wait() is a no-op for a plain launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
#endif

}  // namespace scal3r
