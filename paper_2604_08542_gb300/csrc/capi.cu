// extern "C" entry points of the test-time-training layer: argument checks,
// schedule cache and the launch sequence of one forward / backward call.
//
// Forward, for a layout whose longest sequence has n chunks:
//   prep (copy w0, row-norm targets)
//   for j = 0 .. n:  sweep(j)   gradient pieces of chunk j + apply pieces of
//                               chunk j-1, all at the weights W_j
//                    update(j)  W_{j+1} = normalise(W_j + sum of pieces)
// Backward, for j = n .. 0: sweep(j) (VJP pieces of chunk j's update and
// chunk j-1's apply, at W_j), update(j) (normalisation VJP), then dw0.
#include <algorithm>
#include <cstdio>
#include <cuda_bf16.h>
#include <cstring>
#include <initializer_list>
#include <functional>
#include <mutex>

#include "../../include/scal3r_gcm.h"
#include "bounds.cuh"
#include "ttt_internal.h"

namespace scal3r {
cudaError_t wide_gemm_bf16(const void* a, int64_t lda, int a_kmajor, const void* b, int64_t ldb, int b_kmajor, void* c,
                           int64_t ldc, int out_fp32, int accumulate, int64_t M, int64_t N, int64_t K, void* ws,
                           size_t ws_bytes, int timeout_test, int* status, cudaStream_t st);
size_t wide_gemm_workspace_bytes(int64_t M, int64_t N, int64_t K, int out_fp32);
bool gcm_heads_supported(int H);
size_t gcm_workspace_bytes(int64_t T, int H, int D);
cudaError_t gcm_qkv(const void* x, const void* wqkv, const float* bqkv, const float* w_eta, const float* b_eta,
                    float base, int64_t T, int H, int D, void* q, void* k, void* v, float* lr, float* qn, float* kn,
                    float* sig, void* ws, int* status, int sms, cudaStream_t st);
cudaError_t gcm_out(const void* o, const void* wo, const void* x, const float* alpha, int64_t T, int d, void* out,
                    void* y, int* status, cudaStream_t st);
cudaError_t gcm_out_backward(const void* d_out, const void* o, const void* wo, const void* y, const float* alpha,
                             int64_t T, int d, void* d_o, float* dwo, float* dalpha, void* ws, int* status, int sms,
                             cudaStream_t st);
cudaError_t gcm_qkv_backward(const void* dq, const void* dk, const void* dv, const float* dlr, const void* q,
                             const void* k, const float* qn, const float* kn, const float* sig, float base,
                             const void* x, const void* wqkv, const float* w_eta, const void* d_out, int64_t T, int H,
                             int D, float* dx, float* dwqkv, float* dbqkv, float* dw_eta, float* db_eta, void* ws,
                             int* status, int sms, cudaStream_t st);
bool fp32_shape_supported(int D, int F);
bool bf16_shape_supported(int D, int F);
bool update_shape_supported(int D, int F);
cudaError_t launch_bprep(const Params& prm, int chains, cudaStream_t st);
cudaError_t prepare_fp32();
cudaError_t prepare_bf16_forward();
cudaError_t prepare_bf16_backward();
bool wide_shape_supported(int D, int F);
size_t wide_workspace_bytes(const Plan& p, const Shape& s, bool with_backward, int ckpt_every, int loss,
                            int lr_per_matrix);
int64_t wide_ckpt_slot(const Plan& p, int s, int j, int n);
using WideLaunch = std::function<cudaError_t(int, double, double, const std::function<cudaError_t()>&)>;
cudaError_t wide_partial_grad(const Plan& pl, const Shape& sh, const Params& prm, float* grad, void* ws,
                              const WideLaunch& launch, cudaStream_t st);
cudaError_t wide_apply_update(const Shape& sh, const Params& prm, int S, const float* w, int64_t w_stride,
                              const float* grad, float* w_out, float* wnorm, const WideLaunch& launch, cudaStream_t st);
cudaError_t wide_apply(const Plan& pl, const Shape& sh, const Params& prm, void* ws, const WideLaunch& launch,
                       cudaStream_t st);
cudaError_t prepare_wide();
#ifdef SCAL3R_DEBUG_BOUNDS
cudaError_t wide_upload_bounds(const BoundsTable& t, cudaStream_t st);
cudaError_t bf16_fwd_upload_bounds(const BoundsTable& t, cudaStream_t st);
cudaError_t bf16_bwd_upload_bounds(const BoundsTable& t, cudaStream_t st);
cudaError_t update_upload_bounds(const BoundsTable& t, cudaStream_t st);
// Every translation unit with checked kernels keeps its own table.
static void upload_all_bounds(const BoundsTable& t, cudaStream_t st) {
  wide_upload_bounds(t, st);
  bf16_fwd_upload_bounds(t, st);
  bf16_bwd_upload_bounds(t, st);
  update_upload_bounds(t, st);
}
#endif
cudaError_t wide_forward(const Plan& pl, const Shape& sh, const Params& prm, int ckpt_every, void* ws,
                         const std::function<cudaError_t(int, double, double, const std::function<cudaError_t()>&)>& launch,
                         cudaStream_t st);
cudaError_t wide_backward(const Plan& pl, const Shape& sh, const Params& prm, int ckpt_every, void* ws,
                          const std::function<cudaError_t(int, double, double, const std::function<cudaError_t()>&)>& launch,
                          cudaStream_t st);
cudaError_t prepare_kernels() {
  cudaError_t e = prepare_fp32();
  if (e == cudaSuccess) e = prepare_bf16_forward();
  if (e == cudaSuccess) e = prepare_bf16_backward();
  if (e == cudaSuccess) e = prepare_wide();
  if (e == cudaSuccess) e = prepare_linear_kernels();
  return e;
}
}  // namespace scal3r

using namespace scal3r;

struct ProfRecord {
  int kind;
  cudaEvent_t a, b;
  double flops, bytes;
};

struct GraphSlot {
  bool valid = false;
  uint64_t key = 0;
  cudaGraphExec_t exec = nullptr;
};

struct scal3r_ttt_handle {
  scal3r_ttt_config cfg{};
  Shape shape{};
  Schedule sched{};
  int device = 0;
  int num_sms = 0;
  Plan plan;
  uint64_t plan_gen = 0;        // bumped whenever the plan changes
  int* d_status = nullptr;
  bool prof_on = false;
  std::vector<ProfRecord> prof;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  bool graph_on = false;
  bool wide = false;            // BF16 wide-weight path (head_dim, hidden multiples of 256)
  bool timeout_test = false;    // scal3r_ttt_gemm runs the bounded-wait test
  bool finite_check = false;    // scan each call's tensors for NaN / infinity afterwards
  int64_t bounds_shrink[16] = {};   // bounds-checking build: bytes taken off each registered tensor
  cudaStream_t capture_stream = nullptr;
  GraphSlot gfwd, gbwd;
};

namespace {

// Sets the status word to SCAL3R_ERR_NONFINITE (unless it already holds an
// error) if any element of the tensor is a NaN or an infinity: an all-ones
// exponent, tested on the bit pattern (bf16: 0x7F80, float32: 0x7F800000).
__global__ void finite_scan_kernel(const uint4* __restrict__ p, int64_t nvec, const void* tail, int64_t ntail,
                                   int bf16, int* status) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 x = p[i];
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (bf16)
        bad |= ((w[j] & 0x7F80u) == 0x7F80u) || ((w[j] & 0x7F800000u) == 0x7F800000u);
      else
        bad |= (w[j] & 0x7F800000u) == 0x7F800000u;
    }
  }
  if (blockIdx.x == 0)
    for (int64_t i = threadIdx.x; i < ntail; i += blockDim.x) {
      if (bf16)
        bad |= (reinterpret_cast<const uint16_t*>(tail)[i] & 0x7F80u) == 0x7F80u;
      else
        bad |= (reinterpret_cast<const uint32_t*>(tail)[i] & 0x7F800000u) == 0x7F800000u;
    }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(status, 0, SCAL3R_ERR_NONFINITE);
}

cudaError_t finite_scan(int* status, const void* p, int64_t n, bool bf16, int sms, cudaStream_t st) {
  if (!p || n <= 0) return cudaSuccess;
  const int64_t bytes = n * (bf16 ? 2 : 4);
  const int64_t nvec = bytes / 16;
  const int64_t ntail = (bytes - nvec * 16) / (bf16 ? 2 : 4);
  const void* tail = reinterpret_cast<const uint8_t*>(p) + nvec * 16;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nvec + 255) / 256, 4 * (int64_t)sms));
  finite_scan_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const uint4*>(p), nvec, tail, ntail, bf16 ? 1 : 0,
                                              status);
  return cudaGetLastError();
}

void free_plan(Plan& p) {
  if (p.d_items) cudaFree(p.d_items);
  if (p.d_updates) cudaFree(p.d_updates);
  if (p.d_bitems) cudaFree(p.d_bitems);
  if (p.d_bupdates) cudaFree(p.d_bupdates);
  if (p.d_ritems) cudaFree(p.d_ritems);
  if (p.d_yitems) cudaFree(p.d_yitems);
  p.d_yitems = nullptr;
  if (p.d_rupdates) cudaFree(p.d_rupdates);
  if (p.d_segsrc) cudaFree(p.d_segsrc);
  p.d_ritems = nullptr;
  p.d_rupdates = nullptr;
  p.d_segsrc = nullptr;
  if (p.d_off) cudaFree(p.d_off);
  if (p.d_ptr) cudaFree(p.d_ptr);
  p.d_off = nullptr;
  p.d_ptr = nullptr;
  p.d_items = nullptr;
  p.d_updates = nullptr;
  p.d_bitems = nullptr;
  p.d_bupdates = nullptr;
  p.valid = false;
}

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
  size_t n = std::max<size_t>(v.size(), 1);
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

bool same_layout(const Plan& p, const int64_t* off, int32_t C, const int32_t* ptr, int32_t S) {
  if (!p.valid || p.C != C || p.S != S) return false;
  if (std::memcmp(p.chunk_offsets.data(), off, sizeof(int64_t) * (C + 1)) != 0) return false;
  return std::memcmp(p.seq_chunk_ptr.data(), ptr, sizeof(int32_t) * (S + 1)) == 0;
}

int ensure_plan(scal3r_ttt_handle* hd, const int64_t* off, int32_t C, const int32_t* ptr, int32_t S) {
  if (!off || !ptr || C < 0 || S < 1) return SCAL3R_ERR_INVALID_ARG;
  if (same_layout(hd->plan, off, C, ptr, S)) return SCAL3R_OK;
  Plan np;
  const bool mse_compose = hd->cfg.dtype == SCAL3R_BF16 && !hd->wide && hd->cfg.loss == SCAL3R_LOSS_MSE;
  Schedule sch = hd->sched;
  if (hd->cfg.dtype == SCAL3R_FP32) {   // the float32 kernels take 16-token tiles: short chunks spread over CTAs
    sch.align = 16;
    sch.min_tokens = 16;
  }
  if (hd->cfg.dtype != SCAL3R_BF16 || hd->wide || hd->shape.lin) sch.fill = 0;   // its model is the BF16 kernels'
  int rc = build_plan(np, hd->shape, sch, hd->num_sms, off, C, ptr, S, hd->wide ? 1 : hd->cfg.ckpt_every,
                      mse_compose);
  if (rc != SCAL3R_OK) return rc;
  if (upload(&np.d_items, np.items) != cudaSuccess || upload(&np.d_updates, np.updates) != cudaSuccess ||
      upload(&np.d_bitems, np.bitems) != cudaSuccess || upload(&np.d_bupdates, np.bupdates) != cudaSuccess ||
      upload(&np.d_off, np.chunk_offsets) != cudaSuccess || upload(&np.d_ptr, np.seq_chunk_ptr) != cudaSuccess ||
      upload(&np.d_ritems, np.ritems) != cudaSuccess || upload(&np.d_rupdates, np.rupdates) != cudaSuccess ||
      upload(&np.d_segsrc, np.segsrc) != cudaSuccess || upload(&np.d_yitems, np.yitems) != cudaSuccess) {
    free_plan(np);
    return SCAL3R_ERR_CUDA;
  }
  free_plan(hd->plan);
  hd->plan = std::move(np);
  hd->plan_gen++;
  return SCAL3R_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

void drop_graph(GraphSlot& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g = GraphSlot{};
}

// Record `enqueue` (a sequence of launches on the given stream) into a graph
// on the handle's capture stream, keep it in `slot` under `key` (updating an
// existing executable graph in place when possible) and launch it on `st`.
template <class Fn>
int run_graph(scal3r_ttt_handle* hd, GraphSlot& slot, uint64_t key, cudaStream_t st, Fn enqueue) {
  if (!(slot.valid && slot.key == key)) {
    if (cudaStreamBeginCapture(hd->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return SCAL3R_ERR_CUDA;
    int rc = enqueue(hd->capture_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(hd->capture_stream, &graph);
    if (rc != SCAL3R_OK || e != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      return rc != SCAL3R_OK ? rc : SCAL3R_ERR_CUDA;
    }
    bool updated = false;
    if (slot.valid) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(slot.exec, graph, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        drop_graph(slot);
      }
    }
    if (!updated) {
      cudaGraphExec_t exec = nullptr;
      if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return SCAL3R_ERR_CUDA;
      }
      slot.exec = exec;
    }
    cudaGraphDestroy(graph);
    slot.valid = true;
    slot.key = key;
  }
  return cudaGraphLaunch(slot.exec, st) == cudaSuccess ? SCAL3R_OK : SCAL3R_ERR_CUDA;
}

cudaEvent_t pool_event(scal3r_ttt_handle* hd) {
  if (hd->pool_used == hd->pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    hd->pool.push_back(e);
  }
  return hd->pool[hd->pool_used++];
}

// Algorithmic work of one sweep launch (token-level model, recompute excluded).
void sweep_work(const scal3r_ttt_handle* hd, const WorkItem* items, int n, double& flops, double& bytes) {
  const double DF = (double)hd->shape.D * hd->shape.F;
  const double es = hd->cfg.dtype == SCAL3R_BF16 ? 2.0 : 4.0;
  const double D = hd->shape.D;
  flops = bytes = 0;
  for (int i = 0; i < n; ++i) {
    const double t = (double)(items[i].t1 - items[i].t0);
    switch (items[i].role) {
      case ROLE_KEY: flops += 12 * DF * t; bytes += t * (2 * D * es + 4); break;
      case ROLE_APPLY: flops += 6 * DF * t; bytes += t * (2 * D * es); break;
      case ROLE_BKEY: flops += 24 * DF * t; bytes += t * (4 * D * es + 8); break;
      case ROLE_BAPPLY: flops += 12 * DF * t; bytes += t * (3 * D * es); break;
    }
  }
}

// Run `fn` (one kernel launch on st), bracketed by events when profiling.
template <class Fn>
cudaError_t timed(scal3r_ttt_handle* hd, int kind, double flops, double bytes, cudaStream_t st, Fn fn) {
  if (!hd->prof_on) return fn();
  cudaEvent_t a = pool_event(hd), b = pool_event(hd);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaEventRecord(a, st);
  cudaError_t e = fn();
  cudaEventRecord(b, st);
  hd->prof.push_back({kind, a, b, flops, bytes});
  return e;
}

void fill_common(const scal3r_ttt_handle* hd, Params& prm) {
  prm.H = hd->shape.H;
  prm.D = hd->shape.D;
  prm.F = hd->shape.F;
  prm.S = hd->plan.S;
  prm.T = hd->plan.T;
  prm.loss = hd->cfg.loss;
  prm.lr_mat = hd->cfg.lr_per_matrix ? 1 : 0;
  prm.norm = hd->cfg.weight_norm;
  prm.eps = hd->cfg.norm_eps > 0.f ? hd->cfg.norm_eps : 1e-6f;
  prm.status = hd->d_status;
}

// The forward launch sequence on `st` (see the file comment).
// Composed squared-error loss (BF16, head_dim 64): the residual pieces
// r = v - f_W(k) into prm.rtok, at the step's master weights or (w_items) at
// the weights each piece names.
cudaError_t run_resid(scal3r_ttt_handle* hd, const Params& prm, const WorkItem* host_items, const WorkItem* items,
                      int n, int step, bool w_items, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  Params py = prm;
  py.q = prm.k;
  py.o = prm.rtok;
  py.resid_v = prm.v;
  py.w_items = w_items ? 1 : 0;
  double fl = 0, by = 0;
  if (hd->prof_on) sweep_work(hd, host_items, n, fl, by);
  return timed(hd, SCAL3R_KERNEL_FWD_SWEEP, fl, by, st,
               [&] { return launch_bf16_sweep(py, items, n, step, nullptr, st); });
}

int enqueue_forward(scal3r_ttt_handle* hd, const Params& prm, cudaStream_t st) {
  const Plan& pl = hd->plan;
  const int chains = pl.S * hd->shape.H;
  if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st, [&] { return launch_prep(prm, chains, st); }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  Params pk = prm;   // the gradient pieces see the residuals as their values
  if (pl.mse_compose) {
    pk.v = prm.rtok;
    // a piece's last tile reads rows past its range (masked by a zero rate):
    // they must hold finite values
    if (cudaMemsetAsync(prm.rtok, 0, (size_t)pl.T * hd->shape.H * hd->shape.D * 2, st) != cudaSuccess)
      return SCAL3R_ERR_CUDA;
  }
  for (size_t j = 0; j < pl.steps.size(); ++j) {
    const Step& s = pl.steps[j];
    if (pl.mse_compose) {
      const Step& ys = pl.ysteps[j];
      if (run_resid(hd, prm, pl.yitems.data() + ys.item0, pl.d_yitems + ys.item0, ys.nitems, (int)j, false, st) !=
          cudaSuccess)
        return SCAL3R_ERR_CUDA;
    }
    double fl = 0, by = 0;
    if (hd->prof_on) sweep_work(hd, pl.items.data() + s.item0, s.nitems, fl, by);
    cudaError_t e = cudaSuccess;
    if (s.nitems > 0)
      e = timed(hd, SCAL3R_KERNEL_FWD_SWEEP, fl, by, st, [&] {
        return hd->cfg.dtype == SCAL3R_BF16 ? launch_bf16_sweep(pk, pl.d_items + s.item0, s.nitems, (int)j, nullptr, st)
                                            : launch_fp32_sweep(pk, pl.d_items + s.item0, s.nitems, (int)j, st);
      });
    if (e != cudaSuccess) return SCAL3R_ERR_CUDA;
    if (s.nupd > 0 && timed(hd, SCAL3R_KERNEL_FWD_UPDATE, 0, 0, st, [&] {
          return launch_update(prm, pl.d_updates + s.upd0, s.nupd, (int)j, st);
        }) != cudaSuccess)
      return SCAL3R_ERR_CUDA;
  }
  return SCAL3R_OK;
}

// The backward launch sequence on `st`.
int enqueue_backward(scal3r_ttt_handle* hd, const Params& prm, cudaStream_t st) {
  const Plan& pl = hd->plan;
  const int chains = pl.S * hd->shape.H;
  if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st, [&] { return launch_bprep(prm, chains, st); }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  const bool bf = hd->cfg.dtype == SCAL3R_BF16;
  const size_t wset = (size_t)chains * hd->shape.P();   // floats of one weight set of every chain
  if (pl.mse_compose &&   // rows past a piece's range are read (and masked): keep them finite
      cudaMemsetAsync(prm.rtok, 0, (size_t)pl.T * hd->shape.H * hd->shape.D * 2, st) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  for (size_t j = 0; j < pl.bsteps.size(); ++j) {
    const Step& s = pl.bsteps[j];
    if (s.nrec > 0) {
      // sparse checkpoints: W_{kn+1} .. W_{kn+nrec} into the recompute buffer,
      // by the forward's own gradient pieces and updates from W_{kn}
      const int k0 = s.rec0;
      if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st, [&] {
            return launch_loadw_seg(prm, chains, k0 & 1, pl.d_segsrc + (size_t)s.segk * pl.S, st);
          }) != cudaSuccess)
        return SCAL3R_ERR_CUDA;
      for (int r = k0; r < k0 + s.nrec; ++r) {
        const Step& rs = pl.rsteps[r];
        Params pr = prm;
        pr.w_ckpt = prm.wseg + (size_t)(r - k0) * wset;
        pr.wnorm = nullptr;
        pr.w_final = nullptr;
        if (pl.mse_compose) {
          const Step& ys = pl.ysteps[r];
          if (run_resid(hd, prm, pl.yitems.data() + ys.item0, pl.d_yitems + ys.item0, ys.nitems, r, false, st) !=
              cudaSuccess)
            return SCAL3R_ERR_CUDA;
          pr.v = prm.rtok;
        }
        double fl = 0, by = 0;
        if (hd->prof_on) sweep_work(hd, pl.ritems.data() + rs.item0, rs.nitems, fl, by);
        if (rs.nitems > 0 && timed(hd, SCAL3R_KERNEL_FWD_SWEEP, fl, by, st, [&] {
              return bf ? launch_bf16_sweep(pr, pl.d_ritems + rs.item0, rs.nitems, r, nullptr, st)
                        : launch_fp32_sweep(pr, pl.d_ritems + rs.item0, rs.nitems, r, st);
            }) != cudaSuccess)
          return SCAL3R_ERR_CUDA;
        if (rs.nupd > 0 && timed(hd, SCAL3R_KERNEL_FWD_UPDATE, 0, 0, st, [&] {
              return launch_update(pr, pl.d_rupdates + rs.upd0, rs.nupd, r, st);
            }) != cudaSuccess)
          return SCAL3R_ERR_CUDA;
      }
    }
    Params pb = prm;   // the step's weights: checkpoints / w0, or the recompute buffer
    if (s.wseg > 0) pb.w_ckpt_in = prm.wseg + (size_t)(s.wseg - 1) * wset;
    // composed squared-error loss: the update VJPs see r = v - f_W(k) as their
    // values (their dv is dL/dr = dL/dv); then the apply VJP over the keys with
    // upstream -dr adds its dk and its weight adjoint (the last npost pieces)
    const int nmain = s.nitems - s.npost;
    const WorkItem* post = pl.d_bitems + s.item0 + nmain;
    Params pm = pb;
    if (s.npost > 0) {
      if (run_resid(hd, pb, pl.bitems.data() + s.item0 + nmain, post, s.npost, (int)j, true, st) != cudaSuccess)
        return SCAL3R_ERR_CUDA;
      pm.v = prm.rtok;
    }
    double fl = 0, by = 0;
    if (hd->prof_on) sweep_work(hd, pl.bitems.data() + s.item0, nmain, fl, by);
    cudaError_t e = cudaSuccess;
    if (nmain > 0)
      e = timed(hd, SCAL3R_KERNEL_BWD_SWEEP, fl, by, st, [&] {
        return bf ? launch_bf16_bsweep(pm, pl.d_bitems + s.item0, nmain, (int)j, nullptr, st)
                  : launch_fp32_bsweep(pm, pl.d_bitems + s.item0, nmain, (int)j, st);
      });
    if (e != cudaSuccess) return SCAL3R_ERR_CUDA;
    if (s.npost > 0) {
      Params pp = pb;
      pp.q = prm.k;
      pp.d_o = prm.rtok;
      pp.dq = prm.dk2;
      double fp = 0, bp = 0;
      if (hd->prof_on) sweep_work(hd, pl.bitems.data() + s.item0 + nmain, s.npost, fp, bp);
      if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st,
                [&] { return launch_tok_negate(pb, post, s.npost, prm.dv, prm.rtok, st); }) != cudaSuccess ||
          timed(hd, SCAL3R_KERNEL_BWD_SWEEP, fp, bp, st,
                [&] { return launch_bf16_bsweep(pp, post, s.npost, (int)j, nullptr, st); }) != cudaSuccess ||
          timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st,
                [&] { return launch_tok_add(pb, post, s.npost, prm.dk, prm.dk2, st); }) != cudaSuccess)
        return SCAL3R_ERR_CUDA;
    }
    if (s.nupd > 0 && timed(hd, SCAL3R_KERNEL_BWD_UPDATE, 0, 0, st, [&] {
          return launch_bupdate(pb, pl.d_bupdates + s.upd0, s.nupd, (int)j, st);
        }) != cudaSuccess)
      return SCAL3R_ERR_CUDA;
  }
  if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st, [&] { return launch_bfinal(prm, st); }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  return SCAL3R_OK;
}

bool valid_schedule(const scal3r_ttt_schedule& s) {
  return s.fwd_waves >= 1 && s.fwd_waves <= 8 && s.bwd_waves >= 1 && s.bwd_waves <= 8 &&
         s.min_piece_tokens >= 128 && s.fwd_key_cost > 0.f && s.bwd_key_cost > 0.f && s.tail_fill >= 0 &&
         s.tail_fill <= 3;
}

void to_internal(const scal3r_ttt_schedule& s, Schedule& o) {
  o.fwd_waves = s.fwd_waves;
  o.bwd_waves = s.bwd_waves;
  o.min_tokens = s.min_piece_tokens;
  o.key_cost = s.fwd_key_cost;
  o.bkey_cost = s.bwd_key_cost;
  o.fill = s.tail_fill;
}

void to_public(const Schedule& o, scal3r_ttt_schedule& s) {
  s.fwd_waves = o.fwd_waves;
  s.bwd_waves = o.bwd_waves;
  s.min_piece_tokens = o.min_tokens;
  s.fwd_key_cost = o.key_cost;
  s.bwd_key_cost = o.bkey_cost;
  s.tail_fill = o.fill;
}

}  // namespace

extern "C" {

const char* scal3r_ttt_error_string(int status) {
  switch (status) {
    case SCAL3R_OK: return "ok";
    case SCAL3R_ERR_INVALID_ARG: return "invalid argument";
    case SCAL3R_ERR_UNSUPPORTED: return "unsupported shape, dtype or option";
    case SCAL3R_ERR_MISALIGNED: return "tensor not 16-byte aligned";
    case SCAL3R_ERR_CUDA: return "CUDA error";
    case SCAL3R_ERR_TIMEOUT: return "a bounded device wait timed out";
    case SCAL3R_ERR_WORKSPACE: return "workspace missing or too small";
    case SCAL3R_ERR_NO_DEVICE: return "no sm_103 device";
    case SCAL3R_ERR_NONFINITE: return "a NaN or infinity in an input or output (finite checking on)";
    case SCAL3R_ERR_BOUNDS: return "an access outside every registered range (bounds-checking build)";
    default: return "unknown status";
  }
}

int scal3r_ttt_init(const scal3r_ttt_config* cfg, scal3r_ttt_handle** out) {
  if (!cfg || !out) return SCAL3R_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->num_heads < 1 || cfg->head_dim < 1 || cfg->hidden_dim < 1 || cfg->ckpt_every < 0 ||
      cfg->lr_per_matrix < 0 || cfg->lr_per_matrix > 1)
    return SCAL3R_ERR_INVALID_ARG;
  if (cfg->model != SCAL3R_MODEL_SWIGLU && cfg->model != SCAL3R_MODEL_LINEAR) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->deterministic < 0 || cfg->deterministic > 1) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->dtype != SCAL3R_FP32 && cfg->dtype != SCAL3R_BF16) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->loss != SCAL3R_LOSS_DOT && cfg->loss != SCAL3R_LOSS_MSE) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->weight_norm < 0 || cfg->weight_norm > 2) return SCAL3R_ERR_INVALID_ARG;
  const bool lin = cfg->model == SCAL3R_MODEL_LINEAR;
  // the linear model: float32, hidden_dim = head_dim, one rate per token, a checkpoint per chunk
  if (lin && (cfg->dtype != SCAL3R_FP32 || !linear_shape_supported(cfg->head_dim, cfg->hidden_dim) ||
              cfg->lr_per_matrix || cfg->ckpt_every > 1))
    return SCAL3R_ERR_UNSUPPORTED;
  if (!lin && cfg->dtype == SCAL3R_FP32 && !fp32_shape_supported(cfg->head_dim, cfg->hidden_dim))
    return SCAL3R_ERR_UNSUPPORTED;
  const bool wide = cfg->dtype == SCAL3R_BF16 && wide_shape_supported(cfg->head_dim, cfg->hidden_dim);
  // BF16: the D = 64, F = 128 path or the wide-weight path (both losses)
  if (cfg->dtype == SCAL3R_BF16 && !wide && !bf16_shape_supported(cfg->head_dim, cfg->hidden_dim))
    return SCAL3R_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SCAL3R_ERR_NO_DEVICE;
  int major = 0, minor = 0, sms = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SCAL3R_ERR_NO_DEVICE;
  if (major != 10 || minor != 3) return SCAL3R_ERR_NO_DEVICE;
  if (prepare_kernels() != cudaSuccess) return SCAL3R_ERR_CUDA;
  auto* hd = new scal3r_ttt_handle();
  hd->cfg = *cfg;
  hd->shape = Shape{cfg->num_heads, cfg->head_dim, cfg->hidden_dim, lin ? 1 : 0};
  hd->device = dev;
  hd->num_sms = sms;
  hd->wide = wide;
  if (cfg->dtype == SCAL3R_BF16 && !wide && !lin) {
    // the head_dim-64 kernels' defaults, measured on GB300 (per-CTA timelines
    // and a same-box A/B of the bench layout's step)
    hd->sched.fill = 3;
    hd->sched.key_cost = 2.45f;
  }
  if (cudaMalloc((void**)&hd->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(hd->d_status, 0, sizeof(int)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&hd->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    if (hd->d_status) cudaFree(hd->d_status);
    delete hd;
    return SCAL3R_ERR_CUDA;
  }
  *out = hd;
  return SCAL3R_OK;
}

void scal3r_ttt_destroy(scal3r_ttt_handle* hd) {
  if (!hd) return;
  for (cudaEvent_t e : hd->pool) cudaEventDestroy(e);
  drop_graph(hd->gfwd);
  drop_graph(hd->gbwd);
  if (hd->capture_stream) cudaStreamDestroy(hd->capture_stream);
  free_plan(hd->plan);
  if (hd->d_status) cudaFree(hd->d_status);
  delete hd;
}

int scal3r_ttt_plan(scal3r_ttt_handle* hd, const int64_t* off, int32_t C, const int32_t* ptr, int32_t S) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  return ensure_plan(hd, off, C, ptr, S);
}

int scal3r_ttt_workspace_size(scal3r_ttt_handle* hd, const int64_t* off, int32_t C, const int32_t* ptr,
                              int32_t S, int32_t with_backward, size_t* bytes) {
  if (!hd || !bytes) return SCAL3R_ERR_INVALID_ARG;
  int rc = ensure_plan(hd, off, C, ptr, S);
  if (rc != SCAL3R_OK) return rc;
  if (hd->shape.lin) {   // the backward's per-chain dW0 (shared w0)
    *bytes = with_backward ? (size_t)hd->plan.S * hd->shape.H * hd->shape.P() * sizeof(float) : 0;
    return SCAL3R_OK;
  }
  if (hd->wide) {
    *bytes = wide_workspace_bytes(hd->plan, hd->shape, with_backward != 0, hd->cfg.ckpt_every, hd->cfg.loss,
                                         hd->cfg.lr_per_matrix);
    return SCAL3R_OK;
  }
  *bytes = workspace_bytes(hd->plan, hd->shape, with_backward != 0);
  return SCAL3R_OK;
}

static int forward_impl(scal3r_ttt_handle* hd, const void* q, const void* k, const void* v, const float* lr,
                        const float* w0, int64_t w0_seq_stride, const int64_t* off, int32_t C,
                        const int32_t* ptr, int32_t S, void* o, float* w_ckpt, float* wnorm, float* w_final,
                        void* workspace, size_t workspace_bytes_, void* stream) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  int rc = ensure_plan(hd, off, C, ptr, S);
  if (rc != SCAL3R_OK) return rc;
  const Plan& pl = hd->plan;
  const Shape& sh = hd->shape;
  if (pl.T > 0 && (!q || !k || !v || !lr || !o)) return SCAL3R_ERR_INVALID_ARG;
  if (!w0 || w0_seq_stride < 0) return SCAL3R_ERR_INVALID_ARG;
  if (w0_seq_stride != 0 && w0_seq_stride < (int64_t)sh.H * sh.P()) return SCAL3R_ERR_INVALID_ARG;
  if (!aligned16(q) || !aligned16(k) || !aligned16(v) || !aligned16(o)) return SCAL3R_ERR_MISALIGNED;
  if (!aligned16(lr) || !aligned16(w0) || (w0_seq_stride & 3) != 0) return SCAL3R_ERR_MISALIGNED;
  if (!aligned16(w_ckpt) || !aligned16(w_final)) return SCAL3R_ERR_MISALIGNED;
  if (sh.lin) {   // the linear model: one kernel, one CTA per chain, no workspace
    Params prm;
    std::memset(&prm, 0, sizeof(prm));
    fill_common(hd, prm);
    prm.q = q;
    prm.k = k;
    prm.v = v;
    prm.lr = lr;
    prm.w0 = w0;
    prm.w0_seq_stride = w0_seq_stride;
    prm.o = o;
    prm.w_ckpt = w_ckpt;
    prm.wnorm = wnorm;
    prm.w_final = w_final;
    prm.off = pl.d_off;
    prm.sptr = pl.d_ptr;
    cudaStream_t st = (cudaStream_t)stream;
    return timed(hd, SCAL3R_KERNEL_FWD_SWEEP, 0, 0, st, [&] { return launch_linear_forward(prm, st); }) ==
                   cudaSuccess
               ? SCAL3R_OK
               : SCAL3R_ERR_CUDA;
  }
  const size_t need =
      hd->wide ? wide_workspace_bytes(pl, sh, false, hd->cfg.ckpt_every, hd->cfg.loss,
                                         hd->cfg.lr_per_matrix) : workspace_bytes(pl, sh, false);
  if (!workspace || workspace_bytes_ < need || !aligned16(workspace)) return SCAL3R_ERR_WORKSPACE;
  if (hd->wide) {
    Params prm;
    std::memset(&prm, 0, sizeof(prm));
    fill_common(hd, prm);
    prm.q = q;
    prm.k = k;
    prm.v = v;
    prm.lr = lr;
    prm.w0 = w0;
    prm.w0_seq_stride = w0_seq_stride;
    prm.o = o;
    prm.w_ckpt = w_ckpt;
    prm.wnorm = wnorm;
    prm.w_final = w_final;
    cudaStream_t st = (cudaStream_t)stream;
    auto enqueue = [&](cudaStream_t cs) -> int {
      auto launch = [&](int kind, double flops, double bytes, const std::function<cudaError_t()>& fn) {
        return timed(hd, kind == 0 ? SCAL3R_KERNEL_FWD_SWEEP : SCAL3R_KERNEL_FWD_UPDATE, flops, bytes, cs, fn);
      };
      return wide_forward(pl, sh, prm, hd->cfg.ckpt_every, workspace, launch, cs) == cudaSuccess ? SCAL3R_OK
                                                                                                  : SCAL3R_ERR_CUDA;
    };
    if (hd->graph_on && !hd->prof_on) {
      uint64_t key = fnv1a(&prm, sizeof(prm), hd->plan_gen * 0x9E3779B97F4A7C15ull + 7);
      key = fnv1a(&workspace, sizeof(workspace), key);
      return run_graph(hd, hd->gfwd, key, st, enqueue);
    }
    return enqueue(st);
  }

  Params prm;
  std::memset(&prm, 0, sizeof(prm));   // the graph key hashes the whole struct
  fill_common(hd, prm);
  prm.q = q;
  prm.k = k;
  prm.v = v;
  prm.lr = lr;
  prm.w0 = w0;
  prm.w0_seq_stride = w0_seq_stride;
  prm.o = o;
  prm.w_ckpt = w_ckpt;
  prm.wnorm = wnorm;
  prm.w_final = w_final;
  carve_workspace(pl, sh, false, workspace, prm);
  cudaStream_t st = (cudaStream_t)stream;
  if (hd->graph_on && !hd->prof_on) {
    uint64_t key = fnv1a(&prm, sizeof(prm), hd->plan_gen * 0x9E3779B97F4A7C15ull + 1);
    return run_graph(hd, hd->gfwd, key, st, [&](cudaStream_t cs) { return enqueue_forward(hd, prm, cs); });
  }
  return enqueue_forward(hd, prm, st);
}

static int backward_impl(scal3r_ttt_handle* hd, const void* q, const void* k, const void* v, const float* lr,
                        const float* w0, int64_t w0_seq_stride, const int64_t* off, int32_t C,
                        const int32_t* ptr, int32_t S, const void* d_o, const float* w_ckpt,
                        const float* wnorm, void* dq, void* dk, void* dv, float* dlr, float* dw0,
                        void* workspace, size_t workspace_bytes_, void* stream) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  int rc = ensure_plan(hd, off, C, ptr, S);
  if (rc != SCAL3R_OK) return rc;
  const Plan& pl = hd->plan;
  const Shape& sh = hd->shape;
  if (pl.T > 0 && (!q || !k || !v || !lr || !d_o || !dq || !dk || !dv || !dlr)) return SCAL3R_ERR_INVALID_ARG;
  if (pl.C > 0 && (!wnorm || (!w_ckpt && pl.ckpt_slots > 0))) return SCAL3R_ERR_INVALID_ARG;
  if (!w0 || !dw0 || w0_seq_stride < 0) return SCAL3R_ERR_INVALID_ARG;
  if (w0_seq_stride != 0 && w0_seq_stride < (int64_t)sh.H * sh.P()) return SCAL3R_ERR_INVALID_ARG;
  for (const void* p : {q, k, v, d_o, (const void*)dq, (const void*)dk, (const void*)dv, (const void*)w_ckpt,
                        (const void*)w0, (const void*)dw0})
    if (!aligned16(p)) return SCAL3R_ERR_MISALIGNED;
  if ((w0_seq_stride & 3) != 0) return SCAL3R_ERR_MISALIGNED;
  if (sh.lin) {   // the linear model: one kernel, one CTA per chain (+ the dw0 sum for a shared w0)
    const size_t lneed = w0_seq_stride ? 0 : (size_t)pl.S * sh.H * sh.P() * sizeof(float);
    if (lneed && (!workspace || workspace_bytes_ < lneed || !aligned16(workspace))) return SCAL3R_ERR_WORKSPACE;
    Params prm;
    std::memset(&prm, 0, sizeof(prm));
    fill_common(hd, prm);
    prm.q = q;
    prm.k = k;
    prm.v = v;
    prm.lr = lr;
    prm.w0 = w0;
    prm.w0_seq_stride = w0_seq_stride;
    prm.d_o = d_o;
    prm.w_ckpt_in = w_ckpt;
    prm.wnorm_in = wnorm;
    prm.dq = dq;
    prm.dk = dk;
    prm.dv = dv;
    prm.dlr = dlr;
    prm.dw0 = dw0;
    prm.dw0_chain = static_cast<float*>(workspace);
    prm.off = pl.d_off;
    prm.sptr = pl.d_ptr;
    cudaStream_t st = (cudaStream_t)stream;
    return timed(hd, SCAL3R_KERNEL_BWD_SWEEP, 0, 0, st, [&] { return launch_linear_backward(prm, st); }) ==
                   cudaSuccess
               ? SCAL3R_OK
               : SCAL3R_ERR_CUDA;
  }
  const size_t need =
      hd->wide ? wide_workspace_bytes(pl, sh, true, hd->cfg.ckpt_every, hd->cfg.loss,
                                         hd->cfg.lr_per_matrix) : workspace_bytes(pl, sh, true);
  if (!workspace || workspace_bytes_ < need || !aligned16(workspace)) return SCAL3R_ERR_WORKSPACE;

  Params prm;
  std::memset(&prm, 0, sizeof(prm));   // the graph key hashes the whole struct
  fill_common(hd, prm);
  prm.q = q;
  prm.k = k;
  prm.v = v;
  prm.lr = lr;
  prm.w0 = w0;
  prm.w0_seq_stride = w0_seq_stride;
  prm.d_o = d_o;
  prm.w_ckpt_in = w_ckpt;
  prm.wnorm_in = wnorm;
  prm.dq = dq;
  prm.dk = dk;
  prm.dv = dv;
  prm.dlr = dlr;
  prm.dw0 = dw0;
  cudaStream_t st = (cudaStream_t)stream;
  if (hd->wide) {
    auto enqueue = [&](cudaStream_t cs) -> int {
      auto launch = [&](int kind, double flops, double bytes, const std::function<cudaError_t()>& fn) {
        return timed(hd, kind == 0 ? SCAL3R_KERNEL_BWD_SWEEP : SCAL3R_KERNEL_BWD_UPDATE, flops, bytes, cs, fn);
      };
      return wide_backward(pl, sh, prm, hd->cfg.ckpt_every, workspace, launch, cs) == cudaSuccess ? SCAL3R_OK
                                                                                                   : SCAL3R_ERR_CUDA;
    };
    if (hd->graph_on && !hd->prof_on) {
      uint64_t key = fnv1a(&prm, sizeof(prm), hd->plan_gen * 0x9E3779B97F4A7C15ull + 9);
      key = fnv1a(&workspace, sizeof(workspace), key);
      return run_graph(hd, hd->gbwd, key, st, enqueue);
    }
    return enqueue(st);
  }
  carve_workspace(pl, sh, true, workspace, prm);
  if (hd->graph_on && !hd->prof_on) {
    uint64_t key = fnv1a(&prm, sizeof(prm), hd->plan_gen * 0x9E3779B97F4A7C15ull + 2);
    return run_graph(hd, hd->gbwd, key, st, [&](cudaStream_t cs) { return enqueue_backward(hd, prm, cs); });
  }
  return enqueue_backward(hd, prm, st);
}

int scal3r_ttt_set_schedule(scal3r_ttt_handle* hd, const scal3r_ttt_schedule* sch) {
  if (!hd || !sch || !valid_schedule(*sch)) return SCAL3R_ERR_INVALID_ARG;
  to_internal(*sch, hd->sched);
  free_plan(hd->plan);
  hd->plan = Plan{};
  hd->plan_gen++;
  return SCAL3R_OK;
}

int scal3r_ttt_get_schedule(const scal3r_ttt_handle* hd, scal3r_ttt_schedule* sch) {
  if (!hd || !sch) return SCAL3R_ERR_INVALID_ARG;
  to_public(hd->sched, *sch);
  return SCAL3R_OK;
}

// Bounds-checking build: the byte ranges of a call's tensors, in the order
// of scal3r_ttt_debug_bounds (null entries are not registered), uploaded to
// the wide-weight kernels' table before the call; bounds_end turns checking
// off after it.  Without the build both do nothing.
struct CallTensors {
  const void* p[16] = {};
  int64_t bytes[16] = {};
};

static CallTensors call_tensors(const scal3r_ttt_handle* hd, const void* q, const void* k, const void* v,
                                const float* lr, const float* w0, int64_t w0_seq_stride, const int64_t* off,
                                int32_t C, const int32_t* ptr, int32_t S, void* workspace, size_t workspace_bytes) {
  CallTensors ct;
  const int64_t T = off[C], H = hd->shape.H, D = hd->shape.D, P = hd->shape.P(), R = hd->shape.R();
  const int64_t elt = hd->cfg.dtype == SCAL3R_BF16 ? 2 : 4;
  const int64_t nr = hd->cfg.lr_per_matrix ? 3 : 1;
  const int64_t wbytes = ((w0_seq_stride ? (int64_t)(S - 1) * w0_seq_stride : 0) + H * P) * 4;
  int64_t slots = 0;
  scal3r_ttt_ckpt_slots(hd, ptr, S, &slots);
  const void* p[16] = {q, k, v, lr, w0};
  const int64_t b[16] = {T * H * D * elt, T * H * D * elt, T * H * D * elt, T * H * nr * 4, wbytes,
                         T * H * D * elt, slots * H * P * 4, (int64_t)C * H * R * 4, (int64_t)S * H * P * 4,
                         T * H * D * elt, T * H * D * elt, T * H * D * elt, T * H * D * elt, T * H * nr * 4, wbytes,
                         (int64_t)workspace_bytes};
  for (int i = 0; i < 16; ++i) {
    ct.p[i] = p[i];
    ct.bytes[i] = b[i];
  }
  ct.p[15] = workspace;
  return ct;
}

#ifdef SCAL3R_DEBUG_BOUNDS
constexpr bool kBoundsBuild = true;
#else
constexpr bool kBoundsBuild = false;
#endif

// A checked call: the bounds-checking build, a BF16 handle (the wide-weight
// path, or the fused head_dim-64 kernels and their update kernels) and a
// layout its planner accepts (the tensors' extents come from the plan).
static bool bounds_on(scal3r_ttt_handle* hd, const int64_t* off, int32_t C, const int32_t* ptr, int32_t S) {
  return kBoundsBuild && hd && hd->cfg.dtype == SCAL3R_BF16 && ensure_plan(hd, off, C, ptr, S) == SCAL3R_OK;
}

static void bounds_begin(const scal3r_ttt_handle* hd, const CallTensors& ct, cudaStream_t st) {
#ifdef SCAL3R_DEBUG_BOUNDS
  BoundsTable t{};
  t.status = hd->d_status;
  for (int i = 0; i < 16 && t.n < kMaxBoundsRanges; ++i) {
    if (!ct.p[i] || ct.bytes[i] <= 0) continue;
    const int64_t len = std::max<int64_t>(0, ct.bytes[i] - hd->bounds_shrink[i]);
    t.lo[t.n] = reinterpret_cast<uint64_t>(ct.p[i]);
    t.hi[t.n] = t.lo[t.n] + (uint64_t)len;
    ++t.n;
  }
  if (t.n == 0) t.n = 1;   // nothing registered: every checked access is outside (lo = hi = 0)
  upload_all_bounds(t, st);
#else
  (void)hd; (void)ct; (void)st;
#endif
}

static void bounds_end(cudaStream_t st) {
#ifdef SCAL3R_DEBUG_BOUNDS
  BoundsTable t{};
  upload_all_bounds(t, st);
#else
  (void)st;
#endif
}

int scal3r_ttt_forward(scal3r_ttt_handle* hd, const void* q, const void* k, const void* v, const float* lr,
                       const float* w0, int64_t w0_seq_stride, const int64_t* off, int32_t C,
                       const int32_t* ptr, int32_t S, void* o, float* w_ckpt, float* wnorm, float* w_final,
                       void* workspace, size_t workspace_bytes, void* stream) {
  const bool chk = bounds_on(hd, off, C, ptr, S);
  if (chk) {
    CallTensors ct = call_tensors(hd, q, k, v, lr, w0, w0_seq_stride, off, C, ptr, S, workspace, workspace_bytes);
    ct.p[5] = o;
    ct.p[6] = w_ckpt;
    ct.p[7] = wnorm;
    ct.p[8] = w_final;
    bounds_begin(hd, ct, (cudaStream_t)stream);
  }
  int rc = forward_impl(hd, q, k, v, lr, w0, w0_seq_stride, off, C, ptr, S, o, w_ckpt, wnorm, w_final, workspace,
                        workspace_bytes, stream);
  if (chk) bounds_end((cudaStream_t)stream);
  if (rc != SCAL3R_OK || !hd->finite_check) return rc;
  // inputs and outputs of the call (shapes as checked by forward_impl)
  const int64_t T = off[C], H = hd->shape.H, D = hd->shape.D, P = hd->shape.P();
  const bool bf = hd->cfg.dtype == SCAL3R_BF16;
  const int64_t nr = hd->cfg.lr_per_matrix ? 3 : 1;
  cudaStream_t st = (cudaStream_t)stream;
  int* s_ = hd->d_status;
  const int sms = hd->num_sms;
  cudaError_t e = cudaSuccess;
  for (const void* t : {q, k, v, (const void*)o})
    if (e == cudaSuccess) e = finite_scan(s_, t, T * H * D, bf, sms, st);
  if (e == cudaSuccess) e = finite_scan(s_, lr, T * H * nr, false, sms, st);
  if (e == cudaSuccess) e = finite_scan(s_, w0, (w0_seq_stride ? S : 1) * H * P, false, sms, st);
  if (e == cudaSuccess) e = finite_scan(s_, w_final, (int64_t)S * H * P, false, sms, st);
  return e == cudaSuccess ? SCAL3R_OK : SCAL3R_ERR_CUDA;
}

int scal3r_ttt_backward(scal3r_ttt_handle* hd, const void* q, const void* k, const void* v, const float* lr,
                        const float* w0, int64_t w0_seq_stride, const int64_t* off, int32_t C,
                        const int32_t* ptr, int32_t S, const void* d_o, const float* w_ckpt,
                        const float* wnorm, void* dq, void* dk, void* dv, float* dlr, float* dw0,
                        void* workspace, size_t workspace_bytes, void* stream) {
  const bool chk = bounds_on(hd, off, C, ptr, S);
  if (chk) {
    CallTensors ct = call_tensors(hd, q, k, v, lr, w0, w0_seq_stride, off, C, ptr, S, workspace, workspace_bytes);
    ct.p[6] = w_ckpt;
    ct.p[7] = wnorm;
    ct.p[9] = d_o;
    ct.p[10] = dq;
    ct.p[11] = dk;
    ct.p[12] = dv;
    ct.p[13] = dlr;
    ct.p[14] = dw0;
    bounds_begin(hd, ct, (cudaStream_t)stream);
  }
  int rc = backward_impl(hd, q, k, v, lr, w0, w0_seq_stride, off, C, ptr, S, d_o, w_ckpt, wnorm, dq, dk, dv, dlr,
                         dw0, workspace, workspace_bytes, stream);
  if (chk) bounds_end((cudaStream_t)stream);
  if (rc != SCAL3R_OK || !hd->finite_check) return rc;
  const int64_t T = off[C], H = hd->shape.H, D = hd->shape.D, P = hd->shape.P();
  const bool bf = hd->cfg.dtype == SCAL3R_BF16;
  const int64_t nr = hd->cfg.lr_per_matrix ? 3 : 1;
  cudaStream_t st = (cudaStream_t)stream;
  int* s_ = hd->d_status;
  const int sms = hd->num_sms;
  cudaError_t e = cudaSuccess;
  for (const void* t : {d_o, (const void*)dq, (const void*)dk, (const void*)dv})
    if (e == cudaSuccess) e = finite_scan(s_, t, T * H * D, bf, sms, st);
  if (e == cudaSuccess) e = finite_scan(s_, dlr, T * H * nr, false, sms, st);
  if (e == cudaSuccess) e = finite_scan(s_, dw0, (w0_seq_stride ? S : 1) * H * P, false, sms, st);
  return e == cudaSuccess ? SCAL3R_OK : SCAL3R_ERR_CUDA;
}

int scal3r_ttt_debug_bounds(scal3r_ttt_handle* hd, int32_t tensor, int64_t shrink_bytes) {
  if (!hd || tensor < -1 || tensor >= 16 || shrink_bytes < 0) return SCAL3R_ERR_INVALID_ARG;
#ifdef SCAL3R_DEBUG_BOUNDS
  if (tensor >= 0) hd->bounds_shrink[tensor] = shrink_bytes;
  return SCAL3R_OK;
#else
  return SCAL3R_ERR_UNSUPPORTED;
#endif
}

int scal3r_ttt_set_finite_check(scal3r_ttt_handle* hd, int32_t enable) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  hd->finite_check = enable != 0;
  return SCAL3R_OK;
}

int scal3r_ttt_set_graph_mode(scal3r_ttt_handle* hd, int32_t enable) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  hd->graph_on = enable != 0;
  if (!hd->graph_on) {
    drop_graph(hd->gfwd);
    drop_graph(hd->gbwd);
  }
  return SCAL3R_OK;
}

int scal3r_ttt_autotune(scal3r_ttt_handle* hd, const void* q, const void* k, const void* v, const float* lr,
                        const float* w0, int64_t w0_seq_stride, const int64_t* off, int32_t C, const int32_t* ptr,
                        int32_t S, void* o, float* w_ckpt, float* wnorm, const void* d_o, void* dq, void* dk,
                        void* dv, float* dlr, float* dw0, int32_t with_backward, void* stream,
                        scal3r_ttt_schedule* best, float* best_ms) {
  if (!hd || !best || !best_ms) return SCAL3R_ERR_INVALID_ARG;
  if (hd->wide || hd->shape.lin) return SCAL3R_ERR_UNSUPPORTED;   // the schedule knobs are the head_dim-64 path's
  if (with_backward && (!d_o || !dq || !dk || !dv || !dlr || !dw0 || !w_ckpt || !wnorm))
    return SCAL3R_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const bool graph_was = hd->graph_on, prof_was = hd->prof_on;
  hd->graph_on = false;
  hd->prof_on = false;
  const Schedule saved = hd->sched;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SCAL3R_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SCAL3R_ERR_CUDA;

  // time one schedule: 1 warm-up run, then the mean of 3 timed runs
  auto trial = [&](const Schedule& sc, bool bwd, float& ms) -> int {
    hd->sched = sc;
    free_plan(hd->plan);
    hd->plan = Plan{};
    hd->plan_gen++;
    int r = ensure_plan(hd, off, C, ptr, S);
    if (r != SCAL3R_OK) return r;
    const size_t need = workspace_bytes(hd->plan, hd->shape, true);
    if (need > ws_bytes) {
      if (ws) cudaFree(ws);
      ws = nullptr;
      if (cudaMalloc(&ws, need) != cudaSuccess) return SCAL3R_ERR_CUDA;
      ws_bytes = need;
    }
    auto once = [&]() -> int {
      int x = scal3r_ttt_forward(hd, q, k, v, lr, w0, w0_seq_stride, off, C, ptr, S, o, w_ckpt, wnorm, nullptr, ws,
                                 ws_bytes, stream);
      if (x == SCAL3R_OK && bwd)
        x = scal3r_ttt_backward(hd, q, k, v, lr, w0, w0_seq_stride, off, C, ptr, S, d_o, w_ckpt, wnorm, dq, dk, dv,
                                dlr, dw0, ws, ws_bytes, stream);
      return x;
    };
    r = once();
    if (r != SCAL3R_OK) return r;
    if (cudaEventRecord(e0, st) != cudaSuccess) return SCAL3R_ERR_CUDA;
    for (int i = 0; i < 3 && r == SCAL3R_OK; ++i) r = once();
    if (r != SCAL3R_OK) return r;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return SCAL3R_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return SCAL3R_ERR_CUDA;
    ms = t / 3.f;
    return SCAL3R_OK;
  };

  Schedule bestc = saved;
  float bestt = 0.f;
  if (rc == SCAL3R_OK) {
    // forward: pieces per step (waves; one wave with or without the tail
    // fill) and the gradient/apply cost ratio
    bool first = true;
    for (int wf : {0, 1, 2, 3})
      for (float kc : {1.6f, 1.85f, 2.1f, 2.45f}) {
        Schedule sc = saved;
        sc.fwd_waves = wf < 2 ? 1 : wf;
        sc.fill = (saved.fill & 2) | (wf == 1 ? 1 : 0);
        sc.key_cost = kc;
        float t = 0.f;
        rc = trial(sc, false, t);
        if (rc != SCAL3R_OK) break;
        if (first || t < bestt) {
          bestc = sc;
          bestt = t;
          first = false;
        }
      }
  }
  if (rc == SCAL3R_OK && with_backward) {
    // backward, with the forward fixed at its best schedule
    bool first = true;
    const Schedule fb = bestc;
    for (int wf : {0, 1, 2, 3})
      for (float kc : {2.25f, 2.95f, 3.6f}) {
        Schedule sc = fb;
        sc.bwd_waves = wf < 2 ? 1 : wf;
        sc.fill = (fb.fill & 1) | (wf == 1 ? 2 : 0);
        sc.bkey_cost = kc;
        float t = 0.f;
        rc = trial(sc, true, t);
        if (rc != SCAL3R_OK) break;
        if (first || t < bestt) {
          bestc = sc;
          bestt = t;
          first = false;
        }
      }
  }
  if (ws) {
    cudaStreamSynchronize(st);
    cudaFree(ws);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  hd->sched = rc == SCAL3R_OK ? bestc : saved;
  free_plan(hd->plan);
  hd->plan = Plan{};
  hd->plan_gen++;
  hd->graph_on = graph_was;
  hd->prof_on = prof_was;
  drop_graph(hd->gfwd);
  drop_graph(hd->gbwd);
  if (rc != SCAL3R_OK) return rc;
  to_public(bestc, *best);
  *best_ms = bestt;
  return SCAL3R_OK;
}

int scal3r_ttt_profile_enable(scal3r_ttt_handle* hd, int32_t enable) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  hd->prof.clear();
  hd->pool_used = 0;
  hd->prof_on = enable != 0;
  return SCAL3R_OK;
}

int scal3r_ttt_profile_read(scal3r_ttt_handle* hd, int32_t kind, int64_t* launches, double* total_ms,
                            double* flops, double* bytes) {
  if (!hd || !launches || !total_ms || !flops || !bytes || kind < 0 || kind > SCAL3R_KERNEL_OTHER)
    return SCAL3R_ERR_INVALID_ARG;
  *launches = 0;
  *total_ms = *flops = *bytes = 0;
  for (const auto& r : hd->prof) {
    if (r.kind != kind) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return SCAL3R_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return SCAL3R_ERR_CUDA;
    *launches += 1;
    *total_ms += ms;
    *flops += r.flops;
    *bytes += r.bytes;
  }
  return SCAL3R_OK;
}

// ---- Global Context Synchronisation (Eq. 10) ---------------------------------

namespace {
// The layout gives every sequence at most one chunk (the caller's shard of the
// chunk being synchronised).
bool one_chunk_per_seq(const Plan& pl) {
  for (int32_t s = 0; s < pl.S; ++s)
    if (pl.seq_chunk_ptr[s + 1] - pl.seq_chunk_ptr[s] > 1) return false;
  return true;
}
}  // namespace

int scal3r_ttt_partial_grad(scal3r_ttt_handle* hd, const void* k, const void* v, const float* lr, const float* w,
                            int64_t w_seq_stride, const int64_t* off, int32_t C, const int32_t* ptr, int32_t S,
                            float* grad, void* workspace, size_t workspace_bytes_, void* stream) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  if (hd->shape.lin) return SCAL3R_ERR_UNSUPPORTED;
  int rc = ensure_plan(hd, off, C, ptr, S);
  if (rc != SCAL3R_OK) return rc;
  const Plan& pl = hd->plan;
  const Shape& sh = hd->shape;
  if (!one_chunk_per_seq(pl)) return SCAL3R_ERR_INVALID_ARG;
  if (pl.T > 0 && (!k || !v || !lr)) return SCAL3R_ERR_INVALID_ARG;
  if (!w || !grad || w_seq_stride < 0) return SCAL3R_ERR_INVALID_ARG;
  if (w_seq_stride != 0 && w_seq_stride < (int64_t)sh.H * sh.P()) return SCAL3R_ERR_INVALID_ARG;
  if (!aligned16(k) || !aligned16(v) || !aligned16(lr) || !aligned16(w) || !aligned16(grad) ||
      (w_seq_stride & 3) != 0)
    return SCAL3R_ERR_MISALIGNED;
  const size_t need = hd->wide ? wide_workspace_bytes(pl, sh, false, 1, hd->cfg.loss, hd->cfg.lr_per_matrix) : workspace_bytes(pl, sh, false);
  if (!workspace || workspace_bytes_ < need || !aligned16(workspace)) return SCAL3R_ERR_WORKSPACE;
  if (hd->wide) {
    Params prm;
    std::memset(&prm, 0, sizeof(prm));
    fill_common(hd, prm);
    prm.k = k;
    prm.v = v;
    prm.lr = lr;
    prm.w0 = w;
    prm.w0_seq_stride = w_seq_stride;
    cudaStream_t st = (cudaStream_t)stream;
    auto launch = [&](int kind, double flops, double bytes, const std::function<cudaError_t()>& fn) {
      return timed(hd, kind == 0 ? SCAL3R_KERNEL_FWD_SWEEP : SCAL3R_KERNEL_OTHER, flops, bytes, st, fn);
    };
    return wide_partial_grad(pl, sh, prm, grad, workspace, launch, st) == cudaSuccess ? SCAL3R_OK : SCAL3R_ERR_CUDA;
  }

  Params prm;
  std::memset(&prm, 0, sizeof(prm));
  fill_common(hd, prm);
  prm.q = k;   // no query is read; the token maps need a valid tensor
  prm.k = k;
  prm.v = v;
  prm.lr = lr;
  prm.w0 = w;
  prm.w0_seq_stride = w_seq_stride;
  carve_workspace(pl, sh, false, workspace, prm);
  cudaStream_t st = (cudaStream_t)stream;
  const int chains = pl.S * sh.H;
  if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st, [&] { return launch_prep(prm, chains, st); }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  const Step& s0 = pl.steps[0];   // the gradient pieces of every sequence's chunk, at w
  Params pk = prm;
  if (pl.mse_compose) {   // residuals first; the gradient pieces see them as values
    if (cudaMemsetAsync(prm.rtok, 0, (size_t)pl.T * sh.H * sh.D * 2, st) != cudaSuccess) return SCAL3R_ERR_CUDA;
    const Step& ys = pl.ysteps[0];
    if (run_resid(hd, prm, pl.yitems.data() + ys.item0, pl.d_yitems + ys.item0, ys.nitems, 0, false, st) !=
        cudaSuccess)
      return SCAL3R_ERR_CUDA;
    pk.v = prm.rtok;
  }
  double fl = 0, by = 0;
  if (hd->prof_on) sweep_work(hd, pl.items.data() + s0.item0, s0.nitems, fl, by);
  if (s0.nitems > 0 && timed(hd, SCAL3R_KERNEL_FWD_SWEEP, fl, by, st, [&] {
        return hd->cfg.dtype == SCAL3R_BF16 ? launch_bf16_sweep(pk, pl.d_items + s0.item0, s0.nitems, 0, nullptr, st)
                                            : launch_fp32_sweep(pk, pl.d_items + s0.item0, s0.nitems, 0, st);
      }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st,
            [&] { return launch_gsum(prm, pl.d_updates + s0.upd0, s0.nupd, grad, st); }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  return SCAL3R_OK;
}

int scal3r_ttt_apply_update(scal3r_ttt_handle* hd, const float* w, int64_t w_seq_stride, const float* grad,
                            const float* w0, int64_t w0_seq_stride, int32_t num_seqs, float* w_out, float* wnorm,
                            void* stream) {
  if (!hd || num_seqs < 0) return SCAL3R_ERR_INVALID_ARG;
  if (hd->shape.lin) return SCAL3R_ERR_UNSUPPORTED;
  const Shape& sh = hd->shape;
  if (num_seqs == 0) return SCAL3R_OK;
  if (!w || !grad || !w0 || !w_out || w_seq_stride < 0 || w0_seq_stride < 0) return SCAL3R_ERR_INVALID_ARG;
  for (int64_t stride : {w_seq_stride, w0_seq_stride})
    if (stride != 0 && stride < (int64_t)sh.H * sh.P()) return SCAL3R_ERR_INVALID_ARG;
  if (!aligned16(w) || !aligned16(grad) || !aligned16(w0) || !aligned16(w_out) || (w_seq_stride & 3) != 0 ||
      (w0_seq_stride & 3) != 0)
    return SCAL3R_ERR_MISALIGNED;
  Params prm;
  std::memset(&prm, 0, sizeof(prm));
  fill_common(hd, prm);
  prm.S = num_seqs;
  prm.w0 = w0;
  prm.w0_seq_stride = w0_seq_stride;
  cudaStream_t st = (cudaStream_t)stream;
  if (hd->wide) {
    auto launch = [&](int, double flops, double bytes, const std::function<cudaError_t()>& fn) {
      return timed(hd, SCAL3R_KERNEL_FWD_UPDATE, flops, bytes, st, fn);
    };
    return wide_apply_update(sh, prm, num_seqs, w, w_seq_stride, grad, w_out, wnorm, launch, st) == cudaSuccess
               ? SCAL3R_OK
               : SCAL3R_ERR_CUDA;
  }
  if (timed(hd, SCAL3R_KERNEL_FWD_UPDATE, 0, 0, st, [&] {
        return launch_gcs_update(prm, num_seqs * sh.H, w, w_seq_stride, grad, w_out, wnorm, st);
      }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  return SCAL3R_OK;
}

int scal3r_ttt_apply(scal3r_ttt_handle* hd, const void* q, const float* w, int64_t w_seq_stride, const int64_t* off,
                     int32_t C, const int32_t* ptr, int32_t S, void* o, void* workspace, size_t workspace_bytes_,
                     void* stream) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  if (hd->shape.lin) return SCAL3R_ERR_UNSUPPORTED;
  int rc = ensure_plan(hd, off, C, ptr, S);
  if (rc != SCAL3R_OK) return rc;
  const Plan& pl = hd->plan;
  const Shape& sh = hd->shape;
  if (!one_chunk_per_seq(pl)) return SCAL3R_ERR_INVALID_ARG;
  if (pl.T > 0 && (!q || !o)) return SCAL3R_ERR_INVALID_ARG;
  if (!w || w_seq_stride < 0) return SCAL3R_ERR_INVALID_ARG;
  if (w_seq_stride != 0 && w_seq_stride < (int64_t)sh.H * sh.P()) return SCAL3R_ERR_INVALID_ARG;
  if (!aligned16(q) || !aligned16(o) || !aligned16(w) || (w_seq_stride & 3) != 0) return SCAL3R_ERR_MISALIGNED;
  const size_t need = hd->wide ? wide_workspace_bytes(pl, sh, false, 1, hd->cfg.loss, hd->cfg.lr_per_matrix) : workspace_bytes(pl, sh, false);
  if (!workspace || workspace_bytes_ < need || !aligned16(workspace)) return SCAL3R_ERR_WORKSPACE;
  if (pl.T == 0 || pl.steps.size() < 2) return SCAL3R_OK;   // no token to apply
  if (hd->wide) {
    Params prm;
    std::memset(&prm, 0, sizeof(prm));
    fill_common(hd, prm);
    prm.q = q;
    prm.o = o;
    prm.w0 = w;
    prm.w0_seq_stride = w_seq_stride;
    cudaStream_t st = (cudaStream_t)stream;
    auto launch = [&](int kind, double flops, double bytes, const std::function<cudaError_t()>& fn) {
      return timed(hd, kind == 0 ? SCAL3R_KERNEL_FWD_SWEEP : SCAL3R_KERNEL_OTHER, flops, bytes, st, fn);
    };
    return wide_apply(pl, sh, prm, workspace, launch, st) == cudaSuccess ? SCAL3R_OK : SCAL3R_ERR_CUDA;
  }

  Params prm;
  std::memset(&prm, 0, sizeof(prm));
  fill_common(hd, prm);
  prm.q = q;
  prm.k = q;   // no key or value is read; the token maps need a valid tensor
  prm.v = q;
  prm.o = o;
  prm.w0 = w;
  prm.w0_seq_stride = w_seq_stride;
  carve_workspace(pl, sh, false, workspace, prm);
  cudaStream_t st = (cudaStream_t)stream;
  const int chains = pl.S * sh.H;
  // chunk step 1 applies each sequence's chunk with master buffer 1
  if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st, [&] { return launch_loadw(prm, chains, 1, st); }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  const Step& s1 = pl.steps[1];
  double fl = 0, by = 0;
  if (hd->prof_on) sweep_work(hd, pl.items.data() + s1.item0, s1.nitems, fl, by);
  if (s1.nitems > 0 && timed(hd, SCAL3R_KERNEL_FWD_SWEEP, fl, by, st, [&] {
        return hd->cfg.dtype == SCAL3R_BF16 ? launch_bf16_sweep(prm, pl.d_items + s1.item0, s1.nitems, 1, nullptr, st)
                                            : launch_fp32_sweep(prm, pl.d_items + s1.item0, s1.nitems, 1, st);
      }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  return SCAL3R_OK;
}

int scal3r_ttt_ckpt_slots(const scal3r_ttt_handle* hd, const int32_t* seq_chunk_ptr, int32_t num_seqs,
                          int64_t* slots) {
  if (!hd || !seq_chunk_ptr || num_seqs < 0 || !slots) return SCAL3R_ERR_INVALID_ARG;
  const int n = hd->cfg.ckpt_every > 1 ? hd->cfg.ckpt_every : 1;
  int64_t total = 0;
  for (int s = 0; s < num_seqs; ++s) {
    const int c = seq_chunk_ptr[s + 1] - seq_chunk_ptr[s];
    if (c < 0) return SCAL3R_ERR_INVALID_ARG;
    total += c / n;
  }
  *slots = total;
  return SCAL3R_OK;
}

int scal3r_ttt_gemm_timeout_test(scal3r_ttt_handle* hd, int32_t enable) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  hd->timeout_test = enable != 0;
  return SCAL3R_OK;
}

int scal3r_ttt_gemm_workspace_size(scal3r_ttt_handle* hd, int64_t M, int64_t N, int64_t K, int32_t out_fp32,
                                   size_t* bytes) {
  if (!hd || !bytes || M < 0 || N < 0 || K < 0) return SCAL3R_ERR_INVALID_ARG;
  *bytes = wide_gemm_workspace_bytes(M, N, K, out_fp32);
  return SCAL3R_OK;
}

int scal3r_ttt_gemm(scal3r_ttt_handle* hd, const void* a, int64_t lda, int32_t a_kmajor, const void* b, int64_t ldb,
                    int32_t b_kmajor, void* c, int64_t ldc, int32_t out_fp32, int32_t accumulate, int64_t M, int64_t N,
                    int64_t K, void* workspace, size_t workspace_bytes, void* stream) {
  if (!hd || !a || !b || !c) return SCAL3R_ERR_INVALID_ARG;
  if (M <= 0 || N <= 0 || K <= 0 || N % 256 != 0 || lda % 8 != 0 || ldb % 8 != 0 || ldc < N) return SCAL3R_ERR_UNSUPPORTED;
  if ((a_kmajor ? lda < K : lda < M) || (b_kmajor ? ldb < K : ldb < N)) return SCAL3R_ERR_INVALID_ARG;
  if (!aligned16(a) || !aligned16(b) || !aligned16(c) || (ldc * (out_fp32 ? 4 : 2)) % 16 != 0)
    return SCAL3R_ERR_MISALIGNED;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = timed(hd, SCAL3R_KERNEL_OTHER, 2.0 * M * N * K, 0, st, [&] {
    return wide_gemm_bf16(a, lda, a_kmajor, b, ldb, b_kmajor, c, ldc, out_fp32, accumulate, M, N, K, workspace,
                          workspace_bytes, hd->timeout_test ? 1 : 0, hd->d_status, st);
  });
  if (e == cudaErrorInvalidValue) return SCAL3R_ERR_UNSUPPORTED;
  return e == cudaSuccess ? SCAL3R_OK : SCAL3R_ERR_CUDA;
}

// The GCM module's calls need a BF16 handle, H <= 16 and d = H * D a
// multiple of 256 (the GEMM's output tile).
static int gcm_check(const scal3r_ttt_handle* hd) {
  if (!gcm_heads_supported(hd->shape.H) || hd->cfg.dtype != SCAL3R_BF16 || (hd->shape.H * hd->shape.D) % 256 != 0)
    return SCAL3R_ERR_UNSUPPORTED;
  return SCAL3R_OK;
}

static bool all_aligned(std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (!aligned16(p)) return false;
  return true;
}

int scal3r_gcm_workspace_size(scal3r_ttt_handle* hd, int64_t T, size_t* bytes) {
  if (!hd || !bytes || T < 0) return SCAL3R_ERR_INVALID_ARG;
  *bytes = gcm_workspace_bytes(T, hd->shape.H, hd->shape.D);
  return SCAL3R_OK;
}

int scal3r_gcm_qkv(scal3r_ttt_handle* hd, const void* x, const void* wqkv, const float* bqkv, const float* w_eta,
                   const float* b_eta, float base_lr, int64_t T, void* q, void* k, void* v, float* lr, float* qn,
                   float* kn, float* sig, void* workspace, size_t workspace_bytes, void* stream) {
  if (!hd || T < 0 || !(base_lr > 0.f)) return SCAL3R_ERR_INVALID_ARG;
  int rc = gcm_check(hd);
  if (rc != SCAL3R_OK) return rc;
  if (T == 0) return SCAL3R_OK;
  if (!x || !wqkv || !bqkv || !w_eta || !b_eta || !q || !k || !v || !lr || !qn || !kn || !sig)
    return SCAL3R_ERR_INVALID_ARG;
  if (!all_aligned({x, wqkv, bqkv, w_eta, q, k, v})) return SCAL3R_ERR_MISALIGNED;
  const int H = hd->shape.H, D = hd->shape.D;
  if (!workspace || workspace_bytes < gcm_workspace_bytes(T, H, D) || !aligned16(workspace))
    return SCAL3R_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const double d = (double)H * D;
  cudaError_t e = timed(hd, SCAL3R_KERNEL_OTHER, 6.0 * T * d * d, 0, st, [&] {
    return gcm_qkv(x, wqkv, bqkv, w_eta, b_eta, base_lr, T, H, D, q, k, v, lr, qn, kn, sig, workspace, hd->d_status,
                   hd->num_sms, st);
  });
  return e == cudaSuccess ? SCAL3R_OK : SCAL3R_ERR_CUDA;
}

int scal3r_gcm_out(scal3r_ttt_handle* hd, const void* o, const void* wo, const void* x, const float* alpha, int64_t T,
                   void* out, void* y, void* stream) {
  if (!hd || T < 0) return SCAL3R_ERR_INVALID_ARG;
  int rc = gcm_check(hd);
  if (rc != SCAL3R_OK) return rc;
  if (T == 0) return SCAL3R_OK;
  if (!o || !wo || !x || !alpha || !out || !y) return SCAL3R_ERR_INVALID_ARG;
  if (!all_aligned({o, wo, x, alpha, out, y})) return SCAL3R_ERR_MISALIGNED;
  cudaStream_t st = (cudaStream_t)stream;
  const int d = hd->shape.H * hd->shape.D;
  cudaError_t e = timed(hd, SCAL3R_KERNEL_OTHER, 2.0 * T * d * d, 0, st,
                        [&] { return gcm_out(o, wo, x, alpha, T, d, out, y, hd->d_status, st); });
  return e == cudaSuccess ? SCAL3R_OK : SCAL3R_ERR_CUDA;
}

int scal3r_gcm_out_backward(scal3r_ttt_handle* hd, const void* d_out, const void* o, const void* wo, const void* y,
                            const float* alpha, int64_t T, void* d_o, float* dwo, float* dalpha, void* workspace,
                            size_t workspace_bytes, void* stream) {
  if (!hd || T < 0 || !dwo || !dalpha) return SCAL3R_ERR_INVALID_ARG;
  int rc = gcm_check(hd);
  if (rc != SCAL3R_OK) return rc;
  if (T > 0 && (!d_out || !o || !wo || !y || !alpha || !d_o)) return SCAL3R_ERR_INVALID_ARG;
  if (!all_aligned({d_out, o, wo, y, d_o, dwo, dalpha})) return SCAL3R_ERR_MISALIGNED;
  const int H = hd->shape.H, D = hd->shape.D, d = H * D;
  if (!workspace || workspace_bytes < gcm_workspace_bytes(T, H, D) || !aligned16(workspace))
    return SCAL3R_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = timed(hd, SCAL3R_KERNEL_OTHER, 4.0 * T * d * (double)d, 0, st, [&] {
    return gcm_out_backward(d_out, o, wo, y, alpha, T, d, d_o, dwo, dalpha, workspace, hd->d_status, hd->num_sms, st);
  });
  return e == cudaSuccess ? SCAL3R_OK : SCAL3R_ERR_CUDA;
}

int scal3r_gcm_qkv_backward(scal3r_ttt_handle* hd, const void* dq, const void* dk, const void* dv, const float* dlr,
                            const void* q, const void* k, const float* qn, const float* kn, const float* sig,
                            float base_lr, const void* x, const void* wqkv, const float* w_eta, const void* d_out,
                            int64_t T, float* dx, float* dwqkv, float* dbqkv, float* dw_eta, float* db_eta,
                            void* workspace, size_t workspace_bytes, void* stream) {
  if (!hd || T < 0 || !(base_lr > 0.f) || !dwqkv || !dbqkv || !dw_eta || !db_eta) return SCAL3R_ERR_INVALID_ARG;
  int rc = gcm_check(hd);
  if (rc != SCAL3R_OK) return rc;
  if (T > 0 && (!dq || !dk || !dv || !dlr || !q || !k || !qn || !kn || !sig || !x || !wqkv || !w_eta || !d_out || !dx))
    return SCAL3R_ERR_INVALID_ARG;
  if (!all_aligned({dq, dk, dv, q, k, x, wqkv, w_eta, d_out, dx, dwqkv, dw_eta})) return SCAL3R_ERR_MISALIGNED;
  const int H = hd->shape.H, D = hd->shape.D;
  if (!workspace || workspace_bytes < gcm_workspace_bytes(T, H, D) || !aligned16(workspace))
    return SCAL3R_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const double d = (double)H * D;
  cudaError_t e = timed(hd, SCAL3R_KERNEL_OTHER, 2.0 * T * d * (6.0 * d + 128.0), 0, st, [&] {
    return gcm_qkv_backward(dq, dk, dv, dlr, q, k, qn, kn, sig, base_lr, x, wqkv, w_eta, d_out, T, H, D, dx, dwqkv,
                            dbqkv, dw_eta, db_eta, workspace, hd->d_status, hd->num_sms, st);
  });
  return e == cudaSuccess ? SCAL3R_OK : SCAL3R_ERR_CUDA;
}

int scal3r_ttt_get_status(scal3r_ttt_handle* hd, void* stream) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SCAL3R_ERR_CUDA;
  int s = 0;
  if (cudaMemcpy(&s, hd->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SCAL3R_ERR_CUDA;
  if (s != 0 && cudaMemset(hd->d_status, 0, sizeof(int)) != cudaSuccess) return SCAL3R_ERR_CUDA;
  return s;
}

}  // extern "C"
