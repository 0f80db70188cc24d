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
#include <cstdio>
#include <cstring>
#include <mutex>

#include "ttt_internal.h"

namespace scal3r {
bool fp32_shape_supported(int D, int F);
bool bf16_shape_supported(int D, int F);
bool update_shape_supported(int D, int F);
cudaError_t launch_bprep(const Params& prm, int chains, cudaStream_t st);
}  // namespace scal3r

using namespace scal3r;

struct ProfRecord {
  int kind;
  cudaEvent_t a, b;
  double flops, bytes;
};

struct scal3r_ttt_handle {
  scal3r_ttt_config cfg{};
  Shape shape{};
  Schedule sched{};
  int device = 0;
  int num_sms = 0;
  Plan plan;
  int* d_status = nullptr;
  bool prof_on = false;
  std::vector<ProfRecord> prof;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
};

namespace {

void free_plan(Plan& p) {
  if (p.d_items) cudaFree(p.d_items);
  if (p.d_updates) cudaFree(p.d_updates);
  if (p.d_bitems) cudaFree(p.d_bitems);
  if (p.d_bupdates) cudaFree(p.d_bupdates);
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
  int rc = build_plan(np, hd->shape, hd->sched, hd->num_sms, off, C, ptr, S);
  if (rc != SCAL3R_OK) return rc;
  if (upload(&np.d_items, np.items) != cudaSuccess || upload(&np.d_updates, np.updates) != cudaSuccess ||
      upload(&np.d_bitems, np.bitems) != cudaSuccess || upload(&np.d_bupdates, np.bupdates) != cudaSuccess) {
    free_plan(np);
    return SCAL3R_ERR_CUDA;
  }
  free_plan(hd->plan);
  hd->plan = std::move(np);
  return SCAL3R_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

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
  prm.norm = hd->cfg.weight_norm;
  prm.eps = hd->cfg.norm_eps > 0.f ? hd->cfg.norm_eps : 1e-6f;
  prm.status = hd->d_status;
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
    default: return "unknown status";
  }
}

int scal3r_ttt_init(const scal3r_ttt_config* cfg, scal3r_ttt_handle** out) {
  if (!cfg || !out) return SCAL3R_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->num_heads < 1 || cfg->head_dim < 1 || cfg->hidden_dim < 1 || cfg->reserved != 0)
    return SCAL3R_ERR_INVALID_ARG;
  if (cfg->dtype != SCAL3R_FP32 && cfg->dtype != SCAL3R_BF16) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->loss != SCAL3R_LOSS_DOT && cfg->loss != SCAL3R_LOSS_MSE) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->weight_norm < 0 || cfg->weight_norm > 2) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->dtype == SCAL3R_FP32 && !fp32_shape_supported(cfg->head_dim, cfg->hidden_dim))
    return SCAL3R_ERR_UNSUPPORTED;
  if (cfg->dtype == SCAL3R_BF16 &&
      (!bf16_shape_supported(cfg->head_dim, cfg->hidden_dim) || cfg->loss != SCAL3R_LOSS_DOT))
    return SCAL3R_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SCAL3R_ERR_NO_DEVICE;
  int major = 0, minor = 0, sms = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SCAL3R_ERR_NO_DEVICE;
  if (major != 10 || minor != 3) return SCAL3R_ERR_NO_DEVICE;
  auto* hd = new scal3r_ttt_handle();
  hd->cfg = *cfg;
  hd->shape = Shape{cfg->num_heads, cfg->head_dim, cfg->hidden_dim};
  hd->device = dev;
  hd->num_sms = sms;
  if (cudaMalloc((void**)&hd->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(hd->d_status, 0, sizeof(int)) != cudaSuccess) {
    delete hd;
    return SCAL3R_ERR_CUDA;
  }
  *out = hd;
  return SCAL3R_OK;
}

void scal3r_ttt_destroy(scal3r_ttt_handle* hd) {
  if (!hd) return;
  for (cudaEvent_t e : hd->pool) cudaEventDestroy(e);
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
  *bytes = workspace_bytes(hd->plan, hd->shape, with_backward != 0);
  return SCAL3R_OK;
}

int scal3r_ttt_forward(scal3r_ttt_handle* hd, const void* q, const void* k, const void* v, const float* lr,
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
  const size_t need = workspace_bytes(pl, sh, false);
  if (!workspace || workspace_bytes_ < need || !aligned16(workspace)) return SCAL3R_ERR_WORKSPACE;

  Params prm{};
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
  const int chains = pl.S * sh.H;
  if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st, [&] { return launch_prep(prm, chains, st); }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  for (size_t j = 0; j < pl.steps.size(); ++j) {
    const Step& s = pl.steps[j];
    double fl = 0, by = 0;
    if (hd->prof_on) sweep_work(hd, pl.items.data() + s.item0, s.nitems, fl, by);
    cudaError_t e = cudaSuccess;
    if (s.nitems > 0)
      e = timed(hd, SCAL3R_KERNEL_FWD_SWEEP, fl, by, st, [&] {
        return hd->cfg.dtype == SCAL3R_BF16 ? launch_bf16_sweep(prm, pl.d_items + s.item0, s.nitems, (int)j, nullptr, st)
                                            : launch_fp32_sweep(prm, pl.d_items + s.item0, s.nitems, (int)j, st);
      });
    if (e != cudaSuccess) return SCAL3R_ERR_CUDA;
    if (s.nupd > 0 && timed(hd, SCAL3R_KERNEL_FWD_UPDATE, 0, 0, st, [&] {
          return launch_update(prm, pl.d_updates + s.upd0, s.nupd, (int)j, st);
        }) != cudaSuccess)
      return SCAL3R_ERR_CUDA;
  }
  return SCAL3R_OK;
}

int scal3r_ttt_backward(scal3r_ttt_handle* hd, const void* q, const void* k, const void* v, const float* lr,
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
  if (pl.C > 0 && (!w_ckpt || !wnorm)) return SCAL3R_ERR_INVALID_ARG;
  if (!w0 || !dw0 || w0_seq_stride < 0) return SCAL3R_ERR_INVALID_ARG;
  if (w0_seq_stride != 0 && w0_seq_stride < (int64_t)sh.H * sh.P()) return SCAL3R_ERR_INVALID_ARG;
  for (const void* p : {q, k, v, d_o, (const void*)dq, (const void*)dk, (const void*)dv, (const void*)w_ckpt,
                        (const void*)w0, (const void*)dw0})
    if (!aligned16(p)) return SCAL3R_ERR_MISALIGNED;
  if ((w0_seq_stride & 3) != 0) return SCAL3R_ERR_MISALIGNED;
  const size_t need = workspace_bytes(pl, sh, true);
  if (!workspace || workspace_bytes_ < need || !aligned16(workspace)) return SCAL3R_ERR_WORKSPACE;

  Params prm{};
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
  carve_workspace(pl, sh, true, workspace, prm);
  cudaStream_t st = (cudaStream_t)stream;
  const int chains = pl.S * sh.H;
  if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st, [&] { return launch_bprep(prm, chains, st); }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  for (size_t j = 0; j < pl.bsteps.size(); ++j) {
    const Step& s = pl.bsteps[j];
    double fl = 0, by = 0;
    if (hd->prof_on) sweep_work(hd, pl.bitems.data() + s.item0, s.nitems, fl, by);
    cudaError_t e = cudaSuccess;
    if (s.nitems > 0)
      e = timed(hd, SCAL3R_KERNEL_BWD_SWEEP, fl, by, st, [&] {
        return hd->cfg.dtype == SCAL3R_BF16
                   ? launch_bf16_bsweep(prm, pl.d_bitems + s.item0, s.nitems, (int)j, nullptr, st)
                   : launch_fp32_bsweep(prm, pl.d_bitems + s.item0, s.nitems, (int)j, st);
      });
    if (e != cudaSuccess) return SCAL3R_ERR_CUDA;
    if (s.nupd > 0 && timed(hd, SCAL3R_KERNEL_BWD_UPDATE, 0, 0, st, [&] {
          return launch_bupdate(prm, pl.d_bupdates + s.upd0, s.nupd, (int)j, st);
        }) != cudaSuccess)
      return SCAL3R_ERR_CUDA;
  }
  if (timed(hd, SCAL3R_KERNEL_OTHER, 0, 0, st, [&] { return launch_bfinal(prm, st); }) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
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

int scal3r_ttt_get_status(scal3r_ttt_handle* hd, void* stream) {
  if (!hd) return SCAL3R_ERR_INVALID_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SCAL3R_ERR_CUDA;
  int s = 0;
  if (cudaMemcpy(&s, hd->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SCAL3R_ERR_CUDA;
  if (s != 0 && cudaMemset(hd->d_status, 0, sizeof(int)) != cudaSuccess) return SCAL3R_ERR_CUDA;
  return s;
}

}  // extern "C"
