// scal3r_ttt_forward_noalloc: the forward pass without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another thread
// holds a stream in global-mode graph capture (cudaMalloc is refused then),
// plugins inside a host framework that owns all device memory through its
// own allocator, and latency-critical paths that must not enter the driver's
// allocator (cudaMalloc may synchronise the device).  For them this entry
// point needs no handle and no workspace: its scratch (schedule tables,
// master weights, row-norm targets, partial sums, status word) lives in one
// fixed file-scope device array, kNoallocBytes large, that every GPU which
// loads the library holds until the process exits.
//
// Rules of use:
//  - The first call in a CUDA context looks up the array's device address
//    (cudaGetSymbolAddress, which may load the module) and sets the kernels'
//    shared-memory attributes; make that first call before any stream
//    capture.  The address is cached per context, so a call after a device
//    reset looks it up again.
//  - The schedule tables go to the array through the parameters of small
//    copy kernels (launched on the caller's stream), not through memory
//    copies: the call reads no host memory after it returns and issues no
//    pageable copy.
//  - Every call on a device shares the one array and leaves its contents
//    behind; calls whose GPU work overlaps (different streams, or threads
//    without ordering) race on it.  Order them on one stream.
//  - A problem whose scratch does not fit returns SCAL3R_ERR_WORKSPACE
//    before any work is enqueued.
//  - scal3r_ttt_noalloc_status reads and clears the status word that the
//    kernels' bounded waits set on a timeout.
#include <algorithm>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "ttt_internal.h"

namespace scal3r {
bool fp32_shape_supported(int D, int F);
bool bf16_shape_supported(int D, int F);
}  // namespace scal3r

using namespace scal3r;

namespace {

constexpr size_t kNoallocBytes = 32ull << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_mu;
struct Cached {
  CUcontext ctx;
  void* addr;
};
Cached g_addr[kMaxDevices] = {};

// The current context (the runtime's primary context of the device once the
// runtime has set it up).
CUcontext current_context() {
  using Fn = CUresult (*)(CUcontext*);
  static Fn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<Fn>(f);
  }
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of the array in the current context (looked up once per
// context: a device reset makes a new context and a new lookup).
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return SCAL3R_ERR_NO_DEVICE;
  const CUcontext ctx = current_context();
  if (!ctx) return SCAL3R_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev].addr || g_addr[dev].ctx != ctx) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SCAL3R_ERR_CUDA;
    if (prepare_kernels() != cudaSuccess) return SCAL3R_ERR_CUDA;   // kernel attributes, once per context
    g_addr[dev] = Cached{ctx, p};
  }
  *out = g_addr[dev].addr;
  return SCAL3R_OK;
}

// A block of bytes for the array, carried in the kernel's parameters (the
// launch copies them when it is enqueued).
constexpr int kUploadBytes = 24 * 1024;
struct UploadBlock {
  unsigned long long* dst;   // 8-byte aligned
  int* status;               // zeroed when not null
  int words;                 // 8-byte words to copy
  unsigned long long data[kUploadBytes / 8];
};

__global__ void noalloc_upload_kernel(const __grid_constant__ UploadBlock b) {
  for (int i = threadIdx.x; i < b.words; i += blockDim.x) b.dst[i] = b.data[i];
  if (b.status && threadIdx.x == 0) *b.status = 0;
}

// Copies `bytes` (a multiple of 8) from host memory to dst, in blocks of
// kUploadBytes, on stream st.
int upload(void* dst, const void* src, size_t bytes, int* status, cudaStream_t st) {
  const unsigned char* s = static_cast<const unsigned char*>(src);
  unsigned char* d = static_cast<unsigned char*>(dst);
  static thread_local UploadBlock blk;
  size_t off = 0;
  do {
    const size_t n = std::min<size_t>(kUploadBytes, bytes - off);
    blk.dst = reinterpret_cast<unsigned long long*>(d + off);
    blk.status = off == 0 ? status : nullptr;
    blk.words = (int)(n / 8);
    if (n) std::memcpy(blk.data, s + off, n);
    noalloc_upload_kernel<<<1, 256, 0, st>>>(blk);
    if (cudaGetLastError() != cudaSuccess) return SCAL3R_ERR_CUDA;
    off += n;
  } while (off < bytes);
  return SCAL3R_OK;
}

__global__ void noalloc_clear_kernel(int* status) { *status = 0; }

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int scal3r_ttt_forward_noalloc(const scal3r_ttt_config* cfg, const void* q, const void* k,
                                          const void* v, const float* lr, const float* w0,
                                          int64_t w0_seq_stride, const int64_t* chunk_offsets, int32_t num_chunks,
                                          const int32_t* seq_chunk_ptr, int32_t num_seqs, void* o, float* w_ckpt,
                                          float* wnorm, float* w_final, void* stream) {
  // configuration (the same checks as scal3r_ttt_init)
  if (!cfg) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->num_heads < 1 || cfg->head_dim < 1 || cfg->hidden_dim < 1 || cfg->ckpt_every > 1 || cfg->ckpt_every < 0 ||
      cfg->lr_per_matrix < 0 || cfg->lr_per_matrix > 1)
    return SCAL3R_ERR_INVALID_ARG;
  if (cfg->model != SCAL3R_MODEL_SWIGLU && cfg->model != SCAL3R_MODEL_LINEAR) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->deterministic < 0 || cfg->deterministic > 1) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->model == SCAL3R_MODEL_LINEAR) return SCAL3R_ERR_UNSUPPORTED;   // the handle's forward runs it
  if (cfg->dtype != SCAL3R_FP32 && cfg->dtype != SCAL3R_BF16) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->loss != SCAL3R_LOSS_DOT && cfg->loss != SCAL3R_LOSS_MSE) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->weight_norm < 0 || cfg->weight_norm > 2) return SCAL3R_ERR_INVALID_ARG;
  if (cfg->dtype == SCAL3R_FP32 && !fp32_shape_supported(cfg->head_dim, cfg->hidden_dim))
    return SCAL3R_ERR_UNSUPPORTED;
  if (cfg->dtype == SCAL3R_BF16 &&
      (!bf16_shape_supported(cfg->head_dim, cfg->hidden_dim) || cfg->loss != SCAL3R_LOSS_DOT))
    return SCAL3R_ERR_UNSUPPORTED;
  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SCAL3R_ERR_NO_DEVICE;
  if (major != 10 || minor != 3) return SCAL3R_ERR_NO_DEVICE;

  // schedule (host memory only)
  const Shape sh{cfg->num_heads, cfg->head_dim, cfg->hidden_dim};
  Plan pl;
  Schedule sch{};
  if (cfg->dtype == SCAL3R_FP32) {   // as the handle's plan: 16-token pieces on the float32 path
    sch.align = 16;
    sch.min_tokens = 16;
  }
  int rc = build_plan(pl, sh, sch, sms, chunk_offsets, num_chunks, seq_chunk_ptr, num_seqs);
  if (rc != SCAL3R_OK) return rc;
  if (pl.T > 0 && (!q || !k || !v || !lr || !o)) return SCAL3R_ERR_INVALID_ARG;
  if (!w0 || w0_seq_stride < 0) return SCAL3R_ERR_INVALID_ARG;
  if (w0_seq_stride != 0 && w0_seq_stride < (int64_t)sh.H * sh.P()) return SCAL3R_ERR_INVALID_ARG;
  for (const void* p : {q, k, v, (const void*)o, (const void*)lr, (const void*)w0, (const void*)w_ckpt,
                        (const void*)w_final})
    if (((uintptr_t)p & 15u) != 0) return SCAL3R_ERR_MISALIGNED;
  if ((w0_seq_stride & 3) != 0) return SCAL3R_ERR_MISALIGNED;

  // layout of the static array: status | items | updates | wm | rho | partials
  const size_t chains = (size_t)pl.S * sh.H;
  const size_t b_status = 256;
  const size_t b_items = al256(std::max<size_t>(pl.items.size(), 1) * sizeof(WorkItem));
  const size_t b_upd = al256(std::max<size_t>(pl.updates.size(), 1) * sizeof(UpdateItem));
  const size_t b_wm = al256(2 * chains * sh.P() * sizeof(float));
  const size_t b_rho = al256(chains * sh.R() * sizeof(float));
  const size_t b_part = al256((size_t)std::max(pl.max_slots, 1) * sh.P() * sizeof(float));
  if (b_status + b_items + b_upd + b_wm + b_rho + b_part > kNoallocBytes) return SCAL3R_ERR_WORKSPACE;

  void* base = nullptr;
  rc = scratch_address(dev, &base);
  if (rc != SCAL3R_OK) return rc;
  char* c = static_cast<char*>(base);
  int* status = reinterpret_cast<int*>(c);
  WorkItem* d_items = reinterpret_cast<WorkItem*>(c + b_status);
  UpdateItem* d_upd = reinterpret_cast<UpdateItem*>(c + b_status + b_items);
  char* regions = c + b_status + b_items + b_upd;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the schedule tables, and the status word set to zero with the first
  // block; every other region is written before it is read
  static_assert(sizeof(WorkItem) % 8 == 0 && sizeof(UpdateItem) % 8 == 0, "8-byte words");
  rc = upload(d_items, pl.items.data(), pl.items.size() * sizeof(WorkItem), status, st);
  if (rc == SCAL3R_OK) rc = upload(d_upd, pl.updates.data(), pl.updates.size() * sizeof(UpdateItem), nullptr, st);
  if (rc != SCAL3R_OK) return rc;

  Params prm{};
  prm.H = sh.H;
  prm.D = sh.D;
  prm.F = sh.F;
  prm.S = pl.S;
  prm.T = pl.T;
  prm.loss = cfg->loss;
  prm.lr_mat = cfg->lr_per_matrix;
  prm.norm = cfg->weight_norm;
  prm.eps = cfg->norm_eps > 0.f ? cfg->norm_eps : 1e-6f;
  prm.status = status;
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
  prm.wm = reinterpret_cast<float*>(regions);
  prm.rho = reinterpret_cast<float*>(regions + b_wm);
  prm.part = reinterpret_cast<float*>(regions + b_wm + b_rho);

  if (launch_prep(prm, (int)chains, st) != cudaSuccess) return SCAL3R_ERR_CUDA;
  for (size_t j = 0; j < pl.steps.size(); ++j) {
    const Step& s = pl.steps[j];
    cudaError_t e = cudaSuccess;
    if (s.nitems > 0)
      e = cfg->dtype == SCAL3R_BF16 ? launch_bf16_sweep(prm, d_items + s.item0, s.nitems, (int)j, nullptr, st)
                                    : launch_fp32_sweep(prm, d_items + s.item0, s.nitems, (int)j, st);
    if (e != cudaSuccess) return SCAL3R_ERR_CUDA;
    if (s.nupd > 0 && launch_update(prm, d_upd + s.upd0, s.nupd, (int)j, st) != cudaSuccess) return SCAL3R_ERR_CUDA;
  }
  return SCAL3R_OK;
}

extern "C" int scal3r_ttt_noalloc_status(void* stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SCAL3R_ERR_NO_DEVICE;
  void* base = nullptr;
  const int rc = scratch_address(dev, &base);
  if (rc != SCAL3R_OK) return rc;
  int* status = static_cast<int*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h = 0;
  if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SCAL3R_ERR_CUDA;
  noalloc_clear_kernel<<<1, 1, 0, st>>>(status);
  if (cudaGetLastError() != cudaSuccess) return SCAL3R_ERR_CUDA;
  return h;
}
