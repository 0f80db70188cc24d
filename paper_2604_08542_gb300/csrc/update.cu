// Per-chain kernels that close a chunk step: the weight update of Eq. 8 with
// the row normalisation, and, in the backward, the adjoint of both.
//
// Weights, the adjoint R and every partial-sum slot share one packed layout:
// W1 [F][D], W3 [F][D], W2 [D][F], row-major float32.
//   forward slot  = the chunk's weight increment sum of one piece (W += sum)
//   backward slot = one piece's contribution to dL/dW
// Row r of the packed weights: r < F is W1 row r, r < 2F is W3 row r-F,
// otherwise W2 row r-2F.  Each thread owns four consecutive elements of one
// row (a float4); a row's L2 norm is reduced over the D/4 (or F/4) lanes that
// hold it with shuffles, in a fixed order.  Blocks along y cover the rows:
// first the W1/W3 rows (1024/D per block), then the W2 rows (1024/F per block).
#include <cuda_bf16.h>

#include "bounds.cuh"
#include "ttt_internal.h"

namespace scal3r {
namespace {

constexpr int kThreads = 256;

struct RowSlice {
  bool valid;
  int r;        // packed row index
  size_t off;   // offset of this thread's float4 in the packed layout
  int group;    // lanes per row
  int c4;       // float4 index inside the row
};

__device__ __forceinline__ int blocks13(int D, int F) { return (2 * F * D + 1023) / 1024; }

__device__ __forceinline__ RowSlice row_slice(int by, int D, int F) {
  RowSlice s;
  const int t = threadIdx.x;
  const int nb13 = blocks13(D, F);
  if (by < nb13) {
    s.group = D / 4;
    const int row = by * (1024 / D) + t / s.group;
    s.c4 = t % s.group;
    s.valid = row < 2 * F;
    s.r = row;
    s.off = (size_t)row * D + 4 * s.c4;
  } else {
    s.group = F / 4;
    const int d = (by - nb13) * (1024 / F) + t / s.group;
    s.c4 = t % s.group;
    s.valid = d < D;
    s.r = 2 * F + d;
    s.off = 2 * (size_t)F * D + (size_t)d * F + 4 * s.c4;
  }
  return s;
}

// Sum over the `group` lanes holding one row (group divides 32).
__device__ __forceinline__ float group_sum(float x, int group) {
  for (int o = group >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Every plain global access of these kernels is checked in the bounds-checking
// build (ld4 / st4 and the scalar accesses below); plain otherwise.
__device__ __forceinline__ float4 ld4(const float* p) { return ld_chk(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { st_chk(reinterpret_cast<float4*>(p), v); }
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 scale4(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }
__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

// x + the slots slot0 .. slot0 + n - 1 at element offset `off`, added one by
// one in slot order (fixed-order reduction); the loads of a batch of eight
// slots are issued before any of them is added, so the sum costs one memory
// round trip per eight slots rather than one per slot.
__device__ __forceinline__ float4 add_slots(float4 x, const float* part, int slot0, int n, size_t P, size_t off) {
  constexpr int kBatch = 8;
  for (int b = 0; b < n; b += kBatch) {
    float4 v[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j)
      if (b + j < n) v[j] = ld4(part + (size_t)(slot0 + b + j) * P + off);
#pragma unroll
    for (int j = 0; j < kBatch; ++j)
      if (b + j < n) x = add4(x, v[j]);
  }
  return x;
}

__device__ __forceinline__ const float* chain_w0(const Params& p, int chain) {
  const int s = chain / p.H, h = chain % p.H;
  return p.w0 + (size_t)s * p.w0_seq_stride + (size_t)h * 3 * p.F * p.D;
}

__device__ __forceinline__ float row_target(const Params& p, float ss) {
  return (p.norm == SCAL3R_NORM_UNIT) ? 1.f : sqrtf(ss);
}

// Copy the starting weights of every chain into master buffer 0 and compute
// the row-norm targets.
__global__ void prep_kernel(Params p) {
  pdl_wait();
  const int chain = blockIdx.x;
  const RowSlice s = row_slice(blockIdx.y, p.D, p.F);
  const int P = 3 * p.F * p.D, R = 2 * p.F + p.D;
  const float* w0 = chain_w0(p, chain);
  float4 w = s.valid ? ld4(w0 + s.off) : make_float4(0.f, 0.f, 0.f, 0.f);
  if (s.valid) st4(p.wm + (size_t)chain * P + s.off, w);
  const float ss = group_sum(dot4(w, w), s.group);
  if (s.valid && s.c4 == 0) st_chk(p.rho + (size_t)chain * R + s.r, row_target(p, ss));
}

// Forward update of one chain at step `step`:
//   W~ = W_step + sum_slots partial (fixed slot order),
//   W_{step+1} row = W~ row * rho / max(||W~ row||, eps).
__global__ void update_kernel(Params p, const UpdateItem* __restrict__ upd, int step) {
  pdl_wait();
  const UpdateItem u = upd[blockIdx.x];
  const RowSlice s = row_slice(blockIdx.y, p.D, p.F);
  const int P = 3 * p.F * p.D, R = 2 * p.F + p.D;
  const int chains = p.S * p.H;
  const int h = u.chain % p.H;
  const float* wcur = p.wm + ((size_t)(step & 1) * chains + u.chain) * P;
  float* wnext = p.wm + ((size_t)((step + 1) & 1) * chains + u.chain) * P;
  if (u.chunk < 0) {   // sequence without chunks: w_final = w0
    if (p.w_final && s.valid) st4(p.w_final + ((size_t)u.seq * p.H + h) * P + s.off, ld4(wcur + s.off));
    return;
  }
  float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
  float rho = 1.f;
  if (s.valid) {
    // the row target is loaded before the slot sum so that its round trip
    // overlaps the sum's
    if (p.norm != SCAL3R_NORM_NONE) rho = ld_chk(p.rho + (size_t)u.chain * R + s.r);
    x = add_slots(ld4(wcur + s.off), p.part, u.slot0, u.nslots, P, s.off);
  }
  const float n = sqrtf(group_sum(dot4(x, x), s.group));
  if (!s.valid) return;
  float scale = 1.f;
  if (p.norm != SCAL3R_NORM_NONE) scale = rho / fmaxf(n, p.eps);
  const float4 w = scale4(x, scale);
  st4(wnext + s.off, w);
  if (p.w_ckpt && u.wslot >= 0) st4(p.w_ckpt + ((size_t)u.wslot * p.H + h) * P + s.off, w);
  if (p.w_final && u.last) st4(p.w_final + ((size_t)u.seq * p.H + h) * P + s.off, w);
  if (p.wnorm && s.c4 == 0) st_chk(p.wnorm + ((size_t)u.chunk * p.H + h) * R + s.r, n);
}

// Backward: zero the carried row-norm adjoints and per-chain dW0, compute
// the row-norm targets from w0.
__global__ void bprep_kernel(Params p) {
  pdl_wait();
  const int chain = blockIdx.x;
  const RowSlice s = row_slice(blockIdx.y, p.D, p.F);
  const int P = 3 * p.F * p.D, R = 2 * p.F + p.D;
  const float* w0 = chain_w0(p, chain);
  const float4 w = s.valid ? ld4(w0 + s.off) : make_float4(0.f, 0.f, 0.f, 0.f);
  if (s.valid) st4(p.dw0_chain + (size_t)chain * P + s.off, make_float4(0.f, 0.f, 0.f, 0.f));
  const float ss = group_sum(dot4(w, w), s.group);
  if (s.valid && s.c4 == 0) {
    st_chk(p.rho + (size_t)chain * R + s.r, row_target(p, ss));
    st_chk(p.drho + (size_t)chain * R + s.r, 0.f);
  }
}

// Backward step closing: Lambda = R_next (unless this is the chain's last
// chunk) + sum_slots partial.  Then either the VJP of the row normalisation
// of update `chunk` (R = dL/dW~ into rbuf; the row-norm target's adjoint
// accumulated in drho) or, for the first chunk, dW0 = Lambda + drho * W0 / rho.
//   W_row = rho w~ / max(||w~||, eps), w_hat = W_row / rho:
//   unclamped  R = (rho / ||w~||) (lambda - w_hat (w_hat . lambda))
//   clamped    R = (rho / eps) lambda;      drho += w_hat . lambda in both
__global__ void bupdate_kernel(Params p, const UpdateItem* __restrict__ upd, int step) {
  pdl_wait();
  (void)step;
  const UpdateItem u = upd[blockIdx.x];
  const RowSlice s = row_slice(blockIdx.y, p.D, p.F);
  const int P = 3 * p.F * p.D, R = 2 * p.F + p.D;
  const int h = u.chain % p.H;
  float* rb = p.rbuf + (size_t)u.chain * P;
  // every load that does not depend on the slot sum is issued before it, so
  // that their round trips overlap the sum's
  const bool norm_vjp = !u.first && p.norm != SCAL3R_NORM_NONE;
  float rho = 0.f, drho = 0.f, n = 0.f;
  float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), wck = w0;
  float4 lam = make_float4(0.f, 0.f, 0.f, 0.f);
  if (s.valid) {
    rho = ld_chk(p.rho + (size_t)u.chain * R + s.r);
    if (u.first) {
      if (p.norm == SCAL3R_NORM_ROW_W0) drho = ld_chk(p.drho + (size_t)u.chain * R + s.r);
      w0 = ld4(chain_w0(p, u.chain) + s.off);
    } else if (norm_vjp) {
      wck = ld4(p.w_ckpt_in + ((size_t)u.wslot * p.H + h) * P + s.off);
      n = ld_chk(p.wnorm_in + ((size_t)u.chunk * p.H + h) * R + s.r);
    }
    if (!u.last) lam = ld4(rb + s.off);
    lam = add_slots(lam, p.part, u.slot0, u.nslots, P, s.off);
  }
  if (u.first) {
    if (!s.valid) return;
    float coef = 0.f;
    if (p.norm == SCAL3R_NORM_ROW_W0 && rho > 0.f) coef = drho / rho;
    st4(p.dw0_chain + (size_t)u.chain * P + s.off,
        make_float4(lam.x + coef * w0.x, lam.y + coef * w0.y, lam.z + coef * w0.z, lam.w + coef * w0.w));
    return;
  }
  if (p.norm == SCAL3R_NORM_NONE) {
    if (s.valid) st4(rb + s.off, lam);
    return;
  }
  const float inv_rho = rho > 0.f ? 1.f / rho : 0.f;
  const float4 what = scale4(wck, inv_rho);
  const float proj = group_sum(dot4(what, lam), s.group);
  if (!s.valid) return;
  float4 out;
  if (!(n >= p.eps)) {
    out = scale4(lam, rho / p.eps);
  } else {
    const float c = rho / n;
    out = make_float4(c * (lam.x - what.x * proj), c * (lam.y - what.y * proj), c * (lam.z - what.z * proj),
                      c * (lam.w - what.w * proj));
  }
  st4(rb + s.off, out);
  if (s.c4 == 0 && p.norm == SCAL3R_NORM_ROW_W0) {
    float* dr = p.drho + (size_t)u.chain * R + s.r;
    st_chk(dr, ld_chk(dr) + proj);
  }
}

// dw0 from the per-chain results: summed over sequences in order when w0 is
// shared, copied per sequence otherwise.
__global__ void bfinal_kernel(Params p) {
  pdl_wait();
  const int P = 3 * p.F * p.D;
  const int h = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    if (p.w0_seq_stride == 0) {
      float a = 0.f;
      for (int s = 0; s < p.S; ++s) a += ld_chk(p.dw0_chain + ((size_t)s * p.H + h) * P + i);
      st_chk(p.dw0 + (size_t)h * P + i, a);
    } else {
      for (int s = 0; s < p.S; ++s)
        st_chk(p.dw0 + (size_t)s * p.w0_seq_stride + (size_t)h * P + i,
               ld_chk(p.dw0_chain + ((size_t)s * p.H + h) * P + i));
    }
  }
}

// ---- Global Context Synchronisation (Eq. 10): a chunk's gradient summed over
// token shards held by several callers, then one update applied by each.

// The chunk gradient of every chain over this call's tokens: G = -(sum of the
// step's forward slots, which hold the increments), in the packed layout.
// Chains without a chunk get G = 0.
__global__ void gsum_kernel(Params p, const UpdateItem* __restrict__ upd, float* grad) {
  const UpdateItem u = upd[blockIdx.x];
  const RowSlice s = row_slice(blockIdx.y, p.D, p.F);
  if (!s.valid) return;
  const int P = 3 * p.F * p.D;
  const int h = u.chain % p.H;
  float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
  if (u.chunk >= 0) x = add_slots(x, p.part, u.slot0, u.nslots, P, s.off);
  st4(grad + ((size_t)u.seq * p.H + h) * P + s.off, scale4(x, -1.f));
}

// The weights given in (w0, w0_seq_stride) into master buffer `buf`.
__global__ void loadw_kernel(Params p, int buf) {
  const int chain = blockIdx.x;
  const RowSlice s = row_slice(blockIdx.y, p.D, p.F);
  if (!s.valid) return;
  const int P = 3 * p.F * p.D;
  st4(p.wm + ((size_t)buf * p.S * p.H + chain) * P + s.off, ld4(chain_w0(p, chain) + s.off));
}

// Token rows of the pieces' ranges (head of the piece's chain) of a bf16
// [T][H][D] tensor, 16 bytes per thread step: dst = -src (sign flips, exact).
__global__ void tok_negate_kernel(Params p, const WorkItem* __restrict__ items, const uint4* __restrict__ src,
                                  uint4* __restrict__ dst) {
  const WorkItem it = items[blockIdx.x];
  const int h = it.chain % p.H, nc = p.D / 8;
  const int64_t n = (it.t1 - it.t0) * nc;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const size_t o = (((size_t)(it.t0 + i / nc) * p.H + h) * p.D) / 8 + i % nc;
    uint4 x = ld_chk(src + o);
    x.x ^= 0x80008000u;
    x.y ^= 0x80008000u;
    x.z ^= 0x80008000u;
    x.w ^= 0x80008000u;
    st_chk(dst + o, x);
  }
}

__device__ __forceinline__ uint32_t add_bf16x2(uint32_t a, uint32_t b) {
  const float lo = __uint_as_float(a << 16) + __uint_as_float(b << 16);
  const float hi = __uint_as_float(a & 0xFFFF0000u) + __uint_as_float(b & 0xFFFF0000u);
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// acc += add over the same rows (float32 sum, one rounding to bf16).
__global__ void tok_add_kernel(Params p, const WorkItem* __restrict__ items, uint4* __restrict__ acc,
                               const uint4* __restrict__ add) {
  const WorkItem it = items[blockIdx.x];
  const int h = it.chain % p.H, nc = p.D / 8;
  const int64_t n = (it.t1 - it.t0) * nc;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const size_t o = (((size_t)(it.t0 + i / nc) * p.H + h) * p.D) / 8 + i % nc;
    const uint4 a = ld_chk(acc + o), b = ld_chk(add + o);
    st_chk(acc + o, make_uint4(add_bf16x2(a.x, b.x), add_bf16x2(a.y, b.y), add_bf16x2(a.z, b.z), add_bf16x2(a.w, b.w)));
  }
}

// Sparse checkpoints: the first weights of a backward segment into master
// buffer `buf`, per chain from its sequence's checkpoint slot src[s] (-1: w0,
// -2: the sequence has no step in the segment).
__global__ void loadw_seg_kernel(Params p, int buf, const int32_t* __restrict__ src) {
  const int chain = blockIdx.x;
  const RowSlice s = row_slice(blockIdx.y, p.D, p.F);
  const int idx = src[chain / p.H];
  if (!s.valid || idx == -2) return;
  const int P = 3 * p.F * p.D;
  const float* from = idx < 0 ? chain_w0(p, chain) : p.w_ckpt_in + ((size_t)idx * p.H + chain % p.H) * P;
  st4(p.wm + ((size_t)buf * p.S * p.H + chain) * P + s.off, ld4(from + s.off));
}

// W_next = W - G with every row rescaled to its target (taken from w0, as in
// the forward), per chain; the pre-rescale row norms optionally.
__global__ void gcs_update_kernel(Params p, const float* w, int64_t w_stride, const float* g, float* w_out,
                                  float* wnorm) {
  const int chain = blockIdx.x;
  const int seq = chain / p.H, h = chain % p.H;
  const RowSlice s = row_slice(blockIdx.y, p.D, p.F);
  const int P = 3 * p.F * p.D, R = 2 * p.F + p.D;
  float4 x = make_float4(0.f, 0.f, 0.f, 0.f), t = x;
  if (s.valid) {
    const float4 a = ld4(w + (size_t)seq * w_stride + (size_t)h * P + s.off);
    const float4 b = ld4(g + (size_t)chain * P + s.off);
    x = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    t = ld4(chain_w0(p, chain) + s.off);
  }
  const float n = sqrtf(group_sum(dot4(x, x), s.group));
  const float ss = group_sum(dot4(t, t), s.group);
  if (!s.valid) return;
  float scale = 1.f;
  if (p.norm != SCAL3R_NORM_NONE) scale = row_target(p, ss) / fmaxf(n, p.eps);
  st4(w_out + (size_t)chain * P + s.off, scale4(x, scale));
  if (wnorm && s.c4 == 0) st_chk(wnorm + (size_t)chain * R + s.r, n);
}

int row_blocks(const Params& p) { return (2 * p.F * p.D + 1023) / 1024 + (p.F * p.D + 1023) / 1024; }

}  // namespace

// Shapes the row kernels handle: D/4 and F/4 powers of two dividing 32.
bool update_shape_supported(int D, int F) {
  auto ok = [](int x) { return x % 4 == 0 && x / 4 <= 32 && ((x / 4) & (x / 4 - 1)) == 0; };
  return ok(D) && ok(F);
}

cudaError_t launch_prep(const Params& prm, int chains, cudaStream_t st) {
  if (chains == 0) return cudaSuccess;
  return launch_pdl(prep_kernel, dim3(chains, row_blocks(prm)), dim3(kThreads), 0, st, prm);
}

cudaError_t launch_update(const Params& prm, const UpdateItem* upd, int nupd, int step, cudaStream_t st) {
  if (nupd == 0) return cudaSuccess;
  return launch_pdl(update_kernel, dim3(nupd, row_blocks(prm)), dim3(kThreads), 0, st, prm, upd, step);
}

cudaError_t launch_bupdate(const Params& prm, const UpdateItem* upd, int nupd, int step, cudaStream_t st) {
  if (nupd == 0) return cudaSuccess;
  return launch_pdl(bupdate_kernel, dim3(nupd, row_blocks(prm)), dim3(kThreads), 0, st, prm, upd, step);
}

cudaError_t launch_bprep(const Params& prm, int chains, cudaStream_t st);
cudaError_t launch_bprep(const Params& prm, int chains, cudaStream_t st) {
  if (chains == 0) return cudaSuccess;
  return launch_pdl(bprep_kernel, dim3(chains, row_blocks(prm)), dim3(kThreads), 0, st, prm);
}

cudaError_t launch_gsum(const Params& prm, const UpdateItem* upd, int nupd, float* grad, cudaStream_t st) {
  if (nupd == 0) return cudaSuccess;
  gsum_kernel<<<dim3(nupd, row_blocks(prm)), kThreads, 0, st>>>(prm, upd, grad);
  return cudaGetLastError();
}

cudaError_t launch_loadw(const Params& prm, int chains, int buf, cudaStream_t st) {
  if (chains == 0) return cudaSuccess;
  loadw_kernel<<<dim3(chains, row_blocks(prm)), kThreads, 0, st>>>(prm, buf);
  return cudaGetLastError();
}

cudaError_t launch_tok_negate(const Params& prm, const WorkItem* items, int nitems, const void* src, void* dst,
                              cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  tok_negate_kernel<<<nitems, kThreads, 0, st>>>(prm, items, static_cast<const uint4*>(src), static_cast<uint4*>(dst));
  return cudaGetLastError();
}

cudaError_t launch_tok_add(const Params& prm, const WorkItem* items, int nitems, void* acc, const void* add,
                           cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  tok_add_kernel<<<nitems, kThreads, 0, st>>>(prm, items, static_cast<uint4*>(acc), static_cast<const uint4*>(add));
  return cudaGetLastError();
}

cudaError_t launch_loadw_seg(const Params& prm, int chains, int buf, const int32_t* src, cudaStream_t st) {
  if (chains == 0) return cudaSuccess;
  loadw_seg_kernel<<<dim3(chains, row_blocks(prm)), kThreads, 0, st>>>(prm, buf, src);
  return cudaGetLastError();
}

cudaError_t launch_gcs_update(const Params& prm, int chains, const float* w, int64_t w_stride, const float* g,
                              float* w_out, float* wnorm, cudaStream_t st) {
  if (chains == 0) return cudaSuccess;
  gcs_update_kernel<<<dim3(chains, row_blocks(prm)), kThreads, 0, st>>>(prm, w, w_stride, g, w_out, wnorm);
  return cudaGetLastError();
}

cudaError_t launch_bfinal(const Params& prm, cudaStream_t st) {
  const int P = 3 * prm.F * prm.D;
  dim3 grid((P + 255) / 256, prm.H);
  return launch_pdl(bfinal_kernel, grid, dim3(256), 0, st, prm);
}

#ifdef SCAL3R_DEBUG_BOUNDS
cudaError_t update_upload_bounds(const BoundsTable& t, cudaStream_t st) { return upload_bounds_table(t, st); }
#endif

}  // namespace scal3r
