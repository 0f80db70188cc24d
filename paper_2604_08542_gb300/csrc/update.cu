// Per-chain kernels that close a chunk step: the weight update of Eq. 8 with
// the row normalisation, and, in the backward, the adjoint of both.
//
// Partial sums written by the sweep kernels use one layout for all three
// matrices, [F][D] float32 each (rows = hidden unit):
//   forward  slot = [ A1 | A3 | A2t ] with W1 += A1, W3 += A3, W2 += A2t^T
//   backward slot = [ L1 | L3 | L2t ] with dL/dW1 += L1, dL/dW3 += L3,
//                                         dL/dW2 += L2t^T
// Weights (and the adjoint R) are packed W1 [F][D], W3 [F][D], W2 [D][F].
// Row r of the packed weights: r < F is W1 row r, r < 2F is W3 row r-F,
// otherwise W2 row r-2F (length F).  Row norms are reduced with warp
// shuffles, one warp per row, in a fixed order.
#include "ttt_internal.h"

namespace scal3r {
namespace {

constexpr int kWarps = 8;

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ const float* chain_w0(const Params& p, int chain) {
  const int s = chain / p.H, h = chain % p.H;
  return p.w0 + (size_t)s * p.w0_seq_stride + (size_t)h * 3 * p.F * p.D;
}

// Element j (0 <= j < len) of row r of the packed weights; also the offset of
// the same element in the [F][D] partial-sum layout.
__device__ __forceinline__ void row_geom(int r, int F, int D, int& len, size_t& wbase,
                                         size_t& pbase, int& pstride) {
  if (r < 2 * F) {          // W1 / W3 row: contiguous in both layouts
    len = D;
    wbase = (size_t)r * D;
    pbase = (size_t)r * D;
    pstride = 1;
  } else {                  // W2 row d: column d of the transposed partial
    const int d = r - 2 * F;
    len = F;
    wbase = (size_t)2 * F * D + (size_t)d * F;
    pbase = (size_t)2 * F * D + d;
    pstride = D;
  }
}

// Copy the starting weights of every chain into master buffer 0 and compute
// the row-norm targets.
__global__ void prep_kernel(Params p, int chains) {
  const int chain = blockIdx.x;
  if (chain >= chains) return;
  const int P = 3 * p.F * p.D, R = 2 * p.F + p.D;
  const float* w0 = chain_w0(p, chain);
  float* wm = p.wm + (size_t)chain * P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) wm[i] = w0[i];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int r = warp; r < R; r += blockDim.x / 32) {
    int len, pstride;
    size_t wb, pb;
    row_geom(r, p.F, p.D, len, wb, pb, pstride);
    float ss = 0.f;
    for (int j = lane; j < len; j += 32) ss += w0[wb + j] * w0[wb + j];
    ss = warp_sum(ss);
    if (lane == 0) p.rho[(size_t)chain * R + r] = (p.norm == SCAL3R_NORM_UNIT) ? 1.f : sqrtf(ss);
  }
}

// Forward update of one chain at step `step`:
//   W~ = W_step + sum_slots partial (fixed slot order),
//   W_{step+1} row = W~ row * rho / max(||W~ row||, eps).
__global__ void update_kernel(Params p, const UpdateItem* __restrict__ upd, int step) {
  const UpdateItem u = upd[blockIdx.x];
  const int P = 3 * p.F * p.D, R = 2 * p.F + p.D;
  const int chains = p.S * p.H;
  const int h = u.chain % p.H;
  const float* wcur = p.wm + ((size_t)(step & 1) * chains + u.chain) * P;
  float* wnext = p.wm + ((size_t)((step + 1) & 1) * chains + u.chain) * P;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int rows_per_block = (R + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * rows_per_block;
  const int r1 = min(R, r0 + rows_per_block);
  if (u.chunk < 0) {   // sequence without chunks: w_final = w0
    if (p.w_final && blockIdx.y == 0) {
      float* wf = p.w_final + ((size_t)u.seq * p.H + h) * P;
      for (int i = threadIdx.x; i < P; i += blockDim.x) wf[i] = wcur[i];
    }
    return;
  }
  float* ck = p.w_ckpt ? p.w_ckpt + ((size_t)u.chunk * p.H + h) * P : nullptr;
  float* wf = (p.w_final && u.last) ? p.w_final + ((size_t)u.seq * p.H + h) * P : nullptr;
  constexpr int kMaxPer = 8;  // row length <= 256
  for (int r = r0 + warp; r < r1; r += kWarps) {
    int len, pstride;
    size_t wb, pb;
    row_geom(r, p.F, p.D, len, wb, pb, pstride);
    float x[kMaxPer];
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < kMaxPer; ++i) {
      const int j = lane + 32 * i;
      x[i] = 0.f;
      if (j < len) {
        float a = wcur[wb + j];
        for (int sl = 0; sl < u.nslots; ++sl)
          a += p.part[(size_t)(u.slot0 + sl) * P + pb + (size_t)j * pstride];
        x[i] = a;
        ss += a * a;
      }
    }
    ss = warp_sum(ss);
    const float n = sqrtf(ss);
    float scale = 1.f;
    if (p.norm != SCAL3R_NORM_NONE) scale = p.rho[(size_t)u.chain * R + r] / fmaxf(n, p.eps);
#pragma unroll
    for (int i = 0; i < kMaxPer; ++i) {
      const int j = lane + 32 * i;
      if (j < len) {
        const float w = x[i] * scale;
        wnext[wb + j] = w;
        if (ck) ck[wb + j] = w;
        if (wf) wf[wb + j] = w;
      }
    }
    if (lane == 0 && p.wnorm) p.wnorm[((size_t)u.chunk * p.H + h) * R + r] = n;
  }
}

// Backward: zero the carried row-norm adjoints and per-chain dW0, compute
// the row-norm targets from w0.
__global__ void bprep_kernel(Params p, int chains) {
  const int chain = blockIdx.x;
  if (chain >= chains) return;
  const int P = 3 * p.F * p.D, R = 2 * p.F + p.D;
  const float* w0 = chain_w0(p, chain);
  for (int i = threadIdx.x; i < P; i += blockDim.x) p.dw0_chain[(size_t)chain * P + i] = 0.f;
  for (int i = threadIdx.x; i < R; i += blockDim.x) p.drho[(size_t)chain * R + i] = 0.f;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int r = warp; r < R; r += blockDim.x / 32) {
    int len, pstride;
    size_t wb, pb;
    row_geom(r, p.F, p.D, len, wb, pb, pstride);
    float ss = 0.f;
    for (int j = lane; j < len; j += 32) ss += w0[wb + j] * w0[wb + j];
    ss = warp_sum(ss);
    if (lane == 0) p.rho[(size_t)chain * R + r] = (p.norm == SCAL3R_NORM_UNIT) ? 1.f : sqrtf(ss);
  }
}

// Backward step closing: Lambda = R_next (unless this is the chain's last
// chunk) + sum_slots partial.  Then either the VJP of the row normalisation
// of update `chunk` (R = dL/dW~, written to rbuf; row-norm target adjoint
// accumulated in drho) or, for the first chunk, dW0 = Lambda + drho * W0 / rho.
__global__ void bupdate_kernel(Params p, const UpdateItem* __restrict__ upd, int step) {
  const UpdateItem u = upd[blockIdx.x];
  const int P = 3 * p.F * p.D, R = 2 * p.F + p.D;
  const int h = u.chain % p.H;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int rows_per_block = (R + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * rows_per_block;
  const int r1 = min(R, r0 + rows_per_block);
  float* rb = p.rbuf + (size_t)u.chain * P;
  const float* wc = (u.chunk >= 0) ? p.w_ckpt_in + ((size_t)u.chunk * p.H + h) * P : nullptr;
  const float* nrm = (u.chunk >= 0) ? p.wnorm_in + ((size_t)u.chunk * p.H + h) * R : nullptr;
  const float* w0 = chain_w0(p, u.chain);
  constexpr int kMaxPer = 8;
  for (int r = r0 + warp; r < r1; r += kWarps) {
    int len, pstride;
    size_t wb, pb;
    row_geom(r, p.F, p.D, len, wb, pb, pstride);
    float lam[kMaxPer];
#pragma unroll
    for (int i = 0; i < kMaxPer; ++i) {
      const int j = lane + 32 * i;
      lam[i] = 0.f;
      if (j < len) {
        float a = u.last ? 0.f : rb[wb + j];
        for (int sl = 0; sl < u.nslots; ++sl)
          a += p.part[(size_t)(u.slot0 + sl) * P + pb + (size_t)j * pstride];
        lam[i] = a;
      }
    }
    const float rho = p.rho[(size_t)u.chain * R + r];
    float* drho = p.drho + (size_t)u.chain * R + r;
    if (u.first) {
      // dW0 = Lambda + drho * W0_row / rho   (rho = ||W0 row|| for ROW_W0)
      float coef = 0.f;
      if (p.norm == SCAL3R_NORM_ROW_W0 && rho > 0.f) coef = *drho / rho;
      float* out = p.dw0_chain + (size_t)u.chain * P;
#pragma unroll
      for (int i = 0; i < kMaxPer; ++i) {
        const int j = lane + 32 * i;
        if (j < len) out[wb + j] = lam[i] + coef * w0[wb + j];
      }
      continue;
    }
    if (p.norm == SCAL3R_NORM_NONE) {
#pragma unroll
      for (int i = 0; i < kMaxPer; ++i) {
        const int j = lane + 32 * i;
        if (j < len) rb[wb + j] = lam[i];
      }
      continue;
    }
    // W_row = rho * w~ / max(||w~||, eps);  w_hat = W_row / rho
    float what[kMaxPer];
    float proj = 0.f;
    const float inv_rho = rho > 0.f ? 1.f / rho : 0.f;
#pragma unroll
    for (int i = 0; i < kMaxPer; ++i) {
      const int j = lane + 32 * i;
      what[i] = (j < len) ? wc[wb + j] * inv_rho : 0.f;
      proj += what[i] * lam[i];
    }
    proj = warp_sum(proj);
    const float n = nrm[r];
    const bool clamped = !(n >= p.eps);
#pragma unroll
    for (int i = 0; i < kMaxPer; ++i) {
      const int j = lane + 32 * i;
      if (j < len) {
        float rr;
        if (clamped) rr = (rho / p.eps) * lam[i];
        else rr = (rho / n) * (lam[i] - what[i] * proj);
        rb[wb + j] = rr;
      }
    }
    if (lane == 0 && p.norm == SCAL3R_NORM_ROW_W0) *drho += proj;
  }
}

// dw0 from the per-chain results: summed over sequences in order when w0 is
// shared, copied per sequence otherwise.
__global__ void bfinal_kernel(Params p) {
  const int P = 3 * p.F * p.D;
  const int h = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    if (p.w0_seq_stride == 0) {
      float a = 0.f;
      for (int s = 0; s < p.S; ++s) a += p.dw0_chain[((size_t)s * p.H + h) * P + i];
      p.dw0[(size_t)h * P + i] = a;
    } else {
      for (int s = 0; s < p.S; ++s)
        p.dw0[(size_t)s * p.w0_seq_stride + (size_t)h * P + i] = p.dw0_chain[((size_t)s * p.H + h) * P + i];
    }
  }
}

}  // namespace

cudaError_t launch_prep(const Params& prm, int chains, cudaStream_t st) {
  prep_kernel<<<chains, 256, 0, st>>>(prm, chains);
  return cudaGetLastError();
}

cudaError_t launch_update(const Params& prm, const UpdateItem* upd, int nupd, int step, cudaStream_t st) {
  if (nupd == 0) return cudaSuccess;
  dim3 grid(nupd, 4);
  update_kernel<<<grid, kWarps * 32, 0, st>>>(prm, upd, step);
  return cudaGetLastError();
}

cudaError_t launch_bupdate(const Params& prm, const UpdateItem* upd, int nupd, int step, cudaStream_t st) {
  if (nupd == 0) return cudaSuccess;
  // the drho accumulation is per row and each row belongs to one warp
  dim3 grid(nupd, 4);
  bupdate_kernel<<<grid, kWarps * 32, 0, st>>>(prm, upd, step);
  return cudaGetLastError();
}

cudaError_t launch_bprep(const Params& prm, int chains, cudaStream_t st);
cudaError_t launch_bprep(const Params& prm, int chains, cudaStream_t st) {
  bprep_kernel<<<chains, 256, 0, st>>>(prm, chains);
  return cudaGetLastError();
}

cudaError_t launch_bfinal(const Params& prm, cudaStream_t st) {
  const int P = 3 * prm.F * prm.D;
  dim3 grid((P + 255) / 256, prm.H);
  bfinal_kernel<<<grid, 256, 0, st>>>(prm);
  return cudaGetLastError();
}

}  // namespace scal3r
