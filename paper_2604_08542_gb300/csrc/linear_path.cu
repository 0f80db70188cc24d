// Linear-model mode of the float32 path: f_W(x) = W x with one D x D fast
// weight per chain (Sec. 3.2, Eq. 3-4 with a linear map instead of the SwiGLU
// network).  With the dot loss the forward is chunk-causal linear attention:
// the queries of chunk c see W0 plus the rate-weighted outer products v k^T of
// chunks 0..c (closed form of Eq. 3-4 when nothing is normalised).
//
// One CTA owns one chain (sequence, head) and runs its whole chunk loop: W
// stays in shared memory from the first chunk to the last, token tiles of
// LTT rows are staged through shared memory, and the chunk's gradient sum sits
// in registers (D*D/256 entries per thread) until the step.  Per chunk c with
// tokens [t0, t1) (Eq. 8-9, the update taken at the pre-chunk weights):
//   e_t = -lr_t v_t (dot)  |  lr_t (W k_t - v_t) (MSE)
//   W~  = W - sum_t e_t k_t^T
//   W   = normalise(W~)      (row targets as for the SwiGLU network)
//   o_t = W q_t              (apply after the update, Eq. 4)
// The backward kernel walks the chunks in reverse with the adjoint R = dL/dW
// in registers: apply VJP (dq, R += do q^T), normalisation VJP (from the
// stored pre-normalisation row norms), update VJP at the pre-chunk weights
// (dk, dv, dlr; MSE adds dy k^T to R).  Every sum runs in a fixed order.
#include "ttt_internal.h"

namespace scal3r {
namespace {

constexpr int LNT = 256;   // threads per CTA
constexpr int LTT = 32;    // tokens per tile
constexpr int LWARPS = LNT / 32;

template <int D>
struct Lin {
  static constexpr int LD = D + 1;          // padded row stride of a D x D matrix in smem
  static constexpr int MAT = D * LD;        // floats of one padded matrix
  static constexpr int NE = D * D / LNT;    // register entries per thread
  static constexpr int RS = LNT / D;        // row step between a thread's entries
  static constexpr int TILE = LTT * D;
};

// Thread tid owns entries (row tid / D + RS * j, column tid % D), j < NE.
template <int D>
__device__ __forceinline__ int own_row(int j) {
  return threadIdx.x / D + Lin<D>::RS * j;
}

template <int D>
__device__ void load_matrix(float* dst, const float* __restrict__ src) {
  for (int i = threadIdx.x; i < D * D; i += LNT) dst[(i / D) * Lin<D>::LD + i % D] = src[i];
}

template <int D>
__device__ void store_matrix(float* __restrict__ dst, const float* src) {
  for (int i = threadIdx.x; i < D * D; i += LNT) dst[i] = src[(i / D) * Lin<D>::LD + i % D];
}

// Rows t < n of a [T, H, D] tensor at tokens t0.., zero beyond.
template <int D>
__device__ void load_tile(float* dst, const float* __restrict__ src, int64_t t0, int n, int H, int h) {
  for (int i = threadIdx.x; i < LTT * D; i += LNT) {
    const int r = i / D, c = i % D;
    dst[i] = r < n ? src[((size_t)(t0 + r) * H + h) * D + c] : 0.f;
  }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Sum over the row's D entries by one warp (lanes take columns lane, lane + 32).
template <int D>
__device__ __forceinline__ float row_dot(const float* a, const float* b) {
  const int lane = threadIdx.x & 31;
  float x = 0.f;
  if (lane < D) x = a[lane] * b[lane];
  if (D > 32) x = fmaf(a[lane + 32], b[lane + 32], x);
  return warp_sum(x);
}

// Row-norm targets (the same for every chunk): ||W0 row|| for row_w0, 1 for
// unit rows.
template <int D>
__device__ void row_targets(const Params& p, const float* W0s, float* rho) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  for (int r = warp; r < D; r += LWARPS) {
    const float* row = W0s + r * Lin<D>::LD;
    const float n = sqrtf(row_dot<D>(row, row));
    if (lane == 0) rho[r] = p.norm == SCAL3R_NORM_ROW_W0 ? n : 1.f;
  }
}

// e_t of the tile (rows of Es): -lr v (dot) or lr (W k - v) (MSE); Y keeps W k.
template <int D>
__device__ void tile_errors(const Params& p, const float* Ws, const float* Ks, const float* Vs, const float* etas,
                            float* Es, float* Ys) {
  using L = Lin<D>;
  for (int i = threadIdx.x; i < LTT * D; i += LNT) {
    const int t = i / D, d = i % D;
    if (p.loss == SCAL3R_LOSS_DOT) {
      Es[i] = -etas[t] * Vs[i];
    } else {
      float y = 0.f;
#pragma unroll 16
      for (int e = 0; e < D; ++e) y = fmaf(Ws[d * L::LD + e], Ks[t * D + e], y);
      if (Ys) Ys[i] = y;
      Es[i] = etas[t] * (y - Vs[i]);
    }
  }
}

template <int D>
__device__ void tile_rates(const Params& p, float* etas, int64_t t0, int n, int h) {
  for (int i = threadIdx.x; i < LTT; i += LNT) etas[i] = i < n ? p.lr[(size_t)(t0 + i) * p.H + h] : 0.f;
}

// The chunk's gradient sum G = sum_t e_t k_t^T at the weights Ws (thread-owned
// entries, tokens in order).
template <int D>
__device__ void chunk_gradient(const Params& p, const float* Ws, float* Ks, float* Vs, float* Es, float* etas,
                               int64_t t0, int64_t t1, int h, float (&g)[Lin<D>::NE]) {
  const int e = threadIdx.x % D;
#pragma unroll
  for (int j = 0; j < Lin<D>::NE; ++j) g[j] = 0.f;
  for (int64_t t = t0; t < t1; t += LTT) {
    const int n = (int)(t1 - t < LTT ? t1 - t : LTT);
    __syncthreads();
    load_tile<D>(Ks, (const float*)p.k, t, n, p.H, h);
    load_tile<D>(Vs, (const float*)p.v, t, n, p.H, h);
    tile_rates<D>(p, etas, t, n, h);
    __syncthreads();
    tile_errors<D>(p, Ws, Ks, Vs, etas, Es, nullptr);
    __syncthreads();
    for (int i = 0; i < n; ++i) {
      const float kv = Ks[i * D + e];
#pragma unroll
      for (int j = 0; j < Lin<D>::NE; ++j) g[j] = fmaf(Es[i * D + own_row<D>(j)], kv, g[j]);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------

template <int D>
__global__ void __launch_bounds__(LNT, 1) linear_fwd_kernel(Params p) {
  using L = Lin<D>;
  extern __shared__ float sm[];
  float* Ws = sm;
  float* Ks = Ws + L::MAT;
  float* Vs = Ks + L::TILE;
  float* Es = Vs + L::TILE;
  float* rho = Es + L::TILE;
  float* etas = rho + D;
  const int H = p.H, chain = blockIdx.x, s = chain / H, h = chain % H;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31, e = threadIdx.x % D;
  load_matrix<D>(Ws, p.w0 + (size_t)s * p.w0_seq_stride + (size_t)h * D * D);
  __syncthreads();
  row_targets<D>(p, Ws, rho);
  for (int c = p.sptr[s]; c < p.sptr[s + 1]; ++c) {
    const int64_t t0 = p.off[c], t1 = p.off[c + 1];
    float g[L::NE];
    chunk_gradient<D>(p, Ws, Ks, Vs, Es, etas, t0, t1, h, g);
    // W~ = W - G
#pragma unroll
    for (int j = 0; j < L::NE; ++j) Ws[own_row<D>(j) * L::LD + e] -= g[j];
    __syncthreads();
    // row norms of W~ (stored for the backward) and the rescale
    for (int r = warp; r < D; r += LWARPS) {
      float* row = Ws + r * L::LD;
      const float n = sqrtf(row_dot<D>(row, row));
      if (lane == 0 && p.wnorm) p.wnorm[((size_t)c * H + h) * D + r] = n;
      if (p.norm != SCAL3R_NORM_NONE) {
        const float sc = rho[r] / fmaxf(n, p.eps);
        if (lane < D) row[lane] *= sc;
        if (D > 32) row[lane + 32] *= sc;
      }
    }
    __syncthreads();
    if (p.w_ckpt) store_matrix<D>(p.w_ckpt + ((size_t)c * H + h) * D * D, Ws);
    // o_t = W q_t
    for (int64_t t = t0; t < t1; t += LTT) {
      const int n = (int)(t1 - t < LTT ? t1 - t : LTT);
      __syncthreads();
      load_tile<D>(Ks, (const float*)p.q, t, n, H, h);
      __syncthreads();
      for (int i = threadIdx.x; i < n * D; i += LNT) {
        const int tt = i / D, d = i % D;
        float o = 0.f;
#pragma unroll 16
        for (int k = 0; k < D; ++k) o = fmaf(Ws[d * L::LD + k], Ks[tt * D + k], o);
        ((float*)p.o)[((size_t)(t + tt) * H + h) * D + d] = o;
      }
    }
    __syncthreads();
  }
  if (p.w_final) store_matrix<D>(p.w_final + (size_t)chain * D * D, Ws);
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

template <int D>
__global__ void __launch_bounds__(LNT, 1) linear_bwd_kernel(Params p) {
  using L = Lin<D>;
  extern __shared__ float sm[];
  float* Rs = sm;                 // adjoint rows for row operations, then R~
  float* Wn = Rs + L::MAT;        // weights after the chunk (seen by its queries)
  float* Wp = Wn + L::MAT;        // weights before the chunk (its gradient's point)
  float* Wt = Wp + L::MAT;        // W~ = Wp - G(Wp), before normalisation
  float* Xs = Wt + L::MAT;        // queries / keys
  float* Zs = Xs + L::TILE;       // upstream gradient / values
  float* Es = Zs + L::TILE;       // e
  float* dEs = Es + L::TILE;      // dL/de
  float* Ys = dEs + L::TILE;      // W k (MSE)
  float* rho = Ys + L::TILE;
  float* drho = rho + D;
  float* etas = drho + D;
  const int H = p.H, chain = blockIdx.x, s = chain / H, h = chain % H;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31, e = threadIdx.x % D;
  const bool mse = p.loss == SCAL3R_LOSS_MSE;
  const float* w0 = p.w0 + (size_t)s * p.w0_seq_stride + (size_t)h * D * D;
  load_matrix<D>(Wp, w0);
  for (int i = threadIdx.x; i < D; i += LNT) drho[i] = 0.f;
  __syncthreads();
  row_targets<D>(p, Wp, rho);
  float r[L::NE];   // R = dL/dW after the chunk being differentiated
#pragma unroll
  for (int j = 0; j < L::NE; ++j) r[j] = 0.f;
  const int c0 = p.sptr[s];
  for (int c = p.sptr[s + 1] - 1; c >= c0; --c) {
    const int64_t t0 = p.off[c], t1 = p.off[c + 1];
    __syncthreads();
    load_matrix<D>(Wn, p.w_ckpt_in + ((size_t)c * H + h) * D * D);
    load_matrix<D>(Wp, c == c0 ? w0 : p.w_ckpt_in + ((size_t)(c - 1) * H + h) * D * D);
    // 1. o = Wn q: dq = Wn^T do, R += do q^T
    for (int64_t t = t0; t < t1; t += LTT) {
      const int n = (int)(t1 - t < LTT ? t1 - t : LTT);
      __syncthreads();
      load_tile<D>(Xs, (const float*)p.q, t, n, H, h);
      load_tile<D>(Zs, (const float*)p.d_o, t, n, H, h);
      __syncthreads();
      for (int i = threadIdx.x; i < n * D; i += LNT) {
        const int tt = i / D, k = i % D;
        float g = 0.f;
#pragma unroll 16
        for (int d = 0; d < D; ++d) g = fmaf(Zs[tt * D + d], Wn[d * L::LD + k], g);
        ((float*)p.dq)[((size_t)(t + tt) * H + h) * D + k] = g;
      }
      for (int i = 0; i < n; ++i) {
        const float qv = Xs[i * D + e];
#pragma unroll
        for (int j = 0; j < L::NE; ++j) r[j] = fmaf(Zs[i * D + own_row<D>(j)], qv, r[j]);
      }
    }
    // 2. W~ = Wp - G(Wp), recomputed
    {
      float g[L::NE];
      chunk_gradient<D>(p, Wp, Xs, Zs, Es, etas, t0, t1, h, g);
#pragma unroll
      for (int j = 0; j < L::NE; ++j) {
        const int d = own_row<D>(j);
        Wt[d * L::LD + e] = Wp[d * L::LD + e] - g[j];
        Rs[d * L::LD + e] = r[j];
      }
    }
    __syncthreads();
    // 3. normalisation VJP, row by row (pre-normalisation norms as stored)
    if (p.norm != SCAL3R_NORM_NONE) {
      for (int row = warp; row < D; row += LWARPS) {
        float* rr = Rs + row * L::LD;
        const float* wt = Wt + row * L::LD;
        const float n = p.wnorm_in[((size_t)c * H + h) * D + row];
        const float dot = row_dot<D>(wt, rr);
        float a, b;   // R~ = a R - b W~
        if (n >= p.eps) {
          const float proj = dot / n;          // what . R
          a = rho[row] / n;
          b = a * proj / n;
          if (lane == 0) drho[row] += proj;
        } else {
          a = rho[row] / p.eps;
          b = 0.f;
          if (lane == 0) drho[row] += dot / p.eps;
        }
        __syncwarp();
        if (lane < D) rr[lane] = a * rr[lane] - b * wt[lane];
        if (D > 32) rr[lane + 32] = a * rr[lane + 32] - b * wt[lane + 32];
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < L::NE; ++j) r[j] = Rs[own_row<D>(j) * L::LD + e];
    }
    // 4. VJP of W~ = Wp - sum_t e_t k_t^T at Wp, given R~ (Rs)
    for (int64_t t = t0; t < t1; t += LTT) {
      const int n = (int)(t1 - t < LTT ? t1 - t : LTT);
      __syncthreads();
      load_tile<D>(Xs, (const float*)p.k, t, n, H, h);
      load_tile<D>(Zs, (const float*)p.v, t, n, H, h);
      tile_rates<D>(p, etas, t, n, h);
      __syncthreads();
      tile_errors<D>(p, Wp, Xs, Zs, etas, Es, Ys);
      // dL/de_t = -R~ k_t
      for (int i = threadIdx.x; i < LTT * D; i += LNT) {
        const int tt = i / D, d = i % D;
        float x = 0.f;
#pragma unroll 16
        for (int k = 0; k < D; ++k) x = fmaf(Rs[d * L::LD + k], Xs[tt * D + k], x);
        dEs[i] = -x;
      }
      __syncthreads();
      // dk_t = -R~^T e_t (+ Wp^T dy_t, dy = lr de), dv_t = -lr de_t
      for (int i = threadIdx.x; i < n * D; i += LNT) {
        const int tt = i / D, k = i % D;
        float x = 0.f;
#pragma unroll 16
        for (int d = 0; d < D; ++d) x = fmaf(Rs[d * L::LD + k], Es[tt * D + d], x);
        float dk = -x;
        if (mse) {
          float y = 0.f;
#pragma unroll 16
          for (int d = 0; d < D; ++d) y = fmaf(Wp[d * L::LD + k], dEs[tt * D + d], y);
          dk = fmaf(etas[tt], y, dk);
        }
        const size_t o = ((size_t)(t + tt) * H + h) * D + k;
        ((float*)p.dk)[o] = dk;
        ((float*)p.dv)[o] = -etas[tt] * dEs[tt * D + k];
      }
      // dlr_t = -v . de (dot)  |  (W k - v) . de (MSE)
      for (int tt = warp; tt < n; tt += LWARPS) {
        float x = 0.f;
        for (int d = lane; d < D; d += 32) {
          const float m = mse ? Ys[tt * D + d] - Zs[tt * D + d] : -Zs[tt * D + d];
          x = fmaf(m, dEs[tt * D + d], x);
        }
        x = warp_sum(x);
        if (lane == 0) p.dlr[(size_t)(t + tt) * H + h] = x;
      }
      // MSE: R += dy k^T
      if (mse) {
        for (int i = 0; i < n; ++i) {
          const float kv = Xs[i * D + e], et = etas[i];
#pragma unroll
          for (int j = 0; j < L::NE; ++j) r[j] = fmaf(et * dEs[i * D + own_row<D>(j)], kv, r[j]);
        }
      }
    }
  }
  __syncthreads();
  // dW0 = R (+ the row-target term drho * W0 row / ||W0 row||)
  load_matrix<D>(Wp, w0);
  __syncthreads();
  float* out = p.w0_seq_stride ? p.dw0 + (size_t)s * p.w0_seq_stride + (size_t)h * D * D
                               : p.dw0_chain + (size_t)chain * D * D;
#pragma unroll
  for (int j = 0; j < L::NE; ++j) {
    const int d = own_row<D>(j);
    float v = r[j];
    if (p.norm == SCAL3R_NORM_ROW_W0) v = fmaf(drho[d] / (rho[d] > 0.f ? rho[d] : 1.f), Wp[d * L::LD + e], v);
    out[d * D + e] = v;
  }
}

// Shared w0: dw0[h] = sum over sequences of the chains' dW0, in sequence order.
__global__ void linear_dw0_sum_kernel(Params p, int P) {
  const int64_t n = (int64_t)p.H * P;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < p.S; ++s) acc += p.dw0_chain[(size_t)s * n + i];
    p.dw0[i] = acc;
  }
}

template <int D>
constexpr size_t fwd_smem() {
  return (Lin<D>::MAT + 3 * Lin<D>::TILE + D + LTT) * sizeof(float);
}
template <int D>
constexpr size_t bwd_smem() {
  return (4 * Lin<D>::MAT + 5 * Lin<D>::TILE + 2 * D + LTT) * sizeof(float);
}

template <int D>
cudaError_t prepare_d() {
  cudaError_t e = cudaFuncSetAttribute(linear_fwd_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fwd_smem<D>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(linear_bwd_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bwd_smem<D>());
}

}  // namespace

bool linear_shape_supported(int D, int F) { return F == D && (D == 16 || D == 32 || D == 64); }

cudaError_t prepare_linear_kernels() {
  cudaError_t e = prepare_d<16>();
  if (e == cudaSuccess) e = prepare_d<32>();
  if (e == cudaSuccess) e = prepare_d<64>();
  return e;
}

cudaError_t launch_linear_forward(const Params& prm, cudaStream_t st) {
  const int chains = prm.S * prm.H;
  if (chains == 0) return cudaSuccess;
  switch (prm.D) {
    case 16: linear_fwd_kernel<16><<<chains, LNT, fwd_smem<16>(), st>>>(prm); break;
    case 32: linear_fwd_kernel<32><<<chains, LNT, fwd_smem<32>(), st>>>(prm); break;
    case 64: linear_fwd_kernel<64><<<chains, LNT, fwd_smem<64>(), st>>>(prm); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_linear_backward(const Params& prm, cudaStream_t st) {
  const int chains = prm.S * prm.H;
  if (chains == 0) return cudaSuccess;
  switch (prm.D) {
    case 16: linear_bwd_kernel<16><<<chains, LNT, bwd_smem<16>(), st>>>(prm); break;
    case 32: linear_bwd_kernel<32><<<chains, LNT, bwd_smem<32>(), st>>>(prm); break;
    case 64: linear_bwd_kernel<64><<<chains, LNT, bwd_smem<64>(), st>>>(prm); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || prm.w0_seq_stride != 0) return e;
  const int P = prm.D * prm.D;
  const int64_t n = (int64_t)prm.H * P;
  const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  linear_dw0_sum_kernel<<<blocks, 256, 0, st>>>(prm, P);
  return cudaGetLastError();
}

}  // namespace scal3r
