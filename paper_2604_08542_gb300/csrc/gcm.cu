// The steps either side of the test-time-training layer in the Global
// Context Memory module (Sec. 4.1, Eq. 5; Supp. "Global Context Memory
// module"): the query-key-value projection with per-head L2 normalisation of
// q and k, the token-wise learning-rate predictor, and the gated residual
// out = alpha o (o W_o^T) + x, with their backward.  The projections are GEMMs
// on the tcgen05 kernel of wide_path.cu (scal3r_ttt_gemm); this file holds the
// row kernels around them.  Token tensors are token-major: x, out [T, d],
// qkv [T, 3d] (q | k | v, head h at columns h*D .. h*D+D-1 of each part),
// d = H * D.
#include <cuda_bf16.h>

#include "ttt_internal.h"

namespace scal3r {
namespace {

constexpr int kMaxHeads = 16;

__device__ __forceinline__ float bf(const __nv_bfloat16 x) { return __bfloat162float(x); }

__device__ __forceinline__ float warp_sum(float x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// lr[t, h] = base * sigmoid(x[t] . w_eta[h] + b_eta[h]); one warp per token.
__global__ void gcm_eta_kernel(const __nv_bfloat16* __restrict__ x, const float* __restrict__ w_eta,
                               const float* __restrict__ b_eta, float base, int64_t T, int H, int d,
                               float* __restrict__ lr, float* __restrict__ sig) {
  const int64_t t = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (t >= T) return;
  float acc[kMaxHeads];
#pragma unroll
  for (int h = 0; h < kMaxHeads; ++h) acc[h] = 0.f;
  const __nv_bfloat16* xr = x + (size_t)t * d;
  for (int j = lane; j < d; j += 32) {
    const float xv = bf(xr[j]);
#pragma unroll
    for (int h = 0; h < kMaxHeads; ++h)
      if (h < H) acc[h] = fmaf(xv, w_eta[(size_t)h * d + j], acc[h]);
  }
#pragma unroll
  for (int h = 0; h < kMaxHeads; ++h) {
    if (h >= H) break;
    const float z = warp_sum(acc[h]) + b_eta[h];
    if (lane == 0) {
      const float s = 1.f / (1.f + __expf(-z));
      sig[(size_t)t * H + h] = s;
      lr[(size_t)t * H + h] = base * s;
    }
  }
}

// q, k, v of token t, head h from the projection (plus bias); q and k scaled
// to unit L2 norm over the head's D values; one warp per (t, h).
__global__ void gcm_qkv_kernel(const float* __restrict__ raw, const float* __restrict__ b, int64_t T, int H, int D,
                               __nv_bfloat16* __restrict__ q, __nv_bfloat16* __restrict__ k,
                               __nv_bfloat16* __restrict__ v, float* __restrict__ qn, float* __restrict__ kn) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (w >= T * H) return;
  const int64_t t = w / H;
  const int h = (int)(w % H);
  const int d = H * D;
  const float* r = raw + (size_t)t * 3 * d + (size_t)h * D;
  const size_t o = (size_t)t * d + (size_t)h * D;
  for (int part = 0; part < 2; ++part) {
    const float* rp = r + (size_t)part * d;
    const float* bp = b + (size_t)part * d + (size_t)h * D;
    float ss = 0.f;
    for (int i = lane; i < D; i += 32) {
      const float a = rp[i] + bp[i];
      ss = fmaf(a, a, ss);
    }
    const float n = sqrtf(warp_sum(ss));
    const float inv = 1.f / fmaxf(n, 1e-12f);
    __nv_bfloat16* out = part ? k : q;
    for (int i = lane; i < D; i += 32) out[o + i] = __float2bfloat16((rp[i] + bp[i]) * inv);
    if (lane == 0) (part ? kn : qn)[w] = n;
  }
  const float* rv = r + 2 * (size_t)d;
  const float* bv = b + 2 * (size_t)d + (size_t)h * D;
  for (int i = lane; i < D; i += 32) v[o + i] = __float2bfloat16(rv[i] + bv[i]);
}

// out = alpha o y + x (Eq. 5), bf16.
__global__ void gcm_gate_kernel(const float* __restrict__ y, const __nv_bfloat16* __restrict__ x,
                                const float* __restrict__ alpha, int64_t n, int d, __nv_bfloat16* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(fmaf(alpha[i % d], y[i], bf(x[i])));
}

// Backward of the gate: dy = alpha o d_out (bf16, for the GEMMs), dx = d_out
// (the residual path, float32), and per 128-token block the column sums of
// y o d_out (d alpha partials).
constexpr int kRowBlock = 128;

__global__ void gcm_gate_bwd_kernel(const __nv_bfloat16* __restrict__ dout, const float* __restrict__ y,
                                    const float* __restrict__ alpha, int64_t T, int d, __nv_bfloat16* __restrict__ dy,
                                    float* __restrict__ dx, float* __restrict__ part) {
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= d) return;
  const int64_t t0 = (int64_t)blockIdx.x * kRowBlock, t1 = min(T, t0 + kRowBlock);
  const float a = alpha[j];
  float s = 0.f;
  for (int64_t t = t0; t < t1; ++t) {
    const size_t i = (size_t)t * d + j;
    const float g = bf(dout[i]);
    dy[i] = __float2bfloat16(a * g);
    dx[i] = g;
    s = fmaf(y[i], g, s);
  }
  part[(size_t)blockIdx.x * d + j] = s;
}

// Column sums of `rows` partial rows (`stride` floats apart), columns
// 0 .. n-1, in row order.
__global__ void colsum_kernel(const float* __restrict__ part, int rows, int stride, int n, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += part[(size_t)r * stride + j];
  out[j] = s;
}

// Backward of the normalisation and of the learning-rate predictor, per
// (t, h), one warp:  dq_raw = (dq - q^ (q^ . dq)) / |q|  (same for k),
// dv_raw = dv, dlogit = dlr * base * s (1 - s).  Writes dqkv [T, 3d] (bf16)
// and dlogit into a zero-padded [T, 64] bf16 array.
__global__ void gcm_qkv_bwd_kernel(const __nv_bfloat16* __restrict__ dq, const __nv_bfloat16* __restrict__ dk,
                                   const __nv_bfloat16* __restrict__ dv, const float* __restrict__ dlr,
                                   const __nv_bfloat16* __restrict__ q, const __nv_bfloat16* __restrict__ k,
                                   const float* __restrict__ qn, const float* __restrict__ kn,
                                   const float* __restrict__ sig, float base, int64_t T, int H, int D,
                                   __nv_bfloat16* __restrict__ dqkv, __nv_bfloat16* __restrict__ dlogit) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (w >= T * H) return;
  const int64_t t = w / H;
  const int h = (int)(w % H);
  const int d = H * D;
  const size_t o = (size_t)t * d + (size_t)h * D;
  __nv_bfloat16* out = dqkv + (size_t)t * 3 * d + (size_t)h * D;
  for (int part = 0; part < 2; ++part) {
    const __nv_bfloat16* g = part ? dk : dq;
    const __nv_bfloat16* u = part ? k : q;
    float p = 0.f;
    for (int i = lane; i < D; i += 32) p = fmaf(bf(u[o + i]), bf(g[o + i]), p);
    p = warp_sum(p);
    const float n = (part ? kn : qn)[w];
    const float inv = 1.f / fmaxf(n, 1e-12f);
    for (int i = lane; i < D; i += 32)
      out[(size_t)part * d + i] = __float2bfloat16((bf(g[o + i]) - bf(u[o + i]) * p) * inv);
  }
  for (int i = lane; i < D; i += 32) out[2 * (size_t)d + i] = dv[o + i];
  if (lane == 0) {
    const float s = sig[w];
    dlogit[(size_t)t * 64 + h] = __float2bfloat16(dlr[w] * base * s * (1.f - s));
  }
  if (h == 0)
    for (int c = H + lane; c < 64; c += 32) dlogit[(size_t)t * 64 + c] = __float2bfloat16(0.f);
}

// Per 128-token block, the column sums of dqkv (d bias) and of dlogit (d b_eta).
__global__ void gcm_bias_part_kernel(const __nv_bfloat16* __restrict__ dqkv, const __nv_bfloat16* __restrict__ dlogit,
                                     int64_t T, int n3, int H, float* __restrict__ part) {
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  const int n = n3 + H;
  if (j >= n) return;
  const int64_t t0 = (int64_t)blockIdx.x * kRowBlock, t1 = min(T, t0 + kRowBlock);
  float s = 0.f;
  for (int64_t t = t0; t < t1; ++t) s += (j < n3) ? bf(dqkv[(size_t)t * n3 + j]) : bf(dlogit[(size_t)t * 64 + (j - n3)]);
  part[(size_t)blockIdx.x * n + j] = s;
}

}  // namespace

size_t gcm_partial_bytes(int64_t T, int d, int H) {
  const int64_t blocks = (T + kRowBlock - 1) / kRowBlock;
  return (size_t)blocks * (3 * (size_t)d + H) * sizeof(float) + (size_t)blocks * d * sizeof(float);
}

bool gcm_heads_supported(int H) { return H >= 1 && H <= kMaxHeads; }

cudaError_t gcm_prep(const float* raw, const float* bqkv, const __nv_bfloat16* x, const float* w_eta,
                     const float* b_eta, float base, int64_t T, int H, int D, __nv_bfloat16* q, __nv_bfloat16* k,
                     __nv_bfloat16* v, float* lr, float* qn, float* kn, float* sig, cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  const int d = H * D;
  gcm_eta_kernel<<<(unsigned)((T + 7) / 8), 256, 0, st>>>(x, w_eta, b_eta, base, T, H, d, lr, sig);
  gcm_qkv_kernel<<<(unsigned)((T * H + 7) / 8), 256, 0, st>>>(raw, bqkv, T, H, D, q, k, v, qn, kn);
  return cudaGetLastError();
}

cudaError_t gcm_gate(const float* y, const __nv_bfloat16* x, const float* alpha, int64_t T, int d,
                     __nv_bfloat16* out, cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  gcm_gate_kernel<<<1024, 256, 0, st>>>(y, x, alpha, T * d, d, out);
  return cudaGetLastError();
}

cudaError_t gcm_gate_backward(const __nv_bfloat16* dout, const float* y, const float* alpha, int64_t T, int d,
                              __nv_bfloat16* dy, float* dx, float* dalpha, float* part, cudaStream_t st) {
  if (T <= 0) return cudaMemsetAsync(dalpha, 0, (size_t)d * sizeof(float), st);
  const int blocks = (int)((T + kRowBlock - 1) / kRowBlock);
  gcm_gate_bwd_kernel<<<dim3(blocks, (d + 255) / 256), 256, 0, st>>>(dout, y, alpha, T, d, dy, dx, part);
  colsum_kernel<<<(d + 255) / 256, 256, 0, st>>>(part, blocks, d, d, dalpha);
  return cudaGetLastError();
}

cudaError_t gcm_prep_backward(const __nv_bfloat16* dq, const __nv_bfloat16* dk, const __nv_bfloat16* dv,
                              const float* dlr, const __nv_bfloat16* q, const __nv_bfloat16* k, const float* qn,
                              const float* kn, const float* sig, float base, int64_t T, int H, int D,
                              __nv_bfloat16* dqkv, __nv_bfloat16* dlogit, float* dbqkv, float* db_eta, float* part,
                              cudaStream_t st) {
  const int d = H * D, n3 = 3 * d, n = n3 + H;
  if (T <= 0) {
    cudaMemsetAsync(dbqkv, 0, (size_t)n3 * sizeof(float), st);
    return cudaMemsetAsync(db_eta, 0, (size_t)H * sizeof(float), st);
  }
  gcm_qkv_bwd_kernel<<<(unsigned)((T * H + 7) / 8), 256, 0, st>>>(dq, dk, dv, dlr, q, k, qn, kn, sig, base, T, H, D,
                                                                   dqkv, dlogit);
  const int blocks = (int)((T + kRowBlock - 1) / kRowBlock);
  gcm_bias_part_kernel<<<dim3(blocks, (n + 255) / 256), 256, 0, st>>>(dqkv, dlogit, T, n3, H, part);
  colsum_kernel<<<(n3 + 255) / 256, 256, 0, st>>>(part, blocks, n, n3, dbqkv);
  // d b_eta: the last H columns of the partial rows
  colsum_kernel<<<1, 32, 0, st>>>(part + n3, blocks, n, H, db_eta);
  return cudaGetLastError();
}

}  // namespace scal3r
