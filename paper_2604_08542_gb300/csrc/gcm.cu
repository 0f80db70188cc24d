// The steps either side of the test-time-training layer in the Global
// Context Memory module (Sec. 4.1, Eq. 5; Supp. "Global Context Memory
// module"): the query-key-value projection with per-head L2 normalisation of
// q and k, the token-wise learning-rate predictor, and the gated residual
// out = alpha o (o W_o^T) + x, with their backward.
//
// The projections run on the tcgen05 GEMM of wide_path.cu with the row work
// in their epilogues: the QKV product writes bf16 q, k, v (bias added) and the
// sums of squares of every 64 columns of q and k; the output product writes
// out = alpha o y + x and y itself, both bf16.  No float32 [T, 3d] or [T, d]
// plane is written.  This file holds the row kernels that remain (the per-head
// rescale with the learning-rate predictor, the backward of both, column sums)
// and the host sequences of the four scal3r_gcm_* calls.  Token tensors are
// token-major: x, out [T, d], q, k, v [T, H, D] = [T, d], d = H * D.
#include <cuda_bf16.h>

#include <algorithm>

#include "ttt_internal.h"

namespace scal3r {

cudaError_t wide_gcm_qkv(const void* x, const void* wqkv, const float* bqkv, int64_t T, int d, void* q, void* k,
                         void* v, float* ssq, int* status, cudaStream_t st);
cudaError_t wide_gcm_gate(const void* o, const void* wo, const void* x, const float* alpha, int64_t T, int d,
                          void* out, void* y, int* status, cudaStream_t st);
cudaError_t wide_gemm_addin(const void* a, int64_t lda, const void* b, int64_t ldb, const void* add, float* c,
                            int64_t M, int64_t N, int64_t K, int* status, cudaStream_t st);
cudaError_t wide_gemm_bf16(const void* a, int64_t lda, int a_kmajor, const void* b, int64_t ldb, int b_kmajor, void* c,
                           int64_t ldc, int out_fp32, int accumulate, int64_t M, int64_t N, int64_t K, void* ws,
                           size_t ws_bytes, int timeout_test, int* status, cudaStream_t st);
size_t wide_gemm_workspace_bytes(int64_t M, int64_t N, int64_t K, int out_fp32);

namespace {

constexpr int kMaxHeads = 16;
constexpr int kRowBlock = 128;   // tokens per partial row of a column sum
constexpr int kEtaPad = 64;      // the predictor's logits: 64 extra columns of the dqkv plane (zero beyond H)

__device__ __forceinline__ float warp_sum(float x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Eight bf16 of a 16-byte word as floats (exact), and back (round to nearest even).
__device__ __forceinline__ void unpack8(const uint4 w, float (&f)[8]) {
  const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(u[i] << 16);
    f[2 * i + 1] = __uint_as_float(u[i] & 0xFFFF0000u);
  }
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
  return make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
}

int64_t row_blocks(int64_t T) { return (T + kRowBlock - 1) / kRowBlock; }

// q and k of each token scaled to unit L2 norm per head, in place, from the
// QKV epilogue's sums of squares over 64-column groups (ssq [T][2d/64]: q's
// groups, then k's); the norms kept for the backward.  Then the learning-rate
// predictor lr = base * sigmoid(x . w_eta[h] + b_eta[h]).  One warp per
// token, 16-byte accesses; d is a multiple of 256, so every lane runs the
// same number of 8-value chunks.
__global__ void __launch_bounds__(256) gcm_norm_eta_kernel(const float* __restrict__ ssq,
                                                           const __nv_bfloat16* __restrict__ x,
                                                           const float* __restrict__ w_eta,
                                                           const float* __restrict__ b_eta, float base, int64_t T,
                                                           int H, int D, __nv_bfloat16* __restrict__ q,
                                                           __nv_bfloat16* __restrict__ k, float* __restrict__ lr,
                                                           float* __restrict__ qn, float* __restrict__ kn,
                                                           float* __restrict__ sig) {
  const int lane = threadIdx.x & 31, d = H * D, nc = d / 8, gph = D / 64;
  const int64_t step = (int64_t)gridDim.x * (blockDim.x / 32);
  constexpr int kB = 4;   // 8-value chunks of q, k and x per lane in flight at once
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; t < T; t += step) {
    uint4* qr = reinterpret_cast<uint4*>(q + (size_t)t * d);
    uint4* kr = reinterpret_cast<uint4*>(k + (size_t)t * d);
    const uint4* xr = reinterpret_cast<const uint4*>(x + (size_t)t * d);
    // lane h < H: the norm of q's head h; lane 16 + h: of k's head h
    float n = 0.f;
    const int hh = lane & 15, part = lane >> 4;
    if (hh < H) {
      const float* sp = ssq + (size_t)t * (2 * d / 64) + part * (d / 64) + hh * gph;
      float s = 0.f;
      for (int g = 0; g < gph; ++g) s += sp[g];
      n = sqrtf(s);
      (part ? kn : qn)[(size_t)t * H + hh] = n;
    }
    float acc[kMaxHeads];
#pragma unroll
    for (int h = 0; h < kMaxHeads; ++h) acc[h] = 0.f;
    // kB chunks of q, k and x per lane are loaded before any is used, so a
    // token costs about one memory round trip per kB * 32 chunks, not one
    // per dependent step
    for (int c0 = lane; c0 < nc; c0 += 32 * kB) {
      uint4 qv[kB], kv[kB], xv[kB];
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        const int c = c0 + 32 * b;
        if (c < nc) {
          qv[b] = qr[c];
          kv[b] = kr[c];
          xv[b] = __ldg(xr + c);
        }
      }
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        const int c = c0 + 32 * b;
        const bool in = c < nc;
        const int hc = in ? (8 * c) / D : 0;
        const float inq = 1.f / fmaxf(__shfl_sync(0xffffffffu, n, hc), 1e-12f);
        const float ink = 1.f / fmaxf(__shfl_sync(0xffffffffu, n, 16 + hc), 1e-12f);
        if (!in) continue;
        float f[8];
        unpack8(qv[b], f);
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] *= inq;
        qr[c] = pack8(f);
        unpack8(kv[b], f);
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] *= ink;
        kr[c] = pack8(f);
        unpack8(xv[b], f);
#pragma unroll
        for (int h = 0; h < kMaxHeads; ++h) {
          if (h >= H) break;
          const float4* wp = reinterpret_cast<const float4*>(w_eta + (size_t)h * d + 8 * c);
          const float4 a = __ldg(wp), bq = __ldg(wp + 1);
          acc[h] = fmaf(f[0], a.x, fmaf(f[1], a.y, fmaf(f[2], a.z, fmaf(f[3], a.w, acc[h]))));
          acc[h] = fmaf(f[4], bq.x, fmaf(f[5], bq.y, fmaf(f[6], bq.z, fmaf(f[7], bq.w, acc[h]))));
        }
      }
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
}

// Backward of the rescale and of the predictor, one warp per token, into the
// row of ext [T][3d + 64] bf16: columns [0, d) and [d, 2d) the gradients of
// the pre-normalisation q and k,  dq_raw = (dq - q^ (q^ . dq)) / |q|  (q^ the
// unit-norm q the layer saw), [2d, 3d) dv, then dlogit = dlr base s (1 - s)
// for heads h < H and zeros to column 3d + 63.  A head's D values are G =
// min(32, D/8) lanes' chunks; G lanes reduce its dot with xor shuffles inside
// their aligned group, 32/G heads at a time.  Block b takes the kRowBlock
// tokens from b * kRowBlock; once its rows are written (and still in L2) it
// sums them per column, in token order, into part[b][ld] (the partial rows of
// dbqkv and db_eta).
__global__ void __launch_bounds__(256) gcm_qkv_bwd_kernel(const __nv_bfloat16* __restrict__ dq,
                                                          const __nv_bfloat16* __restrict__ dk,
                                                          const __nv_bfloat16* __restrict__ dv,
                                                          const float* __restrict__ dlr,
                                                          const __nv_bfloat16* __restrict__ q,
                                                          const __nv_bfloat16* __restrict__ k,
                                                          const float* __restrict__ qn, const float* __restrict__ kn,
                                                          const float* __restrict__ sig, float base, int64_t T, int H,
                                                          int D, __nv_bfloat16* __restrict__ ext,
                                                          float* __restrict__ part) {
  const int lane = threadIdx.x & 31, d = H * D, nc = d / 8, cph = D / 8;
  const int G = cph < 32 ? cph : 32, hpi = 32 / G, per = cph / G;
  const size_t ld = 3 * (size_t)d + kEtaPad;
  const int64_t t0 = (int64_t)blockIdx.x * kRowBlock, t1 = min(T, t0 + kRowBlock);
  for (int64_t t = t0 + threadIdx.x / 32; t < t1; t += blockDim.x / 32) {
    __nv_bfloat16* out = ext + (size_t)t * ld;
    for (int part = 0; part < 2; ++part) {
      const uint4* gg = reinterpret_cast<const uint4*>((part ? dk : dq) + (size_t)t * d);
      const uint4* uu = reinterpret_cast<const uint4*>((part ? k : q) + (size_t)t * d);
      uint4* oo = reinterpret_cast<uint4*>(out + (size_t)part * d);
      for (int hb = 0; hb < H; hb += hpi) {
        const int h = hb + lane / G, l = lane % G;
        float p = 0.f;
        for (int j = 0; j < per; ++j) {
          const int c = h * cph + l + G * j;
          float a[8], b[8];
          unpack8(uu[c], a);
          unpack8(gg[c], b);
#pragma unroll
          for (int e = 0; e < 8; ++e) p = fmaf(a[e], b[e], p);
        }
        for (int o = G / 2; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        const float inv = 1.f / fmaxf((part ? kn : qn)[(size_t)t * H + h], 1e-12f);
        for (int j = 0; j < per; ++j) {
          const int c = h * cph + l + G * j;
          float a[8], b[8];
          unpack8(uu[c], a);
          unpack8(gg[c], b);
#pragma unroll
          for (int e = 0; e < 8; ++e) b[e] = (b[e] - a[e] * p) * inv;
          oo[c] = pack8(b);
        }
      }
    }
    const uint4* vv = reinterpret_cast<const uint4*>(dv + (size_t)t * d);
    uint4* ov = reinterpret_cast<uint4*>(out + 2 * (size_t)d);
    for (int c = lane; c < nc; c += 32) ov[c] = vv[c];
    for (int col = lane; col < kEtaPad; col += 32) {
      float g = 0.f;
      if (col < H) {
        const float s = sig[(size_t)t * H + col];
        g = dlr[(size_t)t * H + col] * base * s * (1.f - s);
      }
      out[3 * (size_t)d + col] = __float2bfloat16(g);
    }
  }
  // the block's rows are written: their column sums, 8 columns per thread
  __syncthreads();
  for (int v = threadIdx.x; v < (int)(ld / 8); v += blockDim.x) {
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0.f;
    for (int64_t t = t0; t < t1; ++t) {
      float f[8];
      unpack8(reinterpret_cast<const uint4*>(ext + (size_t)t * ld)[v], f);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] += f[e];
    }
    float4* o = reinterpret_cast<float4*>(part + (size_t)blockIdx.x * ld + 8 * v);
    o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    o[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
  }
}

// Per kRowBlock-token block, column sums of a bf16 [T][ncol] array (or of the
// product of two) into part[block][ncol]; one thread per 8 columns.
template <bool PROD>
__global__ void colsum8_part_kernel(const __nv_bfloat16* __restrict__ a, const __nv_bfloat16* __restrict__ b,
                                    int64_t T, int ncol, float* __restrict__ part) {
  const int v = blockIdx.y * blockDim.x + threadIdx.x;
  if (8 * v >= ncol) return;
  const int64_t t0 = (int64_t)blockIdx.x * kRowBlock, t1 = min(T, t0 + kRowBlock);
  float s[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) s[e] = 0.f;
  for (int64_t t = t0; t < t1; ++t) {
    float f[8];
    unpack8(reinterpret_cast<const uint4*>(a + (size_t)t * ncol)[v], f);
    if (PROD) {
      float g[8];
      unpack8(reinterpret_cast<const uint4*>(b + (size_t)t * ncol)[v], g);
#pragma unroll
      for (int e = 0; e < 8; ++e) s[e] = fmaf(f[e], g[e], s[e]);
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) s[e] += f[e];
    }
  }
  float4* o = reinterpret_cast<float4*>(part + (size_t)blockIdx.x * ncol + 8 * v);
  o[0] = make_float4(s[0], s[1], s[2], s[3]);
  o[1] = make_float4(s[4], s[5], s[6], s[7]);
}

// Column sums of `rows` partial rows (`stride` floats apart), columns
// 0 .. n-1.  A block takes 32 columns (lane = column); warp w sums rows
// w, w + 8, w + 16, ... in order, and the eight warp sums are added in warp
// order, so the result is the same on every run.
constexpr int kColsumWarps = 8;
__global__ void __launch_bounds__(32 * kColsumWarps) colsum_kernel(const float* __restrict__ part, int64_t rows,
                                                                    int stride, int n, float* __restrict__ out) {
  __shared__ float ws[kColsumWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (j < n) {
    const float* pc = part + j;
    int64_t r = w;
    // four independent loads in flight, added in row order
    for (; r + 3 * kColsumWarps < rows; r += 4 * kColsumWarps) {
      const float a = pc[(size_t)r * stride], b = pc[(size_t)(r + kColsumWarps) * stride];
      const float c = pc[(size_t)(r + 2 * kColsumWarps) * stride], d = pc[(size_t)(r + 3 * kColsumWarps) * stride];
      s += a;
      s += b;
      s += c;
      s += d;
    }
    for (; r < rows; r += kColsumWarps) s += pc[(size_t)r * stride];
  }
  ws[w][lane] = s;
  __syncthreads();
  if (w == 0 && j < n) {
    float t = ws[0][lane];
#pragma unroll
    for (int i = 1; i < kColsumWarps; ++i) t += ws[i][lane];
    out[j] = t;
  }
}

// Row j of a [rows][cols] matrix scaled by alpha[j]: a bf16 copy (Wo with
// the gate folded in) or float32 in place (dWo).
__global__ void scale_rows_bf16_kernel(const __nv_bfloat16* __restrict__ w, const float* __restrict__ alpha,
                                       int64_t rows, int cols, __nv_bfloat16* __restrict__ out) {
  const int64_t n = rows * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(alpha[i / cols] * __bfloat162float(w[i]));
}
__global__ void scale_rows_f32_kernel(float* __restrict__ w, const float* __restrict__ alpha, int64_t rows, int cols) {
  const int64_t n = rows * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] *= alpha[i / cols];
}

// The predictor's rows below Wqkv in the dx product: rows r < H of
// dst [64][d] = w_eta (bf16), the rest zero.
__global__ void eta_rows_kernel(const float* __restrict__ w_eta, int H, int d, __nv_bfloat16* __restrict__ dst) {
  const int64_t n = (int64_t)kEtaPad * d;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16(i / d < H ? w_eta[i] : 0.f);
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

int grid_of(int64_t n, int per_block, int cap) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block, cap));
}

}  // namespace

bool gcm_heads_supported(int H) { return H >= 1 && H <= kMaxHeads; }

// Workspace of the four calls for T tokens (each uses it from its start).
size_t gcm_workspace_bytes(int64_t T, int H, int D) {
  const int64_t d = (int64_t)H * D, ld = 3 * d + kEtaPad, nb = row_blocks(T);
  const size_t qkv = al256((size_t)T * (2 * d / 64) * sizeof(float));
  const size_t outb = al256((size_t)d * d * 2) + al256((size_t)nb * d * sizeof(float)) +
                      al256(wide_gemm_workspace_bytes(d, d, T, 1));
  const size_t qkvb = al256((size_t)T * ld * 2) + al256((size_t)ld * d * 2) + al256((size_t)nb * ld * sizeof(float)) +
                      al256(wide_gemm_workspace_bytes(3 * d, d, T, 1)) + al256((size_t)kEtaPad * d * sizeof(float)) +
                      al256(wide_gemm_workspace_bytes(kEtaPad, d, T, 1));
  return std::max(qkv, std::max(outb, qkvb));
}

// [q | k | v] = x Wqkv^T + b with the sums of squares in the epilogue, then
// the per-head rescale and the learning-rate predictor.
cudaError_t gcm_qkv(const void* x, const void* wqkv, const float* bqkv, const float* w_eta, const float* b_eta,
                    float base, int64_t T, int H, int D, void* q, void* k, void* v, float* lr, float* qn, float* kn,
                    float* sig, void* ws, int* status, int sms, cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  float* ssq = static_cast<float*>(ws);
  cudaError_t e = wide_gcm_qkv(x, wqkv, bqkv, T, H * D, q, k, v, ssq, status, st);
  if (e != cudaSuccess) return e;
  gcm_norm_eta_kernel<<<grid_of(T, 8, 8 * sms), 256, 0, st>>>(
      ssq, static_cast<const __nv_bfloat16*>(x), w_eta, b_eta, base, T, H, D, static_cast<__nv_bfloat16*>(q),
      static_cast<__nv_bfloat16*>(k), lr, qn, kn, sig);
  return cudaGetLastError();
}

// out = alpha o (o Wo^T) + x and y = o Wo^T (bf16) in one GEMM.
cudaError_t gcm_out(const void* o, const void* wo, const void* x, const float* alpha, int64_t T, int d, void* out,
                    void* y, int* status, cudaStream_t st) {
  return wide_gcm_gate(o, wo, x, alpha, T, d, out, y, status, st);
}

// Backward of the output product and the gate, with the gate folded into
// the weights:  d_o = d_out (diag(alpha) Wo),  dWo = diag(alpha) (d_out^T o),
// dalpha = sum over tokens of y o d_out.  (The residual's d_out joins dx in
// gcm_qkv_backward.)
cudaError_t gcm_out_backward(const void* d_out, const void* o, const void* wo, const void* y, const float* alpha,
                             int64_t T, int d, void* d_o, float* dwo, float* dalpha, void* ws, int* status, int sms,
                             cudaStream_t st) {
  if (T <= 0) {
    cudaMemsetAsync(dwo, 0, (size_t)d * d * sizeof(float), st);
    return cudaMemsetAsync(dalpha, 0, (size_t)d * sizeof(float), st);
  }
  const int64_t nb = row_blocks(T);
  char* c = static_cast<char*>(ws);
  __nv_bfloat16* wos = reinterpret_cast<__nv_bfloat16*>(c);
  c += al256((size_t)d * d * 2);
  float* part = reinterpret_cast<float*>(c);
  c += al256((size_t)nb * d * sizeof(float));
  const size_t gwb = wide_gemm_workspace_bytes(d, d, T, 1);
  scale_rows_bf16_kernel<<<grid_of((int64_t)d * d, 256, 4 * sms), 256, 0, st>>>(
      static_cast<const __nv_bfloat16*>(wo), alpha, d, d, wos);
  cudaError_t e = wide_gemm_bf16(d_out, d, 1, wos, d, 0, d_o, d, 0, 0, T, d, d, nullptr, 0, 0, status, st);
  if (e == cudaSuccess) e = wide_gemm_bf16(d_out, d, 0, o, d, 0, dwo, d, 1, 0, d, d, T, c, gwb, 0, status, st);
  if (e != cudaSuccess) return e;
  scale_rows_f32_kernel<<<grid_of((int64_t)d * d, 256, 4 * sms), 256, 0, st>>>(dwo, alpha, d, d);
  colsum8_part_kernel<true><<<dim3((unsigned)nb, (d / 8 + 255) / 256), 256, 0, st>>>(
      static_cast<const __nv_bfloat16*>(y), static_cast<const __nv_bfloat16*>(d_out), T, d, part);
  colsum_kernel<<<(d + 31) / 32, 32 * kColsumWarps, 0, st>>>(part, nb, d, d, dalpha);
  return cudaGetLastError();
}

// Backward of the rescale, the predictor and the QKV product:
//   ext = [dqkv | dlogit] (bf16 [T][3d + 64]),  dbqkv, db_eta = its column sums,
//   dx = ext [Wqkv; w_eta (64 rows)] + d_out  (one GEMM; the residual added in its epilogue),
//   dWqkv = dqkv^T x,  dw_eta = (dlogit^T x) rows 0 .. H-1.
cudaError_t gcm_qkv_backward(const void* dq, const void* dk, const void* dv, const float* dlr, const void* q,
                             const void* k, const float* qn, const float* kn, const float* sig, float base,
                             const void* x, const void* wqkv, const float* w_eta, const void* d_out, int64_t T, int H,
                             int D, float* dx, float* dwqkv, float* dbqkv, float* dw_eta, float* db_eta, void* ws,
                             int* status, int sms, cudaStream_t st) {
  const int d = H * D, ld = 3 * d + kEtaPad;
  if (T <= 0) {
    cudaMemsetAsync(dwqkv, 0, (size_t)3 * d * d * sizeof(float), st);
    cudaMemsetAsync(dbqkv, 0, (size_t)3 * d * sizeof(float), st);
    cudaMemsetAsync(dw_eta, 0, (size_t)H * d * sizeof(float), st);
    return cudaMemsetAsync(db_eta, 0, (size_t)H * sizeof(float), st);
  }
  const int64_t nb = row_blocks(T);
  char* c = static_cast<char*>(ws);
  __nv_bfloat16* ext = reinterpret_cast<__nv_bfloat16*>(c);
  c += al256((size_t)T * ld * 2);
  __nv_bfloat16* bext = reinterpret_cast<__nv_bfloat16*>(c);
  c += al256((size_t)ld * d * 2);
  float* part = reinterpret_cast<float*>(c);
  c += al256((size_t)nb * ld * sizeof(float));
  void* gws = c;
  const size_t gwb = wide_gemm_workspace_bytes(3 * d, d, T, 1);
  c += al256(gwb);
  float* deta64 = reinterpret_cast<float*>(c);
  c += al256((size_t)kEtaPad * d * sizeof(float));
  void* gws2 = c;   // the split planes of the dw_eta product (its own region: it splits, dWqkv may not)
  const size_t gwb2 = wide_gemm_workspace_bytes(kEtaPad, d, T, 1);
  using bf = __nv_bfloat16;
  gcm_qkv_bwd_kernel<<<(unsigned)nb, 256, 0, st>>>(
      static_cast<const bf*>(dq), static_cast<const bf*>(dk), static_cast<const bf*>(dv), dlr,
      static_cast<const bf*>(q), static_cast<const bf*>(k), qn, kn, sig, base, T, H, D, ext, part);
  colsum_kernel<<<(3 * d + 31) / 32, 32 * kColsumWarps, 0, st>>>(part, nb, ld, 3 * d, dbqkv);
  colsum_kernel<<<1, 32 * kColsumWarps, 0, st>>>(part + 3 * d, nb, ld, H, db_eta);
  cudaError_t e = cudaMemcpyAsync(bext, wqkv, (size_t)3 * d * d * 2, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  eta_rows_kernel<<<grid_of((int64_t)kEtaPad * d, 256, 4 * sms), 256, 0, st>>>(w_eta, H, d, bext + (size_t)3 * d * d);
  e = wide_gemm_addin(ext, ld, bext, d, d_out, dx, T, d, ld, status, st);
  if (e == cudaSuccess) e = wide_gemm_bf16(ext, ld, 0, x, d, 0, dwqkv, d, 1, 0, 3 * d, d, T, gws, gwb, 0, status, st);
  if (e == cudaSuccess)
    e = wide_gemm_bf16(ext + 3 * d, ld, 0, x, d, 0, deta64, d, 1, 0, kEtaPad, d, T, gws2, gwb2, 0, status, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dw_eta, deta64, (size_t)H * d * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace scal3r
