// Plain FP32 SIMT path of the test-time-training layer (no tensor cores).
//
// One CTA processes one work item: a token range of one chain (sequence,
// head) at one chunk step, in tiles of TT tokens.  Fast weights sit in shared
// memory (rows padded by one float so that lanes reading different rows hit
// different banks); token tiles and their intermediates sit in shared memory;
// the per-piece sums over tokens stay in registers, 3*F*D/256 per thread, and
// are written to the piece's partial-sum slot at the end (packed like the
// weights: W1 [F][D], W3 [F][D], W2 [D][F]).
//
// Forward roles (Sec. 4.2, Eq. 8, Eq. 9, Supp. Sec. A):
//   KEY    gradient partial of the chunk at the pre-chunk weights W:
//            z1 = W1 k, z3 = W3 k, a = SiLU(z1), u = a o z3,
//            e~ = lr v (dot loss)  |  lr (v - W2 u) (MSE),   e~ = -dL/df * lr
//            p~ = W2^T e~, g1 = p~ o z3 o SiLU'(z1), g3 = p~ o a,
//            A1 += g1 k^T, A3 += g3 k^T, A2t += u e~^T     (W += A after the step)
//   APPLY  o = W2 (SiLU(W1 q) o W3 q)                          (Eq. 4)
// Backward roles (reverse-mode differentiation of the forward recurrence):
//   BKEY   VJP of W~ = W - G(W; k, v, lr) given R = dL/dW~, at the weights
//          the chunk's gradient was taken at: dk, dv, dlr and the token sums
//          L1 += dz1 k^T, L3 += dz3 k^T, L2t += dp e^T (+ u dy^T for MSE).
//   BAPPLY VJP of o = f_W(q): dq and L1 += dzq1 q^T, L3 += dzq3 q^T,
//          L2t += uq do^T.
#include <cuda_bf16.h>

#include "ttt_internal.h"

namespace scal3r {
namespace {

constexpr int NTH = 256;

__device__ __forceinline__ float ldio(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ float ldio(const __nv_bfloat16* p, size_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ void stio(float* p, size_t i, float v) { p[i] = v; }
__device__ __forceinline__ void stio(__nv_bfloat16* p, size_t i, float v) { p[i] = __float2bfloat16_rn(v); }

template <int D, int F>
struct Geo {
  static constexpr int LDW = D + 1;        // row stride of W1/W3 in smem
  static constexpr int LD2 = F + 1;        // row stride of W2 in smem
  static constexpr int WS = 2 * F * LDW + D * LD2;   // floats of one weight set
  static constexpr int NF = F / 16;        // accumulator rows per thread
  static constexpr int ND = D / 16;        // accumulator cols per thread
};

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

// Packed weights (W1 [F][D], W3 [F][D], W2 [D][F]) from global into padded smem.
template <int D, int F>
__device__ void load_weights(float* ws, const float* __restrict__ w) {
  using G = Geo<D, F>;
  for (int i = threadIdx.x; i < 2 * F * D; i += NTH) {
    const int r = i / D, c = i % D;
    ws[r * G::LDW + c] = w[i];
  }
  float* w2 = ws + 2 * F * G::LDW;
  for (int i = threadIdx.x; i < D * F; i += NTH) {
    const int r = i / F, c = i % F;
    w2[r * G::LD2 + c] = w[2 * F * D + i];
  }
}

template <int D, int F, int TT, typename TIO>
__device__ void load_rows(float* dst, const TIO* __restrict__ src, int64_t t, int n, int H, int h) {
  for (int i = threadIdx.x; i < TT * D; i += NTH) {
    const int r = i / D, c = i % D;
    dst[i] = (r < n) ? ldio(src, ((size_t)(t + r) * H + h) * D + c) : 0.f;
  }
}

template <int D, int F>
__device__ void store_partial(float* __restrict__ out, const float (&acc)[3][Geo<D, F>::NF][Geo<D, F>::ND]) {
  using G = Geo<D, F>;
  const int dg = threadIdx.x % 16, fg = threadIdx.x / 16;
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int b = 0; b < G::NF; ++b)
#pragma unroll
      for (int a = 0; a < G::ND; ++a)
        out[(size_t)m * F * D + (size_t)(fg + 16 * b) * D + dg + 16 * a] = acc[m][b][a];
  // the W2 part in W2's own orientation [D][F]
#pragma unroll
  for (int b = 0; b < G::NF; ++b)
#pragma unroll
    for (int a = 0; a < G::ND; ++a)
      out[2 * (size_t)F * D + (size_t)(dg + 16 * a) * F + fg + 16 * b] = acc[2][b][a];
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------

template <int D, int F>
__global__ void __launch_bounds__(NTH, 1)
fp32_sweep_kernel(Params p, const WorkItem* __restrict__ items, int step) {
  using G = Geo<D, F>;
  constexpr int TT = 16;
  extern __shared__ float sm[];
  float* W1s = sm;
  float* W3s = W1s + F * G::LDW;
  float* W2s = W3s + F * G::LDW;
  float* Ks = sm + G::WS;          // keys or queries
  float* Vs = Ks + TT * D;
  float* Es = Vs + TT * D;
  float* As = Es + TT * D;         // a, later g3 ; apply: h
  float* Z3s = As + TT * F;
  float* SPs = Z3s + TT * F;       // SiLU'(z1), later g1
  float* Us = SPs + TT * F;
  float* etas = Us + TT * F;       // the token's rate; with per-matrix rates three (W1, W3, W2)

  const WorkItem it = items[blockIdx.x];
  const int H = p.H;
  const int h = it.chain % H;
  const int chains = p.S * H;
  const int nr = p.lr_mat ? 3 : 1;
  const float* w = p.wm + ((size_t)(step & 1) * chains + it.chain) * 3 * F * D;
  load_weights<D, F>(sm, w);
  const int tid = threadIdx.x;

  if (it.role == ROLE_APPLY) {
    const float* q = (const float*)p.q;
    float* o = (float*)p.o;
    for (int64_t t = it.t0; t < it.t1; t += TT) {
      const int n = (int)((it.t1 - t) < TT ? (it.t1 - t) : TT);
      __syncthreads();
      load_rows<D, F, TT, float>(Ks, q, t, n, H, h);
      __syncthreads();
      {
        const int f = tid % F;
        for (int i = tid / F; i < TT; i += NTH / F) {
          float z1 = 0.f, z3 = 0.f;
#pragma unroll 16
          for (int d = 0; d < D; ++d) {
            const float kv = Ks[i * D + d];
            z1 = fmaf(kv, W1s[f * G::LDW + d], z1);
            z3 = fmaf(kv, W3s[f * G::LDW + d], z3);
          }
          As[i * F + f] = z1 * sigm(z1) * z3;
        }
      }
      __syncthreads();
      {
        const int d = tid % D;
        for (int i = tid / D; i < TT; i += NTH / D) {
          float acc = 0.f;
#pragma unroll 16
          for (int f = 0; f < F; ++f) acc = fmaf(As[i * F + f], W2s[d * G::LD2 + f], acc);
          if (i < n) o[((size_t)(t + i) * H + h) * D + d] = acc;
        }
      }
    }
    return;
  }

  // ROLE_KEY
  const float* kk = (const float*)p.k;
  const float* vv = (const float*)p.v;
  float acc[3][G::NF][G::ND];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int b = 0; b < G::NF; ++b)
#pragma unroll
      for (int a = 0; a < G::ND; ++a) acc[m][b][a] = 0.f;

  for (int64_t t = it.t0; t < it.t1; t += TT) {
    const int n = (int)((it.t1 - t) < TT ? (it.t1 - t) : TT);
    __syncthreads();
    load_rows<D, F, TT, float>(Ks, kk, t, n, H, h);
    load_rows<D, F, TT, float>(Vs, vv, t, n, H, h);
    for (int i = tid; i < TT * nr; i += NTH)
      etas[i] = (i / nr < n) ? p.lr[((size_t)(t + i / nr) * H + h) * nr + i % nr] : 0.f;
    __syncthreads();
    {  // z1, z3 and the SiLU pieces
      const int f = tid % F;
      for (int i = tid / F; i < TT; i += NTH / F) {
        float z1 = 0.f, z3 = 0.f;
#pragma unroll 16
        for (int d = 0; d < D; ++d) {
          const float kv = Ks[i * D + d];
          z1 = fmaf(kv, W1s[f * G::LDW + d], z1);
          z3 = fmaf(kv, W3s[f * G::LDW + d], z3);
        }
        const float s = sigm(z1);
        const float a = z1 * s;
        As[i * F + f] = a;
        Z3s[i * F + f] = z3;
        SPs[i * F + f] = s * (1.f + z1 * (1.f - s));
        Us[i * F + f] = a * z3;
      }
    }
    __syncthreads();
    {  // e~ = -lr dL/df (one rate); with per-matrix rates -dL/df, the rates follow
      const int d = tid % D;
      for (int i = tid / D; i < TT; i += NTH / D) {
        float e;
        if (p.loss == SCAL3R_LOSS_DOT) {
          e = Vs[i * D + d];
        } else {
          float y = 0.f;
#pragma unroll 16
          for (int f = 0; f < F; ++f) y = fmaf(Us[i * F + f], W2s[d * G::LD2 + f], y);
          e = Vs[i * D + d] - y;
        }
        Es[i * D + d] = p.lr_mat ? e : etas[i] * e;
      }
    }
    __syncthreads();
    {  // p~ = W2^T e~, g1, g3 (matrix j's gradient weighted by its own rate)
      const int f = tid % F;
      for (int i = tid / F; i < TT; i += NTH / F) {
        float pp = 0.f;
#pragma unroll 16
        for (int d = 0; d < D; ++d) pp = fmaf(Es[i * D + d], W2s[d * G::LD2 + f], pp);
        const float p1 = p.lr_mat ? etas[3 * i] * pp : pp, p3 = p.lr_mat ? etas[3 * i + 1] * pp : pp;
        const float g1 = p1 * Z3s[i * F + f] * SPs[i * F + f];
        const float g3 = p3 * As[i * F + f];
        SPs[i * F + f] = g1;
        As[i * F + f] = g3;
        if (p.lr_mat) Us[i * F + f] *= etas[3 * i + 2];   // W2's increment: u (e2 e~)^T
      }
    }
    __syncthreads();
    {  // token sums
      const int dg = tid % 16, fg = tid / 16;
      for (int i = 0; i < TT; ++i) {
        float kd[G::ND], ed[G::ND];
#pragma unroll
        for (int a = 0; a < G::ND; ++a) {
          kd[a] = Ks[i * D + dg + 16 * a];
          ed[a] = Es[i * D + dg + 16 * a];
        }
#pragma unroll
        for (int b = 0; b < G::NF; ++b) {
          const int f = fg + 16 * b;
          const float g1 = SPs[i * F + f], g3 = As[i * F + f], u = Us[i * F + f];
#pragma unroll
          for (int a = 0; a < G::ND; ++a) {
            acc[0][b][a] = fmaf(g1, kd[a], acc[0][b][a]);
            acc[1][b][a] = fmaf(g3, kd[a], acc[1][b][a]);
            acc[2][b][a] = fmaf(u, ed[a], acc[2][b][a]);
          }
        }
      }
    }
  }
  store_partial<D, F>(p.part + (size_t)it.slot * 3 * F * D, acc);
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

template <int D, int F, typename TIO>
__global__ void __launch_bounds__(NTH, 1)
fp32_bsweep_kernel(Params p, const WorkItem* __restrict__ items, int step) {
  using G = Geo<D, F>;
  constexpr int TT = 8;
  extern __shared__ float sm[];
  float* M1 = sm;                    // W1 or R1
  float* M3 = M1 + F * G::LDW;       // W3 or R3
  float* M2 = M3 + F * G::LDW;       // W2 or R2
  float* Ks = sm + G::WS;            // keys / queries
  float* Vs = Ks + TT * D;           // values / upstream grad
  float* Es = Vs + TT * D;           // e
  float* DEs = Es + TT * D;          // de ; dy (MSE)
  float* DKs = DEs + TT * D;         // dk
  float* Ys = DKs + TT * D;          // y (MSE)
  float* As = Ys + TT * D;
  float* Z3s = As + TT * F;
  float* SPs = Z3s + TT * F;
  float* SPPs = SPs + TT * F;
  float* Us = SPPs + TT * F;
  float* Ps = Us + TT * F;
  float* G1s = Ps + TT * F;
  float* G3s = G1s + TT * F;
  float* DUs = G3s + TT * F;
  float* DPs = DUs + TT * F;
  float* DAs = DPs + TT * F;
  float* DZ1s = DAs + TT * F;
  float* DZ3s = DZ1s + TT * F;
  float* DHs = DZ3s + TT * F;        // per-element terms of dlr (of W2's rate with per-matrix rates)
  float* DH1s = DHs + TT * D;        // per-matrix rates: the terms of W1's and W3's rates
  float* DH3s = DH1s + TT * F;
  float* etas = DH3s + TT * F;       // one rate per token, or three (W1, W3, W2)

  const WorkItem it = items[blockIdx.x];
  const int H = p.H;
  const int h = it.chain % H;
  const int s = it.chain / H;
  const int P = 3 * F * D;
  const float* w = (it.wchunk >= 0) ? p.w_ckpt_in + ((size_t)it.wchunk * H + h) * P
                                    : p.w0 + (size_t)s * p.w0_seq_stride + (size_t)h * P;
  const float* rr = p.rbuf + (size_t)it.chain * P;
  const int tid = threadIdx.x;
  float acc[3][G::NF][G::ND];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int b = 0; b < G::NF; ++b)
#pragma unroll
      for (int a = 0; a < G::ND; ++a) acc[m][b][a] = 0.f;
  const bool mse = (p.loss == SCAL3R_LOSS_MSE);

  if (it.role == ROLE_BAPPLY) {
    load_weights<D, F>(sm, w);
    const TIO* q = (const TIO*)p.q;
    const TIO* go = (const TIO*)p.d_o;
    TIO* dq = (TIO*)p.dq;
    for (int64_t t = it.t0; t < it.t1; t += TT) {
      const int n = (int)((it.t1 - t) < TT ? (it.t1 - t) : TT);
      __syncthreads();
      load_rows<D, F, TT, TIO>(Ks, q, t, n, H, h);
      load_rows<D, F, TT, TIO>(Vs, go, t, n, H, h);
      __syncthreads();
      {
        const int f = tid % F;
        for (int i = tid / F; i < TT; i += NTH / F) {
          float z1 = 0.f, z3 = 0.f, du = 0.f;
#pragma unroll 16
          for (int d = 0; d < D; ++d) {
            const float kv = Ks[i * D + d];
            z1 = fmaf(kv, M1[f * G::LDW + d], z1);
            z3 = fmaf(kv, M3[f * G::LDW + d], z3);
            du = fmaf(Vs[i * D + d], M2[d * G::LD2 + f], du);
          }
          const float sg = sigm(z1);
          const float a = z1 * sg;
          Us[i * F + f] = a * z3;
          DZ3s[i * F + f] = du * a;
          DZ1s[i * F + f] = du * z3 * sg * (1.f + z1 * (1.f - sg));
        }
      }
      __syncthreads();
      {
        const int d = tid % D;
        for (int i = tid / D; i < TT; i += NTH / D) {
          float g = 0.f;
#pragma unroll 16
          for (int f = 0; f < F; ++f)
            g = fmaf(DZ1s[i * F + f], M1[f * G::LDW + d], fmaf(DZ3s[i * F + f], M3[f * G::LDW + d], g));
          if (i < n) stio(dq, ((size_t)(t + i) * H + h) * D + d, g);
        }
      }
      {
        const int dg = tid % 16, fg = tid / 16;
        for (int i = 0; i < TT; ++i) {
          float qd[G::ND], od[G::ND];
#pragma unroll
          for (int a = 0; a < G::ND; ++a) {
            qd[a] = Ks[i * D + dg + 16 * a];
            od[a] = Vs[i * D + dg + 16 * a];
          }
#pragma unroll
          for (int b = 0; b < G::NF; ++b) {
            const int f = fg + 16 * b;
            const float z1g = DZ1s[i * F + f], z3g = DZ3s[i * F + f], u = Us[i * F + f];
#pragma unroll
            for (int a = 0; a < G::ND; ++a) {
              acc[0][b][a] = fmaf(z1g, qd[a], acc[0][b][a]);
              acc[1][b][a] = fmaf(z3g, qd[a], acc[1][b][a]);
              acc[2][b][a] = fmaf(u, od[a], acc[2][b][a]);
            }
          }
        }
      }
    }
    store_partial<D, F>(p.part + (size_t)it.slot * P, acc);
    return;
  }

  // ROLE_BKEY
  const TIO* kk = (const TIO*)p.k;
  const TIO* vv = (const TIO*)p.v;
  TIO* dk = (TIO*)p.dk;
  TIO* dv = (TIO*)p.dv;
  const bool pm = p.lr_mat != 0;
  const int nr = pm ? 3 : 1;
  for (int64_t t = it.t0; t < it.t1; t += TT) {
    const int n = (int)((it.t1 - t) < TT ? (it.t1 - t) : TT);
    __syncthreads();
    load_weights<D, F>(sm, w);
    load_rows<D, F, TT, TIO>(Ks, kk, t, n, H, h);
    load_rows<D, F, TT, TIO>(Vs, vv, t, n, H, h);
    for (int i = tid; i < TT * nr; i += NTH)
      etas[i] = (i / nr < n) ? p.lr[((size_t)(t + i / nr) * H + h) * nr + i % nr] : 0.f;
    __syncthreads();
    // ---- recompute at W -------------------------------------------------
    {
      const int f = tid % F;
      for (int i = tid / F; i < TT; i += NTH / F) {
        float z1 = 0.f, z3 = 0.f;
#pragma unroll 16
        for (int d = 0; d < D; ++d) {
          const float kv = Ks[i * D + d];
          z1 = fmaf(kv, M1[f * G::LDW + d], z1);
          z3 = fmaf(kv, M3[f * G::LDW + d], z3);
        }
        const float sg = sigm(z1);
        const float a = z1 * sg;
        As[i * F + f] = a;
        Z3s[i * F + f] = z3;
        SPs[i * F + f] = sg * (1.f + z1 * (1.f - sg));
        SPPs[i * F + f] = sg * (1.f - sg) * (2.f + z1 * (1.f - 2.f * sg));
        Us[i * F + f] = a * z3;
      }
    }
    __syncthreads();
    {
      const int d = tid % D;
      for (int i = tid / D; i < TT; i += NTH / D) {
        // e = lr (dL/df) with one rate; with per-matrix rates the residual
        // dL/df itself (each matrix's rate enters below)
        const float sc = pm ? 1.f : etas[i];
        if (mse) {
          float y = 0.f;
#pragma unroll 16
          for (int f = 0; f < F; ++f) y = fmaf(Us[i * F + f], M2[d * G::LD2 + f], y);
          Ys[i * D + d] = y;
          Es[i * D + d] = sc * (y - Vs[i * D + d]);
        } else {
          Es[i * D + d] = -sc * Vs[i * D + d];
        }
      }
    }
    __syncthreads();
    {
      const int f = tid % F;
      for (int i = tid / F; i < TT; i += NTH / F) {
        float pp = 0.f;
#pragma unroll 16
        for (int d = 0; d < D; ++d) pp = fmaf(Es[i * D + d], M2[d * G::LD2 + f], pp);
        Ps[i * F + f] = pp;
        // g1, g3 of the step (with per-matrix rates scaled by W1's, W3's rate)
        G3s[i * F + f] = (pm ? etas[3 * i + 1] : 1.f) * pp * As[i * F + f];
        G1s[i * F + f] = (pm ? etas[3 * i] : 1.f) * pp * Z3s[i * F + f] * SPs[i * F + f];
      }
    }
    __syncthreads();
    // ---- products with R = dL/dW~ ----------------------------------------
    load_weights<D, F>(sm, rr);
    __syncthreads();
    {
      const int d = tid % D;
      for (int i = tid / D; i < TT; i += NTH / D) {
        float de = 0.f, dkk = 0.f;
#pragma unroll 16
        for (int f = 0; f < F; ++f) {
          de = fmaf(Us[i * F + f], M2[d * G::LD2 + f], de);
          dkk = fmaf(G1s[i * F + f], M1[f * G::LDW + d], fmaf(G3s[i * F + f], M3[f * G::LDW + d], dkk));
        }
        DEs[i * D + d] = -de;
        DKs[i * D + d] = -dkk;
      }
    }
    {
      const int f = tid % F;
      for (int i = tid / F; i < TT; i += NTH / F) {
        float du = 0.f, dg1 = 0.f, dg3 = 0.f;
#pragma unroll 16
        for (int d = 0; d < D; ++d) {
          const float kv = Ks[i * D + d];
          du = fmaf(Es[i * D + d], M2[d * G::LD2 + f], du);
          dg1 = fmaf(kv, M1[f * G::LDW + d], dg1);
          dg3 = fmaf(kv, M3[f * G::LDW + d], dg3);
        }
        du = -du;
        dg1 = -dg1;
        dg3 = -dg3;
        const float a = As[i * F + f], z3 = Z3s[i * F + f], sp = SPs[i * F + f], pp = Ps[i * F + f];
        if (pm) {
          // per-matrix rates: the adjoints of (e1 h1), (e3 h3) scaled by their
          // rates; dp is dL/dph (the residual's projection); the rates' terms
          // h1 . dg1 and h3 . dg3 (h1 = ph z3 s', h3 = ph a)
          DH1s[i * F + f] = pp * z3 * sp * dg1;
          DH3s[i * F + f] = pp * a * dg3;
          dg1 *= etas[3 * i];
          dg3 *= etas[3 * i + 1];
          du *= etas[3 * i + 2];
        }
        DPs[i * F + f] = dg3 * a + dg1 * z3 * sp;
        DAs[i * F + f] = dg3 * pp;
        DZ3s[i * F + f] = dg1 * pp * sp;
        DZ1s[i * F + f] = dg1 * pp * z3 * SPPs[i * F + f];
        DUs[i * F + f] = du;
      }
    }
    __syncthreads();
    // ---- back at W --------------------------------------------------------
    load_weights<D, F>(sm, w);
    __syncthreads();
    {
      const int d = tid % D;
      for (int i = tid / D; i < TT; i += NTH / D) {
        const float ds2 = DEs[i * D + d];
        float de = pm ? etas[3 * i + 2] * ds2 : ds2;
#pragma unroll 16
        for (int f = 0; f < F; ++f) de = fmaf(DPs[i * F + f], M2[d * G::LD2 + f], de);
        const float eta = etas[i];
        float dvv, dh;
        if (pm) {
          // per-matrix rates: de = dL/d(residual) itself; W2's rate term is
          // residual . ds2; dy = de for the squared error
          DEs[i * D + d] = de;
          dvv = -de;
          dh = Es[i * D + d] * ds2;
        } else if (mse) {
          DEs[i * D + d] = eta * de;                         // dy
          dvv = -eta * de;
          dh = (Ys[i * D + d] - Vs[i * D + d]) * de;
        } else {
          DEs[i * D + d] = de;
          dvv = -eta * de;
          dh = -Vs[i * D + d] * de;
        }
        DHs[i * D + d] = dh;
        if (i < n) stio(dv, ((size_t)(t + i) * H + h) * D + d, dvv);
      }
    }
    __syncthreads();
    {
      const int f = tid % F;
      for (int i = tid / F; i < TT; i += NTH / F) {
        float du = DUs[i * F + f];
        if (mse) {
#pragma unroll 16
          for (int d = 0; d < D; ++d) du = fmaf(DEs[i * D + d], M2[d * G::LD2 + f], du);
        }
        const float a = As[i * F + f], z3 = Z3s[i * F + f];
        const float da = DAs[i * F + f] + du * z3;
        DZ3s[i * F + f] += du * a;
        DZ1s[i * F + f] += da * SPs[i * F + f];
      }
    }
    __syncthreads();
    {
      const int d = tid % D;
      for (int i = tid / D; i < TT; i += NTH / D) {
        float g = DKs[i * D + d];
#pragma unroll 16
        for (int f = 0; f < F; ++f)
          g = fmaf(DZ1s[i * F + f], M1[f * G::LDW + d], fmaf(DZ3s[i * F + f], M3[f * G::LDW + d], g));
        if (i < n) stio(dk, ((size_t)(t + i) * H + h) * D + d, g);
      }
      for (int i = tid; i < n; i += NTH) {
        float a = 0.f;
        for (int d2 = 0; d2 < D; ++d2) a += DHs[i * D + d2];   // fixed order
        if (pm) {
          float a1 = 0.f, a3 = 0.f;
          for (int f = 0; f < F; ++f) {
            a1 += DH1s[i * F + f];
            a3 += DH3s[i * F + f];
          }
          float* dl = p.dlr + ((size_t)(t + i) * H + h) * 3;
          dl[0] = a1;
          dl[1] = a3;
          dl[2] = a;
        } else {
          p.dlr[(size_t)(t + i) * H + h] = a;
        }
      }
    }
    {
      const int dg = tid % 16, fg = tid / 16;
      for (int i = 0; i < TT; ++i) {
        float kd[G::ND], ed[G::ND], yd[G::ND];
#pragma unroll
        for (int a = 0; a < G::ND; ++a) {
          kd[a] = Ks[i * D + dg + 16 * a];
          ed[a] = Es[i * D + dg + 16 * a];
          yd[a] = mse ? DEs[i * D + dg + 16 * a] : 0.f;
        }
#pragma unroll
        for (int b = 0; b < G::NF; ++b) {
          const int f = fg + 16 * b;
          const float z1g = DZ1s[i * F + f], z3g = DZ3s[i * F + f], dp = DPs[i * F + f];
          const float u = mse ? Us[i * F + f] : 0.f;
#pragma unroll
          for (int a = 0; a < G::ND; ++a) {
            acc[0][b][a] = fmaf(z1g, kd[a], acc[0][b][a]);
            acc[1][b][a] = fmaf(z3g, kd[a], acc[1][b][a]);
            acc[2][b][a] = fmaf(dp, ed[a], fmaf(u, yd[a], acc[2][b][a]));
          }
        }
      }
    }
  }
  store_partial<D, F>(p.part + (size_t)it.slot * P, acc);
}

template <int D, int F>
constexpr size_t fwd_smem() {
  return sizeof(float) * (Geo<D, F>::WS + 3 * 16 * D + 4 * 16 * F + 3 * 16);
}
template <int D, int F>
constexpr size_t bwd_smem() {
  return sizeof(float) * (Geo<D, F>::WS + 7 * 8 * D + 15 * 8 * F + 3 * 8);
}

template <int D, int F>
cudaError_t launch_fwd(const Params& prm, const WorkItem* items, int n, int step, cudaStream_t st) {
  const size_t smem = fwd_smem<D, F>();
  fp32_sweep_kernel<D, F><<<n, NTH, smem, st>>>(prm, items, step);
  return cudaGetLastError();
}

template <int D, int F, typename TIO>
cudaError_t launch_bwd(const Params& prm, const WorkItem* items, int n, int step, cudaStream_t st) {
  const size_t smem = bwd_smem<D, F>();
  fp32_bsweep_kernel<D, F, TIO><<<n, NTH, smem, st>>>(prm, items, step);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_fp32() {
  const struct {
    const void* f;
    size_t smem;
  } ks[] = {{(const void*)fp32_sweep_kernel<64, 128>, fwd_smem<64, 128>()},
            {(const void*)fp32_sweep_kernel<16, 32>, fwd_smem<16, 32>()},
            {(const void*)fp32_bsweep_kernel<64, 128, float>, bwd_smem<64, 128>()},
            {(const void*)fp32_bsweep_kernel<16, 32, float>, bwd_smem<16, 32>()},
            {(const void*)fp32_bsweep_kernel<64, 128, __nv_bfloat16>, bwd_smem<64, 128>()}};
  for (const auto& k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k.f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

bool fp32_shape_supported(int D, int F) {
  return (D == 64 && F == 128) || (D == 16 && F == 32);
}

cudaError_t launch_fp32_sweep(const Params& prm, const WorkItem* items, int n, int step, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (prm.D == 64 && prm.F == 128) return launch_fwd<64, 128>(prm, items, n, step, st);
  if (prm.D == 16 && prm.F == 32) return launch_fwd<16, 32>(prm, items, n, step, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fp32_bsweep(const Params& prm, const WorkItem* items, int n, int step, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (prm.D == 64 && prm.F == 128) return launch_bwd<64, 128, float>(prm, items, n, step, st);
  if (prm.D == 16 && prm.F == 32) return launch_bwd<16, 32, float>(prm, items, n, step, st);
  return cudaErrorInvalidValue;
}

// Backward of the BF16 path on CUDA cores: bf16 token tensors, fp32 arithmetic.
cudaError_t launch_simt_bsweep_bf16io(const Params& prm, const WorkItem* items, int n, int step, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (prm.D == 64 && prm.F == 128) return launch_bwd<64, 128, __nv_bfloat16>(prm, items, n, step, st);
  return cudaErrorInvalidValue;
}

}  // namespace scal3r
