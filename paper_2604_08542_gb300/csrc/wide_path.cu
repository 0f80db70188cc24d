// BF16 tensor-core forward for wide fast weights: the paper's own AMU shape
// (one head, hd = 1024, hidden = k * hd, Supp. "Global Context Memory module")
// and any head_dim that is a multiple of 128 with hidden a multiple of 256.
//
// At these sizes a chain's fast weights (3 * F * D values, 50 MB in float32 at
// D = 1024, F = 4096) do not fit on chip, and every product of the chunk step
// is a large GEMM.  One chunk step (Eq. 8, dot loss Eq. 9, then Eq. 4) of
// chain (s, h), tokens of the chunk t in [t0, t1), M = t1 - t0, is
//   P  = V W2                        [M x F]   (p = W2^T e = -eta P, e = -eta v)
//   Z1 = K W1^T, Z3 = K W3^T         [M x F]   -> per (t, f): a = z1 sigmoid(z1),
//        g1 = p z3 s'(z1), g3 = p a, u~ = -eta a z3          (epilogue, bf16 out)
//   G1 = g1^T K, G3 = g3^T K         [F x D],  G2 = V^T u~   [D x F]
//   W <- W - G, rows rescaled (row norm targets of W0)       (wide_update_kernel)
//   O  = (silu(Q W1^T) o (Q W3^T)) W2^T                      (two GEMMs)
// All GEMMs run on one persistent tcgen05 kernel: 128 x 256 output tiles, K
// in steps of 64 through a four-stage TMA pipeline (128-byte swizzle, either
// operand K- or MN-major), one elected thread of a converged warp issuing
// M128 N256 K16 MMAs into two 256-column TMEM accumulators in turn, and two
// groups of four epilogue warps (TMEM lane = output row), one per accumulator.  The Z1/Z3 GEMMs read W1 and W3 rows of the same 128 hidden
// units into one N = 256 operand, so one tile holds both halves of the gate.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <vector>

#include "sm100.cuh"
#include "ttt_internal.h"

namespace scal3r {
namespace {

using namespace sm100;

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr uint32_t A_STAGE = BM * BK * 2;               // 16 KB
constexpr uint32_t B_STAGE = BN * BK * 2;               // 32 KB
constexpr uint32_t STAGE_BYTES = A_STAGE + B_STAGE;
constexpr size_t GEMM_SMEM = 1024 + STAGES * STAGE_BYTES;
constexpr int GEMM_THREADS = 320;                       // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue

enum Epi : int { EPI_F32 = 0, EPI_BF16 = 1, EPI_KEY = 2, EPI_APPLY = 3 };

struct GemmArgs {
  CUtensorMap a, b0, b1;   // operand maps; b1: W3 rows of the gate GEMMs
  int M, N, K;             // output rows, output columns (N = 256 * tiles), reduction length
  int a_mn, b_mn, gate;    // operand major-ness; gate: B = [W1 rows; W3 rows] of 128 hidden units
  int ha, hb;              // coordinate 1 of the A / B maps (the head of a [T, H, D] tensor)
  int ya, yb;              // row offset added to the A / B map's row coordinate
  int epi;
  void* out0;              // F32 / BF16: [M x N]; KEY: g1; APPLY: h
  void* out1;              // KEY: g3
  void* out2;              // KEY: u~
  int64_t ld_out;          // row stride of the outputs (elements)
  const __nv_bfloat16* p;  // KEY: raw P = V W2, [M x F] with row stride ld_out
  const float* eta;        // KEY: learning rate of output row m at eta[m * eta_stride]
  int64_t eta_stride;
  int* status;
};

__device__ __forceinline__ float silu_d(float z, float& sg) {
  sg = sigmoid_fast(z);
  return z * sg;
}

// Persistent: CTA b takes output tiles b, b + gridDim.x, ... (consecutive
// CTAs share an A row-block).  The TMA warp runs the stage ring across tiles;
// the MMA warp alternates between two 256-column accumulators; epilogue group
// g (four warps, all 128 TMEM lanes) drains the tiles of accumulator g, so a
// tile's epilogue overlaps the next tile's MMAs.
__global__ void __launch_bounds__(GEMM_THREADS, 1) wide_gemm_kernel(const __grid_constant__ GemmArgs g) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tiles_n = g.N / BN;
  const int ntiles = ((g.M + BM - 1) / BM) * tiles_n;
  const int nk = (g.K + BK - 1) / BK;
  volatile int* abort = &abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);
    }
    abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&g.a);
    prefetch_tmap(&g.b0);
    if (g.gate) prefetch_tmap(&g.b1);
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int tm = t / tiles_n, tn = t % tiles_n;
        const int m0 = tm * BM, n0 = tn * BN;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % STAGES;
          if (!mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
          uint8_t* as = sm + s * STAGE_BYTES;
          uint8_t* bs = as + A_STAGE;
          const int k0 = kb * BK;
          if (!g.a_mn) {
            tma_load_3d(as, &g.a, &full[s], k0, g.ha, g.ya + m0);
          } else {
            tma_load_3d(as, &g.a, &full[s], m0, g.ha, g.ya + k0);
            tma_load_3d(as + 8192, &g.a, &full[s], m0 + 64, g.ha, g.ya + k0);
          }
          if (g.gate) {
            const int f0 = tn * (BN / 2);
            tma_load_3d(bs, &g.b0, &full[s], k0, g.hb, g.yb + f0);
            tma_load_3d(bs + B_STAGE / 2, &g.b1, &full[s], k0, g.hb, g.yb + f0);
          } else if (!g.b_mn) {
            tma_load_3d(bs, &g.b0, &full[s], k0, g.hb, g.yb + n0);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) tma_load_3d(bs + 8192 * j, &g.b0, &full[s], n0 + 64 * j, g.hb, g.yb + k0);
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    const uint32_t idesc = idesc_bf16(BM, BN, g.a_mn != 0, g.b_mn != 0);
    uint32_t it = 0;
    int i = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
      const int ac = i & 1;
      if (!mbar_wait_w(&acc_empty[ac], ((i >> 1) & 1) ^ 1, abort)) break;
      tc_fence_after();
      const uint32_t acc = tb + ac * 256;
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = it % STAGES;
        if (!mbar_wait_w(&full[s], (it / STAGES) & 1, abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t as = smem_u32(sm + s * STAGE_BYTES), bs = as + A_STAGE;
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
          const uint64_t ad = g.a_mn ? sdesc_sw128(as + ks * 2048, 8192, 1024) : sdesc_sw128(as + ks * 32, 16, 1024);
          const uint64_t bd = g.b_mn ? sdesc_sw128(bs + ks * 2048, 8192, 1024) : sdesc_sw128(bs + ks * 32, 16, 1024);
          mma_ss_w(acc, ad, bd, idesc, (kb > 0 || ks > 0) ? 1u : 0u);
        }
        mma_commit_w(&empty[s]);
      }
      if (ok) mma_commit_w(&acc_full[ac]);
    }
  } else {
    // epilogue group gp = warps 2..5 (gp 0) or 6..9 (gp 1); thread = output
    // row m0 + row of the TMEM lanes of this warp
    const int gp = (warp - 2) >> 2;
    const uint32_t row = 32u * (warp & 3) + lane;
    const uint32_t lane_base = (32u * (warp & 3)) << 16;
    const uint32_t accb = tb + lane_base + gp * 256;
    int i = gp;
    for (int t = blockIdx.x + gp * gridDim.x; t < ntiles; t += 2 * gridDim.x, i += 2) {
      if (!mbar_wait(&acc_full[gp], (i >> 1) & 1, abort)) break;
      tc_fence_after();
      const int tm = t / tiles_n, tn = t % tiles_n;
      const int m0 = tm * BM, n0 = tn * BN;
      const int m = m0 + (int)row;
      const bool valid = m < g.M;
      if (g.epi == EPI_F32 || g.epi == EPI_BF16) {
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          float v0[16], v1[16];
          tmem_ld16(accb + c, v0);
          tmem_ld16(accb + c + 16, v1);
          if (!valid) continue;
          if (g.epi == EPI_F32) {
            float* o = reinterpret_cast<float*>(g.out0) + (size_t)m * g.ld_out + n0 + c;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              reinterpret_cast<float4*>(o)[j] = make_float4(v0[4 * j], v0[4 * j + 1], v0[4 * j + 2], v0[4 * j + 3]);
              reinterpret_cast<float4*>(o + 16)[j] =
                  make_float4(v1[4 * j], v1[4 * j + 1], v1[4 * j + 2], v1[4 * j + 3]);
            }
          } else {
            __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(g.out0) + (size_t)m * g.ld_out + n0 + c;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              reinterpret_cast<uint4*>(o)[j] = make_uint4(pack_bf16(v0[8 * j], v0[8 * j + 1]),
                                                          pack_bf16(v0[8 * j + 2], v0[8 * j + 3]),
                                                          pack_bf16(v0[8 * j + 4], v0[8 * j + 5]),
                                                          pack_bf16(v0[8 * j + 6], v0[8 * j + 7]));
              reinterpret_cast<uint4*>(o + 16)[j] = make_uint4(pack_bf16(v1[8 * j], v1[8 * j + 1]),
                                                               pack_bf16(v1[8 * j + 2], v1[8 * j + 3]),
                                                               pack_bf16(v1[8 * j + 4], v1[8 * j + 5]),
                                                               pack_bf16(v1[8 * j + 6], v1[8 * j + 7]));
            }
          }
        }
      } else {
        // gate epilogues: columns [0, 128) are z1, [128, 256) z3 of hidden
        // units f0 .. f0 + 127
        const int f0 = tn * (BN / 2);
        const float eta = (g.epi == EPI_KEY && valid) ? g.eta[(size_t)m * g.eta_stride] : 0.f;
        // KEY: this row's 128 values of P, loaded at once (one memory latency
        // per tile instead of one per 16 columns)
        uint4 prow[16];
        if (g.epi == EPI_KEY && valid) {
          const uint4* pp = reinterpret_cast<const uint4*>(g.p + (size_t)m * g.ld_out + f0);
#pragma unroll
          for (int j = 0; j < 16; ++j) prow[j] = __ldg(pp + j);
        }
#pragma unroll
        for (int c = 0; c < BN / 2; c += 16) {
          float z1[16], z3[16];
          tmem_ld16(accb + c, z1);
          tmem_ld16(accb + 128 + c, z3);
          if (!valid) continue;
          const size_t off = (size_t)m * g.ld_out + f0 + c;
          if (g.epi == EPI_APPLY) {
            uint32_t h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float s0, s1;
              const float a0 = silu_d(z1[2 * j], s0), a1 = silu_d(z1[2 * j + 1], s1);
              h[j] = pack_bf16(a0 * z3[2 * j], a1 * z3[2 * j + 1]);
            }
            uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(g.out0) + off);
            o[0] = make_uint4(h[0], h[1], h[2], h[3]);
            o[1] = make_uint4(h[4], h[5], h[6], h[7]);
          } else {
            const uint4 pr0 = prow[c / 8], pr1 = prow[c / 8 + 1];
            const uint32_t pw[8] = {pr0.x, pr0.y, pr0.z, pr0.w, pr1.x, pr1.y, pr1.z, pr1.w};
            uint32_t o1[8], o3[8], ou[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float r[2];
              r[0] = __uint_as_float(pw[j] << 16);
              r[1] = __uint_as_float(pw[j] & 0xFFFF0000u);
              float v1[2], v3[2], vu[2];
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const float x1 = z1[2 * j + e], x3 = z3[2 * j + e];
                float sg;
                const float a = silu_d(x1, sg);
                const float sp = fmaf(a, 1.f - sg, sg);     // silu'(z1)
                const float pv = -eta * r[e];               // p = W2^T e, e = -eta v
                v1[e] = pv * x3 * sp;
                v3[e] = pv * a;
                vu[e] = -eta * a * x3;
              }
              o1[j] = pack_bf16(v1[0], v1[1]);
              o3[j] = pack_bf16(v3[0], v3[1]);
              ou[j] = pack_bf16(vu[0], vu[1]);
            }
            uint4* d1 = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(g.out0) + off);
            uint4* d3 = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(g.out1) + off);
            uint4* du = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(g.out2) + off);
            d1[0] = make_uint4(o1[0], o1[1], o1[2], o1[3]);
            d1[1] = make_uint4(o1[4], o1[5], o1[6], o1[7]);
            d3[0] = make_uint4(o3[0], o3[1], o3[2], o3[3]);
            d3[1] = make_uint4(o3[4], o3[5], o3[6], o3[7]);
            du[0] = make_uint4(ou[0], ou[1], ou[2], ou[3]);
            du[1] = make_uint4(ou[4], ou[5], ou[6], ou[7]);
          }
        }
      }
      // the accumulator is drained: the MMA warp may reuse it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[gp]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (abort_flag && threadIdx.x == 0) atomicExch(g.status, SCAL3R_ERR_TIMEOUT);
  if (warp == 1) tmem_dealloc(tb, 512);
}

// ---------------------------------------------------------------------------
// per-row kernels over the packed weights W1 [F][D], W3 [F][D], W2 [D][F]
// ---------------------------------------------------------------------------
constexpr int ROW_THREADS = 256;

__device__ __forceinline__ void row_geometry(int r, int D, int F, size_t& off, int& len) {
  if (r < 2 * F) {
    off = (size_t)r * D;
    len = D;
  } else {
    off = 2 * (size_t)F * D + (size_t)(r - 2 * F) * F;
    len = F;
  }
}

// Fixed-order block sum (each thread's partial, then warps in order).
__device__ __forceinline__ float block_sum(float x, float* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) red[warp] = x;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0) {
    for (int w = 0; w < ROW_THREADS / 32; ++w) t += red[w];
    red[ROW_THREADS / 32] = t;
  }
  __syncthreads();
  t = red[ROW_THREADS / 32];
  __syncthreads();
  return t;
}

// W0 -> master weights, bf16 copy and row-norm targets (one block per row).
__global__ void __launch_bounds__(ROW_THREADS) wide_prep_kernel(const float* __restrict__ w0, float* __restrict__ wm,
                                                                __nv_bfloat16* __restrict__ wb, float* __restrict__ rho,
                                                                int D, int F, int norm) {
  __shared__ float red[ROW_THREADS / 32 + 1];
  size_t off;
  int len;
  row_geometry(blockIdx.x, D, F, off, len);
  float ss = 0.f;
  for (int i = 4 * threadIdx.x; i < len; i += 4 * ROW_THREADS) {
    const float4 x = *reinterpret_cast<const float4*>(w0 + off + i);
    *reinterpret_cast<float4*>(wm + off + i) = x;
    *reinterpret_cast<uint2*>(wb + off + i) = make_uint2(pack_bf16(x.x, x.y), pack_bf16(x.z, x.w));
    ss += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
  }
  ss = block_sum(ss, red);
  if (threadIdx.x == 0) rho[blockIdx.x] = (norm == SCAL3R_NORM_UNIT) ? 1.f : sqrtf(ss);
}

// W <- W - G, then each row rescaled to its target (Eq. 8 and the row
// normalisation); writes the master, its bf16 copy, and optionally the
// checkpoint, the pre-normalisation row norm and the final weights.
__global__ void __launch_bounds__(ROW_THREADS) wide_update_kernel(float* __restrict__ wm, const float* __restrict__ gr,
                                                                  __nv_bfloat16* __restrict__ wb,
                                                                  const float* __restrict__ rho, float* ckpt,
                                                                  float* wnorm, float* wfinal, int D, int F, int norm,
                                                                  float eps) {
  __shared__ float red[ROW_THREADS / 32 + 1];
  size_t off;
  int len;
  row_geometry(blockIdx.x, D, F, off, len);
  constexpr int kMaxPer = 4;   // float4 per thread: row length <= 4 * 4 * ROW_THREADS = 4096
  float4 x[kMaxPer];
  float ss = 0.f;
#pragma unroll
  for (int j = 0; j < kMaxPer; ++j) {
    const int i = 4 * (threadIdx.x + j * ROW_THREADS);
    if (i < len) {
      const float4 a = *reinterpret_cast<const float4*>(wm + off + i);
      const float4 b = *reinterpret_cast<const float4*>(gr + off + i);
      x[j] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
      ss += x[j].x * x[j].x + x[j].y * x[j].y + x[j].z * x[j].z + x[j].w * x[j].w;
    }
  }
  ss = block_sum(ss, red);
  const float n = sqrtf(ss);
  const float scale = (norm == SCAL3R_NORM_NONE) ? 1.f : rho[blockIdx.x] / fmaxf(n, eps);
  if (threadIdx.x == 0 && wnorm) wnorm[blockIdx.x] = n;
#pragma unroll
  for (int j = 0; j < kMaxPer; ++j) {
    const int i = 4 * (threadIdx.x + j * ROW_THREADS);
    if (i < len) {
      const float4 y = make_float4(x[j].x * scale, x[j].y * scale, x[j].z * scale, x[j].w * scale);
      *reinterpret_cast<float4*>(wm + off + i) = y;
      *reinterpret_cast<uint2*>(wb + off + i) = make_uint2(pack_bf16(y.x, y.y), pack_bf16(y.z, y.w));
      if (ckpt) *reinterpret_cast<float4*>(ckpt + off + i) = y;
      if (wfinal) *reinterpret_cast<float4*>(wfinal + off + i) = y;
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

// A bf16 tensor [rows][heads][cols] (heads = 1 for a plain matrix), rows
// `row_stride` elements apart; box = 64 columns x `box_rows` rows of one head.
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int heads, int64_t cols, int64_t row_stride,
              int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)heads, (cuuint64_t)rows};
  cuuint64_t strides[2] = {(cuuint64_t)cols * 2, (cuuint64_t)row_stride * 2};
  cuuint32_t box[3] = {64, 1, (cuuint32_t)box_rows};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool wide_shape_supported(int D, int F) {
  return D >= 128 && D % 256 == 0 && F >= 256 && F % 256 == 0 && F <= 4096 && D <= 4096;
}

size_t wide_workspace_bytes(const Plan& p, const Shape& s) {
  int64_t mmax = 0;
  for (size_t c = 0; c + 1 < p.chunk_offsets.size(); ++c)
    mmax = std::max<int64_t>(mmax, p.chunk_offsets[c + 1] - p.chunk_offsets[c]);
  mmax = (mmax + BM - 1) / BM * BM;
  const size_t P = (size_t)s.P();
  const size_t act = (size_t)mmax * s.F * 2;           // one [M x F] bf16 buffer
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  return 4 * al(act) + 2 * al(P * 4) + al(P * 2) + al((size_t)s.R() * 4);
}

cudaError_t prepare_wide() {
  return cudaFuncSetAttribute(wide_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM);
}

namespace {

struct WideBufs {
  __nv_bfloat16 *pb, *g1, *g3, *ut;   // [mmax x F] each; pb also holds h
  float *wm, *gr, *rho;
  __nv_bfloat16* wb;
};

WideBufs carve(const Plan& p, const Shape& s, void* ws) {
  int64_t mmax = 0;
  for (size_t c = 0; c + 1 < p.chunk_offsets.size(); ++c)
    mmax = std::max<int64_t>(mmax, p.chunk_offsets[c + 1] - p.chunk_offsets[c]);
  mmax = (mmax + BM - 1) / BM * BM;
  const size_t P = (size_t)s.P();
  const size_t act = (size_t)mmax * s.F * 2;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  uint8_t* b = reinterpret_cast<uint8_t*>(ws);
  WideBufs w;
  w.pb = reinterpret_cast<__nv_bfloat16*>(b); b += al(act);
  w.g1 = reinterpret_cast<__nv_bfloat16*>(b); b += al(act);
  w.g3 = reinterpret_cast<__nv_bfloat16*>(b); b += al(act);
  w.ut = reinterpret_cast<__nv_bfloat16*>(b); b += al(act);
  w.wm = reinterpret_cast<float*>(b); b += al(P * 4);
  w.gr = reinterpret_cast<float*>(b); b += al(P * 4);
  w.wb = reinterpret_cast<__nv_bfloat16*>(b); b += al(P * 2);
  w.rho = reinterpret_cast<float*>(b);
  return w;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 148;
  }
  return n;
}

cudaError_t gemm(GemmArgs& a, cudaStream_t st) {
  if (a.M <= 0 || a.N % BN != 0 || a.K <= 0) return cudaErrorInvalidValue;
  const int tiles = ((a.M + BM - 1) / BM) * (a.N / BN);
  const int grid = std::min(tiles, num_sms());
  wide_gemm_kernel<<<grid, GEMM_THREADS, GEMM_SMEM, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

// The forward of every chain, chunk after chunk (see the file comment).
// `launch` wraps each launch (profiling); kind 0 = GEMM, 1 = update / prep.
cudaError_t wide_forward(const Plan& pl, const Shape& sh, const Params& prm, void* ws,
                         const std::function<cudaError_t(int, double, double, const std::function<cudaError_t()>&)>& launch,
                         cudaStream_t st) {
  const int H = sh.H, D = sh.D, F = sh.F;
  const size_t P = (size_t)sh.P();
  const int R = sh.R();
  WideBufs w = carve(pl, sh, ws);
  const int64_t T = pl.T;
  for (int s = 0; s < pl.S; ++s) {
    for (int h = 0; h < H; ++h) {
      const float* w0 = prm.w0 + (size_t)s * prm.w0_seq_stride + (size_t)h * P;
      cudaError_t e = launch(1, 0, 0, [&] {
        wide_prep_kernel<<<R, ROW_THREADS, 0, st>>>(w0, w.wm, w.wb, w.rho, D, F, prm.norm);
        return cudaGetLastError();
      });
      if (e != cudaSuccess) return e;
      // bf16 weight views: W1 [F][D], W3 [F][D], W2 [D][F]
      const __nv_bfloat16* w1 = w.wb;
      const __nv_bfloat16* w3 = w.wb + (size_t)F * D;
      const __nv_bfloat16* w2 = w.wb + 2 * (size_t)F * D;
      const int c0 = pl.seq_chunk_ptr[s], c1 = pl.seq_chunk_ptr[s + 1];
      for (int c = c0; c < c1; ++c) {
        const int64_t t0 = pl.chunk_offsets[c], t1 = pl.chunk_offsets[c + 1];
        const int M = (int)(t1 - t0);
        const double mfd = 2.0 * M * (double)F * D;
        GemmArgs g;
        std::memset(&g, 0, sizeof(g));
        g.status = prm.status;
        // P = V W2: A = v rows of the chunk (K-major), B = W2 as [D][F] (MN-major)
        {
          GemmArgs a = g;
          if (!make_map(&a.a, prm.v, T, H, D, (int64_t)H * D, 128) || !make_map(&a.b0, w2, D, 1, F, F, 64))
            return cudaErrorInvalidValue;
          a.M = M; a.N = F; a.K = D; a.b_mn = 1; a.ha = h; a.ya = (int)t0;
          a.epi = EPI_BF16; a.out0 = w.pb; a.ld_out = F;
          e = launch(0, mfd, 0, [&] { return gemm(a, st); });
          if (e != cudaSuccess) return e;
        }
        // Z1, Z3 = K [W1; W3]^T with the gradient epilogue -> g1, g3, u~
        {
          GemmArgs a = g;
          if (!make_map(&a.a, prm.k, T, H, D, (int64_t)H * D, 128) || !make_map(&a.b0, w1, F, 1, D, D, 128) ||
              !make_map(&a.b1, w3, F, 1, D, D, 128))
            return cudaErrorInvalidValue;
          a.M = M; a.N = 2 * F; a.K = D; a.gate = 1; a.ha = h; a.ya = (int)t0;
          a.epi = EPI_KEY; a.out0 = w.g1; a.out1 = w.g3; a.out2 = w.ut; a.ld_out = F;
          a.p = w.pb; a.eta = prm.lr + (size_t)t0 * H + h; a.eta_stride = H;
          e = launch(0, 2 * mfd, 0, [&] { return gemm(a, st); });
          if (e != cudaSuccess) return e;
        }
        // G1 = g1^T K, G3 = g3^T K: A = g (MN-major, rows = the chunk's tokens), B = k (MN-major)
        for (int j = 0; j < 2; ++j) {
          GemmArgs a = g;
          if (!make_map(&a.a, j ? w.g3 : w.g1, M, 1, F, F, 64) || !make_map(&a.b0, prm.k, T, H, D, (int64_t)H * D, 64))
            return cudaErrorInvalidValue;
          a.M = F; a.N = D; a.K = M; a.a_mn = 1; a.b_mn = 1; a.hb = h; a.yb = (int)t0;
          a.epi = EPI_F32; a.out0 = w.gr + (size_t)j * F * D; a.ld_out = D;
          e = launch(0, mfd, 0, [&] { return gemm(a, st); });
          if (e != cudaSuccess) return e;
        }
        // G2 = V^T u~: A = v (MN-major), B = u~ (MN-major)
        {
          GemmArgs a = g;
          if (!make_map(&a.a, prm.v, T, H, D, (int64_t)H * D, 64) || !make_map(&a.b0, w.ut, M, 1, F, F, 64))
            return cudaErrorInvalidValue;
          a.M = D; a.N = F; a.K = M; a.a_mn = 1; a.b_mn = 1; a.ha = h; a.ya = (int)t0;
          a.epi = EPI_F32; a.out0 = w.gr + 2 * (size_t)F * D; a.ld_out = F;
          e = launch(0, mfd, 0, [&] { return gemm(a, st); });
          if (e != cudaSuccess) return e;
        }
        // update and normalise
        {
          float* ck = prm.w_ckpt ? prm.w_ckpt + ((size_t)c * H + h) * P : nullptr;
          float* wn = prm.wnorm ? prm.wnorm + ((size_t)c * H + h) * R : nullptr;
          float* wf = (prm.w_final && c == c1 - 1) ? prm.w_final + ((size_t)s * H + h) * P : nullptr;
          e = launch(1, 0, 0, [&] {
            wide_update_kernel<<<R, ROW_THREADS, 0, st>>>(w.wm, w.gr, w.wb, w.rho, ck, wn, wf, D, F, prm.norm,
                                                         prm.eps);
            return cudaGetLastError();
          });
          if (e != cudaSuccess) return e;
        }
        // apply: h = silu(Q W1^T) o (Q W3^T), then o = h W2^T
        {
          GemmArgs a = g;
          if (!make_map(&a.a, prm.q, T, H, D, (int64_t)H * D, 128) || !make_map(&a.b0, w1, F, 1, D, D, 128) ||
              !make_map(&a.b1, w3, F, 1, D, D, 128))
            return cudaErrorInvalidValue;
          a.M = M; a.N = 2 * F; a.K = D; a.gate = 1; a.ha = h; a.ya = (int)t0;
          a.epi = EPI_APPLY; a.out0 = w.pb; a.ld_out = F;
          e = launch(0, 2 * mfd, 0, [&] { return gemm(a, st); });
          if (e != cudaSuccess) return e;
        }
        {
          GemmArgs a = g;
          if (!make_map(&a.a, w.pb, M, 1, F, F, 128) || !make_map(&a.b0, w2, D, 1, F, F, 256))
            return cudaErrorInvalidValue;
          a.M = M; a.N = D; a.K = F;
          a.epi = EPI_BF16; a.out0 = reinterpret_cast<__nv_bfloat16*>(prm.o) + ((size_t)t0 * H + h) * D;
          a.ld_out = (int64_t)H * D;
          e = launch(0, mfd, 0, [&] { return gemm(a, st); });
          if (e != cudaSuccess) return e;
        }
      }
    }
  }
  return cudaSuccess;
}

}  // namespace scal3r
