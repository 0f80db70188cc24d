// BF16 tensor-core path of the test-time-training layer (sm_103a):
// tcgen05.mma with TMEM accumulators, operands staged by TMA, warp-specialised
// CTAs, one CTA per SM (all 512 TMEM columns).
//
// Work item roles (see plan.cpp for the chunk-step schedule):
//
// KEY  (gradient partial of a chunk at the pre-chunk weights, Eq. 8, Eq. 9).
//   The token-lane weight-adjoint pass of bf16_token_lane.cuh with the
//   factors scaled by each token's learning rate e (dot loss):
//     Z1 = K W1^T, Z3 = K W3^T, P = V W2 (p = W2^T v)   per hidden quarter
//     g1~ = e p z3 SiLU'(z1), g3~ = e p a, u~ = e a z3   (a = SiLU(z1))
//     S1 += G1~^T K, S3 += G3~^T K, S2t += U~^T V          (M 128 hidden, N 64, K 128 tokens)
//   S accumulates in TMEM for the whole piece and goes to the piece's slot
//   packed like the weights (S2t transposed); W += the fixed-order sum over
//   pieces (update.cu).
// APPLY (o = f_W(q), Eq. 4).  Lanes = token (M = 128 tokens per tile):
//     Zq = Q [W1; W3]^T                                 (M 128, N 256, K 64)
//   the epilogue (thread = token) forms h = SiLU(zq1) zq3 as bf16 into TMEM,
//     O = H W2^T                                        (M 128, N 64, K 128)
//   with H as the TMEM A operand, and stores O as bf16.
//
// Warp roles: warp 0 issues TMA loads, warp 1 allocates TMEM and issues the
// MMAs (one thread; in the KEY role warp 10 issues the S products), warps
// 2..9 are the epilogue (two warps per TMEM lane quarter).  Every wait is an
// mbarrier wait bounded in time: on timeout the CTA raises an abort flag,
// every role leaves its loop, the status word is set to SCAL3R_ERR_TIMEOUT
// and TMEM is freed.
#include <cudaTypedefs.h>

#include "bf16_token_lane.cuh"
#include "bounds.cuh"
#include "sm100.cuh"
#include "ttt_internal.h"

namespace scal3r {
namespace {

using namespace sm100;

constexpr int D = 64;
constexpr int F = 128;
constexpr int NTHREADS = 352;   // the KEY role's second MMA warp is warp 10
constexpr int EPI0 = 2;       // first epilogue warp
constexpr int QT = 128;       // query tile (tokens)
constexpr int QSTAGES = 3;    // Q stages, 16 KB each

// TMEM columns, apply role
constexpr uint32_t A_ZQ = 0;      // z1 0..127, z3 128..255
constexpr uint32_t A_H = 256;     // two buffers of h as bf16 pairs, 64 columns each (tile i: i & 1)
constexpr uint32_t A_O = 384;     // two o accumulators, 64 columns each

constexpr uint32_t IDESC_AZ = idesc_bf16(128, 2 * F, false, false);
constexpr uint32_t IDESC_AO = idesc_bf16(128, D, false, false);

constexpr size_t KEY_SMEM = tl::SMEM_BYTES;
constexpr size_t APPLY_SMEM = 2 * F * 128 + 2 * D * 128 + (size_t)QSTAGES * QT * 128;
constexpr size_t DYN_SMEM = 1024 + (KEY_SMEM > APPLY_SMEM ? KEY_SMEM : APPLY_SMEM);

struct TmaMaps {
  CUtensorMap q;   // box 64 x 1 x 128 tokens
  CUtensorMap k;   // box 64 x 1 x 64 tokens
  CUtensorMap v;   // box 64 x 1 x 64 tokens
};

struct Bars {   // APPLY
  uint64_t q_full[QSTAGES], q_empty[QSTAGES];
  uint64_t zq_full, zq_free, h_full[2], o_full[2], o_free[2];
  uint32_t tmem_base;
  int abort_flag;
};


// ---------------------------------------------------------------------------
// APPLY role
// ---------------------------------------------------------------------------
__device__ void apply_load_weights(const float* w, uint8_t* sm) {
  // [W1; W3] as 256 rows x 64 (K-major, swizzled) and W2 as two [64][64]
  // K-blocks (rows d, columns f).  Chunks of 8 values: 8 of [W1; W3] and 4 of
  // W2 per thread, all loaded before any is stored.
  uint8_t* wb13 = sm;
  uint8_t* wb2 = sm + 2 * F * 128;
  const int t = threadIdx.x - 64;   // epilogue threads 0..255
  constexpr int N13 = 2 * F * 8 / 256, N2 = D * (F / 8) / 256;
  float4 v[N13 + N2][2];
#pragma unroll
  for (int i = 0; i < N13; ++i) {
    const int c = t + 256 * i;
    const float4* src = reinterpret_cast<const float4*>(w + (size_t)(c >> 3) * D + (c & 7) * 8);
    v[i][0] = ldg_chk(src);
    v[i][1] = ldg_chk(src + 1);
  }
  const float* w2 = w + 2 * (size_t)F * D;
#pragma unroll
  for (int i = 0; i < N2; ++i) {
    const int c = t + 256 * i;
    const float4* src = reinterpret_cast<const float4*>(w2 + (size_t)(c / (F / 8)) * F + (c % (F / 8)) * 8);
    v[N13 + i][0] = ldg_chk(src);
    v[N13 + i][1] = ldg_chk(src + 1);
  }
#pragma unroll
  for (int i = 0; i < N13 + N2; ++i) {
    const int c = t + 256 * (i < N13 ? i : i - N13);
    const float4 a = v[i][0], bq = v[i][1];
    const uint4 pk = make_uint4(pack_bf16(a.x, a.y), pack_bf16(a.z, a.w), pack_bf16(bq.x, bq.y), pack_bf16(bq.z, bq.w));
    if (i < N13) {
      *reinterpret_cast<uint4*>(wb13 + sw128_offset(c >> 3, (c & 7) * 8)) = pk;
    } else {
      const int r = c / (F / 8), col = (c % (F / 8)) * 8;   // row d, first f of the chunk
      *reinterpret_cast<uint4*>(wb2 + (col / 64) * (D * 128) + sw128_offset(r, col % 64)) = pk;
    }
  }
  fence_proxy_async_smem();
}

__device__ void apply_role(const TmaMaps& maps, const Params& p, const WorkItem& it, uint8_t* sm, Bars& B,
                           uint32_t tb) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int h = it.chain % p.H;
  const int64_t t0 = it.t0, t1 = it.t1;
  const int ntiles = (int)((t1 - t0 + QT - 1) / QT);
  uint8_t* wb13 = sm;
  uint8_t* wb2 = sm + 2 * F * 128;
  uint8_t* Qs = wb2 + 2 * D * 128;
  volatile int* abort = &B.abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < ntiles; ++i) {
        const int s = i % QSTAGES;
        if (!mbar_wait_spin(&B.q_empty[s], ((i / QSTAGES) & 1) ^ 1, abort)) break;
        mbar_arrive_expect_tx(&B.q_full[s], QT * 128);
        tma_load_3d(Qs + s * QT * 128, &maps.q, &B.q_full[s], 0, h, (int32_t)(t0 + (int64_t)i * QT));
      }
    }
    __syncwarp();
    return;
  }

  if (warp == 1) {
    // the whole warp runs the issue loop; one elected lane issues
    const uint32_t w13 = smem_u32(wb13), w2a = smem_u32(wb2);
    auto issue_zq = [&](int i) -> bool {
      const int s = i % QSTAGES;
      if (!mbar_wait_spin_w(&B.q_full[s], (i / QSTAGES) & 1, abort)) return false;
      if (!mbar_wait_spin_w(&B.zq_free, (i & 1) ^ 1, abort)) return false;
      tc_fence_after();
      const uint32_t qa = smem_u32(Qs + s * QT * 128);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma_ss_w(tb + A_ZQ, sdesc_sw128(qa + kk * 32, 16, 1024), sdesc_sw128(w13 + kk * 32, 16, 1024), IDESC_AZ,
                 kk > 0);
      mma_commit_w(&B.zq_full);
      mma_commit_w(&B.q_empty[s]);
      return true;
    };
    bool ok = issue_zq(0);
    for (int i = 0; i < ntiles && ok; ++i) {
      const int b = i & 1;
      if (i + 1 < ntiles && !issue_zq(i + 1)) break;
      if (!mbar_wait_spin_w(&B.h_full[b], (i >> 1) & 1, abort)) break;
      if (!mbar_wait_spin_w(&B.o_free[b], ((i >> 1) & 1) ^ 1, abort)) break;   // o of tile i - 2 was read
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        mma_ts_w(tb + A_O + 64 * b, tb + A_H + 64 * b + 8 * kk,
                 sdesc_sw128(w2a + (kk / 4) * (D * 128) + (kk % 4) * 32, 16, 1024), IDESC_AO, kk > 0);
      mma_commit_w(&B.o_full[b]);
    }
    return;
  }

  if (warp >= 10) return;   // not a warp of this role
  // epilogue: thread = token row of the tile; half selects f in [64*half, 64*half+64)
  const int ew = warp - 2, half = ew >> 2;
  const uint32_t row = 32u * (warp & 3) + lane;
  const uint32_t lane_base = (32u * (warp & 3)) << 16;
  __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(p.o);
  auto store_o = [&](int i) -> bool {
    const int b = i & 1;
    if (!mbar_wait_spin(&B.o_full[b], (i >> 1) & 1, abort)) return false;
    tc_fence_after();
    float v0[16], v1[16];
    tmem_ld16(tb + lane_base + A_O + 64 * b + 32 * half, v0);
    tmem_ld16(tb + lane_base + A_O + 64 * b + 32 * half + 16, v1);
    // the accumulator is in registers: the next o product into it may start
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&B.o_free[b]);
    const int64_t tok = t0 + (int64_t)i * QT + row;
    if (tok < t1 && p.resid_v) {
      // residual pieces: r = v - f_W(k), rounded once
      const uint4* vv = reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(p.resid_v) +
                                                       ((size_t)tok * p.H + h) * D + 32 * half);
      uint32_t vw[16];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint4 x = ld_chk(vv + c);
        vw[4 * c] = x.x;
        vw[4 * c + 1] = x.y;
        vw[4 * c + 2] = x.z;
        vw[4 * c + 3] = x.w;
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        v0[2 * m] = bf16_lo(vw[m]) - v0[2 * m];
        v0[2 * m + 1] = bf16_hi(vw[m]) - v0[2 * m + 1];
        v1[2 * m] = bf16_lo(vw[8 + m]) - v1[2 * m];
        v1[2 * m + 1] = bf16_hi(vw[8 + m]) - v1[2 * m + 1];
      }
    }
    if (tok < t1) {
      uint4* dst = reinterpret_cast<uint4*>(o + ((size_t)tok * p.H + h) * D + 32 * half);
      st_chk(dst, make_uint4(pack_bf16(v0[0], v0[1]), pack_bf16(v0[2], v0[3]), pack_bf16(v0[4], v0[5]),
                             pack_bf16(v0[6], v0[7])));
      st_chk(dst + 1, make_uint4(pack_bf16(v0[8], v0[9]), pack_bf16(v0[10], v0[11]), pack_bf16(v0[12], v0[13]),
                                 pack_bf16(v0[14], v0[15])));
      st_chk(dst + 2, make_uint4(pack_bf16(v1[0], v1[1]), pack_bf16(v1[2], v1[3]), pack_bf16(v1[4], v1[5]),
                                 pack_bf16(v1[6], v1[7])));
      st_chk(dst + 3, make_uint4(pack_bf16(v1[8], v1[9]), pack_bf16(v1[10], v1[11]), pack_bf16(v1[12], v1[13]),
                                 pack_bf16(v1[14], v1[15])));
    }
    return true;
  };
  // tile i: h(i) into buffer i & 1, then the o of tile i - 1 out while the
  // o product of tile i runs.  h buffer i & 1 was last read by the o product of
  // tile i - 2, which completed before store_o(i - 2) in the previous iteration.
  for (int i = 0; i < ntiles; ++i) {
    if (!mbar_wait_spin(&B.zq_full, i & 1, abort)) break;
    tc_fence_after();
    float z1[64], z3[64];
    {
      // all eight loads in flight together: one TMEM latency
      uint32_t u[8][16];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        tmem_ld16_nowait(tb + lane_base + A_ZQ + 64 * half + 16 * c, u[c]);
        tmem_ld16_nowait(tb + lane_base + A_ZQ + F + 64 * half + 16 * c, u[4 + c]);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) tmem_wait_ld16(u[c]);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          z1[16 * c + j] = __uint_as_float(u[c][j]);
          z3[16 * c + j] = __uint_as_float(u[4 + c][j]);
        }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&B.zq_free);
    uint32_t hp[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) {   // pairs of hidden units on packed float32 lanes
      const f32x2 x = x2(z1[2 * m], z1[2 * m + 1]);
      hp[m] = pack_bf16x2(mul2(mul2(x, sigmoid2(x)), x2(z3[2 * m], z3[2 * m + 1])));
    }
    uint32_t r0[16], r1[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      r0[m] = hp[m];
      r1[m] = hp[16 + m];
    }
    tmem_st16(tb + lane_base + A_H + 64 * (i & 1) + 32 * half, r0);
    tmem_st16(tb + lane_base + A_H + 64 * (i & 1) + 32 * half + 16, r1);
    tmem_st_wait();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&B.h_full[i & 1]);
    if (i > 0 && !store_o(i - 1)) break;
  }
  if (!*abort) store_o(ntiles - 1);
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NTHREADS, 1)
bf16_sweep_kernel(const __grid_constant__ TmaMaps maps, const Params p, const WorkItem* __restrict__ items,
                  int step) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  __shared__ Bars B;
  __shared__ tl::Bars TB;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const WorkItem it = items[blockIdx.x];
  const int chains = p.S * p.H;
  // the step's master weights, or (the backward's residual pieces) the weights
  // the piece names, as the backward's pieces read them
  const int hh = it.chain % p.H, ss = it.chain / p.H;
  const float* w = !p.w_items ? p.wm + ((size_t)(step & 1) * chains + it.chain) * 3 * F * D
                   : it.wchunk >= 0 ? p.w_ckpt_in + ((size_t)it.wchunk * p.H + hh) * 3 * F * D
                                    : p.w0 + (size_t)ss * p.w0_seq_stride + (size_t)hh * 3 * F * D;

  if (threadIdx.x == 0) {
    tl::init_bars(TB);
    for (int i = 0; i < QSTAGES; ++i) {
      mbar_init(&B.q_full[i], 1);
      mbar_init(&B.q_empty[i], 1);
    }
    mbar_init(&B.zq_full, 1);
    mbar_init(&B.zq_free, 8);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&B.h_full[i], 8);   // the epilogue wrote h buffer i
      mbar_init(&B.o_full[i], 1);   // the o product of buffer i completed
      mbar_init(&B.o_free[i], 8);   // the epilogue read o accumulator i
    }
    B.abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&maps.q);
    prefetch_tmap(&maps.k);
    prefetch_tmap(&maps.v);
  }
  if (warp == 1) {
    tmem_alloc(&B.tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = B.tmem_base;
  // the step's weights come from the kernel ahead of this one
  pdl_wait();

  // weights
  if (warp >= 2 && warp < 10) {
    if (it.role == ROLE_KEY) tl::load_weights<EPI0>(w, sm);
    else apply_load_weights(w, sm);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (it.role == ROLE_KEY) {
    if (p.lr_mat) tl::token_lane_pass<false, EPI0, true>(&maps.k, &maps.v, nullptr, p, it, sm, TB, tb);
    else tl::token_lane_pass<false, EPI0>(&maps.k, &maps.v, nullptr, p, it, sm, TB, tb);
  }
  else apply_role(maps, p, it, sm, B, tb);

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((B.abort_flag || TB.abort_flag) && threadIdx.x == 0) atomicExch(p.status, SCAL3R_ERR_TIMEOUT);
  if (warp == 1) tmem_dealloc(tb, 512);
  (void)lane;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn_fwd() {
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

// [T, H, 64] bf16 token tensor, boxes of 64 x 1 x box_tokens, 128-byte swizzle.
bool make_token_map(CUtensorMap* m, const void* base, int64_t T, int H, int box_tokens) {
  auto fn = encode_fn_fwd();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)D, (cuuint64_t)H, (cuuint64_t)T};
  cuuint64_t strides[2] = {(cuuint64_t)D * 2, (cuuint64_t)H * D * 2};
  cuuint32_t box[3] = {(cuuint32_t)D, 1, (cuuint32_t)box_tokens};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool bf16_shape_supported(int Dd, int Ff) { return Dd == D && Ff == F; }

cudaError_t prepare_bf16_forward() {
  return cudaFuncSetAttribute(bf16_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DYN_SMEM);
}

cudaError_t launch_bf16_sweep(const Params& prm, const WorkItem* items, int n, int step, const void*,
                              cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (prm.T <= 0) return cudaErrorInvalidValue;
  TmaMaps maps;
  if (!make_token_map(&maps.q, prm.q, prm.T, prm.H, QT) || !make_token_map(&maps.k, prm.k, prm.T, prm.H, 64) ||
      !make_token_map(&maps.v, prm.v, prm.T, prm.H, 64))
    return cudaErrorInvalidValue;
  return launch_pdl(bf16_sweep_kernel, dim3(n), dim3(NTHREADS), DYN_SMEM, st, maps, prm, items, step);
}

#ifdef SCAL3R_DEBUG_BOUNDS
cudaError_t bf16_fwd_upload_bounds(const BoundsTable& t, cudaStream_t st) { return upload_bounds_table(t, st); }
#endif

}  // namespace scal3r
