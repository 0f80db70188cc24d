// The token-lane weight-adjoint pass, shared by two sweeps (sm_103a).
//
// Both the backward's apply VJP and the forward's gradient pieces form, per
// (token, hidden unit), three factors from Z1 = X W1^T, Z3 = X W3^T and
// P = Y W2 (Y W2 = (W2^T y) per token), and contract them over tokens:
//   L1 += A1^T X, L3 += A3^T X, L2t += A2^T Y          (M 128 hidden, N 64, K = tokens)
// with, for token t of learning rate eta_t (a = SiLU(z1), s' = SiLU'(z1)),
//   apply VJP (X = q, Y = d_o):     A1 = p z3 s', A3 = p a, A2 = a z3,
//                                   plus dq = [A1 A3] [W1; W3] per token;
//   gradient (X = k, Y = v, Eq. 8): A1 = eta p z3 s', A3 = eta p a, A2 = eta a z3,
//                                   the increment of W for the dot loss (Eq. 9),
//                                   -dW of sum eta L: W1 += A1^T K, W3 += A3^T K, W2 += V^T A2.
// TMEM lane = token.  Per 128-token tile and hidden quarter q (32 units):
//   G1 = X [W1_q; W3_q]^T (N 64), G2 = Y [W2^T_q]^T (N 32), double-buffered in TMEM;
// the epilogue stages A1, A3, A2 of the quarter as bf16 [128 tok][32 hidden]
// tiles (64-byte swizzle); all four quarters of a tile stay in shared memory,
// where they are the MN-major A operands of the tile's L products.  The L sums
// stay in TMEM for the whole piece and go to its slot in the layout of W.
//
// Shared memory (224 KB): W1_q, W3_q, W2^T_q for the four quarters (48 KB),
// two X/Y stages (64 KB), the factor tiles (96 KB), dq staging (16 KB).
// TMEM: L at columns 0..191, two G buffers at 192 and 288, dq at 384.
// Warps: 0 TMA loads, 1 issues the G products, (with dq) 2 TMA stores,
// EPI0..EPI0+7 epilogue, EPI0+8 issues the dq and L products: the two MMA
// streams wait on different conditions, so neither holds the other back.
#pragma once

#include <cudaTypedefs.h>

#include "bounds.cuh"
#include "sm100.cuh"
#include "ttt_internal.h"

namespace scal3r {
namespace tl {

using namespace sm100;

constexpr int D = 64;
constexpr int F = 128;
constexpr int BT = 128;                      // tile (tokens)
constexpr int NQ = 4;                        // hidden-unit quarters
constexpr uint32_t ST_TILE = 8192;           // [128 tok][32 hidden] bf16, 64-byte swizzle
constexpr uint32_t AQ_BYTES = 12 * 1024;     // W1_q, W3_q, W2^T_q: 96 rows x 128 B
constexpr uint32_t AW_OFF = 0;               // 4 quarters, 48 KB
constexpr uint32_t AXY_OFF = 48 * 1024;      // 2 stages x (X 16 KB + Y 16 KB)
constexpr uint32_t AST_OFF = 112 * 1024;     // [factor][quarter] tiles of A1, A3, A2 (96 KB)
constexpr uint32_t ADQ_OFF = 208 * 1024;     // dq staging, two 64-token boxes (16 KB)
constexpr uint32_t SMEM_BYTES = 224 * 1024;
constexpr uint32_t B_L = 0;                  // L1 | L3 | L2t, 64 columns each
constexpr uint32_t A_BUF = 192;              // two buffers of G1 (64) | G2 (32)
constexpr uint32_t A_GBUF = 96;
constexpr uint32_t A_DX = 384;               // dq accumulator [tok][64]

constexpr int RG = 4;                        // token-row groups of 32 (one per TMEM lane quarter)

struct Bars {
  uint64_t xy_full[2], xy_empty[2], ga_full[2], ga_free[2], sq_full[NQ], st_free[RG];
  uint64_t acc_full, acc_free, out_full, out_free, bdone;
  int abort_flag;
};

// One thread initialises (the caller fences the inits).
__device__ inline void init_bars(Bars& B) {
  for (int i = 0; i < 2; ++i) {
    mbar_init(&B.xy_full[i], 1);
    mbar_init(&B.xy_empty[i], 1);
    mbar_init(&B.ga_full[i], 1);   // the MMA fills a G buffer
    mbar_init(&B.ga_free[i], 8);   // the 8 epilogue warps free it
  }
  for (int i = 0; i < NQ; ++i) mbar_init(&B.sq_full[i], 8);
  for (int i = 0; i < RG; ++i) mbar_init(&B.st_free[i], 1);
  mbar_init(&B.acc_full, 1);
  mbar_init(&B.acc_free, 8);
  mbar_init(&B.out_full, 8);
  mbar_init(&B.out_free, 1);
  mbar_init(&B.bdone, 1);
  B.abort_flag = 0;
}

__device__ __forceinline__ uint4 pack8(const float* v) {
  return make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}

// 32 fp32 accumulator columns of this thread's token row -> bf16 in a
// [128 tok][64] tile pair (two 64-token boxes, 128-byte swizzle).
__device__ __forceinline__ void stage_row64(uint8_t* base, uint32_t row, int half, const float* v0,
                                            const float* v1) {
  uint8_t* t = base + (row >> 6) * 8192;
  const uint32_t rr = row & 63;
  *reinterpret_cast<uint4*>(t + sw128_offset(rr, 32 * half)) = pack8(v0);
  *reinterpret_cast<uint4*>(t + sw128_offset(rr, 32 * half + 8)) = pack8(v0 + 8);
  *reinterpret_cast<uint4*>(t + sw128_offset(rr, 32 * half + 16)) = pack8(v1);
  *reinterpret_cast<uint4*>(t + sw128_offset(rr, 32 * half + 24)) = pack8(v1 + 8);
}

__device__ __forceinline__ void store_row64(__nv_bfloat16* dst0, int half, const float* v0, const float* v1) {
  uint4* dst = reinterpret_cast<uint4*>(dst0 + 32 * half);
  st_chk(dst, pack8(v0));
  st_chk(dst + 1, pack8(v0 + 8));
  st_chk(dst + 2, pack8(v1));
  st_chk(dst + 3, pack8(v1 + 8));
}

// The L sums of the piece (TMEM lanes = hidden unit) -> its slot, in the
// layout of W: L1 [F][D], L3 [F][D], L2 [D][F].  A thread holds a row of L1
// and L3 (256 B each), so stored directly every warp store would write 32
// scattered 16-byte pieces; they pass through `stage` instead (64 KB of
// shared memory the piece no longer uses), float4 index swizzled by the row,
// and leave as whole rows, two per warp store.  L2t is stored column-wise,
// which is already coalesced.  Run by the 8 epilogue warps only (they meet
// at named barrier 1).
template <int EPI0>
__device__ __noinline__ void store_lambda(const Params& p, const WorkItem& it, uint32_t tb, uint8_t* stage) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int half = (warp - EPI0) >> 2;
  const uint32_t row = 32u * (warp & 3) + lane;
  const uint32_t lane_base = (32u * (warp & 3)) << 16;
  float* slot = p.part + (size_t)it.slot * 3 * F * D;
  // L2t[f][d] is the W2[d][f] entry: stored in W2's orientation
#pragma unroll
  for (int c = 0; c < 32; c += 16) {
    float v[16];
    tmem_ld16(tb + lane_base + B_L + 128 + 32 * half + c, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) st_chk(slot + 2 * (size_t)F * D + (size_t)(32 * half + c + j) * F + row, v[j]);
  }
  float4* st = reinterpret_cast<float4*>(stage);   // [m][f][16 float4]
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    float v[16];
#pragma unroll
    for (int c = 0; c < 32; c += 16) {
      tmem_ld16(tb + lane_base + B_L + 64 * m + 32 * half + c, v);
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const uint32_t c4 = (32 * half + c) / 4 + x;
        st[(m * F + row) * 16 + (c4 ^ (row & 15))] = make_float4(v[4 * x], v[4 * x + 1], v[4 * x + 2], v[4 * x + 3]);
      }
    }
  }
  named_bar_sync(1, 256);
  const int t = threadIdx.x - 32 * EPI0;
#pragma unroll 2
  for (int k = 0; k < 2 * F * 16 / 256; ++k) {
    const int idx = k * 256 + t, mr = idx >> 4, c4 = idx & 15, f = mr & (F - 1);
    st_chk(reinterpret_cast<float4*>(slot + (size_t)mr * D) + c4, st[mr * 16 + (c4 ^ (f & 15))]);
  }
}

// Weights into shared memory, bf16, in the 128-byte swizzled layout: each of
// the 256 epilogue threads takes 8-value chunks (a row of W1, W3, -R1, -R3, or
// a column of W2, R2 = a row of W2^T, -R2^T).  A batch of chunks is loaded
// before any is stored (the stores are ordered against the loads), so the
// load costs a few round trips, not one per chunk.
//   KEY = true:  quarter q rows   0.. 31 W1[32q + r]   32.. 63 W3[32q + r]
//                                64.. 95 -R1[32q + r]  96..127 -R3[32q + r]
//                               128..159 W2[:][32q + r] 160..191 -R2[:][32q + r]
//   KEY = false: quarter q rows   0.. 31 W1[32q + r]   32.. 63 W3[32q + r]
//                                64.. 95 W2[:][32q + r]
// Chunk c = t + 256 k covers block k (quarter k / blocks, 32 rows).  In a row
// block thread t takes row t / 8, chunk t % 8 (a warp reads 4 whole rows); in
// a column block row t % 32, chunk t / 32, so that a warp's load of one d
// reads 32 consecutive entries of W2's (or R2's) row d.
template <bool KEY>
struct ChunkAt {
  static constexpr int BLOCKS = KEY ? 6 : 3;   // 32-row blocks per quarter
  int q, rr, col, blk, f;
  __device__ __forceinline__ ChunkAt(int t, int k) {
    q = k / BLOCKS;
    const int b = k % BLOCKS;
    blk = KEY ? b : (b < 2 ? b : 4);            // 0 W1, 1 W3, 2 R1, 3 R3, 4 W2, 5 R2
    const bool column = blk >= 4;
    const int r = column ? t % 32 : t / 8;
    col = (column ? t / 32 : t % 8) * 8;
    rr = 32 * b + r;
    f = 32 * q + r;
  }
};

template <bool KEY, int BATCH, int EPI0>
__device__ void load_weight_chunks(const float* w, const float* r, uint8_t* dst, uint32_t qbytes) {
  constexpr int QROWS = KEY ? 192 : 96;
  const int t = threadIdx.x - 32 * EPI0;   // 256 epilogue threads
  constexpr int NCH = NQ * QROWS * 8 / 256;   // chunks per thread
  static_assert(NCH % BATCH == 0, "batch");
#pragma unroll 1
  for (int b0 = 0; b0 < NCH; b0 += BATCH) {
    float v[BATCH][8];
#pragma unroll
    for (int i = 0; i < BATCH; ++i) {
      const ChunkAt<KEY> a(t, b0 + i);
      if (a.blk < 4) {   // W1, W3, R1, R3: row f
        const float4* src = reinterpret_cast<const float4*>(
            (a.blk == 0 ? w : a.blk == 1 ? w + F * D : a.blk == 2 ? r : r + F * D) + (size_t)a.f * D + a.col);
        const float4 x = ldg_chk(src), y = ldg_chk(src + 1);
        v[i][0] = x.x; v[i][1] = x.y; v[i][2] = x.z; v[i][3] = x.w;
        v[i][4] = y.x; v[i][5] = y.y; v[i][6] = y.z; v[i][7] = y.w;
      } else {           // W2, R2 [D][F]: column f
        const float* src = (a.blk == 4 ? w : r) + 2 * (size_t)F * D + a.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) v[i][j] = ldg_chk(src + (size_t)(a.col + j) * F);
      }
    }
#pragma unroll
    for (int i = 0; i < BATCH; ++i) {
      const ChunkAt<KEY> a(t, b0 + i);
      if (a.blk == 2 || a.blk == 3 || a.blk == 5) {   // the adjoint enters negated
#pragma unroll
        for (int j = 0; j < 8; ++j) v[i][j] = -v[i][j];
      }
      *reinterpret_cast<uint4*>(dst + a.q * qbytes + sw128_offset(a.rr, a.col)) = pack8(v[i]);
    }
  }
  fence_proxy_async_smem();
}

// W1, W3, W2^T of the pass (the KEY = false layout above).
template <int EPI0>
__device__ void load_weights(const float* w, uint8_t* sm) {
  load_weight_chunks<false, 12, EPI0>(w, w, sm + AW_OFF, AQ_BYTES);
}

// The pass over the item's tokens.  mx, my: tensor maps of X and Y with
// 64-token boxes; mdq: dq's (DQ only).  DQ selects the apply VJP (with dq
// out), else the gradient (factors scaled by the token's learning rate; PM:
// one rate per matrix, lr [T, H, 3] = W1's, W3's, W2's, each factor scaled by
// the rate of the matrix it updates).
template <bool DQ, int EPI0, bool PM = false>
__device__ void token_lane_pass(const CUtensorMap* mx, const CUtensorMap* my, const CUtensorMap* mdq,
                                const Params& p, const WorkItem& it, uint8_t* sm, Bars& B, uint32_t tb) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int H = p.H;
  const int h = it.chain % H;
  const int64_t t0 = it.t0, t1 = it.t1;
  const int ntiles = (int)((t1 - t0 + BT - 1) / BT);
  const int nq = ntiles * NQ;
  volatile int* abort = &B.abort_flag;
  constexpr uint32_t IDESC_G1 = idesc_bf16(128, 64, false, false);
  constexpr uint32_t IDESC_G2 = idesc_bf16(128, 32, false, false);
  constexpr uint32_t IDESC_ACC = idesc_bf16(128, D, false, true);
  constexpr uint32_t IDESC_LAM = idesc_bf16(128, D, true, true);
  const int ew = warp - EPI0, half = ew >> 2;            // epilogue warps only
  const uint32_t row = 32u * (warp & 3) + lane;
  const uint32_t lane_base = (32u * (warp & 3)) << 16;

  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < ntiles; ++i) {
        const int s = i & 1;
        if (!mbar_wait_spin(&B.xy_empty[s], ((i >> 1) & 1) ^ 1, abort)) break;
        mbar_arrive_expect_tx(&B.xy_full[s], 2 * BT * 128);
        uint8_t* xs = sm + AXY_OFF + s * 32768;
        const int32_t tok = (int32_t)(t0 + (int64_t)i * BT);
        tma_load_3d(xs, mx, &B.xy_full[s], 0, h, tok);
        tma_load_3d(xs + 8192, mx, &B.xy_full[s], 0, h, tok + 64);
        tma_load_3d(xs + 16384, my, &B.xy_full[s], 0, h, tok);
        tma_load_3d(xs + 24576, my, &B.xy_full[s], 0, h, tok + 64);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // the G products of every quarter, as soon as a G buffer is free (the
    // whole warp runs the loop; one elected lane issues)
    const uint32_t wq = smem_u32(sm + AW_OFF);
    for (int n = 0; n < nq; ++n) {
      const int i = n / NQ, q = n % NQ, b = n & 1;
      if (q == 0 && !mbar_wait_spin_w(&B.xy_full[i & 1], (i >> 1) & 1, abort)) break;
      if (!mbar_wait_spin_w(&B.ga_free[b], ((n >> 1) & 1) ^ 1, abort)) break;
      tc_fence_after();
      const uint32_t xs = smem_u32(sm + AXY_OFF + (i & 1) * 32768);
      const uint32_t wb = wq + q * AQ_BYTES;
      const uint32_t gb = tb + A_BUF + b * A_GBUF;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        mma_ss_w(gb, sdesc_sw128(xs + ks * 32, 16, 1024), sdesc_sw128(wb + ks * 32, 16, 1024), IDESC_G1, ks > 0);
        mma_ss_w(gb + 64, sdesc_sw128(xs + 16384 + ks * 32, 16, 1024), sdesc_sw128(wb + 8192 + ks * 32, 16, 1024),
                 IDESC_G2, ks > 0);
      }
      mma_commit_w(&B.ga_full[b]);
    }
  } else if (warp == EPI0 + 8) {
    // dq products of every staged quarter (DQ); after a tile's last quarter,
    // its L products (A = the staged factors of all four quarters, hidden-unit
    // blocks of 32 at a stride of one staging tile).  The tile's G products
    // all completed before its last quarter was staged, so the commits after
    // the L products also cover every read of the tile's X/Y stage.  The
    // whole warp runs the loop; one elected lane issues.
    const uint32_t wq = smem_u32(sm + AW_OFF), stg = smem_u32(sm + AST_OFF);
    bool ok = true;
    for (int m = 0; m < nq && ok; ++m) {
      const int i = m / NQ, q = m % NQ;
      if (!mbar_wait_spin_w(&B.sq_full[q], i & 1, abort)) break;
      if (DQ && q == 0 && !mbar_wait_spin_w(&B.acc_free, (i & 1) ^ 1, abort)) break;
      tc_fence_after();
      if (DQ) {
        const uint32_t wb = wq + q * AQ_BYTES;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          mma_ss_w(tb + A_DX, sdesc_sw64(stg + ((ks / 2) * NQ + q) * ST_TILE + (ks % 2) * 32, 16, 512),
                   sdesc_sw128(wb + ks * 2048, 1024, 1024), IDESC_ACC, (q > 0 || ks > 0) ? 1u : 0u);
      }
      if (q == NQ - 1) {
        if (DQ) mma_commit_w(&B.acc_full);
        const uint32_t xs = smem_u32(sm + AXY_OFF + (i & 1) * 32768);
#pragma unroll
        for (int ks = 0; ks < BT / 16; ++ks) {
          const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
          const uint64_t xd = sdesc_sw128(xs + ks * 2048, 1024, 1024);
          const uint64_t yd = sdesc_sw128(xs + 16384 + ks * 2048, 1024, 1024);
          mma_ss_w(tb + B_L, sdesc_sw64(stg + 0 * NQ * ST_TILE + ks * 1024, ST_TILE, 512), xd, IDESC_LAM, acc);
          mma_ss_w(tb + B_L + 64, sdesc_sw64(stg + 1 * NQ * ST_TILE + ks * 1024, ST_TILE, 512), xd, IDESC_LAM, acc);
          mma_ss_w(tb + B_L + 128, sdesc_sw64(stg + 2 * NQ * ST_TILE + ks * 1024, ST_TILE, 512), yd, IDESC_LAM,
                   acc);
          // token rows [32g, 32g + 32) of the staging are read after K-step 2g + 1
          if (ks & 1) mma_commit_w(&B.st_free[ks >> 1]);
        }
        mma_commit_w(&B.xy_empty[i & 1]);    // its X/Y stage may be reloaded
      }
    }
    if (__all_sync(0xffffffffu, ok && !*abort)) mma_commit_w(&B.bdone);
  } else if (DQ && warp == 2) {
    // dq of every full tile by TMA store
    if (lane == 0) {
      for (int i = 0; i < ntiles; ++i) {
        if (!mbar_wait_spin(&B.out_full, i & 1, abort)) break;
        const int64_t tok = t0 + (int64_t)i * BT;
        if (tok + BT <= t1) {
          tma_store_3d(mdq, sm + ADQ_OFF, 0, h, (int32_t)tok);
          tma_store_3d(mdq, sm + ADQ_OFF + 8192, 0, h, (int32_t)(tok + 64));
          bulk_commit();
          bulk_wait_read_all();
        }
        mbar_arrive(&B.out_free);
      }
      bulk_wait_all();
    }
    __syncwarp();
  } else if (warp >= EPI0 && warp < EPI0 + 8) {
    // epilogue: thread = token row of the tile; half selects hidden units
    // [16*half, 16*half + 16) of every quarter.
    uint8_t* stg = sm + AST_OFF;
    float eta = 0.f, eta3 = 0.f, eta2 = 0.f;
    for (int n = 0; n < nq; ++n) {
      const int i = n / NQ, q = n % NQ, b = n & 1;
      const int64_t tok = t0 + (int64_t)i * BT + row;
      const bool valid = tok < t1;
      if (!DQ && q == 0) {
        if (PM) {
          eta = valid ? ld_chk(p.lr + ((size_t)tok * H + h) * 3) : 0.f;
          eta3 = valid ? ld_chk(p.lr + ((size_t)tok * H + h) * 3 + 1) : 0.f;
          eta2 = valid ? ld_chk(p.lr + ((size_t)tok * H + h) * 3 + 2) : 0.f;
        } else {
          eta = valid ? ld_chk(p.lr + (size_t)tok * H + h) : 0.f;
        }
      }
      if (!mbar_wait_spin(&B.ga_full[b], (n >> 1) & 1, abort)) break;
      tc_fence_after();
      const uint32_t buf = tb + lane_base + A_BUF + b * A_GBUF + 16 * half;
      float r[3][16];   // z1 z3 p
      tmem_ld16x3(buf, buf + 32, buf + 64, r[0], r[1], r[2]);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&B.ga_free[b]);
      uint32_t ob[3][8];   // A1 A3 A2 as bf16 pairs (hidden 2j, 2j + 1)
      {
        // the chain rule on pairs of hidden units (packed float32 lanes); the
        // scale is the learning rate (gradient) or the row's validity (dq)
        const f32x2 scale = x2(DQ ? (valid ? 1.f : 0.f) : eta), one = x2(1.f);
        const f32x2 scale3 = x2(eta3), scale2 = x2(eta2);   // PM: W3's and W2's rates
#pragma unroll
        for (int w = 0; w < 8; ++w) {
          const int k = 2 * w;
          const f32x2 z1 = x2(r[0][k], r[0][k + 1]), z3 = x2(r[1][k], r[1][k + 1]);
          const f32x2 sg = sigmoid2(z1);
          const f32x2 a = mul2(z1, sg);
          const f32x2 sp = fma2(a, sub2(one, sg), sg);
          const f32x2 pr = x2(r[2][k], r[2][k + 1]);
          const f32x2 pk = mul2(scale, pr);
          ob[0][w] = pack_bf16x2(mul2(mul2(pk, z3), sp));
          ob[1][w] = pack_bf16x2(mul2(PM ? mul2(scale3, pr) : pk, a));
          ob[2][w] = pack_bf16x2(mul2(PM ? scale2 : scale, mul2(a, z3)));
        }
      }
      // this thread's staging rows are free once the previous tile's L
      // products have read them
      if (q == 0 && !mbar_wait_spin(&B.st_free[warp & 3], (i & 1) ^ 1, abort)) break;
      {
        const uint32_t c = 16u * half;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          uint8_t* t = stg + (m * NQ + q) * ST_TILE;
          *reinterpret_cast<uint4*>(t + sw64_offset(row, c)) = make_uint4(ob[m][0], ob[m][1], ob[m][2], ob[m][3]);
          *reinterpret_cast<uint4*>(t + sw64_offset(row, c + 8)) =
              make_uint4(ob[m][4], ob[m][5], ob[m][6], ob[m][7]);
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      // one barrier per quarter slot: quarters of a tile do not wait for one
      // another, so a single barrier could run two phases ahead of its waiter
      if (lane == 0) mbar_arrive(&B.sq_full[q]);
      if (DQ && q == NQ - 1) {
        // tile finished: dq to shared memory for the TMA store (rows of a
        // partial tile are stored directly)
        if (!mbar_wait_spin(&B.acc_full, i & 1, abort)) break;
        tc_fence_after();
        const bool full_tile = (t0 + (int64_t)i * BT + BT) <= t1;
        if (full_tile && !mbar_wait_spin(&B.out_free, (i & 1) ^ 1, abort)) break;
        float v0[16], v1[16];
        tmem_ld16(tb + lane_base + A_DX + 32 * half, v0);
        tmem_ld16(tb + lane_base + A_DX + 32 * half + 16, v1);
        if (full_tile) {
          stage_row64(sm + ADQ_OFF, row, half, v0, v1);
        } else if (valid) {
          store_row64(reinterpret_cast<__nv_bfloat16*>(p.dq) + ((size_t)tok * H + h) * D, half, v0, v1);
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&B.acc_free);
          mbar_arrive(&B.out_full);
        }
      }
    }
    // the last L products complete before they are read
    mbar_wait_spin(&B.bdone, 0, abort);
  }
  tc_fence_before();
  const int stop = __syncthreads_or(*abort);
  tc_fence_after();
  if (stop || warp < EPI0 || warp >= EPI0 + 8) return;
  store_lambda<EPI0>(p, it, tb, sm + AW_OFF);   // weights and X/Y stages: no longer read
}

}  // namespace tl
}  // namespace scal3r
