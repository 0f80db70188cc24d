// BF16 tensor-core backward sweep of the test-time-training layer (sm_103a).
//
// One CTA = one work item (a token range of one chain at one backward step).
// BKEY items differentiate a chunk update (token tensors X = k, Y = v), BAPPLY
// items a chunk apply (X = q, Y = d_o).  Both form the per-(token, hidden
// unit) adjoints of the SwiGLU chain (reverse-mode differentiation of the
// forward step; dot loss) and contract them twice: over hidden units into the
// token gradients (dk and dv, or dq), and over tokens into the
// weight-adjoint partial sums L of the piece, which go to its partial slot.
// TMEM lane = token for the per-token products; hidden units are taken in
// quarters of 32.
//
// BKEY, per 128-token tile and quarter q:
//   G1 = X [W1_q; W3_q; -R1_q; -R3_q]^T    -> z1, z3, dg1, dg3   (N 128)
//   G2 = Y [W2^T_q; -R2^T_q]^T             -> W2^T v, -R2^T v    (N 64)
//   p = -lr W2^T v, g1 = p z3 s', g3 = p a, du = lr R2^T v,
//   dp = dg3 a + dg1 z3 s', da = dg3 p + du z3,
//   dz3 = dg1 p s' + du a,  dz1 = dg1 p z3 s'' + da s',
//   dlr -= W2^T v . dp - R2^T v . u   (summed over hidden units)
//   dk += [dz1 dz3 g1 g3] [W1_q; W3_q; -R1_q; -R3_q]      (K 128)
//   dv += [-lr dp, -lr u] [W2^T_q; -R2^T_q]               (K 64)
// The factors are staged as bf16 tiles [128 tokens][32 hidden] in the 64-byte
// swizzle (K-major A operands of dk/dv).  The six weight matrices take 96 KB
// of shared memory, so the four quarters of a tile cannot stay resident for
// the token-contracted products (M = 128 hidden units): dz1, dz3 and -lr dp
// are written to the piece's scratch by TMA tile stores, in 32-token groups
// [group][factor][quarter][32 tok][32 hidden], and a second pass reads one
// group per TMA load (the swizzle undone on the way out and redone on the
// way in), as MN-major A operands of
//   L1 += dz1^T X, L3 += dz3^T X, L2t += (-lr dp)^T Y   (M 128, N 64, K 16/step)
// The piece runs in sub-pieces of kBwdSubTiles tiles so that the scratch is
// read back from L2.  The second pass keeps six 32-token stages in flight,
// three of them over the weights, which are copied to the scratch once and
// copied back while the second pass finishes.
//
// BAPPLY needs only W1, W3, W2^T (48 KB), so the tile's factors of all four
// quarters stay in shared memory and every tile is finished in one pass
// (bf16_token_lane.cuh, shared with the forward's gradient pieces):
//   G1 = X [W1_q; W3_q]^T -> zq1, zq3,   G2 = Y [W2^T_q]^T -> du = W2^T d_o
//   dzq1 = du z3 s', dzq3 = du a, uq = a z3
//   dq += [dzq1 dzq3] [W1_q; W3_q]                          (K 64)
//   after the fourth quarter: L1 += dzq1^T X, L3 += dzq3^T X, L2t += uq^T Y
//
// dk/dv/dq are staged in shared memory and written by TMA tile stores.
// Warps: 0 TMA loads, 1 MMA issue, 2 bulk / TMA stores, 3..10 epilogue; in
// BAPPLY warp 11 issues the dq and L products (bf16_token_lane.cuh), in BKEY
// it idles.
#include <cudaTypedefs.h>

#include "bf16_token_lane.cuh"
#include "sm100.cuh"
#include "ttt_internal.h"

namespace scal3r {
namespace {

using namespace sm100;

using tl::BT;
using tl::D;
using tl::F;
using tl::NQ;
using tl::ST_TILE;
using tl::pack8;
using tl::stage_row64;
using tl::store_row64;
constexpr int NTHREADS = 384;
constexpr int EPI0 = 3;                      // first epilogue warp

// BKEY shared memory
constexpr uint32_t QBYTES = 24 * 1024;       // weights of one quarter: 192 rows x 128 B
constexpr uint32_t WQ_OFF = 0;               // 4 quarters, 96 KB
constexpr uint32_t XY_OFF = 96 * 1024;       // 2 stages x (X 16 KB + Y 16 KB); reused for dk/dv staging
constexpr uint32_t ST_OFF = 160 * 1024;      // six tiles: dz1 dz3 g1 g3 dpe ue (48 KB)
constexpr uint32_t ETA_OFF = 208 * 1024;     // half 1's dlr partials [2][3][128] float (one or three rates)
constexpr int PB_T = 32;                     // pass B tile (tokens)
constexpr uint32_t PB_STAGE = 32 * 1024;     // A1, A3, A2 (4 quarter blocks x 2 KB each), X 4 KB, Y 4 KB
constexpr int PB_STAGES = 6;
constexpr uint32_t PB_OFF = 0;               // pass B stages reuse the weights, token and staging regions
constexpr int PB_WQ_STAGES = 3;              // stages 0..2 lie over the weights
constexpr uint32_t WQ_BYTES = 4 * QBYTES;
constexpr uint32_t TILE_SCRATCH = 3 * 4 * ST_TILE;   // [factor][quarter][128 tok][32 hidden] bf16, 96 KB

constexpr size_t DYN_SMEM = 1024 + tl::SMEM_BYTES;   // the apply VJP's layout is the larger
static_assert(ETA_OFF + 2 * 3 * BT * 4 <= tl::SMEM_BYTES, "dlr partials inside the dynamic region");

// TMEM columns (BKEY)
constexpr uint32_t B_L = 0;         // L1 | L3 | L2t, 64 columns each, resident for the whole piece
constexpr uint32_t A_BUF = 192;     // G1 (128) | G2 (64)
constexpr uint32_t A_DX = 384;      // dk accumulator [tok][64]
constexpr uint32_t A_DY = 448;      // dv accumulator [tok][64]

struct TmaMaps {
  CUtensorMap x_k, y_v, x_q, y_do;           // loads, boxes of 64 x 1 x 64 tokens
  CUtensorMap x_k32, y_v32;                  // loads, boxes of 64 x 1 x 32 tokens (BKEY pass B)
  CUtensorMap sc_st, sc_ld;                  // BKEY scratch: one factor tile out, one 32-token group in
  CUtensorMap s_dk, s_dv, s_dq;              // stores, boxes of 64 x 1 x 64 tokens
};

struct Bars {   // BKEY
  uint64_t xy_full[2], xy_empty[2], g_full, g_free;
  uint64_t st_full, st_free, stg_done, acc_full, acc_free, out_full;
  uint64_t eta_full[2], eta_free[2];
  uint64_t b_full[PB_STAGES], b_empty[PB_STAGES], bdone, wq_full;
  uint32_t tmem_base;
  int abort_flag;
};

// BKEY weights, quarter-major:
//   quarter q rows   0.. 31 W1[32q + r][:]      rows  32.. 63 W3[32q + r][:]
//                   64.. 95 -R1[32q + r][:]     rows  96..127 -R3[32q + r][:]
//                  128..159 W2[:][32q + r]      rows 160..191 -R2[:][32q + r]
// each row 64 values (d).
__device__ void load_weights_key(const float* w, const float* r, uint8_t* sm) {
  tl::load_weight_chunks<true, 12, EPI0>(w, r, sm + WQ_OFF, QBYTES);
}

// ---------------------------------------------------------------------------
// BKEY: the VJP of a chunk update (two passes per sub-piece).  PM: one rate
// per matrix (lr [T, H, 3], dlr the same): every factor carries the rate of
// the matrix it came from (W1: dg1 and its products, W3: dg3 and g3, W2: the
// u terms), and dlr has three sums over the hidden units.
// ---------------------------------------------------------------------------
template <bool PM>
__device__ void run_key_vjp(const TmaMaps& maps, const Params& p, const WorkItem& it, uint8_t* sm, Bars& B,
                            uint32_t tb) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int H = p.H;
  const int h = it.chain % H;
  const int64_t t0 = it.t0, t1 = it.t1;
  const int ntiles = (int)((t1 - t0 + BT - 1) / BT);
  const int nsub = (ntiles + kBwdSubTiles - 1) / kBwdSubTiles;
  // The pieces of a launch start together and have equal sub-pieces, so
  // their second passes (the L2-heavy phase) would coincide.  The slack of
  // the last sub-piece (nsub * kBwdSubTiles - ntiles tiles) is taken off the
  // first one by a CTA-dependent amount instead, which staggers the phases
  // without adding a sub-piece.
  const int slack = nsub * kBwdSubTiles - ntiles;
  const int lead = slack > 0 ? (int)(blockIdx.x % (unsigned)(slack + 1)) : 0;
  // the piece's scratch: kBwdSubTiles tiles of factor groups, then the weights
  const int32_t g0 = 4 * it.aux;   // first 32-token group of the piece
  uint8_t* wq_image = reinterpret_cast<uint8_t*>(p.scratch) + (size_t)(it.aux + kBwdSubTiles) * TILE_SCRATCH;
  volatile int* abort = &B.abort_flag;
  constexpr int KDX = 8;    // K-steps of the dk product (16 hidden units each)
  constexpr uint32_t IDESC_G1 = idesc_bf16(128, 128, false, false);
  constexpr uint32_t IDESC_G2 = idesc_bf16(128, 64, false, false);
  constexpr uint32_t IDESC_ACC = idesc_bf16(128, D, false, true);
  constexpr uint32_t IDESC_LAM = idesc_bf16(128, D, true, true);
  const int ew = warp - EPI0, half = ew >> 2;            // epilogue warps only
  const uint32_t row = 32u * (warp & 3) + lane;
  const uint32_t lane_base = (32u * (warp & 3)) << 16;
  // learning rate(s) of this thread's token, one tile ahead
  constexpr int NR = PM ? 3 : 1;
  float eta_next[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j)
    eta_next[j] = (warp >= EPI0 && warp < EPI0 + 8 && t0 + (int64_t)row < t1)
                      ? ld_chk(p.lr + ((size_t)(t0 + row) * H + h) * NR + j) : 0.f;

  // pass B stage use counts (parity per stage), kept alike by the producer
  // and the MMA thread
  uint32_t pb_uses = 0;
  bool aborted = false;
  for (int sp = 0; sp < nsub; ++sp) {
    const int ta = sp == 0 ? 0 : sp * kBwdSubTiles - lead;
    const int te = min(ntiles, (sp + 1) * kBwdSubTiles - lead);
    // ======================= pass A on tiles [ta, te) =======================
    if (warp == 0) {
      if (lane == 0) {
        for (int i = ta; i < te; ++i) {
          const int s = i & 1;
          if (!mbar_wait(&B.xy_empty[s], ((i >> 1) & 1) ^ 1, abort)) break;
          mbar_arrive_expect_tx(&B.xy_full[s], 2 * BT * 128);
          uint8_t* xs = sm + XY_OFF + s * 32768;
          const int32_t tok = (int32_t)(t0 + (int64_t)i * BT);
          tma_load_3d(xs, &maps.x_k, &B.xy_full[s], 0, h, tok);
          tma_load_3d(xs + 8192, &maps.x_k, &B.xy_full[s], 0, h, tok + 64);
          tma_load_3d(xs + 16384, &maps.y_v, &B.xy_full[s], 0, h, tok);
          tma_load_3d(xs + 24576, &maps.y_v, &B.xy_full[s], 0, h, tok + 64);
        }
      }
      __syncwarp();
    } else if (warp == 1) {
      // the whole warp runs the issue loop (uniform control flow); one
      // elected lane issues each MMA and commit
      // descriptor halves: the loops add constant offsets to these bases
      const uint32_t stg_lo = sdesc_lo(smem_u32(sm + ST_OFF), 16);      // staged factors, 64-byte swizzle
      const uint32_t wq_lo16 = sdesc_lo(smem_u32(sm + WQ_OFF), 16);     // weights as B of G (K-major)
      const uint32_t wq_lo1k = sdesc_lo(smem_u32(sm + WQ_OFF), 1024);   // weights as B of dk/dv (MN-major)
      const uint32_t xy_lo = sdesc_lo(smem_u32(sm + XY_OFF), 16);
      constexpr uint32_t HI128 = sdesc_hi(1024, kSwizzle128), HI64 = sdesc_hi(512, kSwizzle64);
      auto issue_acc = [&](int m) -> bool {
        const int i = m / NQ, q = m % NQ;
        if (!mbar_wait_nap_w(&B.st_full, m & 1, abort)) return false;
        if (q == 0 && !mbar_wait_nap_w(&B.acc_free, (i & 1) ^ 1, abort)) return false;
        tc_fence_after();
        const uint32_t wb = wq_lo1k + q * (QBYTES >> 4);
        const uint32_t acc0 = q > 0 ? 1u : 0u;
#pragma unroll
        for (int ks = 0; ks < KDX; ++ks)
          mma_ss_h(tb + A_DX, stg_lo + (((ks / 2) * ST_TILE + (ks % 2) * 32) >> 4), HI64, wb + ((ks * 2048) >> 4),
                   HI128, IDESC_ACC, ks > 0 ? 1u : acc0);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          mma_ss_h(tb + A_DY, stg_lo + (((4 + ks / 2) * ST_TILE + (ks % 2) * 32) >> 4), HI64,
                   wb + ((16384 + ks * 2048) >> 4), HI128, IDESC_ACC, ks > 0 ? 1u : acc0);
        mma_commit_w(&B.st_free);
        if (q == NQ - 1) mma_commit_w(&B.acc_full);
        return true;
      };
      bool ok = true;
      // pass B of the previous sub-piece overwrote the weights
      if (sp > 0 && !mbar_wait_nap_w(&B.wq_full, (sp - 1) & 1, abort)) ok = false;
      for (int n = ta * NQ; n < te * NQ && ok; ++n) {
        const int i = n / NQ, q = n % NQ;
        if (q == 0 && !mbar_wait_nap_w(&B.xy_full[i & 1], (i >> 1) & 1, abort)) break;
        if (!mbar_wait_nap_w(&B.g_free, (n & 1) ^ 1, abort)) break;
        tc_fence_after();
        const uint32_t xs = xy_lo + (i & 1) * (32768 >> 4);
        const uint32_t wb = wq_lo16 + q * (QBYTES >> 4);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          mma_ss_h(tb + A_BUF, xs + ks * 2, HI128, wb + ks * 2, HI128, IDESC_G1, ks > 0);
          mma_ss_h(tb + A_BUF + 128, xs + ((16384 >> 4) + ks * 2), HI128, wb + ((16384 >> 4) + ks * 2), HI128,
                   IDESC_G2, ks > 0);
        }
        mma_commit_w(&B.g_full);
        if (n > ta * NQ) ok = issue_acc(n - 1);
      }
      if (__all_sync(0xffffffffu, ok && !*abort)) issue_acc(te * NQ - 1);
    } else if (warp == 2) {
      // stores: the weights (once), the scratch factors of every quarter,
      // dk/dv of every tile
      if (lane == 0) {
        if (sp == 0 && nsub > 1) {
          bulk_store(wq_image, sm + WQ_OFF, WQ_BYTES);
          bulk_commit();
        }
        // dk / dv of tile i, staged over the tile's X/Y stage by the epilogue
        // (after the next tile's first quarter, see there)
        auto store_dkdv = [&](int i) -> bool {
          if (!mbar_wait(&B.out_full, i & 1, abort)) return false;
          const int64_t tok = t0 + (int64_t)i * BT;
          if (tok + BT <= t1) {
            uint8_t* xs = sm + XY_OFF + (i & 1) * 32768;
            tma_store_3d(&maps.s_dk, xs, 0, h, (int32_t)tok);
            tma_store_3d(&maps.s_dk, xs + 8192, 0, h, (int32_t)(tok + 64));
            tma_store_3d(&maps.s_dv, xs + 16384, 0, h, (int32_t)tok);
            tma_store_3d(&maps.s_dv, xs + 24576, 0, h, (int32_t)(tok + 64));
            bulk_commit();
            bulk_wait_read_all();
          }
          mbar_arrive(&B.xy_empty[i & 1]);
          return true;
        };
        bool ok = true;
        for (int n = ta * NQ; n < te * NQ && ok; ++n) {
          const int i = n / NQ, q = n % NQ;
          if (!mbar_wait(&B.st_full, n & 1, abort)) break;
          const int32_t g = g0 + 4 * (i - ta);
          tma_store_5d(&maps.sc_st, sm + ST_OFF + 0 * ST_TILE, 0, 0, q, 0, g);   // dz1
          tma_store_5d(&maps.sc_st, sm + ST_OFF + 1 * ST_TILE, 0, 0, q, 1, g);   // dz3
          tma_store_5d(&maps.sc_st, sm + ST_OFF + 4 * ST_TILE, 0, 0, q, 2, g);   // -lr dp
          bulk_commit();
          bulk_wait_read_all();
          mbar_arrive(&B.stg_done);
          if (q == 0 && i > ta) ok = store_dkdv(i - 1);
        }
        if (ok && !*abort) store_dkdv(te - 1);
        bulk_wait_all();   // scratch written before pass B reads it back
      }
      __syncwarp();
    } else if (warp < EPI0 + 8) {
      // epilogue: thread = token row of the tile; half selects hidden units
      // [16*half, 16*half + 16) of every quarter.
      uint8_t* stg = sm + ST_OFF;
      float eta[NR], deta[NR], dprev[NR];
#pragma unroll
      for (int j = 0; j < NR; ++j) eta[j] = deta[j] = dprev[j] = 0.f;
      // Tile i finished: dk and dv out of TMEM into the tile's X/Y stage for
      // the TMA store (rows of a partial tile are stored directly), and the
      // dlr halves (dprev) combined.  Run after the next tile's first quarter
      // is staged, so that the wait for the last products overlaps that
      // quarter's chain rule instead of stalling the epilogue.
      auto finish_tile = [&](int i) -> bool {
        const int64_t tok = t0 + (int64_t)i * BT + row;
        const bool valid = tok < t1;
        if (!mbar_wait_spin(&B.acc_full, i & 1, abort)) return false;
        tc_fence_after();
        const bool full_tile = (t0 + (int64_t)i * BT + BT) <= t1;
        uint8_t* xs = sm + XY_OFF + (i & 1) * 32768;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          float v0[16], v1[16];
          tmem_ld16(tb + lane_base + (m ? A_DY : A_DX) + 32 * half, v0);
          tmem_ld16(tb + lane_base + (m ? A_DY : A_DX) + 32 * half + 16, v1);
          if (full_tile) {
            stage_row64(xs + m * 16384, row, half, v0, v1);
          } else if (valid) {
            store_row64(reinterpret_cast<__nv_bfloat16*>(m ? p.dv : p.dk) + ((size_t)tok * H + h) * D, half, v0,
                        v1);
          }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&B.acc_free);
          mbar_arrive(&B.out_full);
        }
        // dlr of the token = sum of the two halves' partials (half 1 hands
        // its partial to half 0 through shared memory)
        const int e = i & 1;
        float* eta_red = reinterpret_cast<float*>(sm + ETA_OFF) + e * 3 * BT;
        if (half == 1) {
          if (!mbar_wait_spin(&B.eta_free[e], ((i >> 1) & 1) ^ 1, abort)) return false;
#pragma unroll
          for (int j = 0; j < NR; ++j) eta_red[j * BT + row] = dprev[j];
          __syncwarp();
          if (lane == 0) mbar_arrive(&B.eta_full[e]);
        } else {
          if (!mbar_wait_spin(&B.eta_full[e], (i >> 1) & 1, abort)) return false;
          if (valid) {
#pragma unroll
            for (int j = 0; j < NR; ++j) st_chk(p.dlr + ((size_t)tok * H + h) * NR + j, dprev[j] + eta_red[j * BT + row]);
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&B.eta_free[e]);
        }
        return true;
      };
      bool ok = true;
      for (int n = ta * NQ; n < te * NQ && ok; ++n) {
        const int i = n / NQ, q = n % NQ;
        const int64_t tok = t0 + (int64_t)i * BT + row;
        if (q == 0) {
          const int64_t tn = tok + BT;
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            dprev[j] = deta[j];
            eta[j] = eta_next[j];
            deta[j] = 0.f;
            eta_next[j] = (i + 1 < ntiles && tn < t1) ? ld_chk(p.lr + ((size_t)tn * H + h) * NR + j) : 0.f;
          }
        }
        if (!mbar_wait_spin(&B.g_full, n & 1, abort)) break;
        tc_fence_after();
        const uint32_t buf = tb + lane_base + A_BUF;
        uint32_t ob[6][8];   // dz1 dz3 g1 g3 dpe ue as bf16 pairs (hidden 2j, 2j + 1)
        float r[2][6][8];
#pragma unroll
        for (int sb = 0; sb < 2; ++sb) {
          const uint32_t c = 16 * half + 8 * sb;
          tmem_ld8x6(buf + c, buf + 32 + c, buf + 64 + c, buf + 96 + c, buf + 128 + c, buf + 160 + c, r[sb]);
        }
        // the quarter's GEMM results are in registers: release the buffer
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.g_free);
        {
          // the chain rule on pairs of hidden units (packed float32 lanes)
          // rates of W1, W3, W2 (all the token's one rate without PM)
          const f32x2 neta = x2(-eta[0]), neta3 = x2(-eta[PM ? 1 : 0]), neta2 = x2(-eta[PM ? 2 : 0]);
          const f32x2 one = x2(1.f), two = x2(2.f), mtwo = x2(-2.f);
          f32x2 dsum = x2(0.f), dsum3 = x2(0.f), dsum2 = x2(0.f);
#pragma unroll
          for (int sb = 0; sb < 2; ++sb) {
#pragma unroll
            for (int jp = 0; jp < 4; ++jp) {
              const int j = 2 * jp;
              const f32x2 z1 = x2(r[sb][0][j], r[sb][0][j + 1]), z3 = x2(r[sb][1][j], r[sb][1][j + 1]);
              const f32x2 dg1 = x2(r[sb][2][j], r[sb][2][j + 1]), dg3 = x2(r[sb][3][j], r[sb][3][j + 1]);
              const f32x2 praw = x2(r[sb][4][j], r[sb][4][j + 1]), ndu = x2(r[sb][5][j], r[sb][5][j + 1]);
              const f32x2 sg = sigmoid2(z1);
              const f32x2 a = mul2(z1, sg);
              const f32x2 oms = sub2(one, sg);
              const f32x2 sp = fma2(a, oms, sg);                                  // silu'(z1)
              const f32x2 spp = mul2(mul2(sg, oms), fma2(z1, fma2(mtwo, sg, one), two));   // silu''(z1)
              const f32x2 u = mul2(a, z3);
              const f32x2 pp = mul2(neta, praw);
              const f32x2 du = mul2(neta2, ndu);
              const f32x2 z3sp = mul2(z3, sp);
              const int w = 4 * sb + jp;
              if (!PM) {
                const f32x2 dp = fma2(dg3, a, mul2(dg1, z3sp));
                const f32x2 da = fma2(dg3, pp, mul2(du, z3));
                const f32x2 gp = mul2(dg1, pp);
                ob[1][w] = pack_bf16x2(fma2(gp, sp, mul2(du, a)));                  // dz3
                ob[0][w] = pack_bf16x2(fma2(mul2(gp, z3), spp, mul2(da, sp)));      // dz1
                ob[2][w] = pack_bf16x2(mul2(pp, z3sp));                            // g1
                ob[3][w] = pack_bf16x2(mul2(pp, a));                               // g3
                ob[4][w] = pack_bf16x2(mul2(neta, dp));                            // -lr dp
                ob[5][w] = pack_bf16x2(mul2(neta, u));                             // -lr u
                dsum = fma2(praw, dp, fma2(ndu, u, dsum));
              } else {
                // W1's terms with its rate, W3's with its rate, u's with W2's
                const f32x2 pp3 = mul2(neta3, praw);
                const f32x2 dg1z = mul2(dg1, z3sp), dg3a = mul2(dg3, a);
                const f32x2 da = fma2(dg3, pp3, mul2(du, z3));
                const f32x2 gp = mul2(dg1, pp);
                ob[1][w] = pack_bf16x2(fma2(gp, sp, mul2(du, a)));                  // dz3
                ob[0][w] = pack_bf16x2(fma2(mul2(gp, z3), spp, mul2(da, sp)));      // dz1
                ob[2][w] = pack_bf16x2(mul2(pp, z3sp));                            // g1
                ob[3][w] = pack_bf16x2(mul2(pp3, a));                              // g3
                ob[4][w] = pack_bf16x2(fma2(neta, dg1z, mul2(neta3, dg3a)));      // -(e1 dg1 z3 s' + e3 dg3 a)
                ob[5][w] = pack_bf16x2(mul2(neta2, u));                            // -e2 u
                dsum = fma2(praw, dg1z, dsum);
                dsum3 = fma2(praw, dg3a, dsum3);
                dsum2 = fma2(ndu, u, dsum2);
              }
            }
          }
          deta[0] -= x2_lo(dsum) + x2_hi(dsum);
          if (PM) {
            deta[1] -= x2_lo(dsum3) + x2_hi(dsum3);
            deta[2] -= x2_lo(dsum2) + x2_hi(dsum2);
          }
        }
        // staging of the quarter: free once the previous quarter's products
        // and its scratch copy have read it
        if (!mbar_wait_spin(&B.st_free, (n & 1) ^ 1, abort)) break;
        if (!mbar_wait_spin(&B.stg_done, (n & 1) ^ 1, abort)) break;
        {
          const uint32_t c = 16u * half;
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            uint8_t* t = stg + m * ST_TILE;
            *reinterpret_cast<uint4*>(t + sw64_offset(row, c)) = make_uint4(ob[m][0], ob[m][1], ob[m][2], ob[m][3]);
            *reinterpret_cast<uint4*>(t + sw64_offset(row, c + 8)) =
                make_uint4(ob[m][4], ob[m][5], ob[m][6], ob[m][7]);
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.st_full);
        if (q == 0 && i > ta) ok = finish_tile(i - 1);
      }
      if (ok && !*abort) {
#pragma unroll
        for (int j = 0; j < NR; ++j) dprev[j] = deta[j];
        finish_tile(te - 1);
      }
    }
    // pass A of the sub-piece done: its MMAs completed (the epilogue waited for
    // the last tile's accumulators) and its scratch copies are complete (the
    // store warp waited for them).  Every thread takes the same abort decision.
    tc_fence_before();
    const int stop_a = __syncthreads_or(*abort);
    tc_fence_after();
    if (stop_a) {
      aborted = true;
      break;
    }

    // ======================= pass B on 32-token tiles of [ta, te) =======================
    // Tile j (0..nb-1) of the sub-piece uses stage (j + rot) % PB_STAGES, so
    // that the last three tiles use the stages off the weights: the weights
    // of the next sub-piece are copied back while those finish.
    const int jb0 = ta * (BT / PB_T), nb = (te - ta) * (BT / PB_T);
    const int rot = (PB_STAGES - nb % PB_STAGES) % PB_STAGES;
    if (warp == 0) {
      if (lane == 0) {
        bool ok = true;
        for (int j = 0; j < nb; ++j) {
          const int s = (j + rot) % PB_STAGES;
          if (!mbar_wait(&B.b_empty[s], ((pb_uses >> s) & 1) ^ 1, abort)) {
            ok = false;
            break;
          }
          pb_uses ^= 1u << s;
          mbar_arrive_expect_tx(&B.b_full[s], PB_STAGE);
          uint8_t* st = sm + PB_OFF + s * PB_STAGE;
          tma_load_5d(st, &maps.sc_ld, &B.b_full[s], 0, 0, 0, 0, g0 + j);
          const int32_t tok = (int32_t)(t0 + (int64_t)(jb0 + j) * PB_T);
          tma_load_3d(st + 24576, &maps.x_k32, &B.b_full[s], 0, h, tok);
          tma_load_3d(st + 28672, &maps.y_v32, &B.b_full[s], 0, h, tok);
        }
        if (ok && sp + 1 < nsub) {
          // the stages over the weights are read: copy the weights back
          for (int s = 0; s < PB_WQ_STAGES && ok; ++s)
            ok = mbar_wait(&B.b_empty[s], ((pb_uses >> s) & 1) ^ 1, abort);
          if (ok) {
            mbar_arrive_expect_tx(&B.wq_full, WQ_BYTES);
            bulk_load(sm + WQ_OFF, wq_image, WQ_BYTES, &B.wq_full);
          }
        }
      }
      __syncwarp();
    } else if (warp == 1) {
      bool ok = true;
      const uint32_t pb_a = sdesc_lo(smem_u32(sm + PB_OFF), 2048);   // factors, MN-major, 64-byte swizzle
      const uint32_t pb_b = sdesc_lo(smem_u32(sm + PB_OFF), 1024);   // X / Y, MN-major, 128-byte swizzle
      constexpr uint32_t HI128 = sdesc_hi(1024, kSwizzle128), HI64 = sdesc_hi(512, kSwizzle64);
      for (int j = 0; j < nb; ++j) {
        const int s = (j + rot) % PB_STAGES;
        if (!mbar_wait_spin_w(&B.b_full[s], (pb_uses >> s) & 1, abort)) {
          ok = false;
          break;
        }
        pb_uses ^= 1u << s;
        tc_fence_after();
        const uint32_t a = pb_a + s * (PB_STAGE >> 4), b = pb_b + s * (PB_STAGE >> 4);
        const uint32_t acc0 = jb0 + j > 0 ? 1u : 0u;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint32_t acc = ks > 0 ? 1u : acc0;
          const uint32_t xd = b + ((24576 + ks * 2048) >> 4), yd = b + ((28672 + ks * 2048) >> 4);
          mma_ss_h(tb + B_L, a + ((ks * 1024) >> 4), HI64, xd, HI128, IDESC_LAM, acc);
          mma_ss_h(tb + B_L + 64, a + ((8192 + ks * 1024) >> 4), HI64, xd, HI128, IDESC_LAM, acc);
          mma_ss_h(tb + B_L + 128, a + ((16384 + ks * 1024) >> 4), HI64, yd, HI128, IDESC_LAM, acc);
        }
        mma_commit_w(&B.b_empty[s]);
      }
      if (ok) mma_commit_w(&B.bdone);
    }
    // everyone waits for the sub-piece's weight-adjoint products before the
    // next pass A reuses their shared memory
    mbar_wait_spin(&B.bdone, sp & 1, abort);
    tc_fence_before();
    const int stop_b = __syncthreads_or(*abort);
    tc_fence_after();
    if (stop_b) {
      aborted = true;
      break;
    }
  }
  if (warp == 2 && lane == 0) bulk_wait_all();   // dk/dv stores complete
  if (aborted || warp < EPI0 || warp >= EPI0 + 8) return;
  tl::store_lambda<EPI0>(p, it, tb, sm + PB_OFF);   // the pass B stages: all read
}

__global__ void __launch_bounds__(NTHREADS, 1)
bf16_bsweep_kernel(const __grid_constant__ TmaMaps maps, const Params p, const WorkItem* __restrict__ items) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  __shared__ Bars B;
  __shared__ tl::Bars TB;
  const int warp = threadIdx.x / 32;
  const WorkItem it = items[blockIdx.x];
  const int H = p.H, P = 3 * F * D;
  const int h = it.chain % H, s = it.chain / H;
  const bool key = (it.role == ROLE_BKEY);
  const float* w = (it.wchunk >= 0) ? p.w_ckpt_in + ((size_t)it.wchunk * H + h) * P
                                    : p.w0 + (size_t)s * p.w0_seq_stride + (size_t)h * P;
  const float* r = p.rbuf + (size_t)it.chain * P;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&B.xy_full[i], 1);
      mbar_init(&B.xy_empty[i], 1);
      mbar_init(&B.eta_full[i], 4);
      mbar_init(&B.eta_free[i], 4);
    }
    mbar_init(&B.g_full, 1);
    mbar_init(&B.g_free, 8);
    mbar_init(&B.st_full, 8);
    mbar_init(&B.st_free, 1);
    mbar_init(&B.stg_done, 1);
    mbar_init(&B.acc_full, 1);
    mbar_init(&B.acc_free, 8);
    mbar_init(&B.out_full, 8);
    for (int i = 0; i < PB_STAGES; ++i) {
      mbar_init(&B.b_full[i], 1);
      mbar_init(&B.b_empty[i], 1);
    }
    mbar_init(&B.bdone, 1);
    mbar_init(&B.wq_full, 1);
    B.abort_flag = 0;
    tl::init_bars(TB);
    fence_barrier_init();
    prefetch_tmap(key ? &maps.x_k : &maps.x_q);
    prefetch_tmap(key ? &maps.y_v : &maps.y_do);
  }
  if (warp == 1) {
    tmem_alloc(&B.tmem_base, 512);
    tmem_relinquish();
  }
  // the weights and the adjoint R come from the kernels ahead of this one
  pdl_wait();
  if (warp >= EPI0 && warp < EPI0 + 8) {
    if (key) load_weights_key(w, r, sm);
    else tl::load_weights<EPI0>(w, sm);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = B.tmem_base;
  if (key) {
    if (p.lr_mat) run_key_vjp<true>(maps, p, it, sm, B, tb);
    else run_key_vjp<false>(maps, p, it, sm, B, tb);
  }
  else tl::token_lane_pass<true, EPI0>(&maps.x_q, &maps.y_do, &maps.s_dq, p, it, sm, TB, tb);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((B.abort_flag || TB.abort_flag) && threadIdx.x == 0) atomicExch(p.status, SCAL3R_ERR_TIMEOUT);
  if (warp == 1) tmem_dealloc(tb, 512);
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

// The BKEY scratch as a 5-D bf16 tensor [group][factor 3][quarter 4][32 tok][32 hidden]
// (64-byte swizzle on the shared-memory side).
bool make_scratch_map(CUtensorMap* m, void* base, int64_t groups, const cuuint32_t (&box)[5]) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[5] = {32, 32, 4, 3, (cuuint64_t)groups};
  cuuint64_t strides[4] = {64, 2048, 8192, 24576};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, const_cast<cuuint32_t*>(box), es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_map(CUtensorMap* m, const void* base, int64_t T, int H, int box_tokens) {
  auto fn = encode_fn();
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

size_t bf16_bwd_scratch_tile_bytes() { return TILE_SCRATCH; }

cudaError_t prepare_bf16_backward() {
  return cudaFuncSetAttribute(bf16_bsweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DYN_SMEM);
}

cudaError_t launch_bf16_bsweep(const Params& prm, const WorkItem* items, int n, int step, const void*,
                               cudaStream_t st) {
  (void)step;
  if (n == 0) return cudaSuccess;
  if (prm.T <= 0 || !prm.scratch || prm.scratch_tiles <= 0) return cudaErrorInvalidValue;
  TmaMaps maps;
  const cuuint32_t box_st[5] = {32, 32, 1, 1, 4}, box_ld[5] = {32, 32, 4, 3, 1};
  if (!make_scratch_map(&maps.sc_st, prm.scratch, 4 * prm.scratch_tiles, box_st) ||
      !make_scratch_map(&maps.sc_ld, prm.scratch, 4 * prm.scratch_tiles, box_ld))
    return cudaErrorInvalidValue;
  if (!make_map(&maps.x_k, prm.k, prm.T, prm.H, 64) || !make_map(&maps.y_v, prm.v, prm.T, prm.H, 64) ||
      !make_map(&maps.x_q, prm.q, prm.T, prm.H, 64) || !make_map(&maps.y_do, prm.d_o, prm.T, prm.H, 64) ||
      !make_map(&maps.x_k32, prm.k, prm.T, prm.H, PB_T) || !make_map(&maps.y_v32, prm.v, prm.T, prm.H, PB_T) ||
      !make_map(&maps.s_dk, prm.dk, prm.T, prm.H, 64) || !make_map(&maps.s_dv, prm.dv, prm.T, prm.H, 64) ||
      !make_map(&maps.s_dq, prm.dq, prm.T, prm.H, 64))
    return cudaErrorInvalidValue;
  return launch_pdl(bf16_bsweep_kernel, dim3(n), dim3(NTHREADS), DYN_SMEM, st, maps, prm, items);
}

#ifdef SCAL3R_DEBUG_BOUNDS
cudaError_t bf16_bwd_upload_bounds(const BoundsTable& t, cudaStream_t st) { return upload_bounds_table(t, st); }
#endif

}  // namespace scal3r
