// BF16 tensor-core path for wide fast weights: the paper's own AMU shape
// (one head, hd = 1024, hidden = k * hd, Supp. "Global Context Memory module")
// and any head_dim and hidden that are multiples of 256 (up to 4096).
//
// At these sizes a chain's fast weights (3 * F * D values, 50 MB in float32 at
// D = 1024, F = 4096) do not fit on chip, and every product of the chunk step
// is a large GEMM.  One chunk step (Eq. 8, dot loss Eq. 9, then Eq. 4) of
// chain (s, h), tokens of the chunk t in [t0, t1), M = t1 - t0, is
//   P  = V W2                        [M x F]   (p = W2^T e, e = -v)
//   Z1 = K W1^T, Z3 = K W3^T         [M x F]   -> per (t, f): a = z1 sigmoid(z1),
//        g1 = -eta1 P z3 s'(z1), g3 = -eta3 P a, u~ = -eta2 a z3   (epilogue, bf16 out)
//   G1 = g1^T K, G3 = g3^T K         [F x D],  G2 = V^T u~   [D x F]
//   W <- W - G, rows rescaled (row norm targets of W0)       (wide_update_kernel)
//   O  = (silu(Q W1^T) o (Q W3^T)) W2^T                      (two GEMMs)
// with one learning rate per token (eta1 = eta3 = eta2) or one per matrix.
// The squared-error loss (key_grad_mse), the backward through the chunk
// loop (wide_backward, update_vjp_mse), the Global Context Synchronisation
// pieces (wide_partial_grad, wide_apply_update, wide_apply) and the plain
// GEMM of the C ABI (wide_gemm_bf16) are built from the same GEMM kernel.
//
// All GEMMs run on one persistent tcgen05 kernel: 128 x 256 output tiles, K
// in steps of 64 through a four-stage TMA pipeline (128-byte swizzle, either
// operand K- or MN-major), one elected thread of a converged warp issuing
// M128 N256 K16 MMAs into two 256-column TMEM accumulators in turn, and two
// groups of four epilogue warps (TMEM lane = output row), one per accumulator.
// The gate GEMMs read W1 and W3 rows (and -R1, -R3 in the backward) of the same
// hidden units into one N = 256 operand, so one tile holds every half of the
// gate.  Epilogues store 32 bytes per thread and row.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <vector>

#include "sm100.cuh"
#include "bounds.cuh"
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

enum Epi : int {
  EPI_F32 = 0,      // out[0] = acc (float32)
  EPI_BF16 = 1,     // out[0] = acc (bf16)
  EPI_KEY = 2,      // forward gradient gate: z1 | z3 of 128 hidden, in0 = P -> g1, g3, u~ (dot loss)
  EPI_APPLY = 3,    // forward apply gate: z1 | z3 -> h
  EPI_F32_ADD = 4,  // out[0] += acc (float32)
  EPI_BAPPLY = 5,   // apply VJP gate: zq1 | zq3 of 128 hidden, in0 = W2^T d_o -> dzq1, dzq3, uq
  EPI_BKEY = 6,     // update VJP gate: z1 | z3 | dg1 | dg3 of 64 hidden, in0 = W2^T v, in1 = -R2^T v
                    //   -> dz1, dz3, g1, g3, -dp, -eta2 u and partials of d eta
  // the squared-error loss; e = W2 u - v without a rate, p = W2^T e:
  EPI_MSE_E = 7,    // acc = W2 u;  in0 = v  -> e = acc - v, and eta2 e if out[1]
  EPI_ADD_BF16 = 8, // out[0] = acc + in0, or acc + eta2 in0 when eta is given
  EPI_MSE_DE = 9,   // acc = dL/de -> out[0] = acc, out[1] = -acc (its own stride)
  EPI_BKEY_MSE1 = 10,  // update VJP gate, pass 1: in0 = p, in1 = -R2^T e -> dp, g1, g3, partials of d eta
  EPI_BKEY_MSE2 = 11,  // update VJP gate, pass 2: in0 = p, in1 = du -> dz1, dz3
  EPI_APPLY2 = 12,  // gate z1 | z3 -> u and eta2 u
  // the GCM module's projections (scal3r_gcm.h):
  EPI_GCM_QKV = 13,   // acc + colvec (bias) -> bf16 into out[0] | out[1] | out[2] (q | k | v, row stride
                      //   ld_out = d); q and k: sum of squares of every 64 columns into out[3] (ld_part)
  EPI_GCM_GATE = 14,  // out[0] = colvec o acc + in0 (alpha o y + x), out[1] = acc; both bf16
  EPI_F32_ADDIN = 15, // out[0] = acc + in0 (float32 out, bf16 in0)
};

struct GemmArgs {
  CUtensorMap a[4], b[4];  // operand maps: K segment s reads a[s] / b[s]; N block j of the B tile reads b[j]
  int M, N, K;             // output rows, output columns (N = 256 * tiles), reduction length
  int kseg, nseg;          // nseg > 1: K is nseg segments of kseg (a multiple of 64)
  int nbn;                 // > 1: the B tile is nbn blocks of 256 / nbn rows (K-major, one segment)
  int a_mn, b_mn;          // operand major-ness
  int ha, hb;              // coordinate 1 of the A / B maps (the head of a [T, H, D] tensor)
  int ya, yb;              // row offset added to the A / B map's row coordinate
  int epi;
  void* out[6];            // outputs (see Epi); token-major [M x ...] with row stride ld_out
  int64_t ld_out;
  const __nv_bfloat16* in0;  // epilogue inputs [M x F], row stride ld_out
  const __nv_bfloat16* in1;
  const float* eta;        // learning rates of output row m: eta[m * eta_stride + j * eta_mat] for
  int64_t eta_stride;      //   W1, W3, W2 (j = 0, 1, 2); eta_mat = 0: one rate shared by all three
  int eta_mat;
  float* part;             // d eta partials of row m, tile column tn: part[m * ld_part + tn] (shared rate:
                           //   the sum), or part[m * ld_part + 3 tn + j] for matrix j
  int64_t ld_part;
  int* status;
  int mse;                 // EPI_KEY: the squared-error loss (in0 = W2^T e; no u~ output)
  int64_t ld_in;           // row stride of in0 / in1 when not ld_out (0: ld_out)
  int64_t ld_out1;         // row stride of out[1] when not ld_out (0: ld_out)
  int timeout_test;        // nonzero: after the last tile the epilogue warps wait, for at most
                           //   50 ms, on a barrier that nothing completes (the bounded-wait test)
  int ksplit;              // > 1: K is cut into ksplit ranges of kb_split K blocks; range s of a tile
  int kb_split;            //   writes (EPI_F32) the partial plane out[0] + s * split_stride
  int64_t split_stride;
  const float* colvec;     // EPI_GCM_QKV: the bias of output column n; EPI_GCM_GATE: its gate alpha
};

__device__ __forceinline__ float silu_d(float z, float& sg) {
  sg = sigmoid_fast(z);
  return z * sg;
}

// One 32-byte store of eight 32-bit words (dst 32-byte aligned).  Each thread
// of an epilogue writes its own row, so a warp's store touches 32 rows: the
// wider store halves the transactions per byte.
__device__ __forceinline__ void st_global_v8(void* dst, const uint32_t (&a)[8]) {
  if (!in_bounds(dst, 32)) return;
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
               :: "l"(dst), "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7])
               : "memory");
}

// Packs 16 floats to 8 bf16x2 words and stores them (one 32-byte store).
__device__ __forceinline__ void st_bf16x16(__nv_bfloat16* dst, const float* v) {
  uint32_t w[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) w[i] = pack_bf16(v[2 * i], v[2 * i + 1]);
  st_global_v8(dst, w);
}

// Four 8-column TMEM loads (z1, z3, dg1, dg3 of the same rows) and one wait.
__device__ __forceinline__ void tmem_ld8x4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, float (&r)[4][8]) {
  uint32_t u[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
        "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]),
        "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]),
        "=r"(u[30]), "=r"(u[31])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
      : "memory");
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int i = 0; i < 8; ++i) r[m][i] = __uint_as_float(u[8 * m + i]);
}

// Unpacks 8 bf16 (one 16-byte word) to floats.
__device__ __forceinline__ void unpack8(const uint4& a, float* v) {
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[2 * j] = __uint_as_float(w[j] << 16);
    v[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
  }
}


// Unpacks 16 bf16 (two 16-byte words) to floats.
__device__ __forceinline__ void unpack16(const uint4& a, const uint4& b, float* v) {
  const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    v[2 * j] = __uint_as_float(w[j] << 16);
    v[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
  }
}

// A 16-byte read-only load (zeros when bounds checking rejects it).
__device__ __forceinline__ uint4 ldg16(const uint4* p) {
  return in_bounds(p, 16) ? __ldg(p) : make_uint4(0, 0, 0, 0);
}

// A null pointer is an unused operand; any other must lie inside a
// registered range (bounds-checking build), else the block skips its work.
#define ROW_CHECK(p, bytes)                                  \
  do {                                                       \
    if ((p) && !in_bounds((p), (uint32_t)(bytes))) return;   \
  } while (0)

// Persistent: CTA b takes output tiles b, b + gridDim.x, ... (consecutive
// CTAs share an A row-block).  The TMA warp runs the stage ring across tiles;
// the MMA warp alternates between two 256-column accumulators; epilogue group
// g (four warps, all 128 TMEM lanes) drains the tiles of accumulator g, so a
// tile's epilogue overlaps the next tile's MMAs.
// XSET: the update-VJP gate and the squared-error loss's epilogues, in their own
// instantiation so that the common ones keep their register allocation.
// The three learning rates of output row m (W1, W3, W2).
__device__ __forceinline__ void row_rates(const GemmArgs& g, int m, float& e1, float& e3, float& e2) {
  const float* ep = g.eta + (size_t)m * g.eta_stride;
  if (!in_bounds(ep, 4 * (2 * g.eta_mat + 1))) {
    e1 = e3 = e2 = 0.f;
    return;
  }
  e1 = ep[0];
  e3 = ep[g.eta_mat];
  e2 = ep[2 * g.eta_mat];
}

// One tile's d eta partials of row m: the three per-matrix sums, or their total.
__device__ __forceinline__ void store_deta(const GemmArgs& g, int m, int tn, float q1, float q3, float q2) {
  float* p = g.part + (size_t)m * g.ld_part;
  if (!in_bounds(p + (g.eta_mat ? 3 * tn : tn), g.eta_mat ? 12 : 4)) return;
  if (g.eta_mat) {
    p[3 * tn] = q1;
    p[3 * tn + 1] = q3;
    p[3 * tn + 2] = q2;
  } else {
    p[tn] = q1 + q3 + q2;
  }
}

template <bool XSET>
__global__ void __launch_bounds__(GEMM_THREADS, 1) wide_gemm_kernel(const __grid_constant__ GemmArgs g) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], never_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tiles_n = g.N / BN;
  const int ntiles = ((g.M + BM - 1) / BM) * tiles_n;
  const int nunits = ntiles * g.ksplit;   // work units: K range s of tile t is unit s * ntiles + t
  const int nk = (g.K + BK - 1) / BK;
  const int kps = g.nseg > 1 ? g.kseg / BK : nk;   // K blocks per segment
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
    mbar_init(&never_bar, 1);   // no thread ever arrives
    abort_flag = 0;
    fence_barrier_init();
    for (int j = 0; j < g.nseg; ++j) prefetch_tmap(&g.a[j]);
    for (int j = 0; j < (g.nbn > g.nseg ? g.nbn : g.nseg); ++j) prefetch_tmap(&g.b[j]);
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
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const int t = u % ntiles, ks0 = (u / ntiles) * g.kb_split;
        const int tm = t / tiles_n, tn = t % tiles_n;
        const int m0 = tm * BM, n0 = tn * BN;
        const int kb_end = min(nk, ks0 + g.kb_split);
        for (int kb = ks0; kb < kb_end; ++kb, ++it) {
          const int s = it % STAGES;
          if (!mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
          uint8_t* as = sm + s * STAGE_BYTES;
          uint8_t* bs = as + A_STAGE;
          const int sg = kb / kps, k0 = (kb % kps) * BK;
          const CUtensorMap* am = &g.a[sg];
          if (!g.a_mn) {
            tma_load_3d(as, am, &full[s], k0, g.ha, g.ya + m0);
          } else {
            tma_load_3d(as, am, &full[s], m0, g.ha, g.ya + k0);
            tma_load_3d(as + 8192, am, &full[s], m0 + 64, g.ha, g.ya + k0);
          }
          if (g.nbn > 1) {
            const int rows = BN / g.nbn;
            for (int j = 0; j < g.nbn; ++j)
              tma_load_3d(bs + j * (B_STAGE / g.nbn), &g.b[j], &full[s], k0, g.hb, g.yb + tn * rows);
          } else if (!g.b_mn) {
            tma_load_3d(bs, &g.b[sg], &full[s], k0, g.hb, g.yb + n0);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) tma_load_3d(bs + 8192 * j, &g.b[sg], &full[s], n0 + 64 * j, g.hb, g.yb + k0);
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
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++i) {
      const int ac = i & 1;
      const int ks0 = (u / ntiles) * g.kb_split, kb_end = min(nk, ks0 + g.kb_split);
      if (!mbar_wait_w(&acc_empty[ac], ((i >> 1) & 1) ^ 1, abort)) break;
      tc_fence_after();
      const uint32_t acc = tb + ac * 256;
      for (int kb = ks0; kb < kb_end; ++kb, ++it) {
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
          mma_ss_w(acc, ad, bd, idesc, (kb > ks0 || ks > 0) ? 1u : 0u);
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
    for (int u = blockIdx.x + gp * gridDim.x; u < nunits; u += 2 * gridDim.x, i += 2) {
      if (!XSET && (g.epi == EPI_GCM_GATE || g.epi == EPI_F32_ADDIN)) {
        // the row's addend (x, or the residual gradient) of this group's next
        // tile (and of its first) into L2 while products finish: the column
        // loop below then waits on L2, not HBM
        for (int up = (i == gp ? u : u + 2 * (int)gridDim.x); up <= u + 2 * (int)gridDim.x && up < nunits;
             up += 2 * (int)gridDim.x) {
          const int tp = up % ntiles;
          const int mp = (tp / tiles_n) * BM + (int)row, np = (tp % tiles_n) * BN;
          if (mp < g.M) {
            const __nv_bfloat16* src = g.in0 + (size_t)mp * (g.ld_in ? g.ld_in : g.ld_out) + np;
            if (in_bounds(src, BN * 2)) bulk_prefetch_l2(src, BN * 2);
          }
        }
      }
      if (!mbar_wait(&acc_full[gp], (i >> 1) & 1, abort)) break;
      tc_fence_after();
      const int t = u % ntiles;
      float* const part_plane = g.ksplit > 1 ? reinterpret_cast<float*>(g.out[0]) + (u / ntiles) * g.split_stride
                                             : reinterpret_cast<float*>(g.out[0]);
      const int tm = t / tiles_n, tn = t % tiles_n;
      const int m0 = tm * BM, n0 = tn * BN;
      const int m = m0 + (int)row;
      const bool valid = m < g.M;
      if (XSET && g.epi != EPI_BKEY) {
        float e1 = 0.f, e3 = 0.f, e2 = 0.f;
        if (g.eta && valid) row_rates(g, m, e1, e3, e2);
        if (g.epi == EPI_MSE_E || g.epi == EPI_ADD_BF16 || g.epi == EPI_MSE_DE) {
          const int64_t ldi = g.ld_in ? g.ld_in : g.ld_out;
          const int64_t ld1 = g.ld_out1 ? g.ld_out1 : g.ld_out;
          const float sx = g.eta ? e2 : 1.f;   // EPI_ADD_BF16: the scale of in0
#pragma unroll 1
          for (int c = 0; c < BN; c += 16) {
            uint4 i0 = make_uint4(0, 0, 0, 0), i1 = i0;
            if (g.in0 && valid) {
              const uint4* ip = reinterpret_cast<const uint4*>(g.in0 + (size_t)m * ldi + n0 + c);
              i0 = ldg16(ip);
              i1 = ldg16(ip + 1);
            }
            float acc[16];
            tmem_ld16(accb + c, acc);
            if (!valid) continue;
            float x[16], o0[16], o1[16];
            unpack16(i0, i1, x);
            const size_t off0 = (size_t)m * g.ld_out + n0 + c, off1 = (size_t)m * ld1 + n0 + c;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              if (g.epi == EPI_MSE_E) {            // x = v
                o0[e] = acc[e] - x[e];
                o1[e] = e2 * o0[e];
              } else if (g.epi == EPI_ADD_BF16) {
                o0[e] = fmaf(sx, x[e], acc[e]);
              } else {                             // EPI_MSE_DE
                o0[e] = acc[e];
                o1[e] = -acc[e];
              }
            }
            st_bf16x16(reinterpret_cast<__nv_bfloat16*>(g.out[0]) + off0, o0);
            if (g.epi != EPI_ADD_BF16 && g.out[1]) st_bf16x16(reinterpret_cast<__nv_bfloat16*>(g.out[1]) + off1, o1);
          }
        } else if (g.epi == EPI_APPLY2) {
          // columns [0, 128) z1, [128, 256) z3 of hidden units f0 .. f0 + 127
          const int f0 = tn * (BN / 2);
#pragma unroll 1
          for (int c = 0; c < BN / 2; c += 16) {
            float z1[16], z3[16];
            tmem_ld16(accb + c, z1);
            tmem_ld16(accb + 128 + c, z3);
            if (!valid) continue;
            float h[16], hs[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              float sg;
              h[e] = silu_d(z1[e], sg) * z3[e];
              hs[e] = e2 * h[e];
            }
            const size_t off = (size_t)m * g.ld_out + f0 + c;
            st_bf16x16(reinterpret_cast<__nv_bfloat16*>(g.out[0]) + off, h);
            st_bf16x16(reinterpret_cast<__nv_bfloat16*>(g.out[1]) + off, hs);
          }
        } else {
          // columns [0,64) z1, [64,128) z3, [128,192) dg1, [192,256) dg3 of
          // hidden units f0 .. f0 + 63 (dg = -R k); squared-error loss
          const int f0 = tn * (BN / 4);
          const uint4* pp = reinterpret_cast<const uint4*>(g.in0 + (size_t)m * g.ld_out + f0);
          const uint4* up = reinterpret_cast<const uint4*>(g.in1 + (size_t)m * g.ld_out + f0);
          const bool second = g.epi == EPI_BKEY_MSE2;
          float q1 = 0.f, q3 = 0.f, q2 = 0.f;
#pragma unroll 1
          for (int c = 0; c < 64; c += 16) {
            uint4 pw[2], uw[2];   // the inputs of the 16 columns, in flight during the TMEM loads
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              pw[j] = valid ? ldg16(pp + c / 8 + j) : make_uint4(0, 0, 0, 0);
              uw[j] = valid ? ldg16(up + c / 8 + j) : make_uint4(0, 0, 0, 0);
            }
            uint32_t pk[3][8];   // 16 columns of each output, packed bf16 pairs
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const int cc = c + 8 * hh;
              float zz[4][8];
              tmem_ld8x4(accb + cc, accb + 64 + cc, accb + 128 + cc, accb + 192 + cc, zz);
              float pv[8], w[8];
              unpack8(pw[hh], pv);
              unpack8(uw[hh], w);
              float o[3][8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                float sg;
                const float x1 = zz[0][e], x3 = zz[1][e], d1 = zz[2][e], d3 = zz[3][e];
                const float a = silu_d(x1, sg);
                const float sp = fmaf(a, 1.f - sg, sg);                               // silu'(z1)
                const float t1 = d1 * x3 * sp;
                if (!second) {                                       // w = -R2^T e
                  o[0][e] = e1 * t1 + e3 * d3 * a;                   // dp
                  o[1][e] = e1 * pv[e] * x3 * sp;                    // g1
                  o[2][e] = e3 * pv[e] * a;                          // g3
                  q1 = fmaf(pv[e], t1, q1);
                  q3 = fmaf(pv[e] * a, d3, q3);
                  q2 = fmaf(w[e], a * x3, q2);
                } else {                                             // w = du
                  const float spp = sg * (1.f - sg) * fmaf(x1, 1.f - 2.f * sg, 2.f);  // silu''(z1)
                  const float da = e3 * d3 * pv[e] + w[e] * x3;
                  o[1][e] = e1 * d1 * pv[e] * sp + w[e] * a;         // dz3
                  o[0][e] = e1 * d1 * pv[e] * x3 * spp + da * sp;    // dz1
                  o[2][e] = 0.f;
                }
              }
#pragma unroll
              for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int i = 0; i < 4; ++i) pk[q][4 * hh + i] = pack_bf16(o[q][2 * i], o[q][2 * i + 1]);
            }
            if (valid) {
              const size_t off = (size_t)m * g.ld_out + f0 + c;
#pragma unroll
              for (int q = 0; q < 3; ++q)
                if (q < (second ? 2 : 3)) st_global_v8(reinterpret_cast<__nv_bfloat16*>(g.out[q]) + off, pk[q]);
            }
          }
          if (!second && valid) store_deta(g, m, tn, q1, q3, q2);
        }
      } else if (!XSET && (g.epi == EPI_F32 || g.epi == EPI_BF16 || g.epi == EPI_F32_ADD)) {
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          float v0[16], v1[16];
          tmem_ld16(accb + c, v0);
          tmem_ld16(accb + c + 16, v1);
          if (!valid) continue;
          if (g.epi == EPI_BF16) {
            __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(g.out[0]) + (size_t)m * g.ld_out + n0 + c;
            st_bf16x16(o, v0);
            st_bf16x16(o + 16, v1);
          } else {
            float4* o = reinterpret_cast<float4*>(part_plane + (size_t)m * g.ld_out + n0 + c);
            if (!in_bounds(o, 128)) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              float4 x0 = make_float4(v0[4 * j], v0[4 * j + 1], v0[4 * j + 2], v0[4 * j + 3]);
              float4 x1 = make_float4(v1[4 * j], v1[4 * j + 1], v1[4 * j + 2], v1[4 * j + 3]);
              if (g.epi == EPI_F32_ADD) {
                const float4 y0 = o[j], y1 = o[4 + j];
                x0 = make_float4(y0.x + x0.x, y0.y + x0.y, y0.z + x0.z, y0.w + x0.w);
                x1 = make_float4(y1.x + x1.x, y1.y + x1.y, y1.z + x1.z, y1.w + x1.w);
              }
              o[j] = x0;
              o[4 + j] = x1;
            }
          }
        }
      } else if (!XSET && g.epi == EPI_GCM_QKV) {
        // the tile's 256 columns lie in one of q, k, v (d is a multiple of 256)
        const int dm = (int)g.ld_out, part = n0 / dm, c0 = n0 - part * dm;
        __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(g.out[part]) + (size_t)m * dm + c0;
        float* ssq = reinterpret_cast<float*>(g.out[3]) + (size_t)m * g.ld_part + (part * dm + c0) / 64;
        float ss = 0.f;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          float v0[16], v1[16];
          tmem_ld16(accb + c, v0);
          tmem_ld16(accb + c + 16, v1);
          if (!valid) continue;
          const float* bb = g.colvec + n0 + c;
          if (!in_bounds(bb, 128)) continue;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            v0[i] += bb[i];
            v1[i] += bb[16 + i];
          }
          st_bf16x16(dst + c, v0);
          st_bf16x16(dst + c + 16, v1);
          if (part < 2) {   // the norm from the float32 values
#pragma unroll
            for (int i = 0; i < 16; ++i) ss = fmaf(v1[i], v1[i], fmaf(v0[i], v0[i], ss));
            if (c & 32) {
              if (in_bounds(ssq + c / 64, 4)) ssq[c / 64] = ss;
              ss = 0.f;
            }
          }
        }
      } else if (!XSET && (g.epi == EPI_GCM_GATE || g.epi == EPI_F32_ADDIN)) {
        const int64_t ldi = g.ld_in ? g.ld_in : g.ld_out;
        // the addend in batches of 64 columns: eight 16-byte loads in flight
        // per thread, so a tile waits four memory round trips, not eight
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 64) {
          const uint4* xin = reinterpret_cast<const uint4*>(g.in0 + (size_t)m * ldi + n0 + c0);
          const bool okx = valid && in_bounds(xin, 128);
          uint4 xw[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) xw[j] = okx ? xin[j] : make_uint4(0, 0, 0, 0);
#pragma unroll
          for (int cc = 0; cc < 64; cc += 32) {
            const int c = c0 + cc;
            float v0[16], v1[16];
            tmem_ld16(accb + c, v0);
            tmem_ld16(accb + c + 16, v1);
            if (!okx) continue;
            float xv[32];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const uint4 w = xw[cc / 8 + j];
              const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                xv[8 * j + 2 * e] = bf16_lo(ww[e]);
                xv[8 * j + 2 * e + 1] = bf16_hi(ww[e]);
              }
            }
            if (g.epi == EPI_F32_ADDIN) {
              float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(g.out[0]) + (size_t)m * g.ld_out + n0 + c);
              if (!in_bounds(o, 128)) continue;
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                o[j] = make_float4(v0[4 * j] + xv[4 * j], v0[4 * j + 1] + xv[4 * j + 1], v0[4 * j + 2] + xv[4 * j + 2],
                                   v0[4 * j + 3] + xv[4 * j + 3]);
                o[4 + j] = make_float4(v1[4 * j] + xv[16 + 4 * j], v1[4 * j + 1] + xv[17 + 4 * j],
                                       v1[4 * j + 2] + xv[18 + 4 * j], v1[4 * j + 3] + xv[19 + 4 * j]);
              }
            } else {
              const size_t off = (size_t)m * g.ld_out + n0 + c;
              __nv_bfloat16* yo = reinterpret_cast<__nv_bfloat16*>(g.out[1]) + off;
              st_bf16x16(yo, v0);
              st_bf16x16(yo + 16, v1);
              const float* al = g.colvec + n0 + c;
              if (!in_bounds(al, 128)) continue;
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                v0[i] = fmaf(al[i], v0[i], xv[i]);
                v1[i] = fmaf(al[16 + i], v1[i], xv[16 + i]);
              }
              __nv_bfloat16* oo = reinterpret_cast<__nv_bfloat16*>(g.out[0]) + off;
              st_bf16x16(oo, v0);
              st_bf16x16(oo + 16, v1);
            }
          }
        }
      } else if (XSET) {   // EPI_BKEY
        // columns [0,64) z1, [64,128) z3, [128,192) dg1, [192,256) dg3 of
        // hidden units f0 .. f0 + 63 (dg = -R k)
        const int f0 = tn * (BN / 4);
        float e1 = 0.f, e3 = 0.f, e2 = 0.f;
        if (valid) row_rates(g, m, e1, e3, e2);
        f32x2 aq1 = x2(0.f), aq3 = x2(0.f), aq2 = x2(0.f);   // d eta partials, negated, per lane
        const uint4* pp = reinterpret_cast<const uint4*>(g.in0 + (size_t)m * g.ld_out + f0);
        const uint4* np = reinterpret_cast<const uint4*>(g.in1 + (size_t)m * g.ld_out + f0);
#pragma unroll 1
        for (int c = 0; c < 64; c += 16) {
          uint4 pcur[2], ncur[2];   // the inputs of the 16 columns, in flight during the TMEM loads
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            pcur[j] = valid ? ldg16(pp + c / 8 + j) : make_uint4(0, 0, 0, 0);
            ncur[j] = valid ? ldg16(np + c / 8 + j) : make_uint4(0, 0, 0, 0);
          }
          uint32_t pk[6][8];   // 16 columns of each output, packed bf16 pairs
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int cc = c + 8 * hh;
            float zz[4][8];
            tmem_ld8x4(accb + cc, accb + 64 + cc, accb + 128 + cc, accb + 192 + cc, zz);
            float praw[8], ndu[8];
            unpack8(pcur[hh], praw);
            unpack8(ncur[hh], ndu);
            // the chain rule on pairs of hidden units (packed float32 lanes)
            const f32x2 n1 = x2(-e1), n3 = x2(-e3), n2 = x2(-e2), one = x2(1.f), two = x2(2.f), mtwo = x2(-2.f);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const int e = 2 * w;
              const f32x2 x1 = x2(zz[0][e], zz[0][e + 1]), x3 = x2(zz[1][e], zz[1][e + 1]);
              const f32x2 d1 = x2(zz[2][e], zz[2][e + 1]), d3 = x2(zz[3][e], zz[3][e + 1]);
              const f32x2 pr = x2(praw[e], praw[e + 1]), nd = x2(ndu[e], ndu[e + 1]);
              const f32x2 sg = sigmoid2(x1);
              const f32x2 a = mul2(x1, sg);
              const f32x2 oms = sub2(one, sg);
              const f32x2 sp = fma2(a, oms, sg);                                         // silu'(z1)
              const f32x2 spp = mul2(mul2(sg, oms), fma2(x1, fma2(mtwo, sg, one), two));  // silu''(z1)
              const f32x2 u = mul2(a, x3);
              const f32x2 p1 = mul2(n1, pr), p3 = mul2(n3, pr);   // rate times p (e = -v)
              const f32x2 du = mul2(n2, nd);
              const f32x2 x3sp = mul2(x3, sp);
              const f32x2 t1 = mul2(d1, x3sp);
              const f32x2 d3a = mul2(d3, a);
              const f32x2 da = fma2(d3, p3, mul2(du, x3));
              const f32x2 dp1 = mul2(d1, p1);
              pk[1][4 * hh + w] = pack_bf16x2(fma2(dp1, sp, mul2(du, a)));                 // dz3
              pk[0][4 * hh + w] = pack_bf16x2(fma2(mul2(dp1, x3), spp, mul2(da, sp)));     // dz1
              pk[2][4 * hh + w] = pack_bf16x2(mul2(p1, x3sp));                           // g1
              pk[3][4 * hh + w] = pack_bf16x2(mul2(p3, a));                              // g3
              pk[4][4 * hh + w] = pack_bf16x2(fma2(n1, t1, mul2(n3, d3a)));              // -dp
              pk[5][4 * hh + w] = pack_bf16x2(mul2(n2, u));                              // -eta2 u
              aq1 = fma2(pr, t1, aq1);
              aq3 = fma2(pr, d3a, aq3);
              aq2 = fma2(nd, u, aq2);
            }
          }
          if (valid) {
            const size_t off = (size_t)m * g.ld_out + f0 + c;
#pragma unroll
            for (int q = 0; q < 6; ++q) st_global_v8(reinterpret_cast<__nv_bfloat16*>(g.out[q]) + off, pk[q]);
          }
        }
        if (valid)
          store_deta(g, m, tn, -(x2_lo(aq1) + x2_hi(aq1)), -(x2_lo(aq3) + x2_hi(aq3)), -(x2_lo(aq2) + x2_hi(aq2)));
      } else {
        // gate epilogues: columns [0, 128) are z1, [128, 256) z3 of hidden
        // units f0 .. f0 + 127
        const int f0 = tn * (BN / 2);
        float e1 = 0.f, e3 = 0.f, e2 = 0.f;
        if (g.epi == EPI_KEY && valid) row_rates(g, m, e1, e3, e2);
        if (!g.mse) {   // dot loss: e = -eta v
          e1 = -e1;
          e3 = -e3;
        }
        // this row's 128 values of the epilogue input (KEY: P; BAPPLY:
        // W2^T d_o), loaded at once: one memory latency per tile
        uint4 prow[16];
        if (g.epi != EPI_APPLY && valid) {
          const uint4* pp = reinterpret_cast<const uint4*>(g.in0 + (size_t)m * g.ld_out + f0);
#pragma unroll
          for (int j = 0; j < 16; ++j) prow[j] = ldg16(pp + j);
        }
        // on pairs of hidden units (packed float32 lanes); KEY scales the
        // factors by the rates, BAPPLY by 1
        const bool key = g.epi == EPI_KEY;
        const f32x2 s1 = x2(key ? e1 : 1.f), s3 = x2(key ? e3 : 1.f), s2 = x2(key ? -e2 : 1.f), one = x2(1.f);
#pragma unroll
        for (int c = 0; c < BN / 2; c += 16) {
          float z1[16], z3[16];
          tmem_ld16(accb + c, z1);
          tmem_ld16(accb + 128 + c, z3);
          if (!valid) continue;
          const size_t off = (size_t)m * g.ld_out + f0 + c;
          if (g.epi == EPI_APPLY) {
            uint32_t hw[8];
#pragma unroll
            for (int w = 0; w < 8; ++w) {
              const f32x2 x = x2(z1[2 * w], z1[2 * w + 1]);
              hw[w] = pack_bf16x2(mul2(mul2(x, sigmoid2(x)), x2(z3[2 * w], z3[2 * w + 1])));
            }
            st_global_v8(reinterpret_cast<__nv_bfloat16*>(g.out[0]) + off, hw);
          } else {
            float r[16];
            unpack16(prow[c / 8], prow[c / 8 + 1], r);
            uint32_t w0[8], w1[8], w2[8];
#pragma unroll
            for (int w = 0; w < 8; ++w) {
              const f32x2 x1 = x2(z1[2 * w], z1[2 * w + 1]), x3 = x2(z3[2 * w], z3[2 * w + 1]);
              const f32x2 rr = x2(r[2 * w], r[2 * w + 1]);
              const f32x2 sg = sigmoid2(x1);
              const f32x2 a = mul2(x1, sg);
              const f32x2 sp = fma2(a, sub2(one, sg), sg);        // silu'(z1)
              // KEY: r = W2^T v (dot) or W2^T e (squared error) -> g1, g3, u~ = -eta2 u;
              // BAPPLY: r = W2^T d_o -> dzq1, dzq3, uq
              w0[w] = pack_bf16x2(mul2(mul2(mul2(s1, rr), x3), sp));
              w1[w] = pack_bf16x2(mul2(mul2(s3, rr), a));
              w2[w] = pack_bf16x2(mul2(s2, mul2(a, x3)));
            }
            st_global_v8(reinterpret_cast<__nv_bfloat16*>(g.out[0]) + off, w0);
            st_global_v8(reinterpret_cast<__nv_bfloat16*>(g.out[1]) + off, w1);
            if (g.out[2]) st_global_v8(reinterpret_cast<__nv_bfloat16*>(g.out[2]) + off, w2);
          }
        }
      }
      // the accumulator is drained: the MMA warp may reuse it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[gp]);
    }
    // bounded-wait test: every tile is stored and no copy or MMA is in flight;
    // the wait runs out, raises the abort flag and the status word reports it
    if (g.timeout_test) mbar_wait(&never_bar, 0, abort, 50000000ull);
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
  ROW_CHECK(w0 + off, 4 * len);
  ROW_CHECK(wm + off, 4 * len);
  ROW_CHECK(wb + off, 2 * len);
  ROW_CHECK(rho ? rho + blockIdx.x : nullptr, 4);
  float ss = 0.f;
  for (int i = 4 * threadIdx.x; i < len; i += 4 * ROW_THREADS) {
    const float4 x = *reinterpret_cast<const float4*>(w0 + off + i);
    *reinterpret_cast<float4*>(wm + off + i) = x;
    *reinterpret_cast<uint2*>(wb + off + i) = make_uint2(pack_bf16(x.x, x.y), pack_bf16(x.z, x.w));
    ss += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
  }
  ss = block_sum(ss, red);
  if (rho && threadIdx.x == 0) rho[blockIdx.x] = (norm == SCAL3R_NORM_UNIT) ? 1.f : sqrtf(ss);
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
  ROW_CHECK(wm + off, 4 * len);
  ROW_CHECK(gr + off, 4 * len);
  ROW_CHECK(wb + off, 2 * len);
  ROW_CHECK(norm == SCAL3R_NORM_NONE ? nullptr : rho + blockIdx.x, 4);
  ROW_CHECK(wnorm ? wnorm + blockIdx.x : nullptr, 4);
  ROW_CHECK(ckpt ? ckpt + off : nullptr, 4 * len);
  ROW_CHECK(wfinal ? wfinal + off : nullptr, 4 * len);
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

// Backward setup of one chain: row-norm targets of W0 and their adjoints.
__global__ void __launch_bounds__(ROW_THREADS) wide_bprep_kernel(const float* __restrict__ w0, float* __restrict__ rho,
                                                                 float* __restrict__ drho, int D, int F, int norm) {
  __shared__ float red[ROW_THREADS / 32 + 1];
  size_t off;
  int len;
  row_geometry(blockIdx.x, D, F, off, len);
  ROW_CHECK(w0 + off, 4 * len);
  ROW_CHECK(rho + blockIdx.x, 4);
  ROW_CHECK(drho + blockIdx.x, 4);
  float ss = 0.f;
  for (int i = 4 * threadIdx.x; i < len; i += 4 * ROW_THREADS) {
    const float4 x = *reinterpret_cast<const float4*>(w0 + off + i);
    ss += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
  }
  ss = block_sum(ss, red);
  if (threadIdx.x == 0) {
    rho[blockIdx.x] = (norm == SCAL3R_NORM_UNIT) ? 1.f : sqrtf(ss);
    drho[blockIdx.x] = 0.f;
  }
}

// Operands of one backward step: bf16 W (from w), bf16 -R (from r, if any),
// and the adjoint accumulator lam = R (or 0).
__global__ void wide_bstep_setup_kernel(const float* __restrict__ w, const float* __restrict__ r,
                                        __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ nrb,
                                        float* __restrict__ lam, size_t P) {
  ROW_CHECK(w, 4 * P);
  ROW_CHECK(wb, 2 * P);
  ROW_CHECK(r, 4 * P);
  ROW_CHECK(r ? nrb : nullptr, 2 * P);
  ROW_CHECK(lam, 4 * P);
  for (size_t i = 4 * ((size_t)blockIdx.x * blockDim.x + threadIdx.x); i < P; i += 4 * (size_t)gridDim.x * blockDim.x) {
    const float4 x = *reinterpret_cast<const float4*>(w + i);
    *reinterpret_cast<uint2*>(wb + i) = make_uint2(pack_bf16(x.x, x.y), pack_bf16(x.z, x.w));
    float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r) {
      y = *reinterpret_cast<const float4*>(r + i);
      *reinterpret_cast<uint2*>(nrb + i) = make_uint2(pack_bf16(-y.x, -y.y), pack_bf16(-y.z, -y.w));
    }
    *reinterpret_cast<float4*>(lam + i) = y;
  }
}

// Closing a backward step (one block per row).  lam = dL/dW_j.  For j > 0 the
// VJP of the row normalisation of update j-1 (W_j = rho w~ / max(|w~|, eps)):
//   unclamped  R = (rho / |w~|) (lam - w_hat (w_hat . lam)),  clamped  R = (rho / eps) lam,
//   w_hat = W_j / rho, drho += w_hat . lam;
// for j = 0, dW0 = lam + drho W0 / rho (added to dw0 when accumulate is set).
__global__ void __launch_bounds__(ROW_THREADS) wide_bupdate_kernel(const float* __restrict__ lam,
                                                                   const float* __restrict__ wj,
                                                                   const float* __restrict__ wnorm,
                                                                   const float* __restrict__ rho, float* drho,
                                                                   float* __restrict__ rout, const float* w0,
                                                                   float* dw0, int accumulate, int D, int F, int norm,
                                                                   float eps) {
  __shared__ float red[ROW_THREADS / 32 + 1];
  size_t off;
  int len;
  row_geometry(blockIdx.x, D, F, off, len);
  ROW_CHECK(rho + blockIdx.x, 4);
  ROW_CHECK(lam + off, 4 * len);
  if (dw0) {
    ROW_CHECK(w0 + off, 4 * len);
    ROW_CHECK(dw0 + off, 4 * len);
    ROW_CHECK(norm == SCAL3R_NORM_ROW_W0 ? drho + blockIdx.x : nullptr, 4);
  } else {
    ROW_CHECK(rout + off, 4 * len);
    if (norm != SCAL3R_NORM_NONE) {
      ROW_CHECK(wj + off, 4 * len);
      ROW_CHECK(wnorm + blockIdx.x, 4);
      ROW_CHECK(norm == SCAL3R_NORM_ROW_W0 ? drho + blockIdx.x : nullptr, 4);
    }
  }
  const float rh = rho[blockIdx.x];
  if (dw0) {
    const float coef = (norm == SCAL3R_NORM_ROW_W0 && rh > 0.f) ? drho[blockIdx.x] / rh : 0.f;
    for (int i = 4 * threadIdx.x; i < len; i += 4 * ROW_THREADS) {
      const float4 l = *reinterpret_cast<const float4*>(lam + off + i);
      const float4 x = *reinterpret_cast<const float4*>(w0 + off + i);
      float4 y = make_float4(l.x + coef * x.x, l.y + coef * x.y, l.z + coef * x.z, l.w + coef * x.w);
      if (accumulate) {
        const float4 z = *reinterpret_cast<const float4*>(dw0 + off + i);
        y = make_float4(z.x + y.x, z.y + y.y, z.z + y.z, z.w + y.w);
      }
      *reinterpret_cast<float4*>(dw0 + off + i) = y;
    }
    return;
  }
  if (norm == SCAL3R_NORM_NONE) {
    for (int i = 4 * threadIdx.x; i < len; i += 4 * ROW_THREADS)
      *reinterpret_cast<float4*>(rout + off + i) = *reinterpret_cast<const float4*>(lam + off + i);
    return;
  }
  const float inv = rh > 0.f ? 1.f / rh : 0.f;
  float pr = 0.f;
  for (int i = 4 * threadIdx.x; i < len; i += 4 * ROW_THREADS) {
    const float4 l = *reinterpret_cast<const float4*>(lam + off + i);
    const float4 x = *reinterpret_cast<const float4*>(wj + off + i);
    pr += (x.x * l.x + x.y * l.y + x.z * l.z + x.w * l.w) * inv;
  }
  const float proj = block_sum(pr, red);
  const float n = wnorm[blockIdx.x];
  const bool clamped = !(n >= eps);
  const float c = clamped ? rh / eps : rh / n;
  for (int i = 4 * threadIdx.x; i < len; i += 4 * ROW_THREADS) {
    const float4 l = *reinterpret_cast<const float4*>(lam + off + i);
    const float4 x = *reinterpret_cast<const float4*>(wj + off + i);
    float4 y;
    if (clamped) {
      y = make_float4(c * l.x, c * l.y, c * l.z, c * l.w);
    } else {
      y = make_float4(c * (l.x - x.x * inv * proj), c * (l.y - x.y * inv * proj), c * (l.z - x.z * inv * proj),
                      c * (l.w - x.w * inv * proj));
    }
    *reinterpret_cast<float4*>(rout + off + i) = y;
  }
  if (threadIdx.x == 0 && norm == SCAL3R_NORM_ROW_W0) drho[blockIdx.x] += proj;
}

// d eta of the chunk's tokens: the per-tile partials summed in tile order
// (nmat = 3: each matrix's rate from its own partials).
__global__ void wide_deta_kernel(const float* __restrict__ part, int64_t ld_part, int ntiles, int nmat,
                                 float* __restrict__ dlr, int64_t stride, int M) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  ROW_CHECK(part + (size_t)m * ld_part, 4 * ntiles * nmat);
  ROW_CHECK(dlr + (size_t)m * stride, 4 * nmat);
  for (int j = 0; j < nmat; ++j) {
    float a = 0.f;
    for (int t = 0; t < ntiles; ++t) a += part[(size_t)m * ld_part + (size_t)t * nmat + j];
    dlr[(size_t)m * stride + j] = a;
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
  return D >= 256 && D % 256 == 0 && F >= 256 && F % 256 == 0 && F <= 4096 && D <= 4096;
}

namespace {

int64_t max_chunk(const Plan& p) {
  int64_t mmax = 0;
  for (size_t c = 0; c + 1 < p.chunk_offsets.size(); ++c)
    mmax = std::max<int64_t>(mmax, p.chunk_offsets[c + 1] - p.chunk_offsets[c]);
  return (mmax + BM - 1) / BM * BM;
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Workspace: activation buffers [mmax x F] bf16 (4 forward, 8 backward),
// then float32 and bf16 weight-sized buffers.
struct WideBufs {
  __nv_bfloat16* act[8];
  float* wm;      // forward: master weights;  backward: lam (dL/dW_j)
  float* gr;      // forward: chunk gradient;  backward: R (dL/dW~ of the next update)
  __nv_bfloat16* wb;    // bf16 weights
  __nv_bfloat16* nrb;   // backward: bf16 -R
  float* rho;
  float* drho;
  float* part;    // backward: d eta partials [mmax x F/64]
  float* rgr;     // backward with sparse checkpoints: the recomputed chunk gradient
  float* seg;     // backward with sparse checkpoints: W_j of one segment, ckpt_every - 1 blocks of P
  __nv_bfloat16* ex[2];   // squared-error loss: [mmax x D] bf16 (forward: e, eta2 e; backward: e, dY)
  float* spl;     // partial planes of the split weight-sized reductions (null: none split)
};

int split_count(int64_t M, int64_t N, int64_t K, int out_fp32);

// d eta partials per token row: one per 64 hidden units (the update-VJP
// gate's tiles), times three with per-matrix rates.
int deta_parts(const Shape& s, int lr_mat) { return (s.F / 64) * (lr_mat ? 3 : 1); }

size_t layout_bytes(const Plan& p, const Shape& s, bool bwd, int ckpt_every, bool mse, int lr_mat, WideBufs* w,
                    void* ws) {
  const size_t P = (size_t)s.P();
  const int64_t mmax = max_chunk(p);
  const size_t act = al256((size_t)mmax * s.F * 2);
  uint8_t* base = reinterpret_cast<uint8_t*>(ws);
  size_t o = 0;
  auto take = [&](size_t n) {
    uint8_t* q = base ? base + o : nullptr;
    o += al256(n);
    return q;
  };
  const int nact = bwd ? 8 : 4;
  WideBufs x{};
  for (int i = 0; i < nact; ++i) x.act[i] = reinterpret_cast<__nv_bfloat16*>(take(act));
  x.wm = reinterpret_cast<float*>(take(P * 4));
  x.gr = reinterpret_cast<float*>(take(P * 4));
  x.wb = reinterpret_cast<__nv_bfloat16*>(take(P * 2));
  if (bwd) x.nrb = reinterpret_cast<__nv_bfloat16*>(take(P * 2));
  x.rho = reinterpret_cast<float*>(take((size_t)s.R() * 4));
  if (bwd) {
    x.drho = reinterpret_cast<float*>(take((size_t)s.R() * 4));
    x.part = reinterpret_cast<float*>(take((size_t)mmax * deta_parts(s, lr_mat) * 4));
    if (ckpt_every > 1) {   // recomputation between stored checkpoints
      x.rgr = reinterpret_cast<float*>(take(P * 4));
      x.seg = reinterpret_cast<float*>(take(P * 4 * (size_t)(ckpt_every - 1)));
    }
  }
  if (mse)
    for (int i = 0; i < 2; ++i) x.ex[i] = reinterpret_cast<__nv_bfloat16*>(take((size_t)mmax * s.D * 2));
  // the [F x D] and [D x F] reductions over a chunk's tokens split their K
  // ranges when their tiles leave SMs idle; the longest chunk needs the most
  // ranges (split_count does not fall as K grows)
  const int nspl = mmax > 0 ? std::max(split_count(s.F, s.D, mmax, 1), split_count(s.D, s.F, mmax, 1)) : 1;
  if (nspl > 1) x.spl = reinterpret_cast<float*>(take((size_t)nspl * s.F * s.D * 4));
  if (w) *w = x;
  return o;
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
  if (a.nseg < 1) a.nseg = 1;
  if (a.nbn < 1) a.nbn = 1;
  if (a.nseg > 1 && (a.kseg % BK != 0 || a.kseg * a.nseg != a.K || a.nbn != 1)) return cudaErrorInvalidValue;
  const int nk = (a.K + BK - 1) / BK;
  if (a.ksplit <= 1) {
    a.ksplit = 1;
    a.kb_split = nk;
  } else if (a.nseg > 1 || a.epi != EPI_F32 || a.kb_split < 1 || (int64_t)(a.ksplit - 1) * a.kb_split >= nk) {
    return cudaErrorInvalidValue;   // every K range non-empty, plain float32 partial planes only
  }
  const int64_t units = (int64_t)((a.M + BM - 1) / BM) * (a.N / BN) * a.ksplit;
  if (units > INT32_MAX) return cudaErrorInvalidValue;
  const int grid = (int)std::min<int64_t>(units, num_sms());
  if ((a.epi >= EPI_MSE_E && a.epi <= EPI_APPLY2) || a.epi == EPI_BKEY)
    wide_gemm_kernel<true><<<grid, GEMM_THREADS, GEMM_SMEM, st>>>(a);
  else
    wide_gemm_kernel<false><<<grid, GEMM_THREADS, GEMM_SMEM, st>>>(a);
  return cudaGetLastError();
}

// Maps: a token tensor [T][H][D] (rows = tokens of head h) and a plain matrix [rows][cols].
bool tok_map(CUtensorMap* m, const void* base, int64_t T, int H, int D, int box_rows) {
  return make_map(m, base, T, H, D, (int64_t)H * D, box_rows);
}
bool mat_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int box_rows) {
  return make_map(m, base, rows, 1, cols, cols, box_rows);
}

using LaunchFn = std::function<cudaError_t(int, double, double, const std::function<cudaError_t()>&)>;

struct Ctx {
  const Plan& pl;
  const Shape& sh;
  const Params& prm;
  const LaunchFn& launch;
  cudaStream_t st;
};

#define WIDE_TRY(x)                          \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) return e_;        \
  } while (0)
#define WIDE_MAP(x)                                  \
  do {                                               \
    if (!(x)) return cudaErrorInvalidValue;          \
  } while (0)

cudaError_t run_gemm(const Ctx& c, GemmArgs& a, double flops) {
  a.status = c.prm.status;
  return c.launch(0, flops, 0, [&] { return gemm(a, c.st); });
}

// The learning rates of head h's tokens from t0 on: lr [T, H] or, with
// per-matrix rates, [T, H, 3].
void set_rates(GemmArgs& a, const Params& prm, int64_t t0, int h) {
  const int n = prm.lr_mat ? 3 : 1;
  a.eta = prm.lr + ((size_t)t0 * prm.H + h) * n;
  a.eta_stride = (int64_t)prm.H * n;
  a.eta_mat = prm.lr_mat ? 1 : 0;
}

// d eta of the chunk's M tokens from t0 (head h) from the gate's partials.
cudaError_t chunk_deta(const Ctx& cx, const float* part, int64_t t0, int h, int M) {
  const Params& prm = cx.prm;
  const int nmat = prm.lr_mat ? 3 : 1;
  const int ntiles = cx.sh.F / 64;
  float* dlr = prm.dlr + ((size_t)t0 * prm.H + h) * nmat;
  return cx.launch(1, 0, 0, [&] {
    wide_deta_kernel<<<(M + 127) / 128, 128, 0, cx.st>>>(part, (int64_t)ntiles * nmat, ntiles, nmat, dlr,
                                                         (int64_t)prm.H * nmat, M);
    return cudaGetLastError();
  });
}

}  // namespace

size_t wide_workspace_bytes(const Plan& p, const Shape& s, bool with_backward, int ckpt_every, int loss,
                            int lr_per_matrix) {
  return layout_bytes(p, s, with_backward, ckpt_every, loss == SCAL3R_LOSS_MSE, lr_per_matrix ? 1 : 0, nullptr,
                      nullptr);
}

// Checkpoint slot of W_j (the weights after local chunk j-1) of sequence s, or
// -1 if it is not stored: every chunk with ckpt_every <= 1, else the weights
// after local chunks n-1, 2n-1, ... (slots of the sequences one after another).
int64_t wide_ckpt_slot(const Plan& p, int s, int j, int n) {
  if (n <= 1) return p.seq_chunk_ptr[s] + j - 1;
  if (j < 1 || j % n != 0) return -1;
  int64_t base = 0;
  for (int t = 0; t < s; ++t) base += (p.seq_chunk_ptr[t + 1] - p.seq_chunk_ptr[t]) / n;
  return base + j / n - 1;
}

namespace {

// K ranges of a float32-output GEMM whose output tiles do not fill the SMs:
// as many ranges as fit the SMs in one wave (tiles x s <= SMs), each at
// least 4 K blocks long; 1 = no split.  Ranges beyond one wave would trim
// the last wave a little, but each adds a partial plane to the fixed-order
// sum: at 32 tiles of 128 x 256 and 16,656 tokens of K, 19 ranges (4 waves)
// take 16 % less GEMM time than 4 ranges (1 wave) and write and re-read
// 76 MB of planes instead of 16 MB, which costs more than it saves.  The
// count never falls as K grows, so a workspace sized for the longest K holds
// the planes of any shorter one.
int split_count(int64_t M, int64_t N, int64_t K, int out_fp32) {
  if (!out_fp32) return 1;
  const int64_t tiles = ((M + BM - 1) / BM) * (N / BN);
  const int64_t nk = (K + BK - 1) / BK;
  if (tiles <= 0) return 1;
  const int64_t s = std::min<int64_t>(std::min<int64_t>(num_sms() / tiles, nk / 4), 64);
  return s >= 2 ? (int)s : 1;
}

// C (+)= the sum of the partial planes in order s = 0 .. S-1 (fixed order:
// the result does not depend on which CTA finished first).
__global__ void split_reduce_kernel(const float* __restrict__ part, int S, int64_t plane, int64_t M, int64_t N,
                                    float* __restrict__ c, int64_t ldc, int accumulate) {
  const int64_t nq = N / 4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M * nq; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = i / nq, n = 4 * (i % nq);
    if (!in_bounds(part + m * N + n, 16) || !in_bounds(part + (S - 1) * plane + m * N + n, 16) ||
        !in_bounds(c + m * ldc + n, 16))
      continue;
    float4 acc = *reinterpret_cast<const float4*>(part + m * N + n);
    for (int s = 1; s < S; ++s) {
      const float4 x = *reinterpret_cast<const float4*>(part + s * plane + m * N + n);
      acc = make_float4(acc.x + x.x, acc.y + x.y, acc.z + x.z, acc.w + x.w);
    }
    float4* dst = reinterpret_cast<float4*>(c + m * ldc + n);
    if (accumulate) {
      const float4 y = *dst;
      acc = make_float4(y.x + acc.x, y.y + acc.y, y.z + acc.z, y.w + acc.w);
    }
    *dst = acc;
  }
}

// A float32 reduction over a chunk's tokens, C = A^T B or C += A^T B with K
// = the chunk's tokens (the weight gradients and adjoints): when its output
// tiles leave SMs idle, K is cut into split_count ranges whose partial planes
// go to `spl`, then summed in a fixed order onto C (the sum does not depend
// on which CTA finished first).  Unsplit when spl is null or the tiles fill
// the SMs.  The reduce is charged to the GEMM's kind.
cudaError_t run_gemm_red(const Ctx& c, GemmArgs& a, double flops, float* spl) {
  const bool acc = a.epi == EPI_F32_ADD;
  const int S = (a.nseg <= 1 && (acc || a.epi == EPI_F32)) ? split_count(a.M, a.N, a.K, 1) : 1;
  if (S <= 1 || !spl) return run_gemm(c, a, flops);
  const int nk = (a.K + BK - 1) / BK;
  float* const out = reinterpret_cast<float*>(a.out[0]);
  const int64_t ldo = a.ld_out, M = a.M, N = a.N;
  a.epi = EPI_F32;
  a.out[0] = spl;
  a.ld_out = N;
  a.kb_split = (nk + S - 1) / S;
  a.ksplit = (nk + a.kb_split - 1) / a.kb_split;   // every range non-empty
  a.split_stride = M * N;
  WIDE_TRY(run_gemm(c, a, flops));
  const int ks = a.ksplit;
  const int blocks = (int)std::min<int64_t>((M * (N / 4) + 255) / 256, 8 * (int64_t)num_sms());
  return c.launch(0, 0, 0, [&] {
    split_reduce_kernel<<<blocks, 256, 0, c.st>>>(spl, ks, M * N, M, N, out, ldo, acc ? 1 : 0);
    return cudaGetLastError();
  });
}

// K ranges of a float32-output product of the C ABI (scal3r_ttt_gemm, and the
// GCM module's weight gradients): the count s with the least estimated time,
// rounds of work units (tiles x ranges over the SMs) times K blocks per range,
// at about 0.34 us per K block of a 128 x 256 tile on one SM (four M128 N256
// K16 MMAs at the measured rate), plus the partial planes' extra traffic
// (written by the GEMM, read by the reduce: 8 s M N bytes at about 6.5 TB/s).
// A larger count is taken only when it saves at least 3 %.  Unlike
// split_count, the count may fall as K grows: these callers size the
// workspace for the product they run (and run unsplit without it).
int api_split_count(int64_t M, int64_t N, int64_t K, int out_fp32) {
  if (!out_fp32) return 1;
  const int64_t tiles = ((M + BM - 1) / BM) * (N / BN);
  const int64_t nk = (K + BK - 1) / BK;
  const int64_t sms = num_sms();
  if (tiles <= 0 || nk < 8 || sms <= 0) return 1;
  auto est_us = [&](int64_t s) {
    const int64_t kb = (nk + s - 1) / s, ranges = (nk + kb - 1) / kb;
    const int64_t rounds = (tiles * ranges + sms - 1) / sms;
    return (double)(rounds * kb) * 0.34 + (ranges > 1 ? 8.0 * (double)ranges * M * N / 6.5e6 : 0.0);
  };
  int best = 1;
  double bt = est_us(1);
  for (int64_t s = 2; s <= 64 && nk / s >= 4; ++s) {
    const double t = est_us(s);
    if (t < 0.97 * bt) {
      bt = t;
      best = (int)s;
    }
  }
  return best;
}

}  // namespace

size_t wide_gemm_workspace_bytes(int64_t M, int64_t N, int64_t K, int out_fp32) {
  if (M <= 0 || N <= 0 || K <= 0 || N % BN != 0) return 0;
  const int s = api_split_count(M, N, K, out_fp32);
  return s > 1 ? (size_t)s * M * N * sizeof(float) : 0;
}

// C = A B^T on the GEMM kernel (bf16 operands, fp32 accumulation); see
// scal3r_ttt_gemm in the header.  A float32-output GEMM with few output tiles
// runs in K ranges into partial planes in `ws` (when it holds them) and a
// fixed-order sum.  Returns cudaErrorInvalidValue on a shape the kernel does
// not take.
// The GCM module's projections with their row steps in the epilogue
// (scal3r_gcm.h).  [q | k | v] = x Wqkv^T + bqkv as bf16 into q, k, v [T][d],
// and the sums of squares of every 64 columns of q and k into ssq [T][2d/64]
// (from the float32 values, for the per-head norms).
cudaError_t wide_gcm_qkv(const void* x, const void* wqkv, const float* bqkv, int64_t T, int d, void* q, void* k,
                         void* v, float* ssq, int* status, cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  if (d <= 0 || d % BN != 0 || T > INT32_MAX) return cudaErrorInvalidValue;
  GemmArgs g{};
  if (!make_map(&g.a[0], x, T, 1, d, d, 128) || !make_map(&g.b[0], wqkv, 3 * (int64_t)d, 1, d, d, 256))
    return cudaErrorInvalidValue;
  g.M = (int)T;
  g.N = 3 * d;
  g.K = d;
  g.epi = EPI_GCM_QKV;
  g.out[0] = q;
  g.out[1] = k;
  g.out[2] = v;
  g.out[3] = ssq;
  g.ld_out = d;
  g.ld_part = 2 * d / 64;
  g.colvec = bqkv;
  g.status = status;
  return gemm(g, st);
}

// out = alpha o (o Wo^T) + x and y = o Wo^T, both bf16 [T][d] (Eq. 5).
cudaError_t wide_gcm_gate(const void* o, const void* wo, const void* x, const float* alpha, int64_t T, int d,
                          void* out, void* y, int* status, cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  if (d <= 0 || d % BN != 0 || T > INT32_MAX) return cudaErrorInvalidValue;
  GemmArgs g{};
  if (!make_map(&g.a[0], o, T, 1, d, d, 128) || !make_map(&g.b[0], wo, d, 1, d, d, 256))
    return cudaErrorInvalidValue;
  g.M = (int)T;
  g.N = d;
  g.K = d;
  g.epi = EPI_GCM_GATE;
  g.out[0] = out;
  g.out[1] = y;
  g.in0 = static_cast<const __nv_bfloat16*>(x);
  g.ld_out = d;
  g.colvec = alpha;
  g.status = status;
  return gemm(g, st);
}

// C = A B + add: A [M][K] bf16 (rows lda apart), B given as [K][N] bf16 (rows
// ldb apart), add [M][N] bf16, C [M][N] float32.
cudaError_t wide_gemm_addin(const void* a, int64_t lda, const void* b, int64_t ldb, const void* add, float* c,
                            int64_t M, int64_t N, int64_t K, int* status, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  if (N % BN != 0 || K <= 0 || M > INT32_MAX || K > INT32_MAX) return cudaErrorInvalidValue;
  GemmArgs g{};
  if (!make_map(&g.a[0], a, M, 1, K, lda, 128) || !make_map(&g.b[0], b, K, 1, N, ldb, 64))
    return cudaErrorInvalidValue;
  g.M = (int)M;
  g.N = (int)N;
  g.K = (int)K;
  g.b_mn = 1;
  g.epi = EPI_F32_ADDIN;
  g.out[0] = c;
  g.ld_out = N;
  g.in0 = static_cast<const __nv_bfloat16*>(add);
  g.status = status;
  return gemm(g, st);
}

cudaError_t wide_gemm_bf16(const void* a, int64_t lda, int a_kmajor, const void* b, int64_t ldb, int b_kmajor, void* c,
                           int64_t ldc, int out_fp32, int accumulate, int64_t M, int64_t N, int64_t K, void* ws,
                           size_t ws_bytes, int timeout_test, int* status, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0 || N % BN != 0 || M > INT32_MAX || K > INT32_MAX) return cudaErrorInvalidValue;
  GemmArgs g{};
  const bool am = !a_kmajor, bm = !b_kmajor;
  if (!(am ? make_map(&g.a[0], a, K, 1, M, lda, 64) : make_map(&g.a[0], a, M, 1, K, lda, 128)))
    return cudaErrorInvalidValue;
  if (!(bm ? make_map(&g.b[0], b, K, 1, N, ldb, 64) : make_map(&g.b[0], b, N, 1, K, ldb, 256)))
    return cudaErrorInvalidValue;
  g.M = (int)M;
  g.N = (int)N;
  g.K = (int)K;
  g.a_mn = am;
  g.b_mn = bm;
  g.epi = out_fp32 ? (accumulate ? EPI_F32_ADD : EPI_F32) : EPI_BF16;
  g.out[0] = c;
  g.ld_out = ldc;
  g.status = status;
  g.timeout_test = timeout_test;
  const int S = api_split_count(M, N, K, out_fp32);
  const size_t need = S > 1 ? (size_t)S * M * N * sizeof(float) : 0;
  if (S <= 1 || !ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 15) != 0) return gemm(g, st);
  const int nk = (int)((K + BK - 1) / BK);
  g.epi = EPI_F32;
  g.out[0] = ws;
  g.ld_out = N;
  g.kb_split = (nk + S - 1) / S;
  g.ksplit = (nk + g.kb_split - 1) / g.kb_split;   // every range non-empty
  g.split_stride = M * N;
  cudaError_t e = gemm(g, st);
  if (e != cudaSuccess) return e;
  const int64_t work = M * (N / 4);
  const int blocks = (int)std::min<int64_t>((work + 255) / 256, 8 * (int64_t)num_sms());
  split_reduce_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const float*>(ws), g.ksplit, M * N, M, N,
                                              reinterpret_cast<float*>(c), ldc, accumulate);
  return cudaGetLastError();
}

cudaError_t prepare_wide() {
  cudaError_t e =
      cudaFuncSetAttribute(wide_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wide_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM);
  return e;
}

namespace {

// The squared-error loss's gradient (Eq. 8 with L = 1/2 |f_W(k) - v|^2): with
// u = silu(z1) o z3, e = W2 u - v and p = W2^T e (no rate yet):
//   U = gate(K), [e, eta2 e] = U W2^T - V, P = e W2, gate(K) with p -> g1 = eta1 p z3 s', g3 = eta3 p a;
//   G1 = g1^T K, G3 = g3^T K, G2 = (eta2 e)^T U.
cudaError_t key_grad_mse(const Ctx& cx, int h, int c, const __nv_bfloat16* wb, float* gr, __nv_bfloat16* const* act,
                         __nv_bfloat16* const* ex, float* spl) {
  const Shape& sh = cx.sh;
  const Params& prm = cx.prm;
  const int H = sh.H, D = sh.D, F = sh.F;
  const int64_t T = cx.pl.T;
  const __nv_bfloat16* w1 = wb;
  const __nv_bfloat16* w3 = wb + (size_t)F * D;
  const __nv_bfloat16* w2 = wb + 2 * (size_t)F * D;
  __nv_bfloat16 *pb = act[0], *g1 = act[1], *g3 = act[2], *ub = act[3];
  __nv_bfloat16 *eb = ex[0], *e2b = ex[1];
  const int64_t t0 = cx.pl.chunk_offsets[c], t1 = cx.pl.chunk_offsets[c + 1];
  const int M = (int)(t1 - t0);
  const double mfd = 2.0 * M * (double)F * D;
  {   // U = silu(K W1^T) o (K W3^T)
    GemmArgs a{};
    WIDE_MAP(tok_map(&a.a[0], prm.k, T, H, D, 128) && mat_map(&a.b[0], w1, F, D, 128) &&
             mat_map(&a.b[1], w3, F, D, 128));
    a.M = M; a.N = 2 * F; a.K = D; a.nbn = 2; a.ha = h; a.ya = (int)t0;
    a.epi = EPI_APPLY; a.out[0] = ub; a.ld_out = F;
    WIDE_TRY(run_gemm(cx, a, 2 * mfd));
  }
  {   // e = U W2^T - V and eta2 e
    GemmArgs a{};
    WIDE_MAP(mat_map(&a.a[0], ub, M, F, 128) && mat_map(&a.b[0], w2, D, F, 256));
    a.M = M; a.N = D; a.K = F;
    a.epi = EPI_MSE_E; a.out[0] = eb; a.out[1] = e2b; a.ld_out = D;
    a.in0 = reinterpret_cast<const __nv_bfloat16*>(prm.v) + ((size_t)t0 * H + h) * D; a.ld_in = (int64_t)H * D;
    set_rates(a, prm, t0, h);
    WIDE_TRY(run_gemm(cx, a, mfd));
  }
  {   // P = e W2
    GemmArgs a{};
    WIDE_MAP(mat_map(&a.a[0], eb, M, D, 128) && mat_map(&a.b[0], w2, D, F, 64));
    a.M = M; a.N = F; a.K = D; a.b_mn = 1;
    a.epi = EPI_BF16; a.out[0] = pb; a.ld_out = F;
    WIDE_TRY(run_gemm(cx, a, mfd));
  }
  {   // Z1, Z3 = K [W1; W3]^T with the gradient epilogue on p -> g1, g3
    GemmArgs a{};
    WIDE_MAP(tok_map(&a.a[0], prm.k, T, H, D, 128) && mat_map(&a.b[0], w1, F, D, 128) &&
             mat_map(&a.b[1], w3, F, D, 128));
    a.M = M; a.N = 2 * F; a.K = D; a.nbn = 2; a.ha = h; a.ya = (int)t0;
    a.epi = EPI_KEY; a.mse = 1; a.out[0] = g1; a.out[1] = g3; a.ld_out = F; a.in0 = pb;
    set_rates(a, prm, t0, h);
    WIDE_TRY(run_gemm(cx, a, 2 * mfd));
  }
  for (int j = 0; j < 2; ++j) {   // G1 = g1^T K, G3 = g3^T K
    GemmArgs a{};
    WIDE_MAP(mat_map(&a.a[0], j ? g3 : g1, M, F, 64) && tok_map(&a.b[0], prm.k, T, H, D, 64));
    a.M = F; a.N = D; a.K = M; a.a_mn = 1; a.b_mn = 1; a.hb = h; a.yb = (int)t0;
    a.epi = EPI_F32; a.out[0] = gr + (size_t)j * F * D; a.ld_out = D;
    WIDE_TRY(run_gemm_red(cx, a, mfd, spl));
  }
  {   // G2 = (eta2 e)^T U
    GemmArgs a{};
    WIDE_MAP(mat_map(&a.a[0], e2b, M, D, 64) && mat_map(&a.b[0], ub, M, F, 64));
    a.M = D; a.N = F; a.K = M; a.a_mn = 1; a.b_mn = 1;
    a.epi = EPI_F32; a.out[0] = gr + 2 * (size_t)F * D; a.ld_out = F;
    WIDE_TRY(run_gemm_red(cx, a, mfd, spl));
  }
  return cudaSuccess;
}

// The gradient G of chunk c (Eq. 8, 9) at the bf16 weights wb of head h,
// into gr (P floats, packed like the weights).  act: four [M x F] bf16 buffers;
// ex: two [M x D] bf16 buffers (squared-error loss only).
cudaError_t key_grad(const Ctx& cx, int h, int c, const __nv_bfloat16* wb, float* gr, __nv_bfloat16* const* act,
                     __nv_bfloat16* const* ex, float* spl) {
  if (cx.prm.loss == SCAL3R_LOSS_MSE) return key_grad_mse(cx, h, c, wb, gr, act, ex, spl);
  const Shape& sh = cx.sh;
  const Params& prm = cx.prm;
  const int H = sh.H, D = sh.D, F = sh.F, R = sh.R();
  const int64_t T = cx.pl.T;
  const __nv_bfloat16* w1 = wb;
  const __nv_bfloat16* w3 = wb + (size_t)F * D;
  const __nv_bfloat16* w2 = wb + 2 * (size_t)F * D;
  __nv_bfloat16 *pb = act[0], *g1 = act[1], *g3 = act[2], *ut = act[3];
  const int64_t t0 = cx.pl.chunk_offsets[c], t1 = cx.pl.chunk_offsets[c + 1];
  const int M = (int)(t1 - t0);
  const double mfd = 2.0 * M * (double)F * D;
  {   // P = V W2
    GemmArgs a{};
    WIDE_MAP(tok_map(&a.a[0], prm.v, T, H, D, 128) && mat_map(&a.b[0], w2, D, F, 64));
    a.M = M; a.N = F; a.K = D; a.b_mn = 1; a.ha = h; a.ya = (int)t0;
    a.epi = EPI_BF16; a.out[0] = pb; a.ld_out = F;
    WIDE_TRY(run_gemm(cx, a, mfd));
  }
  {   // Z1, Z3 = K [W1; W3]^T with the gradient epilogue -> g1, g3, u~
    GemmArgs a{};
    WIDE_MAP(tok_map(&a.a[0], prm.k, T, H, D, 128) && mat_map(&a.b[0], w1, F, D, 128) &&
             mat_map(&a.b[1], w3, F, D, 128));
    a.M = M; a.N = 2 * F; a.K = D; a.nbn = 2; a.ha = h; a.ya = (int)t0;
    a.epi = EPI_KEY; a.out[0] = g1; a.out[1] = g3; a.out[2] = ut; a.ld_out = F; a.in0 = pb;
    set_rates(a, prm, t0, h);
    WIDE_TRY(run_gemm(cx, a, 2 * mfd));
  }
  for (int j = 0; j < 2; ++j) {   // G1 = g1^T K, G3 = g3^T K
    GemmArgs a{};
    WIDE_MAP(mat_map(&a.a[0], j ? g3 : g1, M, F, 64) && tok_map(&a.b[0], prm.k, T, H, D, 64));
    a.M = F; a.N = D; a.K = M; a.a_mn = 1; a.b_mn = 1; a.hb = h; a.yb = (int)t0;
    a.epi = EPI_F32; a.out[0] = gr + (size_t)j * F * D; a.ld_out = D;
    WIDE_TRY(run_gemm_red(cx, a, mfd, spl));
  }
  {   // G2 = V^T u~
    GemmArgs a{};
    WIDE_MAP(tok_map(&a.a[0], prm.v, T, H, D, 64) && mat_map(&a.b[0], ut, M, F, 64));
    a.M = D; a.N = F; a.K = M; a.a_mn = 1; a.b_mn = 1; a.ha = h; a.ya = (int)t0;
    a.epi = EPI_F32; a.out[0] = gr + 2 * (size_t)F * D; a.ld_out = F;
    WIDE_TRY(run_gemm_red(cx, a, mfd, spl));
  }
  return cudaSuccess;
}

// One chunk's gradient step on chain (s, h): W (master wm, bf16 wb) becomes
// normalise(W - G) in place; optionally the checkpoint, the pre-normalisation
// row norms and w_final are written.  gr: the gradient buffer (P floats).
cudaError_t key_update(const Ctx& cx, int h, int c, float* wm, __nv_bfloat16* wb, const float* rho, float* gr,
                       __nv_bfloat16* const* act, __nv_bfloat16* const* ex, float* spl, float* ck, float* wn,
                       float* wf) {
  WIDE_TRY(key_grad(cx, h, c, wb, gr, act, ex, spl));
  const Shape& sh = cx.sh;
  const Params& prm = cx.prm;
  const int D = sh.D, F = sh.F, R = sh.R();
  return cx.launch(1, 0, 0, [&] {   // update and normalise
    wide_update_kernel<<<R, ROW_THREADS, 0, cx.st>>>(wm, gr, wb, rho, ck, wn, wf, D, F, prm.norm, prm.eps);
    return cudaGetLastError();
  });
}

}  // namespace

// The forward of every chain, chunk after chunk (see the file comment).
// `launch` wraps each launch (profiling); kind 0 = GEMM, 1 = update / prep.
cudaError_t wide_forward(const Plan& pl, const Shape& sh, const Params& prm, int ckpt_every, void* ws,
                         const LaunchFn& launch, cudaStream_t st) {
  const Ctx cx{pl, sh, prm, launch, st};
  const int H = sh.H, D = sh.D, F = sh.F;
  const size_t P = (size_t)sh.P();
  const int R = sh.R();
  WideBufs w;
  layout_bytes(pl, sh, false, ckpt_every, prm.loss == SCAL3R_LOSS_MSE, prm.lr_mat, &w, ws);
  __nv_bfloat16* pb = w.act[0];
  const int64_t T = pl.T;
  const __nv_bfloat16* w1 = w.wb;
  const __nv_bfloat16* w3 = w.wb + (size_t)F * D;
  const __nv_bfloat16* w2 = w.wb + 2 * (size_t)F * D;
  for (int s = 0; s < pl.S; ++s) {
    for (int h = 0; h < H; ++h) {
      const float* w0 = prm.w0 + (size_t)s * prm.w0_seq_stride + (size_t)h * P;
      WIDE_TRY(launch(1, 0, 0, [&] {
        wide_prep_kernel<<<R, ROW_THREADS, 0, st>>>(w0, w.wm, w.wb, w.rho, D, F, prm.norm);
        return cudaGetLastError();
      }));
      const int c0 = pl.seq_chunk_ptr[s], c1 = pl.seq_chunk_ptr[s + 1];
      if (c1 == c0 && prm.w_final)   // a sequence without chunks keeps its initial weights
        WIDE_TRY(cudaMemcpyAsync(prm.w_final + ((size_t)s * H + h) * P, w0, P * sizeof(float),
                                 cudaMemcpyDeviceToDevice, st));
      for (int c = c0; c < c1; ++c) {
        const int64_t t0 = pl.chunk_offsets[c], t1 = pl.chunk_offsets[c + 1];
        const int M = (int)(t1 - t0);
        const double mfd = 2.0 * M * (double)F * D;
        const int64_t slot = wide_ckpt_slot(pl, s, c - c0 + 1, ckpt_every);
        float* ck = (prm.w_ckpt && slot >= 0) ? prm.w_ckpt + ((size_t)slot * H + h) * P : nullptr;
        float* wn = prm.wnorm ? prm.wnorm + ((size_t)c * H + h) * R : nullptr;
        float* wf = (prm.w_final && c == c1 - 1) ? prm.w_final + ((size_t)s * H + h) * P : nullptr;
        WIDE_TRY(key_update(cx, h, c, w.wm, w.wb, w.rho, w.gr, w.act, w.ex, w.spl, ck, wn, wf));
        {   // apply: h = silu(Q W1^T) o (Q W3^T)
          GemmArgs a{};
          WIDE_MAP(tok_map(&a.a[0], prm.q, T, H, D, 128) && mat_map(&a.b[0], w1, F, D, 128) &&
                   mat_map(&a.b[1], w3, F, D, 128));
          a.M = M; a.N = 2 * F; a.K = D; a.nbn = 2; a.ha = h; a.ya = (int)t0;
          a.epi = EPI_APPLY; a.out[0] = pb; a.ld_out = F;
          WIDE_TRY(run_gemm(cx, a, 2 * mfd));
        }
        {   // o = h W2^T
          GemmArgs a{};
          WIDE_MAP(mat_map(&a.a[0], pb, M, F, 128) && mat_map(&a.b[0], w2, D, F, 256));
          a.M = M; a.N = D; a.K = F;
          a.epi = EPI_BF16; a.out[0] = reinterpret_cast<__nv_bfloat16*>(prm.o) + ((size_t)t0 * H + h) * D;
          a.ld_out = (int64_t)H * D;
          WIDE_TRY(run_gemm(cx, a, mfd));
        }
      }
    }
  }
  return cudaSuccess;
}

// ---- Global Context Synchronisation (Sec. 4.2, Eq. 10) on the wide path: a
// chunk step in local parts; every sequence holds one chunk.

namespace {

// w_out = normalise(w - g) per row, targets from w0 (one block per row).
__global__ void __launch_bounds__(ROW_THREADS) wide_gcs_update_kernel(const float* __restrict__ w,
                                                                      const float* __restrict__ g,
                                                                      const float* __restrict__ w0,
                                                                      float* __restrict__ w_out, float* wnorm, int D,
                                                                      int F, int norm, float eps) {
  __shared__ float red[ROW_THREADS / 32 + 1];
  size_t off;
  int len;
  row_geometry(blockIdx.x, D, F, off, len);
  float ss = 0.f, st = 0.f;
  for (int i = 4 * threadIdx.x; i < len; i += 4 * ROW_THREADS) {
    const float4 a = *reinterpret_cast<const float4*>(w + off + i);
    const float4 b = *reinterpret_cast<const float4*>(g + off + i);
    const float4 t = *reinterpret_cast<const float4*>(w0 + off + i);
    const float4 x = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    ss += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
    st += t.x * t.x + t.y * t.y + t.z * t.z + t.w * t.w;
  }
  ss = block_sum(ss, red);
  st = block_sum(st, red);
  const float n = sqrtf(ss);
  const float rho = (norm == SCAL3R_NORM_UNIT) ? 1.f : sqrtf(st);
  const float scale = (norm == SCAL3R_NORM_NONE) ? 1.f : rho / fmaxf(n, eps);
  if (threadIdx.x == 0 && wnorm) wnorm[blockIdx.x] = n;
  for (int i = 4 * threadIdx.x; i < len; i += 4 * ROW_THREADS) {
    const float4 a = *reinterpret_cast<const float4*>(w + off + i);
    const float4 b = *reinterpret_cast<const float4*>(g + off + i);
    *reinterpret_cast<float4*>(w_out + off + i) =
        make_float4((a.x - b.x) * scale, (a.y - b.y) * scale, (a.z - b.z) * scale, (a.w - b.w) * scale);
  }
}

}  // namespace

// grad[s, h] = G of sequence s's chunk at w[s, h] (0 without a chunk).
cudaError_t wide_partial_grad(const Plan& pl, const Shape& sh, const Params& prm, float* grad, void* ws,
                              const LaunchFn& launch, cudaStream_t st) {
  const Ctx cx{pl, sh, prm, launch, st};
  const int H = sh.H, D = sh.D, F = sh.F, R = sh.R();
  const size_t P = (size_t)sh.P();
  WideBufs w;
  layout_bytes(pl, sh, false, 1, prm.loss == SCAL3R_LOSS_MSE, prm.lr_mat, &w, ws);
  for (int s = 0; s < pl.S; ++s) {
    for (int h = 0; h < H; ++h) {
      float* gout = grad + ((size_t)s * H + h) * P;
      const int c0 = pl.seq_chunk_ptr[s], c1 = pl.seq_chunk_ptr[s + 1];
      if (c1 == c0) {
        WIDE_TRY(cudaMemsetAsync(gout, 0, P * sizeof(float), st));
        continue;
      }
      const float* wsrc = prm.w0 + (size_t)s * prm.w0_seq_stride + (size_t)h * P;
      WIDE_TRY(launch(1, 0, 0, [&] {
        wide_prep_kernel<<<R, ROW_THREADS, 0, st>>>(wsrc, w.wm, w.wb, nullptr, D, F, prm.norm);
        return cudaGetLastError();
      }));
      WIDE_TRY(key_grad(cx, h, c0, w.wb, gout, w.act, w.ex, w.spl));
    }
  }
  return cudaSuccess;
}

// w_out[s, h] = normalise(w[s, h] - grad[s, h]) with the targets of w0.
cudaError_t wide_apply_update(const Shape& sh, const Params& prm, int S, const float* w, int64_t w_stride,
                              const float* grad, float* w_out, float* wnorm, const LaunchFn& launch, cudaStream_t st) {
  const int H = sh.H, D = sh.D, F = sh.F, R = sh.R();
  const size_t P = (size_t)sh.P();
  for (int s = 0; s < S; ++s)
    for (int h = 0; h < H; ++h) {
      const size_t chain = (size_t)s * H + h;
      WIDE_TRY(launch(1, 0, 0, [&] {
        wide_gcs_update_kernel<<<R, ROW_THREADS, 0, st>>>(w + (size_t)s * w_stride + (size_t)h * P, grad + chain * P,
                                                          prm.w0 + (size_t)s * prm.w0_seq_stride + (size_t)h * P,
                                                          w_out + chain * P, wnorm ? wnorm + chain * R : nullptr, D, F,
                                                          prm.norm, prm.eps);
        return cudaGetLastError();
      }));
    }
  return cudaSuccess;
}

// o = f_w(q) for every sequence's chunk, w[s, h] given in (prm.w0, stride).
cudaError_t wide_apply(const Plan& pl, const Shape& sh, const Params& prm, void* ws, const LaunchFn& launch,
                       cudaStream_t st) {
  const Ctx cx{pl, sh, prm, launch, st};
  const int H = sh.H, D = sh.D, F = sh.F, R = sh.R();
  const size_t P = (size_t)sh.P();
  WideBufs w;
  layout_bytes(pl, sh, false, 1, prm.loss == SCAL3R_LOSS_MSE, prm.lr_mat, &w, ws);
  const int64_t T = pl.T;
  const __nv_bfloat16 *w1 = w.wb, *w3 = w.wb + (size_t)F * D, *w2 = w.wb + 2 * (size_t)F * D;
  __nv_bfloat16* pb = w.act[0];
  for (int s = 0; s < pl.S; ++s)
    for (int h = 0; h < H; ++h) {
      const int c0 = pl.seq_chunk_ptr[s], c1 = pl.seq_chunk_ptr[s + 1];
      if (c1 == c0) continue;
      const float* wsrc = prm.w0 + (size_t)s * prm.w0_seq_stride + (size_t)h * P;
      WIDE_TRY(launch(1, 0, 0, [&] {
        wide_prep_kernel<<<R, ROW_THREADS, 0, st>>>(wsrc, w.wm, w.wb, nullptr, D, F, prm.norm);
        return cudaGetLastError();
      }));
      const int64_t t0 = pl.chunk_offsets[c0];
      const int M = (int)(pl.chunk_offsets[c0 + 1] - t0);
      const double mfd = 2.0 * M * (double)F * D;
      {
        GemmArgs a{};
        WIDE_MAP(tok_map(&a.a[0], prm.q, T, H, D, 128) && mat_map(&a.b[0], w1, F, D, 128) &&
                 mat_map(&a.b[1], w3, F, D, 128));
        a.M = M; a.N = 2 * F; a.K = D; a.nbn = 2; a.ha = h; a.ya = (int)t0;
        a.epi = EPI_APPLY; a.out[0] = pb; a.ld_out = F;
        WIDE_TRY(run_gemm(cx, a, 2 * mfd));
      }
      {
        GemmArgs a{};
        WIDE_MAP(mat_map(&a.a[0], pb, M, F, 128) && mat_map(&a.b[0], w2, D, F, 256));
        a.M = M; a.N = D; a.K = F;
        a.epi = EPI_BF16; a.out[0] = reinterpret_cast<__nv_bfloat16*>(prm.o) + ((size_t)t0 * H + h) * D;
        a.ld_out = (int64_t)H * D;
        WIDE_TRY(run_gemm(cx, a, mfd));
      }
    }
  return cudaSuccess;
}

namespace {

// Update VJP of one chunk under the squared-error loss (Eq. 8 with
// L = 1/2 |f_W(k) - v|^2), at the bf16 weights w.wb with -R in w.nrb; e = W2 u - v
// and p = W2^T e carry no rate, eta1, eta3, eta2 are the rates of W1, W3, W2:
//   [U, eta2 U] = gate(K), e = U W2^T - V, P = e W2, N = e (-R2);
//   gate [W1; W3; -R1; -R3] with p, N -> dp = eta1 dg1 z3 s' + eta3 dg3 a, g1, g3 and the
//     d eta partials (p z3 s' . dg1, p a . dg3, N . u)   (dg = -R k);
//   dE = [eta2 U, dP] [-R2, W2]^T -> dY = dE, dv = -dE;  dU = eta2 N + dY W2;
//   gate again with p, du -> dz1, dz3;  dk = [dz1 dz3 g1 g3] [W1; W3; -R1; -R3];
//   lam1 += dz1^T K, lam3 += dz3^T K, lam2 += e^T dP + dY^T U.
// The d eta partials are left in w.part.
cudaError_t update_vjp_mse(const Ctx& cx, int h, int64_t t0, int M, const WideBufs& w, float* lam1, float* lam3,
                           float* lam2) {
  const Shape& sh = cx.sh;
  const Params& prm = cx.prm;
  const int H = sh.H, D = sh.D, F = sh.F;
  const int64_t T = cx.pl.T;
  const size_t FD = (size_t)F * D;
  const __nv_bfloat16 *w1 = w.wb, *w3 = w.wb + FD, *w2 = w.wb + 2 * FD;
  const __nv_bfloat16 *r1 = w.nrb, *r3 = w.nrb + FD, *r2 = w.nrb + 2 * FD;   // -R
  // du overwrites eta2 U once dE is formed, dz3 overwrites N once du is formed
  __nv_bfloat16 *ub = w.act[0], *pb = w.act[1], *nb = w.act[2], *dp = w.act[3], *g1 = w.act[4], *g3 = w.act[5],
                *u2 = w.act[6], *du = w.act[6], *dz1 = w.act[7], *dz3 = w.act[2];
  __nv_bfloat16 *eb = w.ex[0], *dy = w.ex[1];
  const double mfd = 2.0 * M * (double)F * D;
  {   // U and eta2 U
    GemmArgs a{};
    WIDE_MAP(tok_map(&a.a[0], prm.k, T, H, D, 128) && mat_map(&a.b[0], w1, F, D, 128) &&
             mat_map(&a.b[1], w3, F, D, 128));
    a.M = M; a.N = 2 * F; a.K = D; a.nbn = 2; a.ha = h; a.ya = (int)t0;
    a.epi = EPI_APPLY2; a.out[0] = ub; a.out[1] = u2; a.ld_out = F;
    set_rates(a, prm, t0, h);
    WIDE_TRY(run_gemm(cx, a, 2 * mfd));
  }
  {   // e = U W2^T - V
    GemmArgs a{};
    WIDE_MAP(mat_map(&a.a[0], ub, M, F, 128) && mat_map(&a.b[0], w2, D, F, 256));
    a.M = M; a.N = D; a.K = F;
    a.epi = EPI_MSE_E; a.out[0] = eb; a.ld_out = D;
    a.in0 = reinterpret_cast<const __nv_bfloat16*>(prm.v) + ((size_t)t0 * H + h) * D; a.ld_in = (int64_t)H * D;
    WIDE_TRY(run_gemm(cx, a, mfd));
  }
  for (int i = 0; i < 2; ++i) {   // P = e W2, N = e (-R2)
    GemmArgs a{};
    WIDE_MAP(mat_map(&a.a[0], eb, M, D, 128) && mat_map(&a.b[0], i ? r2 : w2, D, F, 64));
    a.M = M; a.N = F; a.K = D; a.b_mn = 1;
    a.epi = EPI_BF16; a.out[0] = i ? nb : pb; a.ld_out = F;
    WIDE_TRY(run_gemm(cx, a, mfd));
  }
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      {   // dE = -eta2 U R2^T + dP W2^T -> dY, dv
        GemmArgs a{};
        WIDE_MAP(mat_map(&a.a[0], u2, M, F, 128) && mat_map(&a.a[1], dp, M, F, 128) &&
                 mat_map(&a.b[0], r2, D, F, 256) && mat_map(&a.b[1], w2, D, F, 256));
        a.M = M; a.N = D; a.K = 2 * F; a.kseg = F; a.nseg = 2;
        a.epi = EPI_MSE_DE; a.out[0] = dy; a.ld_out = D;
        a.out[1] = reinterpret_cast<__nv_bfloat16*>(prm.dv) + ((size_t)t0 * H + h) * D; a.ld_out1 = (int64_t)H * D;
        WIDE_TRY(run_gemm(cx, a, 2 * mfd));
      }
      {   // dU = eta2 N + dY W2
        GemmArgs a{};
        WIDE_MAP(mat_map(&a.a[0], dy, M, D, 128) && mat_map(&a.b[0], w2, D, F, 64));
        a.M = M; a.N = F; a.K = D; a.b_mn = 1;
        a.epi = EPI_ADD_BF16; a.out[0] = du; a.ld_out = F; a.in0 = nb;
        set_rates(a, prm, t0, h);
        WIDE_TRY(run_gemm(cx, a, mfd));
      }
    }
    // gate [W1; W3; -R1; -R3] on k: pass 0 -> dp, g1, g3, partials; pass 1 -> dz1, dz3
    GemmArgs a{};
    WIDE_MAP(tok_map(&a.a[0], prm.k, T, H, D, 128) && mat_map(&a.b[0], w1, F, D, 64) &&
             mat_map(&a.b[1], w3, F, D, 64) && mat_map(&a.b[2], r1, F, D, 64) && mat_map(&a.b[3], r3, F, D, 64));
    a.M = M; a.N = 4 * F; a.K = D; a.nbn = 4; a.ha = h; a.ya = (int)t0;
    a.ld_out = F; a.in0 = pb;
    set_rates(a, prm, t0, h);
    if (pass == 0) {
      a.epi = EPI_BKEY_MSE1; a.out[0] = dp; a.out[1] = g1; a.out[2] = g3; a.in1 = nb;
      a.part = w.part; a.ld_part = deta_parts(sh, prm.lr_mat);
    } else {
      a.epi = EPI_BKEY_MSE2; a.out[0] = dz1; a.out[1] = dz3; a.in1 = du;
    }
    WIDE_TRY(run_gemm(cx, a, 4 * mfd));
  }
  {   // dk = [dz1 dz3 g1 g3] [W1; W3; -R1; -R3]
    GemmArgs a{};
    WIDE_MAP(mat_map(&a.a[0], dz1, M, F, 128) && mat_map(&a.a[1], dz3, M, F, 128) &&
             mat_map(&a.a[2], g1, M, F, 128) && mat_map(&a.a[3], g3, M, F, 128) &&
             mat_map(&a.b[0], w1, F, D, 64) && mat_map(&a.b[1], w3, F, D, 64) &&
             mat_map(&a.b[2], r1, F, D, 64) && mat_map(&a.b[3], r3, F, D, 64));
    a.M = M; a.N = D; a.K = 4 * F; a.kseg = F; a.nseg = 4; a.b_mn = 1;
    a.epi = EPI_BF16; a.out[0] = reinterpret_cast<__nv_bfloat16*>(prm.dk) + ((size_t)t0 * H + h) * D;
    a.ld_out = (int64_t)H * D;
    WIDE_TRY(run_gemm(cx, a, 4 * mfd));
  }
  for (int i = 0; i < 2; ++i) {   // lam1 += dz1^T K, lam3 += dz3^T K
    GemmArgs a{};
    WIDE_MAP(mat_map(&a.a[0], i ? dz3 : dz1, M, F, 64) && tok_map(&a.b[0], prm.k, T, H, D, 64));
    a.M = F; a.N = D; a.K = M; a.a_mn = 1; a.b_mn = 1; a.hb = h; a.yb = (int)t0;
    a.epi = EPI_F32_ADD; a.out[0] = i ? lam3 : lam1; a.ld_out = D;
    WIDE_TRY(run_gemm_red(cx, a, mfd, w.spl));
  }
  {   // lam2 += e^T dP + dY^T U: one reduction over both token segments
    const int kseg = (M + BK - 1) / BK * BK;
    GemmArgs a{};
    WIDE_MAP(mat_map(&a.a[0], eb, M, D, 64) && mat_map(&a.a[1], dy, M, D, 64) && mat_map(&a.b[0], dp, M, F, 64) &&
             mat_map(&a.b[1], ub, M, F, 64));
    a.M = D; a.N = F; a.K = 2 * kseg; a.kseg = kseg; a.nseg = 2; a.a_mn = 1; a.b_mn = 1;
    a.epi = EPI_F32_ADD; a.out[0] = lam2; a.ld_out = F;
    WIDE_TRY(run_gemm(cx, a, 2 * mfd));
  }
  return cudaSuccess;
}

}  // namespace

// The backward of every chain: for j = n .. 0 (n = the sequence's chunks), at
// W_j (W0, or the checkpoint after update j-1):
//   apply VJP of chunk j-1:   du = W2^T d_o, gate -> dzq1, dzq3, uq;
//                             dq = dzq1 W1 + dzq3 W3;  lam += [dzq1^T Q, dzq3^T Q, d_O^T uq]
//   update VJP of chunk j with R = dL/dW~_{j+1}:  praw = W2^T v, ndu = -R2^T v,
//                             gate [W1; W3; -R1; -R3] -> dz1, dz3, g1, g3, -dp, -eta2 u, d eta
//                             (dp = eta1 dg1 z3 s' + eta3 dg3 a with dg = -R k);
//                             dk = [dz1 dz3 g1 g3] [W1; W3; -R1; -R3], dv = [-dp, -eta2 u] [W2^T; -R2^T];
//                             lam += R + [dz1^T K, dz3^T K, V^T (-dp)]
//   (the squared-error loss: update_vjp_mse)
//   normalisation VJP of update j-1 (R for the next step), or dW0 at j = 0.
cudaError_t wide_backward(const Plan& pl, const Shape& sh, const Params& prm, int ckpt_every, void* ws,
                          const LaunchFn& launch, cudaStream_t st) {
  const Ctx cx{pl, sh, prm, launch, st};
  const int H = sh.H, D = sh.D, F = sh.F;
  const size_t P = (size_t)sh.P();
  const int R = sh.R();
  WideBufs w;
  const bool mse = prm.loss == SCAL3R_LOSS_MSE;
  layout_bytes(pl, sh, true, ckpt_every, mse, prm.lr_mat, &w, ws);
  const int nck = ckpt_every > 1 ? ckpt_every : 1;
  const int64_t T = pl.T;
  const size_t FD = (size_t)F * D;
  const __nv_bfloat16 *w1 = w.wb, *w3 = w.wb + FD, *w2 = w.wb + 2 * FD;
  const __nv_bfloat16 *r1 = w.nrb, *r3 = w.nrb + FD, *r2 = w.nrb + 2 * FD;   // -R
  float *lam1 = w.wm, *lam3 = w.wm + FD, *lam2 = w.wm + 2 * FD;
  const int nparts = deta_parts(sh, prm.lr_mat);
  for (int s = 0; s < pl.S; ++s) {
    for (int h = 0; h < H; ++h) {
      const float* w0 = prm.w0 + (size_t)s * prm.w0_seq_stride + (size_t)h * P;
      float* dw0 = prm.dw0 + (size_t)s * prm.w0_seq_stride + (size_t)h * P;
      const bool acc_dw0 = prm.w0_seq_stride == 0 && s > 0;
      WIDE_TRY(launch(1, 0, 0, [&] {
        wide_bprep_kernel<<<R, ROW_THREADS, 0, st>>>(w0, w.rho, w.drho, D, F, prm.norm);
        return cudaGetLastError();
      }));
      const int c0 = pl.seq_chunk_ptr[s], c1 = pl.seq_chunk_ptr[s + 1];
      const int n = c1 - c0;
      // segments [j0, j1] from the last: W_j0 is stored (or w0); with sparse
      // checkpoints W_j0+1 .. W_j1 are recomputed from it first, by the
      // forward's own gradient steps (the same kernels on the same inputs,
      // so bitwise the weights the forward had)
      for (int j0 = (n / nck) * nck; j0 >= 0; j0 -= nck) {
      const int j1 = std::min(j0 + nck - 1, n);
      const float* wbase = (j0 == 0) ? w0 : prm.w_ckpt_in + ((size_t)wide_ckpt_slot(pl, s, j0, nck) * H + h) * P;
      if (j1 > j0) {
        WIDE_TRY(launch(1, 0, 0, [&] {
          wide_prep_kernel<<<R, ROW_THREADS, 0, st>>>(wbase, w.wm, w.wb, nullptr, D, F, prm.norm);
          return cudaGetLastError();
        }));
        for (int jj = j0; jj < j1; ++jj)
          WIDE_TRY(key_update(cx, h, c0 + jj, w.wm, w.wb, w.rho, w.rgr, w.act, w.ex, w.spl,
                              w.seg + (size_t)(jj - j0) * P, nullptr, nullptr));
      }
      for (int j = j1; j >= j0; --j) {
        const float* wj = (j == j0) ? wbase : w.seg + (size_t)(j - j0 - 1) * P;
        const bool key = j < n;
        WIDE_TRY(launch(1, 0, 0, [&] {
          wide_bstep_setup_kernel<<<4 * num_sms(), 256, 0, st>>>(wj, key ? w.gr : nullptr, w.wb, w.nrb, w.wm, P);
          return cudaGetLastError();
        }));
        if (j >= 1) {   // apply VJP of chunk j-1
          const int c = c0 + j - 1;
          const int64_t t0 = pl.chunk_offsets[c];
          const int M = (int)(pl.chunk_offsets[c + 1] - t0);
          const double mfd = 2.0 * M * (double)F * D;
          __nv_bfloat16 *du = w.act[0], *dz1 = w.act[1], *dz3 = w.act[2], *uq = w.act[3];
          {   // du = d_o W2 (token rows)
            GemmArgs a{};
            WIDE_MAP(tok_map(&a.a[0], prm.d_o, T, H, D, 128) && mat_map(&a.b[0], w2, D, F, 64));
            a.M = M; a.N = F; a.K = D; a.b_mn = 1; a.ha = h; a.ya = (int)t0;
            a.epi = EPI_BF16; a.out[0] = du; a.ld_out = F;
            WIDE_TRY(run_gemm(cx, a, mfd));
          }
          {   // gate on q -> dzq1, dzq3, uq
            GemmArgs a{};
            WIDE_MAP(tok_map(&a.a[0], prm.q, T, H, D, 128) && mat_map(&a.b[0], w1, F, D, 128) &&
                     mat_map(&a.b[1], w3, F, D, 128));
            a.M = M; a.N = 2 * F; a.K = D; a.nbn = 2; a.ha = h; a.ya = (int)t0;
            a.epi = EPI_BAPPLY; a.out[0] = dz1; a.out[1] = dz3; a.out[2] = uq; a.ld_out = F; a.in0 = du;
            WIDE_TRY(run_gemm(cx, a, 2 * mfd));
          }
          {   // dq = dzq1 W1 + dzq3 W3
            GemmArgs a{};
            WIDE_MAP(mat_map(&a.a[0], dz1, M, F, 128) && mat_map(&a.a[1], dz3, M, F, 128) &&
                     mat_map(&a.b[0], w1, F, D, 64) && mat_map(&a.b[1], w3, F, D, 64));
            a.M = M; a.N = D; a.K = 2 * F; a.kseg = F; a.nseg = 2; a.b_mn = 1;
            a.epi = EPI_BF16; a.out[0] = reinterpret_cast<__nv_bfloat16*>(prm.dq) + ((size_t)t0 * H + h) * D;
            a.ld_out = (int64_t)H * D;
            WIDE_TRY(run_gemm(cx, a, 2 * mfd));
          }
          for (int i = 0; i < 2; ++i) {   // lam1 += dzq1^T Q, lam3 += dzq3^T Q
            GemmArgs a{};
            WIDE_MAP(mat_map(&a.a[0], i ? dz3 : dz1, M, F, 64) && tok_map(&a.b[0], prm.q, T, H, D, 64));
            a.M = F; a.N = D; a.K = M; a.a_mn = 1; a.b_mn = 1; a.hb = h; a.yb = (int)t0;
            a.epi = EPI_F32_ADD; a.out[0] = i ? lam3 : lam1; a.ld_out = D;
            WIDE_TRY(run_gemm_red(cx, a, mfd, w.spl));
          }
          {   // lam2 += d_O^T uq
            GemmArgs a{};
            WIDE_MAP(tok_map(&a.a[0], prm.d_o, T, H, D, 64) && mat_map(&a.b[0], uq, M, F, 64));
            a.M = D; a.N = F; a.K = M; a.a_mn = 1; a.b_mn = 1; a.ha = h; a.ya = (int)t0;
            a.epi = EPI_F32_ADD; a.out[0] = lam2; a.ld_out = F;
            WIDE_TRY(run_gemm_red(cx, a, mfd, w.spl));
          }
        }
        if (key && mse) {   // update VJP of chunk j, squared-error loss
          const int c = c0 + j;
          const int64_t t0 = pl.chunk_offsets[c];
          const int M = (int)(pl.chunk_offsets[c + 1] - t0);
          WIDE_TRY(update_vjp_mse(cx, h, t0, M, w, lam1, lam3, lam2));
          WIDE_TRY(chunk_deta(cx, w.part, t0, h, M));
        } else if (key) {   // update VJP of chunk j
          const int c = c0 + j;
          const int64_t t0 = pl.chunk_offsets[c];
          const int M = (int)(pl.chunk_offsets[c + 1] - t0);
          const double mfd = 2.0 * M * (double)F * D;
          __nv_bfloat16 *pr = w.act[0], *nd = w.act[1];
          __nv_bfloat16 *dz1 = w.act[2], *dz3 = w.act[3], *g1 = w.act[4], *g3 = w.act[5], *dpe = w.act[6],
                        *ue = w.act[7];
          for (int i = 0; i < 2; ++i) {   // praw = V W2, ndu = V (-R2)
            GemmArgs a{};
            WIDE_MAP(tok_map(&a.a[0], prm.v, T, H, D, 128) && mat_map(&a.b[0], i ? r2 : w2, D, F, 64));
            a.M = M; a.N = F; a.K = D; a.b_mn = 1; a.ha = h; a.ya = (int)t0;
            a.epi = EPI_BF16; a.out[0] = i ? nd : pr; a.ld_out = F;
            WIDE_TRY(run_gemm(cx, a, mfd));
          }
          {   // gate [W1; W3; -R1; -R3] on k -> the six factors and d eta partials
            GemmArgs a{};
            WIDE_MAP(tok_map(&a.a[0], prm.k, T, H, D, 128) && mat_map(&a.b[0], w1, F, D, 64) &&
                     mat_map(&a.b[1], w3, F, D, 64) && mat_map(&a.b[2], r1, F, D, 64) &&
                     mat_map(&a.b[3], r3, F, D, 64));
            a.M = M; a.N = 4 * F; a.K = D; a.nbn = 4; a.ha = h; a.ya = (int)t0;
            a.epi = EPI_BKEY;
            a.out[0] = dz1; a.out[1] = dz3; a.out[2] = g1; a.out[3] = g3; a.out[4] = dpe; a.out[5] = ue;
            a.ld_out = F; a.in0 = pr; a.in1 = nd;
            set_rates(a, prm, t0, h);
            a.part = w.part; a.ld_part = nparts;
            WIDE_TRY(run_gemm(cx, a, 4 * mfd));
          }
          {   // dk = [dz1 dz3 g1 g3] [W1; W3; -R1; -R3]
            GemmArgs a{};
            WIDE_MAP(mat_map(&a.a[0], dz1, M, F, 128) && mat_map(&a.a[1], dz3, M, F, 128) &&
                     mat_map(&a.a[2], g1, M, F, 128) && mat_map(&a.a[3], g3, M, F, 128) &&
                     mat_map(&a.b[0], w1, F, D, 64) && mat_map(&a.b[1], w3, F, D, 64) &&
                     mat_map(&a.b[2], r1, F, D, 64) && mat_map(&a.b[3], r3, F, D, 64));
            a.M = M; a.N = D; a.K = 4 * F; a.kseg = F; a.nseg = 4; a.b_mn = 1;
            a.epi = EPI_BF16; a.out[0] = reinterpret_cast<__nv_bfloat16*>(prm.dk) + ((size_t)t0 * H + h) * D;
            a.ld_out = (int64_t)H * D;
            WIDE_TRY(run_gemm(cx, a, 4 * mfd));
          }
          {   // dv = [-dp, -eta2 u] [W2^T; -R2^T]
            GemmArgs a{};
            WIDE_MAP(mat_map(&a.a[0], dpe, M, F, 128) && mat_map(&a.a[1], ue, M, F, 128) &&
                     mat_map(&a.b[0], w2, D, F, 256) && mat_map(&a.b[1], r2, D, F, 256));
            a.M = M; a.N = D; a.K = 2 * F; a.kseg = F; a.nseg = 2;
            a.epi = EPI_BF16; a.out[0] = reinterpret_cast<__nv_bfloat16*>(prm.dv) + ((size_t)t0 * H + h) * D;
            a.ld_out = (int64_t)H * D;
            WIDE_TRY(run_gemm(cx, a, 2 * mfd));
          }
          for (int i = 0; i < 2; ++i) {   // lam1 += dz1^T K, lam3 += dz3^T K
            GemmArgs a{};
            WIDE_MAP(mat_map(&a.a[0], i ? dz3 : dz1, M, F, 64) && tok_map(&a.b[0], prm.k, T, H, D, 64));
            a.M = F; a.N = D; a.K = M; a.a_mn = 1; a.b_mn = 1; a.hb = h; a.yb = (int)t0;
            a.epi = EPI_F32_ADD; a.out[0] = i ? lam3 : lam1; a.ld_out = D;
            WIDE_TRY(run_gemm_red(cx, a, mfd, w.spl));
          }
          {   // lam2 += V^T (-dp)
            GemmArgs a{};
            WIDE_MAP(tok_map(&a.a[0], prm.v, T, H, D, 64) && mat_map(&a.b[0], dpe, M, F, 64));
            a.M = D; a.N = F; a.K = M; a.a_mn = 1; a.b_mn = 1; a.ha = h; a.ya = (int)t0;
            a.epi = EPI_F32_ADD; a.out[0] = lam2; a.ld_out = F;
            WIDE_TRY(run_gemm_red(cx, a, mfd, w.spl));
          }
          WIDE_TRY(chunk_deta(cx, w.part, t0, h, M));
        }
        // normalisation VJP of update j-1 -> R, or dW0
        const float* wn = (j >= 1) ? prm.wnorm_in + ((size_t)(c0 + j - 1) * H + h) * R : nullptr;
        WIDE_TRY(launch(1, 0, 0, [&] {
          wide_bupdate_kernel<<<R, ROW_THREADS, 0, st>>>(w.wm, wj, wn, w.rho, w.drho, w.gr, w0,
                                                         j == 0 ? dw0 : nullptr, acc_dw0 ? 1 : 0, D, F, prm.norm,
                                                         prm.eps);
          return cudaGetLastError();
        }));
      }
      }
    }
  }
  return cudaSuccess;
}

#ifdef SCAL3R_DEBUG_BOUNDS
cudaError_t wide_upload_bounds(const BoundsTable& t, cudaStream_t st) { return upload_bounds_table(t, st); }
#endif

}  // namespace scal3r
