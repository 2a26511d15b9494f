// Tensor-core (tcgen05) path: batched GEMMs over BF16 term pairs with the
// fused RK4 stage-combine / forward-Euler-correction epilogues.
//
// Every matrix product of the flows (Section 2, Examples 1 and 2: A Y,
// (I - A) Y, Y P; the square-root flow's Y Y) is computed as
//     D = sum_p L_{a_p} R_{b_p}^T
// where L_a / R_b are the BF16 terms of the left operand (row-major, "L form")
// and of the transposed right operand ("R form"), x = x_0 + x_1 + x_2 with
// x_{k+1} the BF16 rounding of what x_0..x_k leave out.
//
// Accumulation.  The tensor core adds each MMA's products into its float32
// accumulator with truncation toward zero; over the n/16 instructions of a
// long reduction that bias reaches ~1e-5 at n = 2048.  So the main product
// L_0 R_0^T is accumulated one 64-wide k-block at a time in a fresh TMEM chunk
// and drained into float32 registers (round-to-nearest adds); the correction
// products (2^-8 smaller, so their bias is negligible) accumulate in a second
// TMEM buffer for the whole tile.
//
// Roles (one CTA per SM, 10 warps): warp 0 issues TMA loads into a 4-stage
// shared-memory ring; warp 1 issues tcgen05.mma; warps 2-5 drain TMEM into
// registers and hand the finished 128 x 128 tile to warps 6-9 through shared
// memory; warps 6-9 run the epilogue (global memory) while the next tile's
// MMAs proceed.  Tiles are scheduled persistently, M-tile fastest.
#include <cuda_bf16.h>

#include "fa_internal.h"
#include "fa_ptx.cuh"

namespace fa {

namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;
constexpr int STAGES = 4;
constexpr int L_BYTES = BM * BK * 2;
constexpr int R_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = L_BYTES + R_BYTES;
constexpr int KS_LD = BM + 1;                 // hand-off tile: column-major, padded
constexpr int KS_BYTES = BN * KS_LD * 4;
constexpr int THREADS = 320;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t MB_COL0 = 0;               // main-product chunks: columns [0,128), [128,256)
constexpr uint32_t CB_COL0 = 256;             // correction accumulators: [256,384), [384,512)
constexpr size_t SMEM_BYTES = size_t(STAGES) * STAGE_BYTES + KS_BYTES + 1024 + 512;

__device__ __forceinline__ void split_f32(float x, int nt, __nv_bfloat16 *t) {
  float r = x;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k < nt) {
      const __nv_bfloat16 b = __float2bfloat16_rn(r);
      t[k] = b;
      r -= __bfloat162float(b);
    }
  }
}

__device__ __forceinline__ void split_f64(double x, int nt, __nv_bfloat16 *t) {
  double r = x;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k < nt) {
      const __nv_bfloat16 b = __double2bfloat16(r);
      t[k] = b;
      r -= static_cast<double>(__bfloat162float(b));
    }
  }
}

__device__ __forceinline__ void put_r(const EpiParams &e, int b, int i, int j,
                                      const __nv_bfloat16 *t) {
  const size_t off = (static_cast<size_t>(b) * e.n + j) * e.ldp + i;
  for (int k = 0; k < e.terms_r; ++k) e.out_r[k * e.term_stride_r + off] = t[k];
}

__device__ __forceinline__ void put_l(const EpiParams &e, int b, int i, int j,
                                      const __nv_bfloat16 *t) {
  const size_t off = (static_cast<size_t>(b) * e.n + i) * e.ldp + j;
  for (int k = 0; k < e.terms_l; ++k) e.out_l[k * e.term_stride_l + off] = t[k];
}

// RK4 stage combine for element (i, j) of slice b with K = Fl(Y_s)_{ij} (low-storage
// form: acc = K1 + 2K2 + 2K3, Y_{s+1} = X + c_{s+1} h K_s, X <- X + h/6 (acc + K4),
// X kept as an unevaluated float32 sum hi + lo).  Returns the next stage operand
// Y_{s+1}; writes its R-form terms.  On the last step writes F (or F - G_old).
__device__ __forceinline__ float stage_elem(const EpiParams &e, int b, int i, int j, float v) {
  const int n = e.n;
  const size_t nn = static_cast<size_t>(n) * n;
  const size_t c = static_cast<size_t>(j) * n + i;
  float *xh = e.x_hi + b * nn;
  float *xl = e.x_lo + b * nn;
  float *ac = e.acc + b * nn;
  float K = v;
  if (e.flow == FA_FLOW_SQRT) K = (e.a_hi[c] - K) + e.a_lo[c];
  const float ch = static_cast<float>(e.ch);
  float y;
  if (e.stage == 1) {
    ac[c] = K;
    y = xh[c] + ch * K;
  } else if (e.stage < 4) {
    ac[c] = ac[c] + 2.0f * K;
    y = xh[c] + ch * K;
  } else {
    const float inc = static_cast<float>(e.h / 6.0) * (ac[c] + K);
    const float a = xh[c];
    const float s = a + inc;
    const float bp = s - a;
    const float er = (a - (s - bp)) + (inc - bp);   // two-sum error of a + inc
    float lo = xl[c] + er;
    const float hi = s + lo;
    lo = lo - (hi - s);
    xh[c] = hi;
    xl[c] = lo;
    y = hi;
    if (e.last) {
      const double X = static_cast<double>(hi) + static_cast<double>(lo);
      const size_t r = b * nn + static_cast<size_t>(i) * n + j;
      e.f_out[r] = e.g_old ? X - e.g_old[r] : X;
    }
  }
  if (!e.last && e.terms_r) {
    __nv_bfloat16 t[3];
    split_f32(y, e.terms_r > e.terms_l ? e.terms_r : e.terms_l, t);
    put_r(e, b, i, j, t);
  }
  return y;
}

// The same stage combine for four consecutive rows i0..i0+3 of column j (i0 % 4 == 0,
// n % 4 == 0): 16-byte loads/stores of the column-major state and 8-byte stores of the
// R-form terms.  v[u] is the product value of row i0 + u; on return y[u] holds Y_{s+1}.
struct Quad {
  float4 xh, xl, ac, ah, al;
};

__device__ __forceinline__ void stage_quad_load(const EpiParams &e, size_t c, Quad &q) {
  q.xh = *reinterpret_cast<const float4 *>(e.x_hi + c);
  if (e.stage > 1) q.ac = *reinterpret_cast<const float4 *>(e.acc + c);
  if (e.stage == 4) q.xl = *reinterpret_cast<const float4 *>(e.x_lo + c);
}

__device__ __forceinline__ void stage_quad_finish(const EpiParams &e, int b, int i0, int j,
                                                  size_t c, const float (&v)[4], Quad &q,
                                                  float (&y)[4]) {
  const int n = e.n;
  float K[4] = {v[0], v[1], v[2], v[3]};
  if (e.flow == FA_FLOW_SQRT) {
    const size_t ca = static_cast<size_t>(j) * n + i0;
    const float4 ah = *reinterpret_cast<const float4 *>(e.a_hi + ca);
    const float4 al = *reinterpret_cast<const float4 *>(e.a_lo + ca);
    K[0] = (ah.x - K[0]) + al.x;
    K[1] = (ah.y - K[1]) + al.y;
    K[2] = (ah.z - K[2]) + al.z;
    K[3] = (ah.w - K[3]) + al.w;
  }
  float xh[4] = {q.xh.x, q.xh.y, q.xh.z, q.xh.w};
  const float ch = static_cast<float>(e.ch);
  if (e.stage == 1) {
    *reinterpret_cast<float4 *>(e.acc + c) = make_float4(K[0], K[1], K[2], K[3]);
#pragma unroll
    for (int u = 0; u < 4; ++u) y[u] = xh[u] + ch * K[u];
  } else if (e.stage < 4) {
    float ac[4] = {q.ac.x, q.ac.y, q.ac.z, q.ac.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ac[u] = ac[u] + 2.0f * K[u];
      y[u] = xh[u] + ch * K[u];
    }
    *reinterpret_cast<float4 *>(e.acc + c) = make_float4(ac[0], ac[1], ac[2], ac[3]);
  } else {
    const float ac[4] = {q.ac.x, q.ac.y, q.ac.z, q.ac.w};
    float xl[4] = {q.xl.x, q.xl.y, q.xl.z, q.xl.w};
    const float h6 = static_cast<float>(e.h / 6.0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float inc = h6 * (ac[u] + K[u]);
      const float a = xh[u];
      const float s = a + inc;
      const float bp = s - a;
      const float er = (a - (s - bp)) + (inc - bp);
      float lo = xl[u] + er;
      const float hi = s + lo;
      lo = lo - (hi - s);
      xh[u] = hi;
      xl[u] = lo;
      y[u] = hi;
    }
    *reinterpret_cast<float4 *>(e.x_hi + c) = make_float4(xh[0], xh[1], xh[2], xh[3]);
    *reinterpret_cast<float4 *>(e.x_lo + c) = make_float4(xl[0], xl[1], xl[2], xl[3]);
    if (e.last) {
      const size_t nn = static_cast<size_t>(n) * n;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double X = static_cast<double>(xh[u]) + static_cast<double>(xl[u]);
        const size_t r = b * nn + static_cast<size_t>(i0 + u) * n + j;
        e.f_out[r] = e.g_old ? X - e.g_old[r] : X;
      }
    }
  }
}

// BF16 terms of four consecutive rows i0..i0+3 of column j, R form (8-byte stores).
__device__ __forceinline__ void put_r_quad(const EpiParams &e, int b, int i0, int j,
                                           const float (&y)[4], int nt) {
  __nv_bfloat16 t[4][3];
#pragma unroll
  for (int u = 0; u < 4; ++u) split_f32(y[u], nt, t[u]);
  const size_t off = (static_cast<size_t>(b) * e.n + j) * e.ldp + i0;
  for (int k = 0; k < e.terms_r; ++k) {
    __nv_bfloat162 lo2, hi2;
    lo2.x = t[0][k];
    lo2.y = t[1][k];
    hi2.x = t[2][k];
    hi2.y = t[3][k];
    uint2 w;
    w.x = *reinterpret_cast<uint32_t *>(&lo2);
    w.y = *reinterpret_cast<uint32_t *>(&hi2);
    *reinterpret_cast<uint2 *>(e.out_r + k * e.term_stride_r + off) = w;
  }
}

// One forward-Euler substep G = V + dt Fl(V) (single slice, row-major float64); on the
// last substep also G_n out, the correction V_{n+1} = G_n + D_n and the norm terms.
__device__ __forceinline__ void euler_elem(const EpiParams &e, int i, int j, float v, double &s0,
                                           double &s1) {
  const int n = e.n;
  const size_t r = static_cast<size_t>(i) * n + j;
  double K = static_cast<double>(v);
  if (e.flow == FA_FLOW_SQRT) {
    const size_t c = static_cast<size_t>(j) * n + i;
    K = (static_cast<double>(e.a_hi[c]) + static_cast<double>(e.a_lo[c])) - K;
  }
  const double G = e.v_in[r] + e.dt * K;
  double Vn = G;
  if (e.euler_last) {
    e.g_out[r] = G;
    if (e.d_in) Vn = G + e.d_in[r];
    if (e.u_old) {
      const double dl = Vn - e.u_old[r];
      s0 += dl * dl;
      s1 += Vn * Vn;
    }
  }
  e.v_out[r] = Vn;
  const int nt = e.terms_l > e.terms_r ? e.terms_l : e.terms_r;
  if (nt) {
    __nv_bfloat16 t[3];
    split_f64(Vn, nt, t);
    if (e.terms_r) put_r(e, 0, i, j, t);
    if (e.terms_l) put_l(e, 0, i, j, t);
  }
}

__device__ __forceinline__ void fail(volatile int *abort_flag, int *err) {
  *abort_flag = 1;
  if (err) atomicCAS(err, 0, static_cast<int>(FA_ERR_TIMEOUT));
}

__global__ void __launch_bounds__(THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmL,
                   const __grid_constant__ CUtensorMap tmR,
                   const __grid_constant__ TcGemmParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  float *Ks = reinterpret_cast<float *>(smem + STAGES * STAGE_BYTES);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES + KS_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *mbfull = empty + STAGES;
  uint64_t *mbempty = mbfull + 2;
  uint64_t *cbfull = mbempty + 2;
  uint64_t *cbempty = cbfull + 2;
  uint64_t *kfull = cbempty + 2;
  uint64_t *kempty = kfull + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(kempty + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  double *red = reinterpret_cast<double *>(tmem_slot + 2);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(full + s, 1);
      ptx::mbar_init(empty + s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(mbfull + a, 1);
      ptx::mbar_init(mbempty + a, 128);
      ptx::mbar_init(cbfull + a, 1);
      ptx::mbar_init(cbempty + a, 128);
    }
    ptx::mbar_init(kfull, 128);
    ptx::mbar_init(kempty, 128);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    ptx::prefetch_tmap(&tmL);
    ptx::prefetch_tmap(&tmR);
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int tiles_per_slice = p.mt * p.nt;
  const EpiParams &e = p.epi;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < p.num_tiles; tile += gridDim.x) {
        const int mt = tile % p.mt;
        const int rest = tile / p.mt;
        const int ntile = rest % p.nt;
        const int gb = e.b0 + rest / p.nt;
        const int lb = p.l_batched ? gb : 0;
        const int rb = p.r_batched ? gb : 0;
        for (int kb = 0; ok && kb < p.kblocks; ++kb) {
          for (int q = 0; q < p.npairs; ++q) {
            if (!ptx::mbar_wait(empty + stage, phase ^ 1u, abort_flag)) {
              fail(abort_flag, e.err);
              ok = false;
              break;
            }
            uint8_t *sl = smem + stage * STAGE_BYTES;
            ptx::mbar_arrive_expect_tx(full + stage, STAGE_BYTES);
            ptx::tma_load_4d(sl, &tmL, full + stage, kb * BK, mt * BM, lb, p.pair_a[q]);
            ptx::tma_load_4d(sl + L_BYTES, &tmR, full + stage, kb * BK, ntile * BN, rb,
                             p.pair_b[q]);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0, mb = 0, ci = 0;
      uint32_t phase = 0, mph = 0, cph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < p.num_tiles; tile += gridDim.x) {
        if (!ptx::mbar_wait(cbempty + ci, cph ^ 1u, abort_flag)) {
          fail(abort_flag, e.err);
          break;
        }
        ptx::tc_fence_after();
        const uint32_t c_tmem = tmem_base + CB_COL0 + static_cast<uint32_t>(ci * BN);
        for (int kb = 0; ok && kb < p.kblocks; ++kb) {
          if (!ptx::mbar_wait(mbempty + mb, mph ^ 1u, abort_flag)) {
            fail(abort_flag, e.err);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t m_tmem = tmem_base + MB_COL0 + static_cast<uint32_t>(mb * BN);
          for (int q = 0; q < p.npairs; ++q) {
            if (!ptx::mbar_wait(full + stage, phase, abort_flag)) {
              fail(abort_flag, e.err);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t sl = ptx::smem_u32(smem + stage * STAGE_BYTES);
            const uint32_t sr = sl + L_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              const uint32_t acc = (q == 0) ? (k > 0) : (kb > 0 || q > 1 || k > 0);
              ptx::tc_mma_bf16(q == 0 ? m_tmem : c_tmem, ptx::sdesc_sw128(sl + k * 32),
                               ptx::sdesc_sw128(sr + k * 32), p.idesc, acc);
            }
            ptx::tc_commit(empty + stage);
            if (q == 0) ptx::tc_commit(mbfull + mb);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
          mb ^= 1;
          if (mb == 0) mph ^= 1u;
        }
        if (!ok) break;
        ptx::tc_commit(cbfull + ci);
        ci ^= 1;
        if (ci == 0) cph ^= 1u;
      }
    }
    __syncwarp();
  } else if (warp < 6) {
    // ---------------- drain: TMEM -> float32 registers -> shared hand-off tile ----------------
    const int q = warp & 3;              // TMEM lanes [32q, 32q + 32) are reachable from this warp
    const int row = q * 32 + lane;
    const uint32_t lane_base = tmem_base + (static_cast<uint32_t>(q * 32) << 16);
    int mb = 0, ci = 0;
    uint32_t mph = 0, cph = 0, kph = 0;
    bool ok = true;
    for (int tile = blockIdx.x; ok && tile < p.num_tiles; tile += gridDim.x) {
      float acc[BN];
#pragma unroll
      for (int c = 0; c < BN; ++c) acc[c] = 0.0f;
      for (int kb = 0; kb < p.kblocks; ++kb) {
        if (!ptx::mbar_wait(mbfull + mb, mph, abort_flag)) {
          fail(abort_flag, e.err);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
#pragma unroll
        for (int c = 0; c < BN / 32; ++c) {
          float v[32];
          ptx::tmem_ld_32x32b_x32(lane_base + MB_COL0 + static_cast<uint32_t>(mb * BN + c * 32), v);
#pragma unroll
          for (int u = 0; u < 32; ++u) acc[c * 32 + u] += v[u];
        }
        ptx::tc_fence_before();
        ptx::mbar_arrive(mbempty + mb);
        mb ^= 1;
        if (mb == 0) mph ^= 1u;
      }
      if (!ok) break;
      if (!ptx::mbar_wait(cbfull + ci, cph, abort_flag)) {
        fail(abort_flag, e.err);
        break;
      }
      ptx::tc_fence_after();
      if (p.npairs > 1) {
#pragma unroll
        for (int c = 0; c < BN / 32; ++c) {
          float v[32];
          ptx::tmem_ld_32x32b_x32(lane_base + CB_COL0 + static_cast<uint32_t>(ci * BN + c * 32), v);
#pragma unroll
          for (int u = 0; u < 32; ++u) acc[c * 32 + u] += v[u];
        }
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(cbempty + ci);
      ci ^= 1;
      if (ci == 0) cph ^= 1u;
      if (!ptx::mbar_wait(kempty, kph ^ 1u, abort_flag)) {
        fail(abort_flag, e.err);
        break;
      }
#pragma unroll
      for (int c = 0; c < BN; ++c) Ks[c * KS_LD + row] = acc[c];
      ptx::mbar_arrive(kfull);
      kph ^= 1u;
    }
  } else {
    // ---------------- store: epilogue from the shared tile to global memory ----------------
    const int t = threadIdx.x - 192;     // 0..127
    const int sw = t >> 5;
    uint32_t kph = 0;
    const int n = e.n;
    const bool pass1 = (e.mode == EPI_STAGE || e.mode == EPI_PROD);
    const bool pass2 = (e.mode == EPI_STAGE && e.terms_l && !e.last) || e.mode == EPI_EULER ||
                       e.mode == EPI_STORE;
    const bool norms = (e.mode == EPI_EULER) && (e.u_old != nullptr);
    for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
      const int mt = tile % p.mt;
      const int rest = tile / p.mt;
      const int ntile = rest % p.nt;
      const int lb = rest / p.nt;
      const int gb = e.b0 + lb;
      const int m0 = mt * BM, n0 = ntile * BN;
      if (!ptx::mbar_wait(kfull, kph, abort_flag)) {
        fail(abort_flag, e.err);
        break;
      }
      double s0 = 0.0, s1 = 0.0;
      if (pass1) {
        // Four rows per thread (16-byte column-major accesses), columns c = sw + 4k,
        // processed UNR at a time with their global loads issued together.
        const int sub = t & 31;
        const int r0 = 4 * sub;
        const int i0 = m0 + r0;
        const bool vec = ((n & 3) == 0) && (i0 + 3 < n);
        const int nt = e.terms_l > e.terms_r ? e.terms_l : e.terms_r;
        constexpr int UNR = 4;
        if (vec) {
          const size_t nn = static_cast<size_t>(n) * n;
          for (int k0 = 0; k0 < BN / 4; k0 += UNR) {
            Quad qd[UNR];
            size_t cc[UNR];
            bool act[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
              const int c = sw + 4 * (k0 + u);
              const int j = n0 + c;
              act[u] = j < n;
              cc[u] = gb * nn + static_cast<size_t>(j) * n + i0;
              if (act[u] && e.mode == EPI_STAGE) stage_quad_load(e, cc[u], qd[u]);
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
              if (!act[u]) continue;
              const int c = sw + 4 * (k0 + u);
              const int j = n0 + c;
              float v[4], y[4];
#pragma unroll
              for (int w = 0; w < 4; ++w) v[w] = Ks[c * KS_LD + r0 + w];
              if (e.mode == EPI_STAGE) {
                stage_quad_finish(e, gb, i0, j, cc[u], v, qd[u], y);
                if (!e.last) {
                  if (e.terms_r) put_r_quad(e, gb, i0, j, y, nt);
#pragma unroll
                  for (int w = 0; w < 4; ++w) Ks[c * KS_LD + r0 + w] = y[w];
                }
              } else {
                put_r_quad(e, gb, i0, j, v, e.terms_r);
              }
            }
          }
        } else {
          for (int k = 0; k < BN / 4; ++k) {
            const int c = sw + 4 * k;
            const int j = n0 + c;
            if (j >= n) break;
            for (int w = 0; w < 4; ++w) {
              const int i = i0 + w;
              if (i >= n) break;
              const float v = Ks[c * KS_LD + r0 + w];
              if (e.mode == EPI_STAGE) {
                Ks[c * KS_LD + r0 + w] = stage_elem(e, gb, i, j, v);
              } else {
                __nv_bfloat16 tt[3];
                split_f32(v, e.terms_r, tt);
                put_r(e, gb, i, j, tt);
              }
            }
          }
        }
      }
      if (pass2) {
        ptx::named_bar_sync(2, 128);
        // warp = 32 rows, lanes across columns: row-major outputs are coalesced
        for (int rr = 0; rr < 32; ++rr) {
          const int r = sw * 32 + rr;
          const int i = m0 + r;
          if (i >= n) break;
#pragma unroll
          for (int qq = 0; qq < BN / 32; ++qq) {
            const int c = lane + 32 * qq;
            const int j = n0 + c;
            if (j < n) {
              const float v = Ks[c * KS_LD + r];
              if (e.mode == EPI_STAGE) {
                __nv_bfloat16 tt[3];
                split_f32(v, e.terms_l > e.terms_r ? e.terms_l : e.terms_r, tt);
                put_l(e, gb, i, j, tt);
              } else if (e.mode == EPI_EULER) {
                euler_elem(e, i, j, v, s0, s1);
              } else {
                e.store_out[gb * static_cast<size_t>(n) * n + static_cast<size_t>(i) * n + j] =
                    e.alpha * static_cast<double>(v) + (i == j ? e.beta : 0.0);
              }
            }
          }
        }
      }
      if (norms) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          s0 += __shfl_xor_sync(0xffffffffu, s0, off);
          s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        }
        if (lane == 0) {
          red[2 * sw] = s0;
          red[2 * sw + 1] = s1;
        }
        ptx::named_bar_sync(2, 128);
        if (t == 0) {
          const double t0 = ((red[0] + red[2]) + red[4]) + red[6];
          const double t1 = ((red[1] + red[3]) + red[5]) + red[7];
          const size_t slot = static_cast<size_t>(lb) * tiles_per_slice + (tile % tiles_per_slice);
          e.norm_part[2 * slot] = t0;
          e.norm_part[2 * slot + 1] = t1;
        }
      }
      ptx::mbar_arrive(kempty);
      kph ^= 1u;
    }
  }

  if (*abort_flag) {
    // Give in-flight TMA copies and MMAs time to land before TMEM is released.
    const long long t0 = clock64();
    while (clock64() - t0 < 20000000LL) {
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// 32 x 32 tile transposition helpers for the operand-term builders.
constexpr int TT = 32;

__global__ void split_terms_kernel(const double *__restrict__ src, int n, int ldp,
                                   __nv_bfloat16 *out_l, int terms_l, size_t stride_l,
                                   __nv_bfloat16 *out_r, int terms_r, size_t stride_r,
                                   int i_minus) {
  __shared__ double tile[TT][TT + 1];
  const int b = blockIdx.z;
  const int i0 = blockIdx.y * TT, j0 = blockIdx.x * TT;
  const size_t nn = static_cast<size_t>(n) * n;
  const double *S = src + b * nn;
  const int nt = terms_l > terms_r ? terms_l : terms_r;
  for (int r = threadIdx.y; r < TT; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    double x = 0.0;
    if (i < n && j < n) {
      x = S[static_cast<size_t>(i) * n + j];
      if (i_minus) x = (i == j ? 1.0 : 0.0) - x;
      if (terms_l) {
        __nv_bfloat16 t[3];
        split_f64(x, nt, t);
        const size_t off = (static_cast<size_t>(b) * n + i) * ldp + j;
        for (int k = 0; k < terms_l; ++k) out_l[k * stride_l + off] = t[k];
      }
    }
    tile[r][threadIdx.x] = x;
  }
  if (!terms_r) return;
  __syncthreads();
  for (int r = threadIdx.y; r < TT; r += blockDim.y) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (i < n && j < n) {
      __nv_bfloat16 t[3];
      split_f64(tile[threadIdx.x][r], nt, t);
      const size_t off = (static_cast<size_t>(b) * n + j) * ldp + i;
      for (int k = 0; k < terms_r; ++k) out_r[k * stride_r + off] = t[k];
    }
  }
}

__global__ void load_state_kernel(const double *__restrict__ U, int n, int ldp, float *x_hi,
                                  float *x_lo, __nv_bfloat16 *out_l, int terms_l,
                                  size_t stride_l, __nv_bfloat16 *out_r, int terms_r,
                                  size_t stride_r) {
  __shared__ double tile[TT][TT + 1];
  const int b = blockIdx.z;
  const int i0 = blockIdx.y * TT, j0 = blockIdx.x * TT;
  const size_t nn = static_cast<size_t>(n) * n;
  const int nt = terms_l > terms_r ? terms_l : terms_r;
  for (int r = threadIdx.y; r < TT; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    double x = 0.0;
    if (i < n && j < n) {
      x = U[b * nn + static_cast<size_t>(i) * n + j];
      if (terms_l) {
        __nv_bfloat16 t[3];
        split_f32(static_cast<float>(x), nt, t);
        const size_t off = (static_cast<size_t>(b) * n + i) * ldp + j;
        for (int k = 0; k < terms_l; ++k) out_l[k * stride_l + off] = t[k];
      }
    }
    tile[r][threadIdx.x] = x;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < TT; r += blockDim.y) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (i < n && j < n) {
      const double x = tile[threadIdx.x][r];
      const float hi = static_cast<float>(x);
      const float lo = static_cast<float>(x - static_cast<double>(hi));
      const size_t c = b * nn + static_cast<size_t>(j) * n + i;
      x_hi[c] = hi;
      x_lo[c] = lo;
      if (terms_r) {
        __nv_bfloat16 t[3];
        split_f32(hi, nt, t);
        const size_t off = (static_cast<size_t>(b) * n + j) * ldp + i;
        for (int k = 0; k < terms_r; ++k) out_r[k * stride_r + off] = t[k];
      }
    }
  }
}

}  // namespace

PairSet pair_set(int dtype) {
  PairSet s{};
  auto add = [&](int a, int b) {
    s.a[s.npairs] = a;
    s.b[s.npairs] = b;
    ++s.npairs;
  };
  switch (dtype) {
    case FA_BF16: add(0, 0); break;
    case FA_BF16X3: add(0, 0); add(0, 1); add(1, 0); break;
    case FA_BF16X4: add(0, 0); add(0, 1); add(1, 0); add(2, 0); break;
    case FA_BF16X6: add(0, 0); add(0, 1); add(1, 0); add(0, 2); add(1, 1); add(2, 0); break;
    default: break;
  }
  for (int k = 0; k < s.npairs; ++k) {
    if (s.a[k] + 1 > s.terms_l) s.terms_l = s.a[k] + 1;
    if (s.b[k] + 1 > s.terms_r) s.terms_r = s.b[k] + 1;
  }
  return s;
}

cudaError_t launch_tc_gemm(const CUtensorMap *tmL, const CUtensorMap *tmR, const TcGemmParams &p,
                           int num_sms, cudaStream_t s) {
  static thread_local int attr_set_for = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_set_for != dev) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(SMEM_BYTES));
    if (e != cudaSuccess) return e;
    attr_set_for = dev;
  }
  if (p.num_tiles <= 0) return cudaSuccess;
  const int grid = p.num_tiles < num_sms ? p.num_tiles : num_sms;
  tc_gemm_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(*tmL, *tmR, p);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split_terms(const double *src, int nb, int n, int ldp, __nv_bfloat16 *out_l,
                               int terms_l, size_t stride_l, __nv_bfloat16 *out_r, int terms_r,
                               size_t stride_r, int i_minus, cudaStream_t s) {
  dim3 grid((n + TT - 1) / TT, (n + TT - 1) / TT, nb), block(TT, 8);
  split_terms_kernel<<<grid, block, 0, s>>>(src, n, ldp, out_l, terms_l, stride_l, out_r,
                                            terms_r, stride_r, i_minus);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_load_state(const double *U, int nb, int n, int ldp, float *x_hi, float *x_lo,
                              __nv_bfloat16 *out_l, int terms_l, size_t stride_l,
                              __nv_bfloat16 *out_r, int terms_r, size_t stride_r,
                              cudaStream_t s) {
  dim3 grid((n + TT - 1) / TT, (n + TT - 1) / TT, nb), block(TT, 8);
  load_state_kernel<<<grid, block, 0, s>>>(U, n, ldp, x_hi, x_lo, out_l, terms_l, stride_l, out_r,
                                           terms_r, stride_r);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fa
