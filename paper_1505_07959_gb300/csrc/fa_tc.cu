// Tensor-core (tcgen05) path: batched GEMMs over BF16 term pairs with the
// fused RK4 stage-combine / forward-Euler-correction epilogues.
//
// Every matrix product of the flows (Section 2, Examples 1 and 2: A Y,
// (I - A) Y, Y P; the square-root flow's Y Y) is computed as
//     D = sum_p L_{a_p} R_{b_p}^T
// where L_a / R_b are the BF16 terms of the left operand (row-major, "L form")
// and of the transposed right operand ("R form"), x = x_0 + x_1 + x_2 with
// x_{k+1} the BF16 rounding of what x_0..x_k leave out.  Products are
// accumulated in float32 in tensor memory.  A CTA owns one SM: warp 0 issues
// TMA loads into a 4-stage shared-memory ring, warp 1 issues tcgen05.mma into
// one of two 128 x 256 TMEM accumulators, warps 2-5 drain the other
// accumulator through the epilogue, so epilogue traffic overlaps the next
// tile's MMAs.  Tiles are scheduled persistently, M-tile fastest, so CTAs
// that run at the same time share the right operand's tile through L2.
#include <cuda_bf16.h>

#include "fa_internal.h"
#include "fa_ptx.cuh"

namespace fa {

namespace {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int STAGES = 4;
constexpr int L_BYTES = BM * BK * 2;
constexpr int R_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = L_BYTES + R_BYTES;
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 512;
constexpr size_t SMEM_BYTES = size_t(STAGES) * STAGE_BYTES + 1024 + 256;

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

// Write the BF16 terms of element (i, j) of slice b in L form and/or R form.
__device__ __forceinline__ void put_terms(const EpiParams &e, int b, int i, int j,
                                          const __nv_bfloat16 *t) {
  if (e.terms_r) {
    const size_t off = (static_cast<size_t>(b) * e.n + j) * e.ldp + i;
    for (int k = 0; k < e.terms_r; ++k) e.out_r[k * e.term_stride_r + off] = t[k];
  }
  if (e.terms_l) {
    const size_t off = (static_cast<size_t>(b) * e.n + i) * e.ldp + j;
    for (int k = 0; k < e.terms_l; ++k) e.out_l[k * e.term_stride_l + off] = t[k];
  }
}

// Epilogue of 32 consecutive accumulator columns j0..j0+31 of row i, slice b.
__device__ __forceinline__ void epilogue_chunk(const EpiParams &e, int b, int i, int j0,
                                               const float (&v)[32], double &s0, double &s1) {
  const int n = e.n;
  if (i >= n) return;
  const size_t nn = static_cast<size_t>(n) * n;
  const int nt = e.terms_l > e.terms_r ? e.terms_l : e.terms_r;
  const int jend = (n - j0) < 32 ? (n - j0) : 32;
  __nv_bfloat16 t[3];

  if (e.mode == EPI_STAGE) {
    // Classical RK4 in low-storage form: acc = K1 + 2K2 + 2K3, Y_{s+1} = X + c_{s+1} h K_s,
    // X <- X + h/6 (acc + K4), with X kept as an unevaluated float32 sum hi + lo.
    float *xh = e.x_hi + b * nn;
    float *xl = e.x_lo + b * nn;
    float *ac = e.acc + b * nn;
    const float ch = static_cast<float>(e.ch);
    const float h6 = static_cast<float>(e.h / 6.0);
    for (int jj = 0; jj < jend; ++jj) {
      const int j = j0 + jj;
      const size_t c = static_cast<size_t>(j) * n + i;
      float K = v[jj];
      if (e.flow == FA_FLOW_SQRT) K = (e.a_hi[c] - K) + e.a_lo[c];
      float y;
      if (e.stage == 1) {
        ac[c] = K;
        y = xh[c] + ch * K;
      } else if (e.stage < 4) {
        ac[c] = ac[c] + 2.0f * K;
        y = xh[c] + ch * K;
      } else {
        const float inc = h6 * (ac[c] + K);
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
      if (!e.last) {
        split_f32(y, nt, t);
        put_terms(e, b, i, j, t);
      }
    }
  } else if (e.mode == EPI_PROD) {
    for (int jj = 0; jj < jend; ++jj) {
      split_f32(v[jj], nt, t);
      put_terms(e, b, i, j0 + jj, t);
    }
  } else if (e.mode == EPI_EULER) {
    // One forward-Euler substep G = V + dt Fl(V) on a single slice (row-major float64);
    // on the last substep also the parareal correction V_{n+1} = G_n + D_n and the norms.
    for (int jj = 0; jj < jend; ++jj) {
      const int j = j0 + jj;
      const size_t r = static_cast<size_t>(i) * n + j;
      double K = static_cast<double>(v[jj]);
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
      if (nt) {
        split_f64(Vn, nt, t);
        put_terms(e, 0, i, j, t);
      }
    }
  } else {  // EPI_STORE
    for (int jj = 0; jj < jend; ++jj) {
      const int j = j0 + jj;
      e.store_out[b * nn + static_cast<size_t>(i) * n + j] =
          e.alpha * static_cast<double>(v[jj]) + (i == j ? e.beta : 0.0);
    }
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
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *tfull = empty + STAGES;
  uint64_t *tempty = tfull + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  double *red = reinterpret_cast<double *>(tmem_slot + 4);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(full + s, 1);
      ptx::mbar_init(empty + s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(tfull + a, 1);
      ptx::mbar_init(tempty + a, 4 * 32);
    }
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
        const int gb = p.epi.b0 + rest / p.nt;
        const int lb = p.l_batched ? gb : 0;
        const int rb = p.r_batched ? gb : 0;
        for (int kb = 0; ok && kb < p.kblocks; ++kb) {
          for (int q = 0; q < p.npairs; ++q) {
            if (!ptx::mbar_wait(empty + stage, phase ^ 1u, abort_flag)) {
              fail(abort_flag, p.epi.err);
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
      int stage = 0;
      uint32_t phase = 0;
      int ai = 0;
      uint32_t aphase = 0;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < p.num_tiles; tile += gridDim.x) {
        if (!ptx::mbar_wait(tempty + ai, aphase ^ 1u, abort_flag)) {
          fail(abort_flag, p.epi.err);
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(ai * BN);
        uint32_t accumulate = 0;
        for (int kb = 0; ok && kb < p.kblocks; ++kb) {
          for (int q = 0; q < p.npairs; ++q) {
            if (!ptx::mbar_wait(full + stage, phase, abort_flag)) {
              fail(abort_flag, p.epi.err);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t sl = ptx::smem_u32(smem + stage * STAGE_BYTES);
            const uint32_t sr = sl + L_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              ptx::tc_mma_bf16(d_tmem, ptx::sdesc_sw128(sl + k * 32),
                               ptx::sdesc_sw128(sr + k * 32), p.idesc, accumulate);
              accumulate = 1;
            }
            ptx::tc_commit(empty + stage);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (!ok) break;
        ptx::tc_commit(tfull + ai);
        ai ^= 1;
        if (ai == 0) aphase ^= 1u;
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int q = warp & 3;            // this warp may access TMEM lanes [32q, 32q + 32)
    const int row = q * 32 + lane;     // accumulator row owned by this thread
    int ai = 0;
    uint32_t aphase = 0;
    const bool norms = (p.epi.mode == EPI_EULER) && (p.epi.u_old != nullptr);
    for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
      const int mt = tile % p.mt;
      const int rest = tile / p.mt;
      const int ntile = rest % p.nt;
      const int lb = rest / p.nt;
      const int gb = p.epi.b0 + lb;
      if (!ptx::mbar_wait(tfull + ai, aphase, abort_flag)) {
        fail(abort_flag, p.epi.err);
        break;
      }
      ptx::tc_fence_after();
      double s0 = 0.0, s1 = 0.0;
      const int i = mt * BM + row;
      for (int c = 0; c < BN / 32; ++c) {
        const int j0 = ntile * BN + c * 32;
        if (j0 >= p.n) break;
        float v[32];
        ptx::tmem_ld_32x32b_x32(
            tmem_base + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(ai * BN + c * 32),
            v);
        epilogue_chunk(p.epi, gb, i, j0, v, s0, s1);
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(tempty + ai);
      if (norms) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          s0 += __shfl_xor_sync(0xffffffffu, s0, off);
          s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        }
        if (lane == 0) {
          red[2 * q] = s0;
          red[2 * q + 1] = s1;
        }
        ptx::named_bar_sync(1, 128);
        if (warp == 2 && lane == 0) {
          const double t0 = ((red[0] + red[2]) + red[4]) + red[6];
          const double t1 = ((red[1] + red[3]) + red[5]) + red[7];
          const size_t slot = static_cast<size_t>(lb) * tiles_per_slice + (tile % tiles_per_slice);
          p.epi.norm_part[2 * slot] = t0;
          p.epi.norm_part[2 * slot + 1] = t1;
        }
        ptx::named_bar_sync(1, 128);
      }
      ai ^= 1;
      if (ai == 0) aphase ^= 1u;
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
