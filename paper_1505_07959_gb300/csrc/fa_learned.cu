// Learned coarse propagator: features, the coefficient network (inference and training), the
// pair records it is trained on, and the polynomial update.
//
// The coarse step is G_theta(X) = X + sum_{j=1..4} c_j dT^j X_[j], where X_[j] is the j-th
// Taylor coefficient of the flow's solution through X (inverse flow: X (BX)^j with B = I - A;
// exponential flow: A^j X / j!), so c = (1, 0, 0, 0) is the forward-Euler step of Section 2
// (Example 1) and c = (1, 1, 1, 1) the degree-4 Taylor step.  The products R_j (the X_[j]
// without the 1/j!) come from the GEMM kernels; this file holds everything after them:
//
//  * stats: one pass over a state X (and optionally its fine image F and the powers R_j) that
//    accumulates, per block and in a fixed order, the 8 Hutchinson sums z_k^T X z_k (Rademacher
//    probes from SplitMix64, kept as one byte of 8 sign bits per index), ||X||^2, the Gram
//    sums <R_a, R_b>, <R_a, D>, ||D||^2 with D = F - X, and Gershgorin bounds;
//  * records: per pair, the 8 features and the Gram data of the quadratic loss;
//  * the network 8 -> 128 -> 128 -> 4 (GELU, exact erf form): BF16 weights (rounded from the
//    float32 master copy at load), float32 activations and accumulation.  Forward for
//    inference; forward + backward per sample and a fixed-order float64 reduction of the
//    weight gradients over the batch for training; Adam;
//  * combine: G = X + sum_j a_j R_j, the parareal correction X_{n+1} = G + D_n and the
//    convergence-norm partial sums.
// Every reduction runs in a fixed order, so results are bitwise reproducible.
#include <cstring>

#include <cuda_bf16.h>

#include "fa_internal.h"

namespace fa {

namespace {

constexpr int NF = FA_MLP_FEATURES, HID = FA_MLP_HIDDEN, NC = FA_MLP_COEFS;
constexpr int OFF_MU = 0, OFF_SD = OFF_MU + NF, OFF_W1 = OFF_SD + NF, OFF_B1 = OFF_W1 + HID * NF,
              OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID,
              OFF_B3 = OFF_W3 + NC * HID, NPARAM = OFF_B3 + NC;
static_assert(NPARAM == FA_MLP_PARAMS, "parameter blob layout");
constexpr int REC = FA_RECORD_DOUBLES;
constexpr int STATS_THREADS = 256;
constexpr int MLP_S = 8;                 // samples per block
constexpr int W2LD = HID + 2;            // BF16 row stride of W2 in shared memory (65 words)

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// ---- probes -------------------------------------------------------------------------------------

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output c of the stream seeded with `seed`.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long c) {
  unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// bits[j], bit k: probe k has -1 at index j (bit 63 of output k n + j).
__global__ void probes_kernel(int n, unsigned long long seed, uint8_t *bits) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  unsigned int m = 0;
  for (int k = 0; k < FA_PROBES; ++k)
    m |= static_cast<unsigned int>(splitmix64_at(seed, static_cast<unsigned long long>(k) * n + j) >> 63)
         << k;
  bits[j] = static_cast<uint8_t>(m);
}

// ---- stats --------------------------------------------------------------------------------------

// Index of the Gram sum <R_a, R_b> (a <= b) in the stats vector.
__host__ __device__ constexpr int rr_index(int a, int b) {
  return ST_RR + (a == 0 ? b : a == 1 ? 3 + b : a == 2 ? 5 + b : 9);
}

// Per block: rows [blockIdx.x * rows, ...) of slice blockIdx.y, one warp per row at a time,
// lanes striding the columns.  Partial sums go to part[(slice * blocks + block) * NSTAT].
__global__ void __launch_bounds__(STATS_THREADS) stats_kernel(const StatsArgs a) {
  const int n = a.n;
  const int b = blockIdx.y;
  const int rows = a.rows_per_block;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double *X = a.X + b * a.x_stride;
  const double *F = a.F ? a.F + b * a.f_stride : nullptr;
  const double *G = a.G ? a.G + b * a.f_stride : nullptr;
  const double *R0 = a.nR > 0 ? a.R[0] + b * a.r_stride : nullptr;
  const double *R1 = a.nR > 1 ? a.R[1] + b * a.r_stride : nullptr;
  const double *R2 = a.nR > 1 ? a.R[2] + b * a.r_stride : nullptr;
  const double *R3 = a.nR > 1 ? a.R[3] + b * a.r_stride : nullptr;
  double s[NSTAT];
#pragma unroll
  for (int q = 0; q < NSTAT; ++q) s[q] = 0.0;
  double glo = 1e300, ghi = -1e300;
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  for (int i = r0 + warp; i < r1; i += STATS_THREADS / 32) {
    const unsigned int zi = a.probes[i];
    const size_t row = static_cast<size_t>(i) * n;
    double off = 0.0, dg = 0.0;
    for (int j = lane; j < n; j += 32) {
      const double x = X[row + j];
      const unsigned int sg = zi ^ a.probes[j];
#pragma unroll
      for (int k = 0; k < FA_PROBES; ++k) s[ST_HUT + k] += ((sg >> k) & 1u) ? -x : x;
      s[ST_XX] += x * x;
      if (a.gersh) {
        if (j == i) dg = x;
        else off += fabs(x);
      }
      if (R0) {
        const double q0 = R0[row + j];
        s[rr_index(0, 0)] += q0 * q0;
        if (R1) {
          const double q1 = R1[row + j], q2 = R2[row + j], q3 = R3[row + j];
          s[rr_index(0, 1)] += q0 * q1;
          s[rr_index(0, 2)] += q0 * q2;
          s[rr_index(0, 3)] += q0 * q3;
          s[rr_index(1, 1)] += q1 * q1;
          s[rr_index(1, 2)] += q1 * q2;
          s[rr_index(1, 3)] += q1 * q3;
          s[rr_index(2, 2)] += q2 * q2;
          s[rr_index(2, 3)] += q2 * q3;
          s[rr_index(3, 3)] += q3 * q3;
          if (F) {
            const double d = (G ? F[row + j] + G[row + j] : F[row + j]) - x;
            s[ST_RD + 0] += q0 * d;
            s[ST_RD + 1] += q1 * d;
            s[ST_RD + 2] += q2 * d;
            s[ST_RD + 3] += q3 * d;
            s[ST_DD] += d * d;
          }
        }
      }
    }
    if (a.gersh) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        dg += __shfl_xor_sync(0xffffffffu, dg, o);
      }
      glo = fmin(glo, dg - off);
      ghi = fmax(ghi, dg + off);
    }
  }
  // Fixed-order reduction: lanes by xor butterfly, then warps in index order.
  __shared__ double red[STATS_THREADS / 32][NSTAT];
#pragma unroll
  for (int q = 0; q < NSTAT; ++q) {
    double v = s[q];
    if (q == ST_GLO) v = glo;
    if (q == ST_GHI) v = ghi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = (q == ST_GLO) ? fmin(v, w) : (q == ST_GHI) ? fmax(v, w) : v + w;
    }
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NSTAT) {
    const int q = threadIdx.x;
    double v = red[0][q];
    for (int w = 1; w < STATS_THREADS / 32; ++w)
      v = (q == ST_GLO) ? fmin(v, red[w][q]) : (q == ST_GHI) ? fmax(v, red[w][q]) : v + red[w][q];
    a.part[(static_cast<size_t>(b) * gridDim.x + blockIdx.x) * NSTAT + q] = v;
  }
}

// Sum of slice b's block partials for stat q, blocks in index order.
__device__ __forceinline__ double stat_sum(const double *part, int b, int blocks, int q) {
  const double *p = part + static_cast<size_t>(b) * blocks * NSTAT + q;
  double v = p[0];
  for (int k = 1; k < blocks; ++k) {
    const double w = p[static_cast<size_t>(k) * NSTAT];
    v = (q == ST_GLO) ? fmin(v, w) : (q == ST_GHI) ? fmax(v, w) : v + w;
  }
  return v;
}

// The matrix's own features: Gershgorin lower/upper bound and Hutchinson tr(A).
__global__ void matrix_stats_kernel(const double *part, int blocks, double *mstats) {
  if (threadIdx.x != 0) return;
  mstats[0] = stat_sum(part, 0, blocks, ST_GLO);
  mstats[1] = stat_sum(part, 0, blocks, ST_GHI);
  double h = 0.0;
  for (int k = 0; k < FA_PROBES; ++k) h += stat_sum(part, 0, blocks, ST_HUT + k);
  mstats[2] = h / FA_PROBES;
}

// The 8 raw features of slice b from its stats (see the network's docstring in fa.h).
__device__ __forceinline__ void slice_features(const double *part, int b, int blocks, int n,
                                               double t_over_T, double dT, const double *mstats,
                                               double *f) {
  double h = 0.0;
  for (int k = 0; k < FA_PROBES; ++k) h += stat_sum(part, b, blocks, ST_HUT + k);
  const double rn = sqrt(static_cast<double>(n));
  f[0] = t_over_T;
  f[1] = dT;
  f[2] = mstats[0];
  f[3] = mstats[1];
  f[4] = mstats[2] / n;
  f[5] = h / FA_PROBES / n;
  f[6] = sqrt(stat_sum(part, b, blocks, rr_index(0, 0))) / rn;
  f[7] = sqrt(stat_sum(part, b, blocks, ST_XX)) / rn;
}

// One thread per pair: features, Gram matrix M_ab = s_a s_b <R_a, R_b>, vector
// v_a = s_a <R_a, D> and dd = ||D||^2, with s_a = dT^a kappa_a the Taylor scale of R_a.
__global__ void records_kernel(const double *part, int nslices, int blocks, int n, int N_total,
                               int slice0, double dT, RecordScale sc, const double *mstats,
                               double *rec) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nslices) return;
  double *r = rec + static_cast<size_t>(b) * REC;
  slice_features(part, b, blocks, n, static_cast<double>(slice0 + b) / N_total, dT, mstats, r);
  for (int x = 0; x < 4; ++x) {
    for (int y = 0; y < 4; ++y) {
      const int lo = x < y ? x : y, hi = x < y ? y : x;
      r[NF + 4 * x + y] = sc.s[x] * sc.s[y] * stat_sum(part, b, blocks, rr_index(lo, hi));
    }
    r[NF + 16 + x] = sc.s[x] * stat_sum(part, b, blocks, ST_RD + x);
  }
  r[NF + 20] = stat_sum(part, b, blocks, ST_DD);
  for (int q = NF + 21; q < REC; ++q) r[q] = 0.0;
}

// ---- the network ----------------------------------------------------------------------------------

struct MlpShared {
  __nv_bfloat16 w2[HID * W2LD];  // w2[o * W2LD + i] = W2[o][i] (row and column reads conflict-free)
  float xs[MLP_S][NF];           // standardised features
  float h1[MLP_S][HID];
  float h2[MLP_S][HID];
  float dz2[MLP_S][HID];
  float c[MLP_S][NC];
  float dc[MLP_S][NC];
};

// Forward pass of the block's samples (xs filled, valid samples < nvalid).  Thread t owns hidden
// unit t; returns z1, z2 of unit t per sample in registers.  Ends with c in shared memory.
__device__ __forceinline__ void mlp_forward(const float *__restrict__ P, MlpShared &sm,
                                            float (&z1)[MLP_S], float (&z2)[MLP_S]) {
  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  float w1[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) w1[f] = bf16r(P[OFF_W1 + t * NF + f]);
  const float b1 = P[OFF_B1 + t];
#pragma unroll
  for (int s = 0; s < MLP_S; ++s) {
    float a = b1;
#pragma unroll
    for (int f = 0; f < NF; ++f) a = fmaf(w1[f], sm.xs[s][f], a);
    z1[s] = a;
    sm.h1[s][t] = gelu(a);
  }
  __syncthreads();
  const float b2 = P[OFF_B2 + t];
#pragma unroll
  for (int s = 0; s < MLP_S; ++s) z2[s] = b2;
  for (int i = 0; i < HID; ++i) {
    const float w = __bfloat162float(sm.w2[t * W2LD + i]);
#pragma unroll
    for (int s = 0; s < MLP_S; ++s) z2[s] = fmaf(w, sm.h1[s][i], z2[s]);
  }
#pragma unroll
  for (int s = 0; s < MLP_S; ++s) sm.h2[s][t] = gelu(z2[s]);
  __syncthreads();
  // Output o = warp: lanes take units lane + 32 q, then an xor butterfly.
  const int o = warp;
  float w3[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) w3[q] = bf16r(P[OFF_W3 + o * HID + lane + 32 * q]);
#pragma unroll
  for (int s = 0; s < MLP_S; ++s) {
    float v = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) v = fmaf(w3[q], sm.h2[s][lane + 32 * q], v);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) sm.c[s][o] = v + P[OFF_B3 + o];
  }
  __syncthreads();
}

__device__ __forceinline__ void load_w2(const float *__restrict__ P, MlpShared &sm) {
  for (int idx = threadIdx.x; idx < HID * HID; idx += HID)
    sm.w2[(idx / HID) * W2LD + idx % HID] = __float2bfloat16_rn(P[OFF_W2 + idx]);
}

__device__ __forceinline__ void load_features(const float *__restrict__ P, MlpShared &sm,
                                              const double *feat, int fstride, int b0, int B) {
  for (int idx = threadIdx.x; idx < MLP_S * NF; idx += HID) {
    const int s = idx / NF, f = idx % NF;
    const int b = b0 + s;
    const float x = b < B ? static_cast<float>(feat[static_cast<size_t>(b) * fstride + f]) : 0.0f;
    sm.xs[s][f] = (x - P[OFF_MU + f]) / P[OFF_SD + f];
  }
}

// Inference: coef[b][0..3] for B feature rows (stride fstride doubles); non-finite outputs are
// replaced by the Euler coefficients (1, 0, 0, 0) and counted in *fallbacks (when not null).
__global__ void __launch_bounds__(HID) mlp_forward_kernel(const float *__restrict__ P, int B,
                                                          const double *feat, int fstride,
                                                          float *coef, int *fallbacks) {
  __shared__ MlpShared sm;
  const int b0 = blockIdx.x * MLP_S;
  load_w2(P, sm);
  load_features(P, sm, feat, fstride, b0, B);
  __syncthreads();
  float z1[MLP_S], z2[MLP_S];
  mlp_forward(P, sm, z1, z2);
  if (threadIdx.x < MLP_S) {
    const int s = threadIdx.x, b = b0 + s;
    if (b < B) {
      bool ok = true;
      for (int o = 0; o < NC; ++o) ok = ok && isfinite(sm.c[s][o]);
      for (int o = 0; o < NC; ++o) coef[static_cast<size_t>(b) * NC + o] = ok ? sm.c[s][o] : (o == 0 ? 1.0f : 0.0f);
      if (!ok && fallbacks) atomicAdd(fallbacks, 1);
    }
  }
}

// Training, per sample: forward, loss (c^T M c - 2 c^T v + dd) / dd and its gradient
// dc = 2 (M c - v) / (dd B) (in float64 from the record), then backprop to dz2, dz1.  Stores
// what the weight-gradient reduction needs.
__global__ void __launch_bounds__(HID) mlp_train_kernel(const float *__restrict__ P, int B,
                                                        const double *rec, MlpTrainBuffers tb) {
  __shared__ MlpShared sm;
  const int t = threadIdx.x;
  const int b0 = blockIdx.x * MLP_S;
  load_w2(P, sm);
  load_features(P, sm, rec, REC, b0, B);
  __syncthreads();
  float z1[MLP_S], z2[MLP_S];
  mlp_forward(P, sm, z1, z2);
  if (t < MLP_S) {
    const int b = b0 + t;
    double dcv[NC] = {0.0, 0.0, 0.0, 0.0};
    double loss = 0.0;
    if (b < B) {
      const double *r = rec + static_cast<size_t>(b) * REC;
      const double *M = r + NF, *v = r + NF + 16;
      const double dd = r[NF + 20];
      double c[NC], Mc[NC];
      for (int o = 0; o < NC; ++o) c[o] = static_cast<double>(sm.c[t][o]);
      double cMc = 0.0, cv = 0.0;
      for (int o = 0; o < NC; ++o) {
        double m = 0.0;
        for (int q = 0; q < NC; ++q) m += M[4 * o + q] * c[q];
        Mc[o] = m;
        cMc += c[o] * m;
        cv += c[o] * v[o];
      }
      loss = (cMc - 2.0 * cv + dd) / dd;
      for (int o = 0; o < NC; ++o) dcv[o] = 2.0 * (Mc[o] - v[o]) / dd / B;
      tb.loss[b] = loss;
      for (int o = 0; o < NC; ++o) tb.dc[static_cast<size_t>(b) * NC + o] = static_cast<float>(dcv[o]);
    }
    for (int o = 0; o < NC; ++o) sm.dc[t][o] = static_cast<float>(dcv[o]);
  }
  __syncthreads();
  float w3[NC];
#pragma unroll
  for (int o = 0; o < NC; ++o) w3[o] = bf16r(P[OFF_W3 + o * HID + t]);
#pragma unroll
  for (int s = 0; s < MLP_S; ++s) {
    float g = 0.0f;
#pragma unroll
    for (int o = 0; o < NC; ++o) g = fmaf(w3[o], sm.dc[s][o], g);
    sm.dz2[s][t] = g * gelu_grad(z2[s]);
  }
  __syncthreads();
  float dz1[MLP_S];
#pragma unroll
  for (int s = 0; s < MLP_S; ++s) dz1[s] = 0.0f;
  for (int o = 0; o < HID; ++o) {
    const float w = __bfloat162float(sm.w2[o * W2LD + t]);
#pragma unroll
    for (int s = 0; s < MLP_S; ++s) dz1[s] = fmaf(w, sm.dz2[s][o], dz1[s]);
  }
#pragma unroll
  for (int s = 0; s < MLP_S; ++s) {
    const int b = b0 + s;
    if (b >= B) continue;
    const size_t o = static_cast<size_t>(b) * HID + t;
    tb.h1[o] = sm.h1[s][t];
    tb.h2[o] = sm.h2[s][t];
    tb.dz2[o] = sm.dz2[s][t];
    tb.dz1[o] = dz1[s] * gelu_grad(z1[s]);
    if (t < NF) tb.xs[static_cast<size_t>(b) * NF + t] = sm.xs[s][t];
  }
}

// Weight gradients: one thread per parameter, the batch summed in index order in float64.
// Thread NPARAM writes the mean loss.  mu and sd get zero gradient (they are not trained).
__global__ void mlp_grad_kernel(int B, MlpTrainBuffers tb, float *grad, double *loss_out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g == NPARAM) {
    double l = 0.0;
    for (int b = 0; b < B; ++b) l += tb.loss[b];
    *loss_out = l / B;
    return;
  }
  if (g >= NPARAM) return;
  double acc = 0.0;
  if (g < OFF_W1) {
    acc = 0.0;
  } else if (g < OFF_B1) {
    const int o = (g - OFF_W1) / NF, f = (g - OFF_W1) % NF;
    for (int b = 0; b < B; ++b)
      acc += static_cast<double>(tb.dz1[static_cast<size_t>(b) * HID + o]) * tb.xs[static_cast<size_t>(b) * NF + f];
  } else if (g < OFF_W2) {
    const int o = g - OFF_B1;
    for (int b = 0; b < B; ++b) acc += tb.dz1[static_cast<size_t>(b) * HID + o];
  } else if (g < OFF_B2) {
    const int o = (g - OFF_W2) / HID, i = (g - OFF_W2) % HID;
    for (int b = 0; b < B; ++b)
      acc += static_cast<double>(tb.dz2[static_cast<size_t>(b) * HID + o]) * tb.h1[static_cast<size_t>(b) * HID + i];
  } else if (g < OFF_W3) {
    const int o = g - OFF_B2;
    for (int b = 0; b < B; ++b) acc += tb.dz2[static_cast<size_t>(b) * HID + o];
  } else if (g < OFF_B3) {
    const int o = (g - OFF_W3) / HID, i = (g - OFF_W3) % HID;
    for (int b = 0; b < B; ++b)
      acc += static_cast<double>(tb.dc[static_cast<size_t>(b) * NC + o]) * tb.h2[static_cast<size_t>(b) * HID + i];
  } else {
    const int o = g - OFF_B3;
    for (int b = 0; b < B; ++b) acc += tb.dc[static_cast<size_t>(b) * NC + o];
  }
  grad[g] = static_cast<float>(acc);
}

// Adam on the trained parameters (W1..b3); c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t).
__global__ void adam_kernel(float *P, const float *grad, float *m, float *v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const int g = OFF_W1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= NPARAM) return;
  const float gr = grad[g];
  const float mm = b1 * m[g] + (1.0f - b1) * gr;
  const float vv = b2 * v[g] + (1.0f - b2) * gr * gr;
  m[g] = mm;
  v[g] = vv;
  P[g] = P[g] - lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

// Learned coarse step, network part (one block): features of slice `slice` from its stats,
// standardisation, forward pass, Euler fallback on non-finite output; coef[0..3] for the slice.
__global__ void __launch_bounds__(HID) coarse_coef_kernel(const float *__restrict__ P,
                                                          const double *part, int blocks, int n,
                                                          int slice, int N, double dT,
                                                          const double *mstats, float *coef,
                                                          int *fallbacks) {
  __shared__ MlpShared sm;
  __shared__ double feat[NF];
  load_w2(P, sm);
  if (threadIdx.x == 0) slice_features(part, 0, blocks, n, static_cast<double>(slice) / N, dT, mstats, feat);
  __syncthreads();
  load_features(P, sm, feat, NF, 0, 1);
  __syncthreads();
  float z1[MLP_S], z2[MLP_S];
  mlp_forward(P, sm, z1, z2);
  if (threadIdx.x == 0) {
    bool ok = true;
    for (int o = 0; o < NC; ++o) ok = ok && isfinite(sm.c[0][o]);
    for (int o = 0; o < NC; ++o) coef[o] = ok ? sm.c[0][o] : (o == 0 ? 1.0f : 0.0f);
    if (!ok) atomicAdd(fallbacks, 1);
  }
}

// G = X + sum_j (c_j s_j) R_j on one slice (s_j = dT^j kappa_j), then the correction
// X_{n+1} = G + D (D may be null: Step 0) and the partial norm sums of
// ||X_{n+1} - U_old||^2, ||X_{n+1}||^2 per block (u_old may be null).  Block k handles the
// contiguous elements [k chunk, (k + 1) chunk).
__global__ void __launch_bounds__(256) combine_kernel(const CombineArgs a) {
  const size_t nn = static_cast<size_t>(a.n) * a.n;
  const size_t chunk = (nn + gridDim.x - 1) / gridDim.x;
  const size_t e0 = blockIdx.x * chunk;
  const size_t e1 = e0 + chunk < nn ? e0 + chunk : nn;
  double w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) w[j] = static_cast<double>(a.coef[j]) * a.scale[j];
  double s0 = 0.0, s1 = 0.0;
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double x = a.v_in[e];
    const double G = x + (w[0] * a.R[0][e] + w[1] * a.R[1][e] + w[2] * a.R[2][e] + w[3] * a.R[3][e]);
    const double V = a.d_in ? G + a.d_in[e] : G;
    if (a.u_old) {
      const double dl = V - a.u_old[e];
      s0 += dl * dl;
      s1 += V * V;
    }
    a.g_out[e] = G;
    a.v_out[e] = V;
  }
  if (!a.norm_part) return;
  __shared__ double red[8][2];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[warp][0] = s0;
    red[warp][1] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int k = 0; k < 8; ++k) {
      t0 += red[k][0];
      t1 += red[k][1];
    }
    a.norm_part[2 * blockIdx.x] = t0;
    a.norm_part[2 * blockIdx.x + 1] = t1;
  }
}

}  // namespace

int stats_rows_per_block(int n) { return n <= 512 ? 8 : 16; }
int stats_blocks(int n) { return (n + stats_rows_per_block(n) - 1) / stats_rows_per_block(n); }

cudaError_t launch_probes(int n, uint8_t *bits, cudaStream_t s) {
  count_launch();
  probes_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, FA_PROBE_SEED, bits);
  return cudaGetLastError();
}

cudaError_t launch_stats(const StatsArgs &a, int nslices, cudaStream_t s) {
  count_launch();
  stats_kernel<<<dim3(stats_blocks(a.n), nslices), STATS_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_matrix_stats(const double *part, int n, double *mstats, cudaStream_t s) {
  count_launch();
  matrix_stats_kernel<<<1, 32, 0, s>>>(part, stats_blocks(n), mstats);
  return cudaGetLastError();
}

cudaError_t launch_records(const double *part, int nslices, int n, int N_total, int slice0,
                           double dT, const RecordScale &sc, const double *mstats, double *rec,
                           cudaStream_t s) {
  count_launch();
  records_kernel<<<(nslices + 63) / 64, 64, 0, s>>>(part, nslices, stats_blocks(n), n, N_total,
                                                    slice0, dT, sc, mstats, rec);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float *P, int B, const double *feat, int fstride, float *coef,
                               int *fallbacks, cudaStream_t s) {
  count_launch();
  mlp_forward_kernel<<<(B + MLP_S - 1) / MLP_S, HID, 0, s>>>(P, B, feat, fstride, coef, fallbacks);
  return cudaGetLastError();
}

size_t mlp_train_scratch_bytes(int B) {
  const size_t b = static_cast<size_t>(B);
  return 256 + b * sizeof(double) + b * (NF + 4 * HID + NC) * sizeof(float) + 6 * 256;
}

MlpTrainBuffers mlp_train_buffers(void *scratch, int B) {
  MlpTrainBuffers tb;
  char *p = static_cast<char *>(scratch);
  auto take = [&](size_t bytes) {
    char *r = p;
    p += (bytes + 255) / 256 * 256;
    return r;
  };
  const size_t b = static_cast<size_t>(B);
  tb.loss = reinterpret_cast<double *>(take(b * sizeof(double)));
  tb.xs = reinterpret_cast<float *>(take(b * NF * sizeof(float)));
  tb.h1 = reinterpret_cast<float *>(take(b * HID * sizeof(float)));
  tb.h2 = reinterpret_cast<float *>(take(b * HID * sizeof(float)));
  tb.dz1 = reinterpret_cast<float *>(take(b * HID * sizeof(float)));
  tb.dz2 = reinterpret_cast<float *>(take(b * HID * sizeof(float)));
  tb.dc = reinterpret_cast<float *>(take(b * NC * sizeof(float)));
  return tb;
}

cudaError_t launch_mlp_loss_grad(const float *P, int B, const double *rec, void *scratch,
                                 float *grad, double *loss, cudaStream_t s) {
  const MlpTrainBuffers tb = mlp_train_buffers(scratch, B);
  count_launch();
  mlp_train_kernel<<<(B + MLP_S - 1) / MLP_S, HID, 0, s>>>(P, B, rec, tb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  mlp_grad_kernel<<<(NPARAM + 1 + 127) / 128, 128, 0, s>>>(B, tb, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float *P, const float *grad, float *m, float *v, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t s) {
  count_launch();
  adam_kernel<<<(NPARAM - OFF_W1 + 255) / 256, 256, 0, s>>>(P, grad, m, v, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_coarse_coef(const float *P, const double *part, int n, int slice, int N,
                               double dT, const double *mstats, float *coef, int *fallbacks,
                               cudaStream_t s) {
  count_launch();
  coarse_coef_kernel<<<1, HID, 0, s>>>(P, part, stats_blocks(n), n, slice, N, dT, mstats, coef,
                                       fallbacks);
  return cudaGetLastError();
}

cudaError_t launch_combine(const CombineArgs &a, int blocks, cudaStream_t s) {
  count_launch();
  combine_kernel<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fa
