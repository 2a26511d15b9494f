// Float64 path: a batched SIMT GEMM (float64 FMA; sm_103 has no float64
// tensor-core kind) with the same fused epilogues as the tensor-core path,
// on row-major float64 state.  This is the plain float64 GPU parareal, used
// where 1e-12 agreement with the oracle is required and for the float64
// refinement steps.  Each output element accumulates its dot product in a
// fixed k order, so results are bitwise reproducible.
#include <math_constants.h>

#include "fa_internal.h"
#include "fa_ptx.cuh"

namespace fa {

namespace {

constexpr int F64_BK = 16;
constexpr int F64_THREADS = 256;

// Epilogue of one element (i, j) of slice b with product value v.
__device__ __forceinline__ void epi_f64(const EpiParams &e, int b, int i, int j, double v,
                                        double &s0, double &s1) {
  const int n = e.n;
  const size_t nn = static_cast<size_t>(n) * n;
  const size_t r = static_cast<size_t>(i) * n + j;
  switch (e.mode) {
    case EPI_STAGE: {
      const size_t g = b * nn + r;
      double K = v;
      if (e.flow == FA_FLOW_SQRT) K = e.a64[r] - v;
      double *X = e.x64, *ac = e.acc64;
      if (e.stage == 1) {
        ac[g] = K;
        e.out64[g] = X[g] + e.ch * K;
      } else if (e.stage < 4) {
        ac[g] = ac[g] + 2.0 * K;
        e.out64[g] = X[g] + e.ch * K;
      } else {
        const double Xn = e.euler_step ? X[g] + e.h * K : X[g] + (e.h / 6.0) * (ac[g] + K);
        X[g] = Xn;
        if (e.last) {
          e.f_out[g] = e.g_old ? Xn - e.g_old[g] : Xn;
        } else {
          e.out64[g] = Xn;
        }
      }
      break;
    }
    case EPI_PROD:
    case EPI_TAYLOR:
      e.out64[b * nn + r] = v;
      break;
    case EPI_EULER: {
      double K = v;
      if (e.flow == FA_FLOW_SQRT) K = e.a64[r] - v;
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
      break;
    }
    case EPI_AIMA: {
      // Algorithm 8: slice 0 is X, slice 1 the control u (float64, current state in x64, next in
      // out64); v = (A X)_ij or (A u)_ij.  The residual (I - A X)_ij of the current X is summed.
      if (b == 0) {
        const double res = (i == j ? 1.0 : 0.0) - v;
        s0 += res * res;
        if (!e.last) e.out64[r] = e.x64[r] + e.dt * (res + e.x64[nn + r]);
      } else if (!e.last) {
        e.out64[nn + r] = e.x64[nn + r] - e.dt * v;
      }
      break;
    }
    default:
      e.store_out[b * nn + r] = e.alpha * v + (i == j ? e.beta : 0.0) +
                                (e.store_add ? e.store_add[b * nn + r] : 0.0);
      break;
  }
}

template <int TM>
__global__ void __launch_bounds__(F64_THREADS)
    f64_gemm_kernel(const __grid_constant__ F64GemmParams p) {
  constexpr int TPT = TM / 16;
  __shared__ double Ls[F64_BK][TM + 1];
  __shared__ double Rs[F64_BK][TM + 1];
  __shared__ double red[F64_THREADS / 32][2];
  const int n = p.n;
  const int b = blockIdx.z;
  const int gb = p.epi.b0 + b;
  const double *L = p.L + static_cast<size_t>(gb) * p.l_stride;
  const double *R = p.R + static_cast<size_t>(gb) * p.r_stride;
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TM;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[TPT][TPT];
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int w = 0; w < TPT; ++w) acc[u][w] = 0.0;

  for (int k0 = 0; k0 < n; k0 += F64_BK) {
    for (int idx = threadIdx.x; idx < TM * F64_BK; idx += F64_THREADS) {
      const int rr = idx / F64_BK, c = idx % F64_BK;
      const int gi = i0 + rr, gk = k0 + c;
      Ls[c][rr] = (gi < n && gk < n) ? L[static_cast<size_t>(gi) * n + gk] : 0.0;
    }
    for (int idx = threadIdx.x; idx < F64_BK * TM; idx += F64_THREADS) {
      const int rr = idx / TM, c = idx % TM;
      const int gk = k0 + rr, gj = j0 + c;
      Rs[rr][c] = (gk < n && gj < n) ? R[static_cast<size_t>(gk) * n + gj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < F64_BK; ++k) {
      double a[TPT], bb[TPT];
#pragma unroll
      for (int u = 0; u < TPT; ++u) {
        a[u] = Ls[k][ty + 16 * u];
        bb[u] = Rs[k][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < TPT; ++u)
#pragma unroll
        for (int w = 0; w < TPT; ++w) acc[u][w] = fma(a[u], bb[w], acc[u][w]);
    }
    __syncthreads();
  }

  double s0 = 0.0, s1 = 0.0;
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int w = 0; w < TPT; ++w) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * w;
      if (i < n && j < n) epi_f64(p.epi, gb, i, j, acc[u][w], s0, s1);
    }

  if ((p.epi.mode == EPI_EULER && p.epi.u_old != nullptr) || (p.epi.mode == EPI_AIMA && gb == 0)) {
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
      for (int w = 0; w < F64_THREADS / 32; ++w) {
        t0 += red[w][0];
        t1 += red[w][1];
      }
      const size_t slot = static_cast<size_t>(blockIdx.y) * gridDim.x + blockIdx.x;
      p.epi.norm_part[2 * slot] = t0;
      p.epi.norm_part[2 * slot + 1] = t1;
    }
  }
}

}  // namespace

int f64_tile(int n, int nb) {
  const long t64 = static_cast<long>((n + 63) / 64) * ((n + 63) / 64) * nb;
  return t64 >= 2 * 152 ? 64 : 32;
}

int f64_tiles_per_slice(int n, int nb) {
  const int tm = f64_tile(n, nb);
  return ((n + tm - 1) / tm) * ((n + tm - 1) / tm);
}

cudaError_t launch_f64_gemm(const F64GemmParams &p, cudaStream_t s) {
  const int tm = f64_tile(p.n, p.nb);
  dim3 grid((p.n + tm - 1) / tm, (p.n + tm - 1) / tm, p.nb);
  if (tm == 64) {
    f64_gemm_kernel<64><<<grid, F64_THREADS, 0, s>>>(p);
  } else {
    f64_gemm_kernel<32><<<grid, F64_THREADS, 0, s>>>(p);
  }
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Small helpers.

namespace {

__global__ void reduce_norms_kernel(const double *part, int nslices, int tiles, double *norms) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nslices) return;
  double t0 = 0.0, t1 = 0.0;
  for (int t = 0; t < tiles; ++t) {
    t0 += part[2 * (static_cast<size_t>(b) * tiles + t)];
    t1 += part[2 * (static_cast<size_t>(b) * tiles + t) + 1];
  }
  norms[2 * b] = t0;
  norms[2 * b + 1] = t1;
}

__global__ void max_ratio_kernel(const double *norms, int nslices, double *dx, int *err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double m = 0.0;
  bool bad = false;
  for (int b = 0; b < nslices; ++b) {
    const double r = sqrt(norms[2 * b]) / sqrt(norms[2 * b + 1]);
    if (!isfinite(r)) bad = true;
    if (r > m) m = r;
  }
  dx[0] = bad ? CUDART_INF : m;
  if (bad && err) atomicCAS(err, 0, static_cast<int>(FA_ERR_NONFINITE));
}

__global__ void batch_norms_kernel(const BatchNorm *bn, int count, int N, double *dx, int *err) {
  const int p = blockIdx.x;
  if (p >= count) return;
  const double *part = bn[p].part;
  const int tiles = bn[p].tiles;
  double m = 0.0;
  bool bad = false;
  for (int b = threadIdx.x; b < N; b += blockDim.x) {
    double t0 = 0.0, t1 = 0.0;
    for (int t = 0; t < tiles; ++t) {
      t0 += part[2 * (static_cast<size_t>(b) * tiles + t)];
      t1 += part[2 * (static_cast<size_t>(b) * tiles + t) + 1];
    }
    const double r = sqrt(t0) / sqrt(t1);
    if (!isfinite(r)) bad = true;
    if (r > m) m = r;
  }
  for (int off = 16; off > 0; off >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    bad = __any_sync(0xffffffffu, bad);
  }
  if (threadIdx.x == 0) {
    dx[p] = bad ? CUDART_INF : m;
    if (bad && err) atomicCAS(err, 0, static_cast<int>(FA_ERR_NONFINITE));
  }
}

__global__ void i_minus_kernel(const double *A, int n, double *out) {
  const size_t nn = static_cast<size_t>(n) * n;
  for (size_t k = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; k < nn;
       k += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t i = k / n, j = k % n;
    out[k] = (i == j ? 1.0 : 0.0) - A[k];
  }
}

__global__ void colmajor_pair_kernel(const double *A, int n, float *hi, float *lo) {
  __shared__ double tile[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && j < n) ? A[static_cast<size_t>(i) * n + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (i < n && j < n) {
      const double x = tile[threadIdx.x][r];
      const float h = static_cast<float>(x);
      hi[static_cast<size_t>(j) * n + i] = h;
      lo[static_cast<size_t>(j) * n + i] = static_cast<float>(x - static_cast<double>(h));
    }
  }
}

__global__ void check_finite_kernel(const double *x, size_t count, int *err) {
  for (size_t k = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; k < count;
       k += static_cast<size_t>(gridDim.x) * blockDim.x) {
    if (!isfinite(x[k])) {
      atomicCAS(err, 0, static_cast<int>(FA_ERR_NONFINITE));
      return;
    }
  }
}

__global__ void identity_kernel(double *X, int n) {
  const size_t nn = static_cast<size_t>(n) * n;
  for (size_t k = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; k < nn;
       k += static_cast<size_t>(gridDim.x) * blockDim.x) {
    X[k] = (k / n == k % n) ? 1.0 : 0.0;
  }
}

int blocks_for(size_t count) {
  size_t b = (count + 255) / 256;
  return static_cast<int>(b < 4096 ? (b ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_reduce_norms(const double *part, int nslices, int tiles, double *norms,
                                cudaStream_t s) {
  reduce_norms_kernel<<<(nslices + 127) / 128, 128, 0, s>>>(part, nslices, tiles, norms);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_max_ratio(const double *norms, int nslices, double *dx, int *err,
                             cudaStream_t s) {
  max_ratio_kernel<<<1, 32, 0, s>>>(norms, nslices, dx, err);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch_norms(const BatchNorm *bn, int count, int N, double *dx, int *err,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  batch_norms_kernel<<<count, 32, 0, s>>>(bn, count, N, dx, err);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_i_minus(const double *A, int n, double *out, cudaStream_t s) {
  i_minus_kernel<<<blocks_for(static_cast<size_t>(n) * n), 256, 0, s>>>(A, n, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_colmajor_pair(const double *A, int n, float *hi, float *lo, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  colmajor_pair_kernel<<<grid, block, 0, s>>>(A, n, hi, lo);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const double *x, size_t count, int *err, cudaStream_t s) {
  check_finite_kernel<<<blocks_for(count), 256, 0, s>>>(x, count, err);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_identity(double *X, int n, cudaStream_t s) {
  identity_kernel<<<blocks_for(static_cast<size_t>(n) * n), 256, 0, s>>>(X, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fa
