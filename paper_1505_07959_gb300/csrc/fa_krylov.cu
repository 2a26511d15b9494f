// Kernels of the modified parareal (Section 3 of the paper): Frobenius inner products of float64
// matrices (entries of the diamond product), the Gram-Schmidt steps of globalQR (Algorithm 2),
// and the projection update of Algorithm 3.  These are streaming kernels (each reads a few
// n x n float64 matrices once); every reduction runs on a fixed grid in a fixed order, so the
// results are bitwise reproducible.
#include "fa_internal.h"

namespace fa {

namespace {

constexpr int KT = 256;   // threads per block

// Sum of a block's per-thread values (fixed tree order); the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < KT / 32; ++w) t += red[w];
  __syncthreads();
  return t;
}

// Element range [k0, k1) of block b when `count` elements are split over the grid.
__device__ __forceinline__ void block_range(size_t count, size_t &k0, size_t &k1) {
  const size_t chunk = (count + gridDim.x - 1) / gridDim.x;
  k0 = static_cast<size_t>(blockIdx.x) * chunk;
  k1 = k0 + chunk < count ? k0 + chunk : count;
}

// One step of the Gram-Schmidt loop on the work matrix q:
//   if prev: c = sum of part_in[0 .. kKrylovBlocks) (the previous step's <q, prev>), q -= c prev;
//   part_out[block] = partial sum of <q, next> (next != null) or of <q, q> (next == null).
__global__ void __launch_bounds__(KT) gs_step_kernel(double *q, const double *__restrict__ prev,
                                                     const double *__restrict__ part_in,
                                                     const double *__restrict__ next,
                                                     size_t count, double *part_out) {
  __shared__ double red[KT / 32];
  __shared__ double coef;
  if (prev) {
    double s = 0.0;
    for (int i = threadIdx.x; i < kKrylovBlocks; i += KT) s += part_in[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) coef = s;
    __syncthreads();
  }
  const double c = prev ? coef : 0.0;
  size_t k0, k1;
  block_range(count, k0, k1);
  double acc = 0.0;
  for (size_t k = k0 + threadIdx.x; k < k1; k += KT) {
    double v = q[k];
    if (prev) {
      v -= c * prev[k];
      q[k] = v;
    }
    acc += v * (next ? next[k] : v);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part_out[blockIdx.x] = acc;
}

__global__ void scale_copy_kernel(const double *__restrict__ q, double s, size_t count,
                                  double *__restrict__ out) {
  for (size_t k = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; k < count;
       k += static_cast<size_t>(gridDim.x) * blockDim.x)
    out[k] = q[k] * s;
}

constexpr int MD = 8;   // basis blocks per multi-dot block row

// part[j][block] = partial <V, Q_j> for j in [0, d), MD blocks per grid row (blockIdx.y).
__global__ void __launch_bounds__(KT) multi_dot_kernel(const double *__restrict__ V,
                                                       const double *__restrict__ Q, size_t count,
                                                       int d, double *part) {
  __shared__ double red[KT / 32];
  const int j0 = blockIdx.y * MD;
  const int nj = d - j0 < MD ? d - j0 : MD;
  size_t k0, k1;
  block_range(count, k0, k1);
  double acc[MD];
#pragma unroll
  for (int t = 0; t < MD; ++t) acc[t] = 0.0;
  for (size_t k = k0 + threadIdx.x; k < k1; k += KT) {
    const double v = V[k];
#pragma unroll
    for (int t = 0; t < MD; ++t)
      if (t < nj) acc[t] += v * Q[static_cast<size_t>(j0 + t) * count + k];
  }
#pragma unroll
  for (int t = 0; t < MD; ++t) {
    if (t >= nj) break;
    const double s = block_sum(acc[t], red);
    if (threadIdx.x == 0) part[static_cast<size_t>(j0 + t) * kKrylovBlocks + blockIdx.x] = s;
  }
}

// alpha[j] = sum over blocks of part[j][.] (sequential, fixed order).
__global__ void reduce_alpha_kernel(const double *__restrict__ part, int d, double *alpha) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  double s = 0.0;
  for (int b = 0; b < kKrylovBlocks; ++b) s += part[static_cast<size_t>(j) * kKrylovBlocks + b];
  alpha[j] = s;
}

// R = V - sum_j alpha_j Q_j (the part of V outside the space), W = sum_j alpha_j FQ_j (the fine
// image of its projection), j in order.
__global__ void __launch_bounds__(KT) project_combine_kernel(
    const double *__restrict__ V, const double *__restrict__ Q, const double *__restrict__ FQ,
    const double *__restrict__ alpha, int d, size_t count, double *__restrict__ R,
    double *__restrict__ W) {
  extern __shared__ double a_s[];
  for (int j = threadIdx.x; j < d; j += blockDim.x) a_s[j] = alpha[j];
  __syncthreads();
  for (size_t k = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; k < count;
       k += static_cast<size_t>(gridDim.x) * blockDim.x) {
    double r = V[k], w = 0.0;
    for (int j = 0; j < d; ++j) {
      const double a = a_s[j];
      r -= a * Q[static_cast<size_t>(j) * count + k];
      w += a * FQ[static_cast<size_t>(j) * count + k];
    }
    R[k] = r;
    W[k] = w;
  }
}

int stream_blocks(size_t count) {
  const size_t b = (count + KT - 1) / KT;
  return static_cast<int>(b < 2048 ? (b ? b : 1) : 2048);
}

}  // namespace

cudaError_t launch_gs_step(double *q, const double *prev, const double *part_in,
                           const double *next, size_t count, double *part_out, cudaStream_t s) {
  gs_step_kernel<<<kKrylovBlocks, KT, 0, s>>>(q, prev, part_in, next, count, part_out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(const double *q, double scale, size_t count, double *out,
                              cudaStream_t s) {
  scale_copy_kernel<<<stream_blocks(count), KT, 0, s>>>(q, scale, count, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_project_alpha(const double *V, const double *Q, size_t count, int d,
                                 double *part, double *alpha, cudaStream_t s) {
  if (d <= 0) return cudaSuccess;
  dim3 grid(kKrylovBlocks, (d + MD - 1) / MD);
  multi_dot_kernel<<<grid, KT, 0, s>>>(V, Q, count, d, part);
  count_launch();
  reduce_alpha_kernel<<<(d + 127) / 128, 128, 0, s>>>(part, d, alpha);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_project_combine(const double *V, const double *Q, const double *FQ,
                                   const double *alpha, int d, size_t count, double *R, double *W,
                                   cudaStream_t s) {
  project_combine_kernel<<<stream_blocks(count), KT, static_cast<size_t>(d > 0 ? d : 1) * sizeof(double),
                           s>>>(V, Q, FQ, alpha, d, count, R, W);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fa
