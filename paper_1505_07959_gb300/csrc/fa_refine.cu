// Helpers of the square-root refinement (Newton steps for X^2 = A whose Sylvester equations are
// solved by the Newton-Schulz sign iteration on the tensor cores): a power iteration for the
// largest eigenvalue, symmetric combinations of matrices and their transposes, and the
// deviation norm that stops the sign iteration.  Every reduction runs in a fixed order.
#include "fa_internal.h"

namespace fa {

namespace {

constexpr int RT = 32;   // transpose tile

// y = X v, one warp per row, lanes striding the columns, xor-butterfly sum.
__global__ void matvec_kernel(const double *__restrict__ X, int n, const double *__restrict__ v,
                              double *__restrict__ y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double *row = X + static_cast<size_t>(warp) * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += row[j] * v[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[warp] = s;
}

// v = y / ||y||, lam = ||y|| (one block of 1024 threads, fixed-order reduction).
__global__ void __launch_bounds__(1024) normalize_kernel(const double *__restrict__ y, int n,
                                                         double *__restrict__ v, double *lam) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += y[i] * y[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 32; ++w) t += red[w];
    red[0] = sqrt(t);
    *lam = red[0];
  }
  __syncthreads();
  const double nrm = red[0];
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = nrm > 0.0 ? y[i] / nrm : 0.0;
}

// out = a (A + A^T)/2 + b B + c (C + C^T)/2 (null operands contribute nothing); tiles of 32 x 32
// so that the transposed reads are coalesced.  out may alias B (each element of B is read by
// the thread that writes it), not A or C.
__global__ void sym_combine_kernel(int n, double a, const double *__restrict__ A, double b,
                                   const double *B, double c, const double *__restrict__ C,
                                   double *out) {
  __shared__ double ta[RT][RT + 1], tc[RT][RT + 1];
  const int i0 = blockIdx.y * RT, j0 = blockIdx.x * RT;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int r = ty; r < RT; r += 8) {
    const int gi = j0 + r, gj = i0 + tx;          // transposed tile (rows j0.., cols i0..)
    const bool ok = gi < n && gj < n;
    ta[r][tx] = (A && ok) ? A[static_cast<size_t>(gi) * n + gj] : 0.0;
    tc[r][tx] = (C && ok) ? C[static_cast<size_t>(gi) * n + gj] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < RT; r += 8) {
    const int i = i0 + r, j = j0 + tx;
    if (i >= n || j >= n) continue;
    const size_t e = static_cast<size_t>(i) * n + j;
    double v = 0.0;
    if (A) v += a * 0.5 * (A[e] + ta[tx][r]);
    if (B) v += b * B[e];
    if (C) v += c * 0.5 * (C[e] + tc[tx][r]);
    out[e] = v;
  }
}

// part[block] = sum over the block's elements of (T - d I)^2.
__global__ void __launch_bounds__(256) dev_norm_kernel(const double *__restrict__ T, int n,
                                                       double d, double *part) {
  const size_t nn = static_cast<size_t>(n) * n;
  const size_t chunk = (nn + gridDim.x - 1) / gridDim.x;
  const size_t e0 = blockIdx.x * chunk;
  const size_t e1 = e0 + chunk < nn ? e0 + chunk : nn;
  double s = 0.0;
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) s += T[e] * T[e];
  // diagonal corrections (t - d)^2 - t^2, the diagonal shared out over all blocks
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double t = T[static_cast<size_t>(i) * n + i];
    s += (t - d) * (t - d) - t * t;
  }
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void fill_kernel(double *x, size_t count, double v) {
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < count) x[i] = v;
}

__global__ void sum_parts_kernel(const double *part, int count, double *out) {
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int k = 0; k < count; ++k) t += part[k];
  *out = t;
}

}  // namespace

cudaError_t launch_power_step(const double *X, int n, double *v, double *y, double *lam,
                              cudaStream_t s) {
  count_launch();
  matvec_kernel<<<(n + 7) / 8, 256, 0, s>>>(X, n, v, y);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  normalize_kernel<<<1, 1024, 0, s>>>(y, n, v, lam);
  return cudaGetLastError();
}

cudaError_t launch_sym_combine(int n, double a, const double *A, double b, const double *B,
                               double c, const double *C, double *out, cudaStream_t s) {
  count_launch();
  sym_combine_kernel<<<dim3((n + RT - 1) / RT, (n + RT - 1) / RT), dim3(RT, 8), 0, s>>>(
      n, a, A, b, B, c, C, out);
  return cudaGetLastError();
}

cudaError_t launch_fill(double *x, size_t count, double v, cudaStream_t s) {
  count_launch();
  fill_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, s>>>(x, count, v);
  return cudaGetLastError();
}

cudaError_t launch_dev_norm(const double *T, int n, double d, double *part, double *out,
                            cudaStream_t s) {
  count_launch();
  dev_norm_kernel<<<kDevNormBlocks, 256, 0, s>>>(T, n, d, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  sum_parts_kernel<<<1, 32, 0, s>>>(part, kDevNormBlocks, out);
  return cudaGetLastError();
}

}  // namespace fa
