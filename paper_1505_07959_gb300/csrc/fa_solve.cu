// Dense float64 solve for the Crank-Nicolson propagators of the linear flow (Section 2,
// Example 2).  A Crank-Nicolson step of dX/dt = A X with step h is
//     (I - h/2 A) X_{j+1} = (I + h/2 A) X_j,   i.e.   X_{j+1} = X_j + h M X_j,
// M = (I - h/2 A)^{-1} A (since (I + h/2 A) - (I - h/2 A) = h A).  M is constant, so it is formed
// once per matrix by Gauss-Jordan elimination with partial pivoting on the augmented matrix
// [I - c A | A], c = h/2, after which every step is one product in the increment form above.
// One pivot column per pair of launches (pivot search, row swap and scaling in one block; the
// elimination over the grid), so the work is O(n^3) float64 and the order of operations is
// fixed: bitwise reproducible.
#include "fa_internal.h"

namespace fa {

namespace {

constexpr int GJ_THREADS = 1024;

// aug (n x 2n, row-major) = [I - c A | A]
__global__ void gj_build_kernel(const double *__restrict__ A, int n, double c, double *aug) {
  const size_t total = static_cast<size_t>(n) * 2 * n;
  for (size_t k = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t i = k / (2 * static_cast<size_t>(n)), j = k % (2 * static_cast<size_t>(n));
    if (j < static_cast<size_t>(n))
      aug[k] = (i == j ? 1.0 : 0.0) - c * A[i * n + j];
    else
      aug[k] = A[i * n + (j - n)];
  }
}

// Column k: the row r >= k of largest |aug[r][k]| (the first such row on ties) is swapped into
// row k, and row k is divided by its pivot.  A zero pivot marks the matrix singular (*err).
__global__ void __launch_bounds__(GJ_THREADS) gj_pivot_kernel(double *aug, int n, int k,
                                                               int *err) {
  __shared__ double bv[GJ_THREADS / 32];
  __shared__ int bi[GJ_THREADS / 32];
  __shared__ int piv;
  __shared__ double pval;
  const size_t w = 2 * static_cast<size_t>(n);
  double best = -1.0;
  int bidx = n;
  for (int r = k + threadIdx.x; r < n; r += GJ_THREADS) {
    const double a = fabs(aug[r * w + k]);
    if (a > best) {            // rows visited in increasing order: the first maximum stays
      best = a;
      bidx = r;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) {
      best = ob;
      bidx = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    bv[threadIdx.x >> 5] = best;
    bi[threadIdx.x >> 5] = bidx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -1.0;
    int ix = n;
    for (int q = 0; q < GJ_THREADS / 32; ++q)
      if (bv[q] > b || (bv[q] == b && bi[q] < ix)) {
        b = bv[q];
        ix = bi[q];
      }
    piv = ix;
    pval = ix < n ? aug[ix * w + k] : 0.0;
    if (!(b > 0.0) && err) atomicCAS(err, 0, static_cast<int>(FA_ERR_NONFINITE));
  }
  __syncthreads();
  const int r = piv;
  if (r >= n) return;
  const double inv = 1.0 / pval;
  for (size_t j = threadIdx.x; j < w; j += GJ_THREADS) {
    const double a = aug[static_cast<size_t>(r) * w + j];
    if (r != k) aug[static_cast<size_t>(r) * w + j] = aug[static_cast<size_t>(k) * w + j];
    aug[static_cast<size_t>(k) * w + j] = a * inv;
  }
}

// Eliminate column k from every other row: aug[i][j] -= aug[i][k] aug[k][j] for j > k (column k
// itself is never read again, so it is left as it is and no thread reads a value another
// thread of this launch writes).
__global__ void gj_eliminate_kernel(double *aug, int n, int k) {
  const size_t w = 2 * static_cast<size_t>(n);
  const size_t cols = w - k - 1;
  const size_t total = static_cast<size_t>(n) * cols;
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t i = t / cols, j = k + 1 + t % cols;
    if (i == static_cast<size_t>(k)) continue;
    const double f = aug[i * w + k];
    if (f != 0.0) aug[i * w + j] -= f * aug[static_cast<size_t>(k) * w + j];
  }
}

__global__ void gj_extract_kernel(const double *__restrict__ aug, int n, double *__restrict__ M) {
  const size_t nn = static_cast<size_t>(n) * n;
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < nn;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t i = t / n, j = t % n;
    M[t] = aug[i * 2 * n + n + j];
  }
}

int grid_for(size_t count) {
  const size_t b = (count + 255) / 256;
  return static_cast<int>(b < 8192 ? (b ? b : 1) : 8192);
}

}  // namespace

cudaError_t launch_cn_matrix(const double *A, int n, double c, double *aug, double *M, int *err,
                             cudaStream_t s) {
  const size_t nn = static_cast<size_t>(n) * n;
  gj_build_kernel<<<grid_for(2 * nn), 256, 0, s>>>(A, n, c, aug);
  count_launch();
  for (int k = 0; k < n; ++k) {
    gj_pivot_kernel<<<1, GJ_THREADS, 0, s>>>(aug, n, k, err);
    count_launch();
    gj_eliminate_kernel<<<grid_for(static_cast<size_t>(n) * (2 * n - k - 1)), 256, 0, s>>>(aug, n, k);
    count_launch();
  }
  gj_extract_kernel<<<grid_for(nn), 256, 0, s>>>(aug, n, M);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fa

// ---- cosine by Algorithm 5 (Section 3, Example 3) -------------------------------------------

namespace fa {

namespace {

// out[0] = ||A||_inf = max_i sum_j |A_ij| (one block; rows summed in order, maximum in a fixed
// tree order).
__global__ void __launch_bounds__(1024) inf_norm_kernel(const double *__restrict__ A, int n,
                                                         double *out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += fabs(A[static_cast<size_t>(i) * n + j]);
    m = fmax(m, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) t = fmax(t, red[w]);
    out[0] = t;
  }
}

// B = [[0, s A], [-s A, 0]] (order 2n) and X0 = [[0, 0], [0, I]] (eq. eqB from U(0) = (0; I),
// embedded as the second block column of an order-2n state).
__global__ void cos_block_kernel(const double *__restrict__ A, int n, double s, double *B,
                                 double *X0) {
  const size_t m = 2 * static_cast<size_t>(n), total = m * m;
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t i = t / m, j = t % m;
    double b = 0.0;
    if (i < static_cast<size_t>(n) && j >= static_cast<size_t>(n)) b = s * A[i * n + (j - n)];
    if (i >= static_cast<size_t>(n) && j < static_cast<size_t>(n)) b = -s * A[(i - n) * n + j];
    B[t] = b;
    X0[t] = (i == j && i >= static_cast<size_t>(n)) ? 1.0 : 0.0;
  }
}

// out (n x n) = the block (r0.., c0..) of the order-2n matrix U.
__global__ void extract_block_kernel(const double *__restrict__ U, int n, int r0, int c0,
                                     double *__restrict__ out) {
  const size_t nn = static_cast<size_t>(n) * n, m = 2 * static_cast<size_t>(n);
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < nn;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t i = t / n, j = t % n;
    out[t] = U[(r0 + i) * m + c0 + j];
  }
}

}  // namespace

cudaError_t launch_inf_norm(const double *A, int n, double *out, cudaStream_t s) {
  inf_norm_kernel<<<1, 1024, 0, s>>>(A, n, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cos_block(const double *A, int n, double scale, double *B, double *X0,
                             cudaStream_t s) {
  cos_block_kernel<<<grid_for(4 * static_cast<size_t>(n) * n), 256, 0, s>>>(A, n, scale, B, X0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_extract_block(const double *U, int n, int r0, int c0, double *out,
                                 cudaStream_t s) {
  extract_block_kernel<<<grid_for(static_cast<size_t>(n) * n), 256, 0, s>>>(U, n, r0, c0, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fa
