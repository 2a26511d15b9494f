// Allocation-free split-BF16 matrix product.
//
// Some callers cannot allocate device memory: their device memory is budgeted up front by a
// host application that forbids allocations after start-up, or they hold only their inputs and
// outputs and have no way to own a workspace for the library.  fa_product_noalloc serves them:
// it runs the same tensor-core product as the planned path, but keeps its BF16 operand terms
// in a fixed array compiled into this library (every GPU that loads the library holds it, about
// 12 MB, until the process exits) and calls no cudaMalloc, cudaFree or allocating library
// routine.  It is a convenience outside the paper's method.
#include <cstring>
#include <mutex>

#include "fa_internal.h"

namespace {

constexpr int kMaxN = 1024;                                  // largest n the array holds
constexpr size_t kTermElems = 3ull * kMaxN * kMaxN;          // three BF16 terms of one operand
constexpr int kMaxDevices = 64;

// Scratch: the left operand's L-form terms, then the right operand's R-form terms.  Every call
// rewrites the part it reads, so nothing needs clearing between calls; calls that overlap on
// the GPU (different streams, or host threads) share this array and race.
__device__ __align__(256) __nv_bfloat16 g_scratch[2 * kTermElems];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Device address of the scratch array on the current device (first call per device looks it
// up with that device current and caches it; the lookup may load the module, so the first call
// on a device should come before any stream capture).
fa_status scratch_for_device(int dev, void **ptr, int *sms) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return fa::record_error(FA_ERR_UNSUPPORTED, "device index too large");
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return fa::record_error(FA_ERR_CUDA, cudaGetErrorString(e));
    int n = 0;
    const cudaError_t e2 = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e2 != cudaSuccess) return fa::record_error(FA_ERR_CUDA, cudaGetErrorString(e2));
    g_scratch_ptr[dev] = p;
    g_num_sms[dev] = n;
  }
  *ptr = g_scratch_ptr[dev];
  *sms = g_num_sms[dev];
  return FA_OK;
}

}  // namespace

extern "C" fa_status fa_product_noalloc(int n, int dtype, const double *dL, const double *dR,
                                        double *dC, void *stream) {
  if (n < 1 || n > kMaxN)
    return fa::record_error(FA_ERR_ARG, "fa_product_noalloc: n must be in [1, 1024]");
  if (dtype < FA_BF16 || dtype > FA_BF16X6)
    return fa::record_error(FA_ERR_ARG, "fa_product_noalloc: dtype must be one of FA_BF16*");
  if (!dL || !dR || !dC) return fa::record_error(FA_ERR_ARG, "fa_product_noalloc: null pointer");
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fa::record_error(FA_ERR_CUDA, cudaGetErrorString(ce));
  int major = 0, minor = 0;
  ce = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (ce != cudaSuccess) return fa::record_error(FA_ERR_CUDA, cudaGetErrorString(ce));
  if (major != 10 || minor != 3)
    return fa::record_error(FA_ERR_UNSUPPORTED, "fa_product_noalloc: device is not sm_103");
  void *scratch = nullptr;
  int sms = 0;
  fa_status st = scratch_for_device(dev, &scratch, &sms);
  if (st != FA_OK) return st;

  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const fa::PairSet ps = fa::pair_set(dtype);
  const int ldp = (n + 7) / 8 * 8;
  const size_t stride = static_cast<size_t>(n) * ldp;        // elements between terms
  __nv_bfloat16 *lterms = static_cast<__nv_bfloat16 *>(scratch);
  __nv_bfloat16 *rterms = lterms + kTermElems;

  ce = fa::launch_split_terms(dL, 1, n, ldp, lterms, ps.terms_l, stride, nullptr, 0, 0, 0, s);
  if (ce == cudaSuccess)
    ce = fa::launch_split_terms(dR, 1, n, ldp, nullptr, 0, 0, rterms, ps.terms_r, stride, 0, s);
  if (ce != cudaSuccess) return fa::record_error(FA_ERR_CUDA, cudaGetErrorString(ce));

  CUtensorMap tmL, tmR;
  st = fa::encode_terms_map(&tmL, lterms, n, ldp, 1, ps.terms_l, stride, 128);
  if (st != FA_OK) return st;
  st = fa::encode_terms_map(&tmR, rterms, n, ldp, 1, ps.terms_r, stride, 128);
  if (st != FA_OK) return st;

  fa::TcGemmParams g = fa::tc_launch_params(n, 1, 0, 0, ps);
  memset(&g.epi, 0, sizeof(g.epi));
  g.epi.mode = fa::EPI_STORE;
  g.epi.n = n;
  g.epi.ldp = ldp;
  g.epi.alpha = 1.0;
  g.epi.beta = 0.0;
  g.epi.store_out = dC;
  ce = fa::launch_tc_gemm(&tmL, &tmR, g, sms, s);
  if (ce != cudaSuccess) return fa::record_error(FA_ERR_CUDA, cudaGetErrorString(ce));
  return FA_OK;
}
