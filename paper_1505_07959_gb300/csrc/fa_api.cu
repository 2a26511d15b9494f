// Host driver and C ABI of libfa: plans, workspace layout, the fine and
// coarse sweeps of classical parareal (Algorithm 1) and the solve loop.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fa_internal.h"
#include "fa_ptx.cuh"

using fa::EpiParams;
using fa::F64GemmParams;
using fa::TcGemmParams;

namespace {

thread_local std::string g_last_error;
unsigned long long *g_prof = nullptr;   // diagnostics: per-role cycle counters of the TC kernel
long long g_wait_cycles = 0;            // diagnostics: wait limit of TC launches (0 = default)
int g_skip_loads_cta = -1;              // diagnostics: CTA that issues no loads (-1 = none)
thread_local unsigned long long g_launches = 0;

fa_status set_err(fa_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
fa_status set_err(fa_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define FA_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return set_err(FA_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                     __FILE__, __LINE__);                                                 \
  } while (0)

#define FA_TRY(call)              \
  do {                            \
    fa_status s_ = (call);        \
    if (s_ != FA_OK) return s_;   \
  } while (0)

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool is_mixed(int dt) { return dt >= FA_BF16 && dt <= FA_BF16X6; }

// Bump allocator over the workspace (256-byte aligned sub-buffers).  With a
// null base it only measures.
struct Carver {
  char *base;
  size_t off = 0;
  template <typename T>
  T *take(size_t count) {
    off = (off + 255) & ~static_cast<size_t>(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

}  // namespace

namespace fa {
void count_launch() { ++g_launches; }
fa_status record_error(fa_status s, const char *msg) { return set_err(s, "%s", msg); }
}  // namespace fa

struct fa_plan_s {
  fa_problem_desc d{};
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  bool mixed = false, cmixed = false;
  fa::PairSet ps{};
  int ldp = 0;
  size_t nn = 0;
  size_t ws_need = 0;
  char *ws = nullptr;
  bool matrix_set = false;

  // parareal state (float64 row-major)
  double *U = nullptr, *Gold = nullptr, *Gnew = nullptr, *D = nullptr;
  double *part = nullptr, *norms = nullptr, *dx = nullptr;
  double *Vtmp[2] = {nullptr, nullptr};
  double *A64 = nullptr, *B64 = nullptr, *Xin = nullptr, *Xout = nullptr, *R1 = nullptr,
         *R2 = nullptr;
  int *err = nullptr;
  int part_tiles = 0;   // partial-norm slots per slice

  // mixed fine state
  float *x_hi = nullptr, *x_lo = nullptr, *acc = nullptr, *a_hi = nullptr, *a_lo = nullptr;
  __nv_bfloat16 *Aop = nullptr, *Yl[2] = {nullptr, nullptr}, *Yr[2] = {nullptr, nullptr},
                *Pr = nullptr;
  // mixed coarse operands (single slice)
  __nv_bfloat16 *Vl[2] = {nullptr, nullptr}, *Vr[2] = {nullptr, nullptr}, *Pcr = nullptr;
  size_t strideY = 0, strideV = 0, strideA = 0;   // elements between terms
  // float64 fine state
  double *X64 = nullptr, *acc64 = nullptr, *Y64[2] = {nullptr, nullptr}, *P64 = nullptr,
         *Pc64 = nullptr;

  CUtensorMap tmA{}, tmYl[2]{}, tmYr[2]{}, tmPr{}, tmVl[2]{}, tmVr[2]{}, tmPcr{};

  // features (every plan: pair records need them)
  uint8_t *probes = nullptr;     // n bytes of probe sign bits
  double *mstats = nullptr;      // Gershgorin lower / upper bound, Hutchinson tr(A)
  double *spart = nullptr;       // stats partials of one slice
  bool mstats_valid = false;
  // learned coarse propagator
  bool learned = false;          // coarse_kind == FA_COARSE_LEARNED
  bool learned_active = false;   // cleared by the fallback to Euler inside a solve
  bool learned_check = false;    // compare the first iteration with Euler's (opt-in fallback)
  bool params_set = false;
  float *mlp = nullptr;          // network blob
  float *coef = nullptr;         // [N][4] coefficients of the last coarse sweep
  int *fallbacks = nullptr;      // slices whose network output was not finite
  double *Rc[4] = {nullptr, nullptr, nullptr, nullptr};   // raw Taylor powers of the coarse state
  __nv_bfloat16 *Tl[2] = {nullptr, nullptr}, *Tr[2] = {nullptr, nullptr};  // chain operand terms
  CUtensorMap tmTl[2]{}, tmTr[2]{};
  // square-root refinement: Newton steps whose Sylvester equations are solved by the
  // Newton-Schulz sign iteration in BF16x6 term products on the tensor cores
  double *Xs = nullptr, *Rm = nullptr, *Pm[2] = {nullptr, nullptr}, *Tm = nullptr,
         *Wm = nullptr, *Vm = nullptr, *Qm = nullptr, *pv = nullptr;
  __nv_bfloat16 *Lp[2] = {nullptr, nullptr}, *Lt = nullptr, *Lq = nullptr, *Lpq = nullptr;
  CUtensorMap tmLp[2]{}, tmLt{}, tmLq{}, tmLpq{};
  size_t strideS = 0;
  int sign_steps_last = 0;       // sign-iteration steps of the last Newton step (diagnostics)
  // launch schedule of the tensor-core products (fa_plan_autotune; -1 = the default rule)
  int tune_prefetch = -1, tune_raster = -1;
  std::string tuning;
  // pair recorder of fa_parareal_solve
  double *rec = nullptr;
  int rec_cap = 0, rec_count = 0;
  void *rec_scratch = nullptr;
  size_t rec_scratch_bytes = 0;

  // E4M3 fine operands (FA_FP8E4M3): bytes [N][n][ldp8] in L and R form, double-buffered by
  // stage, and the per-tile scales [parity][inverse scale, amax][N][qT][qT]
  bool fp8 = false;
  int ldp8 = 0, qT = 0;
  uint8_t *Yl8[2] = {nullptr, nullptr}, *Yr8[2] = {nullptr, nullptr};
  float *qbuf = nullptr;
  CUtensorMap tmYl8[2]{}, tmYr8[2]{};
  float *qinv(int par) const { return qbuf + (static_cast<size_t>(par) * 2) * d.N * qT * qT; }
  float *qamax(int par) const { return qbuf + (static_cast<size_t>(par) * 2 + 1) * d.N * qT * qT; }

  // modified parareal (Algorithm 3): the F-orthonormal basis Q of the space, the fine images
  // F(Q_i), reduction partials and the projection coefficients
  bool modified = false;
  int cap = 0;                   // capacity of the space in blocks
  double drop = 0.0;             // removal threshold of globalQR
  double *Qb = nullptr, *FQb = nullptr, *kpart = nullptr, *apart = nullptr, *alpha = nullptr;

  // time-stepping schemes (FA_SCHEME_*) of F and G; with Crank-Nicolson the exponential flow's
  // products use the step matrices M = (I - h/2 A)^{-1} A (fine) and (I - dt/2 A)^{-1} A
  // (coarse) in place of A
  int fsch = FA_SCHEME_RK4, csch = FA_SCHEME_EULER;
  double *MF64 = nullptr, *MG64 = nullptr, *aug = nullptr;
  __nv_bfloat16 *AopF = nullptr, *AopG = nullptr;
  CUtensorMap tmAF{}, tmAG{};
  const CUtensorMap &fine_tmA() const { return fsch == FA_SCHEME_CN ? tmAF : tmA; }
  const CUtensorMap &coarse_tmA() const { return csch == FA_SCHEME_CN ? tmAG : tmA; }
  const double *fine_A64() const { return fsch == FA_SCHEME_CN ? MF64 : A64; }
  const double *coarse_A64() const { return csch == FA_SCHEME_CN ? MG64 : A64; }

  bool aima = false;             // a plan of fa_aima_plan (Algorithm 8)
  // FA_FLOW_COS: the order-2n exponential-flow plan of eq. eqB's block flow, and the outer
  // plan's own buffers (block matrix, start state, result, double-angle iterates, scalar)
  fa_plan_s *inner = nullptr;
  size_t inner_ws = 0;
  double *Bm = nullptr, *X0b = nullptr, *Ub = nullptr, *Cw[2] = {nullptr, nullptr},
         *scal = nullptr;
  ~fa_plan_s() { delete inner; }

  bool needs_l() const { return d.flow != FA_FLOW_EXP; }  // Y in L form (left factor)
};

namespace {

constexpr int TC_BM = 128, TC_BN = 128;

size_t carve(fa_plan_s *p, char *base) {
  Carver c{base};
  const fa_problem_desc &d = p->d;
  if (p->inner) {
    // FA_FLOW_COS: the inner plan's workspace first, then the outer buffers
    c.take<char>(p->inner_ws);
    const size_t n2 = 4 * static_cast<size_t>(d.n) * d.n;
    p->Bm = c.take<double>(n2);
    p->X0b = c.take<double>(n2);
    p->Ub = c.take<double>(n2);
    p->Cw[0] = c.take<double>(static_cast<size_t>(d.n) * d.n);
    p->Cw[1] = c.take<double>(static_cast<size_t>(d.n) * d.n);
    p->scal = c.take<double>(4);
    p->err = c.take<int>(4);
    p->A64 = c.take<double>(static_cast<size_t>(d.n) * d.n);     // host-buffer solve: A, X
    p->Xout = c.take<double>(static_cast<size_t>(d.n) * d.n);
    return c.off + 256;
  }
  const size_t nn = p->nn;
  const size_t N = static_cast<size_t>(d.N);
  p->U = c.take<double>((N + 1) * nn);
  p->Gold = c.take<double>(N * nn);
  p->Gnew = c.take<double>(N * nn);
  p->D = c.take<double>(N * nn);
  p->part = c.take<double>(N * static_cast<size_t>(p->part_tiles) * 2);
  p->norms = c.take<double>(N * 2);
  p->dx = c.take<double>(4);
  p->err = c.take<int>(4);
  if (d.coarse_steps > 1) {
    p->Vtmp[0] = c.take<double>(nn);
    p->Vtmp[1] = c.take<double>(nn);
  }
  p->A64 = c.take<double>(nn);
  p->Xin = c.take<double>(nn);
  p->Xout = c.take<double>(nn);
  if (d.flow == FA_FLOW_INV && (!p->mixed || !p->cmixed)) p->B64 = c.take<double>(nn);
  p->R1 = c.take<double>(nn);
  p->R2 = c.take<double>(nn);
  const size_t ldp = static_cast<size_t>(p->ldp);
  const size_t tl = static_cast<size_t>(p->ps.terms_l), tr = static_cast<size_t>(p->ps.terms_r);
  if (p->mixed || p->cmixed) {
    p->strideA = static_cast<size_t>(d.n) * ldp;
    if (d.flow != FA_FLOW_SQRT) p->Aop = c.take<__nv_bfloat16>(tl * p->strideA);
    if (d.flow == FA_FLOW_SQRT) {
      p->a_hi = c.take<float>(nn);
      p->a_lo = c.take<float>(nn);
    }
  }
  if (p->fp8) {
    p->x_hi = c.take<float>(N * nn);
    p->x_lo = c.take<float>(N * nn);
    p->acc = c.take<float>(N * nn);
    for (int k = 0; k < 2; ++k) {
      p->Yl8[k] = c.take<uint8_t>(N * static_cast<size_t>(d.n) * p->ldp8);
      p->Yr8[k] = c.take<uint8_t>(N * static_cast<size_t>(d.n) * p->ldp8);
    }
    p->qbuf = c.take<float>(4 * N * static_cast<size_t>(p->qT) * p->qT);
  } else if (p->mixed) {
    p->x_hi = c.take<float>(N * nn);
    p->x_lo = c.take<float>(N * nn);
    p->acc = c.take<float>(N * nn);
    p->strideY = N * static_cast<size_t>(d.n) * ldp;
    for (int k = 0; k < 2; ++k) {
      p->Yr[k] = c.take<__nv_bfloat16>(tr * p->strideY);
      if (p->needs_l()) p->Yl[k] = c.take<__nv_bfloat16>(tl * p->strideY);
    }
    if (d.flow == FA_FLOW_INV) p->Pr = c.take<__nv_bfloat16>(tr * p->strideY);
  } else {
    p->X64 = c.take<double>(N * nn);
    p->acc64 = c.take<double>(N * nn);
    p->Y64[0] = c.take<double>(N * nn);
    p->Y64[1] = c.take<double>(N * nn);
    if (d.flow == FA_FLOW_INV) p->P64 = c.take<double>(N * nn);
  }
  if (p->cmixed) {
    p->strideV = static_cast<size_t>(d.n) * ldp;
    for (int k = 0; k < 2; ++k) {
      p->Vr[k] = c.take<__nv_bfloat16>(tr * p->strideV);
      if (p->needs_l()) p->Vl[k] = c.take<__nv_bfloat16>(tl * p->strideV);
    }
    if (d.flow == FA_FLOW_INV) p->Pcr = c.take<__nv_bfloat16>(tr * p->strideV);
  } else {
    if (d.flow == FA_FLOW_INV) p->Pc64 = c.take<double>(nn);
  }
  if (d.flow == FA_FLOW_SQRT && d.refine_steps > 0) {
    p->Xs = c.take<double>(nn);
    p->Rm = c.take<double>(nn);
    p->Pm[0] = c.take<double>(nn);
    p->Pm[1] = c.take<double>(nn);
    p->Tm = c.take<double>(nn);
    p->Wm = c.take<double>(nn);
    p->Vm = c.take<double>(nn);
    p->Qm = c.take<double>(nn);
    p->pv = c.take<double>(2 * static_cast<size_t>(d.n) + 8 + fa::kDevNormBlocks);
    p->strideS = static_cast<size_t>(d.n) * ldp;
    p->Lp[0] = c.take<__nv_bfloat16>(3 * p->strideS);
    p->Lp[1] = c.take<__nv_bfloat16>(3 * p->strideS);
    p->Lt = c.take<__nv_bfloat16>(3 * p->strideS);
    p->Lq = c.take<__nv_bfloat16>(3 * p->strideS);
    p->Lpq = c.take<__nv_bfloat16>(3 * p->strideS);
  }
  if (p->fsch == FA_SCHEME_CN) p->MF64 = c.take<double>(nn);
  if (p->csch == FA_SCHEME_CN) p->MG64 = c.take<double>(nn);
  if (p->fsch == FA_SCHEME_CN || p->csch == FA_SCHEME_CN) p->aug = c.take<double>(2 * nn);
  if (p->mixed && p->fsch == FA_SCHEME_CN) p->AopF = c.take<__nv_bfloat16>(tl * p->strideA);
  if (p->cmixed && p->csch == FA_SCHEME_CN) p->AopG = c.take<__nv_bfloat16>(tl * p->strideA);
  if (p->modified) {
    p->Qb = c.take<double>(static_cast<size_t>(p->cap) * nn);
    p->FQb = c.take<double>(static_cast<size_t>(p->cap) * nn);
    p->kpart = c.take<double>(3 * static_cast<size_t>(fa::kKrylovBlocks));
    p->apart = c.take<double>(static_cast<size_t>(p->cap) * fa::kKrylovBlocks);
    p->alpha = c.take<double>(static_cast<size_t>(p->cap));
  }
  p->probes = c.take<uint8_t>(static_cast<size_t>(d.n));
  p->mstats = c.take<double>(8);
  p->spart = c.take<double>(static_cast<size_t>(fa::stats_blocks(d.n)) * fa::NSTAT);
  p->coef = c.take<float>(N * FA_MLP_COEFS);
  p->fallbacks = c.take<int>(4);
  if (p->learned) {
    p->mlp = c.take<float>(FA_MLP_PARAMS);
    for (int j = 0; j < 4; ++j) p->Rc[j] = c.take<double>(nn);
    if (p->cmixed) {
      for (int k = 0; k < 2; ++k) {
        if (d.flow == FA_FLOW_INV) p->Tl[k] = c.take<__nv_bfloat16>(tl * p->strideV);
        else p->Tr[k] = c.take<__nv_bfloat16>(tr * p->strideV);
      }
    }
  }
  return c.off + 256;
}

fa_status encode(CUtensorMap *m, void *base, int n, int ldp, int nslices, int nterms,
                 size_t term_stride, int box_rows);

}  // namespace

namespace fa {
fa_status encode_terms_map(CUtensorMap *m, void *base, int n, int ldp, int nslices, int nterms,
                           size_t term_stride, int box_rows) {
  return encode(m, base, n, ldp, nslices, nterms, term_stride, box_rows);
}

TcGemmParams tc_launch_params(int n, int nb, int l_batched, int r_batched, const PairSet &ps) {
  TcGemmParams g;
  memset(&g, 0, sizeof(g));
  g.n = n;
  g.nb = nb;
  g.l_batched = l_batched;
  g.r_batched = r_batched;
  g.mt = (n + TC_BM - 1) / TC_BM;
  g.nt = (n + TC_BN - 1) / TC_BN;
  g.num_tiles = g.mt * g.nt * nb;
  g.kblocks = (n + 63) / 64;
  tc_schedule(ps, g);
  g.prof = g_prof;
  g.wait_cycles = g_wait_cycles;
  g.skip_loads_cta = g_skip_loads_cta;
  g.prefetch_state = ps.npairs == 1 ? 1 : 0;   // measured: +10 % at one pair, -2 % at six
  g.idesc = ptx::idesc_bf16_f32(TC_BM, TC_BN);
  return g;
}
}  // namespace fa

namespace {

fa_status encode(CUtensorMap *m, void *base, int n, int ldp, int nslices, int nterms,
                 size_t term_stride, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return set_err(FA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[4] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(n),
                        static_cast<cuuint64_t>(nslices), static_cast<cuuint64_t>(nterms)};
  cuuint64_t strides[3] = {static_cast<cuuint64_t>(ldp) * 2,
                           static_cast<cuuint64_t>(n) * ldp * 2,
                           static_cast<cuuint64_t>(term_stride) * 2};
  cuuint32_t box[4] = {64, static_cast<cuuint32_t>(box_rows), 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_err(FA_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return FA_OK;
}

// Tensor map over E4M3 operand bytes [nslices][n][ldp8] with a 128 x 128 box (128-byte rows).
fa_status encode8(CUtensorMap *m, void *base, int n, int ldp8, int nslices) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return set_err(FA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[4] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(n),
                        static_cast<cuuint64_t>(nslices), 1};
  cuuint64_t strides[3] = {static_cast<cuuint64_t>(ldp8),
                           static_cast<cuuint64_t>(n) * ldp8,
                           static_cast<cuuint64_t>(nslices) * n * ldp8};
  cuuint32_t box[4] = {128, 128, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_err(FA_ERR_CUDA, "cuTensorMapEncodeTiled (E4M3) failed (%d)", (int)r);
  return FA_OK;
}

fa_status encode_all(fa_plan_s *p) {
  const int n = p->d.n, ldp = p->ldp, N = p->d.N;
  const int tl = p->ps.terms_l, tr = p->ps.terms_r;
  if (p->fp8) {
    for (int k = 0; k < 2; ++k) {
      FA_TRY(encode8(&p->tmYl8[k], p->Yl8[k], n, p->ldp8, N));
      FA_TRY(encode8(&p->tmYr8[k], p->Yr8[k], n, p->ldp8, N));
    }
  }
  if (p->Lq) {
    // refinement operands are symmetric (or left factors): one row-major term map serves as
    // either operand (BM = BN)
    for (int k = 0; k < 2; ++k) FA_TRY(encode(&p->tmLp[k], p->Lp[k], n, ldp, 1, 3, p->strideS, TC_BM));
    FA_TRY(encode(&p->tmLt, p->Lt, n, ldp, 1, 3, p->strideS, TC_BM));
    FA_TRY(encode(&p->tmLq, p->Lq, n, ldp, 1, 3, p->strideS, TC_BM));
    FA_TRY(encode(&p->tmLpq, p->Lpq, n, ldp, 1, 3, p->strideS, TC_BM));
  }
  if (p->Aop) FA_TRY(encode(&p->tmA, p->Aop, n, ldp, 1, tl, p->strideA, TC_BM));
  if (p->AopF) FA_TRY(encode(&p->tmAF, p->AopF, n, ldp, 1, tl, p->strideA, TC_BM));
  if (p->AopG) FA_TRY(encode(&p->tmAG, p->AopG, n, ldp, 1, tl, p->strideA, TC_BM));
  if (p->mixed && !p->fp8) {
    for (int k = 0; k < 2; ++k) {
      FA_TRY(encode(&p->tmYr[k], p->Yr[k], n, ldp, N, tr, p->strideY, TC_BN));
      if (p->Yl[k]) FA_TRY(encode(&p->tmYl[k], p->Yl[k], n, ldp, N, tl, p->strideY, TC_BM));
    }
    if (p->Pr) FA_TRY(encode(&p->tmPr, p->Pr, n, ldp, N, tr, p->strideY, TC_BN));
  }
  if (p->cmixed) {
    for (int k = 0; k < 2; ++k) {
      FA_TRY(encode(&p->tmVr[k], p->Vr[k], n, ldp, 1, tr, p->strideV, TC_BN));
      if (p->Vl[k]) FA_TRY(encode(&p->tmVl[k], p->Vl[k], n, ldp, 1, tl, p->strideV, TC_BM));
    }
    if (p->Pcr) FA_TRY(encode(&p->tmPcr, p->Pcr, n, ldp, 1, tr, p->strideV, TC_BN));
    for (int k = 0; k < 2; ++k) {
      if (p->Tl[k]) FA_TRY(encode(&p->tmTl[k], p->Tl[k], n, ldp, 1, tl, p->strideV, TC_BM));
      if (p->Tr[k]) FA_TRY(encode(&p->tmTr[k], p->Tr[k], n, ldp, 1, tr, p->strideV, TC_BN));
    }
  }
  return FA_OK;
}

EpiParams base_epi(const fa_plan_s *p) {
  EpiParams e;
  memset(&e, 0, sizeof(e));
  e.flow = p->d.flow;
  e.n = p->d.n;
  e.ldp = p->ldp;
  e.err = p->err;
  return e;
}

TcGemmParams tc_params(const fa_plan_s *p, int nb, int l_batched, int r_batched,
                       const EpiParams &e) {
  TcGemmParams g = fa::tc_launch_params(p->d.n, nb, l_batched, r_batched, p->ps);
  if (p->tune_prefetch >= 0) g.prefetch_state = p->tune_prefetch;
  if (p->tune_raster >= 0) g.raster = p->tune_raster;
  g.epi = e;
  return g;
}

fa_status tc(const fa_plan_s *p, const CUtensorMap &L, const CUtensorMap &R, const TcGemmParams &g) {
  FA_CUDA(fa::launch_tc_gemm(&L, &R, g, p->num_sms, p->stream));
  return FA_OK;
}

fa_status f64(const fa_plan_s *p, const double *L, size_t ls, const double *R, size_t rs, int nb,
              const EpiParams &e) {
  F64GemmParams g;
  memset(&g, 0, sizeof(g));
  g.n = p->d.n;
  g.nb = nb;
  g.L = L;
  g.R = R;
  g.l_stride = ls;
  g.r_stride = rs;
  g.epi = e;
  FA_CUDA(fa::launch_f64_gemm(g, p->stream));
  return FA_OK;
}

fa_status check_ready(const fa_plan_s *p, bool need_matrix) {
  if (!p) return set_err(FA_ERR_ARG, "null plan");
  if (!p->ws) return set_err(FA_ERR_WORKSPACE, "no workspace bound");
  if (need_matrix && !p->matrix_set)
    return set_err(FA_ERR_ARG, "fa_plan_set_matrix has not been called");
  return FA_OK;
}

// ---- fine sweep ------------------------------------------------------------------------------

// The fine sweep with E4M3 stage operands (square-root flow).
fa_status fine_sweep_fp8(fa_plan_s *p, const double *U, double *out, const double *g_old) {
  const fa_problem_desc &d = p->d;
  const int n = d.n, N = d.N, J = d.fine_steps;
  const double h = d.T / static_cast<double>(N) / static_cast<double>(J);
  FA_CUDA(fa::launch_load_state(U, N, n, p->ldp, p->x_hi, p->x_lo, nullptr, 0, 0, nullptr, 0, 0,
                                p->stream));
  FA_CUDA(fa::launch_fp8_load(U, N, n, p->ldp8, p->Yl8[0], p->Yr8[0], p->qamax(0), p->qinv(0),
                              p->stream));
  fa::PairSet one;
  memset(&one, 0, sizeof(one));
  one.npairs = 1;
  one.terms_l = one.terms_r = 1;
  int cur = 0;
  for (int j = 0; j < J; ++j) {
    for (int s = 1; s <= 4; ++s) {
      const bool last = (j == J - 1 && s == 4);
      EpiParams e = base_epi(p);
      e.mode = fa::EPI_STAGE;
      e.stage = s;
      e.last = last ? 1 : 0;
      e.h = h;
      e.ch = (s == 3) ? h : (s < 3 ? 0.5 * h : 0.0);
      e.f_out = out;
      e.g_old = g_old;
      e.x_hi = p->x_hi;
      e.x_lo = p->x_lo;
      e.acc = p->acc;
      e.a_hi = p->a_hi;
      e.a_lo = p->a_lo;
      if (!last) {
        e.out_l8 = p->Yl8[cur ^ 1];
        e.out_r8 = p->Yr8[cur ^ 1];
        e.ldp8 = p->ldp8;
        e.q_T = p->qT;
        e.q_amax_in = p->qamax(cur);
        e.q_inv_out = p->qinv(cur ^ 1);
        e.q_amax_out = p->qamax(cur ^ 1);
      }
      TcGemmParams g = fa::tc_launch_params(n, N, 1, 1, one);
      g.fp8 = 1;
      g.kblocks = (n + 127) / 128;
      g.idesc = fa::ptx::idesc_e4m3_f32(TC_BM, TC_BN);
      g.q_inv_l = g.q_inv_r = p->qinv(cur);
      g.q_T = p->qT;
      if (p->tune_prefetch >= 0) g.prefetch_state = p->tune_prefetch;
      if (p->tune_raster >= 0) g.raster = p->tune_raster;
      g.epi = e;
      FA_TRY(tc(p, p->tmYl8[cur], p->tmYr8[cur], g));
      cur ^= 1;
    }
  }
  return FA_OK;
}

// F on every slice: out = F(U_b) (g_old == null) or F(U_b) - g_old_b, for b < nb (nb < 0: all
// N slices; at most N, the capacity of the fine state).
fa_status fine_sweep(fa_plan_s *p, const double *U, double *out, const double *g_old, int nb = -1) {
  if (p->fp8) return fine_sweep_fp8(p, U, out, g_old);
  const fa_problem_desc &d = p->d;
  const int n = d.n, N = nb < 0 ? d.N : nb, J = d.fine_steps;
  const double h = d.T / static_cast<double>(d.N) / static_cast<double>(J);
  const size_t nn = p->nn;
  const int tl = p->ps.terms_l, tr = p->ps.terms_r;
  if (N <= 0) return FA_OK;
  if (p->mixed) {
    FA_CUDA(fa::launch_load_state(U, N, n, p->ldp, p->x_hi, p->x_lo, p->Yl[0],
                                  p->needs_l() ? tl : 0, p->strideY, p->Yr[0], tr, p->strideY,
                                  p->stream));
  } else {
    FA_CUDA(cudaMemcpyAsync(p->X64, U, N * nn * sizeof(double), cudaMemcpyDeviceToDevice,
                            p->stream));
    FA_CUDA(cudaMemcpyAsync(p->Y64[0], U, N * nn * sizeof(double), cudaMemcpyDeviceToDevice,
                            p->stream));
  }
  int cur = 0;
  // RK4: four stage launches per step; explicit Euler and Crank-Nicolson: one explicit step
  // X <- X + h K per launch (the stage-4 epilogue with acc = 0 and h in place of h/6), K = Fl(X)
  // or, for Crank-Nicolson, M X
  const bool rk4 = p->fsch == FA_SCHEME_RK4;
  for (int j = 0; j < J; ++j) {
    for (int s = rk4 ? 1 : 4; s <= 4; ++s) {
      const bool last = (j == J - 1 && s == 4);
      EpiParams e = base_epi(p);
      e.mode = fa::EPI_STAGE;
      e.stage = s;
      e.last = last ? 1 : 0;
      e.h = h;
      e.ch = (s == 3) ? h : (s < 3 ? 0.5 * h : 0.0);
      e.euler_step = rk4 ? 0 : 1;
      e.f_out = out;
      e.g_old = g_old;
      if (p->mixed) {
        e.x_hi = p->x_hi;
        e.x_lo = p->x_lo;
        e.acc = p->acc;
        e.a_hi = p->a_hi;
        e.a_lo = p->a_lo;
        e.out_r = p->Yr[cur ^ 1];
        e.out_l = p->Yl[cur ^ 1];
        e.terms_r = tr;
        e.terms_l = p->needs_l() ? tl : 0;
        e.term_stride_r = e.term_stride_l = p->strideY;
        if (d.flow == FA_FLOW_EXP) {
          FA_TRY(tc(p, p->fine_tmA(), p->tmYr[cur], tc_params(p, N, 0, 1, e)));
        } else if (d.flow == FA_FLOW_SQRT) {
          FA_TRY(tc(p, p->tmYl[cur], p->tmYr[cur], tc_params(p, N, 1, 1, e)));
        } else {
          EpiParams e1 = base_epi(p);
          e1.mode = fa::EPI_PROD;
          e1.out_r = p->Pr;
          e1.terms_r = tr;
          e1.term_stride_r = p->strideY;
          FA_TRY(tc(p, p->tmA, p->tmYr[cur], tc_params(p, N, 0, 1, e1)));
          FA_TRY(tc(p, p->tmYl[cur], p->tmPr, tc_params(p, N, 1, 1, e)));
        }
      } else {
        e.x64 = p->X64;
        e.acc64 = p->acc64;
        e.a64 = p->A64;
        e.out64 = p->Y64[cur ^ 1];
        const double *Y = p->Y64[cur];
        if (d.flow == FA_FLOW_EXP) {
          FA_TRY(f64(p, p->fine_A64(), 0, Y, nn, N, e));
        } else if (d.flow == FA_FLOW_SQRT) {
          FA_TRY(f64(p, Y, nn, Y, nn, N, e));
        } else {
          EpiParams e1 = base_epi(p);
          e1.mode = fa::EPI_PROD;
          e1.out64 = p->P64;
          FA_TRY(f64(p, p->B64, 0, Y, nn, N, e1));
          FA_TRY(f64(p, Y, nn, p->P64, nn, N, e));
        }
      }
      cur ^= 1;
    }
  }
  return FA_OK;
}

// ---- coarse sweep ----------------------------------------------------------------------------

// Whether a tensor-core launch may compute the transposed product (X Y)^T = Y^T X^T with the
// two operands' term buffers swapped (an L-form buffer read as the R form of the transpose, and
// the other way round): the term pairs must be symmetric, so that the swapped launch forms the
// same term products.
bool transposable(const fa_plan_s *p) {
  const fa::PairSet &s = p->ps;
  if (s.terms_l != s.terms_r) return false;
  for (int k = 0; k < s.npairs; ++k) {
    bool found = false;
    for (int q = 0; q < s.npairs; ++q) found = found || (s.a[q] == s.b[k] && s.b[q] == s.a[k]);
    if (!found) return false;
  }
  return true;
}

// The product(s) of one forward-Euler substep on the single-slice coarse state vin (operand
// terms in Vl/Vr[cur] when the coarse arithmetic is mixed), with the Euler epilogue e.  Where
// the pair set allows, the Euler launch computes the transposed product ((A V)^T = V^T A^T;
// (V P)^T = P^T V^T; (V V)^T = V^T V^T), whose epilogue reaches the row-major float64 state with
// coalesced accesses.
fa_status euler_gemm(fa_plan_s *p, int cur, const double *vin, EpiParams e) {
  const fa_problem_desc &d = p->d;
  const int tr = p->ps.terms_r;
  if (p->cmixed) {
    e.a_hi = p->a_hi;
    e.a_lo = p->a_lo;
    const bool tp = transposable(p);
    if (d.flow == FA_FLOW_EXP) {
      if (tp) {
        e.transposed = 1;
        FA_TRY(tc(p, p->tmVr[cur], p->coarse_tmA(), tc_params(p, 1, 0, 0, e)));
      } else {
        FA_TRY(tc(p, p->coarse_tmA(), p->tmVr[cur], tc_params(p, 1, 0, 0, e)));
      }
    } else if (d.flow == FA_FLOW_SQRT) {
      if (tp) {
        // (V V)^T = V^T V^T; K = A - P takes A's entries from the row-major float64 copy
        e.transposed = 1;
        e.a64 = p->A64;
        FA_TRY(tc(p, p->tmVr[cur], p->tmVl[cur], tc_params(p, 1, 0, 0, e)));
      } else {
        FA_TRY(tc(p, p->tmVl[cur], p->tmVr[cur], tc_params(p, 1, 0, 0, e)));
      }
    } else {
      EpiParams e1 = base_epi(p);
      e1.mode = fa::EPI_PROD;
      e1.out_r = p->Pcr;
      e1.terms_r = tr;
      e1.term_stride_r = p->strideV;
      FA_TRY(tc(p, p->tmA, p->tmVr[cur], tc_params(p, 1, 0, 0, e1)));
      if (tp) {
        e.transposed = 1;
        FA_TRY(tc(p, p->tmPcr, p->tmVl[cur], tc_params(p, 1, 0, 0, e)));
      } else {
        FA_TRY(tc(p, p->tmVl[cur], p->tmPcr, tc_params(p, 1, 0, 0, e)));
      }
    }
  } else {
    e.a64 = p->A64;
    if (d.flow == FA_FLOW_EXP) {
      FA_TRY(f64(p, p->coarse_A64(), 0, vin, 0, 1, e));
    } else if (d.flow == FA_FLOW_SQRT) {
      FA_TRY(f64(p, vin, 0, vin, 0, 1, e));
    } else {
      EpiParams e1 = base_epi(p);
      e1.mode = fa::EPI_PROD;
      e1.out64 = p->Pc64;
      FA_TRY(f64(p, p->B64, 0, vin, 0, 1, e1));
      FA_TRY(f64(p, vin, 0, p->Pc64, 0, 1, e));
    }
  }
  return FA_OK;
}

// BF16 operand terms of a single-slice coarse state into Vl/Vr[k], split from the float32
// rounding as the Euler epilogue splits the states it writes: a sweep that starts from a state
// (Step 0, or a slice range's first state received from elsewhere) computes the same bits as one
// that reached it.
fa_status split_coarse(fa_plan_s *p, const double *v, int k) {
  FA_CUDA(fa::launch_split_terms(v, 1, p->d.n, p->ldp, p->Vl[k], p->needs_l() ? p->ps.terms_l : 0,
                                 p->strideV, p->Vr[k], p->ps.terms_r, p->strideV,
                                 fa::SPLIT_FROM_F32, p->stream));
  return FA_OK;
}

fa_status euler_coarse_sweep(fa_plan_s *p, const double *U0, const double *D, double *Unew,
                             double *Gout, double *norms, const double *Uold) {
  const fa_problem_desc &d = p->d;
  const int N = d.N, m = d.coarse_steps;
  const size_t nn = p->nn;
  const double dt = d.T / static_cast<double>(N) / static_cast<double>(m);
  const int tl = p->ps.terms_l, tr = p->ps.terms_r;
  int cur = 0;
  if (p->cmixed) FA_TRY(split_coarse(p, U0, 0));
  const int tiles = p->part_tiles;
  for (int s = 0; s < N; ++s) {
    for (int sub = 0; sub < m; ++sub) {
      const bool last = (sub == m - 1);
      const double *vin = (sub == 0) ? Unew + static_cast<size_t>(s) * nn : p->Vtmp[(sub - 1) & 1];
      double *vout = last ? Unew + static_cast<size_t>(s + 1) * nn : p->Vtmp[sub & 1];
      EpiParams e = base_epi(p);
      e.mode = fa::EPI_EULER;
      e.dt = dt;
      e.v_in = vin;
      e.v_out = vout;
      e.euler_last = last ? 1 : 0;
      if (last) {
        e.g_out = Gout + static_cast<size_t>(s) * nn;
        e.d_in = D ? D + static_cast<size_t>(s) * nn : nullptr;
        e.u_old = (norms && Uold) ? Uold + static_cast<size_t>(s + 1) * nn : nullptr;
        e.norm_part = p->part + static_cast<size_t>(s) * tiles * 2;
      }
      if (p->cmixed) {
        e.out_r = p->Vr[cur ^ 1];
        e.out_l = p->Vl[cur ^ 1];
        e.terms_r = tr;
        e.terms_l = p->needs_l() ? tl : 0;
        e.term_stride_r = e.term_stride_l = p->strideV;
      }
      FA_TRY(euler_gemm(p, cur, vin, e));
      if (p->cmixed) cur ^= 1;
    }
  }
  return FA_OK;
}

// Gershgorin bounds and Hutchinson tr(A) of the plan's matrix (once per matrix).
fa_status ensure_mstats(fa_plan_s *p) {
  if (p->mstats_valid) return FA_OK;
  fa::StatsArgs a;
  memset(&a, 0, sizeof(a));
  a.n = p->d.n;
  a.rows_per_block = fa::stats_rows_per_block(a.n);
  a.X = p->A64;
  a.probes = p->probes;
  a.gersh = 1;
  a.part = p->spart;
  FA_CUDA(fa::launch_stats(a, 1, p->stream));
  FA_CUDA(fa::launch_matrix_stats(p->spart, a.n, p->mstats, p->stream));
  p->mstats_valid = true;
  return FA_OK;
}

// Taylor scale s_j = dT^j kappa_j of the raw power R_j (kappa_j = 1 for the inverse flow,
// 1 / j! for the exponential flow).
fa::RecordScale taylor_scale(const fa_plan_s *p) {
  fa::RecordScale sc;
  const double dT = p->d.T / static_cast<double>(p->d.N);
  double pw = 1.0, fact = 1.0;
  for (int j = 0; j < 4; ++j) {
    pw *= dT;
    fact *= (j + 1);
    sc.s[j] = p->d.flow == FA_FLOW_EXP ? pw / fact : pw;
  }
  return sc;
}

// Raw Taylor powers R_1..R_4 of the single-slice coarse state vin into Rc (inverse flow:
// P = B V, R_1 = V P, R_{j+1} = R_j P; exponential flow: R_1 = A V, R_{j+1} = A R_j).
fa_status coarse_taylor(fa_plan_s *p, int cur, const double *vin) {
  const bool inv = p->d.flow == FA_FLOW_INV;
  const int tl = p->ps.terms_l, tr = p->ps.terms_r;
  if (p->cmixed) {
    if (inv) {
      EpiParams e1 = base_epi(p);
      e1.mode = fa::EPI_PROD;
      e1.out_r = p->Pcr;
      e1.terms_r = tr;
      e1.term_stride_r = p->strideV;
      FA_TRY(tc(p, p->tmA, p->tmVr[cur], tc_params(p, 1, 0, 0, e1)));
    }
    for (int j = 0; j < 4; ++j) {
      EpiParams e = base_epi(p);
      e.mode = fa::EPI_TAYLOR;
      e.out64 = p->Rc[j];
      if (j < 3) {
        if (inv) {
          e.out_l = p->Tl[j & 1];
          e.terms_l = tl;
          e.term_stride_l = p->strideV;
        } else {
          e.out_r = p->Tr[j & 1];
          e.terms_r = tr;
          e.term_stride_r = p->strideV;
        }
      }
      if (inv) {
        const CUtensorMap &L = j == 0 ? p->tmVl[cur] : p->tmTl[(j - 1) & 1];
        FA_TRY(tc(p, L, p->tmPcr, tc_params(p, 1, 0, 0, e)));
      } else {
        const CUtensorMap &R = j == 0 ? p->tmVr[cur] : p->tmTr[(j - 1) & 1];
        FA_TRY(tc(p, p->tmA, R, tc_params(p, 1, 0, 0, e)));
      }
    }
  } else {
    if (inv) {
      EpiParams e1 = base_epi(p);
      e1.mode = fa::EPI_PROD;
      e1.out64 = p->Pc64;
      FA_TRY(f64(p, p->B64, 0, vin, 0, 1, e1));
    }
    for (int j = 0; j < 4; ++j) {
      EpiParams e = base_epi(p);
      e.mode = fa::EPI_TAYLOR;
      e.out64 = p->Rc[j];
      const double *src = j == 0 ? vin : p->Rc[j - 1];
      if (inv) FA_TRY(f64(p, src, 0, p->Pc64, 0, 1, e));
      else FA_TRY(f64(p, p->A64, 0, src, 0, 1, e));
    }
  }
  return FA_OK;
}

// Coarse sweep with the learned polynomial step: per slice, the Taylor powers, the stats of
// the state, the network (one block) and the update with correction and norms.
fa_status learned_coarse_sweep(fa_plan_s *p, const double *U0, const double *D, double *Unew,
                               double *Gout, double *norms, const double *Uold) {
  const fa_problem_desc &d = p->d;
  if (!p->params_set) return set_err(FA_ERR_ARG, "fa_plan_set_learned has not been called");
  FA_TRY(ensure_mstats(p));
  const int n = d.n, N = d.N;
  const size_t nn = p->nn;
  const double dT = d.T / static_cast<double>(N);
  const fa::RecordScale sc = taylor_scale(p);
  const int tiles = p->part_tiles;
  int cur = 0;
  if (p->cmixed) FA_TRY(split_coarse(p, U0, 0));
  for (int s = 0; s < N; ++s) {
    const double *vin = Unew + static_cast<size_t>(s) * nn;
    double *vout = Unew + static_cast<size_t>(s + 1) * nn;
    FA_TRY(coarse_taylor(p, cur, vin));
    fa::StatsArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.rows_per_block = fa::stats_rows_per_block(n);
    a.X = vin;
    a.R[0] = p->Rc[0];
    a.nR = 1;
    a.probes = p->probes;
    a.part = p->spart;
    FA_CUDA(fa::launch_stats(a, 1, p->stream));
    float *cf = p->coef + static_cast<size_t>(s) * FA_MLP_COEFS;
    FA_CUDA(fa::launch_coarse_coef(p->mlp, p->spart, n, s, N, dT, p->mstats, cf, p->fallbacks,
                                   p->stream));
    fa::CombineArgs c;
    memset(&c, 0, sizeof(c));
    c.n = n;
    c.v_in = vin;
    for (int j = 0; j < 4; ++j) {
      c.R[j] = p->Rc[j];
      c.scale[j] = sc.s[j];
    }
    c.coef = cf;
    c.d_in = D ? D + static_cast<size_t>(s) * nn : nullptr;
    const bool nrm = norms && Uold;
    c.u_old = nrm ? Uold + static_cast<size_t>(s + 1) * nn : nullptr;
    c.g_out = Gout + static_cast<size_t>(s) * nn;
    c.v_out = vout;
    c.norm_part = nrm ? p->part + static_cast<size_t>(s) * tiles * 2 : nullptr;
    FA_CUDA(fa::launch_combine(c, tiles, p->stream));
    if (p->cmixed && s + 1 < N) {
      FA_TRY(split_coarse(p, vout, cur ^ 1));
      cur ^= 1;
    }
  }
  return FA_OK;
}

fa_status coarse_sweep(fa_plan_s *p, const double *U0, const double *D, double *Unew, double *Gout,
                       double *norms, const double *Uold) {
  const fa_problem_desc &d = p->d;
  if (Unew != U0)
    FA_CUDA(cudaMemcpyAsync(Unew, U0, p->nn * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  if (p->learned_active) FA_TRY(learned_coarse_sweep(p, U0, D, Unew, Gout, norms, Uold));
  else FA_TRY(euler_coarse_sweep(p, U0, D, Unew, Gout, norms, Uold));
  if (norms && Uold) FA_CUDA(fa::launch_reduce_norms(p->part, d.N, p->part_tiles, norms, p->stream));
  return FA_OK;
}

// Forward-Euler G of every slice of U into Gout (independent steps; the fallback of the learned
// propagator recomputes the cached G(U^k_n) with it).
fa_status euler_all(fa_plan_s *p, const double *U, double *Gout) {
  const fa_problem_desc &d = p->d;
  const size_t nn = p->nn;
  const double dt = d.T / static_cast<double>(d.N);
  for (int s = 0; s < d.N; ++s) {
    const double *vin = U + static_cast<size_t>(s) * nn;
    if (p->cmixed) FA_TRY(split_coarse(p, vin, 0));
    EpiParams e = base_epi(p);
    e.mode = fa::EPI_EULER;
    e.dt = dt;
    e.v_in = vin;
    e.v_out = Gout + static_cast<size_t>(s) * nn;
    e.g_out = Gout + static_cast<size_t>(s) * nn;
    e.euler_last = 1;
    FA_TRY(euler_gemm(p, 0, vin, e));
  }
  return FA_OK;
}

// ---- pair records ------------------------------------------------------------------------------

size_t records_scratch_bytes(const fa_plan_s *p) {
  const size_t N = static_cast<size_t>(p->d.N);
  return 4 * (N * p->nn * sizeof(double) + 256) +
         N * fa::stats_blocks(p->d.n) * fa::NSTAT * sizeof(double) + 256;
}

// Records of the pairs (U_b, F_b) (F_b = F[b] + G[b] when G is given) for b = 0..N-1, Taylor
// powers in the fine arithmetic (the fine sweep's operand buffers serve as chain storage).
fa_status records(fa_plan_s *p, const double *U, const double *F, const double *G, double *out,
                  void *scratch, size_t scratch_bytes) {
  const fa_problem_desc &d = p->d;
  if (d.flow == FA_FLOW_SQRT)
    return set_err(FA_ERR_UNSUPPORTED, "pair records are implemented for the inverse and exponential flows");
  if (p->fp8) return set_err(FA_ERR_UNSUPPORTED, "pair records need a BF16 or float64 fine dtype");
  if (!scratch || scratch_bytes < records_scratch_bytes(p))
    return set_err(FA_ERR_WORKSPACE, "records scratch of %zu bytes < %zu needed", scratch_bytes,
                   records_scratch_bytes(p));
  FA_TRY(ensure_mstats(p));
  const int n = d.n, N = d.N;
  const size_t nn = p->nn;
  Carver c{static_cast<char *>(scratch)};
  double *R[4];
  for (int j = 0; j < 4; ++j) R[j] = c.take<double>(N * nn);
  double *part = c.take<double>(static_cast<size_t>(N) * fa::stats_blocks(n) * fa::NSTAT);
  const bool inv = d.flow == FA_FLOW_INV;
  const int tl = p->ps.terms_l, tr = p->ps.terms_r;
  if (p->mixed) {
    FA_CUDA(fa::launch_split_terms(U, N, n, p->ldp, inv ? p->Yl[0] : nullptr, inv ? tl : 0,
                                   p->strideY, p->Yr[0], tr, p->strideY, 0, p->stream));
    if (inv) {
      EpiParams e1 = base_epi(p);
      e1.mode = fa::EPI_PROD;
      e1.out_r = p->Pr;
      e1.terms_r = tr;
      e1.term_stride_r = p->strideY;
      FA_TRY(tc(p, p->tmA, p->tmYr[0], tc_params(p, N, 0, 1, e1)));
    }
    for (int j = 0; j < 4; ++j) {
      EpiParams e = base_epi(p);
      e.mode = fa::EPI_TAYLOR;
      e.out64 = R[j];
      const int src = j & 1, dst = (j + 1) & 1;
      if (j < 3) {
        if (inv) {
          e.out_l = p->Yl[dst];
          e.terms_l = tl;
          e.term_stride_l = p->strideY;
        } else {
          e.out_r = p->Yr[dst];
          e.terms_r = tr;
          e.term_stride_r = p->strideY;
        }
      }
      if (inv) FA_TRY(tc(p, p->tmYl[src], p->tmPr, tc_params(p, N, 1, 1, e)));
      else FA_TRY(tc(p, p->tmA, p->tmYr[src], tc_params(p, N, 0, 1, e)));
    }
  } else {
    if (inv) {
      EpiParams e1 = base_epi(p);
      e1.mode = fa::EPI_PROD;
      e1.out64 = p->P64;
      FA_TRY(f64(p, p->B64, 0, U, nn, N, e1));
    }
    for (int j = 0; j < 4; ++j) {
      EpiParams e = base_epi(p);
      e.mode = fa::EPI_TAYLOR;
      e.out64 = R[j];
      const double *src = j == 0 ? U : R[j - 1];
      if (inv) FA_TRY(f64(p, src, nn, p->P64, nn, N, e));
      else FA_TRY(f64(p, p->A64, 0, src, nn, N, e));
    }
  }
  fa::StatsArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.rows_per_block = fa::stats_rows_per_block(n);
  a.X = U;
  a.x_stride = nn;
  a.F = F;
  a.G = G;
  a.f_stride = nn;
  for (int j = 0; j < 4; ++j) a.R[j] = R[j];
  a.r_stride = nn;
  a.nR = 4;
  a.probes = p->probes;
  a.part = part;
  FA_CUDA(fa::launch_stats(a, N, p->stream));
  FA_CUDA(fa::launch_records(part, N, n, N, 0, d.T / N, taylor_scale(p), p->mstats, out,
                             p->stream));
  return FA_OK;
}

fa_status read_err(fa_plan_s *p) {
  int h = 0;
  FA_CUDA(cudaMemcpyAsync(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  FA_CUDA(cudaStreamSynchronize(p->stream));
  if (h == FA_ERR_TIMEOUT) return set_err(FA_ERR_TIMEOUT, "a device-side wait timed out");
  if (h == FA_ERR_NONFINITE) return set_err(FA_ERR_NONFINITE, "non-finite values in the iterates");
  if (h != 0) return set_err(static_cast<fa_status>(h), "device error %d", h);
  return FA_OK;
}

// Square-root refinement: Newton steps X <- X + E with X E + E X = A - X^2.  Per step: X is
// symmetrised, R = A - X^2 in float64, mu = the largest eigenvalue of X (power iteration), and
// the Sylvester equation is solved through sign([[X, R], [0, -X]] / mu) = [[I, 2E], [0, -I]]
// (Roberts 1980) by the Newton-Schulz sign iteration on the blocks,
//     T = 3I - P^2,  Q <- (T Q + Q T - 3Q + P Q P) / 2,  P <- P T / 2,
// from P = X / mu, Q = R / mu, with every product a BF16x6 term product on the tensor cores
// (the products' epilogues write the operand terms of the next products).  The iteration stops
// two steps after ||I - P^2||_F / sqrt(n) < 1e-6.
fa_status refine_sqrt(fa_plan_s *p, double *X) {
  const int n = p->d.n;
  const fa::PairSet ps6 = fa::pair_set(FA_BF16X6);
  double *v = p->pv, *y = v + n, *lam = y + n, *dn = lam + 1, *parts = lam + 8;
  auto prod = [&](const CUtensorMap &L, const CUtensorMap &R, double alpha, double beta,
                  double *out64, __nv_bfloat16 *terms) -> fa_status {
    EpiParams e = base_epi(p);
    e.mode = fa::EPI_STORE;
    e.alpha = alpha;
    e.beta = beta;
    e.store_out = out64;
    if (terms) {
      e.out_l = terms;
      e.terms_l = 3;
      e.term_stride_l = p->strideS;
    }
    TcGemmParams g = fa::tc_launch_params(n, 1, 0, 0, ps6);
    g.epi = e;
    return tc(p, L, R, g);
  };
  auto split = [&](const double *src, __nv_bfloat16 *dst) -> fa_status {
    FA_CUDA(fa::launch_split_terms(src, 1, n, p->ldp, dst, 3, p->strideS, nullptr, 0, 0, 0,
                                   p->stream));
    return FA_OK;
  };
  for (int st = 0; st < p->d.refine_steps; ++st) {
    FA_CUDA(fa::launch_sym_combine(n, 1.0, X, 0.0, nullptr, 0.0, nullptr, p->Xs, p->stream));
    EpiParams e = base_epi(p);
    e.mode = fa::EPI_STORE;
    e.alpha = -1.0;
    e.beta = 0.0;
    e.store_add = p->A64;
    e.store_out = p->Rm;
    FA_TRY(f64(p, p->Xs, 0, p->Xs, 0, 1, e));                       // R = A - X^2
    FA_CUDA(fa::launch_fill(v, n, 1.0 / std::sqrt(static_cast<double>(n)), p->stream));
    for (int it = 0; it < 40; ++it) FA_CUDA(fa::launch_power_step(p->Xs, n, v, y, lam, p->stream));
    double mu = 0.0;
    FA_CUDA(cudaMemcpyAsync(&mu, lam, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    FA_CUDA(cudaStreamSynchronize(p->stream));
    if (!(mu > 0.0) || !std::isfinite(mu))
      return set_err(FA_ERR_NONFINITE, "square-root refinement: no positive spectral scale");
    FA_CUDA(fa::launch_sym_combine(n, 1.0 / mu, p->Xs, 0.0, nullptr, 0.0, nullptr, p->Pm[0],
                                   p->stream));
    FA_TRY(split(p->Pm[0], p->Lp[0]));
    FA_CUDA(fa::launch_sym_combine(n, 1.0 / mu, p->Rm, 0.0, nullptr, 0.0, nullptr, p->Qm,
                                   p->stream));
    FA_TRY(split(p->Qm, p->Lq));
    int cur = 0, extra = -1, k = 0;
    const double stop = 1e-12 * n;                     // ||I - P^2||_F^2 < (1e-6)^2 n
    for (; k < 60; ++k) {
      FA_TRY(prod(p->tmLp[cur], p->tmLp[cur], -1.0, 3.0, p->Tm, p->Lt));          // T
      FA_TRY(prod(p->tmLp[cur], p->tmLt, 0.5, 0.0, p->Pm[cur ^ 1], p->Lp[cur ^ 1]));  // P'
      FA_TRY(prod(p->tmLt, p->tmLq, 1.0, 0.0, p->Wm, nullptr));                   // W = T Q
      FA_TRY(prod(p->tmLp[cur], p->tmLq, 1.0, 0.0, nullptr, p->Lpq));             // P Q
      FA_TRY(prod(p->tmLpq, p->tmLp[cur], 1.0, 0.0, p->Vm, nullptr));             // V = P Q P
      FA_CUDA(fa::launch_sym_combine(n, 1.0, p->Wm, -1.5, p->Qm, 0.5, p->Vm, p->Qm, p->stream));
      FA_TRY(split(p->Qm, p->Lq));
      cur ^= 1;
      FA_CUDA(fa::launch_dev_norm(p->Tm, n, 2.0, parts, dn, p->stream));
      double dev = 0.0;
      FA_CUDA(cudaMemcpyAsync(&dev, dn, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
      FA_CUDA(cudaStreamSynchronize(p->stream));
      if (!std::isfinite(dev))
        return set_err(FA_ERR_NONFINITE, "square-root refinement: sign iteration diverged");
      if (extra < 0 && dev < stop) extra = 2;
      if (extra == 0) break;
      if (extra > 0) --extra;
    }
    p->sign_steps_last = k + 1;
    FA_CUDA(fa::launch_sym_combine(n, 1.0, p->Xs, 0.0, nullptr, 0.5, p->Qm, X, p->stream));
  }
  return FA_OK;
}

fa_status refine(fa_plan_s *p, double *X) {
  const fa_problem_desc &d = p->d;
  if (d.refine_steps <= 0) return FA_OK;
  if (d.flow == FA_FLOW_SQRT) return refine_sqrt(p, X);
  if (d.flow != FA_FLOW_INV)
    return set_err(FA_ERR_UNSUPPORTED, "the exponential flow has no refinement");
  for (int s = 0; s < d.refine_steps; ++s) {
    // T = 2I - A X ; X <- X T  (Newton-Schulz)
    EpiParams e = base_epi(p);
    e.mode = fa::EPI_STORE;
    e.alpha = -1.0;
    e.beta = 2.0;
    e.store_out = p->R1;
    FA_TRY(f64(p, p->A64, 0, X, 0, 1, e));
    e.alpha = 1.0;
    e.beta = 0.0;
    e.store_out = p->R2;
    FA_TRY(f64(p, X, 0, p->R1, 0, 1, e));
    FA_CUDA(cudaMemcpyAsync(X, p->R2, p->nn * sizeof(double), cudaMemcpyDeviceToDevice,
                            p->stream));
  }
  return FA_OK;
}

}  // namespace


// ---- batched solve: many problems of mixed order and flow --------------------------------------

struct fa_batch_s {
  struct Table {
    size_t first = 0;   // index of the first segment in the device array
    int nseg = 0;
    int tiles = 0;
  };
  int count = 0, N = 0, J = 0, max_iters = 0, dtype = 0, max_m = 1;
  double tol = 0.0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  std::vector<fa_plan_s *> plans;
  std::vector<size_t> offs;
  size_t ws_need = 0, seg_off = 0, norm_off = 0, dx_off = 0, err_off = 0, nseg_total = 0;
  char *ws = nullptr;
  fa::TcSegment *d_segs = nullptr;
  fa::BatchNorm *d_norm = nullptr;
  double *d_dx = nullptr;
  int *d_err = nullptr;
  Table fine[5][2];              // [stage 1..4, 4-last][phase: main, inverse second product]
  std::vector<Table> coarse;     // [((mode * N + n) * max_m + sub) * 2 + phase]
  cudaGraphExec_t graph = nullptr;
  bool graph_tried = false;
  // launch schedule of the fine-sweep tables (fa_batch_autotune): per size bucket of n, the
  // epilogue's L2 prefetch and the tile order; per launch, the order of the problems
  static constexpr int kBuckets = 6;     // n <= 64, 128, 256, 512, 1024, larger
  int prefetch_b[kBuckets] = {0, 0, 0, 0, 0, 0}, raster_b[kBuckets] = {0, 0, 0, 0, 0, 0};
  int order = 0;                         // 0: problems as given, 1: largest n first
  std::string tuning;
  // problems still iterating in the current solve (empty = all): a problem that met the
  // tolerance leaves the segment tables, so later launches skip its tiles
  std::vector<char> active;
  bool is_active(int i) const { return active.empty() || active[i]; }
  ~fa_batch_s() {
    for (auto *p : plans) delete p;
    if (graph) cudaGraphExecDestroy(graph);
  }
  size_t coarse_index(int mode, int n, int sub, int phase) const {
    return ((static_cast<size_t>(mode) * N + n) * max_m + sub) * 2 + phase;
  }
};

namespace {

int size_bucket(int n) {
  int k = 0;
  for (int edge = 64; k < fa_batch_s::kBuckets - 1 && n > edge; edge *= 2) ++k;
  return k;
}

// Problem indices in the order of the batch's segment tables.
std::vector<int> problem_order(const fa_batch_s *b) {
  std::vector<int> ord(b->count);
  for (int i = 0; i < b->count; ++i) ord[i] = i;
  if (b->order == 1)
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int x, int y) { return b->plans[x]->d.n > b->plans[y]->d.n; });
  return ord;
}

void push_segment(std::vector<fa::TcSegment> &host, fa_batch_s::Table &t, const fa_plan_s *p,
                  const CUtensorMap &L, const CUtensorMap &R, int nb, int lbat, int rbat,
                  const EpiParams &e, int prefetch = -1, int raster = 0) {
  fa::TcSegment sg;
  memset(&sg, 0, sizeof(sg));
  sg.tmL = L;
  sg.tmR = R;
  sg.epi = e;
  sg.n = p->d.n;
  sg.nb = nb;
  sg.l_batched = lbat;
  sg.r_batched = rbat;
  sg.mt = (p->d.n + TC_BM - 1) / TC_BM;
  sg.nt = (p->d.n + TC_BN - 1) / TC_BN;
  sg.kblocks = (p->d.n + 63) / 64;
  sg.prefetch = prefetch >= 0 ? prefetch : (p->ps.npairs == 1 ? 1 : 0);
  sg.raster = raster;
  sg.tile_begin = t.tiles;
  t.tiles += sg.mt * sg.nt * nb;
  ++t.nseg;
  host.push_back(sg);
}

// Segment tables of every launch of a batch iteration (fixed pointers: the coarse sweep
// overwrites G in place, after the fine sweep has consumed it).
void build_tables(fa_batch_s *b, std::vector<fa::TcSegment> &host) {
  host.clear();
  const int N = b->N, J = b->J;
  const std::vector<int> ord = problem_order(b);
  // fine sweep: config c = stage 1..4 (c = 0..3), or stage 4 of the last step (c = 4)
  for (int c = 0; c < 5; ++c) {
    const int st = c < 4 ? c + 1 : 4;
    const bool last = (c == 4);
    const int cur = (st - 1) & 1;
    for (int phase = 0; phase < 2; ++phase) {
      fa_batch_s::Table &t = b->fine[c][phase];
      t = fa_batch_s::Table();
      t.first = host.size();
      for (int idx : ord) {
        if (!b->is_active(idx)) continue;
        fa_plan_s *p = b->plans[idx];
        const fa_problem_desc &d = p->d;
        const int bk = size_bucket(d.n);
        const int pf = b->prefetch_b[bk], rs = b->raster_b[bk];
        const double h = d.T / static_cast<double>(N) / static_cast<double>(J);
        EpiParams e = base_epi(p);
        e.mode = fa::EPI_STAGE;
        e.stage = st;
        e.last = last ? 1 : 0;
        e.h = h;
        e.ch = (st == 3) ? h : (st < 3 ? 0.5 * h : 0.0);
        e.f_out = p->D;
        e.g_old = p->Gold;
        e.x_hi = p->x_hi;
        e.x_lo = p->x_lo;
        e.acc = p->acc;
        e.a_hi = p->a_hi;
        e.a_lo = p->a_lo;
        e.out_r = p->Yr[cur ^ 1];
        e.out_l = p->Yl[cur ^ 1];
        e.terms_r = p->ps.terms_r;
        e.terms_l = p->needs_l() ? p->ps.terms_l : 0;
        e.term_stride_r = e.term_stride_l = p->strideY;
        e.err = b->d_err;
        if (phase == 0) {
          if (d.flow == FA_FLOW_EXP) {
            push_segment(host, t, p, p->tmA, p->tmYr[cur], N, 0, 1, e, pf, rs);
          } else if (d.flow == FA_FLOW_SQRT) {
            push_segment(host, t, p, p->tmYl[cur], p->tmYr[cur], N, 1, 1, e, pf, rs);
          } else {
            EpiParams e1 = base_epi(p);
            e1.mode = fa::EPI_PROD;
            e1.out_r = p->Pr;
            e1.terms_r = p->ps.terms_r;
            e1.term_stride_r = p->strideY;
            e1.err = b->d_err;
            push_segment(host, t, p, p->tmA, p->tmYr[cur], N, 0, 1, e1, pf, rs);
          }
        } else if (d.flow == FA_FLOW_INV) {
          push_segment(host, t, p, p->tmYl[cur], p->tmPr, N, 1, 1, e, pf, rs);
        }
      }
    }
  }
  // coarse sweep: mode 0 = Step 0, mode 1 = correction with norms
  b->coarse.assign(static_cast<size_t>(2) * N * b->max_m * 2, fa_batch_s::Table());
  for (int mode = 0; mode < 2; ++mode)
    for (int n = 0; n < N; ++n)
      for (int sub = 0; sub < b->max_m; ++sub)
        for (int phase = 0; phase < 2; ++phase) {
          fa_batch_s::Table &t = b->coarse[b->coarse_index(mode, n, sub, phase)];
          t.first = host.size();
          for (int idx : ord) {
            if (!b->is_active(idx)) continue;
            fa_plan_s *p = b->plans[idx];
            const fa_problem_desc &d = p->d;
            const int m = d.coarse_steps;
            if (sub >= m) continue;
            if (phase == 0 && d.flow != FA_FLOW_INV) continue;
            const size_t nn = p->nn;
            const int tglob = n * m + sub;
            const int cur = tglob & 1;
            const bool lastsub = (sub == m - 1);
            if (phase == 0) {
              EpiParams e1 = base_epi(p);
              e1.mode = fa::EPI_PROD;
              e1.out_r = p->Pcr;
              e1.terms_r = p->ps.terms_r;
              e1.term_stride_r = p->strideV;
              e1.err = b->d_err;
              push_segment(host, t, p, p->tmA, p->tmVr[cur], 1, 0, 0, e1);
              continue;
            }
            EpiParams e = base_epi(p);
            e.mode = fa::EPI_EULER;
            e.dt = d.T / static_cast<double>(N) / static_cast<double>(m);
            e.v_in = (sub == 0) ? p->U + static_cast<size_t>(n) * nn : p->Vtmp[(sub - 1) & 1];
            e.v_out = lastsub ? p->U + static_cast<size_t>(n + 1) * nn : p->Vtmp[sub & 1];
            e.euler_last = lastsub ? 1 : 0;
            if (lastsub) {
              e.g_out = p->Gold + static_cast<size_t>(n) * nn;
              e.d_in = mode ? p->D + static_cast<size_t>(n) * nn : nullptr;
              e.u_old = mode ? p->U + static_cast<size_t>(n + 1) * nn : nullptr;
              e.norm_part = p->part + static_cast<size_t>(n) * p->part_tiles * 2;
            }
            e.a_hi = p->a_hi;
            e.a_lo = p->a_lo;
            e.out_r = p->Vr[cur ^ 1];
            e.out_l = p->Vl[cur ^ 1];
            e.terms_r = p->ps.terms_r;
            e.terms_l = p->needs_l() ? p->ps.terms_l : 0;
            e.term_stride_r = e.term_stride_l = p->strideV;
            e.err = b->d_err;
            // the same launches as the single-problem sweep (euler_gemm), transposed alike
            const bool tp = transposable(p);
            e.transposed = tp ? 1 : 0;
            if (tp && d.flow == FA_FLOW_SQRT) e.a64 = p->A64;
            if (d.flow == FA_FLOW_EXP && tp)
              push_segment(host, t, p, p->tmVr[cur], p->tmA, 1, 0, 0, e);
            else if (d.flow == FA_FLOW_EXP)
              push_segment(host, t, p, p->tmA, p->tmVr[cur], 1, 0, 0, e);
            else if (d.flow == FA_FLOW_SQRT && tp)
              push_segment(host, t, p, p->tmVr[cur], p->tmVl[cur], 1, 0, 0, e);
            else if (d.flow == FA_FLOW_SQRT)
              push_segment(host, t, p, p->tmVl[cur], p->tmVr[cur], 1, 0, 0, e);
            else if (tp)
              push_segment(host, t, p, p->tmPcr, p->tmVl[cur], 1, 0, 0, e);
            else
              push_segment(host, t, p, p->tmVl[cur], p->tmPcr, 1, 0, 0, e);
          }
        }
}

// Segment tables to the device (after any change of the schedule); the captured iteration
// graph refers to the old tables' contents only through the device array, but is rebuilt anyway.
fa_status upload_tables(fa_batch_s *b) {
  std::vector<fa::TcSegment> host;
  host.reserve(b->nseg_total);
  build_tables(b, host);
  if (host.size() > b->nseg_total) return set_err(FA_ERR_WORKSPACE, "segment table overflow");
  FA_CUDA(cudaMemcpyAsync(b->d_segs, host.data(), host.size() * sizeof(fa::TcSegment),
                          cudaMemcpyHostToDevice, b->stream));
  FA_CUDA(cudaStreamSynchronize(b->stream));
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->graph_tried = false;
  return FA_OK;
}

// Every problem back in the segment tables (the start of a solve, and the autotuner).
fa_status activate_all(fa_batch_s *b) {
  if (b->active.empty()) return FA_OK;
  b->active.clear();
  return upload_tables(b);
}

fa_status launch_table(fa_batch_s *b, const fa_batch_s::Table &t) {
  if (t.nseg == 0) return FA_OK;
  TcGemmParams g = fa::tc_launch_params(128, 1, 0, 0, b->plans[0]->ps);
  g.epi.err = b->d_err;
  FA_CUDA(fa::launch_tc_gemm_ragged(b->d_segs + t.first, t.nseg, t.tiles, g, b->num_sms,
                                    b->stream));
  return FA_OK;
}

fa_status batch_coarse(fa_batch_s *b, int mode) {
  for (int i = 0; i < b->count; ++i) {
    if (!b->is_active(i)) continue;
    fa_plan_s *p = b->plans[i];
    FA_CUDA(fa::launch_split_terms(p->U, 1, p->d.n, p->ldp, p->Vl[0],
                                   p->needs_l() ? p->ps.terms_l : 0, p->strideV, p->Vr[0],
                                   p->ps.terms_r, p->strideV, fa::SPLIT_FROM_F32, b->stream));
  }
  for (int n = 0; n < b->N; ++n)
    for (int sub = 0; sub < b->max_m; ++sub)
      for (int phase = 0; phase < 2; ++phase)
        FA_TRY(launch_table(b, b->coarse[b->coarse_index(mode, n, sub, phase)]));
  return FA_OK;
}

fa_status batch_iteration(fa_batch_s *b) {
  for (int i = 0; i < b->count; ++i) {
    if (!b->is_active(i)) continue;
    fa_plan_s *p = b->plans[i];
    FA_CUDA(fa::launch_load_state(p->U, b->N, p->d.n, p->ldp, p->x_hi, p->x_lo, p->Yl[0],
                                  p->needs_l() ? p->ps.terms_l : 0, p->strideY, p->Yr[0],
                                  p->ps.terms_r, p->strideY, b->stream));
  }
  for (int j = 0; j < b->J; ++j)
    for (int st = 1; st <= 4; ++st) {
      const int c = (st == 4 && j == b->J - 1) ? 4 : st - 1;
      FA_TRY(launch_table(b, b->fine[c][0]));
      FA_TRY(launch_table(b, b->fine[c][1]));
    }
  FA_TRY(batch_coarse(b, 1));
  FA_CUDA(fa::launch_batch_norms(b->d_norm, b->count, b->N, b->d_dx, b->d_err, b->stream));
  return FA_OK;
}

// ---- modified parareal (Algorithm 3) ---------------------------------------------------------

// Sum of kKrylovBlocks partials read back to the host (fixed order).
double host_sum(const double *h) {
  double s = 0.0;
  for (int b = 0; b < fa::kKrylovBlocks; ++b) s += h[b];
  return s;
}

// globalQR step (Algorithm 2) for one block z against the basis Q_0 .. Q_{d-1}: two modified
// Gram-Schmidt sweeps on a copy q, then r = ||q||_F; the block joins the basis as q / r when
// r > drop ||z||_F and the space has room.  ||q|| is also read after the first sweep: the second
// sweep removes only what rounding left along the basis and cannot lengthen q, so a block that
// is already below the threshold is removed without it (the decision the full two sweeps would
// take).  Returns through *kept.
fa_status gs_extend(fa_plan_s *p, const double *z, int *d, bool *kept) {
  const size_t nn = p->nn;
  const int dd = *d;
  *kept = false;
  if (dd >= p->cap) return FA_OK;                 // no room: the block is left to G
  double *q = p->Xout;
  double *pz = p->kpart, *pa = p->kpart + fa::kKrylovBlocks, *pb = pa + fa::kKrylovBlocks;
  FA_CUDA(cudaMemcpyAsync(q, z, nn * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  FA_CUDA(fa::launch_gs_step(q, nullptr, nullptr, nullptr, nn, pz, p->stream));   // ||z||^2
  double hz[fa::kKrylovBlocks], hr[fa::kKrylovBlocks];
  double zn = 0.0, r = 0.0;
  double *pin = pa, *pout = pb;
  auto read_norms = [&](const double *pr) -> fa_status {
    FA_CUDA(cudaMemcpyAsync(hz, pz, sizeof(hz), cudaMemcpyDeviceToHost, p->stream));
    FA_CUDA(cudaMemcpyAsync(hr, pr, sizeof(hr), cudaMemcpyDeviceToHost, p->stream));
    FA_CUDA(cudaStreamSynchronize(p->stream));
    zn = std::sqrt(host_sum(hz));
    r = std::sqrt(host_sum(hr));
    if (!std::isfinite(zn) || !std::isfinite(r))
      return set_err(FA_ERR_NONFINITE, "non-finite block in the parareal space");
    return FA_OK;
  };
  if (dd == 0) {
    FA_TRY(read_norms(pz));                       // the reduced block is z itself
  } else {
    for (int pass = 0; pass < 2; ++pass) {
      const double *prev = nullptr;
      for (int j = 0; j < dd; ++j) {
        const double *next = p->Qb + static_cast<size_t>(j) * nn;
        FA_CUDA(fa::launch_gs_step(q, prev, pin, next, nn, pout, p->stream));
        prev = next;
        std::swap(pin, pout);
      }
      FA_CUDA(fa::launch_gs_step(q, prev, pin, nullptr, nn, pout, p->stream));     // ||q||^2
      std::swap(pin, pout);
      FA_TRY(read_norms(pin));
      if (!(r > p->drop * zn && r > 0.0)) return FA_OK;   // removed
    }
  }
  *kept = r > p->drop * zn && r > 0.0;
  if (*kept) {
    FA_CUDA(fa::launch_scale_copy(q, 1.0 / r, nn, p->Qb + static_cast<size_t>(dd) * nn, p->stream));
    *d = dd + 1;
  }
  return FA_OK;
}

// Sequential update of Algorithm 3 (eq. eq_update): for n = 0..N-1,
//   alpha = Q^T <> U_n,  R = U_n - sum alpha_i Q_i,  W = sum alpha_i F(Q_i),
//   U_{n+1} = G(R) + W (forward-Euler substeps on R, W added on the last one),
// in place on p->U with the convergence norms against the previous iterate.
fa_status modified_update(fa_plan_s *p, int d) {
  const fa_problem_desc &d_ = p->d;
  const int N = d_.N, m = d_.coarse_steps;
  const size_t nn = p->nn;
  const double dt = d_.T / static_cast<double>(N) / static_cast<double>(m);
  const int tl = p->ps.terms_l, tr = p->ps.terms_r;
  double *R = p->R1, *W = p->R2;
  const int tiles = p->part_tiles;
  for (int s = 0; s < N; ++s) {
    const double *V = p->U + static_cast<size_t>(s) * nn;
    FA_CUDA(fa::launch_project_alpha(V, p->Qb, nn, d, p->apart, p->alpha, p->stream));
    FA_CUDA(fa::launch_project_combine(V, p->Qb, p->FQb, p->alpha, d, nn, R, W, p->stream));
    int cur = 0;
    if (p->cmixed) FA_TRY(split_coarse(p, R, 0));
    for (int sub = 0; sub < m; ++sub) {
      const bool last = (sub == m - 1);
      const double *vin = (sub == 0) ? R : p->Vtmp[(sub - 1) & 1];
      double *vout = last ? p->U + static_cast<size_t>(s + 1) * nn : p->Vtmp[sub & 1];
      EpiParams e = base_epi(p);
      e.mode = fa::EPI_EULER;
      e.dt = dt;
      e.v_in = vin;
      e.v_out = vout;
      e.euler_last = last ? 1 : 0;
      if (last) {
        e.g_out = p->Gnew + static_cast<size_t>(s) * nn;   // G(R): not needed later
        e.d_in = W;
        e.u_old = p->U + static_cast<size_t>(s + 1) * nn;
        e.norm_part = p->part + static_cast<size_t>(s) * tiles * 2;
      }
      if (p->cmixed) {
        e.out_r = p->Vr[cur ^ 1];
        e.out_l = p->Vl[cur ^ 1];
        e.terms_r = tr;
        e.terms_l = p->needs_l() ? tl : 0;
        e.term_stride_r = e.term_stride_l = p->strideV;
      }
      FA_TRY(euler_gemm(p, cur, vin, e));
      if (p->cmixed) cur ^= 1;
    }
  }
  FA_CUDA(fa::launch_reduce_norms(p->part, N, tiles, p->norms, p->stream));
  FA_CUDA(fa::launch_max_ratio(p->norms, N, p->dx, p->err, p->stream));
  return FA_OK;
}

// The whole modified solve (matrix already set): Step 0, then per iteration the space's
// enlargement, F on the new blocks, and the sequential update.
fa_status modified_solve(fa_plan_s *p, const double *dX0, double *dXout, fa_report *r) {
  const fa_problem_desc &d = p->d;
  const size_t nn = p->nn;
  cudaEvent_t ev[4];
  for (auto &e : ev) FA_CUDA(cudaEventCreate(&e));
  struct EvGuard {
    cudaEvent_t *e;
    ~EvGuard() {
      for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
    }
  } guard{ev};
  FA_CUDA(cudaEventRecord(ev[0], p->stream));
  if (dX0) {
    FA_CUDA(cudaMemcpyAsync(p->U, dX0, nn * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  } else {
    FA_CUDA(fa::launch_identity(p->U, d.n, p->stream));
  }
  // Step 0 (eq. eqStep0): the coarse sweep
  FA_TRY(coarse_sweep(p, p->U, nullptr, p->U, p->Gold, nullptr, nullptr));
  FA_CUDA(cudaEventRecord(ev[1], p->stream));
  FA_CUDA(cudaEventSynchronize(ev[1]));
  float ms = 0.f;
  FA_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
  double t_init = ms, t_fine = 0.0, t_coarse = 0.0;
  int basis = 0, iters = 0, fine_blocks = 0;
  bool converged = false;
  double dx = INFINITY;
  for (int k = 0; k < d.max_iters; ++k) {
    // S^k = Span(S^{k-1}, U^k_0 .. U^k_N): globalQR of [Q, U_0, ..., U_N] (the old basis is
    // kept and completed)
    FA_CUDA(cudaEventRecord(ev[1], p->stream));
    const int d0 = basis;
    for (int s = 0; s <= d.N && basis < p->cap; ++s) {
      bool kept = false;
      FA_TRY(gs_extend(p, p->U + static_cast<size_t>(s) * nn, &basis, &kept));
    }
    // F on the new blocks only, all at once (in chunks of the fine state's N slices)
    for (int c = d0; c < basis; c += d.N) {
      const int cnt = basis - c < d.N ? basis - c : d.N;
      FA_TRY(fine_sweep(p, p->Qb + static_cast<size_t>(c) * nn, p->FQb + static_cast<size_t>(c) * nn,
                        nullptr, cnt));
    }
    fine_blocks += basis - d0;
    FA_CUDA(cudaEventRecord(ev[2], p->stream));
    FA_TRY(modified_update(p, basis));
    FA_CUDA(cudaEventRecord(ev[3], p->stream));
    FA_CUDA(cudaMemcpyAsync(&dx, p->dx, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    FA_CUDA(cudaStreamSynchronize(p->stream));
    FA_CUDA(cudaEventElapsedTime(&ms, ev[1], ev[2]));
    t_fine += ms;
    FA_CUDA(cudaEventElapsedTime(&ms, ev[2], ev[3]));
    t_coarse += ms;
    ++iters;
    if (r && r->dx_history) r->dx_history[k] = dx;
    if (!std::isfinite(dx)) break;
    if (dx < d.tol) {
      converged = true;
      break;
    }
  }
  FA_CUDA(cudaMemcpyAsync(dXout, p->U + static_cast<size_t>(d.N) * nn, nn * sizeof(double),
                          cudaMemcpyDeviceToDevice, p->stream));
  const fa_status es = read_err(p);
  if (r) {
    r->iters = iters;
    r->converged = converged ? 1 : 0;
    r->last_dx = dx;
    r->t_init_ms = t_init;
    r->t_fine_ms = t_fine;
    r->t_coarse_ms = t_coarse;
    r->t_refine_ms = 0.0;
    r->g_fallback_iter = 0;
    r->coef_fallbacks = 0;
    r->records = 0;
    r->basis_dim = basis;
    r->fine_blocks = fine_blocks;
  }
  if (es != FA_OK) return es;
  if (!std::isfinite(dx))
    return set_err(FA_ERR_NONFINITE, "non-finite convergence measure at iteration %d", iters);
  if (!converged && d.tol > 0.0)
    return set_err(FA_ERR_NOT_CONVERGED, "tolerance %.3g not reached in %d iterations (dx %.3g)",
                   d.tol, iters, dx);
  return FA_OK;
}

}  // namespace

// ---- C ABI -----------------------------------------------------------------------------------

extern "C" {

fa_status cos_plan(fa_plan_t *out, const fa_problem_desc *d, void *stream, size_t *ws_bytes);

fa_status fa_plan(fa_plan_t *out, const fa_problem_desc *d, void *stream, size_t *ws_bytes) {
  if (!out || !d || !ws_bytes) return set_err(FA_ERR_ARG, "null argument");
  *out = nullptr;
  if (d->flow == FA_FLOW_COS) return cos_plan(out, d, stream, ws_bytes);
  if (d->n < 1 || d->n > 16384) return set_err(FA_ERR_ARG, "n = %d out of range [1, 16384]", d->n);
  if (d->N < 1) return set_err(FA_ERR_ARG, "N = %d must be >= 1", d->N);
  if (d->fine_steps < 1) return set_err(FA_ERR_ARG, "fine_steps = %d must be >= 1", d->fine_steps);
  if (d->coarse_steps < 1)
    return set_err(FA_ERR_ARG, "coarse_steps = %d must be >= 1", d->coarse_steps);
  if (!(d->T > 0.0) || !std::isfinite(d->T)) return set_err(FA_ERR_ARG, "T must be finite and > 0");
  if (d->max_iters < 0) return set_err(FA_ERR_ARG, "max_iters must be >= 0");
  if (!(d->tol >= 0.0)) return set_err(FA_ERR_ARG, "tol must be >= 0");
  if (d->flow < FA_FLOW_INV || d->flow > FA_FLOW_SQRT)
    return set_err(FA_ERR_ARG, "unknown flow %d", d->flow);
  if (d->fine_dtype < FA_F64 || d->fine_dtype > FA_FP8E4M3)
    return set_err(FA_ERR_ARG, "unknown fine dtype %d", d->fine_dtype);
  if (d->fine_dtype == FA_FP8E4M3) {
    if (d->coarse_dtype < FA_F64 || d->coarse_dtype > FA_BF16X6)
      return set_err(FA_ERR_ARG, "with FA_FP8E4M3 F the coarse dtype is FA_F64 or a BF16 form");
  } else if (d->coarse_dtype != FA_F64 && d->coarse_dtype != d->fine_dtype) {
    return set_err(FA_ERR_ARG, "coarse dtype must be FA_F64 or the fine dtype");
  }
  if (d->refine_steps < 0) return set_err(FA_ERR_ARG, "refine_steps must be >= 0");
  if (d->coarse_kind != FA_COARSE_EULER && d->coarse_kind != FA_COARSE_LEARNED)
    return set_err(FA_ERR_ARG, "unknown coarse kind %d", d->coarse_kind);
  if (d->fine_dtype == FA_FP8E4M3 && d->flow != FA_FLOW_SQRT)
    return set_err(FA_ERR_UNSUPPORTED, "FA_FP8E4M3 operands are implemented for the square-root flow");
  if (d->method != FA_METHOD_CLASSICAL && d->method != FA_METHOD_MODIFIED)
    return set_err(FA_ERR_ARG, "unknown method %d", d->method);
  if (d->method == FA_METHOD_MODIFIED) {
    if (d->flow != FA_FLOW_EXP)
      return set_err(FA_ERR_UNSUPPORTED,
                     "the modified parareal is for linear homogeneous flows (the exponential flow)");
    if (d->coarse_kind != FA_COARSE_EULER)
      return set_err(FA_ERR_UNSUPPORTED, "the modified parareal uses the forward-Euler G");
    if (d->max_basis < 0 || d->max_basis > 4096)
      return set_err(FA_ERR_ARG, "max_basis = %d out of range [0, 4096]", d->max_basis);
    if (!(d->span_drop >= 0.0) || !std::isfinite(d->span_drop))
      return set_err(FA_ERR_ARG, "span_drop must be finite and >= 0");
  }
  if (d->fine_scheme < FA_SCHEME_DEFAULT || d->fine_scheme > FA_SCHEME_CN)
    return set_err(FA_ERR_ARG, "unknown fine scheme %d", d->fine_scheme);
  if (d->coarse_scheme != FA_SCHEME_DEFAULT && d->coarse_scheme != FA_SCHEME_EULER &&
      d->coarse_scheme != FA_SCHEME_CN)
    return set_err(d->coarse_scheme == FA_SCHEME_RK4 ? FA_ERR_UNSUPPORTED : FA_ERR_ARG,
                   "coarse scheme %d: G is forward Euler or Crank-Nicolson", d->coarse_scheme);
  if ((d->fine_scheme == FA_SCHEME_CN || d->coarse_scheme == FA_SCHEME_CN) &&
      d->flow != FA_FLOW_EXP)
    return set_err(FA_ERR_UNSUPPORTED, "Crank-Nicolson propagators are for the exponential flow");
  if ((d->fine_scheme > FA_SCHEME_RK4 || d->coarse_scheme == FA_SCHEME_CN) &&
      (d->fine_dtype == FA_FP8E4M3 || d->coarse_kind != FA_COARSE_EULER))
    return set_err(FA_ERR_UNSUPPORTED,
                   "explicit-Euler and Crank-Nicolson schemes need BF16 or float64 products and "
                   "the Euler coarse kind");
  if (d->coarse_kind == FA_COARSE_LEARNED) {
    if (d->flow == FA_FLOW_SQRT)
      return set_err(FA_ERR_UNSUPPORTED,
                     "the learned coarse propagator supports the inverse and exponential flows");
    if (d->coarse_steps != 1)
      return set_err(FA_ERR_ARG, "the learned coarse propagator takes one step per slice");
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return set_err(FA_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
  cudaDeviceProp prop;
  ce = cudaGetDeviceProperties(&prop, dev);
  if (ce != cudaSuccess)
    return set_err(FA_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(ce));
  if (prop.major != 10 || prop.minor != 3)
    return set_err(FA_ERR_UNSUPPORTED, "device %s is sm_%d%d; this library is built for sm_103a",
                   prop.name, prop.major, prop.minor);
  fa_plan_s *p = new (std::nothrow) fa_plan_s();
  if (!p) return set_err(FA_ERR_ARG, "out of host memory");
  p->d = *d;
  p->stream = static_cast<cudaStream_t>(stream);
  p->device = dev;
  p->num_sms = prop.multiProcessorCount;
  p->fp8 = d->fine_dtype == FA_FP8E4M3;
  p->mixed = is_mixed(d->fine_dtype) || p->fp8;
  p->cmixed = is_mixed(d->coarse_dtype);
  p->ps = fa::pair_set(p->fp8 ? (p->cmixed ? d->coarse_dtype : FA_BF16)
                              : (p->mixed ? d->fine_dtype : d->coarse_dtype));
  p->ldp8 = (d->n + 15) / 16 * 16;
  p->qT = (d->n + 127) / 128;
  p->ldp = (d->n + 7) / 8 * 8;
  p->nn = static_cast<size_t>(d->n) * d->n;
  p->learned = d->coarse_kind == FA_COARSE_LEARNED;
  p->learned_active = p->learned;
  p->fsch = d->fine_scheme == FA_SCHEME_DEFAULT ? FA_SCHEME_RK4 : d->fine_scheme;
  p->csch = d->coarse_scheme == FA_SCHEME_DEFAULT ? FA_SCHEME_EULER : d->coarse_scheme;
  p->modified = d->method == FA_METHOD_MODIFIED;
  if (p->modified) {
    // default: three iterations' worth of new blocks (the linear flows here need two or three)
    const long long k = d->max_iters < 1 ? 1 : (d->max_iters < 3 ? d->max_iters : 3);
    const long long def = (static_cast<long long>(d->N) + 1) * k;
    p->cap = d->max_basis > 0 ? d->max_basis : static_cast<int>(def < 4096 ? def : 4096);
    p->drop = d->span_drop > 0.0 ? d->span_drop : (p->mixed ? 1e-7 : 1e-12);
  }
  p->part_tiles = p->cmixed ? ((d->n + TC_BM - 1) / TC_BM) * ((d->n + TC_BN - 1) / TC_BN)
                            : fa::f64_tiles_per_slice(d->n, 1);
  p->ws_need = carve(p, nullptr);
  *ws_bytes = p->ws_need;
  *out = p;
  return FA_OK;
}

// FA_FLOW_COS plans: an inner exponential-flow plan of order 2n for eq. eqB's block flow.
fa_status cos_plan(fa_plan_t *out, const fa_problem_desc *d, void *stream, size_t *ws_bytes) {
  if (d->n < 1 || d->n > 8192) return set_err(FA_ERR_ARG, "n = %d out of range [1, 8192]", d->n);
  if (d->T != 1.0) return set_err(FA_ERR_ARG, "FA_FLOW_COS integrates over [0, 1]: T must be 1");
  if (d->fine_scheme == FA_SCHEME_CN || d->coarse_scheme == FA_SCHEME_CN)
    return set_err(FA_ERR_UNSUPPORTED, "FA_FLOW_COS uses RK4 or explicit-Euler propagators");
  if (d->refine_steps != 0) return set_err(FA_ERR_UNSUPPORTED, "FA_FLOW_COS has no refinement");
  fa_problem_desc d2 = *d;
  d2.n = 2 * d->n;
  d2.flow = FA_FLOW_EXP;
  fa_plan_t inner = nullptr;
  size_t iws = 0;
  FA_TRY(fa_plan(&inner, &d2, stream, &iws));
  fa_plan_s *p = new (std::nothrow) fa_plan_s();
  if (!p) {
    delete inner;
    return set_err(FA_ERR_ARG, "out of host memory");
  }
  p->d = *d;
  p->stream = static_cast<cudaStream_t>(stream);
  p->device = inner->device;
  p->num_sms = inner->num_sms;
  p->nn = static_cast<size_t>(d->n) * d->n;
  p->inner = inner;
  p->inner_ws = (iws + 255) / 256 * 256;
  p->ws_need = carve(p, nullptr);
  *ws_bytes = p->ws_need;
  *out = p;
  return FA_OK;
}

// cos(A) by Algorithm 5 on an FA_FLOW_COS plan.
fa_status cos_solve(fa_plan_s *p, const double *dA, double *dXout, fa_report *r) {
  const int n = p->d.n;
  FA_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), p->stream));
  FA_CUDA(fa::launch_check_finite(dA, p->nn, p->err, p->stream));
  // step 1: the smallest m >= 0 with 2^-m ||A||_inf <= 1
  FA_CUDA(fa::launch_inf_norm(dA, n, p->scal, p->stream));
  double a = 0.0;
  FA_CUDA(cudaMemcpyAsync(&a, p->scal, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  FA_CUDA(cudaStreamSynchronize(p->stream));
  if (!std::isfinite(a)) return set_err(FA_ERR_NONFINITE, "non-finite entries in A");
  int m = 0;
  double scale = 1.0;
  while (a > 1.0) {
    a *= 0.5;
    scale *= 0.5;
    ++m;
  }
  // steps 2-3: eq. eqB's block flow for A0 = 2^-m A from (0; I), by the inner plan
  FA_CUDA(fa::launch_cos_block(dA, n, scale, p->Bm, p->X0b, p->stream));
  const fa_status st = fa_parareal_solve(p->inner, p->Bm, p->X0b, p->Ub, r);
  if (st != FA_OK && st != FA_ERR_NOT_CONVERGED) return st;
  // C_0 = cos(A0): the lower-right block; step 4: C <- 2 C^2 - I, m times (float64)
  FA_CUDA(fa::launch_extract_block(p->Ub, n, n, n, p->Cw[0], p->stream));
  int cur = 0;
  for (int i = 0; i < m; ++i) {
    F64GemmParams g;
    memset(&g, 0, sizeof(g));
    g.n = n;
    g.nb = 1;
    g.L = p->Cw[cur];
    g.R = p->Cw[cur];
    g.epi.mode = fa::EPI_STORE;
    g.epi.n = n;
    g.epi.alpha = 2.0;
    g.epi.beta = -1.0;
    g.epi.store_out = p->Cw[cur ^ 1];
    g.epi.err = p->err;
    FA_CUDA(fa::launch_f64_gemm(g, p->stream));
    cur ^= 1;
  }
  FA_CUDA(cudaMemcpyAsync(dXout, p->Cw[cur], p->nn * sizeof(double), cudaMemcpyDeviceToDevice,
                          p->stream));
  if (r) r->double_angle_steps = m;
  const fa_status es = read_err(p);
  if (es != FA_OK) return es;
  return st;
}

fa_status fa_aima_plan(fa_plan_t *out, int n, int dtype, void *stream, size_t *ws_bytes) {
  if (!out || !ws_bytes) return set_err(FA_ERR_ARG, "null argument");
  if (dtype != FA_F64 && !is_mixed(dtype))
    return set_err(FA_ERR_ARG, "dtype must be FA_F64 or a BF16 form");
  // the machinery of a two-slice exponential-flow plan: the shared left factor A, the right
  // factor [X | u] (slices 0 and 1)
  fa_problem_desc d{};
  d.n = n;
  d.flow = FA_FLOW_EXP;
  d.T = 1.0;
  d.N = 2;
  d.coarse_steps = 1;
  d.fine_steps = 1;
  d.max_iters = 0;
  d.fine_dtype = dtype;
  d.coarse_dtype = dtype;
  FA_TRY(fa_plan(out, &d, stream, ws_bytes));
  fa_plan_s *p = *out;
  p->aima = true;
  if (!p->mixed) {
    // residual partials per tile of slice 0 in the two-slice float64 launch
    p->part_tiles = fa::f64_tiles_per_slice(n, 2);
    p->ws_need = carve(p, nullptr);
    *ws_bytes = p->ws_need;
  }
  return FA_OK;
}

fa_status fa_aima(fa_plan_t p, const double *dA, const double *dX0, const double *dE, double dt,
                  int steps, double *dXout, double *h_res) {
  FA_TRY(check_ready(p, false));
  if (!p->aima) return set_err(FA_ERR_ARG, "the plan was not made by fa_aima_plan");
  if (!dA || !dX0 || !dE || !dXout) return set_err(FA_ERR_ARG, "null pointer");
  const int n = p->d.n;
  const size_t nn = p->nn;
  if (steps < 0 || static_cast<size_t>(steps) + 1 > nn)
    return set_err(FA_ERR_ARG, "steps = %d out of range [0, n^2 - 1]", steps);
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(FA_ERR_ARG, "dt must be finite and > 0");
  FA_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), p->stream));
  FA_TRY(fa_plan_set_matrix(p, dA));
  // state [X | u] (float64 [2][n][n]) double-buffered in Gold / Gnew; residuals in D
  double *S[2] = {p->Gold, p->Gnew};
  double *res = p->D;
  FA_CUDA(cudaMemcpyAsync(S[0], dX0, nn * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  FA_CUDA(cudaMemcpyAsync(S[0] + nn, dE, nn * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  const int tr = p->ps.terms_r;
  if (p->mixed)
    FA_CUDA(fa::launch_split_terms(S[0], 2, n, p->ldp, nullptr, 0, 0, p->Yr[0], tr, p->strideY,
                                   fa::SPLIT_FROM_F32, p->stream));
  int cur = 0;
  for (int k = 0; k <= steps; ++k) {
    EpiParams e = base_epi(p);
    e.mode = fa::EPI_AIMA;
    e.last = (k == steps) ? 1 : 0;   // the final launch forms the residual only
    e.dt = dt;
    e.x64 = S[cur];
    e.out64 = S[cur ^ 1];
    e.norm_part = p->part;
    if (p->mixed) {
      e.out_r = p->Yr[cur ^ 1];
      e.terms_r = tr;
      e.term_stride_r = p->strideY;
      if (transposable(p)) {
        // (A Y)^T = Y^T A^T: coalesced float64 state accesses in the epilogue
        e.transposed = 1;
        FA_TRY(tc(p, p->tmYr[cur], p->tmA, tc_params(p, 2, 1, 0, e)));
      } else {
        FA_TRY(tc(p, p->tmA, p->tmYr[cur], tc_params(p, 2, 0, 1, e)));
      }
    } else {
      FA_TRY(f64(p, p->A64, 0, S[cur], nn, 2, e));
    }
    FA_CUDA(fa::launch_reduce_norms(p->part, 1, p->part_tiles, res + 2 * static_cast<size_t>(k),
                                    p->stream));
    if (k < steps) cur ^= 1;
  }
  FA_CUDA(cudaMemcpyAsync(dXout, S[cur], nn * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  if (h_res) {
    std::vector<double> r2(2 * (static_cast<size_t>(steps) + 1));
    FA_CUDA(cudaMemcpyAsync(r2.data(), res, r2.size() * sizeof(double), cudaMemcpyDeviceToHost,
                            p->stream));
    FA_CUDA(cudaStreamSynchronize(p->stream));
    for (int k = 0; k <= steps; ++k) h_res[k] = std::sqrt(r2[2 * static_cast<size_t>(k)]);
  }
  return read_err(p);
}

fa_status fa_plan_bind_workspace(fa_plan_t p, void *ws, size_t bytes) {
  if (!p) return set_err(FA_ERR_ARG, "null plan");
  if (!ws) return set_err(FA_ERR_WORKSPACE, "null workspace");
  if (bytes < p->ws_need)
    return set_err(FA_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", bytes, p->ws_need);
  if (reinterpret_cast<uintptr_t>(ws) & 255)
    return set_err(FA_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  // the plan's device current on this thread (tensor maps are encoded through the driver API,
  // which needs a current context; a thread that made no runtime call yet has none)
  FA_CUDA(cudaSetDevice(p->device));
  if (p->inner) {
    FA_TRY(fa_plan_bind_workspace(p->inner, ws, p->inner->ws_need));
    p->ws = static_cast<char *>(ws);
    carve(p, p->ws);
    return FA_OK;
  }
  p->ws = static_cast<char *>(ws);
  carve(p, p->ws);
  p->matrix_set = false;
  p->mstats_valid = false;
  p->params_set = false;
  FA_TRY(encode_all(p));
  FA_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), p->stream));
  FA_CUDA(cudaMemsetAsync(p->fallbacks, 0, sizeof(int), p->stream));
  FA_CUDA(fa::launch_probes(p->d.n, p->probes, p->stream));
  return FA_OK;
}

fa_status fa_plan_set_matrix(fa_plan_t p, const double *dA) {
  if (p && p->inner)
    return set_err(FA_ERR_UNSUPPORTED, "FA_FLOW_COS plans are solved with fa_parareal_solve only");
  FA_TRY(check_ready(p, false));
  if (!dA) return set_err(FA_ERR_ARG, "null A");
  const int n = p->d.n;
  const size_t nn = p->nn;
  if (dA != p->A64)
    FA_CUDA(cudaMemcpyAsync(p->A64, dA, nn * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  FA_CUDA(fa::launch_check_finite(p->A64, nn, p->err, p->stream));
  p->mstats_valid = false;
  if (p->B64) FA_CUDA(fa::launch_i_minus(p->A64, n, p->B64, p->stream));
  {
    // Crank-Nicolson step matrices M = (I - c A)^{-1} A, c = half the step
    const fa_problem_desc &d = p->d;
    const double hF = d.T / d.N / d.fine_steps, hG = d.T / d.N / d.coarse_steps;
    const int tl = p->ps.terms_l;
    if (p->MF64) {
      FA_CUDA(fa::launch_cn_matrix(p->A64, n, 0.5 * hF, p->aug, p->MF64, p->err, p->stream));
      if (p->AopF)
        FA_CUDA(fa::launch_split_terms(p->MF64, 1, n, p->ldp, p->AopF, tl, p->strideA, nullptr,
                                       0, 0, 0, p->stream));
    }
    if (p->MG64) {
      FA_CUDA(fa::launch_cn_matrix(p->A64, n, 0.5 * hG, p->aug, p->MG64, p->err, p->stream));
      if (p->AopG)
        FA_CUDA(fa::launch_split_terms(p->MG64, 1, n, p->ldp, p->AopG, tl, p->strideA, nullptr,
                                       0, 0, 0, p->stream));
    }
  }
  if (p->mixed || p->cmixed) {
    const int tl = p->ps.terms_l;
    if (p->d.flow == FA_FLOW_EXP)
      FA_CUDA(fa::launch_split_terms(p->A64, 1, n, p->ldp, p->Aop, tl, p->strideA, nullptr, 0, 0,
                                     0, p->stream));
    else if (p->d.flow == FA_FLOW_INV)
      FA_CUDA(fa::launch_split_terms(p->A64, 1, n, p->ldp, p->Aop, tl, p->strideA, nullptr, 0, 0,
                                     1, p->stream));
    else
      FA_CUDA(fa::launch_colmajor_pair(p->A64, n, p->a_hi, p->a_lo, p->stream));
  }
  p->matrix_set = true;
  return FA_OK;
}

fa_status fa_fine_sweep(fa_plan_t p, const double *dU, double *dF) {
  if (p && p->inner)
    return set_err(FA_ERR_UNSUPPORTED, "FA_FLOW_COS plans are solved with fa_parareal_solve only");
  FA_TRY(check_ready(p, true));
  if (!dU || !dF) return set_err(FA_ERR_ARG, "null pointer");
  return fine_sweep(p, dU, dF, nullptr);
}

fa_status fa_coarse_sweep(fa_plan_t p, const double *dU0, const double *dD, double *dUnew,
                          double *dGnew, double *dNorms, const double *dUold) {
  if (p && p->inner)
    return set_err(FA_ERR_UNSUPPORTED, "FA_FLOW_COS plans are solved with fa_parareal_solve only");
  FA_TRY(check_ready(p, true));
  if (!dU0 || !dUnew || !dGnew) return set_err(FA_ERR_ARG, "null pointer");
  if (dNorms && !dUold) return set_err(FA_ERR_ARG, "dNorms requires dUold");
  return coarse_sweep(p, dU0, dD, dUnew, dGnew, dNorms, dUold);
}

fa_status fa_refine(fa_plan_t p, double *dX) {
  if (p && p->inner)
    return set_err(FA_ERR_UNSUPPORTED, "FA_FLOW_COS plans are solved with fa_parareal_solve only");
  FA_TRY(check_ready(p, true));
  if (!dX) return set_err(FA_ERR_ARG, "null pointer");
  if (p->d.flow == FA_FLOW_EXP)
    return set_err(FA_ERR_UNSUPPORTED, "the exponential flow has no refinement");
  return refine(p, dX);
}

fa_status fa_parareal_solve(fa_plan_t p, const double *dA, const double *dX0, double *dXout,
                            fa_report *r) {
  FA_TRY(check_ready(p, false));
  if (!dA || !dXout) return set_err(FA_ERR_ARG, "null pointer");
  if (p->inner) {
    if (dX0) return set_err(FA_ERR_ARG, "FA_FLOW_COS starts from (0; I): dX0 must be NULL");
    return cos_solve(p, dA, dXout, r);
  }
  if (p->aima) return set_err(FA_ERR_ARG, "AIMA plans are run with fa_aima");
  if (p->d.refine_steps > 0 && p->d.flow == FA_FLOW_EXP)
    return set_err(FA_ERR_UNSUPPORTED, "the exponential flow has no refinement");
  const fa_problem_desc &d = p->d;
  const size_t nn = p->nn;
  cudaEvent_t ev[4];
  for (auto &e : ev) FA_CUDA(cudaEventCreate(&e));
  struct EvGuard {
    cudaEvent_t *e;
    ~EvGuard() {
      for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
    }
  } guard{ev};
  if (p->learned && !p->params_set)
    return set_err(FA_ERR_ARG, "fa_plan_set_learned has not been called");
  FA_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), p->stream));
  FA_CUDA(cudaMemsetAsync(p->fallbacks, 0, sizeof(int), p->stream));
  if (p->modified) {
    FA_TRY(fa_plan_set_matrix(p, dA));
    return modified_solve(p, dX0, dXout, r);
  }

  p->learned_active = p->learned;
  p->rec_count = 0;
  int g_fallback_iter = 0;
  FA_CUDA(cudaEventRecord(ev[0], p->stream));
  FA_TRY(fa_plan_set_matrix(p, dA));
  double dx_euler1 = INFINITY;   // Euler G's first convergence measure (the opt-in guard's bar)
  if (p->learned && p->learned_check && d.max_iters > 0) {
    p->learned_active = false;
    if (dX0) {
      FA_CUDA(cudaMemcpyAsync(p->U, dX0, nn * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    } else {
      FA_CUDA(fa::launch_identity(p->U, d.n, p->stream));
    }
    FA_TRY(coarse_sweep(p, p->U, nullptr, p->U, p->Gold, nullptr, nullptr));
    FA_TRY(fine_sweep(p, p->U, p->D, p->Gold));
    FA_TRY(coarse_sweep(p, p->U, p->D, p->U, p->Gnew, p->norms, p->U));
    FA_CUDA(fa::launch_max_ratio(p->norms, d.N, p->dx, p->err, p->stream));
    FA_CUDA(cudaMemcpyAsync(&dx_euler1, p->dx, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    FA_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), p->stream));
    FA_CUDA(cudaStreamSynchronize(p->stream));
    p->learned_active = true;
  }
  if (dX0) {
    FA_CUDA(cudaMemcpyAsync(p->U, dX0, nn * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  } else {
    FA_CUDA(fa::launch_identity(p->U, d.n, p->stream));
  }
  // Step 0 (eq. eqStep0): U^0_{n+1} = G(U^0_n), G(U^0_n) kept as G_old.
  FA_TRY(coarse_sweep(p, p->U, nullptr, p->U, p->Gold, nullptr, nullptr));
  FA_CUDA(cudaEventRecord(ev[1], p->stream));
  FA_CUDA(cudaEventSynchronize(ev[1]));
  float ms = 0.f;
  FA_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
  double t_init = ms, t_fine = 0.0, t_coarse = 0.0, t_ref = 0.0;
  int iters = 0;
  bool converged = false;
  double dx = INFINITY, prev_dx = INFINITY;
  fa_status st = FA_OK;
  for (int k = 0; k < d.max_iters; ++k) {
    // Step k+1: the fine propagator on every slice at once, D_n = F(U^k_n) - G(U^k_n) ...
    FA_CUDA(cudaEventRecord(ev[1], p->stream));
    FA_TRY(fine_sweep(p, p->U, p->D, p->Gold));
    if (p->rec && p->rec_count + d.N <= p->rec_cap) {
      // training pairs (U^k_n, F(U^k_n)), F(U^k_n) = D_n + G(U^k_n)
      FA_TRY(records(p, p->U, p->D, p->Gold, p->rec + static_cast<size_t>(p->rec_count) * FA_RECORD_DOUBLES,
                     p->rec_scratch, p->rec_scratch_bytes));
      p->rec_count += d.N;
    }
    FA_CUDA(cudaEventRecord(ev[2], p->stream));
    // ... then the sequential correction U^{k+1}_{n+1} = G(U^{k+1}_n) + D_n (eq. eqStepk+1).
    FA_TRY(coarse_sweep(p, p->U, p->D, p->U, p->Gnew, p->norms, p->U));
    FA_CUDA(fa::launch_max_ratio(p->norms, d.N, p->dx, p->err, p->stream));
    FA_CUDA(cudaEventRecord(ev[3], p->stream));
    FA_CUDA(cudaMemcpyAsync(&dx, p->dx, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    FA_CUDA(cudaStreamSynchronize(p->stream));
    FA_CUDA(cudaEventElapsedTime(&ms, ev[1], ev[2]));
    t_fine += ms;
    FA_CUDA(cudaEventElapsedTime(&ms, ev[2], ev[3]));
    t_coarse += ms;
    double *t = p->Gold;
    p->Gold = p->Gnew;
    p->Gnew = t;
    ++iters;
    if (r && r->dx_history) r->dx_history[k] = dx;
    if (!std::isfinite(dx)) {
      st = set_err(FA_ERR_NONFINITE, "non-finite convergence measure at iteration %d", k + 1);
      break;
    }
    if (dx < d.tol) {
      converged = true;
      break;
    }
    if (p->learned_active && ((k > 0 && dx > prev_dx) || (k == 0 && dx > dx_euler1))) {
      // Fallback: the rest of the solve runs with Euler G; G(U^k_n) is recomputed with it so
      // that the next correction F(U^k_n) - G(U^k_n) uses one propagator.
      p->learned_active = false;
      g_fallback_iter = k + 1;
      FA_TRY(euler_all(p, p->U, p->Gold));
    }
    prev_dx = dx;
  }
  FA_CUDA(cudaMemcpyAsync(dXout, p->U + static_cast<size_t>(d.N) * nn, nn * sizeof(double),
                          cudaMemcpyDeviceToDevice, p->stream));
  if (d.refine_steps > 0 && st == FA_OK) {
    FA_CUDA(cudaEventRecord(ev[1], p->stream));
    FA_TRY(refine(p, dXout));
    FA_CUDA(cudaEventRecord(ev[2], p->stream));
    FA_CUDA(cudaEventSynchronize(ev[2]));
    FA_CUDA(cudaEventElapsedTime(&ms, ev[1], ev[2]));
    t_ref = ms;
  }
  p->learned_active = p->learned;
  fa_status es = read_err(p);
  int coef_fb = 0;
  FA_CUDA(cudaMemcpyAsync(&coef_fb, p->fallbacks, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  FA_CUDA(cudaStreamSynchronize(p->stream));
  if (r) {
    r->g_fallback_iter = g_fallback_iter;
    r->coef_fallbacks = coef_fb;
    r->records = p->rec_count;
    r->basis_dim = 0;
    r->fine_blocks = iters * d.N;
    r->iters = iters;
    r->converged = converged ? 1 : 0;
    r->last_dx = dx;
    r->t_init_ms = t_init;
    r->t_fine_ms = t_fine;
    r->t_coarse_ms = t_coarse;
    r->t_refine_ms = t_ref;
  }
  if (es != FA_OK) return es;
  if (st != FA_OK) return st;
  if (!converged && d.tol > 0.0)
    return set_err(FA_ERR_NOT_CONVERGED, "tolerance %.3g not reached in %d iterations (dx %.3g)",
                   d.tol, iters, dx);
  return FA_OK;
}

fa_status fa_parareal_solve_host(fa_plan_t p, const double *hA, const double *hX0, double *hXout,
                                 fa_report *r) {
  FA_TRY(check_ready(p, false));
  if (!hA || !hXout) return set_err(FA_ERR_ARG, "null pointer");
  if (p->inner && hX0) return set_err(FA_ERR_ARG, "FA_FLOW_COS starts from (0; I): hX0 must be NULL");
  if (p->aima) return set_err(FA_ERR_ARG, "AIMA plans are run with fa_aima");
  const size_t bytes = p->nn * sizeof(double);
  FA_CUDA(cudaMemcpyAsync(p->A64, hA, bytes, cudaMemcpyHostToDevice, p->stream));
  if (hX0) FA_CUDA(cudaMemcpyAsync(p->Xin, hX0, bytes, cudaMemcpyHostToDevice, p->stream));
  fa_status s = fa_parareal_solve(p, p->A64, hX0 ? p->Xin : nullptr, p->Xout, r);
  if (s != FA_OK && s != FA_ERR_NOT_CONVERGED) return s;
  FA_CUDA(cudaMemcpyAsync(hXout, p->Xout, bytes, cudaMemcpyDeviceToHost, p->stream));
  FA_CUDA(cudaStreamSynchronize(p->stream));
  return s;
}

fa_status fa_debug_product(fa_plan_t p, const double *dL, const double *dR, double *dC) {
  if (p && p->inner)
    return set_err(FA_ERR_UNSUPPORTED, "FA_FLOW_COS plans are solved with fa_parareal_solve only");
  FA_TRY(check_ready(p, false));
  if (!dL || !dR || !dC) return set_err(FA_ERR_ARG, "null pointer");
  EpiParams e = base_epi(p);
  e.mode = fa::EPI_STORE;
  e.alpha = 1.0;
  e.beta = 0.0;
  e.store_out = dC;
  if (p->cmixed) {
    const int tl = p->ps.terms_l, tr = p->ps.terms_r;
    if (!p->Vl[0]) return set_err(FA_ERR_UNSUPPORTED, "debug product needs an L-form buffer (flow inv/sqrt)");
    FA_CUDA(fa::launch_split_terms(dL, 1, p->d.n, p->ldp, p->Vl[0], tl, p->strideV, nullptr, 0, 0,
                                   0, p->stream));
    FA_CUDA(fa::launch_split_terms(dR, 1, p->d.n, p->ldp, nullptr, 0, 0, p->Vr[0], tr, p->strideV,
                                   0, p->stream));
    return tc(p, p->tmVl[0], p->tmVr[0], tc_params(p, 1, 0, 0, e));
  }
  return f64(p, dL, 0, dR, 0, 1, e);
}

fa_status fa_debug_set_wait_fault(long long wait_cycles, int skip_loads_cta) {
  if (wait_cycles < 0) return set_err(FA_ERR_ARG, "wait_cycles must be >= 0");
  g_wait_cycles = wait_cycles;
  g_skip_loads_cta = skip_loads_cta < 0 ? -1 : skip_loads_cta;
  return FA_OK;
}

fa_status fa_debug_set_profile(unsigned long long *d_counters) {
  g_prof = d_counters;
  return FA_OK;
}


fa_status fa_plan_set_learned(fa_plan_t p, const float *d_params) {
  FA_TRY(check_ready(p, false));
  if (!p->learned) return set_err(FA_ERR_ARG, "the plan's coarse kind is not FA_COARSE_LEARNED");
  if (!d_params) return set_err(FA_ERR_ARG, "null parameter blob");
  FA_CUDA(cudaMemcpyAsync(p->mlp, d_params, FA_MLP_PARAMS * sizeof(float),
                          cudaMemcpyDeviceToDevice, p->stream));
  p->params_set = true;
  return FA_OK;
}

fa_status fa_plan_learned_coefs(fa_plan_t p, float *d_coef) {
  FA_TRY(check_ready(p, false));
  if (!d_coef) return set_err(FA_ERR_ARG, "null pointer");
  FA_CUDA(cudaMemcpyAsync(d_coef, p->coef, static_cast<size_t>(p->d.N) * FA_MLP_COEFS * sizeof(float),
                          cudaMemcpyDeviceToDevice, p->stream));
  return FA_OK;
}

fa_status fa_learned_records_scratch(fa_plan_t p, size_t *bytes) {
  if (!p || !bytes) return set_err(FA_ERR_ARG, "null argument");
  *bytes = records_scratch_bytes(p);
  return FA_OK;
}

fa_status fa_learned_records(fa_plan_t p, const double *dU, const double *dF, double *d_records,
                             void *d_scratch, size_t scratch_bytes) {
  FA_TRY(check_ready(p, true));
  if (!dU || !dF || !d_records) return set_err(FA_ERR_ARG, "null pointer");
  return records(p, dU, dF, nullptr, d_records, d_scratch, scratch_bytes);
}

fa_status fa_plan_set_learned_check(fa_plan_t p, int enable) {
  FA_TRY(check_ready(p, false));
  if (!p->learned) return set_err(FA_ERR_ARG, "the plan's coarse propagator is not the learned one");
  p->learned_check = enable != 0;
  return FA_OK;
}

fa_status fa_plan_set_recorder(fa_plan_t p, double *d_records, int capacity_pairs, void *d_scratch,
                               size_t scratch_bytes) {
  FA_TRY(check_ready(p, false));
  if (!d_records) {
    p->rec = nullptr;
    p->rec_cap = 0;
    return FA_OK;
  }
  if (p->d.flow == FA_FLOW_SQRT)
    return set_err(FA_ERR_UNSUPPORTED, "pair records are implemented for the inverse and exponential flows");
  if (capacity_pairs < 0) return set_err(FA_ERR_ARG, "capacity must be >= 0");
  if (!d_scratch || scratch_bytes < records_scratch_bytes(p))
    return set_err(FA_ERR_WORKSPACE, "records scratch of %zu bytes < %zu needed", scratch_bytes,
                   records_scratch_bytes(p));
  p->rec = d_records;
  p->rec_cap = capacity_pairs;
  p->rec_scratch = d_scratch;
  p->rec_scratch_bytes = scratch_bytes;
  return FA_OK;
}

fa_status fa_mlp_forward(const float *d_params, int batch, const double *d_feat, int feat_stride,
                         float *d_coef, void *stream) {
  if (!d_params || !d_feat || !d_coef) return set_err(FA_ERR_ARG, "null pointer");
  if (batch < 0 || feat_stride < FA_MLP_FEATURES) return set_err(FA_ERR_ARG, "bad batch or stride");
  if (batch == 0) return FA_OK;
  FA_CUDA(fa::launch_mlp_forward(d_params, batch, d_feat, feat_stride, d_coef, nullptr,
                                 static_cast<cudaStream_t>(stream)));
  return FA_OK;
}

fa_status fa_mlp_scratch_bytes(int batch, size_t *bytes) {
  if (batch < 1 || !bytes) return set_err(FA_ERR_ARG, "batch must be >= 1");
  *bytes = fa::mlp_train_scratch_bytes(batch);
  return FA_OK;
}

fa_status fa_mlp_loss_grad(const float *d_params, int batch, const double *d_records,
                           float *d_grad, double *d_loss, void *d_scratch, size_t scratch_bytes,
                           void *stream) {
  if (!d_params || !d_records || !d_grad || !d_loss || !d_scratch)
    return set_err(FA_ERR_ARG, "null pointer");
  if (batch < 1) return set_err(FA_ERR_ARG, "batch must be >= 1");
  if (scratch_bytes < fa::mlp_train_scratch_bytes(batch))
    return set_err(FA_ERR_WORKSPACE, "scratch of %zu bytes < %zu needed", scratch_bytes,
                   fa::mlp_train_scratch_bytes(batch));
  if (reinterpret_cast<uintptr_t>(d_scratch) & 255)
    return set_err(FA_ERR_WORKSPACE, "scratch must be 256-byte aligned");
  FA_CUDA(fa::launch_mlp_loss_grad(d_params, batch, d_records, d_scratch, d_grad, d_loss,
                                   static_cast<cudaStream_t>(stream)));
  return FA_OK;
}

fa_status fa_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int step,
                      float lr, float beta1, float beta2, float eps, void *stream) {
  if (!d_params || !d_grad || !d_m || !d_v) return set_err(FA_ERR_ARG, "null pointer");
  if (step < 1) return set_err(FA_ERR_ARG, "step must be >= 1");
  const float c1 = static_cast<float>(1.0 / (1.0 - std::pow(static_cast<double>(beta1), step)));
  const float c2 = static_cast<float>(1.0 / (1.0 - std::pow(static_cast<double>(beta2), step)));
  FA_CUDA(fa::launch_adam(d_params, d_grad, d_m, d_v, lr, beta1, beta2, eps, c1, c2,
                          static_cast<cudaStream_t>(stream)));
  return FA_OK;
}

fa_status fa_batch_plan(fa_batch_t *out, int count, const int *ns, const int *flows,
                        const double *Ts, const int *coarse_steps, int N, int fine_steps,
                        int max_iters, double tol, int dtype, void *stream,
                        size_t *workspace_bytes) {
  if (!out || !ns || !flows || !Ts || !coarse_steps || !workspace_bytes)
    return set_err(FA_ERR_ARG, "null argument");
  *out = nullptr;
  if (count < 1) return set_err(FA_ERR_ARG, "count must be >= 1");
  if (dtype < FA_BF16 || dtype > FA_BF16X6)
    return set_err(FA_ERR_ARG, "batched solves use a BF16 form (FA_BF16*)");
  fa_batch_s *b = new (std::nothrow) fa_batch_s();
  if (!b) return set_err(FA_ERR_ARG, "out of host memory");
  b->count = count;
  b->N = N;
  b->J = fine_steps;
  b->max_iters = max_iters;
  b->tol = tol;
  b->dtype = dtype;
  b->stream = static_cast<cudaStream_t>(stream);
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    fa_problem_desc d{};
    d.n = ns[i];
    d.flow = flows[i];
    d.T = Ts[i];
    d.N = N;
    d.coarse_steps = coarse_steps[i];
    d.fine_steps = fine_steps;
    d.max_iters = max_iters;
    d.tol = tol;
    d.fine_dtype = dtype;
    d.coarse_dtype = dtype;
    d.refine_steps = 0;
    fa_plan_t p = nullptr;
    size_t need = 0;
    const fa_status st = fa_plan(&p, &d, stream, &need);
    if (st != FA_OK) {
      delete b;
      return set_err(st, "problem %d: %s", i, fa_last_error());
    }
    b->plans.push_back(p);
    b->offs.push_back(off);
    off += (need + 255) & ~static_cast<size_t>(255);
    if (d.coarse_steps > b->max_m) b->max_m = d.coarse_steps;
    b->num_sms = p->num_sms;
  }
  // segment tables: fine 10 x count, coarse 2 x N x max_m x 2 x count (upper bound)
  b->nseg_total = static_cast<size_t>(count) * (10 + 4 * static_cast<size_t>(N) * b->max_m);
  b->seg_off = off;
  off += b->nseg_total * sizeof(fa::TcSegment);
  off = (off + 255) & ~static_cast<size_t>(255);
  b->norm_off = off;
  off += static_cast<size_t>(count) * sizeof(fa::BatchNorm);
  off = (off + 255) & ~static_cast<size_t>(255);
  b->dx_off = off;
  off += static_cast<size_t>(count) * sizeof(double);
  off = (off + 255) & ~static_cast<size_t>(255);
  b->err_off = off;
  off += 256;
  b->ws_need = off;
  *workspace_bytes = off;
  *out = b;
  return FA_OK;
}

fa_status fa_batch_bind_workspace(fa_batch_t b, void *d_ws, size_t bytes) {
  if (!b) return set_err(FA_ERR_ARG, "null batch");
  if (!d_ws) return set_err(FA_ERR_WORKSPACE, "null workspace");
  if (bytes < b->ws_need)
    return set_err(FA_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", bytes, b->ws_need);
  if (reinterpret_cast<uintptr_t>(d_ws) & 255)
    return set_err(FA_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  FA_CUDA(cudaSetDevice(b->plans[0]->device));
  b->ws = static_cast<char *>(d_ws);
  b->d_segs = reinterpret_cast<fa::TcSegment *>(b->ws + b->seg_off);
  b->d_norm = reinterpret_cast<fa::BatchNorm *>(b->ws + b->norm_off);
  b->d_dx = reinterpret_cast<double *>(b->ws + b->dx_off);
  b->d_err = reinterpret_cast<int *>(b->ws + b->err_off);
  for (int i = 0; i < b->count; ++i) {
    fa_plan_s *p = b->plans[i];
    FA_TRY(fa_plan_bind_workspace(p, b->ws + b->offs[i], p->ws_need));
  }
  const int pf = b->plans[0]->ps.npairs == 1 ? 1 : 0;
  for (int k = 0; k < fa_batch_s::kBuckets; ++k) {
    b->prefetch_b[k] = pf;
    b->raster_b[k] = 0;
  }
  b->order = 0;
  b->active.clear();
  FA_TRY(upload_tables(b));
  std::vector<fa::BatchNorm> norms(b->count);
  for (int i = 0; i < b->count; ++i) {
    norms[i].part = b->plans[i]->part;
    norms[i].tiles = b->plans[i]->part_tiles;
  }
  FA_CUDA(cudaMemcpyAsync(b->d_norm, norms.data(), norms.size() * sizeof(fa::BatchNorm),
                          cudaMemcpyHostToDevice, b->stream));
  FA_CUDA(cudaStreamSynchronize(b->stream));
  return FA_OK;
}

namespace {

// Valid operands for timing launches: every slice of U = I, the RK4 state loaded from it.
fa_status timing_state(fa_plan_s *p, cudaStream_t s) {
  for (int k = 0; k < p->d.N; ++k)
    FA_CUDA(fa::launch_identity(p->U + static_cast<size_t>(k) * p->nn, p->d.n, s));
  if (p->mixed)
    FA_CUDA(fa::launch_load_state(p->U, p->d.N, p->d.n, p->ldp, p->x_hi, p->x_lo, p->Yl[0],
                                  p->needs_l() ? p->ps.terms_l : 0, p->strideY, p->Yr[0],
                                  p->ps.terms_r, p->strideY, s));
  return FA_OK;
}

// A short signature of a batch's problems (FNV-1a over n, flow, T and m).
unsigned long long batch_signature(const fa_batch_s *b) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) {
    for (int k = 0; k < 8; ++k) {
      h ^= (v >> (8 * k)) & 0xffu;
      h *= 1099511628211ull;
    }
  };
  for (const fa_plan_s *p : b->plans) {
    unsigned long long tb;
    memcpy(&tb, &p->d.T, sizeof(tb));
    mix(static_cast<unsigned long long>(p->d.n));
    mix(static_cast<unsigned long long>(p->d.flow));
    mix(tb);
    mix(static_cast<unsigned long long>(p->d.coarse_steps));
  }
  return h;
}

std::string schedule_string(const fa_batch_s *b) {
  std::string s = "order=" + std::to_string(b->order) + " buckets=";
  for (int k = 0; k < fa_batch_s::kBuckets; ++k) {
    if (k) s += ",";
    s += std::to_string(b->prefetch_b[k]) + std::to_string(b->raster_b[k]);
  }
  return s;
}

bool parse_schedule(fa_batch_s *b, const char *line) {
  int order = 0;
  char bk[128] = {0};
  if (sscanf(line, "order=%d buckets=%127s", &order, bk) != 2) return false;
  int pf[fa_batch_s::kBuckets], rs[fa_batch_s::kBuckets];
  const char *c = bk;
  for (int k = 0; k < fa_batch_s::kBuckets; ++k) {
    if (c[0] < '0' || c[0] > '1' || c[1] < '0' || c[1] > '1') return false;
    pf[k] = c[0] - '0';
    rs[k] = c[1] - '0';
    c += 2;
    if (k + 1 < fa_batch_s::kBuckets) {
      if (*c != ',') return false;
      ++c;
    }
  }
  b->order = order ? 1 : 0;
  for (int k = 0; k < fa_batch_s::kBuckets; ++k) {
    b->prefetch_b[k] = pf[k];
    b->raster_b[k] = rs[k];
  }
  return true;
}

}  // namespace

fa_status fa_batch_autotune(fa_batch_t b, const double *const *dA, const char *cache_path) {
  if (!b) return set_err(FA_ERR_ARG, "null batch");
  if (!b->ws) return set_err(FA_ERR_WORKSPACE, "no workspace bound");
  if (!dA) return set_err(FA_ERR_ARG, "null pointer");
  FA_TRY(activate_all(b));
  char key[160];
  snprintf(key, sizeof(key), "fa-batch count=%d N=%d J=%d dtype=%d sig=%016llx", b->count, b->N,
           b->J, b->dtype, batch_signature(b));
  if (cache_path) {
    if (FILE *f = fopen(cache_path, "r")) {
      char line[512];
      bool hit = false;
      while (fgets(line, sizeof(line), f)) {
        const size_t kl = strlen(key);
        if (strncmp(line, key, kl) == 0 && line[kl] == ' ' && parse_schedule(b, line + kl + 1)) hit = true;
      }
      fclose(f);
      if (hit) {
        FA_TRY(upload_tables(b));
        b->tuning = std::string("from cache: ") + schedule_string(b);
        return FA_OK;
      }
    }
  }
  for (int i = 0; i < b->count; ++i) {
    fa_plan_s *p = b->plans[i];
    if (!dA[i]) return set_err(FA_ERR_ARG, "null pointer for problem %d", i);
    p->err = b->d_err;
    FA_TRY(fa_plan_set_matrix(p, dA[i]));
    FA_TRY(timing_state(p, b->stream));
  }
  cudaEvent_t e0, e1;
  FA_CUDA(cudaEventCreate(&e0));
  FA_CUDA(cudaEventCreate(&e1));
  // time of the fine sweep's stage-2 launches (both product phases), 3 repetitions
  auto measure = [&](float *ms) -> fa_status {
    FA_TRY(upload_tables(b));
    FA_TRY(launch_table(b, b->fine[1][0]));
    FA_TRY(launch_table(b, b->fine[1][1]));
    FA_CUDA(cudaEventRecord(e0, b->stream));
    for (int r = 0; r < 3; ++r) {
      FA_TRY(launch_table(b, b->fine[1][0]));
      FA_TRY(launch_table(b, b->fine[1][1]));
    }
    FA_CUDA(cudaEventRecord(e1, b->stream));
    FA_CUDA(cudaEventSynchronize(e1));
    FA_CUDA(cudaEventElapsedTime(ms, e0, e1));
    *ms /= 3.0f;
    return FA_OK;
  };
  bool present[fa_batch_s::kBuckets] = {false, false, false, false, false, false};
  for (const fa_plan_s *p : b->plans) present[size_bucket(p->d.n)] = true;
  float best = 0.f, t = 0.f, base = 0.f;
  fa_status st = measure(&best);
  base = best;
  std::string log;
  // coordinate descent: keep a change only if it saves more than 1 %
  auto trial = [&](int *knob, const char *name) -> fa_status {
    *knob ^= 1;
    const fa_status s2 = measure(&t);
    if (s2 != FA_OK) return s2;
    const bool keep = t < 0.99f * best;
    char buf[96];
    snprintf(buf, sizeof(buf), "%s:%.3f%s ", name, t, keep ? "*" : "");
    log += buf;
    if (keep) best = t;
    else *knob ^= 1;
    return FA_OK;
  };
  if (st == FA_OK) st = trial(&b->order, "order");
  for (int k = 0; st == FA_OK && k < fa_batch_s::kBuckets; ++k) {
    if (!present[k]) continue;
    char nm[32];
    snprintf(nm, sizeof(nm), "b%d.prefetch", k);
    st = trial(&b->prefetch_b[k], nm);
    if (st != FA_OK) break;
    snprintf(nm, sizeof(nm), "b%d.raster", k);
    st = trial(&b->raster_b[k], nm);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FA_OK) return st;
  FA_TRY(upload_tables(b));
  char head[160];
  snprintf(head, sizeof(head), "tuned: stage launch %.3f -> %.3f ms; ", base, best);
  b->tuning = std::string(head) + schedule_string(b) + "; trials " + log;
  if (cache_path) {
    if (FILE *f = fopen(cache_path, "a")) {
      fprintf(f, "%s %s\n", key, schedule_string(b).c_str());
      fclose(f);
    } else {
      return set_err(FA_ERR_ARG, "cannot write the tuning cache %s", cache_path);
    }
  }
  return FA_OK;
}

const char *fa_batch_tuning(fa_batch_t b) { return b ? b->tuning.c_str() : ""; }

fa_status fa_plan_autotune(fa_plan_t p) {
  if (p && p->inner)
    return set_err(FA_ERR_UNSUPPORTED, "FA_FLOW_COS plans are solved with fa_parareal_solve only");
  FA_TRY(check_ready(p, true));
  if (p->fp8) {
    p->tuning = "E4M3 operands: the default schedule";
    return FA_OK;
  }
  if (!p->mixed) {
    p->tuning = "float64 products: nothing to tune";
    return FA_OK;
  }
  FA_TRY(timing_state(p, p->stream));
  cudaEvent_t e0, e1;
  FA_CUDA(cudaEventCreate(&e0));
  FA_CUDA(cudaEventCreate(&e1));
  const int N = p->d.N, tl = p->ps.terms_l, tr = p->ps.terms_r;
  // the fine sweep's stage-2 product(s) under a schedule
  auto stage = [&]() -> fa_status {
    EpiParams e = base_epi(p);
    e.mode = fa::EPI_STAGE;
    e.stage = 2;
    e.h = 1e-3;
    e.ch = 5e-4;
    e.x_hi = p->x_hi;
    e.x_lo = p->x_lo;
    e.acc = p->acc;
    e.a_hi = p->a_hi;
    e.a_lo = p->a_lo;
    e.out_r = p->Yr[1];
    e.out_l = p->Yl[1];
    e.terms_r = tr;
    e.terms_l = p->needs_l() ? tl : 0;
    e.term_stride_r = e.term_stride_l = p->strideY;
    if (p->d.flow == FA_FLOW_EXP) return tc(p, p->tmA, p->tmYr[0], tc_params(p, N, 0, 1, e));
    if (p->d.flow == FA_FLOW_SQRT) return tc(p, p->tmYl[0], p->tmYr[0], tc_params(p, N, 1, 1, e));
    EpiParams e1 = base_epi(p);
    e1.mode = fa::EPI_PROD;
    e1.out_r = p->Pr;
    e1.terms_r = tr;
    e1.term_stride_r = p->strideY;
    FA_TRY(tc(p, p->tmA, p->tmYr[0], tc_params(p, N, 0, 1, e1)));
    return tc(p, p->tmYl[0], p->tmPr, tc_params(p, N, 1, 1, e));
  };
  float best = 1e30f;
  int bp = 0, br = 0;
  std::string log;
  fa_status st = FA_OK;
  for (int pf = 0; pf < 2 && st == FA_OK; ++pf)
    for (int rs = 0; rs < 2 && st == FA_OK; ++rs) {
      p->tune_prefetch = pf;
      p->tune_raster = rs;
      st = stage();
      if (st != FA_OK) break;
      cudaEventRecord(e0, p->stream);
      for (int r = 0; r < 3 && st == FA_OK; ++r) st = stage();
      cudaEventRecord(e1, p->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= 3.0f;
      char buf[64];
      snprintf(buf, sizeof(buf), "p%d r%d %.3f ms; ", pf, rs, ms);
      log += buf;
      if (ms < best * 0.99f) {
        best = ms;
        bp = pf;
        br = rs;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FA_OK) return st;
  p->tune_prefetch = bp;
  p->tune_raster = br;
  p->tuning = "chose prefetch=" + std::to_string(bp) + " raster=" + std::to_string(br) + " (" + log + ")";
  return FA_OK;
}

const char *fa_plan_tuning(fa_plan_t p) { return p ? p->tuning.c_str() : ""; }

fa_status fa_batch_solve(fa_batch_t b, const double *const *dA, double *const *dXout, int *iters,
                         double *last_dx) {
  if (!b) return set_err(FA_ERR_ARG, "null batch");
  if (!b->ws) return set_err(FA_ERR_WORKSPACE, "no workspace bound");
  if (!dA || !dXout) return set_err(FA_ERR_ARG, "null pointer");
  FA_TRY(activate_all(b));
  FA_CUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
  for (int i = 0; i < b->count; ++i) {
    fa_plan_s *p = b->plans[i];
    if (!dA[i] || !dXout[i]) return set_err(FA_ERR_ARG, "null pointer for problem %d", i);
    p->err = b->d_err;
    FA_TRY(fa_plan_set_matrix(p, dA[i]));
    FA_CUDA(fa::launch_identity(p->U, p->d.n, b->stream));
  }
  FA_TRY(batch_coarse(b, 0));       // Step 0 (eq. eqStep0) for every problem
  std::vector<double> dx(b->count, INFINITY), dx_at(b->count, INFINITY);
  std::vector<int> conv_at(b->count, 0);
  int done = 0, k = 0;
  for (; k < b->max_iters && done < b->count; ++k) {
    if (b->graph) {
      FA_CUDA(cudaGraphLaunch(b->graph, b->stream));
    } else if (!b->graph_tried && k > 0 && b->stream) {
      // capture one iteration (every launch has fixed arguments) and replay it from now on
      b->graph_tried = true;
      cudaGraph_t gr = nullptr;
      if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const fa_status st = batch_iteration(b);
        const cudaError_t ce = cudaStreamEndCapture(b->stream, &gr);
        if (st != FA_OK) return st;
        if (ce == cudaSuccess && gr &&
            cudaGraphInstantiate(&b->graph, gr, 0) == cudaSuccess) {
          cudaGraphDestroy(gr);
          FA_CUDA(cudaGraphLaunch(b->graph, b->stream));
        } else {
          if (gr) cudaGraphDestroy(gr);
          b->graph = nullptr;
          cudaGetLastError();
          FA_TRY(batch_iteration(b));
        }
      } else {
        cudaGetLastError();
        FA_TRY(batch_iteration(b));
      }
    } else {
      FA_TRY(batch_iteration(b));
    }
    FA_CUDA(cudaMemcpyAsync(dx.data(), b->d_dx, b->count * sizeof(double), cudaMemcpyDeviceToHost,
                            b->stream));
    FA_CUDA(cudaStreamSynchronize(b->stream));
    bool changed = false;
    for (int i = 0; i < b->count; ++i) {
      if (!conv_at[i] && dx[i] < b->tol) {
        // converged: its result is U_N of this iteration, and it leaves the later launches
        conv_at[i] = k + 1;
        dx_at[i] = dx[i];
        ++done;
        fa_plan_s *p = b->plans[i];
        FA_CUDA(cudaMemcpyAsync(dXout[i], p->U + static_cast<size_t>(b->N) * p->nn,
                                p->nn * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
        if (b->active.empty()) b->active.assign(b->count, 1);
        b->active[i] = 0;
        changed = true;
      }
    }
    if (changed && done < b->count && k + 1 < b->max_iters) FA_TRY(upload_tables(b));
  }
  for (int i = 0; i < b->count; ++i) {
    fa_plan_s *p = b->plans[i];
    if (!conv_at[i])
      FA_CUDA(cudaMemcpyAsync(dXout[i], p->U + static_cast<size_t>(b->N) * p->nn,
                              p->nn * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    if (iters) iters[i] = conv_at[i] ? conv_at[i] : k;
    if (last_dx) last_dx[i] = conv_at[i] ? dx_at[i] : dx[i];
  }
  int h = 0;
  FA_CUDA(cudaMemcpyAsync(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  FA_CUDA(cudaStreamSynchronize(b->stream));
  if (h) return set_err(static_cast<fa_status>(h), "device error %d in the batch", h);
  if (done < b->count && b->tol > 0.0)
    return set_err(FA_ERR_NOT_CONVERGED, "%d of %d problems did not reach the tolerance",
                   b->count - done, b->count);
  return FA_OK;
}

fa_status fa_batch_destroy(fa_batch_t b) {
  delete b;
  return FA_OK;
}

fa_status fa_plan_destroy(fa_plan_t p) {
  delete p;
  return FA_OK;
}

const char *fa_status_string(fa_status s) {
  switch (s) {
    case FA_OK: return "ok";
    case FA_ERR_ARG: return "invalid argument";
    case FA_ERR_CUDA: return "CUDA error";
    case FA_ERR_WORKSPACE: return "workspace missing or too small";
    case FA_ERR_NONFINITE: return "non-finite values";
    case FA_ERR_NOT_CONVERGED: return "not converged";
    case FA_ERR_TIMEOUT: return "device wait timed out";
    case FA_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *fa_last_error(void) { return g_last_error.c_str(); }

unsigned long long fa_launch_count(void) { return g_launches; }

void fa_launch_count_reset(void) { g_launches = 0; }

}  // extern "C"
