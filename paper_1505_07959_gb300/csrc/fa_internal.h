// Internal declarations shared by the kernels and the host driver of libfa.
//
// Storage conventions inside the workspace (the boundary is always float64
// row-major):
//  * parareal state U, G, D: float64 row-major [count][n][n];
//  * mixed-precision RK4 state (x_hi, x_lo, acc): float32 column-major
//    [N][n][n] (element (i,j) of slice b at b n^2 + j n + i), so that the
//    epilogue's thread-per-row mapping gives coalesced warp accesses;
//  * BF16 operand terms: [term][slice][n][ldp] with ldp = n rounded up to 8
//    (16-byte rows for TMA).  The "L form" of a matrix Y is row-major
//    (row i holds Y[i][:]); the "R form" is its transpose (row j holds
//    Y[:][j]).  A tensor-core product D = L R^T therefore computes
//    D[i][j] = sum_k L[i][k] R[j][k] = (Y_left * Y_right)[i][j] when the left
//    factor is given in L form and the right factor in R form.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/fa.h"

namespace fa {

constexpr int kMaxPairs = 6;

enum EpiMode : int {
  EPI_STAGE = 0,   // RK4 stage combine (fine sweep)
  EPI_PROD = 1,    // write the product as operand terms (inverse flow: P = (I-A) Y)
  EPI_EULER = 2,   // forward-Euler substep of G, with the parareal correction on the last one
  EPI_STORE = 3,   // plain float64 store: out = alpha * v + beta * (i == j)
  EPI_TAYLOR = 4,  // a product of a Taylor-term chain: float64 copy (out64) + operand terms
  EPI_AIMA = 5,    // a step of Algorithm 8 on [X | u] (slices 0 and 1) + the residual norm
};

// Parameters of the fused epilogue.  One struct serves the tensor-core and the
// float64 kernels; fields that a mode does not use are ignored.
struct EpiParams {
  int mode;
  int flow;
  int stage;          // 1..4 (EPI_STAGE)
  int last;           // EPI_STAGE: stage 4 of the slice's last RK4 step -> write F or D
  int n;
  int ldp;            // leading dimension of BF16 operand storage
  int terms_l;        // BF16 terms to write in L form (0 = do not write)
  int terms_r;        // BF16 terms to write in R form (0 = do not write)
  size_t term_stride_l, term_stride_r;   // elements between consecutive terms
  int b0;             // slice offset of this launch inside the state arrays
  // RK4 coefficients
  double h;           // fine step
  double ch;          // c_{s+1} h: Y_{s+1} = X + ch K_s (stages 1..3)
  // mixed-precision fine state (column-major float32)
  float *x_hi, *x_lo, *acc;
  // float64 fine state (row-major)
  double *x64, *acc64;
  // the constant matrix for K = A - v (square-root flow)
  const float *a_hi, *a_lo;     // column-major float32 pair (mixed)
  const double *a64;            // row-major float64
  // new operand output (mixed: BF16 terms; f64: row-major float64)
  __nv_bfloat16 *out_l, *out_r;
  double *out64;
  // E4M3 operand output (FA_FP8E4M3 fine sweeps): bytes in L form and R form [slice][n][ldp8],
  // quantised with one float32 scale per 128 x 128 tile of the operand (delayed scaling: the
  // tile's scale is 448 / (2 amax) of the same tile of the previous operand); the epilogue
  // records the new operand's per-tile amax and the inverse scales it used.  Tile arrays are
  // [slice][T][T], T = ceil(n / 128).
  uint8_t *out_l8, *out_r8;
  int ldp8, q_T;
  const float *q_amax_in;
  float *q_inv_out, *q_amax_out;
  // fine sweep outputs (row-major float64): f_out = X (or X - g_old when g_old != 0)
  double *f_out;
  const double *g_old;
  // EPI_EULER
  double dt;                    // Euler substep dT/m
  const double *v_in;           // V (row-major float64) of this substep
  double *v_out;                // next V (intermediate substep) or V_{n+1} (last substep)
  double *g_out;                // G_n (last substep)
  const double *d_in;           // D_n (last substep; 0 = Step 0)
  const double *u_old;          // previous iterate U_{n+1} for the norms (0 = no norms)
  double *norm_part;            // per-tile partial sums [tiles][2]
  int euler_last;               // 1 on the last substep
  // EPI_STORE: store_out = alpha v + beta (i == j) (+ store_add when set), and the operand
  // terms of that value (L and/or R form) when terms_l / terms_r are set
  double alpha, beta;
  double *store_out;
  const double *store_add;
  int *err;                     // device error word
  int euler_step;               // EPI_STAGE with stage 4: an explicit step X <- X + h K (the
                                // explicit-Euler and Crank-Nicolson fine schemes), no acc read
  int transposed;               // EPI_EULER, EPI_AIMA: the launch computes the transposed
                                // product (tile element (i, j) is entry (j, i) of the method's
                                // product), so that a thread's float64 accesses to the
                                // row-major state run along a row, coalesced across the warp
};

// One problem of a ragged (multi-problem) tensor-core launch: its tensor maps, epilogue
// and shape, and the index of its first tile in the launch's tile sequence.
struct alignas(64) TcSegment {
  CUtensorMap tmL, tmR;
  EpiParams epi;
  int n, nb, l_batched, r_batched, mt, nt, kblocks, tile_begin;
  int prefetch;   // epilogue state prefetch into L2 for this problem's tiles (0 / 1)
  int raster;     // tile order inside a slice: 0 = M-tile fastest, 1 = N-tile fastest
};

// One tensor-core GEMM launch: for every slice b in [0, nb) and tile,
// D = sum_p L_{a_p} R_{b_p}^T over the BF16 term pairs, then the epilogue.
// Each 64-wide k-block loads its operand term tiles once (tl_side / tl_term,
// in load order) and issues pair p once tile pair_at[p] has landed; pair 0 is
// the main product L_0 R_0^T.
struct TcGemmParams {
  int n;            // rows of both operands and reduction length
  int nb;           // slices in this launch
  int l_batched;    // 1: L has one matrix per slice; 0: shared (slice coordinate 0)
  int r_batched;
  int mt, nt;       // tiles per slice along M and N (128 rows each)
  int num_tiles;
  int kblocks;      // ceil(n / 64)
  int ntl;          // operand tiles per k-block
  int tl_side[2 * 3];   // 0 = left operand (L form), 1 = right operand (R form)
  int tl_term[2 * 3];
  int npairs;
  int pair_tl[kMaxPairs], pair_tr[kMaxPairs], pair_at[kMaxPairs];
  uint32_t idesc;   // tcgen05 instruction descriptor
  unsigned long long *prof;   // optional per-role cycle counters (diagnostics), may be null
  int raster;                 // uniform launches: 0 = M-tile fastest, 1 = N-tile fastest
  int fp8;                    // 1: E4M3 operands (kind::f8f6f4, 128-element k-blocks), the drain
                              // scales each k-block by the two operand tiles' inverse scales
  const float *q_inv_l, *q_inv_r;   // [slice][T][T] inverse scales of L's and R's source matrix
  int q_T;
  int prefetch_state;         // 1: the epilogue warps prefetch their tile's state into L2 while
                              // the tile's products run (pays where the epilogue dominates:
                              // one term pair; with six it competes with the operand feed)
  const TcSegment *segs;      // ragged launch: per-problem segments (device), else null
  int nseg;
  long long wait_cycles;      // limit of every mbarrier wait (<= 0: ptx::kWaitCycles)
  int skip_loads_cta;         // diagnostics: this CTA issues no operand loads (-1: none), so
                              // its waits run out and the launch reports FA_ERR_TIMEOUT
  EpiParams epi;
};

// One float64 SIMT GEMM launch: C_b = L_b * R_b (row-major float64), then the epilogue.
struct F64GemmParams {
  int n;
  int nb;
  const double *L, *R;
  size_t l_stride, r_stride;     // elements between slices (0 = shared)
  EpiParams epi;
};

// Pairs of BF16 terms for each dtype and the number of terms each side needs.
struct PairSet {
  int npairs;
  int a[kMaxPairs], b[kMaxPairs];
  int terms_l, terms_r;
};
PairSet pair_set(int dtype);
// Fill the tile list and pair schedule of a launch from a pair set.
void tc_schedule(const PairSet &ps, TcGemmParams &g);

// --- launchers (return cudaGetLastError()) ---
cudaError_t launch_tc_gemm(const CUtensorMap *tmL, const CUtensorMap *tmR,
                           const TcGemmParams &p, int num_sms, cudaStream_t s);
cudaError_t launch_f64_gemm(const F64GemmParams &p, cudaStream_t s);
// Ragged launch: `nseg` device segments holding `num_tiles` tiles in total (schedule fields of
// `p` give the term tiles and pairs shared by all segments; p.epi.err the error word).
cudaError_t launch_tc_gemm_ragged(const TcSegment *segs, int nseg, int num_tiles,
                                  const TcGemmParams &p, int num_sms, cudaStream_t s);
// Tile edge the float64 GEMM uses for (n, nb), and its tiles per slice.
int f64_tile(int n, int nb);
int f64_tiles_per_slice(int n, int nb);

// float64 row-major [nb][n][n] -> BF16 terms (L form and/or R form).  Flags: SPLIT_I_MINUS
// forms I - x first (to build I - A); SPLIT_FROM_F32 splits x rounded to float32, as the
// epilogues split the states they write (so a state re-split on the host side gets the same
// bits as the one an epilogue wrote); otherwise the split is taken from the float64 value.
constexpr int SPLIT_I_MINUS = 1, SPLIT_FROM_F32 = 2;
cudaError_t launch_split_terms(const double *src, int nb, int n, int ldp, __nv_bfloat16 *out_l,
                               int terms_l, size_t stride_l, __nv_bfloat16 *out_r, int terms_r,
                               size_t stride_r, int flags, cudaStream_t s);
// float64 row-major [nb][n][n] -> column-major float32 hi/lo pair, plus BF16 terms
// of hi (the first RK4 stage operand).
cudaError_t launch_load_state(const double *U, int nb, int n, int ldp, float *x_hi, float *x_lo,
                              __nv_bfloat16 *out_l, int terms_l, size_t stride_l,
                              __nv_bfloat16 *out_r, int terms_r, size_t stride_r,
                              cudaStream_t s);
// E4M3 operand of the first RK4 stage from U (float64 [nb][n][n]): per 128 x 128 tile the
// amax of U, then bytes in L and R form quantised with scale 448 / (2 amax); writes amax and the
// inverse scales ([nb][T][T]).
cudaError_t launch_fp8_load(const double *U, int nb, int n, int ldp8, uint8_t *out_l,
                            uint8_t *out_r, float *amax, float *inv, cudaStream_t s);
// Sum per-tile partial norms in a fixed order: norms[b][2] = sum over tiles.
cudaError_t launch_reduce_norms(const double *part, int nslices, int tiles_per_slice,
                                double *norms, cudaStream_t s);
// dx = max_b sqrt(norms[b][0] / norms[b][1]); flags non-finite values.
cudaError_t launch_max_ratio(const double *norms, int nslices, double *dx, int *err,
                             cudaStream_t s);
// Per-problem convergence measure of a batch: for problem p, dx[p] = max over its N slices of
// sqrt(sum of d^2 partials / sum of v^2 partials), partials summed in a fixed order.
struct BatchNorm {
  const double *part;   // [N][tiles][2]
  int tiles;
};
cudaError_t launch_batch_norms(const BatchNorm *bn, int count, int N, double *dx, int *err,
                               cudaStream_t s);
// I - A (row-major float64).
cudaError_t launch_i_minus(const double *A, int n, double *out, cudaStream_t s);
// Column-major float32 hi/lo copy of A (for K = A - X^2 in the mixed epilogue).
cudaError_t launch_colmajor_pair(const double *A, int n, float *hi, float *lo, cudaStream_t s);
// Check an array for non-finite values (sets *err = FA_ERR_NONFINITE).
cudaError_t launch_check_finite(const double *x, size_t count, int *err, cudaStream_t s);
// X = I (row-major, count matrices)
cudaError_t launch_identity(double *X, int n, cudaStream_t s);

// --- learned coarse propagator (fa_learned.cu) ---
// Slots of the per-block stats vector.
enum StatSlot : int {
  ST_HUT = 0,          // 8 Hutchinson sums z_k^T X z_k
  ST_XX = 8,           // ||X||^2
  ST_RR = 9,           // 10 Gram sums <R_a, R_b>, a <= b (rr_index)
  ST_RD = 19,          // 4 sums <R_a, D>, D = F - X
  ST_DD = 23,          // ||D||^2
  ST_GLO = 24,         // Gershgorin lower bound (min over rows), when requested
  ST_GHI = 25,         // Gershgorin upper bound (max over rows)
  NSTAT = 26
};

// One stats pass over `nslices` slices (row-major float64 [slice][n][n] arrays).
struct StatsArgs {
  int n;
  int rows_per_block;            // stats_rows_per_block(n)
  const double *X;               // states
  size_t x_stride;
  const double *F;               // fine images (or D = F - G when G is set); null: no D sums
  const double *G;               // added to F when not null
  size_t f_stride;               // of F and G
  const double *R[4];            // raw Taylor powers R_1..R_4 (nR = 0, 1 or 4 of them)
  size_t r_stride;
  int nR;
  const uint8_t *probes;         // n bytes, bit k = sign of probe k
  int gersh;                     // 1: Gershgorin bounds of X
  double *part;                  // [nslices][stats_blocks(n)][NSTAT]
};

// Taylor scale s_a = dT^(a+1) kappa_a of the raw power R_(a+1).
struct RecordScale {
  double s[4];
};

// Per-sample activations and gradients kept between the two training kernels.
struct MlpTrainBuffers {
  double *loss;
  float *xs, *h1, *h2, *dz1, *dz2, *dc;
};

// The learned coarse step's update on one slice (row-major float64 n x n).
struct CombineArgs {
  int n;
  const double *v_in;            // X
  const double *R[4];            // raw powers R_1..R_4
  double scale[4];               // s_j = dT^j kappa_j
  const float *coef;             // c_1..c_4 (device)
  const double *d_in;            // correction D_n, or null (Step 0)
  const double *u_old;           // previous iterate for the norms, or null
  double *g_out;                 // G_theta(X)
  double *v_out;                 // X_{n+1} = G + D
  double *norm_part;             // [blocks][2], or null
};

int stats_rows_per_block(int n);
int stats_blocks(int n);
cudaError_t launch_probes(int n, uint8_t *bits, cudaStream_t s);
cudaError_t launch_stats(const StatsArgs &a, int nslices, cudaStream_t s);
// mstats[0..2] = Gershgorin lower / upper bound, Hutchinson tr(A), from a one-slice stats pass.
cudaError_t launch_matrix_stats(const double *part, int n, double *mstats, cudaStream_t s);
cudaError_t launch_records(const double *part, int nslices, int n, int N_total, int slice0,
                           double dT, const RecordScale &sc, const double *mstats, double *rec,
                           cudaStream_t s);
cudaError_t launch_mlp_forward(const float *P, int B, const double *feat, int fstride, float *coef,
                               int *fallbacks, cudaStream_t s);
size_t mlp_train_scratch_bytes(int B);
cudaError_t launch_mlp_loss_grad(const float *P, int B, const double *rec, void *scratch,
                                 float *grad, double *loss, cudaStream_t s);
cudaError_t launch_adam(float *P, const float *grad, float *m, float *v, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t s);
cudaError_t launch_coarse_coef(const float *P, const double *part, int n, int slice, int N,
                               double dT, const double *mstats, float *coef, int *fallbacks,
                               cudaStream_t s);
cudaError_t launch_combine(const CombineArgs &a, int blocks, cudaStream_t s);

// --- modified parareal (fa_krylov.cu) ---
constexpr int kKrylovBlocks = 304;   // fixed grid of the reductions (2 x 152 SMs)
// One Gram-Schmidt step on q: with prev, q -= c prev where c sums part_in[0 .. kKrylovBlocks);
// part_out[block] = partial <q, next> (or <q, q> when next is null).
cudaError_t launch_gs_step(double *q, const double *prev, const double *part_in,
                           const double *next, size_t count, double *part_out, cudaStream_t s);
// out = scale q
cudaError_t launch_scale_copy(const double *q, double scale, size_t count, double *out,
                              cudaStream_t s);
// alpha[j] = <V, Q_j> for j < d (Q: d consecutive matrices of `count` elements); part holds
// d x kKrylovBlocks partial sums.
cudaError_t launch_project_alpha(const double *V, const double *Q, size_t count, int d,
                                 double *part, double *alpha, cudaStream_t s);
// R = V - sum_j alpha_j Q_j, W = sum_j alpha_j FQ_j.
cudaError_t launch_project_combine(const double *V, const double *Q, const double *FQ,
                                   const double *alpha, int d, size_t count, double *R, double *W,
                                   cudaStream_t s);

// --- Crank-Nicolson step matrices (fa_solve.cu) ---
// M = (I - c A)^{-1} A by Gauss-Jordan elimination with partial pivoting on aug = [I - c A | A]
// (scratch of 2 n^2 doubles); a zero pivot sets *err = FA_ERR_NONFINITE.
cudaError_t launch_cn_matrix(const double *A, int n, double c, double *aug, double *M, int *err,
                             cudaStream_t s);

// --- cosine by Algorithm 5 (fa_solve.cu) ---
// out[0] = ||A||_inf (largest absolute row sum)
cudaError_t launch_inf_norm(const double *A, int n, double *out, cudaStream_t s);
// B = [[0, scale A], [-scale A, 0]] and X0 = diag(0, I), both of order 2n
cudaError_t launch_cos_block(const double *A, int n, double scale, double *B, double *X0,
                             cudaStream_t s);
// out = the n x n block at (r0, c0) of the order-2n matrix U
cudaError_t launch_extract_block(const double *U, int n, int r0, int c0, double *out,
                                 cudaStream_t s);

// --- square-root refinement helpers (fa_refine.cu) ---
constexpr int kDevNormBlocks = 256;
// One power-iteration step: y = X v, lam = ||y||, v = y / ||y||.
cudaError_t launch_power_step(const double *X, int n, double *v, double *y, double *lam,
                              cudaStream_t s);
// out = a (A + A^T)/2 + b B + c (C + C^T)/2 (null operands skipped; out may alias B).
cudaError_t launch_sym_combine(int n, double a, const double *A, double b, const double *B,
                               double c, const double *C, double *out, cudaStream_t s);
cudaError_t launch_fill(double *x, size_t count, double v, cudaStream_t s);
// *out = ||T - d I||_F^2 (part: kDevNormBlocks doubles of scratch), fixed order.
cudaError_t launch_dev_norm(const double *T, int n, double d, double *part, double *out,
                            cudaStream_t s);

// Per-thread launch counter (incremented by every launcher).
void count_launch();

// Record a failure as the calling thread's last error; returns s.
fa_status record_error(fa_status s, const char *msg);
// 4-D tensor map over BF16 operand terms [nterms][nslices][n][ldp] with a 64 x box_rows box.
fa_status encode_terms_map(CUtensorMap *m, void *base, int n, int ldp, int nslices, int nterms,
                           size_t term_stride, int box_rows);
// Launch parameters of one tensor-core product over a pair set (no epilogue fields set).
TcGemmParams tc_launch_params(int n, int nb, int l_batched, int r_batched, const PairSet &ps);

}  // namespace fa
