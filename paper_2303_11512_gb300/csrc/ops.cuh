// Host-side launchers of the library's CUDA kernels.  All vectors use the
// canonical layout [rhs][site][dof] with complex entries (float2 / double2).
// `active` (device int[nrhs] or nullptr) masks right-hand sides: kernels skip
// every rhs whose flag is 0.
#pragma once

#include "common.cuh"

namespace mg {

// ---------------------------------------------------------------- fine level
// links out[site][mu] = -1/2 * eta * U_mu(site); eta = -1 on the t links of the
// last time slice (antiperiodic fermion boundary folded into the link).
void prepare_links(cudaStream_t st, const double2* U, int L, double2* l64, float2* l32);
// *bad = 1 if some link of U is NaN or infinite (bad is not cleared)
void check_links(cudaStream_t st, const double2* U, int L, int* bad);
// y = D x, or y = b - D x when b != nullptr.
template <typename R>
void wilson_apply(cudaStream_t st, const typename CT<R>::T* links, R diag, int L,
                  const typename CT<R>::T* x, typename CT<R>::T* y, const typename CT<R>::T* b,
                  int nrhs, const int* active);
// dense diagonal blocks D_BB (bs x bs sites, 2 dof) of the fine operator: out[block][bd][bd]
void fine_block_matrices(cudaStream_t st, const double2* l64, double diag, int L, int bs, double2* out);

// ---------------------------------------------------------------- coarse levels
template <typename R>
void coarse_apply(cudaStream_t st, const typename CT<R>::T* stencil, int Ls, int d,
                  const typename CT<R>::T* x, typename CT<R>::T* y, const typename CT<R>::T* b,
                  int nrhs, const int* active);
void coarse_block_matrices(cudaStream_t st, const double2* stencil, int Ls, int d, int bs, double2* out);

// ---------------------------------------------------------------- SAP
// one colour half-sweep: x_B += inv_B (f - D x)_B on the blocks of colour `color`.
// inv_transposed: block inverses stored transposed (inv[b][j][i]), as blocks_to_fp32_transposed writes them
template <typename R>
void sap_half_fine(cudaStream_t st, const typename CT<R>::T* links, R diag, int L, int bs,
                   const typename CT<R>::T* inv, const typename CT<R>::T* f, typename CT<R>::T* x,
                   int color, int nrhs, const int* active, bool inv_transposed = false);
void blocks_to_fp32_transposed(cudaStream_t st, const double2* in, int nb, int bd, float2* out);
template <typename R>
void sap_half_coarse(cudaStream_t st, const typename CT<R>::T* stencil, int Ls, int d, int bs,
                     const typename CT<R>::T* inv, const typename CT<R>::T* f, typename CT<R>::T* x,
                     int color, int nrhs, const int* active);

// ---------------------------------------------------------------- transfer
// P layout: [aggregate][chirality 2][bsz = agg*agg*d/2][ntv]
template <typename R>
void restrict_op(cudaStream_t st, const typename CT<R>::T* P, int Ls, int d, int agg, int ntv,
                 const typename CT<R>::T* xf, typename CT<R>::T* xc, int nrhs, const int* active);
template <typename R>
void prolong_op(cudaStream_t st, const typename CT<R>::T* P, int Ls, int d, int agg, int ntv,
                const typename CT<R>::T* xc, typename CT<R>::T* xf, bool add, int nrhs,
                const int* active, void* xf16 = nullptr, int bf = 0);  // xf16: planar 16-bit copy of xf (d 16)
// gather test-vector blocks from V[m][n] into P layout
void gather_tv_blocks(cudaStream_t st, const double2* V, int Ls, int d, int agg, int ntv, double2* P);
// orthonormalise every (aggregate, chirality) block of P (bsz x ntv): QR with real positive diag
void orthonormalise_blocks(cudaStream_t st, double2* P, int nblocks, int bsz, int ntv, int* fail);
// Galerkin coarse stencil out[site][5][dc][dc] = P^H D_l P, D_l given by the prepared links
// (wilson, d = 2, diagonal diag) or by the level-l stencil A[site][5][d][d]
void galerkin(cudaStream_t st, const double2* A, bool wilson, double diag, int Ls, int d, int agg, int ntv,
              const double2* P, double2* out);

// ---------------------------------------------------------------- dense (coarsest)
void dense_from_stencil(cudaStream_t st, const double2* stencil, int Ls, int d, double2* A);
// batched in-place Gauss-Jordan inverse with partial pivoting (one CTA per matrix, bd <= 64), C = double2 / float2
template <typename C>
void invert_small_batched(cudaStream_t st, C* A, int nmat, int bd, int* fail);
// in-place inverse of one n x n matrix (large n), one cooperative kernel; work: invert_large_work_bytes(n);
// fail set on a zero pivot, timeout on an expired grid barrier; C = double2 / float2
size_t invert_large_work_bytes(int n);
// polls: poll limit of each grid-barrier wait (0 = default, about a second; < 0 = bounded-wait self-test:
// the barrier expects one arrival more than the grid has, so every wait runs out after -polls polls)
template <typename C>
void invert_large(cudaStream_t st, C* A, int n, int* piv, void* work, int* fail, int* timeout, long polls = 0);
template <typename R>
void dense_apply(cudaStream_t st, const typename CT<R>::T* A, int n, const typename CT<R>::T* x,
                 typename CT<R>::T* y, int nrhs, const int* active);
// sum_i A_ii, or with g5_dof > 0 sum_i gamma5_i A_ii (gamma5_i = -1 for dof i % g5_dof >= g5_dof / 2)
void trace_dense(cudaStream_t st, const double2* A, int n, double2* out, int g5_dof = 0);

// ---------------------------------------------------------------- BLAS-1 (per rhs)
template <typename C> void vzero(cudaStream_t st, C* x, long n, int nrhs);
template <typename Cd, typename Cs>
void vconvert(cudaStream_t st, const Cs* x, Cd* y, long n, int nrhs, const double* scale /*per rhs or null*/,
              const int* active);
// y = a * x + y  (a per rhs, double2 on device; sign: +1 or -1 multiplies a)
template <typename C>
void vaxpy(cudaStream_t st, const double2* a, double sign, const C* x, C* y, long n, int nrhs, const int* active);
// y = x * (1 / s[rhs]) where s is a double (norm)
template <typename C>
void vscale_inv(cudaStream_t st, const double* s, const C* x, C* y, long n, int nrhs, const int* active);
template <typename C> void vcopy(cudaStream_t st, const C* x, C* y, long n, int nrhs);
// x (FP64) += scale[rhs] * e (R)
template <typename R>
void vaccum_mixed(cudaStream_t st, const double* scale, const typename CT<R>::T* e, double2* x, long n,
                  int nrhs, const int* active);
// y = x - y  (FP64)
void vsub_from(cudaStream_t st, const double2* x, double2* y, long n, int nrhs);
// v[i] = sqrt(v[i])
void sqrt_inplace(cudaStream_t st, double* v, int n);

// reductions: out[rhs] (double / double2) on device; work = partial buffer
size_t reduce_work_bytes(long n, int nrhs, int nvec);
template <typename C>
void vnorm2(cudaStream_t st, const C* x, long n, int nrhs, double* out, void* work, const int* active);
template <typename C>
void vdot(cudaStream_t st, const C* x, const C* y, long n, int nrhs, double2* out, void* work, const int* active);
// h[i * nrhs + rhs] = V_i^H w for i < k; V_i = V + i * vstride
template <typename C>
void vmultidot(cudaStream_t st, const C* V, long vstride, int k, const C* w, long n, int nrhs, double2* h,
               void* work, const int* active);
// w -= sum_i h[i][rhs] V_i
template <typename C>
void vgs_update(cudaStream_t st, const C* V, long vstride, int k, const double2* h, C* w, long n, int nrhs,
                const int* active);
// the two classical Gram-Schmidt passes, each update fused with the reduction that follows it:
// w -= sum_i h[i][rhs] V_i, then h2[i][rhs] = V_i^H w   /   w -= sum_i h[i][rhs] V_i, then out[rhs] = ||w||^2
template <typename C>
void vgs_update_dot(cudaStream_t st, const C* V, long vstride, int k, const double2* h, C* w, long n, int nrhs,
                    double2* h2, void* work, const int* active);
template <typename C>
void vgs_update_norm(cudaStream_t st, const C* V, long vstride, int k, const double2* h, C* w, long n, int nrhs,
                     double* out, void* work, const int* active);
// x += sum_i y[i][rhs] Z_i
template <typename C>
void vcombine(cudaStream_t st, const C* Z, long zstride, int k, const double2* y, C* x, long n, int nrhs,
              const int* active);

// ---------------------------------------------------------------- RNG
void rademacher_fill(cudaStream_t st, uint64_t seed, int level, int phase, int64_t sample0, long n,
                     int nrhs, double2* out);
void complex_rademacher_fill(cudaStream_t st, uint64_t seed, int level, int phase, int64_t sample0, long n,
                             int nrhs, double2* out);
// isotropic noise of eq. random_props: kind MGMLMC_NOISE_RADEMACHER (real +-1) or MGMLMC_NOISE_Z4 (i^q)
void noise_fill(cudaStream_t st, int kind, uint64_t seed, int level, int phase, int64_t sample0, long n, int nrhs,
                double2* out);
// y <- gamma5 y (chirality-1 components negated; dof per site `dof`)
void gamma5_apply(cudaStream_t st, double2* y, int dof, long n, int nrhs);

// ---------------------------------------------------------------- Hutch++ (FP64)
constexpr int SK_MAXD = 64;  // largest sketch size d (deflation vectors per level difference)
// G = Y^H Y, Y = [d][n]; out d x d (row-major, G[i][j] = y_i^H y_j)
void gram(cudaStream_t st, const double2* Y, int d, long n, double2* G, void* work);
size_t gram_work_bytes(int d, long n);
// Cholesky G = R^H R, then Rinv = R^{-1} (upper); fail != 0 if not positive definite
void chol_inv_upper(cudaStream_t st, const double2* G, int d, double2* Rinv, int* fail);
// Y <- Y Rinv (in place, Rinv upper triangular)
void right_mul_upper(cudaStream_t st, double2* Y, int d, long n, const double2* Rinv);
// c[i][rhs] = Q_i^H x_rhs, Q = [d][n], x = [nrhs][n]
void proj_coeffs(cudaStream_t st, const double2* Q, int d, const double2* x, long n, int nrhs, double2* c,
                 void* work);
size_t proj_work_bytes(int d, long n, int nrhs);

// ---------------------------------------------------------------- tensor cores (coarse levels, d = 16)
// Pre-swizzled weight images of the real-embedded coarse operators, Re rows only, in TF32 (bf = 0, K in the
// interleaved Re/Im order of the FP32 vectors) or BF16 / FP16 (bf = 1 / 2, planar K: 16 Re then 16 Im parts per
// site): stencil [site][dir 5][16 x 32]; SAP block inverses of one colour [item][4][64 x 32].
// The 16-bit copy x16 of a coarse FP32 vector x ([rhs][site][16 complex]) is [rhs][site][16 Re | 16 Im] in the
// operand format, rounded to nearest even; the 2x2-block stencil reads it by TMA.
// coarse stencil y = D x (or y = b - D x) with 16-bit operands (bf 1 BF16, 2 FP16), one 2x2 block of sites per
// item: all blocks (bmode 0) or the blocks of colour `color` (bmode 1); W is the per-site weight image, x16 the
// 16-bit copy of x; y FP32 (y16 = 0) or, for bmode 1, the planar 16-bit form of y (y16 = 1)
void tc_block_stencil(cudaStream_t st, int bf, const void* W, int Ls, const void* x16, void* y, int y16,
                      const float2* b, int bmode, int color, int nrhs, const int* active, int* err, double bytes,
                      double flops);
// SAP block update x_B += inv_B r_B on the colour-`color` 2x2 blocks, rhs on the MMA M dimension: r16 the planar
// 16-bit residual tiles (tc_block_stencil with y16 = 1), Winv the colour's block-inverse image; x (FP32) and its
// 16-bit copy x16 are updated on the colour's sites
void tc_block_update(cudaStream_t st, int bf, const void* Winv, int Ls, const void* r16, float2* x, void* x16,
                     int color, int nrhs, const int* active, int* err, double bytes, double flops);
size_t tc_stencil_weight_bytes(int nsite, int bf);
size_t tc_blockinv_weight_bytes(int Ls, int bf);  // the blocks of one colour
void tc_stencil_weights(cudaStream_t st, const float2* st32, int nsite, void* W, int bf);
void tc_blockinv_weights(cudaStream_t st, const float2* inv32, int Ls, int color, void* W, int bf);
// true where the stencil launches for (bf, Ls, nrhs) take the 2x2-block kernel: their callers then pass x16
bool tc_block_selected(int bf, int Ls, int nrhs);
// x16 = the 16-bit copy of x (all rhs rows)
void tc_round16(cudaStream_t st, int bf, const float2* x, void* x16, int nsite, int nrhs);
// y = D x (b == nullptr) or y = b - D x, FP32 vectors, TF32, BF16 or FP16 products with FP32 accumulation;
// x16 (the 16-bit copy of x) is required where tc_block_selected, else unused
void tc_stencil_apply(cudaStream_t st, const void* W, int bf, int Ls, const float2* x, const void* x16, float2* y,
                      const float2* b, int nrhs, const int* active, int* err);
// res = f - D x on colour-0 block sites, 0 on colour-1 block sites (the residual right after a SAP sweep: it
// vanishes on the blocks solved last up to the rounding of the tensor-core products)
void tc_residual_after_sap(cudaStream_t st, const void* Wst, int bf, int Ls, const float2* x, const void* x16,
                           float2* res, const float2* f, int nrhs, const int* active, int* err);
// one SAP colour half sweep with 2x2-site blocks: res = f - D x on the colour's sites, x_B += inv_B res_B; where
// tc_block_selected, x16 is read by the residual and updated with x_B (res then holds the 16-bit residual)
void tc_sap_half(cudaStream_t st, const void* Wst, const void* Winv, int bf, int Ls, const float2* f, float2* x,
                 void* x16, float2* res, int color, int nrhs, const int* active, int* err);

// ---------------------------------------------------------------- launch-shape tuning table (tune.cu)
enum { TUNE_WILSON32 = 0, TUNE_TC0 = 1, TUNE_TC1 = 2 };
int tune_bucket(int nrhs);  // batch bucket: the power of two >= nrhs in 8..256
// variant of (kernel kind, lattice side, bucket of nrhs, weight format) or dflt when the table has none
int tune_lookup(int kind, int shape, int nrhs, int fmt, int dflt);
void tune_store(int kind, int shape, int bucket, int fmt, int variant, float us);
bool tune_known(int kind, int shape, int bucket, int fmt);
std::string tune_table_text();  // lines "device kind side bucket fmt variant microseconds"
void tune_clear();               // drops the entries of the current device

// ---------------------------------------------------------------- misc
void fill_int(cudaStream_t st, int* p, int v, int n);

}  // namespace mg
