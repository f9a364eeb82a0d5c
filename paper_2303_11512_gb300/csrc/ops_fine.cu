// Fine-level kernels: the Schwinger Wilson-Dirac stencil (multi-rhs), its
// SAP block matrices and the fine SAP smoother.
//
// Operator (Section 4, Schwinger discretisation, Wilson form):
//   (D x)(s) = (m0+2) x(s) + sum_mu [ (1-sigma_mu) W_mu(s) x(s+mu)
//                                    + (1+sigma_mu) conj(W_mu(s-mu)) x(s-mu) ]
// with W_mu(s) = -1/2 eta U_mu(s) the prepared link (eta = -1 on the t links
// of the last time slice: antiperiodic fermions).  (1 -+ sigma_mu) has rank 1,
// so each hop is one complex projection, one complex multiply by the link and
// a reconstruction of the lower spin:
//   (1 - sigma_1) x = h (1, -1),  h = x0 - x1
//   (1 + sigma_1) x = h (1,  1),  h = x0 + x1
//   (1 - sigma_2) x = h (1, -i),  h = x0 + i x1
//   (1 + sigma_2) x = h (1,  i),  h = x0 - i x1
#include "ops.cuh"

namespace mg {

__global__ void k_prepare_links(const double2* __restrict__ U, int L, double2* __restrict__ l64,
                                float2* __restrict__ l32) {
  const int V = L * L;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * V) return;
  int s = i >> 1, mu = i & 1;
  int t = s / L;
  double f = -0.5;
  if (mu == 1 && t == L - 1) f = 0.5;
  double2 u = U[i];
  double2 w = make_double2(f * u.x, f * u.y);
  l64[i] = w;
  if (l32) l32[i] = make_float2((float)w.x, (float)w.y);
}

// bad = 1 if some link is not a finite complex number
__global__ void k_check_links(const double2* __restrict__ U, long count, int* bad) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const double2 u = U[i];
    if (!isfinite(u.x) || !isfinite(u.y)) atomicExch(bad, 1);
  }
}
void check_links(cudaStream_t st, const double2* U, int L, int* bad) {
  MG_LAUNCH(k_check_links, cdiv(2L * L * L, 256), 256, 0, st, U, 2L * L * L, bad);
}

void prepare_links(cudaStream_t st, const double2* U, int L, double2* l64, float2* l32) {
  MG_LAUNCH(k_prepare_links, cdiv(2L * L * L, 256), 256, 0, st, U, L, l64, l32);
}

// ---- spinor loads ----------------------------------------------------------
__device__ __forceinline__ void ld_sp(const float2* __restrict__ p, long s, float2& a, float2& b) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p) + s);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_sp(const double2* __restrict__ p, long s, double2& a, double2& b) {
  a = __ldg(p + 2 * s);
  b = __ldg(p + 2 * s + 1);
}
__device__ __forceinline__ void st_sp(float2* p, long s, float2 a, float2 b) {
  reinterpret_cast<float4*>(p)[s] = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_sp(double2* p, long s, double2 a, double2 b) {
  p[2 * s] = a;
  p[2 * s + 1] = b;
}

// (D x)(s) for one site of one rhs (X points at that rhs).
template <typename R>
__device__ __forceinline__ void wilson_site(const typename CT<R>::T* __restrict__ lk, R diag, int L,
                                            const typename CT<R>::T* __restrict__ X, int s,
                                            typename CT<R>::T& o0, typename CT<R>::T& o1) {
  typedef typename CT<R>::T C;
  const int V = L * L;
  const int t = s / L, xx = s - t * L;
  const int sxp = s + (xx == L - 1 ? 1 - L : 1);
  const int sxm = s + (xx == 0 ? L - 1 : -1);
  const int stp = (t == L - 1) ? xx : s + L;
  const int stm = (t == 0) ? s + V - L : s - L;
  C a0, a1;
  ld_sp(X, s, a0, a1);
  o0 = cscale(a0, diag);
  o1 = cscale(a1, diag);
  {  // +x : (1 - sigma_1) W_0(s) x(s+x)
    ld_sp(X, sxp, a0, a1);
    C u = cmul(__ldg(lk + 2 * s), csub(a0, a1));
    o0 = cadd(o0, u);
    o1 = csub(o1, u);
  }
  {  // -x : (1 + sigma_1) conj(W_0(s-x)) x(s-x)
    ld_sp(X, sxm, a0, a1);
    C u = cmulc(__ldg(lk + 2 * sxm), cadd(a0, a1));
    o0 = cadd(o0, u);
    o1 = cadd(o1, u);
  }
  {  // +t : (1 - sigma_2) W_1(s) x(s+t)
    ld_sp(X, stp, a0, a1);
    C u = cmul(__ldg(lk + 2 * s + 1), cadd(a0, cmuli(a1)));
    o0 = cadd(o0, u);
    o1 = cadd(o1, cmulmi(u));
  }
  {  // -t : (1 + sigma_2) conj(W_1(s-t)) x(s-t)
    ld_sp(X, stm, a0, a1);
    C u = cmulc(__ldg(lk + 2 * stm + 1), cadd(a0, cmulmi(a1)));
    o0 = cadd(o0, u);
    o1 = cadd(o1, cmuli(u));
  }
}

// One thread per site and RPT right-hand sides (blockIdx.y * RPT + j): the RPT sites' neighbour loads are
// independent, so each thread keeps RPT times as many loads in flight (the tuner picks RPT per batch size).
template <typename R, bool RES, int RPT>
__global__ void __launch_bounds__(256) k_wilson(const typename CT<R>::T* __restrict__ lk, R diag, int L,
                                                const typename CT<R>::T* __restrict__ x,
                                                typename CT<R>::T* __restrict__ y,
                                                const typename CT<R>::T* __restrict__ b,
                                                const int* __restrict__ active, int nrhs) {
  typedef typename CT<R>::T C;
  const int V = L * L;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  C o0[RPT], o1[RPT];
  bool on[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) {
    const int rhs = blockIdx.y * RPT + j;
    on[j] = rhs < nrhs && !(active && !active[rhs]);
    if (on[j]) wilson_site<R>(lk, diag, L, x + (size_t)rhs * 2 * V, s, o0[j], o1[j]);
  }
#pragma unroll
  for (int j = 0; j < RPT; ++j) {
    if (!on[j]) continue;
    const size_t off = (size_t)(blockIdx.y * RPT + j) * 2 * V;
    if (RES) {
      C b0, b1;
      ld_sp(b + off, s, b0, b1);
      o0[j] = csub(b0, o0[j]);
      o1[j] = csub(b1, o1[j]);
    }
    st_sp(y + off, s, o0[j], o1[j]);
  }
}

template <typename R>
void wilson_apply(cudaStream_t st, const typename CT<R>::T* links, R diag, int L, const typename CT<R>::T* x,
                  typename CT<R>::T* y, const typename CT<R>::T* b, int nrhs, const int* active) {
  if (nrhs <= 0) return;
  const int rpt = sizeof(R) == 4 ? tune_lookup(TUNE_WILSON32, L, nrhs, 0, 1) : 1;
  dim3 grid(cdiv((long)L * L, 256), cdiv(nrhs, rpt));
  // algorithmic traffic: x read + y written once per site and rhs (+ b), links once per launch
  const double V = (double)L * L, sp = 2.0 * sizeof(typename CT<R>::T), ar = act_rhs(nrhs);
  const double bytes = ar * V * sp * (b ? 3 : 2) + V * sp;
  const double flops = ar * V * (b ? 56.0 : 52.0);
#define MG_WILSON_LAUNCH(RPT_)                                                                                  \
  do {                                                                                                          \
    if (b)                                                                                                      \
      MG_LAUNCH_W(bytes, flops, (k_wilson<R, true, RPT_>), grid, 256, 0, st, links, diag, L, x, y, b, active, nrhs); \
    else                                                                                                        \
      MG_LAUNCH_W(bytes, flops, (k_wilson<R, false, RPT_>), grid, 256, 0, st, links, diag, L, x, y, b, active, nrhs); \
  } while (0)
  if (rpt == 4)
    MG_WILSON_LAUNCH(4);
  else if (rpt == 2)
    MG_WILSON_LAUNCH(2);
  else
    MG_WILSON_LAUNCH(1);
#undef MG_WILSON_LAUNCH
}
template void wilson_apply<float>(cudaStream_t, const float2*, float, int, const float2*, float2*, const float2*,
                                  int, const int*);
template void wilson_apply<double>(cudaStream_t, const double2*, double, int, const double2*, double2*,
                                   const double2*, int, const int*);

// ---- SAP block matrices ------------------------------------------------------
// Block (BT, BX) of bs x bs sites; local dof index (jt * bs + jx) * 2 + spin.
// out[block][bd][bd], bd = 2 bs^2, blocks ordered BT slow, BX fast.
__global__ void k_fine_blocks(const double2* __restrict__ lk, double diag, int L, int bs, double2* __restrict__ out) {
  const int nbx = L / bs;
  const int blk = blockIdx.x;
  const int BT = blk / nbx, BX = blk % nbx;
  const int bd = 2 * bs * bs;
  double2* A = out + (size_t)blk * bd * bd;
  for (int e = threadIdx.x; e < bd * bd; e += blockDim.x) A[e] = make_double2(0, 0);
  __syncthreads();
  for (int j = threadIdx.x; j < bs * bs; j += blockDim.x) {
    const int jt = j / bs, jx = j % bs;
    const int t = BT * bs + jt, x = BX * bs + jx;
    const int s = t * L + x;
    A[(2 * j) * bd + 2 * j] = make_double2(diag, 0);
    A[(2 * j + 1) * bd + 2 * j + 1] = make_double2(diag, 0);
    // (row spin a, col spin b) coefficients of the four projectors
    if (jx + 1 < bs) {  // +x, link W_0(s)
      const int k = j + 1;
      double2 w = lk[2 * s];
      A[(2 * j) * bd + 2 * k] = w;
      A[(2 * j) * bd + 2 * k + 1] = cneg(w);
      A[(2 * j + 1) * bd + 2 * k] = cneg(w);
      A[(2 * j + 1) * bd + 2 * k + 1] = w;
    }
    if (jx > 0) {  // -x, conj(W_0(s-x))
      const int k = j - 1;
      double2 w = cconj(lk[2 * (s - 1)]);
      A[(2 * j) * bd + 2 * k] = w;
      A[(2 * j) * bd + 2 * k + 1] = w;
      A[(2 * j + 1) * bd + 2 * k] = w;
      A[(2 * j + 1) * bd + 2 * k + 1] = w;
    }
    if (jt + 1 < bs) {  // +t, W_1(s); (1 - sigma_2) = [[1, i], [-i, 1]]
      const int k = j + bs;
      double2 w = lk[2 * s + 1];
      A[(2 * j) * bd + 2 * k] = w;
      A[(2 * j) * bd + 2 * k + 1] = cmuli(w);
      A[(2 * j + 1) * bd + 2 * k] = cmulmi(w);
      A[(2 * j + 1) * bd + 2 * k + 1] = w;
    }
    if (jt > 0) {  // -t, conj(W_1(s-t)); (1 + sigma_2) = [[1, -i], [i, 1]]
      const int k = j - bs;
      double2 w = cconj(lk[2 * (s - L) + 1]);
      A[(2 * j) * bd + 2 * k] = w;
      A[(2 * j) * bd + 2 * k + 1] = cmulmi(w);
      A[(2 * j + 1) * bd + 2 * k] = cmuli(w);
      A[(2 * j + 1) * bd + 2 * k + 1] = w;
    }
  }
}

void fine_block_matrices(cudaStream_t st, const double2* l64, double diag, int L, int bs, double2* out) {
  const int nb = (L / bs) * (L / bs);
  MG_LAUNCH(k_fine_blocks, nb, 128, 0, st, l64, diag, L, bs, out);
}

// ---- SAP half sweep on the fine level ----------------------------------------
// One CTA per block of the colour; the block inverse is staged in shared memory
// once and applied to all right-hand sides in groups of G.
template <typename R, int BS, bool TRANS>
__global__ void __launch_bounds__(256) k_sap_fine(const typename CT<R>::T* __restrict__ lk, R diag, int L,
                                                  const typename CT<R>::T* __restrict__ inv,
                                                  const typename CT<R>::T* __restrict__ f,
                                                  typename CT<R>::T* __restrict__ x, int color, int nrhs,
                                                  const int* __restrict__ active) {
  typedef typename CT<R>::T C;
  constexpr int NS = BS * BS;      // sites per block
  constexpr int BD = 2 * NS;       // dof per block
  constexpr int G = 256 / NS;      // rhs per group (one thread per site and rhs in the residual phase)
  __shared__ C sinv[BD * BD];      // transposed: sinv[j * BD + i] = inv[i][j] (conflict-free over i)
  __shared__ C sres[G * BD];
  const int nbx = L / BS;
  const int half = nbx / 2;
  const int k = blockIdx.x;
  const int BT = k / half;
  const int BX = 2 * (k % half) + ((BT + color) & 1);
  const int blk = BT * nbx + BX;
  const C* I = inv + (size_t)blk * BD * BD;
  if (TRANS)  // stored transposed already: a straight, conflict-free copy
    for (int e = threadIdx.x; e < BD * BD; e += blockDim.x) sinv[e] = I[e];
  else
    for (int e = threadIdx.x; e < BD * BD; e += blockDim.x) sinv[(e % BD) * BD + e / BD] = I[e];
  const int V = L * L;
  const size_t n = 2 * (size_t)V;
  for (int r0 = 0; r0 < nrhs; r0 += G) {
    __syncthreads();
    // residual of the block sites
    for (int q = threadIdx.x; q < G * NS; q += blockDim.x) {
      const int g = q / NS, j = q % NS;
      const int rhs = r0 + g;
      if (rhs < nrhs && !(active && !active[rhs])) {
        const int s = (BT * BS + j / BS) * L + BX * BS + (j % BS);
        C o0, o1, f0, f1;
        wilson_site<R>(lk, diag, L, x + rhs * n, s, o0, o1);
        ld_sp(f + rhs * n, s, f0, f1);
        sres[g * BD + 2 * j] = csub(f0, o0);
        sres[g * BD + 2 * j + 1] = csub(f1, o1);
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < G * BD; q += blockDim.x) {
      const int g = q / BD, i = q % BD;
      const int rhs = r0 + g;
      if (rhs < nrhs && !(active && !active[rhs])) {
        C acc = czero<C>();
#pragma unroll 8
        for (int j = 0; j < BD; ++j) acc = cfma(sinv[j * BD + i], sres[g * BD + j], acc);
        const int js = i >> 1;
        const int s = (BT * BS + js / BS) * L + BX * BS + (js % BS);
        C* px = x + rhs * n + 2 * s + (i & 1);
        *px = cadd(*px, acc);
      }
    }
  }
}

template <typename R>
void sap_half_fine(cudaStream_t st, const typename CT<R>::T* links, R diag, int L, int bs,
                   const typename CT<R>::T* inv, const typename CT<R>::T* f, typename CT<R>::T* x, int color,
                   int nrhs, const int* active, bool inv_transposed) {
  MG_CHECK_ARG(bs == 4 || bs == 2, "fine SAP block side must be 2 or 4");
  const int nb = (L / bs) * (L / bs) / 2;
  // per block and rhs: x, f read and x written on the block (bd complex each); inverse once per block
  const double bd = 2.0 * bs * bs, cs = sizeof(typename CT<R>::T), ar = act_rhs(nrhs);
  const double bytes = nb * (ar * 3 * bd * cs + bd * bd * cs);
  const double flops = nb * ar * (bs * bs * 56.0 + 8.0 * bd * bd);
  if (bs == 4 && inv_transposed)
    MG_LAUNCH_W(bytes, flops, (k_sap_fine<R, 4, true>), nb, 256, 0, st, links, diag, L, inv, f, x, color, nrhs, active);
  else if (bs == 4)
    MG_LAUNCH_W(bytes, flops, (k_sap_fine<R, 4, false>), nb, 256, 0, st, links, diag, L, inv, f, x, color, nrhs,
                active);
  else if (inv_transposed)
    MG_LAUNCH_W(bytes, flops, (k_sap_fine<R, 2, true>), nb, 256, 0, st, links, diag, L, inv, f, x, color, nrhs, active);
  else
    MG_LAUNCH_W(bytes, flops, (k_sap_fine<R, 2, false>), nb, 256, 0, st, links, diag, L, inv, f, x, color, nrhs,
                active);
}
template void sap_half_fine<float>(cudaStream_t, const float2*, float, int, int, const float2*, const float2*,
                                   float2*, int, int, const int*, bool);
template void sap_half_fine<double>(cudaStream_t, const double2*, double, int, int, const double2*,
                                    const double2*, double2*, int, int, const int*, bool);

// out[b][j][i] = (float) in[b][i][j] for nb blocks of bd x bd
__global__ void k_blocks_to_fp32_transposed(const double2* __restrict__ in, int nb, int bd, float2* __restrict__ out) {
  const size_t total = (size_t)nb * bd * bd;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / ((size_t)bd * bd);
    const int r = (int)(e - b * bd * bd), i = r / bd, j = r - i * bd;
    const double2 v = in[e];
    out[b * bd * bd + (size_t)j * bd + i] = make_float2((float)v.x, (float)v.y);
  }
}

void blocks_to_fp32_transposed(cudaStream_t st, const double2* in, int nb, int bd, float2* out) {
  MG_LAUNCH(k_blocks_to_fp32_transposed, 1024, 256, 0, st, in, nb, bd, out);
}

}  // namespace mg
