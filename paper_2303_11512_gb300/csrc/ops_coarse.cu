// Coarse-level kernels: 5-point block stencil apply, SAP block matrices and
// smoother on coarse levels, aggregation restriction/prolongation (R = P^H,
// Section 3.1), the per-aggregate orthonormalisation of the test vectors and
// the Galerkin construction D_{l+1} = P_l^H D_l P_l, block by block.
//
// Stencil layout: st[site][dir][i][j], dir = 0 self, 1 +x, 2 -x, 3 +t, 4 -t;
// (D x)(s)_i = sum_dir sum_j st[s][dir][i][j] x(s + dir)_j, periodic (the
// fermion boundary sign is already inside the Galerkin blocks).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ops.cuh"

namespace mg {

__device__ __forceinline__ int nbr_site(int s, int dir, int Ls) {
  const int t = s / Ls, x = s - t * Ls;
  switch (dir) {
    case 1: return t * Ls + (x + 1 == Ls ? 0 : x + 1);
    case 2: return t * Ls + (x == 0 ? Ls - 1 : x - 1);
    case 3: return (t + 1 == Ls ? 0 : t + 1) * Ls + x;
    case 4: return (t == 0 ? Ls - 1 : t - 1) * Ls + x;
    default: return s;
  }
}

// ---- coarse stencil apply -----------------------------------------------------
// CTA per site: the 5 stencil blocks (transposed in shared memory) are applied to the
// rhs in groups of 256 / d; DT = d at compile time (0: runtime d).
template <typename R, bool RES, int DT>
__global__ void __launch_bounds__(256) k_coarse_apply(const typename CT<R>::T* __restrict__ st, int Ls, int d_,
                                                      const typename CT<R>::T* __restrict__ x,
                                                      typename CT<R>::T* __restrict__ y,
                                                      const typename CT<R>::T* __restrict__ b, int nrhs,
                                                      const int* __restrict__ active) {
  typedef typename CT<R>::T C;
  const int d = DT ? DT : d_;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sst = reinterpret_cast<C*>(smem_raw);  // [dir][j][i] (transposed)
  const int G = 256 / d;
  C* sx = sst + 5 * d * d;                  // [g][dir][j]
  const int s = blockIdx.x;
  const int dd = d * d;
  const C* S = st + (size_t)s * 5 * dd;
  for (int e = threadIdx.x; e < 5 * dd; e += 256) {
    const int dir = e / dd, r = e - dir * dd, i = r / d, j = r - i * d;
    sst[dir * dd + j * d + i] = S[e];
  }
  const size_t n = (size_t)Ls * Ls * d;
  const int g = threadIdx.x / d, i = threadIdx.x - g * d;
  for (int r0 = 0; r0 < nrhs; r0 += G) {
    __syncthreads();
    for (int q = threadIdx.x; q < G * 5 * d; q += 256) {
      const int gg = q / (5 * d), rem = q - gg * 5 * d, dir = rem / d, j = rem - dir * d;
      const int rhs = r0 + gg;
      if (rhs < nrhs && !(active && !active[rhs]))
        sx[q] = __ldg(x + rhs * n + (size_t)nbr_site(s, dir, Ls) * d + j);
    }
    __syncthreads();
    const int rhs = r0 + g;
    if (rhs < nrhs && !(active && !active[rhs])) {
      C acc = czero<C>();
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        const C* a = sst + dir * dd + i;
        const C* v = sx + (g * 5 + dir) * d;
#pragma unroll 16
        for (int j = 0; j < d; ++j) acc = cfma(a[j * d], v[j], acc);
      }
      const size_t o = rhs * n + (size_t)s * d + i;
      y[o] = RES ? csub(b[o], acc) : acc;
    }
  }
}

template <typename K>
static void set_smem_attr(K kernel) {
  ensure_max_smem((const void*)kernel, 200 * 1024);
}

template <typename R, bool RES>
static void coarse_apply_launch(cudaStream_t stm, const typename CT<R>::T* st, int Ls, int d,
                                const typename CT<R>::T* x, typename CT<R>::T* y, const typename CT<R>::T* b,
                                int nrhs, const int* active, size_t sm, double bytes, double flops) {
  if (d == 16) {
    set_smem_attr(k_coarse_apply<R, RES, 16>);
    MG_LAUNCH_W(bytes, flops, (k_coarse_apply<R, RES, 16>), Ls * Ls, 256, sm, stm, st, Ls, d, x, y, b, nrhs, active);
  } else {
    set_smem_attr(k_coarse_apply<R, RES, 0>);
    MG_LAUNCH_W(bytes, flops, (k_coarse_apply<R, RES, 0>), Ls * Ls, 256, sm, stm, st, Ls, d, x, y, b, nrhs, active);
  }
}

template <typename R>
void coarse_apply(cudaStream_t stm, const typename CT<R>::T* st, int Ls, int d, const typename CT<R>::T* x,
                  typename CT<R>::T* y, const typename CT<R>::T* b, int nrhs, const int* active) {
  typedef typename CT<R>::T C;
  MG_CHECK_ARG(d <= 64 && 256 % d == 0, "coarse dof must divide 256");
  const int G = 256 / d;
  size_t sm = sizeof(C) * (5 * d * d + G * 5 * d);
  const double ns = (double)Ls * Ls, cs = sizeof(C), ar = act_rhs(nrhs);
  const double bytes = ar * ns * d * cs * (b ? 3 : 2) + ns * 5.0 * d * d * cs;
  const double flops = ar * ns * 8.0 * 5.0 * d * d;
  if (b)
    coarse_apply_launch<R, true>(stm, st, Ls, d, x, y, b, nrhs, active, sm, bytes, flops);
  else
    coarse_apply_launch<R, false>(stm, st, Ls, d, x, y, b, nrhs, active, sm, bytes, flops);
}
template void coarse_apply<float>(cudaStream_t, const float2*, int, int, const float2*, float2*, const float2*,
                                  int, const int*);
template void coarse_apply<double>(cudaStream_t, const double2*, int, int, const double2*, double2*,
                                   const double2*, int, const int*);

// ---- SAP on coarse levels --------------------------------------------------------
// Block (BT, BX) of bs x bs sites, local index (jt * bs + jx) * d + k.
__global__ void k_coarse_blocks(const double2* __restrict__ st, int Ls, int d, int bs, double2* __restrict__ out) {
  const int nbx = Ls / bs;
  const int blk = blockIdx.x;
  const int BT = blk / nbx, BX = blk % nbx;
  const int ns = bs * bs, bd = ns * d, dd = d * d;
  double2* A = out + (size_t)blk * bd * bd;
  for (int e = threadIdx.x; e < bd * bd; e += blockDim.x) A[e] = make_double2(0, 0);
  __syncthreads();
  for (int j = 0; j < ns; ++j) {
    const int s = (BT * bs + j / bs) * Ls + BX * bs + j % bs;
    for (int dir = 0; dir < 5; ++dir) {
      const int nbs = nbr_site(s, dir, Ls);
      const int nt = nbs / Ls, nx = nbs % Ls;
      if (nt / bs != BT || nx / bs != BX) continue;
      const int jj = (nt % bs) * bs + nx % bs;
      const double2* S = st + ((size_t)s * 5 + dir) * dd;
      for (int e = threadIdx.x; e < dd; e += blockDim.x) {
        const int i = e / d, k = e % d;
        double2* a = A + (size_t)(j * d + i) * bd + jj * d + k;
        *a = cadd(*a, S[e]);
      }
      __syncthreads();
    }
  }
}

void coarse_block_matrices(cudaStream_t stm, const double2* st, int Ls, int d, int bs, double2* out) {
  const int nb = (Ls / bs) * (Ls / bs);
  MG_LAUNCH(k_coarse_blocks, nb, 256, 0, stm, st, Ls, d, bs, out);
}

template <typename R>
__global__ void __launch_bounds__(256) k_sap_coarse(const typename CT<R>::T* __restrict__ st, int Ls, int d, int bs,
                                                    const typename CT<R>::T* __restrict__ inv,
                                                    const typename CT<R>::T* __restrict__ f,
                                                    typename CT<R>::T* __restrict__ x, int color, int nrhs,
                                                    const int* __restrict__ active) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ns = bs * bs, bd = ns * d, dd = d * d;
  const int G = max(1, (int)blockDim.x / bd);
  C* sinv = reinterpret_cast<C*>(smem_raw);     // [bd][bd]
  C* sst = sinv + bd * bd;                      // [j][dir][k'][k] transposed stencil of block sites
  C* sres = sst + ns * 5 * dd;                  // [g][bd]
  const int nbx = Ls / bs, half = nbx / 2;
  const int kb = blockIdx.x;
  const int BT = kb / half;
  const int BX = 2 * (kb % half) + ((BT + color) & 1);
  const int blk = BT * nbx + BX;
  const C* I = inv + (size_t)blk * bd * bd;
  // transposed, sinv[j * bd + i] = inv[i][j]: threads of a warp differ in i
  for (int e = threadIdx.x; e < bd * bd; e += blockDim.x) sinv[(e % bd) * bd + e / bd] = I[e];
  for (int e = threadIdx.x; e < ns * 5 * dd; e += blockDim.x) {
    const int j = e / (5 * dd), r = e % (5 * dd), dir = r / dd, q = r % dd, i = q / d, k = q % d;
    const int s = (BT * bs + j / bs) * Ls + BX * bs + j % bs;
    sst[(j * 5 + dir) * dd + k * d + i] = st[((size_t)s * 5 + dir) * dd + q];
  }
  const size_t n = (size_t)Ls * Ls * d;
  for (int r0 = 0; r0 < nrhs; r0 += G) {
    __syncthreads();
    for (int q = threadIdx.x; q < G * bd; q += blockDim.x) {
      const int g = q / bd, i = q % bd, j = i / d, k = i % d;
      const int rhs = r0 + g;
      if (rhs < nrhs && !(active && !active[rhs])) {
        const int s = (BT * bs + j / bs) * Ls + BX * bs + j % bs;
        const C* X = x + rhs * n;
        C acc = __ldg(f + rhs * n + (size_t)s * d + k);
        for (int dir = 0; dir < 5; ++dir) {
          const C* xv = X + (size_t)nbr_site(s, dir, Ls) * d;
          const C* a = sst + (j * 5 + dir) * dd + k;
          for (int kk = 0; kk < d; ++kk) acc = csub(acc, cmul(a[kk * d], xv[kk]));
        }
        sres[g * bd + i] = acc;
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < G * bd; q += blockDim.x) {
      const int g = q / bd, i = q % bd, j = i / d, k = i % d;
      const int rhs = r0 + g;
      if (rhs < nrhs && !(active && !active[rhs])) {
        C acc = czero<C>();
        for (int jj = 0; jj < bd; ++jj) acc = cfma(sinv[jj * bd + i], sres[g * bd + jj], acc);
        const int s = (BT * bs + j / bs) * Ls + BX * bs + j % bs;
        C* px = x + rhs * n + (size_t)s * d + k;
        *px = cadd(*px, acc);
      }
    }
  }
}

template <typename R>
void sap_half_coarse(cudaStream_t stm, const typename CT<R>::T* st, int Ls, int d, int bs,
                     const typename CT<R>::T* inv, const typename CT<R>::T* f, typename CT<R>::T* x, int color,
                     int nrhs, const int* active) {
  typedef typename CT<R>::T C;
  const int ns = bs * bs, bd = ns * d;
  const int G = std::max(1, 256 / bd);
  size_t sm = sizeof(C) * ((size_t)bd * bd + (size_t)ns * 5 * d * d + (size_t)G * bd);
  MG_CHECK_ARG(sm <= 220 * 1024, "coarse SAP block too large for shared memory");
  ensure_max_smem((const void*)k_sap_coarse<R>, 220 * 1024);
  const int nb = (Ls / bs) * (Ls / bs) / 2;
  const double cs = sizeof(C), ar = act_rhs(nrhs);
  const double bytes = nb * (ar * 3.0 * bd * cs + ((double)bd * bd + ns * 5.0 * d * d) * cs);
  const double flops = nb * ar * (8.0 * bd * 5.0 * d + 8.0 * bd * bd);
  MG_LAUNCH_W(bytes, flops, k_sap_coarse<R>, nb, 256, sm, stm, st, Ls, d, bs, inv, f, x, color, nrhs, active);
}
template void sap_half_coarse<float>(cudaStream_t, const float2*, int, int, int, const float2*, const float2*,
                                     float2*, int, int, const int*);
template void sap_half_coarse<double>(cudaStream_t, const double2*, int, int, int, const double2*,
                                      const double2*, double2*, int, int, const int*);

// ---- restriction / prolongation ---------------------------------------------------
// Aggregate (T, X) of agg x agg sites; block of chirality c has rows
// j = js * hd + k' (js = jt * agg + jx local site, hd = d / 2 dof per chirality)
// mapping to fine dof (site(js)) * d + c * hd + k'.  One CTA per aggregate, its P blocks
// in shared memory, rhs in groups.  DT / AT / NT = d / agg / ntv at compile time (0: runtime).
template <typename R, int DT, int AT, int NT>
__global__ void __launch_bounds__(256) k_restrict(const typename CT<R>::T* __restrict__ P, int Ls, int d_, int agg_,
                                                  int ntv_, const typename CT<R>::T* __restrict__ xf,
                                                  typename CT<R>::T* __restrict__ xc, int nrhs,
                                                  const int* __restrict__ active) {
  typedef typename CT<R>::T C;
  const int d = DT ? DT : d_, agg = AT ? AT : agg_, ntv = NT ? NT : ntv_;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int hd = d / 2, na = agg * agg, bsz = na * hd, dc = 2 * ntv, fa = na * d;
  const int G = max(1, 256 / dc);
  C* sP = reinterpret_cast<C*>(smem_raw);  // [c][j][m]
  C* sx = sP + 2 * bsz * ntv;              // [g][js * d + k]
  const int Lc = Ls / agg;
  const int a = blockIdx.x, T = a / Lc, X = a - T * Lc;
  const C* Pa = P + (size_t)a * 2 * bsz * ntv;
  for (int e = threadIdx.x; e < 2 * bsz * ntv; e += 256) sP[e] = Pa[e];
  const size_t n = (size_t)Ls * Ls * d, nc = (size_t)Lc * Lc * dc;
  for (int r0 = 0; r0 < nrhs; r0 += G) {
    __syncthreads();
    for (int q = threadIdx.x; q < G * fa; q += 256) {
      const int g = q / fa, rem = q - g * fa, js = rem / d, k = rem - js * d;
      const int rhs = r0 + g;
      if (rhs < nrhs && !(active && !active[rhs])) {
        const int jt = js / agg, jx = js - jt * agg;
        const size_t site = (size_t)(agg * T + jt) * Ls + agg * X + jx;
        sx[q] = __ldg(xf + rhs * n + site * d + k);
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < G * dc; q += 256) {
      const int g = q / dc, o = q - g * dc, c = o / ntv, m = o - c * ntv;
      const int rhs = r0 + g;
      if (rhs < nrhs && !(active && !active[rhs])) {
        C acc = czero<C>();
        const C* pc = sP + (size_t)c * bsz * ntv + m;
        const C* xv = sx + g * fa + c * hd;
#pragma unroll 16
        for (int j = 0; j < bsz; ++j) {
          const int js = j / hd, kp = j - js * hd;
          acc = cfmac(pc[j * ntv], xv[js * d + kp], acc);
        }
        xc[rhs * nc + (size_t)a * dc + o] = acc;
      }
    }
  }
}

template <typename R, bool ADD, int DT, int AT, int NT>
__global__ void __launch_bounds__(256) k_prolong(const typename CT<R>::T* __restrict__ P, int Ls, int d_, int agg_,
                                                 int ntv_, const typename CT<R>::T* __restrict__ xc,
                                                 typename CT<R>::T* __restrict__ xf,
                                                 unsigned short* __restrict__ xf16, int bf, int nrhs,
                                                 const int* __restrict__ active) {
  typedef typename CT<R>::T C;
  const int d = DT ? DT : d_, agg = AT ? AT : agg_, ntv = NT ? NT : ntv_;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int hd = d / 2, na = agg * agg, bsz = na * hd, dc = 2 * ntv, fa = na * d;
  const int G = max(1, 256 / fa);
  C* sP = reinterpret_cast<C*>(smem_raw);  // [c][m][j] (transposed)
  C* sc = sP + 2 * bsz * ntv;              // [g][dc]
  const int Lc = Ls / agg;
  const int a = blockIdx.x, T = a / Lc, X = a - T * Lc;
  const C* Pa = P + (size_t)a * 2 * bsz * ntv;
  for (int e = threadIdx.x; e < 2 * bsz * ntv; e += 256) {
    const int c = e / (bsz * ntv), r = e - c * bsz * ntv, j = r / ntv, m = r - j * ntv;
    sP[(c * ntv + m) * bsz + j] = Pa[e];
  }
  const size_t n = (size_t)Ls * Ls * d, nc = (size_t)Lc * Lc * dc;
  for (int r0 = 0; r0 < nrhs; r0 += G) {
    __syncthreads();
    for (int q = threadIdx.x; q < G * dc; q += 256) {
      const int g = q / dc, o = q - g * dc;
      const int rhs = r0 + g;
      if (rhs < nrhs && !(active && !active[rhs])) sc[q] = __ldg(xc + rhs * nc + (size_t)a * dc + o);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < G * fa; q += 256) {
      const int g = q / fa, rem = q - g * fa, js = rem / d, k = rem - js * d;
      const int rhs = r0 + g;
      if (rhs < nrhs && !(active && !active[rhs])) {
        const int c = k / hd, kp = k - c * hd, j = js * hd + kp;
        C acc = czero<C>();
        const C* pc = sP + (size_t)c * ntv * bsz + j;
        const C* cv = sc + g * dc + c * ntv;
#pragma unroll 8
        for (int m = 0; m < ntv; ++m) acc = cfma(pc[m * bsz], cv[m], acc);
        const int jt = js / agg, jx = js - jt * agg;
        const size_t site = (size_t)(agg * T + jt) * Ls + agg * X + jx;
        C* p = xf + rhs * n + site * d + k;
        const C v = ADD ? cadd(*p, acc) : acc;
        *p = v;
        if constexpr (sizeof(R) == 4) {
          if (xf16) {  // planar 16-bit copy of an FP32 coarse vector: Re parts of the site's d dofs, then Im
            unsigned short* p16 = xf16 + 2 * (rhs * n + site * d) + k;
            p16[0] = bf == 2 ? __half_as_ushort(__float2half_rn(v.x)) : __bfloat16_as_ushort(__float2bfloat16_rn(v.x));
            p16[d] = bf == 2 ? __half_as_ushort(__float2half_rn(v.y)) : __bfloat16_as_ushort(__float2bfloat16_rn(v.y));
          }
        }
      }
    }
  }
}

// compile-time shapes of the default hierarchy (agg 4, ntv 8: fine d = 2, coarse d = 16)
enum { SHAPE_GENERIC = 0, SHAPE_FINE = 1, SHAPE_COARSE = 2 };
static int transfer_shape(int d, int agg, int ntv) {
  if (agg == 4 && ntv == 8 && d == 2) return SHAPE_FINE;
  if (agg == 4 && ntv == 8 && d == 16) return SHAPE_COARSE;
  return SHAPE_GENERIC;
}

template <typename R>
void restrict_op(cudaStream_t stm, const typename CT<R>::T* P, int Ls, int d, int agg, int ntv,
                 const typename CT<R>::T* xf, typename CT<R>::T* xc, int nrhs, const int* active) {
  typedef typename CT<R>::T C;
  const int na = agg * agg, bsz = na * d / 2, dc = 2 * ntv;
  const int G = std::max(1, 256 / dc);
  size_t sm = sizeof(C) * ((size_t)2 * bsz * ntv + (size_t)G * na * d);
  const int Lc = Ls / agg;
  const double nag = (double)Lc * Lc, cs = sizeof(C), ar = act_rhs(nrhs);
  const double bytes = nag * (ar * (na * d + dc) * cs + 2.0 * bsz * ntv * cs);
  const double flops = nag * ar * 8.0 * 2.0 * bsz * ntv;
  switch (transfer_shape(d, agg, ntv)) {
    case SHAPE_FINE:
      set_smem_attr(k_restrict<R, 2, 4, 8>);
      MG_LAUNCH_W(bytes, flops, (k_restrict<R, 2, 4, 8>), Lc * Lc, 256, sm, stm, P, Ls, d, agg, ntv, xf, xc, nrhs,
                  active);
      break;
    case SHAPE_COARSE:
      set_smem_attr(k_restrict<R, 16, 4, 8>);
      MG_LAUNCH_W(bytes, flops, (k_restrict<R, 16, 4, 8>), Lc * Lc, 256, sm, stm, P, Ls, d, agg, ntv, xf, xc, nrhs,
                  active);
      break;
    default:
      set_smem_attr(k_restrict<R, 0, 0, 0>);
      MG_LAUNCH_W(bytes, flops, (k_restrict<R, 0, 0, 0>), Lc * Lc, 256, sm, stm, P, Ls, d, agg, ntv, xf, xc, nrhs,
                  active);
  }
}

template <typename R, bool ADD>
static void prolong_launch(cudaStream_t stm, const typename CT<R>::T* P, int Ls, int d, int agg, int ntv,
                           const typename CT<R>::T* xc, typename CT<R>::T* xf, unsigned short* xf16, int bf,
                           int nrhs, const int* active, size_t sm, double bytes, double flops) {
  const int Lc = Ls / agg;
  switch (transfer_shape(d, agg, ntv)) {
    case SHAPE_FINE:
      set_smem_attr(k_prolong<R, ADD, 2, 4, 8>);
      MG_LAUNCH_W(bytes, flops, (k_prolong<R, ADD, 2, 4, 8>), Lc * Lc, 256, sm, stm, P, Ls, d, agg, ntv, xc, xf,
                  xf16, bf, nrhs, active);
      break;
    case SHAPE_COARSE:
      set_smem_attr(k_prolong<R, ADD, 16, 4, 8>);
      MG_LAUNCH_W(bytes, flops, (k_prolong<R, ADD, 16, 4, 8>), Lc * Lc, 256, sm, stm, P, Ls, d, agg, ntv, xc, xf,
                  xf16, bf, nrhs, active);
      break;
    default:
      set_smem_attr(k_prolong<R, ADD, 0, 0, 0>);
      MG_LAUNCH_W(bytes, flops, (k_prolong<R, ADD, 0, 0, 0>), Lc * Lc, 256, sm, stm, P, Ls, d, agg, ntv, xc, xf,
                  xf16, bf, nrhs, active);
  }
}

template <typename R>
void prolong_op(cudaStream_t stm, const typename CT<R>::T* P, int Ls, int d, int agg, int ntv,
                const typename CT<R>::T* xc, typename CT<R>::T* xf, bool add, int nrhs, const int* active,
                void* xf16, int bf) {
  MG_CHECK_ARG(!xf16 || (sizeof(R) == 4 && (bf == 1 || bf == 2)), "16-bit copy: FP32 vectors, BF16 or FP16");
  typedef typename CT<R>::T C;
  const int na = agg * agg, bsz = na * d / 2, dc = 2 * ntv, fa = na * d;
  const int G = std::max(1, 256 / fa);
  size_t sm = sizeof(C) * ((size_t)2 * bsz * ntv + (size_t)G * dc);
  const int Lc = Ls / agg;
  const double nag = (double)Lc * Lc, cs = sizeof(C), ar = act_rhs(nrhs);
  const double bytes = nag * (ar * ((add ? 2.0 : 1.0) * fa + dc) * cs + 2.0 * bsz * ntv * cs) +
                       (xf16 ? nag * ar * fa * 4.0 : 0.0);
  const double flops = nag * ar * 8.0 * 2.0 * bsz * ntv;
  unsigned short* x16 = (unsigned short*)xf16;
  if (add)
    prolong_launch<R, true>(stm, P, Ls, d, agg, ntv, xc, xf, x16, bf, nrhs, active, sm, bytes, flops);
  else
    prolong_launch<R, false>(stm, P, Ls, d, agg, ntv, xc, xf, x16, bf, nrhs, active, sm, bytes, flops);
}
template void restrict_op<float>(cudaStream_t, const float2*, int, int, int, int, const float2*, float2*, int,
                                 const int*);
template void restrict_op<double>(cudaStream_t, const double2*, int, int, int, int, const double2*, double2*, int,
                                  const int*);
template void prolong_op<float>(cudaStream_t, const float2*, int, int, int, int, const float2*, float2*, bool, int,
                                const int*, void*, int);
template void prolong_op<double>(cudaStream_t, const double2*, int, int, int, int, const double2*, double2*, bool,
                                 int, const int*, void*, int);

// ---- test vectors -> prolongator blocks --------------------------------------------
__global__ void k_gather_tv(const double2* __restrict__ V, int Ls, int d, int agg, int ntv, double2* __restrict__ P) {
  const int hd = d / 2, na = agg * agg, bsz = na * hd;
  const int Lc = Ls / agg;
  const size_t total = (size_t)Lc * Lc * 2 * bsz * ntv;
  const size_t n = (size_t)Ls * Ls * d;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int m = e % ntv;
    const size_t r = e / ntv;
    const int j = r % bsz;
    const size_t r2 = r / bsz;
    const int c = r2 % 2;
    const int a = (int)(r2 / 2), T = a / Lc, X = a % Lc;
    const int js = j / hd, kp = j % hd;
    const size_t site = (size_t)(agg * T + js / agg) * Ls + agg * X + js % agg;
    P[e] = V[m * n + site * d + c * hd + kp];
  }
}

void gather_tv_blocks(cudaStream_t stm, const double2* V, int Ls, int d, int agg, int ntv, double2* P) {
  MG_LAUNCH(k_gather_tv, 1024, 256, 0, stm, V, Ls, d, agg, ntv, P);
}

// Modified Gram-Schmidt with one re-orthogonalisation pass, one warp per block:
// Q has orthonormal columns and R a real positive diagonal (the QR normalisation
// of the oracle), FP64.
__global__ void k_orthonormalise(double2* __restrict__ P, int nblocks, int bsz, int ntv, int* fail) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (w >= nblocks) return;
  double2* B = P + (size_t)w * bsz * ntv;  // B[j][m]
  for (int m = 0; m < ntv; ++m) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = 0; i < m; ++i) {
        double2 acc = make_double2(0, 0);
        for (int j = lane; j < bsz; j += 32) acc = cfmac(B[j * ntv + i], B[j * ntv + m], acc);
        for (int o = 16; o; o >>= 1) {
          acc.x += __shfl_xor_sync(0xffffffff, acc.x, o);
          acc.y += __shfl_xor_sync(0xffffffff, acc.y, o);
        }
        for (int j = lane; j < bsz; j += 32) B[j * ntv + m] = csub(B[j * ntv + m], cmul(B[j * ntv + i], acc));
        __syncwarp();
      }
    }
    double nr = 0;
    for (int j = lane; j < bsz; j += 32) {
      double2 v = B[j * ntv + m];
      nr += v.x * v.x + v.y * v.y;
    }
    for (int o = 16; o; o >>= 1) nr += __shfl_xor_sync(0xffffffff, nr, o);
    if (!(nr > 0.0)) {
      if (lane == 0) atomicExch(fail, 1);
      return;
    }
    const double inv = 1.0 / sqrt(nr);
    for (int j = lane; j < bsz; j += 32) B[j * ntv + m] = cscale(B[j * ntv + m], inv);
    __syncwarp();
  }
}

void orthonormalise_blocks(cudaStream_t stm, double2* P, int nblocks, int bsz, int ntv, int* fail) {
  MG_LAUNCH(k_orthonormalise, cdiv(nblocks, 4), 128, 0, stm, P, nblocks, bsz, ntv, fail);
}

// ---- Galerkin coarse operator ------------------------------------------------------
// D_{l+1} = P^H D_l P (Section 3.1), one CTA per coarse site B, block by block: for every fine
// site s of aggregate B and stencil direction f, with s' the f-neighbour of s,
//   D_{l+1}[B, f or self] += P(s)^H D_l(s, f) P(s'),
// where P(s) (d x dc) is block diagonal in chirality and s' lies in B itself or in the aggregate
// adjacent to B in direction f (a fine hop crosses only the aggregate face it points to).
__device__ __forceinline__ void wilson_hop(const double2* __restrict__ lk, double diag, int L, int s, int f,
                                           double2* M) {
  double2 w;
  switch (f) {
    case 0:
      M[0] = make_double2(diag, 0); M[1] = make_double2(0, 0);
      M[2] = make_double2(0, 0); M[3] = make_double2(diag, 0);
      return;
    case 1:  // +x: (1 - sigma_1) W_0(s)
      w = lk[2 * s];
      M[0] = w; M[1] = cneg(w); M[2] = cneg(w); M[3] = w;
      return;
    case 2:  // -x: (1 + sigma_1) conj(W_0(s - x))
      w = cconj(lk[2 * nbr_site(s, 2, L)]);
      M[0] = w; M[1] = w; M[2] = w; M[3] = w;
      return;
    case 3:  // +t: (1 - sigma_2) W_1(s)
      w = lk[2 * s + 1];
      M[0] = w; M[1] = cmuli(w); M[2] = cmulmi(w); M[3] = w;
      return;
    default:  // -t: (1 + sigma_2) conj(W_1(s - t))
      w = cconj(lk[2 * nbr_site(s, 4, L) + 1]);
      M[0] = w; M[1] = cmulmi(w); M[2] = cmuli(w); M[3] = w;
      return;
  }
}

constexpr int GAL_T = 256;   // threads per coarse site
constexpr int GAL_E = 4;     // coarse block entries per thread (dc <= 32)

template <bool WILSON>
__global__ void __launch_bounds__(GAL_T) k_galerkin(const double2* __restrict__ A, double diag, int Ls, int d,
                                                    int agg, int ntv, const double2* __restrict__ P,
                                                    double2* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int hd = d / 2, na = agg * agg, bsz = na * hd, dc = 2 * ntv, Lc = Ls / agg;
  const int dd = d * d, ddc = d * dc, dcc = dc * dc;
  double2* sA = reinterpret_cast<double2*>(smem_raw);  // [f][r][k]   D_l(s, f)
  double2* sT = sA + 5 * dd;                            // [f][r][j]   D_l(s, f) P(s'_f)
  __shared__ int s_nb[5], s_js[5];                      // aggregate and local site of s'_f
  const int B = blockIdx.x, BT = B / Lc, BX = B % Lc;
  const size_t pblk = (size_t)2 * bsz * ntv;
  const double2* PB = P + (size_t)B * pblk;
  double2 acc[5][GAL_E];
#pragma unroll
  for (int c = 0; c < 5; ++c)
#pragma unroll
    for (int q = 0; q < GAL_E; ++q) acc[c][q] = make_double2(0, 0);
  for (int js = 0; js < na; ++js) {
    const int s = (BT * agg + js / agg) * Ls + BX * agg + js % agg;
    bool inside[5];  // s'_f in B: the f contribution goes to the self block
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const int s2 = nbr_site(s, f, Ls), t2 = s2 / Ls, x2 = s2 % Ls;
      inside[f] = (t2 / agg) * Lc + x2 / agg == B;
    }
    __syncthreads();  // the previous site's sA / sT / s_nb / s_js are consumed
    if (threadIdx.x < 5) {
      const int s2 = nbr_site(s, threadIdx.x, Ls), t2 = s2 / Ls, x2 = s2 % Ls;
      s_nb[threadIdx.x] = (t2 / agg) * Lc + x2 / agg;
      s_js[threadIdx.x] = (t2 % agg) * agg + x2 % agg;
    }
    if (WILSON) {
      if (threadIdx.x < 5) wilson_hop(A, diag, Ls, s, threadIdx.x, sA + threadIdx.x * 4);
    } else {
      const double2* As = A + (size_t)s * 5 * dd;
      for (int e = threadIdx.x; e < 5 * dd; e += GAL_T) sA[e] = __ldg(As + e);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 5 * ddc; e += GAL_T) {
      const int f = e / ddc, rem = e % ddc, r = rem / dc, j = rem % dc, cj = j / ntv, m = j % ntv;
      const double2* p = P + (size_t)s_nb[f] * pblk + ((size_t)cj * bsz + s_js[f] * hd) * ntv + m;
      const double2* a = sA + f * dd + r * d + cj * hd;
      double2 t = make_double2(0, 0);
      for (int k = 0; k < hd; ++k) t = cfma(a[k], __ldg(p + (size_t)k * ntv), t);
      sT[e] = t;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GAL_E; ++q) {
      const int e = threadIdx.x + q * GAL_T;
      if (e < dcc) {
        const int i = e / dc, j = e % dc, ci = i / ntv, mi = i % ntv;
        const double2* p = PB + ((size_t)ci * bsz + js * hd) * ntv + mi;
#pragma unroll
        for (int f = 0; f < 5; ++f) {
          const double2* t = sT + f * ddc + (ci * hd) * dc + j;
          double2 v = make_double2(0, 0);
          for (int k = 0; k < hd; ++k) v = cfmac(__ldg(p + (size_t)k * ntv), t[k * dc], v);
          if (inside[f])
            acc[0][q] = cadd(acc[0][q], v);
          else
            acc[f][q] = cadd(acc[f][q], v);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < GAL_E; ++q) {
    const int e = threadIdx.x + q * GAL_T;
    if (e < dcc)
#pragma unroll
      for (int c = 0; c < 5; ++c) out[((size_t)B * 5 + c) * dcc + e] = acc[c][q];
  }
}

void galerkin(cudaStream_t stm, const double2* A, bool wilson, double diag, int Ls, int d, int agg, int ntv,
              const double2* P, double2* out) {
  const int dc = 2 * ntv, Lc = Ls / agg;
  MG_CHECK_ARG(dc * dc <= GAL_E * GAL_T && d % 2 == 0 && (!wilson || d == 2), "Galerkin block sizes");
  const size_t sm = sizeof(double2) * 5 * ((size_t)d * d + (size_t)d * dc);
  MG_CHECK_ARG(sm <= 200 * 1024, "Galerkin blocks too large for shared memory");
  const double na = agg * agg, hd = d / 2;
  const double flops = (double)Lc * Lc * na * 5.0 * 8.0 * hd * ((double)d * dc + (double)dc * dc);
  const double bytes = (double)Lc * Lc * (na * (wilson ? 32.0 : 5.0 * d * d * 16.0) + 5.0 * dc * dc * 16.0 +
                                          2.0 * na * hd * ntv * 16.0);
  if (wilson) {
    ensure_max_smem((const void*)k_galerkin<true>, 200 * 1024);
    MG_LAUNCH_W(bytes, flops, k_galerkin<true>, Lc * Lc, GAL_T, sm, stm, A, diag, Ls, d, agg, ntv, P, out);
  } else {
    ensure_max_smem((const void*)k_galerkin<false>, 200 * 1024);
    MG_LAUNCH_W(bytes, flops, k_galerkin<false>, Lc * Lc, GAL_T, sm, stm, A, diag, Ls, d, agg, ntv, P, out);
  }
}

// ---- coarsest level as a dense matrix -------------------------------------------------
__global__ void k_dense_from_stencil(const double2* __restrict__ st, int Ls, int d, double2* __restrict__ A) {
  const int nsite = Ls * Ls;
  const size_t N = (size_t)nsite * d;
  const size_t total = (size_t)nsite * d * d;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = e % d, i = (e / d) % d, s = (int)(e / ((size_t)d * d));
    for (int dir = 0; dir < 5; ++dir) {
      const int nb = nbr_site(s, dir, Ls);
      double2* a = A + ((size_t)s * d + i) * N + (size_t)nb * d + j;
      *a = cadd(*a, st[((size_t)s * 5 + dir) * d * d + i * d + j]);
    }
  }
}

void dense_from_stencil(cudaStream_t stm, const double2* st, int Ls, int d, double2* A) {
  const size_t N = (size_t)Ls * Ls * d;
  MG_CUDA(cudaMemsetAsync(A, 0, N * N * sizeof(double2), stm));
  // one thread per (site, i, j): the five neighbour columns are distinct for Ls >= 3
  MG_LAUNCH(k_dense_from_stencil, 512, 256, 0, stm, st, Ls, d, A);
}

}  // namespace mg
