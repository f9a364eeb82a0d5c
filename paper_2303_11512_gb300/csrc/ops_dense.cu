// Dense FP64 kernels: Gauss-Jordan inverses (SAP blocks, the coarsest level of
// Algorithm 2 whose trace is tau_L), the coarsest-level inverse apply, and the
// Hutch++ pieces of Algorithm 2: the Gram matrix and Cholesky factor of
// CholeskyQR2 and the projection coefficients Q^H x.
#include "ops.cuh"

namespace mg {

namespace {
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
  return v;
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double cabs2(float2 a) { return (double)a.x * a.x + (double)a.y * a.y; }
__device__ __forceinline__ double2 crecip(double2 a) {
  const double s = 1.0 / cabs2(a);
  return make_double2(a.x * s, -a.y * s);
}
__device__ __forceinline__ float2 crecip(float2 a) {
  const float s = 1.0f / (a.x * a.x + a.y * a.y);
  return make_float2(a.x * s, -a.y * s);
}
}  // namespace

// ---- batched small inverse (one CTA per matrix) ------------------------------------------------
// Gauss-Jordan with partial pivoting in shared memory, three barriers per column: pivot search (warp 0, also
// the reciprocal of the pivot), then the row swap, pivot-row scaling and multipliers (read all, barrier,
// write all), then the rank-1 elimination.  BD = block dimension at compile time (0: runtime bd).
template <typename C, int BD>
__global__ void __launch_bounds__(256) k_invert_small(C* __restrict__ Ag, int bd_, int* fail) {
  const int bd = BD ? BD : bd_;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);
  C* sf = A + bd * bd;
  int* perm = reinterpret_cast<int*>(sf + bd);
  __shared__ int s_p;
  __shared__ int s_bad;
  __shared__ C s_a;
  C* G = Ag + (size_t)blockIdx.x * bd * bd;
  for (int e = threadIdx.x; e < bd * bd; e += 256) A[e] = G[e];
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int k = 0; k < bd; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + threadIdx.x; i < bd; i += 32) {
        double v = cabs2(A[i * bd + k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffff, best, o);
        int oi = __shfl_xor_sync(0xffffffff, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        s_p = bi;
        perm[k] = bi;
        if (!(best > 0.0)) s_bad = 1;
        s_a = best > 0.0 ? crecip(A[bi * bd + k]) : czero<C>();
      }
    }
    __syncthreads();
    if (s_bad) break;
    const int p = s_p;
    const C a = s_a;
    // swap rows k and p, scale the pivot row, multipliers of the swapped column k
    C tk, tp, ck, akk;
    const int t = threadIdx.x;
    if (t < bd) {
      tk = A[k * bd + t];
      tp = A[p * bd + t];
      ck = A[t * bd + k];
      akk = A[k * bd + k];
    }
    __syncthreads();
    if (t < bd) {
      if (p != k) A[p * bd + t] = tk;
      A[k * bd + t] = (t == k) ? a : cmul(tp, a);
      sf[t] = (t == k) ? czero<C>() : (t == p ? akk : ck);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < bd * bd; e += 256) {
      const int i = e / bd, j = e - i * bd;
      if (i != k) A[e] = csub(j == k ? czero<C>() : A[e], cmul(sf[i], A[k * bd + j]));
    }
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) atomicExch(fail, 1);
    return;
  }
  for (int k = bd - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = threadIdx.x; i < bd; i += 256) {
        C t = A[i * bd + k];
        A[i * bd + k] = A[i * bd + p];
        A[i * bd + p] = t;
      }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < bd * bd; e += 256) G[e] = A[e];
}

template <typename C>
void invert_small_batched(cudaStream_t st, C* A, int nmat, int bd, int* fail) {
  MG_CHECK_ARG(bd <= 64, "small inverse limited to 64 x 64");
  size_t sm = sizeof(C) * ((size_t)bd * bd + bd) + sizeof(int) * bd + 16;
  auto attr = [&](auto kern, int) { ensure_max_smem((const void*)kern, 100 * 1024); };
  if (bd == 64) {
    attr(k_invert_small<C, 64>, 0);
    MG_LAUNCH((k_invert_small<C, 64>), nmat, 256, sm, st, A, bd, fail);
  } else if (bd == 32) {
    attr(k_invert_small<C, 32>, 1);
    MG_LAUNCH((k_invert_small<C, 32>), nmat, 256, sm, st, A, bd, fail);
  } else {
    attr(k_invert_small<C, 0>, 2);
    MG_LAUNCH((k_invert_small<C, 0>), nmat, 256, sm, st, A, bd, fail);
  }
}
template void invert_small_batched<double2>(cudaStream_t, double2*, int, int, int*);
template void invert_small_batched<float2>(cudaStream_t, float2*, int, int, int*);

// ---- large in-place inverse: Gauss-Jordan with partial pivoting in one cooperative kernel ------------
// The CTAs of the grid (all resident, cooperative launch) sweep the columns in step: per column k the pivot
// p = argmax_{i >= k} |A_ik| (ties: smallest i) comes from per-CTA partial maxima, rows k and p are swapped,
// the pivot row is scaled by a = 1 / A_pk (its column-k entry becomes a) and every other row i loses
// f_i x (pivot row), its column-k entry becoming -f_i a.  Column k reads one matrix buffer and writes the
// other (ping-pong), so every CTA can read the pivot row and column while others already write: one grid
// barrier per column.  The barrier spins on a generation counter with an iteration limit (timeout flag, all
// CTAs then leave).  Columns are unscrambled afterwards by the recorded swaps in reverse order.
constexpr int GJ_T = 512;
constexpr long GJ_SPIN = 1L << 28;  // default polls of the generation counter (well over a second)

// `expect` arrivals release the barrier (the grid size; one more in the bounded-wait self-test, where nothing
// releases it and every wait runs out after `polls` polls)
__device__ __forceinline__ bool gj_barrier(unsigned* bar, unsigned expect, long polls, int* timeout, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == expect - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long it = 0;
      while (*gen == g) {
        if (++it > polls) {
          atomicExch(timeout, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    *s_ok = ok && !*(volatile int*)timeout;
  }
  __syncthreads();
  return *s_ok;
}

// block-wide argmax (value, smallest index on ties), result in thread 0
__device__ __forceinline__ void gj_block_argmax(double& best, int& idx, double* sb, int* si) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffff, best, o);
    const int oi = __shfl_xor_sync(0xffffffff, idx, o);
    if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sb[w] = best; si[w] = idx; }
  __syncthreads();
  if (w == 0) {
    best = l < GJ_T / 32 ? sb[l] : -1.0;
    idx = l < GJ_T / 32 ? si[l] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffff, best, o);
      const int oi = __shfl_xor_sync(0xffffffff, idx, o);
      if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
    }
  }
}

// A0: the matrix (result written back here); A1: scratch of the same size; slots: per-CTA (max, index)
// of the next pivot column, double-buffered by column parity
template <typename C>
__global__ void __launch_bounds__(GJ_T, 1) k_gj_coop(C* __restrict__ A0, C* __restrict__ A1, int n,
                                                    int* __restrict__ piv, double* __restrict__ slot_v,
                                                    int* __restrict__ slot_i, unsigned* bar, int* fail,
                                                    int* timeout, long polls, unsigned expect) {
  __shared__ double sb[GJ_T / 32];
  __shared__ int si[GJ_T / 32];
  __shared__ int s_ok, s_p;
  __shared__ C s_a;
  extern __shared__ __align__(16) unsigned char gj_smem[];
  C* s_row = reinterpret_cast<C*>(gj_smem);  // the scaled pivot row of the current column
  const unsigned nb = gridDim.x;
  // column 0 partial maxima into slot set 0
  {
    double best = -1.0;
    int idx = 0x7fffffff;
    for (int i = blockIdx.x * GJ_T + threadIdx.x; i < n; i += nb * GJ_T) {
      const double v = cabs2(A0[(size_t)i * n]);
      if (v > best || (v == best && i < idx)) { best = v; idx = i; }
    }
    gj_block_argmax(best, idx, sb, si);
    if (threadIdx.x == 0) { slot_v[blockIdx.x] = best; slot_i[blockIdx.x] = idx; }
  }
  if (!gj_barrier(bar, expect, polls, timeout, &s_ok)) return;
  for (int k = 0; k < n; ++k) {
    const C* __restrict__ cur = (k & 1) ? A1 : A0;
    C* __restrict__ nxt = (k & 1) ? A0 : A1;
    const double* sv = slot_v + (k & 1) * 1024;
    const int* sx = slot_i + (k & 1) * 1024;
    // pivot from the partial maxima (every CTA reaches the same decision)
    if (threadIdx.x < 32) {
      double best = -1.0;
      int idx = 0x7fffffff;
      for (unsigned c = threadIdx.x; c < nb; c += 32) {
        const double v = sv[c];
        const int i = sx[c];
        if (v > best || (v == best && i < idx)) { best = v; idx = i; }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffff, best, o);
        const int oi = __shfl_xor_sync(0xffffffff, idx, o);
        if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
      }
      if (threadIdx.x == 0) {
        const bool good = best > 0.0 && idx >= k && idx < n;
        s_p = good ? idx : k;
        if (!good && blockIdx.x == 0) atomicExch(fail, 1);
        s_a = good ? crecip(cur[(size_t)s_p * n + k]) : czero<C>();
        if (blockIdx.x == 0) piv[k] = s_p;
      }
    }
    __syncthreads();
    const int p = s_p;
    const C a = s_a;
    const C fk = cur[(size_t)k * n + k];  // multiplier of row p after the swap
    for (int j = threadIdx.x; j < n; j += GJ_T) s_row[j] = (j == k) ? a : cmul(cur[(size_t)p * n + j], a);
    __syncthreads();
    // eliminate into nxt; track the next pivot column's partial maximum
    double best = -1.0;
    int idx = 0x7fffffff;
    const int kn = k + 1;
#pragma unroll 2
    for (int i = blockIdx.x; i < n; i += (int)nb) {
      const C f = (i == k) ? czero<C>() : (i == p ? fk : cur[(size_t)i * n + k]);
      const C* src = cur + (size_t)(i == p ? k : i) * n;  // row p takes the old row k
#pragma unroll 4
      for (int j = threadIdx.x; j < n; j += GJ_T) {
        const C r = s_row[j];  // new pivot row
        C v;
        if (i == k)
          v = r;
        else if (j == k)
          v = cneg(cmul(f, r));
        else
          v = csub(src[j], cmul(f, r));
        nxt[(size_t)i * n + j] = v;
        if (j == kn && i >= kn) {
          const double m = cabs2(v);
          if (m > best || (m == best && i < idx)) { best = m; idx = i; }
        }
      }
    }
    gj_block_argmax(best, idx, sb, si);
    if (threadIdx.x == 0) {
      slot_v[((k + 1) & 1) * 1024 + blockIdx.x] = best;
      slot_i[((k + 1) & 1) * 1024 + blockIdx.x] = idx;
    }
    if (!gj_barrier(bar, expect, polls, timeout, &s_ok)) return;
  }
}

// Undo the column swaps of the recorded pivots.  Skipped when the elimination stopped early (a barrier ran out or
// a zero pivot), since the pivot record is then incomplete; entries outside [k, n) are ignored.
template <typename C>
__global__ void k_gj_unscramble(C* __restrict__ A, int n, const int* __restrict__ piv, const int* __restrict__ fail,
                                const int* __restrict__ timeout) {
  if (*(volatile const int*)timeout || *(volatile const int*)fail) return;
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k && p > k && p < n)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        C t = A[(size_t)i * n + k];
        A[(size_t)i * n + k] = A[(size_t)i * n + p];
        A[(size_t)i * n + p] = t;
      }
    __syncthreads();
  }
}

size_t invert_large_work_bytes(int n) {
  return sizeof(double2) * (size_t)n * n + (sizeof(double) + sizeof(int)) * 2048 + 64;
}

template <typename C>
void invert_large(cudaStream_t st, C* A, int n, int* piv, void* work, int* fail, int* timeout, long polls) {
  int dev = 0, nsm = 0, per = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const size_t sm = sizeof(C) * (size_t)n;
  ensure_max_smem((const void*)k_gj_coop<C>, 160 * 1024);
  MG_CHECK_ARG(sm <= 160 * 1024, "coarsest level too large for the pivot row in shared memory");
  MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gj_coop<C>, GJ_T, sm));
  // one resident CTA per SM (at most one row per CTA), all co-resident as the cooperative launch requires
  const int grid = std::max(1, std::min(std::min(nsm * std::min(std::max(per, 1), 1), 1024), n));
  char* w = (char*)work;
  C* A1 = (C*)w;
  double* slot_v = (double*)(w + sizeof(double2) * (size_t)n * n);
  int* slot_i = (int*)(slot_v + 2048);
  unsigned* bar = (unsigned*)(slot_i + 2048);
  MG_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
  // polls == 0: the default limit; polls < 0: bounded-wait self-test (one arrival more than the grid has)
  long lim = polls == 0 ? GJ_SPIN : (polls > 0 ? polls : -polls);
  unsigned expect = (unsigned)grid + (polls < 0 ? 1u : 0u);
  void* args[] = {&A, &A1, &n, &piv, &slot_v, &slot_i, &bar, &fail, &timeout, &lim, &expect};
  KTimer* t = g_timer;
  cudaEvent_t ea = nullptr, eb = nullptr;
  const char* name = sizeof(C) == 8 ? "k_gj_coop<float2>" : "k_gj_coop<double2>";
  if (t && t->want(name)) { ea = t->get(); eb = t->get(); MG_CUDA(cudaEventRecord(ea, st)); }
  MG_CUDA(cudaLaunchCooperativeKernel((void*)k_gj_coop<C>, dim3(grid), dim3(GJ_T), args, sm, st));
  if (ea) {
    MG_CUDA(cudaEventRecord(eb, st));
    t->recs.push_back({name, __PRETTY_FUNCTION__, 2.0 * sizeof(C) * n * (double)n * n, 8.0 * n * (double)n * n, ea, eb});
  }
  if (g_launch_counter) ++*g_launch_counter;
  if (n & 1)  // odd column count: the last column wrote the scratch buffer
    MG_CUDA(cudaMemcpyAsync(A, A1, sizeof(C) * (size_t)n * n, cudaMemcpyDeviceToDevice, st));
  MG_LAUNCH(k_gj_unscramble<C>, 1, 1024, 0, st, A, n, piv, fail, timeout);
}
template void invert_large<double2>(cudaStream_t, double2*, int, int*, void*, int*, int*, long);
template void invert_large<float2>(cudaStream_t, float2*, int, int*, void*, int*, int*, long);

// ---- y = A x for the coarsest level (n x n dense, nrhs columns) --------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_dense_apply(const typename CT<R>::T* __restrict__ A, int n,
                                                     const typename CT<R>::T* __restrict__ x,
                                                     typename CT<R>::T* __restrict__ y, int nrhs,
                                                     const int* __restrict__ active) {
  typedef typename CT<R>::T C;
  __shared__ C As[16][17];
  __shared__ C Xs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = blockIdx.x * 16 + tx;   // row of A
  const int r = blockIdx.y * 16 + ty;   // rhs
  C acc = czero<C>();
  for (int j0 = 0; j0 < n; j0 += 16) {
    {
      const int ii = blockIdx.x * 16 + ty, jj = j0 + tx;
      As[ty][tx] = (ii < n && jj < n) ? A[(size_t)ii * n + jj] : czero<C>();
      const int rr = blockIdx.y * 16 + ty;
      Xs[ty][tx] = (rr < nrhs && jj < n) ? x[(size_t)rr * n + jj] : czero<C>();
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) acc = cfma(As[tx][q], Xs[ty][q], acc);
    __syncthreads();
  }
  if (i < n && r < nrhs && !(active && !active[r])) y[(size_t)r * n + i] = acc;
}

template <typename R>
void dense_apply(cudaStream_t st, const typename CT<R>::T* A, int n, const typename CT<R>::T* x,
                 typename CT<R>::T* y, int nrhs, const int* active) {
  dim3 grid(cdiv(n, 16), cdiv(nrhs, 16));
  MG_LAUNCH(k_dense_apply<R>, grid, 256, 0, st, A, n, x, y, nrhs, active);
}
template void dense_apply<float>(cudaStream_t, const float2*, int, const float2*, float2*, int, const int*);
template void dense_apply<double>(cudaStream_t, const double2*, int, const double2*, double2*, int, const int*);

// sum_i w_i A_ii with w_i = 1, or (g5_dof > 0) the gamma5 sign of dof i % g5_dof (-1 in its upper half)
__global__ void k_trace(const double2* __restrict__ A, int n, int g5_dof, double2* out) {
  __shared__ double sr[32], si[32];
  double re = 0, im = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double w = (g5_dof > 0 && i % g5_dof >= g5_dof / 2) ? -1.0 : 1.0;
    re += w * A[(size_t)i * n + i].x;
    im += w * A[(size_t)i * n + i].y;
  }
  re = warp_sum(re);
  im = warp_sum(im);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sr[w] = re; si[w] = im; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    re = l < nw ? sr[l] : 0;
    im = l < nw ? si[l] : 0;
    re = warp_sum(re);
    im = warp_sum(im);
    if (l == 0) *out = make_double2(re, im);
  }
}
void trace_dense(cudaStream_t st, const double2* A, int n, double2* out, int g5_dof) {
  MG_LAUNCH(k_trace, 1, 1024, 0, st, A, n, g5_dof, out);
}

// ---- CholeskyQR2 pieces ---------------------------------------------------------------------------
namespace {
constexpr int GCH = 32;     // rows per shared-memory chunk
constexpr int GBLK = 128;   // blocks (partials)
}

size_t gram_work_bytes(int d, long n) {
  (void)n;
  return sizeof(double2) * (size_t)GBLK * d * d;
}

// G is Hermitian: the upper-triangle entries (i, j), i <= j, are packed in order (t = 0 .. d(d+1)/2 - 1) and
// thread tid accumulates entries tid, tid + blockDim.x, ... (at most GACC of them), writing each and its
// conjugate mirror.
constexpr int GACC = (SK_MAXD * (SK_MAXD + 1) / 2 + 1023) / 1024;
__global__ void __launch_bounds__(1024) k_gram_part(const double2* __restrict__ Y, int d, long n,
                                                    double2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* Ys = reinterpret_cast<double2*>(smem_raw);  // [GCH][d]
  const int tid = threadIdx.x, ntri = d * (d + 1) / 2;
  int ii[GACC], jj[GACC];
#pragma unroll
  for (int u = 0; u < GACC; ++u) {
    int t = tid + u * (int)blockDim.x, i = 0;
    if (t >= ntri) { ii[u] = -1; jj[u] = 0; continue; }
    while (t >= d - i) { t -= d - i; ++i; }
    ii[u] = i;
    jj[u] = i + t;
  }
  double2 acc[GACC];
#pragma unroll
  for (int u = 0; u < GACC; ++u) acc[u] = make_double2(0, 0);
  for (long e0 = (long)blockIdx.x * GCH; e0 < n; e0 += (long)gridDim.x * GCH) {
    __syncthreads();
    for (int q = tid; q < GCH * d; q += blockDim.x) {
      const int c = q / GCH, e = q % GCH;
      Ys[e * d + c] = (e0 + e < n) ? Y[(size_t)c * n + e0 + e] : make_double2(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < GACC; ++u)
      if (ii[u] >= 0)
#pragma unroll 8
        for (int e = 0; e < GCH; ++e) acc[u] = cfmac(Ys[e * d + ii[u]], Ys[e * d + jj[u]], acc[u]);
  }
#pragma unroll
  for (int u = 0; u < GACC; ++u) {
    if (ii[u] < 0) continue;
    const int i = ii[u], j = jj[u];
    part[((size_t)blockIdx.x * d + i) * d + j] = acc[u];
    if (i != j) part[((size_t)blockIdx.x * d + j) * d + i] = cconj(acc[u]);
  }
}

__global__ void k_gram_final(const double2* __restrict__ part, int d, int nb, double2* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d * d) return;
  double2 s = make_double2(0, 0);
  for (int b = 0; b < nb; ++b) s = cadd(s, part[(size_t)b * d * d + e]);
  G[e] = s;
}

void gram(cudaStream_t st, const double2* Y, int d, long n, double2* G, void* work) {
  MG_CHECK_ARG(d >= 1 && d <= SK_MAXD, "sketch size d limited to 64");
  const int nb = (int)std::min<long>(GBLK, cdiv(n, GCH));
  double2* part = reinterpret_cast<double2*>(work);
  MG_LAUNCH(k_gram_part, nb, 1024, sizeof(double2) * GCH * d, st, Y, d, n, part);
  MG_LAUNCH(k_gram_final, cdiv(d * d, 256), 256, 0, st, part, d, nb, G);
}

// G = R^H R (R upper, real positive diagonal), Rinv = R^{-1}; R and its inverse in dynamic shared memory
__global__ void k_chol_inv(const double2* __restrict__ Gg, int d, double2* __restrict__ Rinv, int* fail) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* R = reinterpret_cast<double2*>(smem_raw);
  double2* X = R + d * d;
  __shared__ int bad;
  const int tid = threadIdx.x;
  for (int e = tid; e < d * d; e += blockDim.x) { R[e] = Gg[e]; X[e] = make_double2(0, 0); }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < d; ++k) {
    if (tid == 0) {
      double s = R[k * d + k].x;
      for (int i = 0; i < k; ++i) s -= cabs2(R[i * d + k]);
      if (!(s > 0.0)) bad = 1;
      R[k * d + k] = make_double2(sqrt(fmax(s, 1e-300)), 0);
    }
    __syncthreads();
    const double rkk = R[k * d + k].x;
    for (int j = k + 1 + tid; j < d; j += blockDim.x) {
      double2 s = R[k * d + j];
      for (int i = 0; i < k; ++i) s = csub(s, cmulc(R[i * d + k], R[i * d + j]));
      R[k * d + j] = cscale(s, 1.0 / rkk);
    }
    __syncthreads();
  }
  // upper-triangular inverse, column j per thread
  for (int j = tid; j < d; j += blockDim.x) {
    X[j * d + j] = make_double2(1.0 / R[j * d + j].x, 0);
    for (int i = j - 1; i >= 0; --i) {
      double2 s = make_double2(0, 0);
      for (int m = i + 1; m <= j; ++m) s = cfma(R[i * d + m], X[m * d + j], s);
      X[i * d + j] = cscale(cneg(s), 1.0 / R[i * d + i].x);
    }
  }
  __syncthreads();
  for (int e = tid; e < d * d; e += blockDim.x) Rinv[e] = X[e];
  if (tid == 0 && bad) atomicExch(fail, 1);
}

void chol_inv_upper(cudaStream_t st, const double2* G, int d, double2* Rinv, int* fail) {
  MG_CHECK_ARG(d >= 1 && d <= SK_MAXD, "sketch size d limited to 64");
  const int sm = (int)sizeof(double2) * 2 * d * d;
  ensure_max_smem((const void*)k_chol_inv, sizeof(double2) * 2 * SK_MAXD * SK_MAXD);
  MG_LAUNCH(k_chol_inv, 1, 128, sm, st, G, d, Rinv, fail);
}

// Y <- Y Rinv for Y = [d][n]: a block takes RMT consecutive elements e of all d vectors into shared memory and
// each thread forms new_j(e) = sum_{i <= j} Y_i(e) Rinv_ij for several (e, j)
constexpr int RMT = 32;
__global__ void __launch_bounds__(256) k_right_mul_upper(double2* __restrict__ Y, int d, long n,
                                                         const double2* __restrict__ Rinv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* Rs = reinterpret_cast<double2*>(smem_raw);  // [d][d]
  double2* Ys = Rs + d * d;                             // [RMT][d + 1]
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) Rs[e] = Rinv[e];
  for (long e0 = (long)blockIdx.x * RMT; e0 < n; e0 += (long)gridDim.x * RMT) {
    __syncthreads();
    for (int q = threadIdx.x; q < RMT * d; q += blockDim.x) {
      const int i = q / RMT, e = q % RMT;
      Ys[e * (d + 1) + i] = (e0 + e < n) ? Y[(size_t)i * n + e0 + e] : make_double2(0, 0);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < RMT * d; q += blockDim.x) {
      const int j = q / RMT, e = q % RMT;
      if (e0 + e >= n) continue;
      double2 acc = make_double2(0, 0);
      for (int i = 0; i <= j; ++i) acc = cfma(Ys[e * (d + 1) + i], Rs[i * d + j], acc);
      Y[(size_t)j * n + e0 + e] = acc;
    }
  }
}

void right_mul_upper(cudaStream_t st, double2* Y, int d, long n, const double2* Rinv) {
  MG_CHECK_ARG(d >= 1 && d <= SK_MAXD, "sketch size d limited to 64");
  const size_t sm = sizeof(double2) * ((size_t)d * d + (size_t)RMT * (d + 1));
  ensure_max_smem((const void*)k_right_mul_upper,
                  (int)(sizeof(double2) * ((size_t)SK_MAXD * SK_MAXD + (size_t)RMT * (SK_MAXD + 1))));
  MG_LAUNCH(k_right_mul_upper, std::min<long>(cdiv(n, RMT), 2048), 256, sm, st, Y, d, n, Rinv);
}

// ---- projection coefficients c[i][r] = Q_i^H x_r -----------------------------------------------------
namespace {
constexpr int PCH = 32;    // rows per chunk (the Q tile of up to 64 vectors stays under 48 KB)
constexpr int PRG = 8;     // rhs per block
constexpr int PBLK = 96;   // chunks (partials)
}

size_t proj_work_bytes(int d, long n, int nrhs) {
  (void)n;
  return sizeof(double2) * (size_t)PBLK * d * nrhs;
}

// 32 x 8 threads: lane i accumulates basis vectors i and i + 32 (d <= 64) against rhs r0 + g
__global__ void __launch_bounds__(256) k_proj_part(const double2* __restrict__ Q, int d, const double2* __restrict__ x,
                                                   long n, int nrhs, double2* __restrict__ part) {
  __shared__ double2 Qs[PCH * (SK_MAXD + 1)];
  __shared__ double2 Xs[PRG * PCH];
  const int tid = threadIdx.x;
  const int r0 = blockIdx.y * PRG;
  const int i = tid % 32, g = tid / 32;
  double2 acc0 = make_double2(0, 0), acc1 = make_double2(0, 0);
  for (long e0 = (long)blockIdx.x * PCH; e0 < n; e0 += (long)gridDim.x * PCH) {
    __syncthreads();
    for (int q = tid; q < d * PCH; q += blockDim.x) {
      const int c = q / PCH, e = q % PCH;
      Qs[e * (SK_MAXD + 1) + c] = (e0 + e < n) ? Q[(size_t)c * n + e0 + e] : make_double2(0, 0);
    }
    for (int q = tid; q < PRG * PCH; q += blockDim.x) {
      const int rr = q / PCH, e = q % PCH;
      Xs[q] = (r0 + rr < nrhs && e0 + e < n) ? x[(size_t)(r0 + rr) * n + e0 + e] : make_double2(0, 0);
    }
    __syncthreads();
    if (i < d)
#pragma unroll 8
      for (int e = 0; e < PCH; ++e) {
        const double2 xv = Xs[g * PCH + e];
        acc0 = cfmac(Qs[e * (SK_MAXD + 1) + i], xv, acc0);
        if (i + 32 < d) acc1 = cfmac(Qs[e * (SK_MAXD + 1) + i + 32], xv, acc1);
      }
  }
  if (r0 + g < nrhs) {
    if (i < d) part[((size_t)blockIdx.x * d + i) * nrhs + r0 + g] = acc0;
    if (i + 32 < d) part[((size_t)blockIdx.x * d + i + 32) * nrhs + r0 + g] = acc1;
  }
}

__global__ void k_proj_final(const double2* __restrict__ part, int cnt, int nb, double2* __restrict__ c) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= cnt) return;
  double2 s = make_double2(0, 0);
  for (int b = 0; b < nb; ++b) s = cadd(s, part[(size_t)b * cnt + e]);
  c[e] = s;
}

void proj_coeffs(cudaStream_t st, const double2* Q, int d, const double2* x, long n, int nrhs, double2* c, void* work) {
  MG_CHECK_ARG(d >= 1 && d <= SK_MAXD, "sketch size d limited to 64");
  const int nb = (int)std::min<long>(PBLK, cdiv(n, PCH));
  double2* part = reinterpret_cast<double2*>(work);
  MG_LAUNCH(k_proj_part, dim3(nb, cdiv(nrhs, PRG)), 256, 0, st, Q, d, x, n, nrhs, part);
  MG_LAUNCH(k_proj_final, cdiv((long)d * nrhs, 256), 256, 0, st, part, d * nrhs, nb, c);
}

}  // namespace mg
