// Batched BLAS-1 over right-hand sides ([rhs][n] complex vectors), the
// deterministic two-stage reductions used by the Krylov solver (warp-shuffle
// trees, fixed partition, so repeated runs give identical bits), and the
// counter-based Rademacher generator.
#include "ops.cuh"

namespace mg {

namespace {
constexpr int RT = 256;   // threads per reduction block
constexpr int RBLK = 64;  // reduction blocks per rhs

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
  return v;
}
// block-wide sum of a double (RT threads); result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0;
  if (w == 0) {
    r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

template <typename C> struct Acc;
template <> struct Acc<float2> { typedef float R; };
template <> struct Acc<double2> { typedef double R; };
}  // namespace

size_t reduce_work_bytes(long n, int nrhs, int nvec) {
  (void)n;
  return sizeof(double2) * (size_t)nrhs * nvec * RBLK;
}

// ---- norm^2 ------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(RT) k_norm2_part(const C* __restrict__ x, long n, double* __restrict__ part,
                                                   const int* __restrict__ active) {
  typedef typename Acc<C>::R R;
  __shared__ double sh[32];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) {
    if (threadIdx.x == 0) part[(size_t)rhs * RBLK + blockIdx.x] = 0.0;
    return;
  }
  const C* X = x + (size_t)rhs * n;
  R acc = 0;
  for (long i = blockIdx.x * (long)RT + threadIdx.x; i < n; i += (long)RBLK * RT) {
    C v = X[i];
    acc += v.x * v.x + v.y * v.y;
  }
  double r = block_sum((double)acc, sh);
  if (threadIdx.x == 0) part[(size_t)rhs * RBLK + blockIdx.x] = r;
}

__global__ void k_finalize_real(const double* __restrict__ part, int nrhs, double* __restrict__ out) {
  const int rhs = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int l = threadIdx.x & 31;
  if (rhs >= nrhs) return;
  double v = part[(size_t)rhs * RBLK + l] + part[(size_t)rhs * RBLK + l + 32];
  v = warp_sum(v);
  if (l == 0) out[rhs] = v;
}

template <typename C>
void vnorm2(cudaStream_t st, const C* x, long n, int nrhs, double* out, void* work, const int* active) {
  double* part = reinterpret_cast<double*>(work);
  MG_LAUNCH_W(act_rhs(nrhs) * n * sizeof(C), act_rhs(nrhs) * n * 4.0, k_norm2_part<C>, dim3(RBLK, nrhs), RT, 0, st,
              x, n, part, active);
  MG_LAUNCH(k_finalize_real, cdiv(nrhs, 4), 128, 0, st, part, nrhs, out);
}
template void vnorm2<float2>(cudaStream_t, const float2*, long, int, double*, void*, const int*);
template void vnorm2<double2>(cudaStream_t, const double2*, long, int, double*, void*, const int*);

// ---- multi-dot: h[i][rhs] = V_i^H w ---------------------------------------------------
// Each thread accumulates its share of a chunk of dot products in registers; the block then
// reduces all 2*chunk real values together (block_sum_many), one shared-memory pass in all.
template <typename C> struct MdChunk { static constexpr int value = 16; };
template <> struct MdChunk<double2> { static constexpr int value = 8; };

// Transposed warp reduction of NV values per lane: at each step the lanes of a pair swap
// halves of their value sets, so NV values take NV - 1 + log2(32 / NV) shuffles instead of
// 5 NV.  Lane l returns the warp total of value (l >> s), s = log2(32 / NV).
template <int NV>
__device__ __forceinline__ double warp_sum_many(double (&v)[NV]) {
  static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "NV must be a power of two <= 32");
  const int lane = threadIdx.x & 31;
  int o = 16;
#pragma unroll
  for (int half = NV / 2; half >= 1; half >>= 1, o >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int q = 0; q < half; ++q) {
      const double send = up ? v[q] : v[q + half];
      const double keep = up ? v[q + half] : v[q];
      v[q] = keep + __shfl_xor_sync(0xffffffff, send, o);
    }
  }
  double r = v[0];
  for (; o; o >>= 1) r += __shfl_xor_sync(0xffffffff, r, o);
  return r;
}

// Block (RT threads) totals of NV values; thread t < NV returns the total of value t
// (other threads return 0).  sh holds (RT / 32) * NV doubles.
template <int NV>
__device__ __forceinline__ double block_sum_many(double (&v)[NV], double* sh) {
  constexpr int S = (NV == 32) ? 0 : (NV == 16) ? 1 : (NV == 8) ? 2 : (NV == 4) ? 3 : (NV == 2) ? 4 : 5;
  const double r = warp_sum_many<NV>(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();  // sh may still be read by a previous call
  if ((l & ((1 << S) - 1)) == 0) sh[w * NV + (l >> S)] = r;
  __syncthreads();
  double t = 0;
  if ((int)threadIdx.x < NV) {
#pragma unroll
    for (int q = 0; q < RT / 32; ++q) t += sh[q * NV + threadIdx.x];
  }
  return t;
}

// part[(i * nrhs + rhs) * RBLK + block] (component c) = t, for dot i, real (c = 0) / imaginary (c = 1)
__device__ __forceinline__ void store_part(double2* part, int i, int nrhs, int rhs, int c, double t) {
  reinterpret_cast<double*>(part + ((size_t)i * nrhs + rhs) * RBLK + blockIdx.x)[c] = t;
}

template <typename C, int MDC>
__global__ void __launch_bounds__(RT) k_multidot_part(const C* __restrict__ V, long vstride, int k,
                                                      const C* __restrict__ w, long n, double2* __restrict__ part,
                                                      const int* __restrict__ active) {
  typedef typename Acc<C>::R R;
  __shared__ double sh[(RT / 32) * 2 * MDC];
  const int rhs = blockIdx.y;
  const int nrhs = gridDim.y;
  const bool on = !(active && !active[rhs]);
  const C* W = w + (size_t)rhs * n;
  const C* Vr = V + (size_t)rhs * n;
  for (int i0 = 0; i0 < k; i0 += MDC) {
    R ar[MDC], ai[MDC];
#pragma unroll
    for (int q = 0; q < MDC; ++q) { ar[q] = 0; ai[q] = 0; }
    const int cnt = min(MDC, k - i0);
    if (on) {
      for (long e = blockIdx.x * (long)RT + threadIdx.x; e < n; e += (long)RBLK * RT) {
        const C b = W[e];
#pragma unroll
        for (int q = 0; q < MDC; ++q) {
          if (q < cnt) {
            const C a = Vr[(size_t)(i0 + q) * vstride + e];
            ar[q] = fma(a.x, b.x, fma(a.y, b.y, ar[q]));
            ai[q] = fma(a.x, b.y, fma(-a.y, b.x, ai[q]));
          }
        }
      }
    }
    double v[2 * MDC];
#pragma unroll
    for (int q = 0; q < MDC; ++q) { v[2 * q] = ar[q]; v[2 * q + 1] = ai[q]; }
    const double t = block_sum_many<2 * MDC>(v, sh);
    if ((int)threadIdx.x < 2 * cnt) store_part(part, i0 + (threadIdx.x >> 1), nrhs, rhs, threadIdx.x & 1, t);
  }
}

__global__ void k_finalize_cplx(const double2* __restrict__ part, int count, double2* __restrict__ out) {
  const int idx = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int l = threadIdx.x & 31;
  if (idx >= count) return;
  double2 a = part[(size_t)idx * RBLK + l], b = part[(size_t)idx * RBLK + l + 32];
  double re = warp_sum(a.x + b.x), im = warp_sum(a.y + b.y);
  if (l == 0) out[idx] = make_double2(re, im);
}

template <typename C>
void vmultidot(cudaStream_t st, const C* V, long vstride, int k, const C* w, long n, int nrhs, double2* h,
               void* work, const int* active) {
  double2* part = reinterpret_cast<double2*>(work);
  // chunk of dot products per pass: 8 when that covers k (fewer registers, more resident blocks)
  const double bytes = act_rhs(nrhs) * n * sizeof(C) * (k + 1.0), flops = act_rhs(nrhs) * n * 8.0 * k;
  if (k <= 8)
    MG_LAUNCH_W(bytes, flops, (k_multidot_part<C, 8>), dim3(RBLK, nrhs), RT, 0, st, V, vstride, k, w, n, part,
                active);
  else
    MG_LAUNCH_W(bytes, flops, (k_multidot_part<C, MdChunk<C>::value>), dim3(RBLK, nrhs), RT, 0, st, V, vstride, k,
                w, n, part, active);
  MG_LAUNCH(k_finalize_cplx, cdiv((long)k * nrhs, 4), 128, 0, st, part, k * nrhs, h);
}
template void vmultidot<float2>(cudaStream_t, const float2*, long, int, const float2*, long, int, double2*, void*,
                                const int*);
template void vmultidot<double2>(cudaStream_t, const double2*, long, int, const double2*, long, int, double2*,
                                 void*, const int*);

template <typename C>
void vdot(cudaStream_t st, const C* x, const C* y, long n, int nrhs, double2* out, void* work, const int* active) {
  vmultidot<C>(st, x, 0, 1, y, n, nrhs, out, work, active);
}
template void vdot<float2>(cudaStream_t, const float2*, const float2*, long, int, double2*, void*, const int*);
template void vdot<double2>(cudaStream_t, const double2*, const double2*, long, int, double2*, void*, const int*);

// ---- w -= sum_i h_i V_i ; x += sum_i y_i Z_i -----------------------------------------------
template <typename C, bool SUB>
__global__ void __launch_bounds__(256) k_lincomb(const C* __restrict__ V, long vstride, int k,
                                                 const double2* __restrict__ h, C* __restrict__ w, long n,
                                                 const int* __restrict__ active) {
  typedef typename Acc<C>::R R;
  __shared__ C hs[64];
  const int rhs = blockIdx.y, nrhs = gridDim.y;
  if (active && !active[rhs]) return;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double2 v = h[(size_t)i * nrhs + rhs];
    hs[i] = cmake((R)v.x, (R)v.y);
  }
  __syncthreads();
  C* W = w + (size_t)rhs * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    C acc = czero<C>();
    for (int i = 0; i < k; ++i) {
      if (hs[i].x == 0 && hs[i].y == 0) continue;  // unused basis vectors may hold stale data
      acc = cfma(hs[i], V[(size_t)i * vstride + (size_t)rhs * n + e], acc);
    }
    W[e] = SUB ? csub(W[e], acc) : cadd(W[e], acc);
  }
}

static unsigned ew_blocks(long n) { return std::min<long>(cdiv(n, 256 * 4), 1024); }

template <typename C>
void vgs_update(cudaStream_t st, const C* V, long vstride, int k, const double2* h, C* w, long n, int nrhs,
                const int* active) {
  MG_CHECK_ARG(k <= 64, "at most 64 basis vectors");
  MG_LAUNCH_W(act_rhs(nrhs) * n * sizeof(C) * (k + 2.0), act_rhs(nrhs) * n * 8.0 * k, (k_lincomb<C, true>),
              dim3(ew_blocks(n), nrhs), 256, 0, st, V, vstride, k, h, w, n, active);
}
template <typename C>
void vcombine(cudaStream_t st, const C* Z, long zstride, int k, const double2* y, C* x, long n, int nrhs,
              const int* active) {
  MG_CHECK_ARG(k <= 64, "at most 64 basis vectors");
  MG_LAUNCH_W(act_rhs(nrhs) * n * sizeof(C) * (k + 2.0), act_rhs(nrhs) * n * 8.0 * k, (k_lincomb<C, false>),
              dim3(ew_blocks(n), nrhs), 256, 0, st, Z, zstride, k, y, x, n, active);
}
template void vgs_update<float2>(cudaStream_t, const float2*, long, int, const double2*, float2*, long, int, const int*);
template void vgs_update<double2>(cudaStream_t, const double2*, long, int, const double2*, double2*, long, int,
                                  const int*);
template void vcombine<float2>(cudaStream_t, const float2*, long, int, const double2*, float2*, long, int, const int*);
template void vcombine<double2>(cudaStream_t, const double2*, long, int, const double2*, double2*, long, int,
                                const int*);

// ---- fused classical Gram-Schmidt passes ------------------------------------------------------
// First-pass update fused with the second pass's dot products: w -= sum_i h_i V_i, then
// V_i^H w with the updated w; each thread keeps its V_i elements in registers between the two.
template <typename C, int KM>
__global__ void __launch_bounds__(RT, sizeof(C) == 8 ? 2 : 1) k_gs_update_dot(const C* __restrict__ V, long vstride, int k,
                                                      const double2* __restrict__ h, C* __restrict__ w, long n,
                                                      double2* __restrict__ part, const int* __restrict__ active) {
  typedef typename Acc<C>::R R;
  __shared__ C hs[KM];
  __shared__ double sh[(RT / 32) * 2 * KM];
  const int rhs = blockIdx.y, nrhs = gridDim.y;
  const bool on = !(active && !active[rhs]);
  if ((int)threadIdx.x < k) {
    const double2 v = h[(size_t)threadIdx.x * nrhs + rhs];
    hs[threadIdx.x] = cmake((R)v.x, (R)v.y);
  }
  __syncthreads();
  R dr[KM], di[KM];
#pragma unroll
  for (int q = 0; q < KM; ++q) { dr[q] = 0; di[q] = 0; }
  if (on) {
    C* W = w + (size_t)rhs * n;
    const C* Vr = V + (size_t)rhs * n;
    for (long e = blockIdx.x * (long)RT + threadIdx.x; e < n; e += (long)RBLK * RT) {
      C a[KM];
      C acc = czero<C>();
#pragma unroll
      for (int q = 0; q < KM; ++q) {
        if (q < k) {
          a[q] = Vr[(size_t)q * vstride + e];
          acc = cfma(hs[q], a[q], acc);
        }
      }
      const C x = csub(W[e], acc);
      W[e] = x;
#pragma unroll
      for (int q = 0; q < KM; ++q) {
        if (q < k) {
          dr[q] = fma(a[q].x, x.x, fma(a[q].y, x.y, dr[q]));
          di[q] = fma(a[q].x, x.y, fma(-a[q].y, x.x, di[q]));
        }
      }
    }
  }
  double v[2 * KM];
#pragma unroll
  for (int q = 0; q < KM; ++q) { v[2 * q] = dr[q]; v[2 * q + 1] = di[q]; }
  const double t = block_sum_many<2 * KM>(v, sh);
  if ((int)threadIdx.x < 2 * k) store_part(part, threadIdx.x >> 1, nrhs, rhs, threadIdx.x & 1, t);
}

// Second-pass update fused with the norm of the result: w -= sum_i h_i V_i, part = ||w||^2.
template <typename C, int KM>
__global__ void __launch_bounds__(RT) k_gs_update_norm(const C* __restrict__ V, long vstride, int k,
                                                       const double2* __restrict__ h, C* __restrict__ w, long n,
                                                       double* __restrict__ part, const int* __restrict__ active) {
  typedef typename Acc<C>::R R;
  __shared__ C hs[KM];
  __shared__ double sh[32];
  const int rhs = blockIdx.y, nrhs = gridDim.y;
  if (active && !active[rhs]) {
    if (threadIdx.x == 0) part[(size_t)rhs * RBLK + blockIdx.x] = 0.0;
    return;
  }
  if ((int)threadIdx.x < k) {
    const double2 v = h[(size_t)threadIdx.x * nrhs + rhs];
    hs[threadIdx.x] = cmake((R)v.x, (R)v.y);
  }
  __syncthreads();
  C* W = w + (size_t)rhs * n;
  const C* Vr = V + (size_t)rhs * n;
  R s = 0;
  for (long e = blockIdx.x * (long)RT + threadIdx.x; e < n; e += (long)RBLK * RT) {
    C acc = czero<C>();
#pragma unroll
    for (int q = 0; q < KM; ++q)
      if (q < k) acc = cfma(hs[q], Vr[(size_t)q * vstride + e], acc);
    const C x = csub(W[e], acc);
    W[e] = x;
    s += x.x * x.x + x.y * x.y;
  }
  const double r = block_sum((double)s, sh);
  if (threadIdx.x == 0) part[(size_t)rhs * RBLK + blockIdx.x] = r;
}

template <typename C>
void vgs_update_dot(cudaStream_t st, const C* V, long vstride, int k, const double2* h, C* w, long n, int nrhs,
                    double2* h2, void* work, const int* active) {
  if (k > 16) {
    vgs_update<C>(st, V, vstride, k, h, w, n, nrhs, active);
    vmultidot<C>(st, V, vstride, k, w, n, nrhs, h2, work, active);
    return;
  }
  double2* part = reinterpret_cast<double2*>(work);
  const double bytes = act_rhs(nrhs) * n * sizeof(C) * (k + 2.0), flops = act_rhs(nrhs) * n * 16.0 * k;
  if (k <= 8)
    MG_LAUNCH_W(bytes, flops, (k_gs_update_dot<C, 8>), dim3(RBLK, nrhs), RT, 0, st, V, vstride, k, h, w, n, part,
                active);
  else
    MG_LAUNCH_W(bytes, flops, (k_gs_update_dot<C, 16>), dim3(RBLK, nrhs), RT, 0, st, V, vstride, k, h, w, n, part,
                active);
  MG_LAUNCH(k_finalize_cplx, cdiv((long)k * nrhs, 4), 128, 0, st, part, k * nrhs, h2);
}

template <typename C>
void vgs_update_norm(cudaStream_t st, const C* V, long vstride, int k, const double2* h, C* w, long n, int nrhs,
                     double* out, void* work, const int* active) {
  if (k > 16) {
    vgs_update<C>(st, V, vstride, k, h, w, n, nrhs, active);
    vnorm2<C>(st, w, n, nrhs, out, work, active);
    return;
  }
  double* part = reinterpret_cast<double*>(work);
  const double bytes = act_rhs(nrhs) * n * sizeof(C) * (k + 2.0), flops = act_rhs(nrhs) * n * (8.0 * k + 4.0);
  if (k <= 8)
    MG_LAUNCH_W(bytes, flops, (k_gs_update_norm<C, 8>), dim3(RBLK, nrhs), RT, 0, st, V, vstride, k, h, w, n, part,
                active);
  else
    MG_LAUNCH_W(bytes, flops, (k_gs_update_norm<C, 16>), dim3(RBLK, nrhs), RT, 0, st, V, vstride, k, h, w, n, part,
                active);
  MG_LAUNCH(k_finalize_real, cdiv(nrhs, 4), 128, 0, st, part, nrhs, out);
}
template void vgs_update_dot<float2>(cudaStream_t, const float2*, long, int, const double2*, float2*, long, int,
                                     double2*, void*, const int*);
template void vgs_update_dot<double2>(cudaStream_t, const double2*, long, int, const double2*, double2*, long, int,
                                      double2*, void*, const int*);
template void vgs_update_norm<float2>(cudaStream_t, const float2*, long, int, const double2*, float2*, long, int,
                                      double*, void*, const int*);
template void vgs_update_norm<double2>(cudaStream_t, const double2*, long, int, const double2*, double2*, long, int,
                                       double*, void*, const int*);

// ---- elementwise -------------------------------------------------------------------------------
template <typename C> void vzero(cudaStream_t st, C* x, long n, int nrhs) {
  MG_CUDA(cudaMemsetAsync(x, 0, sizeof(C) * (size_t)n * nrhs, st));
}
template void vzero<float2>(cudaStream_t, float2*, long, int);
template void vzero<double2>(cudaStream_t, double2*, long, int);

template <typename C> void vcopy(cudaStream_t st, const C* x, C* y, long n, int nrhs) {
  MG_CUDA(cudaMemcpyAsync(y, x, sizeof(C) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice, st));
}
template void vcopy<float2>(cudaStream_t, const float2*, float2*, long, int);
template void vcopy<double2>(cudaStream_t, const double2*, double2*, long, int);

template <typename Cd, typename Cs>
__global__ void k_convert(const Cs* __restrict__ x, Cd* __restrict__ y, long n, const double* __restrict__ scale,
                          const int* __restrict__ active) {
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const double s = scale ? 1.0 / scale[rhs] : 1.0;
  const Cs* X = x + (size_t)rhs * n;
  Cd* Y = y + (size_t)rhs * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    Cs v = X[e];
    Cd o;
    o.x = (double)v.x * s;
    o.y = (double)v.y * s;
    Y[e] = o;
  }
}
template <typename Cd, typename Cs>
void vconvert(cudaStream_t st, const Cs* x, Cd* y, long n, int nrhs, const double* scale, const int* active) {
  MG_LAUNCH((k_convert<Cd, Cs>), dim3(ew_blocks(n), nrhs), 256, 0, st, x, y, n, scale, active);
}
template void vconvert<float2, double2>(cudaStream_t, const double2*, float2*, long, int, const double*, const int*);
template void vconvert<double2, float2>(cudaStream_t, const float2*, double2*, long, int, const double*, const int*);
template void vconvert<double2, double2>(cudaStream_t, const double2*, double2*, long, int, const double*,
                                         const int*);
template void vconvert<float2, float2>(cudaStream_t, const float2*, float2*, long, int, const double*, const int*);

template <typename C>
__global__ void k_axpy(const double2* __restrict__ a, double sign, const C* __restrict__ x, C* __restrict__ y,
                       long n, const int* __restrict__ active) {
  typedef typename Acc<C>::R R;
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const double2 av = a[rhs];
  const C ac = cmake((R)(sign * av.x), (R)(sign * av.y));
  const C* X = x + (size_t)rhs * n;
  C* Y = y + (size_t)rhs * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    Y[e] = cfma(ac, X[e], Y[e]);
}
template <typename C>
void vaxpy(cudaStream_t st, const double2* a, double sign, const C* x, C* y, long n, int nrhs, const int* active) {
  MG_LAUNCH(k_axpy<C>, dim3(ew_blocks(n), nrhs), 256, 0, st, a, sign, x, y, n, active);
}
template void vaxpy<float2>(cudaStream_t, const double2*, double, const float2*, float2*, long, int, const int*);
template void vaxpy<double2>(cudaStream_t, const double2*, double, const double2*, double2*, long, int, const int*);

template <typename C>
__global__ void k_scale_inv(const double* __restrict__ s, const C* __restrict__ x, C* __restrict__ y, long n,
                            const int* __restrict__ active) {
  typedef typename Acc<C>::R R;
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const R f = (R)(1.0 / s[rhs]);
  const C* X = x + (size_t)rhs * n;
  C* Y = y + (size_t)rhs * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    Y[e] = cscale(X[e], f);
}
template <typename C>
void vscale_inv(cudaStream_t st, const double* s, const C* x, C* y, long n, int nrhs, const int* active) {
  MG_LAUNCH(k_scale_inv<C>, dim3(ew_blocks(n), nrhs), 256, 0, st, s, x, y, n, active);
}
template void vscale_inv<float2>(cudaStream_t, const double*, const float2*, float2*, long, int, const int*);
template void vscale_inv<double2>(cudaStream_t, const double*, const double2*, double2*, long, int, const int*);

template <typename R>
__global__ void k_accum_mixed(const double* __restrict__ scale, const typename CT<R>::T* __restrict__ e,
                              double2* __restrict__ x, long n, const int* __restrict__ active) {
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const double s = scale ? scale[rhs] : 1.0;
  const typename CT<R>::T* E = e + (size_t)rhs * n;
  double2* X = x + (size_t)rhs * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    typename CT<R>::T v = E[i];
    double2 o = X[i];
    o.x = fma(s, (double)v.x, o.x);
    o.y = fma(s, (double)v.y, o.y);
    X[i] = o;
  }
}
template <typename R>
void vaccum_mixed(cudaStream_t st, const double* scale, const typename CT<R>::T* e, double2* x, long n, int nrhs,
                  const int* active) {
  MG_LAUNCH(k_accum_mixed<R>, dim3(ew_blocks(n), nrhs), 256, 0, st, scale, e, x, n, active);
}
template void vaccum_mixed<float>(cudaStream_t, const double*, const float2*, double2*, long, int, const int*);
template void vaccum_mixed<double>(cudaStream_t, const double*, const double2*, double2*, long, int, const int*);

__global__ void k_sub_from(const double2* __restrict__ x, double2* __restrict__ y, size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    y[e] = csub(x[e], y[e]);
}
void vsub_from(cudaStream_t st, const double2* x, double2* y, long n, int nrhs) {
  MG_LAUNCH(k_sub_from, 1024, 256, 0, st, x, y, (size_t)n * nrhs);
}

__global__ void k_sqrt(double* v, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = sqrt(v[i]);
}
void sqrt_inplace(cudaStream_t st, double* v, int n) { MG_LAUNCH(k_sqrt, cdiv(n, 256), 256, 0, st, v, n); }

__global__ void k_fill_int(int* p, int v, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
void fill_int(cudaStream_t st, int* p, int v, int n) { MG_LAUNCH(k_fill_int, cdiv(n, 256), 256, 0, st, p, v, n); }

// ---- counter-based Rademacher ------------------------------------------------------------------
template <bool CPLX>
__global__ void k_rademacher(uint64_t seed, int level, int phase, int64_t sample0, long n, double2* __restrict__ out) {
  const int rhs = blockIdx.y;
  const uint64_t key = stream_key(seed, level, phase, (uint64_t)(sample0 + rhs));
  double2* O = out + (size_t)rhs * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    if (CPLX)
      O[i] = make_double2(rad_sign(key, 2 * (uint64_t)i), rad_sign(key, 2 * (uint64_t)i + 1));
    else
      O[i] = make_double2(rad_sign(key, (uint64_t)i), 0.0);
  }
}
void rademacher_fill(cudaStream_t st, uint64_t seed, int level, int phase, int64_t sample0, long n, int nrhs,
                     double2* out) {
  MG_LAUNCH(k_rademacher<false>, dim3(ew_blocks(n), nrhs), 256, 0, st, seed, level, phase, sample0, n, out);
}
void complex_rademacher_fill(cudaStream_t st, uint64_t seed, int level, int phase, int64_t sample0, long n, int nrhs,
                             double2* out) {
  MG_LAUNCH(k_rademacher<true>, dim3(ew_blocks(n), nrhs), 256, 0, st, seed, level, phase, sample0, n, out);
}

// Z4 noise: entry i = i^q, q = the top two bits of the same counter word whose top bit gives the Rademacher sign
__global__ void k_z4(uint64_t seed, int level, int phase, int64_t sample0, long n, double2* __restrict__ out) {
  const int rhs = blockIdx.y;
  const uint64_t key = stream_key(seed, level, phase, (uint64_t)(sample0 + rhs));
  double2* O = out + (size_t)rhs * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const unsigned q = (unsigned)(mix64(key + 0x9E3779B97F4A7C15ull * ((uint64_t)i + 1)) >> 62);
    const double re = q == 0 ? 1.0 : q == 2 ? -1.0 : 0.0;
    const double im = q == 1 ? 1.0 : q == 3 ? -1.0 : 0.0;
    O[i] = make_double2(re, im);
  }
}
void noise_fill(cudaStream_t st, int kind, uint64_t seed, int level, int phase, int64_t sample0, long n, int nrhs,
                double2* out) {
  if (kind == MGMLMC_NOISE_Z4)
    MG_LAUNCH(k_z4, dim3(ew_blocks(n), nrhs), 256, 0, st, seed, level, phase, sample0, n, out);
  else
    rademacher_fill(st, seed, level, phase, sample0, n, nrhs, out);
}

// y <- gamma5 y in place: the components of chirality 1 change sign (dof index >= dof / 2 of each site; on the
// fine level dof = 2, so spin 1)
__global__ void k_gamma5(double2* __restrict__ y, int dof, size_t total) {
  const int half = dof / 2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    if ((int)(e % dof) >= half) y[e] = cneg(y[e]);
}
void gamma5_apply(cudaStream_t st, double2* y, int dof, long n, int nrhs) {
  MG_LAUNCH_W(32.0 * n * nrhs, 0, k_gamma5, 1024, 256, 0, st, y, dof, (size_t)n * nrhs);
}

}  // namespace mg
