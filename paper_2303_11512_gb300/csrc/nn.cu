// Learned gauge-covariant preconditioner: a stack of 3x3 parallel-transport
// convolutions over complex channels (bf16 weights, FP32 accumulation) with a
// phase-preserving activation, its forward and backward kernels, and Adam.
//
//   z(x)_k = sum_d sum_c W[d][k][c] T_d(x) a(x + d)_c,  d = 3 (dt + 1) + (dx + 1)
//   a'(x)_k = z_k max(0, |z_k| + b_k) / |z_k|   (hidden layers; the last one is linear)
//
// T_d(x) transports a field from x + d to x (links with the antiperiodic sign on
// time-boundary crossings; diagonals average the two L-shaped paths), so the net
// commutes with gauge transformations.  Fields are [rhs][site][channel] complex.
// Gradients follow the complex convention g = dL/dRe + i dL/dIm:
// y = W u  ->  g_W += g_y conj(u),  g_u = conj(W) g_y.
#include <cuda_bf16.h>

#include "nn.cuh"

namespace mg {

namespace {

__device__ __forceinline__ int nn_nbr(int s, int d, int L) {
  const int t = s / L, x = s - t * L;
  const int dx = d % 3 - 1, dt = d / 3 - 1;
  int xx = x + dx, tt = t + dt;
  xx = xx < 0 ? xx + L : (xx >= L ? xx - L : xx);
  tt = tt < 0 ? tt + L : (tt >= L ? tt - L : tt);
  return tt * L + xx;
}

__global__ void k_nn_transport(const double2* __restrict__ U, int L, float2* __restrict__ T) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= L * L) return;
  const int t = s / L, x = s - t * L;
  auto site = [&](int tt, int xx) { return ((tt + L) % L) * L + (xx + L) % L; };
  auto ux = [&](int tt, int xx) -> double2 { return U[2 * site(tt, xx)]; };
  auto ut = [&](int tt, int xx) -> double2 {  // t-link with the boundary sign of the hop t -> t+1
    const int t0 = (tt + L) % L;
    double2 u = U[2 * site(tt, xx) + 1];
    return t0 == L - 1 ? cneg(u) : u;
  };
  // single hops from (t, x) to a neighbour: transport from neighbour back to (t, x)
  auto hx = [&](int tt, int xx, int dx) -> double2 {
    if (dx == 0) return make_double2(1, 0);
    return dx > 0 ? ux(tt, xx) : cconj(ux(tt, xx - 1));
  };
  auto ht = [&](int tt, int xx, int dt) -> double2 {
    if (dt == 0) return make_double2(1, 0);
    return dt > 0 ? ut(tt, xx) : cconj(ut(tt - 1, xx));
  };
  for (int d = 0; d < 9; ++d) {
    const int dx = d % 3 - 1, dt = d / 3 - 1;
    double2 v;
    if (dx == 0 || dt == 0) {
      v = cmul(hx(t, x, dx), ht(t, x, dt));
    } else {
      const double2 p1 = cmul(hx(t, x, dx), ht(t, x + dx, dt));
      const double2 p2 = cmul(ht(t, x, dt), hx(t + dt, x, dx));
      v = cscale(cadd(p1, p2), 0.5);
    }
    T[(size_t)s * 9 + d] = make_float2((float)v.x, (float)v.y);
  }
}

// params (FP32 master) -> bf16 weights of one layer
__global__ void k_nn_round(const float* __restrict__ p, int count, __nv_bfloat16* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) w[i] = __float2bfloat16_rn(p[i]);
}

template <int CI, int CO, bool ACT>
__global__ void __launch_bounds__(128) k_nn_fwd(const float2* __restrict__ T, const float2* __restrict__ a,
                                                const __nv_bfloat16* __restrict__ W, const float* __restrict__ b,
                                                float2* __restrict__ z, float2* __restrict__ out, int L) {
  __shared__ float2 sW[9 * CO * CI];
  for (int e = threadIdx.x; e < 9 * CO * CI; e += blockDim.x)
    sW[e] = make_float2(__bfloat162float(W[2 * e]), __bfloat162float(W[2 * e + 1]));
  __syncthreads();
  const int V = L * L;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (s >= V) return;
  const float2* A = a + (size_t)rhs * V * CI;
  float2 acc[CO];
#pragma unroll
  for (int k = 0; k < CO; ++k) acc[k] = make_float2(0.f, 0.f);
  for (int d = 0; d < 9; ++d) {
    const float2 t = T[(size_t)s * 9 + d];
    const float2* an = A + (size_t)nn_nbr(s, d, L) * CI;
#pragma unroll
    for (int c = 0; c < CI; ++c) {
      const float2 u = cmul(t, an[c]);
#pragma unroll
      for (int k = 0; k < CO; ++k) acc[k] = cfma(sW[(d * CO + k) * CI + c], u, acc[k]);
    }
  }
  float2* O = out + ((size_t)rhs * V + s) * CO;
  float2* Z = z ? z + ((size_t)rhs * V + s) * CO : nullptr;
#pragma unroll
  for (int k = 0; k < CO; ++k) {
    if (Z) Z[k] = acc[k];
    if (ACT) {
      const float m = sqrtf(acc[k].x * acc[k].x + acc[k].y * acc[k].y);
      const float f = m > 0.f ? fmaxf(0.f, m + b[k]) / m : 0.f;
      O[k] = make_float2(acc[k].x * f, acc[k].y * f);
    } else {
      O[k] = acc[k];
    }
  }
}

// activation backward in place: g (w.r.t. the activation output) -> g_z; bias partials per block
template <int CO>
__global__ void __launch_bounds__(128) k_nn_act_bwd(const float2* __restrict__ z, const float* __restrict__ b,
                                                    float2* __restrict__ g, long count_sites, float* __restrict__ bpart) {
  __shared__ float red[4][CO];
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;  // (rhs, site) row
  float rb[CO];
#pragma unroll
  for (int k = 0; k < CO; ++k) rb[k] = 0.f;
  if (i < count_sites) {
#pragma unroll
    for (int k = 0; k < CO; ++k) {
      const float2 zz = z[i * CO + k];
      const float2 gg = g[i * CO + k];
      const float m = sqrtf(zz.x * zz.x + zz.y * zz.y);
      float2 out = make_float2(0.f, 0.f);
      if (m > 0.f && m + b[k] > 0.f) {
        const float2 ph = make_float2(zz.x / m, zz.y / m);
        const float rad = ph.x * gg.x + ph.y * gg.y;
        const float sc = (m + b[k]) / m;
        out = make_float2(rad * ph.x + sc * (gg.x - rad * ph.x), rad * ph.y + sc * (gg.y - rad * ph.y));
        rb[k] = rad;
      }
      g[i * CO + k] = out;
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < CO; ++k) {
    float v = rb[k];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
    if (l == 0) red[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < CO)
    bpart[(size_t)blockIdx.x * CO + threadIdx.x] =
        red[0][threadIdx.x] + red[1][threadIdx.x] + red[2][threadIdx.x] + red[3][threadIdx.x];
}

// gradient w.r.t. the layer input: ga(y)_c = sum_d conj(T_d(x)) sum_k conj(W[d][k][c]) gz(x)_k, x = y - d
template <int CI, int CO>
__global__ void __launch_bounds__(128) k_nn_bwd_in(const float2* __restrict__ T, const float2* __restrict__ gz,
                                                   const __nv_bfloat16* __restrict__ W, float2* __restrict__ ga,
                                                   int L) {
  __shared__ float2 sW[9 * CO * CI];
  for (int e = threadIdx.x; e < 9 * CO * CI; e += blockDim.x)
    sW[e] = make_float2(__bfloat162float(W[2 * e]), __bfloat162float(W[2 * e + 1]));
  __syncthreads();
  const int V = L * L;
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (y >= V) return;
  float2 acc[CI];
#pragma unroll
  for (int c = 0; c < CI; ++c) acc[c] = make_float2(0.f, 0.f);
  for (int d = 0; d < 9; ++d) {
    const int x = nn_nbr(y, 8 - d, L);  // y - offset(d)
    const float2 t = cconj(T[(size_t)x * 9 + d]);
    const float2* G = gz + ((size_t)rhs * V + x) * CO;
    float2 sv[CI];
#pragma unroll
    for (int c = 0; c < CI; ++c) sv[c] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < CO; ++k) {
      const float2 gk = G[k];
#pragma unroll
      for (int c = 0; c < CI; ++c) sv[c] = cfmac(sW[(d * CO + k) * CI + c], gk, sv[c]);
    }
#pragma unroll
    for (int c = 0; c < CI; ++c) acc[c] = cfma(t, sv[c], acc[c]);
  }
  float2* O = ga + ((size_t)rhs * V + y) * CI;
#pragma unroll
  for (int c = 0; c < CI; ++c) O[c] = acc[c];
}

// weight-gradient partials: one block per 64 consecutive sites of one rhs
constexpr int NN_WCH = 64;
template <int CI, int CO>
__global__ void __launch_bounds__(256) k_nn_bwd_w(const float2* __restrict__ T, const float2* __restrict__ a,
                                                  const float2* __restrict__ gz, int L, float2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* su = reinterpret_cast<float2*>(smem_raw);  // [NN_WCH][9][CI]
  float2* sg = su + NN_WCH * 9 * CI;                 // [NN_WCH][CO]
  const int V = L * L;
  const int chunks = (V + NN_WCH - 1) / NN_WCH;
  const int rhs = blockIdx.x / chunks, x0 = (blockIdx.x % chunks) * NN_WCH;
  const float2* A = a + (size_t)rhs * V * CI;
  for (int e = threadIdx.x; e < NN_WCH * 9 * CI; e += blockDim.x) {
    const int xi = e / (9 * CI), r = e % (9 * CI), d = r / CI, c = r % CI;
    const int x = x0 + xi;
    float2 v = make_float2(0.f, 0.f);
    if (x < V) v = cmul(T[(size_t)x * 9 + d], A[(size_t)nn_nbr(x, d, L) * CI + c]);
    su[e] = v;
  }
  for (int e = threadIdx.x; e < NN_WCH * CO; e += blockDim.x) {
    const int xi = e / CO, k = e % CO;
    const int x = x0 + xi;
    sg[e] = x < V ? gz[((size_t)rhs * V + x) * CO + k] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int w = threadIdx.x; w < 9 * CO * CI; w += blockDim.x) {
    const int d = w / (CO * CI), k = (w / CI) % CO, c = w % CI;
    float2 acc = make_float2(0.f, 0.f);
    for (int xi = 0; xi < NN_WCH; ++xi) acc = cfmac(su[(xi * 9 + d) * CI + c], sg[xi * CO + k], acc);  // g conj(u)
    part[(size_t)blockIdx.x * 9 * CO * CI + w] = acc;
  }
}

// sum partials over blocks in a fixed order into the flat gradient (float pairs)
__global__ void k_nn_reduce_c(const float2* __restrict__ part, int nblk, int count, float* __restrict__ grad) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= count) return;
  double re = 0, im = 0;
  for (int b = 0; b < nblk; ++b) {
    const float2 v = part[(size_t)b * count + w];
    re += v.x;
    im += v.y;
  }
  grad[2 * w] = (float)re;
  grad[2 * w + 1] = (float)im;
}
__global__ void k_nn_reduce_r(const float* __restrict__ part, int nblk, int count, float* __restrict__ grad) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= count) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * count + w];
  grad[w] = (float)s;
}

// loss gradient: g = 2 (y - e) / (nrhs ||e||^2)
__global__ void k_nn_diff(const float2* __restrict__ y, const float2* __restrict__ e, float2* __restrict__ g, long n) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= n) return;
  const size_t o = (size_t)rhs * n + i;
  g[o] = csub(y[o], e[o]);
}
__global__ void k_nn_scale(float2* __restrict__ g, long n, const double* __restrict__ en, int nrhs) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= n) return;
  const float f = (float)(2.0 / (nrhs * en[rhs]));
  g[(size_t)rhs * n + i] = cscale(g[(size_t)rhs * n + i], f);
}

__global__ void k_nn_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, int count, float lr, float b1, float b2, float c1, float c2,
                          float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_nn_add(float2* __restrict__ z, const float2* __restrict__ c, long n, const double* __restrict__ s) {
  const int rhs = blockIdx.y;
  const float f = s ? (float)s[rhs] : 1.f;
  if (f == 0.f) return;  // masked or zero residual: no correction
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const size_t o = (size_t)rhs * n + i;
    z[o] = cadd(z[o], cscale(c[o], f));
  }
}

// ---- dispatch over the supported channel counts -------------------------------------------
template <typename F>
void with_dims(int ci, int co, F&& f) {
#define MG_NN_CASE(A, B) \
  if (ci == A && co == B) return f(std::integral_constant<int, A>(), std::integral_constant<int, B>());
  MG_NN_CASE(2, 4) MG_NN_CASE(4, 4) MG_NN_CASE(4, 2)
  MG_NN_CASE(2, 8) MG_NN_CASE(8, 8) MG_NN_CASE(8, 2)
  MG_NN_CASE(2, 16) MG_NN_CASE(16, 16) MG_NN_CASE(16, 2)
#undef MG_NN_CASE
  throw Error(MGMLMC_ERR_INVALID_ARG, "unsupported channel count (4, 8 or 16)");
}

}  // namespace

int NNet::dim(int l) const { return (l == 0 || l == layers) ? 2 : channels; }
size_t NNet::w_offset(int l) const {
  size_t o = 0;
  for (int j = 0; j < l; ++j) o += 2 * 9 * (size_t)dim(j + 1) * dim(j) + (j + 1 < layers ? dim(j + 1) : 0);
  return o;
}

void nn_init(NNet* net, const double2* U, int L, int layers, int channels, uint64_t seed, cudaStream_t st) {
  MG_CHECK_ARG(layers >= 2 && layers <= 8, "layers must be 2..8");
  MG_CHECK_ARG(channels == 4 || channels == 8 || channels == 16, "channels must be 4, 8 or 16");
  MG_CHECK_ARG(L >= 4 && L % 2 == 0, "L must be even and >= 4");
  net->L = L;
  net->layers = layers;
  net->channels = channels;
  net->st = st;
  net->nparams = net->w_offset(layers);
  net->T.alloc(sizeof(float2) * 9 * L * L, st);
  MG_LAUNCH(k_nn_transport, cdiv(L * L, 128), 128, 0, st, U, L, net->T.as<float2>());
  // seeded initial weights: complex Gaussian / sqrt(9 c_in) by Box-Muller on the SplitMix64 stream, zero biases
  std::vector<float> p(net->nparams, 0.f);
  uint64_t ctr = 0;
  auto unif = [&]() { return ((mix64(seed * 0x9E3779B97F4A7C15ull + (++ctr)) >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
  for (int l = 0; l < layers; ++l) {
    const size_t o = net->w_offset(l);
    const int ci = net->dim(l), co = net->dim(l + 1);
    const double s = 1.0 / std::sqrt(9.0 * ci) / std::sqrt(2.0);
    for (int i = 0; i < 2 * 9 * co * ci; ++i) {
      const double u1 = unif(), u2 = unif();
      p[o + i] = (float)(s * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  }
  net->params.alloc(sizeof(float) * net->nparams, st);
  net->m.alloc(sizeof(float) * net->nparams, st);
  net->v.alloc(sizeof(float) * net->nparams, st);
  net->grad.alloc(sizeof(float) * net->nparams, st);
  net->w16.alloc(sizeof(__nv_bfloat16) * net->nparams, st);
  MG_CUDA(cudaMemcpyAsync(net->params.p, p.data(), sizeof(float) * net->nparams, cudaMemcpyHostToDevice, st));
  MG_CUDA(cudaMemsetAsync(net->m.p, 0, sizeof(float) * net->nparams, st));
  MG_CUDA(cudaMemsetAsync(net->v.p, 0, sizeof(float) * net->nparams, st));
  net->err.alloc(sizeof(int), st);
  MG_CUDA(cudaMemsetAsync(net->err.p, 0, sizeof(int), st));
  MG_CUDA(cudaStreamSynchronize(st));
  net->step = 0;
  net->tc = nn_tc_supported(L) ? 1 : 0;
}

void nn_check(NNet* net, cudaStream_t st) {
  int flag = 0;
  MG_CUDA(cudaMemcpyAsync(&flag, net->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  MG_CUDA(cudaStreamSynchronize(st));
  if (flag) {
    MG_CUDA(cudaMemsetAsync(net->err.p, 0, sizeof(int), st));
    throw Error(MGMLMC_ERR_TIMEOUT, "tensor-core layer: a bounded wait expired (code " + std::to_string(flag) + ")");
  }
}

void nn_bind_field(NNet* net, const double2* U, int L, cudaStream_t st) {
  MG_CHECK_ARG(L >= 4 && L % 2 == 0, "L must be even and >= 4");
  MG_CHECK_ARG(!net->tc || nn_tc_supported(L), "tensor-core layers need L a multiple of 16");
  MG_CUDA(cudaStreamSynchronize(net->st));
  net->L = L;
  net->st = st;
  net->T.alloc(sizeof(float2) * 9 * L * L, st);
  MG_LAUNCH(k_nn_transport, cdiv(L * L, 128), 128, 0, st, U, L, net->T.as<float2>());
  net->acts.clear();
  net->zs.clear();
  net->acts16.clear();
}

static void nn_round(NNet* net, cudaStream_t st) {
  MG_LAUNCH(k_nn_round, cdiv((long)net->nparams, 256), 256, 0, st, net->params.as<float>(), (int)net->nparams,
            net->w16.as<__nv_bfloat16>());
}

// forward; with a tape (training) the inputs of every layer and hidden pre-activations are kept
void nn_forward(NNet* net, const float2* r, float2* y, int nrhs, bool tape, cudaStream_t st) {
  if (net->tc) return nn_tc_forward(net, r, nullptr, y, nrhs, tape, net->err.as<int>(), st);
  const int L = net->L, V = L * L;
  nn_round(net, st);
  const size_t fsz = (size_t)nrhs * V * 16;
  if (tape) {
    net->acts.resize(net->layers);
    net->zs.resize(net->layers);
  }
  std::vector<DBuf> tmp(2);
  const float2* in = r;
  for (int l = 0; l < net->layers; ++l) {
    const int ci = net->dim(l), co = net->dim(l + 1);
    const bool last = l == net->layers - 1;
    float2* out;
    float2* z = nullptr;
    if (last) {
      out = y;
    } else if (tape) {
      net->acts[l + 1].ensure(sizeof(float2) * (size_t)nrhs * V * co, st);
      out = net->acts[l + 1].as<float2>();
    } else {
      tmp[l & 1].ensure(sizeof(float2) * (size_t)nrhs * V * co, st);
      out = tmp[l & 1].as<float2>();
    }
    if (tape && !last) {
      net->zs[l].ensure(sizeof(float2) * (size_t)nrhs * V * co, st);
      z = net->zs[l].as<float2>();
    }
    const __nv_bfloat16* W = net->w16.as<__nv_bfloat16>() + net->w_offset(l);
    const float* b = last ? nullptr : net->params.as<float>() + net->w_offset(l) + 2 * 9 * co * ci;
    dim3 grid(cdiv(V, 128), nrhs);
    const double flops = 8.0 * 9 * ci * co * V * nrhs;
    with_dims(ci, co, [&](auto CI, auto CO) {
      if (last)
        MG_LAUNCH_W(0, flops, (k_nn_fwd<CI.value, CO.value, false>), grid, 128, 0, st, net->T.as<float2>(), in, W, b,
                    z, out, L);
      else
        MG_LAUNCH_W(0, flops, (k_nn_fwd<CI.value, CO.value, true>), grid, 128, 0, st, net->T.as<float2>(), in, W, b, z,
                    out, L);
    });
    in = out;
    (void)fsz;
  }
}

// loss and gradient (w.r.t. the bf16-rounded weights and the biases) into net->grad; returns the loss
double nn_backward(NNet* net, const float2* r, const float2* e, int nrhs, cudaStream_t st, int* pinned) {
  const int L = net->L, V = L * L;
  const long n = 2L * V;  // complex per rhs of the input/output fields
  DBuf y(sizeof(float2) * n * nrhs, st), g(sizeof(float2) * n * nrhs, st);
  nn_forward(net, r, y.as<float2>(), nrhs, true, st);
  DBuf nrm(sizeof(double) * 2 * nrhs, st), red(reduce_work_bytes(n, nrhs, 1), st);
  vnorm2<float2>(st, e, n, nrhs, nrm.as<double>(), red.p, nullptr);
  MG_LAUNCH(k_nn_diff, dim3(cdiv(n, 256), nrhs), 256, 0, st, y.as<float2>(), e, g.as<float2>(), n);
  vnorm2<float2>(st, g.as<float2>(), n, nrhs, nrm.as<double>() + nrhs, red.p, nullptr);
  std::vector<double> hn(2 * nrhs);
  MG_CUDA(cudaMemcpyAsync(hn.data(), nrm.p, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
  MG_CUDA(cudaStreamSynchronize(st));
  double loss = 0;
  for (int i = 0; i < nrhs; ++i) loss += hn[nrhs + i] / hn[i];
  loss /= nrhs;
  MG_LAUNCH(k_nn_scale, dim3(cdiv(n, 256), nrhs), 256, 0, st, g.as<float2>(), n, nrm.as<double>(), nrhs);
  if (net->tc) {
    nn_tc_backward(net, g.as<float2>(), nrhs, net->err.as<int>(), st);
    return loss;
  }
  // walk the layers backwards; g holds the gradient w.r.t. the current layer's output
  DBuf gprev;
  for (int l = net->layers - 1; l >= 0; --l) {
    const int ci = net->dim(l), co = net->dim(l + 1);
    const bool last = l == net->layers - 1;
    float2* gz = g.as<float2>();
    const size_t woff = net->w_offset(l);
    if (!last) {  // activation backward and bias gradient
      const long rows = (long)nrhs * V;
      const int nb = (int)cdiv(rows, 128);
      DBuf bpart(sizeof(float) * nb * co, st);
      const float* b = net->params.as<float>() + woff + 2 * 9 * co * ci;
      with_dims(ci, co, [&](auto CI, auto CO) {
        (void)CI;
        MG_LAUNCH((k_nn_act_bwd<CO.value>), nb, 128, 0, st, net->zs[l].as<float2>(), b, gz, rows, bpart.as<float>());
      });
      MG_LAUNCH(k_nn_reduce_r, cdiv(co, 64), 64, 0, st, bpart.as<float>(), nb, co,
                net->grad.as<float>() + woff + 2 * 9 * co * ci);
    }
    const float2* a_in = l == 0 ? r : net->acts[l].as<float2>();
    const int chunks = (V + NN_WCH - 1) / NN_WCH;
    const int nblk = chunks * nrhs;
    const int cnt = 9 * co * ci;
    DBuf part(sizeof(float2) * (size_t)nblk * cnt, st);
    const size_t sm = sizeof(float2) * NN_WCH * (9 * ci + co);
    with_dims(ci, co, [&](auto CI, auto CO) {
      ensure_max_smem((const void*)k_nn_bwd_w<CI.value, CO.value>, 160 * 1024);
      MG_LAUNCH((k_nn_bwd_w<CI.value, CO.value>), nblk, 256, sm, st, net->T.as<float2>(), a_in, gz, L,
                part.as<float2>());
    });
    MG_LAUNCH(k_nn_reduce_c, cdiv(cnt, 128), 128, 0, st, part.as<float2>(), nblk, cnt,
              net->grad.as<float>() + woff);
    if (l > 0) {
      gprev.alloc(sizeof(float2) * (size_t)nrhs * V * ci, st);
      const __nv_bfloat16* W = net->w16.as<__nv_bfloat16>() + woff;
      with_dims(ci, co, [&](auto CI, auto CO) {
        MG_LAUNCH((k_nn_bwd_in<CI.value, CO.value>), dim3(cdiv(V, 128), nrhs), 128, 0, st, net->T.as<float2>(), gz, W,
                  gprev.as<float2>(), L);
      });
      g = std::move(gprev);
    }
  }
  (void)pinned;
  return loss;
}

void nn_adam(NNet* net, double lr, cudaStream_t st) {
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
  MG_LAUNCH(k_nn_adam, cdiv((long)net->nparams, 256), 256, 0, st, net->params.as<float>(), net->grad.as<float>(),
            net->m.as<float>(), net->v.as<float>(), (int)net->nparams, (float)lr, b1, b2, c1, c2, 1e-8f);
}

void nn_add(cudaStream_t st, float2* z, const float2* c, long n, int nrhs, const double* scale) {
  MG_LAUNCH(k_nn_add, dim3(std::min<long>(cdiv(n, 1024), 512), nrhs), 256, 0, st, z, c, n, scale);
}

}  // namespace mg
