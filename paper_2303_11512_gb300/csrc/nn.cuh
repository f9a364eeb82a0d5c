// Learned gauge-covariant preconditioner (see nn.cu).
#pragma once

#include <vector>

#include "ops.cuh"

namespace mg {

struct NNet {
  int L = 0, layers = 0, channels = 0;
  size_t nparams = 0;  // floats: per layer W[9][c_out][c_in] complex (interleaved), then b[c_out] (hidden layers)
  int step = 0;
  cudaStream_t st = 0;
  DBuf T;                     // transporters [site][9] complex64
  DBuf params, m, v, grad;    // FP32 master weights, Adam moments, gradient
  DBuf w16;                   // bf16 copy used by the forward/backward kernels
  std::vector<DBuf> acts, zs; // training tape
  int dim(int l) const;
  size_t w_offset(int l) const;
};

void nn_init(NNet* net, const double2* U, int L, int layers, int channels, uint64_t seed, cudaStream_t st);
// y = M(r), r/y fine-level fields [nrhs][site][2] complex64
void nn_forward(NNet* net, const float2* r, float2* y, int nrhs, bool tape, cudaStream_t st);
// loss (1/nrhs) sum ||M(r) - e||^2 / ||e||^2 and its gradient into net->grad
double nn_backward(NNet* net, const float2* r, const float2* e, int nrhs, cudaStream_t st, int* pinned);
void nn_adam(NNet* net, double lr, cudaStream_t st);
// z[rhs] += scale[rhs] * c[rhs]  (scale may be null: 1)
void nn_add(cudaStream_t st, float2* z, const float2* c, long n, int nrhs, const double* scale);

}  // namespace mg
