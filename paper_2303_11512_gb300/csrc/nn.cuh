// Learned gauge-covariant preconditioner (see nn.cu).
#pragma once

#include <vector>

#include "ops.cuh"

namespace mg {

struct NNet {
  int L = 0, layers = 0, channels = 0;
  int tc = 0;                 // 1: tensor-core layers (BF16 operands, nn_tc.cu), 0: FP32 CUDA-core layers
  size_t nparams = 0;  // floats: per layer W[9][c_out][c_in] complex (interleaved), then b[c_out] (hidden layers)
  int step = 0;
  cudaStream_t st = 0;
  DBuf T;                     // transporters [site][9] complex64
  DBuf params, m, v, grad;    // FP32 master weights, Adam moments, gradient
  DBuf w16;                   // bf16 copy used by the forward/backward kernels
  std::vector<DBuf> acts, zs; // training tape (FP32 layer inputs, hidden pre-activations)
  std::vector<DBuf> acts16;   // tensor-core layers: BF16 layer inputs (the tape, or two ping-pong buffers)
  std::vector<DBuf> wimg;     // tensor-core weight images per layer: forward, conjugate-transposed
  DBuf err;                   // device int: set by a tensor-core kernel whose bounded wait expired
  int dim(int l) const;
  size_t w_offset(int l) const;
};

void nn_init(NNet* net, const double2* U, int L, int layers, int channels, uint64_t seed, cudaStream_t st);
// rebinds the net to another gauge field (lattice side L): new transporters, same weights and Adam state
void nn_bind_field(NNet* net, const double2* U, int L, cudaStream_t st);
// y = M(r), r/y fine-level fields [nrhs][site][2] complex64
void nn_forward(NNet* net, const float2* r, float2* y, int nrhs, bool tape, cudaStream_t st);
// loss (1/nrhs) sum ||M(r) - e||^2 / ||e||^2 and its gradient into net->grad
double nn_backward(NNet* net, const float2* r, const float2* e, int nrhs, cudaStream_t st, int* pinned);
void nn_adam(NNet* net, double lr, cudaStream_t st);
// z[rhs] += scale[rhs] * c[rhs]  (scale may be null: 1)
void nn_add(cudaStream_t st, float2* z, const float2* c, long n, int nrhs, const double* scale);
// raises MGMLMC_ERR_TIMEOUT (and clears the flag) when a tensor-core layer gave up waiting
void nn_check(NNet* net, cudaStream_t st);

// tensor-core layers (nn_tc.cu): lattice sides that are multiples of 16 (whole 128-site tiles per rhs)
bool nn_tc_supported(int L);
void nn_tc_weights(NNet* net, cudaStream_t st);
// y = M(r / rscale[rhs]) (rscale null: 1); with a tape the BF16 layer inputs and FP32 pre-activations are kept
void nn_tc_forward(NNet* net, const float2* r, const double* rscale, float2* y, int nrhs, bool tape, int* err,
                   cudaStream_t st);
// gradient into net->grad from the FP32 output gradient g (overwritten) of a taped forward
void nn_tc_backward(NNet* net, float2* g, int nrhs, int* err, cudaStream_t st);
// E = (x - v) / s[rhs], R = R / s[rhs]  (training pairs from the residual R, the solution x, the V-cycle v)
void nn_pair_finish(cudaStream_t st, float2* R, float2* E, const float2* x, const float2* v, const double* s, long n,
                    int nrhs);

}  // namespace mg
