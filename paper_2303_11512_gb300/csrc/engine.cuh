// Host-side engine: context, multigrid hierarchy, V-cycle, batched FGMRES,
// MG-MLMC level differences, Hutch++ sketches and the Algorithm 2 driver.
#pragma once

#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "nn.cuh"
#include "ops.cuh"

struct mgmlmc_ctx {
  cudaStream_t stream = 0;
  int device = 0;
  std::string err;
  int64_t launches = 0;
  int* pinned = nullptr;  // small pinned host buffer for flags
  double* pinned_d = nullptr;
  mg::KTimer timer;
  std::map<std::string, mg::DBuf> ws;  // workspaces of calls that have no hierarchy (projection)
  void* work(const std::string& tag, size_t bytes) {
    auto& b = ws[tag];
    if (bytes > b.bytes) b.alloc(bytes, stream);
    return b.p;
  }
};

namespace mg {

struct LevelData {
  int side = 0, dof = 0;
  long n = 0;
  // fine level
  DBuf links64, links32;
  double diag = 0;
  // coarse levels (and the coarsest, for mg_apply)
  DBuf st64, st32;
  // SAP smoother (all but the coarsest)
  int sap_bs = 0, sap_bd = 0;
  DBuf sapinv64, sapinv32;
  // test vectors (ntv x n, FP64) and the prolongator to the next coarser level
  DBuf tv;
  DBuf P64, P32;
  // tensor-core images (coarse levels with 16 dof): stencil and per-colour SAP block inverses
  DBuf tcW, tcInv[2];
  int tc_bf = 0;  // format of the tensor-core images: 0 TF32, 1 BF16, 2 FP16
  // coarsest level: dense inverse
  DBuf inv64, inv32;
  double2 trace = make_double2(0, 0);     // coarsest level: tr(D_L^{-1})
  double2 trace_g5 = make_double2(0, 0);  // coarsest level: tr(gamma5_L D_L^{-1})
  // FP64 SAP inverses / coarsest inverse current (intermediate bootstrap rounds build FP32 ones only)
  bool sap64_ok = false, inv64_ok = false;
  bool sapinv32_t = false;  // FP32 SAP inverses stored transposed (fine level)
};

}  // namespace mg

struct mgmlmc_hier {
  mgmlmc_ctx* ctx = nullptr;   // context of the most recent call (set by every entry point)
  cudaStream_t stream = 0;     // stream the hierarchy's memory is ordered on
  int L = 0;
  double m0 = 0;
  mg_params prm;
  int nlev = 0;
  std::vector<mg::LevelData> lv;
  std::map<std::tuple<std::string, int>, mg::DBuf> ws;  // workspaces
  mg::DBuf tc_err;  // device int: set by a tensor-core kernel whose bounded wait expired
  mg::NNet* nn = nullptr;  // learned fine-level correction (precond = 2), not owned
  bool use_tc(int l) const {
    return prm.tensor_cores && l >= 1 && l < nlev && lv[l].dof == 16 && lv[l].tcW.p != nullptr;
  }
  // generation of device buffers: bumped whenever a workspace is (re)allocated or the hierarchy is
  // rebuilt, so captured CUDA graphs that hold old pointers are never replayed
  uint64_t gen = 0;
  bool capturing = false;
  void* work(const std::string& tag, int level, size_t bytes) {
    auto& b = ws[std::make_tuple(tag, level)];
    if (bytes > b.bytes) {
      if (capturing) throw mg::Error(MGMLMC_ERR_INVALID_ARG, "workspace growth during graph capture");
      b.alloc(bytes, stream);
      ++gen;
    }
    return b.p;
  }
  // captured V-cycles: key (level, precision, nrhs, active mask) -> executable graph on fixed in/out buffers
  struct VGraph {
    cudaGraphExec_t exec = nullptr;
    void* in = nullptr;
    void* out = nullptr;
    uint64_t gen = 0;
    int64_t launches = 0;  // kernels per replay
    int uses = 0;
  };
  std::map<std::tuple<int, int, int, const void*>, VGraph> vgraphs;
  cudaStream_t capture_stream = nullptr;  // private stream to capture on (the legacy stream cannot be captured)
  void drop_graphs() {
    for (auto& kv : vgraphs)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    vgraphs.clear();
  }
  ~mgmlmc_hier() {
    drop_graphs();
    if (capture_stream) cudaStreamDestroy(capture_stream);
  }
};

struct mgmlmc_sketch {
  int level = 0, d = 0;
  long n = 0;
  mg::DBuf Q;  // [d][n] complex128
  cudaStream_t st = 0;
  double2 tau = make_double2(0, 0);  // direct part: tau_lr of a Hutch++ sketch, tr(Q^H D^{-1} Q) of a deflation basis
};

namespace mg {

// RAII binding of the launch counter to a context
struct LaunchScope {
  LaunchScope(mgmlmc_ctx* c) {
    g_launch_counter = &c->launches;
    g_timer = c->timer.on ? &c->timer : nullptr;
    g_nact_hint = -1;
  }
  ~LaunchScope() {
    g_launch_counter = nullptr;
    g_timer = nullptr;
    g_nact_hint = -1;
  }
};

void build_hierarchy(mgmlmc_ctx* ctx, mgmlmc_hier* h, const double2* U);

// One SAP sweep (colour 0 then 1) for D_l x = f.  x16: the planar 16-bit copy of x that the tensor-core sweep
// keeps up to date where the 2x2-block stencil is selected (tc_block_selected); nullptr makes the sweep derive
// one from x first.
template <typename R>
void sap_sweep(mgmlmc_hier* h, int l, const typename CT<R>::T* f, typename CT<R>::T* x, int nrhs, const int* active,
               void* x16 = nullptr);
// Batched flexible GMRES(m) in precision R, x0 = 0; see engine.cu.
template <typename R>
void fgmres_core(mgmlmc_hier* h, int l, const typename CT<R>::T* b, typename CT<R>::T* x, int nrhs, int m,
                 double tol, int maxit, int precond, const int* act_in, int* its_acc, double* relres_out,
                 int* cycles_out);

template <typename R>
void op_apply(mgmlmc_hier* h, int l, const typename CT<R>::T* x, typename CT<R>::T* y, const typename CT<R>::T* b,
              int nrhs, const int* active);
template <typename R>
void vcycle(mgmlmc_hier* h, int l, const typename CT<R>::T* r, typename CT<R>::T* e, int nrhs, const int* active);
template <typename R>
void restrict_level(mgmlmc_hier* h, int l, const typename CT<R>::T* xf, typename CT<R>::T* xc, int nrhs);
template <typename R>
void prolong_level(mgmlmc_hier* h, int l, const typename CT<R>::T* xc, typename CT<R>::T* xf, int nrhs);

struct SolveOut {
  int iters = 0, outer = 0, converged = 1;
  double max_relres = 0;
  int64_t total_iters = 0;
  std::vector<int> its;  // per rhs
};
// b, x device vectors in the precision implied by sp.prec (FP64 for MIXED)
SolveOut solve(mgmlmc_hier* h, int l, const void* b, void* x, int nrhs, const solve_params& sp);
// y = (D_l^{-1} - P_l D_{l+1}^{-1} P_l^H) zeta, FP64 vectors
SolveOut level_sample(mgmlmc_hier* h, int l, const double2* zeta, double2* y, int nrhs, const solve_params& sp);
// several level differences in one pass, solves on a shared level batched together (see engine.cu)
struct LsItem {
  int l = 0;
  const double2* zeta = nullptr;
  double2* y = nullptr;
  int nrhs = 0;
  SolveOut out;
  double flops = 0;  // counted operator flops of the item's solves: 8 nnz(D_m) (iterations + 1) per rhs
};
void multi_level_sample(mgmlmc_hier* h, std::vector<LsItem>& items, const solve_params& sp);
void restrict_to_level(mgmlmc_hier* h, int l, const double2* zfine, double2* out, int nrhs);
// fills zeta (level-l vectors, FP64) for samples sample0.. of level difference l
void make_level_vectors(mgmlmc_hier* h, int l, int form, uint64_t seed, int phase, int64_t sample0, int nrhs,
                        double2* out, int noise = MGMLMC_NOISE_RADEMACHER);
// the accumulated level difference on fine-size vectors: y = Phat_l A_l Rhat_l zeta
SolveOut level_sample_accumulated(mgmlmc_hier* h, int l, const double2* zeta_fine, double2* y_fine, int nrhs,
                                  const solve_params& sp);
void hutchinson(mgmlmc_hier* h, const hutch_params& p, hutch_result* r);
// time the launch variants of h's tunable kernels for these batch sizes and record the fastest (tune.cu)
void autotune(mgmlmc_hier* h, const std::vector<int>& nrhs_list, bool force);
// FMA throughput of the CUDA cores (FP64 or FP32), TFLOP/s, measured on the current device
double alu_peak_tflops(cudaStream_t st, bool fp64);
// block subspace iteration on D^{-1} gamma5 (fine level): the deflation basis of the exactly deflated Hutchinson
// comparator, its direct part tr(Q^H D^{-1} Q) in sk->tau and the relative residual of the invariant subspace
mgmlmc_sketch* deflation_basis(mgmlmc_hier* h, int k, int sweeps, uint64_t seed, const solve_params& sp,
                               double* residual, int64_t* solves);
// in-place CholeskyQR2 of Y = [d][n] (FP64): Y <- Q with Q^H Q = I, R with real positive diagonal
void cholesky_qr2(mgmlmc_ctx* ctx, double2* Y, int d, long n);
mgmlmc_sketch* sketch_qr(mgmlmc_hier* h, int l, int d, int k, uint64_t seed, int form, const solve_params& sp,
                         double2* tau_lr);
void project(mgmlmc_ctx* ctx, const mgmlmc_sketch* s, const double2* zeta, const double2* y, long n, int nrhs,
             double2* tau_host);
void estimate(mgmlmc_hier* h, const est_params& p, est_result* r);
int update_active(int nd, int* active, const double* V, const int64_t* N, const double* C, double eps,
                  double tau_abs, int policy, int min_samples);

}  // namespace mg
