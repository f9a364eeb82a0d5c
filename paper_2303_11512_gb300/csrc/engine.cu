// Host engine: hierarchy set-up, V-cycle, batched flexible GMRES with FP64
// iterative refinement, MG-MLMC level differences, Hutch++ sketch/projection
// and the Algorithm 2 driver.  Every arithmetic step is a kernel of ops_*.cu;
// the host only sequences launches and takes the per-batch decisions.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "engine.cuh"

namespace mg {

thread_local int64_t* g_launch_counter = nullptr;
thread_local KTimer* g_timer = nullptr;
thread_local int g_nact_hint = -1;

// ---------------------------------------------------------------- helpers
template <typename R> static inline const typename CT<R>::T* links_of(const LevelData& L) {
  if constexpr (sizeof(R) == 8) return L.links64.as<double2>(); else return L.links32.as<float2>();
}
template <typename R> static inline const typename CT<R>::T* st_of(const LevelData& L) {
  if constexpr (sizeof(R) == 8) return L.st64.as<double2>(); else return L.st32.as<float2>();
}
template <typename R> static inline const typename CT<R>::T* sapinv_of(const LevelData& L) {
  if constexpr (sizeof(R) == 8) return L.sapinv64.as<double2>(); else return L.sapinv32.as<float2>();
}
template <typename R> static inline const typename CT<R>::T* P_of(const LevelData& L) {
  if constexpr (sizeof(R) == 8) return L.P64.as<double2>(); else return L.P32.as<float2>();
}
template <typename R> static inline const typename CT<R>::T* inv_of(const LevelData& L) {
  if constexpr (sizeof(R) == 8) return L.inv64.as<double2>(); else return L.inv32.as<float2>();
}

static int read_flag(mgmlmc_ctx* ctx, const int* dflag) {
  MG_CUDA(cudaMemcpyAsync(ctx->pinned, dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  MG_CUDA(cudaStreamSynchronize(ctx->stream));
  return ctx->pinned[0];
}

// ---------------------------------------------------------------- operator pieces
template <typename R>
void op_apply(mgmlmc_hier* h, int l, const typename CT<R>::T* x, typename CT<R>::T* y, const typename CT<R>::T* b,
              int nrhs, const int* active) {
  const LevelData& L = h->lv[l];
  cudaStream_t st = h->ctx->stream;
  if (l == 0)
    wilson_apply<R>(st, links_of<R>(L), (R)L.diag, L.side, x, y, b, nrhs, active);
  else
    coarse_apply<R>(st, st_of<R>(L), L.side, L.dof, x, y, b, nrhs, active);
}

template <typename R>
void sap_sweep(mgmlmc_hier* h, int l, const typename CT<R>::T* f, typename CT<R>::T* x, int nrhs,
               const int* active, void* x16) {
  const LevelData& L = h->lv[l];
  cudaStream_t st = h->ctx->stream;
  if (sizeof(R) == 8 && !L.sap64_ok) throw Error(MGMLMC_ERR_INVALID_ARG, "FP64 SAP inverse not built at this level");
  if constexpr (sizeof(R) == 4) {
    if (h->use_tc(l) && L.sap_bs == 2 && L.tcInv[0].p) {
      float2* res = (float2*)h->work("tc_res", l, sizeof(float2) * L.n * nrhs);
      if (!x16 && tc_block_selected(L.tc_bf, L.side, nrhs)) {  // the block stencil reads a 16-bit copy of x
        x16 = h->work("sap_x16", l, sizeof(uint32_t) * L.n * nrhs);
        tc_round16(st, L.tc_bf, x, x16, L.side * L.side, nrhs);
      }
      for (int color = 0; color < 2; ++color)
        tc_sap_half(st, L.tcW.p, L.tcInv[color].p, L.tc_bf, L.side, f, x, x16, res, color, nrhs, active,
                    h->tc_err.as<int>());
      return;
    }
  }
  for (int color = 0; color < 2; ++color) {
    if (l == 0)
      sap_half_fine<R>(st, links_of<R>(L), (R)L.diag, L.side, L.sap_bs, sapinv_of<R>(L), f, x, color, nrhs, active,
                       sizeof(R) == 4 && L.sapinv32_t);
    else
      sap_half_coarse<R>(st, st_of<R>(L), L.side, L.dof, L.sap_bs, sapinv_of<R>(L), f, x, color, nrhs, active);
  }
}

template <typename R>
void restrict_level(mgmlmc_hier* h, int l, const typename CT<R>::T* xf, typename CT<R>::T* xc, int nrhs) {
  const LevelData& L = h->lv[l];
  restrict_op<R>(h->ctx->stream, P_of<R>(L), L.side, L.dof, h->prm.agg, h->prm.ntv, xf, xc, nrhs, nullptr);
}
template <typename R>
void prolong_level(mgmlmc_hier* h, int l, const typename CT<R>::T* xc, typename CT<R>::T* xf, int nrhs) {
  const LevelData& L = h->lv[l];
  prolong_op<R>(h->ctx->stream, P_of<R>(L), L.side, L.dof, h->prm.agg, h->prm.ntv, xc, xf, false, nrhs, nullptr);
}

template <typename R>
void vcycle(mgmlmc_hier* h, int l, const typename CT<R>::T* r, typename CT<R>::T* e, int nrhs, const int* active) {
  typedef typename CT<R>::T C;
  cudaStream_t st = h->ctx->stream;
  const LevelData& L = h->lv[l];
  if (l == h->nlev - 1) {
    if (sizeof(R) == 8 && !L.inv64_ok) throw Error(MGMLMC_ERR_INVALID_ARG, "FP64 coarsest inverse not built");
    dense_apply<R>(st, inv_of<R>(L), (int)L.n, r, e, nrhs, active);
    return;
  }
  const LevelData& Lc = h->lv[l + 1];
  const int pr = sizeof(R) == 8;
  C* res = (C*)h->work(pr ? "vc_res64" : "vc_res32", l, sizeof(C) * L.n * nrhs);
  C* rc = (C*)h->work(pr ? "vc_rc64" : "vc_rc32", l, sizeof(C) * Lc.n * nrhs);
  C* ec = (C*)h->work(pr ? "vc_ec64" : "vc_ec32", l, sizeof(C) * Lc.n * nrhs);
  // the 16-bit copy of e that the 2x2-block tensor-core stencil reads, kept up to date by every kernel that
  // writes e below (SAP block updates, the coarse-grid correction)
  void* e16 = nullptr;
  if constexpr (sizeof(R) == 4) {
    if (h->use_tc(l) && tc_block_selected(L.tc_bf, L.side, nrhs))
      e16 = h->work("vc_e16", l, sizeof(uint32_t) * L.n * nrhs);
  }
  vzero<C>(st, e, L.n, nrhs);
  if (e16) MG_CUDA(cudaMemsetAsync(e16, 0, sizeof(uint32_t) * L.n * nrhs, st));
  for (int s = 0; s < h->prm.pre_smooth; ++s) sap_sweep<R>(h, l, r, e, nrhs, active, e16);
  bool done = false;
  if constexpr (sizeof(R) == 4) {
    if (h->use_tc(l)) {  // res = r - D e on the tensor cores (preconditioner accuracy)
      if (h->prm.pre_smooth > 0 && L.sap_bs == 2 && L.tcInv[0].p)  // zero on the blocks the sweep solved last
        tc_residual_after_sap(st, L.tcW.p, L.tc_bf, L.side, e, e16, res, r, nrhs, active, h->tc_err.as<int>());
      else
        tc_stencil_apply(st, L.tcW.p, L.tc_bf, L.side, e, e16, res, r, nrhs, active, h->tc_err.as<int>());
      done = true;
    }
  }
  if (!done) op_apply<R>(h, l, e, res, r, nrhs, active);  // res = r - D e
  restrict_op<R>(st, P_of<R>(L), L.side, L.dof, h->prm.agg, h->prm.ntv, res, rc, nrhs, active);
  if (h->prm.kcycle_its > 0 && l + 1 < h->nlev - 1)  // K-cycle: a few FGMRES steps on level l+1
    fgmres_core<R>(h, l + 1, rc, ec, nrhs, h->prm.kcycle_its, h->prm.kcycle_tol, h->prm.kcycle_its, true, active,
                   nullptr, nullptr, nullptr);
  else
    vcycle<R>(h, l + 1, rc, ec, nrhs, active);
  prolong_op<R>(st, P_of<R>(L), L.side, L.dof, h->prm.agg, h->prm.ntv, ec, e, true, nrhs, active, e16, L.tc_bf);
  for (int s = 0; s < h->prm.post_smooth; ++s) sap_sweep<R>(h, l, r, e, nrhs, active, e16);
}

template void sap_sweep<float>(mgmlmc_hier*, int, const float2*, float2*, int, const int*, void*);
template void sap_sweep<double>(mgmlmc_hier*, int, const double2*, double2*, int, const int*, void*);
template void op_apply<float>(mgmlmc_hier*, int, const float2*, float2*, const float2*, int, const int*);
template void op_apply<double>(mgmlmc_hier*, int, const double2*, double2*, const double2*, int, const int*);
template void vcycle<float>(mgmlmc_hier*, int, const float2*, float2*, int, const int*);
template void vcycle<double>(mgmlmc_hier*, int, const double2*, double2*, int, const int*);
template void restrict_level<float>(mgmlmc_hier*, int, const float2*, float2*, int);
template void restrict_level<double>(mgmlmc_hier*, int, const double2*, double2*, int);
template void prolong_level<float>(mgmlmc_hier*, int, const float2*, float2*, int);
template void prolong_level<double>(mgmlmc_hier*, int, const double2*, double2*, int);

// ---------------------------------------------------------------- FGMRES
// Per-rhs bookkeeping kernels of the batched flexible GMRES(m).
__global__ void k_gm_init(const double* __restrict__ bn2, const int* __restrict__ act_in, int* act, double* bnorm,
                          int* its, double* relres, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const double b = sqrt(bn2[r]);
  bnorm[r] = b;
  act[r] = (b > 0.0) && isfinite(b) && (act_in ? act_in[r] : 1);
  relres[r] = isfinite(b) ? 0.0 : b;  // a NaN/Inf right-hand side is reported, not solved
  its[r] = 0;
}

__global__ void k_gm_cycle(const double* __restrict__ beta2, int* act, int* cact, int* iact, int* kvec,
                           double* beta, double2* g, const double* __restrict__ bnorm, const int* __restrict__ its,
                           double* relres, double tol, int maxit, int m, int nrhs, int* count) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  kvec[r] = 0;
  if (!act[r]) { cact[r] = 0; iact[r] = 0; return; }
  const double b = sqrt(beta2[r]);
  beta[r] = b;
  relres[r] = b / bnorm[r];
  const bool nanb = !(b == b) || isinf(b);
  if (b <= tol * bnorm[r] || its[r] >= maxit || nanb || b == 0.0) {
    act[r] = 0; cact[r] = 0; iact[r] = 0;
    if (nanb) relres[r] = b;
    return;
  }
  cact[r] = 1;
  iact[r] = 1;
  g[r] = make_double2(b, 0);
  for (int i = 1; i <= m; ++i) g[(size_t)i * nrhs + r] = make_double2(0, 0);
  atomicAdd(count, 1);
}

__global__ void k_gm_arnoldi(int j, int m, int nrhs, const double2* __restrict__ h1, const double2* __restrict__ h2,
                             const double* __restrict__ hn2, double* hn, double2* H, double* cs, double2* sn,
                             double2* g, int* iact, int* kvec, int* its, const double* __restrict__ bnorm,
                             double tol, int maxit, int* count) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs || !iact[r]) return;
  double2 col[65];
  for (int i = 0; i <= j; ++i) col[i] = cadd(h1[(size_t)i * nrhs + r], h2[(size_t)i * nrhs + r]);
  const double hh = sqrt(hn2[r]);
  col[j + 1] = make_double2(hh, 0);
  for (int i = 0; i < j; ++i) {
    const double c = cs[(size_t)i * nrhs + r];
    const double2 s = sn[(size_t)i * nrhs + r];
    const double2 a = col[i], b = col[i + 1];
    col[i] = cadd(cscale(a, c), cmul(s, b));
    col[i + 1] = csub(cscale(b, c), cmulc(s, a));
  }
  // new rotation zeroing col[j+1]
  const double2 a = col[j], b = col[j + 1];
  const double na = sqrt(a.x * a.x + a.y * a.y), nb = sqrt(b.x * b.x + b.y * b.y);
  double c;
  double2 s, rr;
  if (na == 0.0) {
    c = 0.0; s = make_double2(1, 0); rr = b;
  } else {
    const double t = sqrt(na * na + nb * nb);
    const double2 ph = make_double2(a.x / na, a.y / na);
    c = na / t;
    s = cscale(cmul(ph, cconj(b)), 1.0 / t);
    rr = cscale(ph, t);
  }
  cs[(size_t)j * nrhs + r] = c;
  sn[(size_t)j * nrhs + r] = s;
  col[j] = rr;
  for (int i = 0; i <= j; ++i) H[((size_t)i * m + j) * nrhs + r] = col[i];
  const double2 gj = g[(size_t)j * nrhs + r];
  g[(size_t)(j + 1) * nrhs + r] = cneg(cmulc(s, gj));
  g[(size_t)j * nrhs + r] = cscale(gj, c);
  const double2 gn = g[(size_t)(j + 1) * nrhs + r];
  const double res = sqrt(gn.x * gn.x + gn.y * gn.y);
  its[r] += 1;
  kvec[r] = j + 1;
  hn[r] = hh;
  if (res <= tol * bnorm[r] || its[r] >= maxit || hh == 0.0 || j + 1 == m || !(res == res)) {
    iact[r] = 0;
  } else {
    atomicAdd(count, 1);
  }
}

__global__ void k_gm_trisolve(int m, int nrhs, const double2* __restrict__ H, const double2* __restrict__ g,
                              const int* __restrict__ kvec, const int* __restrict__ cact, double2* y) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int k = cact[r] ? kvec[r] : 0;
  for (int i = m - 1; i >= 0; --i) {
    if (i >= k) { y[(size_t)i * nrhs + r] = make_double2(0, 0); continue; }
    double2 s = g[(size_t)i * nrhs + r];
    for (int q = i + 1; q < k; ++q) s = csub(s, cmul(H[((size_t)i * m + q) * nrhs + r], y[(size_t)q * nrhs + r]));
    const double2 d = H[((size_t)i * m + i) * nrhs + r];
    const double dn = d.x * d.x + d.y * d.y;
    y[(size_t)i * nrhs + r] = dn > 0 ? cscale(cmulc(d, s), 1.0 / dn) : make_double2(0, 0);
  }
}

// The V-cycle as a CUDA graph: a fixed launch sequence for a given (level, precision, nrhs, mask), captured
// once on fixed input/output buffers after an eager warm-up pass has allocated every workspace it touches,
// then replayed between two vector copies.  Not used while the per-kernel timer runs or with K-cycles
// (their host decisions cannot be captured); a graph is re-captured whenever a buffer it refers to changed.
template <typename R>
static void vcycle_maybe_graph(mgmlmc_hier* h, int l, const typename CT<R>::T* in_vec, typename CT<R>::T* out_vec,
                               int nrhs, const int* active) {
  typedef typename CT<R>::T C;
  if (!h->prm.graphs || g_timer || h->prm.kcycle_its > 0 || l == h->nlev - 1) {
    vcycle<R>(h, l, in_vec, out_vec, nrhs, active);
    return;
  }
  cudaStream_t st = h->ctx->stream;
  const long n = h->lv[l].n;
  const size_t bytes = sizeof(C) * n * nrhs;
  const bool dp = sizeof(R) == 8;
  C* gin = (C*)h->work(dp ? "vg_in64" : "vg_in32", l, bytes);
  C* gout = (C*)h->work(dp ? "vg_out64" : "vg_out32", l, bytes);
  auto& g = h->vgraphs[std::make_tuple(l, (int)sizeof(R), nrhs, (const void*)active)];
  if (g.exec && (g.gen != h->gen || g.in != gin || g.out != gout)) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.uses = 0;
  }
  if (!g.exec && g.uses == 0) {  // eager warm-up: allocates the workspaces of this shape
    vcycle<R>(h, l, in_vec, out_vec, nrhs, active);
    g.uses = 1;
    return;
  }
  if (!g.exec) {
    const uint64_t gen0 = h->gen;
    const int64_t before = g_launch_counter ? *g_launch_counter : 0;
    cudaGraph_t graph = nullptr;
    if (!h->capture_stream) MG_CUDA(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    cudaStream_t cs = h->capture_stream;
    MG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    h->ctx->stream = cs;  // the V-cycle's launches go to the capturing stream
    try {
      vcycle<R>(h, l, gin, gout, nrhs, active);
    } catch (...) {
      h->ctx->stream = st;
      h->capturing = false;
      cudaStreamEndCapture(cs, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      throw;
    }
    h->ctx->stream = st;
    h->capturing = false;
    MG_CUDA(cudaStreamEndCapture(cs, &graph));
    const int64_t captured = g_launch_counter ? *g_launch_counter - before : 0;
    if (g_launch_counter) *g_launch_counter = before;  // capturing issued nothing
    if (h->gen != gen0) {
      cudaGraphDestroy(graph);
      vcycle<R>(h, l, in_vec, out_vec, nrhs, active);
      return;
    }
    MG_CUDA(cudaGraphInstantiate(&g.exec, graph, 0));
    cudaGraphDestroy(graph);
    g.gen = h->gen;
    g.in = gin;
    g.out = gout;
    g.launches = captured;
  }
  MG_CUDA(cudaMemcpyAsync(gin, in_vec, bytes, cudaMemcpyDeviceToDevice, st));
  MG_CUDA(cudaGraphLaunch(g.exec, st));
  MG_CUDA(cudaMemcpyAsync(out_vec, gout, bytes, cudaMemcpyDeviceToDevice, st));
  if (g_launch_counter) *g_launch_counter += g.launches;
  ++g.uses;
}

template <typename R>
struct GmState {
  typedef typename CT<R>::T C;
  C *V, *Z;
  int *act, *cact, *iact, *kvec, *its, *count;
  double *bnorm, *beta, *beta2, *hn, *hn2, *cs, *relres;
  double2 *g, *H, *sn, *h1, *h2, *y;
  void* red;
};

template <typename R>
static GmState<R> gm_state(mgmlmc_hier* h, int l, int nrhs, int m) {
  typedef typename CT<R>::T C;
  GmState<R> s;
  const long n = h->lv[l].n;
  const char* tg = sizeof(R) == 8 ? "gm64" : "gm32";
  char* b = (char*)h->work(std::string(tg) + "_V", l, sizeof(C) * n * nrhs * (m + 1));
  s.V = (C*)b;
  s.Z = (C*)h->work(std::string(tg) + "_Z", l, sizeof(C) * n * nrhs * m);
  size_t ints = (size_t)nrhs * 6 + 8;
  int* ip = (int*)h->work(std::string(tg) + "_i", l, sizeof(int) * ints);
  s.act = ip; s.cact = ip + nrhs; s.iact = ip + 2 * nrhs; s.kvec = ip + 3 * nrhs; s.its = ip + 4 * nrhs;
  s.count = ip + 6 * nrhs;
  double* dp = (double*)h->work(std::string(tg) + "_d", l, sizeof(double) * (size_t)nrhs * (7 + m));
  s.bnorm = dp; s.beta = dp + nrhs; s.beta2 = dp + 2 * nrhs; s.hn = dp + 3 * nrhs; s.hn2 = dp + 4 * nrhs;
  s.relres = dp + 5 * nrhs; s.cs = dp + 7 * nrhs;
  double2* cp = (double2*)h->work(std::string(tg) + "_c", l,
                                  sizeof(double2) * (size_t)nrhs * ((m + 1) + (size_t)(m + 1) * m + m + 2 * (m + 1) + m));
  s.g = cp; cp += (size_t)(m + 1) * nrhs;
  s.H = cp; cp += (size_t)(m + 1) * m * nrhs;
  s.sn = cp; cp += (size_t)m * nrhs;
  s.h1 = cp; cp += (size_t)(m + 1) * nrhs;
  s.h2 = cp; cp += (size_t)(m + 1) * nrhs;
  s.y = cp;
  s.red = h->work(std::string(tg) + "_r", l, reduce_work_bytes(n, nrhs, m + 1));
  return s;
}

// Batched flexible GMRES(m), x0 = 0, each rhs stops at ||b - D x|| <= tol ||b||
// (true residual, checked at every restart) or after maxit inner iterations.
// Per-rhs iteration counts are added to its_acc (device, may be null).
template <typename R>
void fgmres_core(mgmlmc_hier* h, int l, const typename CT<R>::T* b, typename CT<R>::T* x, int nrhs, int m,
                 double tol, int maxit, int precond, const int* act_in, int* its_acc, double* relres_out,
                 int* cycles_out) {
  typedef typename CT<R>::T C;
  struct HintGuard {  // nested solves (K-cycle, bootstrap) restore the caller's hint
    int saved = g_nact_hint;
    ~HintGuard() { g_nact_hint = saved; }
  } hint_guard;
  mgmlmc_ctx* ctx = h->ctx;
  cudaStream_t st = ctx->stream;
  const long n = h->lv[l].n;
  MG_CHECK_ARG(m >= 1 && m <= 64, "FGMRES restart length must be 1..64");
  GmState<R> s = gm_state<R>(h, l, nrhs, m);
  const long vs = n * nrhs;
  const unsigned nb = cdiv(nrhs, 64);
  vnorm2<C>(st, b, n, nrhs, s.beta2, s.red, act_in);
  MG_LAUNCH(k_gm_init, nb, 64, 0, st, s.beta2, act_in, s.act, s.bnorm, s.its, s.relres, nrhs);
  vzero<C>(st, x, n, nrhs);
  int cycles = 0;
  for (;; ++cycles) {
    if (cycles == 0)
      vcopy<C>(st, b, s.V, n, nrhs);
    else
      op_apply<R>(h, l, x, s.V, b, nrhs, s.act);  // V0 = b - D x
    vnorm2<C>(st, s.V, n, nrhs, s.beta2, s.red, s.act);
    MG_CUDA(cudaMemsetAsync(s.count, 0, sizeof(int), st));
    MG_LAUNCH(k_gm_cycle, nb, 64, 0, st, s.beta2, s.act, s.cact, s.iact, s.kvec, s.beta, s.g, s.bnorm, s.its,
              s.relres, tol, maxit, m, nrhs, s.count);
    const int nstart = read_flag(ctx, s.count);
    if (nstart == 0) break;
    g_nact_hint = nstart;
    vscale_inv<C>(st, s.beta, s.V, s.V, n, nrhs, s.cact);
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      C* Vj = s.V + (size_t)j * vs;
      C* Vj1 = s.V + (size_t)(j + 1) * vs;
      C* Zj = s.Z + (size_t)j * vs;
      if (precond)
      {
        vcycle_maybe_graph<R>(h, l, Vj, Zj, nrhs, s.iact);
        if constexpr (sizeof(R) == 4) {
          if (precond == 2 && l == 0 && h->nn) {  // learned correction: z += |t| M(t / |t|), t = v - D z
            MG_CHECK_ARG(h->nn->L == h->L, "the attached network is bound to another lattice");
            C* tt = (C*)h->work("nn_t", l, sizeof(C) * n * nrhs);
            C* cc = (C*)h->work("nn_c", l, sizeof(C) * n * nrhs);
            double* tn = (double*)h->work("nn_n", l, sizeof(double) * nrhs);
            void* red = h->work("nn_red", l, reduce_work_bytes(n, nrhs, 1));
            op_apply<R>(h, l, Zj, tt, Vj, nrhs, s.iact);
            vnorm2<C>(st, tt, n, nrhs, tn, red, s.iact);
            sqrt_inplace(st, tn, nrhs);
            if (h->nn->tc) {  // the tensor-core net scales while rounding its input to BF16
              nn_tc_forward(h->nn, tt, tn, cc, nrhs, false, h->tc_err.as<int>(), st);
            } else {
              vscale_inv<C>(st, tn, tt, tt, n, nrhs, s.iact);
              nn_forward(h->nn, tt, cc, nrhs, false, st);
            }
            nn_add(st, Zj, cc, n, nrhs, tn);
          }
        }
      }
      else
        vcopy<C>(st, Vj, Zj, n, nrhs);
      op_apply<R>(h, l, Zj, Vj1, nullptr, nrhs, s.iact);
      vmultidot<C>(st, s.V, vs, j + 1, Vj1, n, nrhs, s.h1, s.red, s.iact);
      vgs_update_dot<C>(st, s.V, vs, j + 1, s.h1, Vj1, n, nrhs, s.h2, s.red, s.iact);
      vgs_update_norm<C>(st, s.V, vs, j + 1, s.h2, Vj1, n, nrhs, s.hn2, s.red, s.iact);
      MG_CUDA(cudaMemsetAsync(s.count, 0, sizeof(int), st));
      MG_LAUNCH(k_gm_arnoldi, nb, 64, 0, st, j, m, nrhs, s.h1, s.h2, s.hn2, s.hn, s.H, s.cs, s.sn, s.g, s.iact,
                s.kvec, s.its, s.bnorm, tol, maxit, s.count);
      jdone = j + 1;
      vscale_inv<C>(st, s.hn, Vj1, Vj1, n, nrhs, s.iact);
      const int nit = read_flag(ctx, s.count);
      if (nit == 0) break;
      g_nact_hint = nit;
    }
    g_nact_hint = nstart;
    MG_LAUNCH(k_gm_trisolve, nb, 64, 0, st, m, nrhs, s.H, s.g, s.kvec, s.cact, s.y);
    vcombine<C>(st, s.Z, vs, jdone, s.y, x, n, nrhs, s.cact);
    g_nact_hint = -1;
  }
  g_nact_hint = -1;
  if (its_acc) {
    // its_acc += its
    std::vector<int> a(nrhs), b2(nrhs);
    MG_CUDA(cudaMemcpyAsync(a.data(), s.its, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaMemcpyAsync(b2.data(), its_acc, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < nrhs; ++r) b2[r] += a[r];
    MG_CUDA(cudaMemcpyAsync(its_acc, b2.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
    MG_CUDA(cudaStreamSynchronize(st));
  }
  if (relres_out) MG_CUDA(cudaMemcpyAsync(relres_out, s.relres, sizeof(double) * nrhs, cudaMemcpyDeviceToDevice, st));
  if (cycles_out) *cycles_out = cycles;
}
template void fgmres_core<float>(mgmlmc_hier*, int, const float2*, float2*, int, int, double, int, int, const int*,
                                 int*, double*, int*);
template void fgmres_core<double>(mgmlmc_hier*, int, const double2*, double2*, int, int, double, int, int,
                                  const int*, int*, double*, int*);

__global__ void k_mixed_check(const double* __restrict__ rn2, const double* __restrict__ bn2, int* act,
                              double* scale, double* relres, double tol, int nrhs, int* count) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const double rn = sqrt(rn2[r]), bn = sqrt(bn2[r]);
  scale[r] = rn;
  if (!act[r]) return;
  relres[r] = bn > 0 ? rn / bn : 0.0;
  if (!(rn > tol * bn) || !(rn == rn)) {
    act[r] = 0;
    if (!(rn == rn)) relres[r] = rn;
    return;
  }
  atomicAdd(count, 1);
}

__global__ void k_init_act(const double* __restrict__ bn2, int* act, double* relres, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  act[r] = bn2[r] > 0.0 && isfinite(bn2[r]);
  relres[r] = isfinite(bn2[r]) ? 0.0 : bn2[r];  // a NaN/Inf right-hand side is reported, not solved
}

static SolveOut finish_out(mgmlmc_ctx* ctx, const int* its_dev, const double* relres_dev, int nrhs, double tol,
                           int cycles, const int* tc_err = nullptr) {
  SolveOut o;
  o.its.resize(nrhs);
  std::vector<double> rr(nrhs);
  int tcflag = 0;
  MG_CUDA(cudaMemcpyAsync(o.its.data(), its_dev, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  MG_CUDA(cudaMemcpyAsync(rr.data(), relres_dev, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  if (tc_err) MG_CUDA(cudaMemcpyAsync(&tcflag, tc_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  MG_CUDA(cudaStreamSynchronize(ctx->stream));
  if (tcflag) throw Error(MGMLMC_ERR_TIMEOUT, "a tensor-core kernel ran out of its bounded wait");
  o.outer = cycles;
  for (int r = 0; r < nrhs; ++r) {
    o.iters = std::max(o.iters, o.its[r]);
    o.total_iters += o.its[r];
    if (!std::isfinite(rr[r]))
      throw Error(MGMLMC_ERR_NAN, "a residual norm became NaN or infinite (right-hand side " + std::to_string(r) + ")");
    o.max_relres = std::max(o.max_relres, rr[r]);
    if (rr[r] > tol) o.converged = 0;
  }
  return o;
}

SolveOut solve(mgmlmc_hier* h, int l, const void* b, void* x, int nrhs, const solve_params& sp) {
  mgmlmc_ctx* ctx = h->ctx;
  cudaStream_t st = ctx->stream;
  const long n = h->lv[l].n;
  MG_CHECK_ARG(l >= 0 && l < h->nlev, "level out of range");
  if (l == h->nlev - 1) {  // coarsest: dense inverse, exact up to rounding
    if (sp.prec != MGMLMC_FP32 && !h->lv[l].inv64_ok)
      throw Error(MGMLMC_ERR_INVALID_ARG, "FP64 coarsest inverse not built");
    if (sp.prec == MGMLMC_FP32)
      dense_apply<float>(st, h->lv[l].inv32.as<float2>(), (int)n, (const float2*)b, (float2*)x, nrhs, nullptr);
    else
      dense_apply<double>(st, h->lv[l].inv64.as<double2>(), (int)n, (const double2*)b, (double2*)x, nrhs, nullptr);
    SolveOut o;
    o.its.assign(nrhs, 0);
    return o;
  }
  int* its = (int*)h->work("sv_its", l, sizeof(int) * nrhs);
  double* relres = (double*)h->work("sv_rr", l, sizeof(double) * nrhs);
  MG_CUDA(cudaMemsetAsync(its, 0, sizeof(int) * nrhs, st));
  const int pc = sp.precond;
  if (sp.prec == MGMLMC_FP64) {
    int cyc = 0;
    fgmres_core<double>(h, l, (const double2*)b, (double2*)x, nrhs, sp.m, sp.tol, sp.maxit, pc, nullptr, its, relres,
                        &cyc);
    return finish_out(ctx, its, relres, nrhs, sp.tol, cyc, h->tc_err.as<int>());
  }
  if (sp.prec == MGMLMC_FP32) {
    int cyc = 0;
    fgmres_core<float>(h, l, (const float2*)b, (float2*)x, nrhs, sp.m, sp.tol, sp.maxit, pc, nullptr, its, relres,
                       &cyc);
    return finish_out(ctx, its, relres, nrhs, sp.tol, cyc, h->tc_err.as<int>());
  }
  // MIXED: FP64 outer iterative refinement on the true residual, FP32 inner FGMRES
  MG_CHECK_ARG(sp.prec == MGMLMC_MIXED, "unknown precision");
  const double2* b64 = (const double2*)b;
  double2* x64 = (double2*)x;
  double2* r64 = (double2*)h->work("mx_r", l, sizeof(double2) * n * nrhs);
  float2* r32 = (float2*)h->work("mx_r32", l, sizeof(float2) * n * nrhs);
  float2* e32 = (float2*)h->work("mx_e32", l, sizeof(float2) * n * nrhs);
  double* dd = (double*)h->work("mx_d", l, sizeof(double) * 3 * nrhs);
  double *bn2 = dd, *rn2 = dd + nrhs, *scale = dd + 2 * nrhs;
  int* ip = (int*)h->work("mx_i", l, sizeof(int) * (nrhs + 2));
  int *act = ip, *count = ip + nrhs;
  void* red = h->work("mx_red", l, reduce_work_bytes(n, nrhs, 1));
  const unsigned nb = cdiv(nrhs, 64);
  vnorm2<double2>(st, b64, n, nrhs, bn2, red, nullptr);
  MG_LAUNCH(k_init_act, nb, 64, 0, st, bn2, act, relres, nrhs);
  vzero<double2>(st, x64, n, nrhs);
  const int max_outer = 30;
  int outer = 0, used = 0;
  for (;; ++outer) {
    if (outer == 0)
      vcopy<double2>(st, b64, r64, n, nrhs);
    else
      op_apply<double>(h, l, x64, r64, b64, nrhs, act);
    vnorm2<double2>(st, r64, n, nrhs, rn2, red, act);
    MG_CUDA(cudaMemsetAsync(count, 0, sizeof(int), st));
    MG_LAUNCH(k_mixed_check, nb, 64, 0, st, rn2, bn2, act, scale, relres, sp.tol, nrhs, count);
    const int nout = read_flag(ctx, count);
    if (nout == 0 || outer >= max_outer || used >= sp.maxit) break;
    g_nact_hint = nout;
    vconvert<float2, double2>(st, r64, r32, n, nrhs, scale, act);
    const int inner_max = std::min(sp.maxit - used, std::max(sp.m * 4, 8));
    int cyc = 0;
    fgmres_core<float>(h, l, r32, e32, nrhs, sp.m, sp.inner_tol, inner_max, pc, act, its, nullptr, &cyc);
    used += inner_max;
    vaccum_mixed<float>(st, scale, e32, x64, n, nrhs, act);
    g_nact_hint = nout;  // the next true residual covers the rhs active in this pass
  }
  g_nact_hint = -1;
  return finish_out(ctx, its, relres, nrhs, sp.tol, outer, h->tc_err.as<int>());
}

// ---------------------------------------------------------------- MG-MLMC level differences
SolveOut level_sample(mgmlmc_hier* h, int l, const double2* zeta, double2* y, int nrhs, const solve_params& sp) {
  MG_CHECK_ARG(l >= 0 && l + 1 < h->nlev, "level difference index out of range");
  cudaStream_t st = h->ctx->stream;
  const long n = h->lv[l].n, nc = h->lv[l + 1].n;
  solve_params s2 = sp;
  if (s2.prec == MGMLMC_FP32) s2.prec = MGMLMC_MIXED;  // samples are FP64 vectors
  double2* x1 = (double2*)h->work("ls_x1", l, sizeof(double2) * n * nrhs);
  double2* zc = (double2*)h->work("ls_zc", l, sizeof(double2) * nc * nrhs);
  double2* x2 = (double2*)h->work("ls_x2", l, sizeof(double2) * nc * nrhs);
  SolveOut o1 = solve(h, l, zeta, x1, nrhs, s2);
  restrict_level<double>(h, l, zeta, zc, nrhs);
  SolveOut o2 = solve(h, l + 1, zc, x2, nrhs, s2);
  prolong_level<double>(h, l, x2, y, nrhs);
  vsub_from(st, x1, y, n, nrhs);  // y = x1 - P x2
  SolveOut o = o1;
  o.converged = o1.converged && o2.converged;
  o.max_relres = std::max(o1.max_relres, o2.max_relres);
  o.iters = std::max(o1.iters, o2.iters);
  o.total_iters = o1.total_iters + o2.total_iters;
  // per-rhs cost proxy: iterations weighted by the nnz of each level's operator
  return o;
}

// non-zeros of D_m as the cost model counts them: 9 per fine row, a 5-point block stencil on coarse levels, the
// dense inverse on the coarsest level
static double level_nnz(const mgmlmc_hier* h, int m) {
  const LevelData& L = h->lv[m];
  if (m == h->nlev - 1) return (double)L.n * (double)L.n;
  return (double)L.n * (m == 0 ? 9.0 : 5.0 * L.dof);
}

// Level-difference applications of several levels at once (items with distinct levels).  Difference l needs
// solves on levels l and l+1, so the second term of difference m-1 and the first term of difference m fall on
// the same level m; each level is solved once with those right-hand sides side by side.  Every right-hand side
// is iterated independently (per-rhs masks, reductions and stopping), so each item's result and iteration
// counts are those of level_sample on its own.
void multi_level_sample(mgmlmc_hier* h, std::vector<LsItem>& items, const solve_params& sp) {
  cudaStream_t st = h->ctx->stream;
  solve_params s2 = sp;
  if (s2.prec == MGMLMC_FP32) s2.prec = MGMLMC_MIXED;  // samples are FP64 vectors
  const int nlev = h->nlev;
  struct Part { const double2* src; int nrhs, item, term; };
  std::vector<std::vector<Part>> parts(nlev);
  std::vector<double2*> x1(items.size()), x2(items.size());
  std::vector<int> seen(nlev, 0);
  for (size_t i = 0; i < items.size(); ++i) {
    const LsItem& it = items[i];
    MG_CHECK_ARG(it.l >= 0 && it.l + 1 < nlev, "level difference index out of range");
    MG_CHECK_ARG(!seen[it.l], "one item per level difference");
    seen[it.l] = 1;
    if (it.nrhs <= 0) continue;
    double2* zc = (double2*)h->work("mls_zc", it.l, sizeof(double2) * h->lv[it.l + 1].n * it.nrhs);
    restrict_level<double>(h, it.l, it.zeta, zc, it.nrhs);
    parts[it.l].push_back({it.zeta, it.nrhs, (int)i, 0});
    parts[it.l + 1].push_back({zc, it.nrhs, (int)i, 1});
  }
  std::vector<SolveOut> first(items.size()), second(items.size());
  std::vector<double> flops(items.size(), 0.0);
  for (int m = 0; m < nlev; ++m) {
    if (parts[m].empty()) continue;
    const long n = h->lv[m].n;
    int tot = 0;
    for (const Part& q : parts[m]) tot += q.nrhs;
    const double2* b = parts[m][0].src;
    if (parts[m].size() > 1) {
      double2* bb = (double2*)h->work("mls_b", m, sizeof(double2) * n * tot);
      int off = 0;
      for (const Part& q : parts[m]) {
        MG_CUDA(cudaMemcpyAsync(bb + (size_t)off * n, q.src, sizeof(double2) * n * q.nrhs, cudaMemcpyDeviceToDevice,
                                st));
        off += q.nrhs;
      }
      b = bb;
    }
    double2* x = (double2*)h->work("mls_x", m, sizeof(double2) * n * tot);
    SolveOut o = solve(h, m, b, x, tot, s2);
    int off = 0;
    for (const Part& q : parts[m]) {
      SolveOut& d = q.term == 0 ? first[q.item] : second[q.item];
      d = o;
      d.its.assign(o.its.begin() + off, o.its.begin() + off + q.nrhs);
      d.total_iters = 0;
      d.iters = 0;
      for (int v : d.its) { d.total_iters += v; d.iters = std::max(d.iters, v); }
      (q.term == 0 ? x1 : x2)[q.item] = x + (size_t)off * n;
      flops[q.item] += 8.0 * level_nnz(h, m) * (double)(d.total_iters + q.nrhs);
      off += q.nrhs;
    }
  }
  for (size_t i = 0; i < items.size(); ++i) {
    LsItem& it = items[i];
    if (it.nrhs <= 0) continue;
    prolong_level<double>(h, it.l, x2[i], it.y, it.nrhs);
    vsub_from(st, x1[i], it.y, h->lv[it.l].n, it.nrhs);  // y = x1 - P x2
    SolveOut o = first[i];
    o.converged = first[i].converged && second[i].converged;
    o.max_relres = std::max(first[i].max_relres, second[i].max_relres);
    o.iters = std::max(first[i].iters, second[i].iters);
    o.total_iters = first[i].total_iters + second[i].total_iters;
    it.out = o;
    it.flops = flops[i];
  }
}

void restrict_to_level(mgmlmc_hier* h, int l, const double2* zfine, double2* out, int nrhs) {
  cudaStream_t st = h->ctx->stream;
  if (l == 0) {
    vcopy<double2>(st, zfine, out, h->lv[0].n, nrhs);
    return;
  }
  const double2* src = zfine;
  for (int k = 0; k < l; ++k) {
    double2* dst = (k == l - 1) ? out
                                : (double2*)h->work((k & 1) ? "rt_b" : "rt_a", 0, sizeof(double2) * h->lv[k + 1].n * nrhs);
    restrict_level<double>(h, k, src, dst, nrhs);
    src = dst;
  }
}

void make_level_vectors(mgmlmc_hier* h, int l, int form, uint64_t seed, int phase, int64_t sample0, int nrhs,
                        double2* out, int noise) {
  cudaStream_t st = h->ctx->stream;
  if (form == MGMLMC_REDUCED || l == 0) {
    noise_fill(st, noise, seed, l, phase, sample0, h->lv[l].n, nrhs, out);
    return;
  }
  double2* zf = (double2*)h->work("mlv_fine", 0, sizeof(double2) * h->lv[0].n * nrhs);
  noise_fill(st, noise, seed, l, phase, sample0, h->lv[0].n, nrhs, zf);
  restrict_to_level(h, l, zf, out, nrhs);
}

SolveOut level_sample_accumulated(mgmlmc_hier* h, int l, const double2* zeta_fine, double2* y_fine, int nrhs,
                                  const solve_params& sp) {
  if (l == 0) return level_sample(h, 0, zeta_fine, y_fine, nrhs, sp);
  const long nl = h->lv[l].n;
  double2* zl = (double2*)h->work("lsa_z", l, sizeof(double2) * nl * nrhs);
  double2* yl = (double2*)h->work("lsa_y", l, sizeof(double2) * nl * nrhs);
  restrict_to_level(h, l, zeta_fine, zl, nrhs);
  SolveOut o = level_sample(h, l, zl, yl, nrhs, sp);
  const double2* src = yl;  // y_fine = P_0 ... P_{l-1} yl
  for (int k = l - 1; k >= 0; --k) {
    double2* dst = k == 0 ? y_fine : (double2*)h->work("lsa_p", k, sizeof(double2) * h->lv[k].n * nrhs);
    prolong_level<double>(h, k, src, dst, nrhs);
    src = dst;
  }
  return o;
}

// ---------------------------------------------------------------- Hutch++
void cholesky_qr2(mgmlmc_ctx* ctx, double2* Y, int d, long n) {
  cudaStream_t st = ctx->stream;
  void* work = ctx->work("cq_work", gram_work_bytes(d, n));
  double2* G = (double2*)ctx->work("cq_G", sizeof(double2) * d * d * 2);
  double2* Rinv = G + d * d;
  int* fail = (int*)ctx->work("cq_fail", sizeof(int));
  MG_CUDA(cudaMemsetAsync(fail, 0, sizeof(int), st));
  for (int pass = 0; pass < 2; ++pass) {
    gram(st, Y, d, n, G, work);
    chol_inv_upper(st, G, d, Rinv, fail);
    right_mul_upper(st, Y, d, n, Rinv);
  }
  if (read_flag(ctx, fail)) throw Error(MGMLMC_ERR_NOT_POSDEF, "CholeskyQR2: Gram matrix not positive definite");
}

mgmlmc_sketch* sketch_qr(mgmlmc_hier* h, int l, int d, int k, uint64_t seed, int form, const solve_params& sp,
                         double2* tau_lr) {
  MG_CHECK_ARG(d >= 1 && d <= SK_MAXD, "sketch size d must be 1..64");
  MG_CHECK_ARG(k >= 1, "at least one power sweep");
  cudaStream_t st = h->ctx->stream;
  const long n = h->lv[l].n;
  std::unique_ptr<mgmlmc_sketch> sk(new mgmlmc_sketch);
  sk->level = l; sk->d = d; sk->n = n; sk->st = st;
  sk->Q.alloc(sizeof(double2) * n * d, st);
  double2* S = sk->Q.as<double2>();
  double2* Y = (double2*)h->work("sk_Y", l, sizeof(double2) * n * d);
  make_level_vectors(h, l, form, seed, MGMLMC_PHASE_SKETCH, 0, d, S);
  for (int it = 0; it < k; ++it) {
    SolveOut o = level_sample(h, l, S, Y, d, sp);
    if (!o.converged) throw Error(MGMLMC_ERR_NOT_CONVERGED, "sketch solves did not converge");
    cholesky_qr2(h->ctx, Y, d, n);
    vcopy<double2>(st, Y, S, n, d);
  }
  SolveOut o = level_sample(h, l, S, Y, d, sp);
  if (!o.converged) throw Error(MGMLMC_ERR_NOT_CONVERGED, "low-rank solves did not converge");
  double2* dots = (double2*)h->work("sk_dots", l, sizeof(double2) * d);
  void* red = h->work("sk_red", l, reduce_work_bytes(n, d, 1));
  vdot<double2>(st, S, Y, n, d, dots, red, nullptr);
  std::vector<double2> hd(d);
  MG_CUDA(cudaMemcpyAsync(hd.data(), dots, sizeof(double2) * d, cudaMemcpyDeviceToHost, st));
  MG_CUDA(cudaStreamSynchronize(st));
  double2 t = make_double2(0, 0);
  for (int i = 0; i < d; ++i) t = cadd(t, hd[i]);
  *tau_lr = t;
  sk->tau = t;
  return sk.release();
}

// Exactly deflated Hutchinson (the paper's comparator, Section 2): the deflating subspace approximates the right
// singular vectors of D with the smallest singular values, i.e. the eigenvectors of the Hermitian gamma5 D with
// the smallest |mu|: block power method on Q^{-1} = D^{-1} gamma5, V <- CholeskyQR2(D^{-1} gamma5 V), from k
// Rademacher vectors (stream: seed, level 0, phase 4).  The direct part tr(V^H D^{-1} V) takes k more solves and
// is exact for any orthonormal V, so the estimator stays unbiased however far the iteration converged.
// residual = ||Y - V (V^H Y)||_F / ||Y||_F with Y = D^{-1} gamma5 V after the last sweep (0 for an invariant
// subspace), from ||Y||^2 - ||V^H Y||^2 (V orthonormal).
mgmlmc_sketch* deflation_basis(mgmlmc_hier* h, int k, int sweeps, uint64_t seed, const solve_params& sp0,
                               double* residual, int64_t* solves) {
  MG_CHECK_ARG(k >= 1 && k <= SK_MAXD, "deflation basis size must be 1..64");
  MG_CHECK_ARG(sweeps >= 1, "at least one sweep");
  mgmlmc_ctx* ctx = h->ctx;
  cudaStream_t st = ctx->stream;
  const long n = h->lv[0].n;
  solve_params sp = sp0;
  if (sp.prec == MGMLMC_FP32) sp.prec = MGMLMC_MIXED;  // FP64 basis
  std::unique_ptr<mgmlmc_sketch> sk(new mgmlmc_sketch);
  sk->level = 0; sk->d = k; sk->n = n; sk->st = st;
  sk->Q.alloc(sizeof(double2) * n * k, st);
  double2* V = sk->Q.as<double2>();
  double2* T = (double2*)h->work("df_T", 0, sizeof(double2) * n * k);
  double2* Y = (double2*)h->work("df_Y", 0, sizeof(double2) * n * k);
  rademacher_fill(st, seed, 0, 4, 0, n, k, V);
  int64_t ns = 0;
  auto solve_g5 = [&](const double2* in, double2* out) {  // out = D^{-1} gamma5 in
    vcopy<double2>(st, in, T, n, k);
    gamma5_apply(st, T, h->lv[0].dof, n, k);
    SolveOut o = solve(h, 0, T, out, k, sp);
    if (!o.converged) throw Error(MGMLMC_ERR_NOT_CONVERGED, "deflation-basis solves did not converge");
    ns += k;
  };
  for (int it = 0; it < sweeps; ++it) {
    solve_g5(V, Y);
    cholesky_qr2(ctx, Y, k, n);
    vcopy<double2>(st, Y, V, n, k);
  }
  // residual of the subspace
  solve_g5(V, Y);
  {
    double* yn = (double*)h->work("df_yn", 0, sizeof(double) * k);
    double2* G = (double2*)h->work("df_G", 0, sizeof(double2) * k * k);
    vnorm2<double2>(st, Y, n, k, yn, h->work("df_red", 0, reduce_work_bytes(n, k, 1)), nullptr);
    proj_coeffs(st, V, k, Y, n, k, G, h->work("df_pw", 0, proj_work_bytes(k, n, k)));
    std::vector<double> hy(k);
    std::vector<double2> hg((size_t)k * k);
    MG_CUDA(cudaMemcpyAsync(hy.data(), yn, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaMemcpyAsync(hg.data(), G, sizeof(double2) * k * k, cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    double ty = 0, tg = 0;
    for (double v : hy) ty += v;
    for (const double2& g : hg) tg += g.x * g.x + g.y * g.y;
    if (residual) *residual = ty > 0 ? std::sqrt(std::max(0.0, ty - tg) / ty) : 0.0;
  }
  // direct part tr(V^H D^{-1} V)
  {
    SolveOut o = solve(h, 0, V, Y, k, sp);
    if (!o.converged) throw Error(MGMLMC_ERR_NOT_CONVERGED, "deflation-trace solves did not converge");
    ns += k;
    double2* dots = (double2*)h->work("df_dots", 0, sizeof(double2) * k);
    vdot<double2>(st, V, Y, n, k, dots, h->work("df_red", 0, reduce_work_bytes(n, k, 1)), nullptr);
    std::vector<double2> hd(k);
    MG_CUDA(cudaMemcpyAsync(hd.data(), dots, sizeof(double2) * k, cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    double2 t = make_double2(0, 0);
    for (int i = 0; i < k; ++i) t = cadd(t, hd[i]);
    sk->tau = t;
  }
  if (solves) *solves = ns;
  return sk.release();
}

// The sketches of all level differences at once (Algorithm 2's deflation part for every l with d[l] > 0): the
// power sweeps and the low-rank traces of the levels advance together so that the solves of neighbouring
// differences on a shared level run as one batch (multi_level_sample).  Each level's Q and tau_lr equal those of
// sketch_qr for that level.
// With weight = MGMLMC_TRACE_GAMMA5 every level difference A_l is replaced by gamma5_l A_l (the matrix whose trace
// is estimated), so Y = gamma5_l A_l S and tau_lr = sum_i q_i^H gamma5_l A_l q_i.  `flops` accumulates the counted
// operator flops of the sketch solves.
void sketch_qr_all(mgmlmc_hier* h, const int* d, int k, uint64_t seed, int form, const solve_params& sp,
                   std::vector<std::unique_ptr<mgmlmc_sketch>>& out, std::vector<double2>& tau_lr, int noise,
                   int weight, double* flops) {
  MG_CHECK_ARG(k >= 1, "at least one power sweep");
  cudaStream_t st = h->ctx->stream;
  const int nd = h->nlev - 1;
  out.clear();
  out.resize(nd);
  tau_lr.assign(nd, make_double2(0, 0));
  std::vector<LsItem> items;
  std::vector<double2*> S(nd, nullptr), Y(nd, nullptr);
  for (int l = 0; l < nd; ++l) {
    if (d[l] <= 0) continue;
    MG_CHECK_ARG(d[l] <= SK_MAXD, "sketch size d must be 1..64");
    const long n = h->lv[l].n;
    out[l].reset(new mgmlmc_sketch);
    out[l]->level = l; out[l]->d = d[l]; out[l]->n = n; out[l]->st = st;
    out[l]->Q.alloc(sizeof(double2) * n * d[l], st);
    S[l] = out[l]->Q.as<double2>();
    Y[l] = (double2*)h->work("sk_Y", l, sizeof(double2) * n * d[l]);
    make_level_vectors(h, l, form, seed, MGMLMC_PHASE_SKETCH, 0, d[l], S[l], noise);
    LsItem it;
    it.l = l; it.zeta = S[l]; it.y = Y[l]; it.nrhs = d[l];
    items.push_back(it);
  }
  if (items.empty()) return;
  for (int sweep = 0; sweep <= k; ++sweep) {
    multi_level_sample(h, items, sp);
    for (const LsItem& it : items) {
      if (!it.out.converged)
        throw Error(MGMLMC_ERR_NOT_CONVERGED, sweep < k ? "sketch solves did not converge"
                                                        : "low-rank solves did not converge");
      if (flops) *flops += it.flops;
      if (weight == MGMLMC_TRACE_GAMMA5) gamma5_apply(st, Y[it.l], h->lv[it.l].dof, h->lv[it.l].n, it.nrhs);
    }
    if (sweep == k) break;
    for (const LsItem& it : items) {
      cholesky_qr2(h->ctx, Y[it.l], d[it.l], h->lv[it.l].n);
      vcopy<double2>(st, Y[it.l], S[it.l], h->lv[it.l].n, d[it.l]);
    }
  }
  for (const LsItem& it : items) {
    const int l = it.l;
    double2* dots = (double2*)h->work("sk_dots", l, sizeof(double2) * d[l]);
    void* red = h->work("sk_red", l, reduce_work_bytes(h->lv[l].n, d[l], 1));
    vdot<double2>(st, S[l], Y[l], h->lv[l].n, d[l], dots, red, nullptr);
    std::vector<double2> hd(d[l]);
    MG_CUDA(cudaMemcpyAsync(hd.data(), dots, sizeof(double2) * d[l], cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    double2 t = make_double2(0, 0);
    for (int i = 0; i < d[l]; ++i) t = cadd(t, hd[i]);
    tau_lr[l] = t;
    out[l]->tau = t;
  }
}

// tau_r = a_r - sum_i conj(c_ir) g_ir with c = Q^H zeta, g = Q^H y (stored after c), in a fixed order
__global__ void k_proj_combine(double2* __restrict__ a, const double2* __restrict__ c, int d, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  double2 t = a[r];
  for (int i = 0; i < d; ++i) t = csub(t, cmulc(c[(size_t)i * nrhs + r], c[(size_t)(d + i) * nrhs + r]));
  a[r] = t;
}

void project(mgmlmc_ctx* ctx, const mgmlmc_sketch* s, const double2* zeta, const double2* y, long n, int nrhs,
             double2* tau_host) {
  cudaStream_t st = ctx->stream;
  const int d = s ? s->d : 0;
  double2* a = (double2*)ctx->work("pj_a", sizeof(double2) * nrhs);
  vdot<double2>(st, zeta, y, n, nrhs, a, ctx->work("pj_red", reduce_work_bytes(n, nrhs, 1)), nullptr);
  if (d > 0) {
    MG_CHECK_ARG(s->n == n, "sketch and vectors differ in size");
    double2* c = (double2*)ctx->work("pj_c", sizeof(double2) * d * nrhs * 2);
    void* w = ctx->work("pj_w", proj_work_bytes(d, n, nrhs));
    proj_coeffs(st, s->Q.as<double2>(), d, zeta, n, nrhs, c, w);
    proj_coeffs(st, s->Q.as<double2>(), d, y, n, nrhs, c + (size_t)d * nrhs, w);
    MG_LAUNCH(k_proj_combine, cdiv(nrhs, 64), 64, 0, st, a, c, d, nrhs);
  }
  MG_CUDA(cudaMemcpyAsync(tau_host, a, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, st));
  MG_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------- Algorithm 2
int update_active(int nd, int* active, const double* V, const int64_t* N, const double* C, double eps,
                  double tau_abs, int policy, int min_samples) {
  for (int j = 0; j < nd; ++j)
    if (N[j] < 2) return 0;
  double denom = 0;
  for (int j = 0; j < nd; ++j) denom += std::sqrt(C[j] * V[j]);
  const double t2 = (eps * tau_abs) * (eps * tau_abs);
  int changed = 0;
  for (int l = 0; l < nd; ++l) {
    if (!active[l] || N[l] < min_samples) continue;
    double rho2;
    if (policy == MGMLMC_UNIFORM)
      rho2 = t2 / nd;
    else
      rho2 = (denom > 0 ? std::sqrt(C[l] * V[l]) / denom : 1.0 / nd) * t2;
    if (V[l] / (double)N[l] <= rho2) {
      active[l] = 0;
      changed = 1;
    }
  }
  return changed;
}

struct LevelStats {  // Welford on real and imaginary parts
  int64_t N = 0;
  double mr = 0, mi = 0, sr = 0, si = 0, csum = 0;
  void add(double2 t, double c) {
    ++N;
    const double dr = t.x - mr, di = t.y - mi;
    mr += dr / N;
    mi += di / N;
    sr += dr * (t.x - mr);
    si += di * (t.y - mi);
    csum += c;
  }
  double var() const { return N >= 2 ? (sr + si) / (N - 1) : NAN; }
  double cost() const { return N ? csum / N : 0; }
};

void estimate(mgmlmc_hier* h, const est_params& p, est_result* res) {
  mgmlmc_ctx* ctx = h->ctx;
  const int nd = h->nlev - 1;
  MG_CHECK_ARG(p.eps > 0, "eps must be positive");
  MG_CHECK_ARG(p.nrhs_max >= 1 && p.nrhs_first >= 1, "batch sizes must be positive");
  MG_CHECK_ARG(p.min_samples >= 2, "min_samples must be >= 2");
  std::memset(res, 0, sizeof(*res));
  res->nlev = h->nlev;
  std::vector<std::unique_ptr<mgmlmc_sketch>> sk;
  std::vector<double2> tau_lr;
  MG_CHECK_ARG(p.noise == MGMLMC_NOISE_RADEMACHER || p.noise == MGMLMC_NOISE_Z4, "unknown noise");
  MG_CHECK_ARG(p.weight == MGMLMC_TRACE_PLAIN || p.weight == MGMLMC_TRACE_GAMMA5, "unknown trace weight");
  const bool g5 = p.weight == MGMLMC_TRACE_GAMMA5;
  double flops = 0;
  sketch_qr_all(h, p.d, p.k, p.seed, p.form, p.solve, sk, tau_lr, p.noise, p.weight, &flops);
  for (int l = 0; l < nd; ++l)
    if (p.d[l] > 0) res->solves += (int64_t)2 * p.d[l] * (p.k + 1);
  const double2 tauL = g5 ? h->lv[h->nlev - 1].trace_g5 : h->lv[h->nlev - 1].trace;
  std::vector<std::vector<double2>> samp(nd);
  std::vector<std::vector<double>> scost(nd);
  std::vector<LevelStats> stats(nd);
  std::vector<int> active(nd, 1);
  int64_t s = 0;
  const int64_t maxs = p.max_samples > 0 ? p.max_samples : (int64_t)1 << 40;
  // one round: a batch of nb[l] new samples for every level with nb[l] > 0, all level differences applied
  // together (shared-level solves batched; each sample is the one level_sample would give)
  auto run_batches = [&](const std::vector<int>& nb) {
    std::vector<LsItem> items;
    for (int l = 0; l < nd; ++l) {
      if (nb[l] <= 0) continue;
      const long n = h->lv[l].n;
      LsItem it;
      it.l = l;
      it.nrhs = nb[l];
      double2* z = (double2*)h->work("est_z", l, sizeof(double2) * n * nb[l]);
      it.zeta = z;
      it.y = (double2*)h->work("est_y", l, sizeof(double2) * n * nb[l]);
      make_level_vectors(h, l, p.form, p.seed, MGMLMC_PHASE_STOCH, (int64_t)samp[l].size(), nb[l], z, p.noise);
      items.push_back(it);
    }
    if (items.empty()) return;
    multi_level_sample(h, items, p.solve);
    for (const LsItem& it : items) {
      const int l = it.l, b = it.nrhs;
      const SolveOut& o = it.out;
      if (!o.converged) throw Error(MGMLMC_ERR_NOT_CONVERGED, "sample solves did not converge");
      flops += it.flops;
      if (g5) gamma5_apply(ctx->stream, it.y, h->lv[l].dof, h->lv[l].n, b);
      std::vector<double2> t(b);
      project(ctx, sk[l].get(), it.zeta, it.y, h->lv[l].n, b, t.data());
      const double nnz_l = (double)h->lv[l].n * (l == 0 ? 9.0 : 5.0 * h->lv[l].dof);
      for (int r = 0; r < b; ++r) {
        samp[l].push_back(t[r]);
        scost[l].push_back(p.cost_mode == 1 ? (double)(o.its[r] + 1) * nnz_l : p.cost[l]);
      }
      res->solves += 2 * b;
      res->inner_iters += o.total_iters;
    }
  };
  auto batch_size = [&](int l) -> int {
    if (samp[l].empty()) return p.nrhs_first;
    // predicted samples from the current variances: V_l / rho_l^2
    bool ok = true;
    double denom = 0;
    for (int j = 0; j < nd; ++j) {
      if (stats[j].N < 2) ok = false; else denom += std::sqrt(stats[j].cost() * stats[j].var());
    }
    double tr;
    double tre = tauL.x, tim = tauL.y;
    for (int j = 0; j < nd; ++j) { tre += stats[j].mr + tau_lr[j].x; tim += stats[j].mi + tau_lr[j].y; }
    tr = std::hypot(tre, tim);
    int64_t want = p.nrhs_first;
    if (ok && denom > 0 && tr > 0) {
      const double rho2 = (p.policy == MGMLMC_UNIFORM ? 1.0 / nd
                                                       : std::sqrt(stats[l].cost() * stats[l].var()) / denom) *
                          (p.eps * tr) * (p.eps * tr);
      const double need = stats[l].var() / rho2;
      want = (int64_t)std::ceil(1.15 * need) - (int64_t)samp[l].size() + 1;
    }
    want = std::max<int64_t>(want, 8);
    want = ((want + 7) / 8) * 8;
    want = std::min<int64_t>(want, p.nrhs_max);
    want = std::min<int64_t>(want, maxs - (int64_t)samp[l].size());
    return (int)std::max<int64_t>(1, want);
  };
  while (s < maxs) {
    bool any = false;
    for (int l = 0; l < nd; ++l) any |= active[l] != 0;
    if (!any) break;
    std::vector<int> nb(nd, 0);
    for (int l = 0; l < nd; ++l)
      if (active[l] && (int64_t)samp[l].size() <= s) nb[l] = batch_size(l);
    run_batches(nb);
    ++s;
    for (int l = 0; l < nd; ++l)
      if (active[l]) stats[l].add(samp[l][s - 1], scost[l][s - 1]);
    double tre = tauL.x, tim = tauL.y;
    for (int l = 0; l < nd; ++l) { tre += stats[l].mr + tau_lr[l].x; tim += stats[l].mi + tau_lr[l].y; }
    std::vector<double> V(nd), C(nd);
    std::vector<int64_t> N(nd);
    for (int l = 0; l < nd; ++l) { V[l] = stats[l].var(); C[l] = stats[l].cost(); N[l] = stats[l].N; }
    update_active(nd, active.data(), V.data(), N.data(), C.data(), p.eps, std::hypot(tre, tim), p.policy,
                  p.min_samples);
  }
  double tre = tauL.x, tim = tauL.y, var = 0;
  for (int l = 0; l < nd; ++l) {
    const LevelStats& S = stats[l];
    res->N[l] = S.N;
    res->computed[l] = (int64_t)samp[l].size();
    res->mean[l][0] = S.mr;
    res->mean[l][1] = S.mi;
    res->V[l] = S.var();
    res->C[l] = S.cost();
    res->tau_lr[l][0] = tau_lr[l].x;
    res->tau_lr[l][1] = tau_lr[l].y;
    tre += S.mr + tau_lr[l].x;
    tim += S.mi + tau_lr[l].y;
    if (S.N >= 2) var += S.var() / S.N;
    if (p.sample_out[l]) {
      const int64_t cnt = std::min<int64_t>(p.sample_cap, (int64_t)samp[l].size());
      for (int64_t i = 0; i < cnt; ++i) {
        p.sample_out[l][2 * i] = samp[l][i].x;
        p.sample_out[l][2 * i + 1] = samp[l][i].y;
      }
    }
  }
  res->tau[0] = tre;
  res->tau[1] = tim;
  res->tau_L[0] = tauL.x;
  res->tau_L[1] = tauL.y;
  res->sigma = std::sqrt(var);
  res->steps = (int)s;
  res->flops = flops;
}

// ---------------------------------------------------------------- Algorithm 1
void hutchinson(mgmlmc_hier* h, const hutch_params& p, hutch_result* res) {
  mgmlmc_ctx* ctx = h->ctx;
  cudaStream_t st = ctx->stream;
  MG_CHECK_ARG(p.eps > 0, "eps must be positive");
  MG_CHECK_ARG(p.nrhs_max >= 1 && p.nrhs_first >= 1, "batch sizes must be positive");
  MG_CHECK_ARG(p.min_samples >= 2, "min_samples must be >= 2");
  MG_CHECK_ARG(p.noise == MGMLMC_NOISE_RADEMACHER || p.noise == MGMLMC_NOISE_Z4, "unknown noise");
  MG_CHECK_ARG(p.weight == MGMLMC_TRACE_PLAIN || p.weight == MGMLMC_TRACE_GAMMA5, "unknown trace weight");
  std::memset(res, 0, sizeof(*res));
  solve_params sp = p.solve;
  if (sp.prec == MGMLMC_FP32) sp.prec = MGMLMC_MIXED;  // samples are FP64 vectors
  const long n = h->lv[0].n;
  const mgmlmc_sketch* df = p.deflate;
  MG_CHECK_ARG(!df || (df->level == 0 && df->n == n), "deflation basis must be of the fine level");
  MG_CHECK_ARG(!df || p.weight == MGMLMC_TRACE_PLAIN, "deflation with the plain trace only");
  const double2 tdf = df ? df->tau : make_double2(0, 0);
  const int64_t maxs = p.max_samples > 0 ? p.max_samples : (int64_t)1 << 40;
  std::vector<double2> samp;
  LevelStats S;
  bool done = false;
  while (!done && (int64_t)samp.size() < maxs) {
    int64_t want = p.nrhs_first;
    if (S.N >= 2) {  // samples still needed by the current variance: V / (eps |tau|)^2
      const double t = std::hypot(S.mr + tdf.x, S.mi + tdf.y) * p.eps;
      if (t > 0) want = (int64_t)std::ceil(1.15 * S.var() / (t * t)) - S.N + 1;
      want = std::max<int64_t>(want, 8);
      want = ((want + 7) / 8) * 8;
    }
    want = std::min<int64_t>(std::min<int64_t>(want, p.nrhs_max), maxs - (int64_t)samp.size());
    const int b = (int)std::max<int64_t>(1, want);
    double2* z = (double2*)h->work("hu_z", 0, sizeof(double2) * n * b);
    double2* x = (double2*)h->work("hu_x", 0, sizeof(double2) * n * b);
    noise_fill(st, p.noise, p.seed, 0, MGMLMC_PHASE_HUTCH, (int64_t)samp.size(), n, b, z);
    SolveOut o = solve(h, 0, z, x, b, sp);
    if (!o.converged) throw Error(MGMLMC_ERR_NOT_CONVERGED, "Hutchinson solves did not converge");
    if (p.weight == MGMLMC_TRACE_GAMMA5) gamma5_apply(st, x, h->lv[0].dof, n, b);
    std::vector<double2> t(b);
    project(ctx, df, z, x, n, b, t.data());  // with a deflation basis: zeta^H (I - V V^H) D^{-1} zeta
    res->solves += b;
    res->inner_iters += o.total_iters;
    samp.insert(samp.end(), t.begin(), t.end());
    for (int r = 0; r < b && !done; ++r) {  // Algorithm 1, one sample at a time
      S.add(t[r], 0.0);
      if (S.N >= p.min_samples) {
        const double tol = std::hypot(S.mr + tdf.x, S.mi + tdf.y) * p.eps;
        if (S.var() / S.N <= tol * tol) done = true;
      }
    }
  }
  res->tau[0] = S.mr + tdf.x;
  res->tau[1] = S.mi + tdf.y;
  res->tau_defl[0] = tdf.x;
  res->tau_defl[1] = tdf.y;
  res->sigma = S.N >= 2 ? std::sqrt(S.var() / S.N) : NAN;
  res->N = S.N;
  res->computed = res->solves;
  if (p.sample_out) {
    const int64_t cnt = std::min<int64_t>(p.sample_cap, (int64_t)samp.size());
    for (int64_t i = 0; i < cnt; ++i) {
      p.sample_out[2 * i] = samp[i].x;
      p.sample_out[2 * i + 1] = samp[i].y;
    }
  }
}

}  // namespace mg
