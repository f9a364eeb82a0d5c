// Multigrid set-up (Section 3.1 / Section 4): SAP block inverses, test
// vectors, orthonormal aggregation prolongators, Galerkin coarse stencils
// P^H D P, the coarsest dense inverse (its trace is tau_L of
// Algorithm 2), and the optional bootstrap rounds.
#include <algorithm>

#include <cmath>

#include "engine.cuh"

namespace mg {

static void to_fp32(cudaStream_t st, const DBuf& src, DBuf& dst, size_t count) {
  dst.alloc(count * sizeof(float2), st);
  vconvert<float2, double2>(st, src.as<double2>(), dst.as<float2>(), (long)count, 1, nullptr, nullptr);
}

static int default_levels(int L, int agg) {
  int lv = 1, side = L;
  while (side > 8 && side % (4 * agg) == 0) {
    side /= agg;
    ++lv;
  }
  return lv;
}

// SAP block inverses of level l: the block matrices in FP64, inverted in FP64 (FP32 copy alongside) or, for an
// intermediate bootstrap round whose hierarchy only serves FP32 solves, inverted in FP32 only
static void build_sap(mgmlmc_hier* h, int l, int* dfail, bool fp64) {
  cudaStream_t st = h->stream;
  LevelData& lv = h->lv[l];
  const int Ls = lv.side, d = lv.dof, bs = lv.sap_bs, bd = lv.sap_bd;
  const int nb = (Ls / bs) * (Ls / bs);
  lv.sapinv64.alloc(sizeof(double2) * (size_t)nb * bd * bd, st);
  if (l == 0)
    fine_block_matrices(st, lv.links64.as<double2>(), lv.diag, Ls, bs, lv.sapinv64.as<double2>());
  else
    coarse_block_matrices(st, lv.st64.as<double2>(), Ls, d, bs, lv.sapinv64.as<double2>());
  lv.sapinv32_t = false;
  if (fp64 && l == 0) {  // the fine CUDA-core smoother reads its FP32 inverses transposed
    invert_small_batched<double2>(st, lv.sapinv64.as<double2>(), nb, bd, dfail);
    lv.sapinv32.alloc(sizeof(float2) * (size_t)nb * bd * bd, st);
    blocks_to_fp32_transposed(st, lv.sapinv64.as<double2>(), nb, bd, lv.sapinv32.as<float2>());
    lv.sapinv32_t = true;
  } else if (fp64) {
    invert_small_batched<double2>(st, lv.sapinv64.as<double2>(), nb, bd, dfail);
    to_fp32(st, lv.sapinv64, lv.sapinv32, (size_t)nb * bd * bd);
  } else {
    to_fp32(st, lv.sapinv64, lv.sapinv32, (size_t)nb * bd * bd);
    invert_small_batched<float2>(st, lv.sapinv32.as<float2>(), nb, bd, dfail);
  }
  lv.sap64_ok = fp64;
  if (h->prm.tensor_cores && l >= 1 && d == 16 && bs == 2) {
    lv.tc_bf = h->prm.tensor_cores == 1 ? 1 : h->prm.tensor_cores == 3 ? 2 : 0;
    for (int c = 0; c < 2; ++c) {
      lv.tcInv[c].alloc(tc_blockinv_weight_bytes(Ls, lv.tc_bf), st);
      tc_blockinv_weights(st, lv.sapinv32.as<float2>(), Ls, c, lv.tcInv[c].p, lv.tc_bf);
    }
  }
}

// dense inverse of the coarsest level: FP64 with its trace (tau_L of Algorithm 2), or FP32 only for an
// intermediate bootstrap round
static void build_coarsest(mgmlmc_hier* h, int* dfail, bool fp64) {
  cudaStream_t st = h->stream;
  LevelData& lc = h->lv[h->nlev - 1];
  const int n = (int)lc.n;
  MG_CHECK_ARG(n <= 8192, "coarsest level too large for the dense inverse");
  lc.inv64.alloc(sizeof(double2) * (size_t)n * n, st);
  dense_from_stencil(st, lc.st64.as<double2>(), lc.side, lc.dof, lc.inv64.as<double2>());
  DBuf piv(sizeof(int) * n, st), work(invert_large_work_bytes(n), st), tr(2 * sizeof(double2), st);
  lc.inv64_ok = fp64;
  if (!fp64) {
    to_fp32(st, lc.inv64, lc.inv32, (size_t)n * n);
    invert_large<float2>(st, lc.inv32.as<float2>(), n, piv.as<int>(), work.p, dfail, dfail + 1);
    MG_CUDA(cudaStreamSynchronize(st));  // piv / work are released at return
    return;
  }
  invert_large<double2>(st, lc.inv64.as<double2>(), n, piv.as<int>(), work.p, dfail, dfail + 1);
  to_fp32(st, lc.inv64, lc.inv32, (size_t)n * n);
  trace_dense(st, lc.inv64.as<double2>(), n, tr.as<double2>());
  trace_dense(st, lc.inv64.as<double2>(), n, tr.as<double2>() + 1, lc.dof);
  double2 both[2];
  MG_CUDA(cudaMemcpyAsync(both, tr.p, 2 * sizeof(double2), cudaMemcpyDeviceToHost, st));
  MG_CUDA(cudaStreamSynchronize(st));
  lc.trace = both[0];
  lc.trace_g5 = both[1];
}

// P_l from the level-l test vectors lv.tv (ntv x n_l, FP64), D_{l+1} = P^H D_l P,
// then the smoother (or dense inverse) of level l+1.
static void build_from_tv(mgmlmc_hier* h, int l, int* dfail, bool sap64, bool coarsest64) {
  cudaStream_t st = h->stream;
  const mg_params& p = h->prm;
  LevelData& lv = h->lv[l];
  LevelData& lc = h->lv[l + 1];
  const int Ls = lv.side, d = lv.dof, ntv = p.ntv;
  const int Lc = Ls / p.agg, dc = 2 * ntv;
  const int bsz = p.agg * p.agg * d / 2;
  const size_t pcount = (size_t)Lc * Lc * 2 * bsz * ntv;
  lv.P64.alloc(sizeof(double2) * pcount, st);
  gather_tv_blocks(st, lv.tv.as<double2>(), Ls, d, p.agg, ntv, lv.P64.as<double2>());
  orthonormalise_blocks(st, lv.P64.as<double2>(), Lc * Lc * 2, bsz, ntv, dfail + 1);
  to_fp32(st, lv.P64, lv.P32, pcount);
  // Galerkin coarse operator, block by block
  {
    const size_t scount = (size_t)Lc * Lc * 5 * dc * dc;
    lc.st64.alloc(sizeof(double2) * scount, st);
    if (l == 0)
      galerkin(st, lv.links64.as<double2>(), true, lv.diag, Ls, d, p.agg, ntv, lv.P64.as<double2>(),
               lc.st64.as<double2>());
    else
      galerkin(st, lv.st64.as<double2>(), false, 0.0, Ls, d, p.agg, ntv, lv.P64.as<double2>(), lc.st64.as<double2>());
    to_fp32(st, lc.st64, lc.st32, scount);
    if (p.tensor_cores && dc == 16) {
      lc.tc_bf = p.tensor_cores == 1 ? 1 : p.tensor_cores == 3 ? 2 : 0;
      lc.tcW.alloc(tc_stencil_weight_bytes(Lc * Lc, lc.tc_bf), st);
      tc_stencil_weights(st, lc.st32.as<float2>(), Lc * Lc, lc.tcW.p, lc.tc_bf);
    }
  }
  if (l + 1 < h->nlev - 1)
    build_sap(h, l + 1, dfail + 0, sap64);
  else
    build_coarsest(h, dfail + 2, coarsest64);
  ++h->gen;  // operators changed: captured V-cycles must be rebuilt
}

static void check_fail(mgmlmc_hier* h, const int* dfail) {
  int fl[4];
  MG_CUDA(cudaMemcpyAsync(fl, dfail, sizeof(fl), cudaMemcpyDeviceToHost, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  if (fl[0]) throw Error(MGMLMC_ERR_NAN, "singular SAP block");
  if (fl[1]) throw Error(MGMLMC_ERR_NAN, "test-vector block of zero norm");
  if (fl[2]) throw Error(MGMLMC_ERR_NAN, "singular coarsest operator");
  if (fl[3]) throw Error(MGMLMC_ERR_TIMEOUT, "coarsest inversion: grid barrier timed out");
}

void build_hierarchy(mgmlmc_ctx* ctx, mgmlmc_hier* h, const double2* U) {
  cudaStream_t st = h->stream;
  const mg_params& p = h->prm;
  const int L = h->L;
  MG_CHECK_ARG(p.agg >= 2 && p.ntv >= 1 && 2 * p.ntv <= 32 && 256 % (2 * p.ntv) == 0,
               "mg_params: agg >= 2, 2*ntv must divide 256 and be <= 32");
  MG_CHECK_ARG(p.setup_sweeps >= 0 && p.pre_smooth >= 0 && p.post_smooth >= 0 && p.bootstrap >= 0 &&
                   p.kcycle_its >= 0 && p.kcycle_its <= 64 && p.bootstrap_its >= 1 && p.bootstrap_its <= 64,
               "mg_params: negative or too large iteration counts");
  h->nlev = p.levels > 0 ? p.levels : default_levels(L, p.agg);
  MG_CHECK_ARG(h->nlev >= 2 && h->nlev <= MGMLMC_MAX_LEVELS, "need 2..8 levels");
  h->lv.clear();
  h->lv.resize(h->nlev);
  {
    int side = L;
    for (int l = 0; l < h->nlev; ++l) {
      LevelData& lv = h->lv[l];
      lv.side = side;
      lv.dof = l == 0 ? 2 : 2 * p.ntv;
      lv.n = (long)side * side * lv.dof;
      if (l < h->nlev - 1) {
        const int bs = l == 0 ? p.sap_block_fine : p.sap_block_coarse;
        MG_CHECK_ARG(side % p.agg == 0 && side / p.agg >= 4, "every coarse side must be >= 4 and divide evenly");
        MG_CHECK_ARG(bs >= 1 && side % bs == 0 && (side / bs) % 2 == 0,
                     "SAP block must tile the level in an even grid");
        MG_CHECK_ARG(bs * bs * lv.dof <= 64, "SAP block dimension limited to 64");
        lv.sap_bs = bs;
        lv.sap_bd = bs * bs * lv.dof;
        side /= p.agg;
      }
    }
  }
  DBuf failbuf(sizeof(int) * 4, st);
  int* dfail = failbuf.as<int>();
  MG_CUDA(cudaMemsetAsync(dfail, 0, sizeof(int) * 4, st));
  h->tc_err.alloc(sizeof(int), st);
  MG_CUDA(cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), st));

  MG_CHECK_ARG(std::isfinite(h->m0), "m0 must be finite");
  check_links(st, U, L, dfail + 1);
  {
    int bad = 0;
    MG_CUDA(cudaMemcpyAsync(&bad, dfail + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    if (bad) throw Error(MGMLMC_ERR_NAN, "gauge field holds a NaN or infinite link");
  }
  LevelData& l0 = h->lv[0];
  l0.diag = h->m0 + 2.0;
  l0.links64.alloc(sizeof(double2) * 2 * L * L, st);
  l0.links32.alloc(sizeof(float2) * 2 * L * L, st);
  prepare_links(st, U, L, l0.links64.as<double2>(), l0.links32.as<float2>());
  build_sap(h, 0, dfail + 0, true);

  // initial phase: complex Rademacher test vectors smoothed by SAP sweeps for D_l v = 0
  const int ntv = p.ntv;
  for (int l = 0; l + 1 < h->nlev; ++l) {
    LevelData& lv = h->lv[l];
    const long n = lv.n;
    lv.tv.alloc(sizeof(double2) * n * ntv, st);
    complex_rademacher_fill(st, p.seed, l, MGMLMC_PHASE_TESTVEC, 0, n, ntv, lv.tv.as<double2>());
    if (p.bootstrap == 0) {  // this hierarchy is the final one: FP64 throughout
      DBuf f0(sizeof(double2) * n * ntv, st);
      vzero<double2>(st, f0.as<double2>(), n, ntv);
      for (int s = 0; s < p.setup_sweeps; ++s) sap_sweep<double>(h, l, f0.as<double2>(), lv.tv.as<double2>(), ntv, nullptr);
    } else {  // only a seed for the bootstrap rounds: smoothed in FP32
      DBuf f0(sizeof(float2) * n * ntv, st), t32(sizeof(float2) * n * ntv, st);
      vzero<float2>(st, f0.as<float2>(), n, ntv);
      vconvert<float2, double2>(st, lv.tv.as<double2>(), t32.as<float2>(), n, ntv, nullptr, nullptr);
      for (int s = 0; s < p.setup_sweeps; ++s) sap_sweep<float>(h, l, f0.as<float2>(), t32.as<float2>(), ntv, nullptr);
      vconvert<double2, float2>(st, t32.as<float2>(), lv.tv.as<double2>(), n, ntv, nullptr, nullptr);
    }
    // without bootstrap rounds this is the final hierarchy (FP64 inverses); otherwise FP32 inverses serve the
    // FP32 smoothing above and the bootstrap solves
    build_from_tv(h, l, dfail, p.bootstrap == 0, p.bootstrap == 0);
  }
  check_fail(h, dfail);

  // bootstrap rounds: inverse iteration with the current hierarchy as approximate inverse
  for (int it = 0; it < p.bootstrap; ++it) {
    for (int l = 0; l + 1 < h->nlev; ++l) {
      LevelData& lv = h->lv[l];
      const long n = lv.n;
      DBuf b32(sizeof(float2) * n * ntv, st), x32(sizeof(float2) * n * ntv, st), nrm(sizeof(double) * ntv, st);
      DBuf red(reduce_work_bytes(n, ntv, 1), st);
      vnorm2<double2>(st, lv.tv.as<double2>(), n, ntv, nrm.as<double>(), red.p, nullptr);
      sqrt_inplace(st, nrm.as<double>(), ntv);
      vconvert<float2, double2>(st, lv.tv.as<double2>(), b32.as<float2>(), n, ntv, nrm.as<double>(), nullptr);
      fgmres_core<float>(h, l, b32.as<float2>(), x32.as<float2>(), ntv, p.bootstrap_its, 1e-30, p.bootstrap_its, true,
                         nullptr, nullptr, nullptr, nullptr);
      vconvert<double2, float2>(st, x32.as<float2>(), lv.tv.as<double2>(), n, ntv, nullptr, nullptr);
      const bool final_round = it == p.bootstrap - 1;  // earlier rounds only feed FP32 bootstrap solves
      build_from_tv(h, l, dfail, final_round, final_round);
    }
    check_fail(h, dfail);
  }
  (void)ctx;
}

}  // namespace mg
