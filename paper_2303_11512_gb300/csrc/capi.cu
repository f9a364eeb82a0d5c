// extern "C" entry points of libmgmlmc (declared in include/mgmlmc.h).  Each
// call validates its arguments, binds the launch counter of its context, runs
// the engine and maps exceptions to status codes.
#include <cstring>

#include "engine.cuh"

using namespace mg;

namespace {

template <typename F>
int guarded(mgmlmc_ctx* ctx, F&& f) {
  if (!ctx) return MGMLMC_ERR_INVALID_ARG;
  LaunchScope scope(ctx);
  try {
    MG_CUDA(cudaSetDevice(ctx->device));
    f();
    ctx->err.clear();
    return MGMLMC_OK;
  } catch (const Error& e) {
    ctx->err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    ctx->err = "host allocation failed";
    return MGMLMC_ERR_OOM;
  } catch (const std::exception& e) {
    ctx->err = e.what();
    return MGMLMC_ERR_CUDA;
  }
}

void check_prec(int prec) {
  MG_CHECK_ARG(prec == MGMLMC_FP64 || prec == MGMLMC_FP32 || prec == MGMLMC_MIXED, "unknown precision");
}

}  // namespace

extern "C" {

int mgmlmc_version(void) { return 100; }

int mgmlmc_ctx_create(void* stream, mgmlmc_ctx** out) {
  if (!out) return MGMLMC_ERR_INVALID_ARG;
  *out = nullptr;
  mgmlmc_ctx* c = new (std::nothrow) mgmlmc_ctx;
  if (!c) return MGMLMC_ERR_OOM;
  c->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaMallocHost((void**)&c->pinned, 64) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MGMLMC_ERR_CUDA;
  }
  c->pinned_d = reinterpret_cast<double*>(c->pinned + 8);
  *out = c;
  return MGMLMC_OK;
}

void mgmlmc_ctx_destroy(mgmlmc_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  delete ctx;
}

const char* mgmlmc_last_error(const mgmlmc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t mgmlmc_launch_count(const mgmlmc_ctx* ctx) { return ctx ? ctx->launches : 0; }

int mgmlmc_alu_peak(mgmlmc_ctx* ctx, int fp64, double* tflops) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(tflops, "null pointer");
    *tflops = mg::alu_peak_tflops(ctx->stream, fp64 != 0);
  });
}

int mgmlmc_timing_enable(mgmlmc_ctx* ctx, int on, const char* filter) {
  if (!ctx) return MGMLMC_ERR_INVALID_ARG;
  ctx->timer.on = on != 0;
  ctx->timer.filter = filter ? filter : "";
  return MGMLMC_OK;
}

int mgmlmc_timing_report(mgmlmc_ctx* ctx, char* buf, int64_t len) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(buf && len > 0, "null buffer");
    struct Agg { int64_t n = 0; double ms = 0, bytes = 0, flops = 0; };
    std::map<std::string, Agg> agg;
    for (auto& r : ctx->timer.recs) {
      MG_CUDA(cudaEventSynchronize(r.b));
      float ms = 0;
      MG_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      std::string key = r.name;
      const char* w = std::strstr(r.where, "[with ");
      if (w) {  // append the launcher's template arguments, e.g. "[with R = float]"
        const char* e = std::strchr(w, ']');
        key += " ";
        key.append(w + 6, e ? (size_t)(e - w - 6) : std::strlen(w + 6));
      }
      Agg& a = agg[key];
      a.n += 1;
      a.ms += ms;
      a.bytes += r.bytes;
      a.flops += r.flops;
      ctx->timer.pool.push_back(r.a);
      ctx->timer.pool.push_back(r.b);
    }
    ctx->timer.recs.clear();
    std::string out;
    char line[512];
    for (auto& kv : agg) {
      std::snprintf(line, sizeof(line), "%s\t%lld\t%.6f\t%.6e\t%.6e\n", kv.first.c_str(), (long long)kv.second.n,
                    kv.second.ms, kv.second.bytes, kv.second.flops);
      out += line;
    }
    MG_CHECK_ARG((int64_t)out.size() < len, "report buffer too small");
    std::memcpy(buf, out.c_str(), out.size() + 1);
  });
}

int schwinger_apply(mgmlmc_ctx* ctx, const double* U, int L, double m0, const void* x, void* y, int nrhs, int prec) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(nrhs >= 0, "nrhs must be >= 0");
    if (nrhs == 0) return;
    MG_CHECK_ARG(U && x && y, "null pointer");
    MG_CHECK_ARG(L >= 4 && L % 2 == 0, "L must be even and >= 4");
    MG_CHECK_ARG(x != y, "x and y must not alias");
    check_prec(prec);
    if (nrhs == 0) return;
    cudaStream_t st = ctx->stream;
    DBuf l64(sizeof(double2) * 2 * L * L, st);
    DBuf l32(prec == MGMLMC_FP32 ? sizeof(float2) * 2 * L * L : 0, st);
    prepare_links(st, (const double2*)U, L, l64.as<double2>(), prec == MGMLMC_FP32 ? l32.as<float2>() : nullptr);
    if (prec == MGMLMC_FP32)
      wilson_apply<float>(st, l32.as<float2>(), (float)(m0 + 2.0), L, (const float2*)x, (float2*)y, nullptr, nrhs,
                          nullptr);
    else
      wilson_apply<double>(st, l64.as<double2>(), m0 + 2.0, L, (const double2*)x, (double2*)y, nullptr, nrhs,
                           nullptr);
  });
}

int mgmlmc_rademacher(mgmlmc_ctx* ctx, uint64_t seed, int level, int phase, int64_t sample0, int64_t n, int nrhs,
                      double* out) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(out, "null pointer");
    MG_CHECK_ARG(level >= 0 && level < 256 && phase >= 0 && phase < 256, "level/phase out of range");
    MG_CHECK_ARG(sample0 >= 0 && n >= 0 && nrhs >= 0, "negative size");
    if (n == 0 || nrhs == 0) return;
    rademacher_fill(ctx->stream, seed, level, phase, sample0, (long)n, nrhs, (double2*)out);
  });
}

int mgmlmc_noise(mgmlmc_ctx* ctx, int kind, uint64_t seed, int level, int phase, int64_t sample0, int64_t n,
                 int nrhs, double* out) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(out, "null pointer");
    MG_CHECK_ARG(kind == MGMLMC_NOISE_RADEMACHER || kind == MGMLMC_NOISE_Z4, "unknown noise");
    MG_CHECK_ARG(level >= 0 && level < 256 && phase >= 0 && phase < 256, "level/phase out of range");
    MG_CHECK_ARG(sample0 >= 0 && n >= 0 && nrhs >= 0, "negative size");
    if (n == 0 || nrhs == 0) return;
    noise_fill(ctx->stream, kind, seed, level, phase, sample0, (long)n, nrhs, (double2*)out);
  });
}

int mg_params_default(mg_params* p) {
  if (!p) return MGMLMC_ERR_INVALID_ARG;
  p->levels = 0;
  p->agg = 4;
  p->ntv = 8;
  p->sap_block_fine = 4;
  p->sap_block_coarse = 2;
  p->setup_sweeps = 4;
  p->pre_smooth = 1;
  p->post_smooth = 1;
  p->seed = 0;
  p->bootstrap = 0;
  p->bootstrap_its = 6;
  p->kcycle_its = 0;
  p->kcycle_tol = 0.1;
  p->tensor_cores = 2;
  p->graphs = 1;
  p->autotune = 0;
  return MGMLMC_OK;
}

int mg_setup(mgmlmc_ctx* ctx, const double* U, int L, double m0, const mg_params* params, mgmlmc_hier** out) {
  if (out) *out = nullptr;
  return guarded(ctx, [&] {
    MG_CHECK_ARG(U && out, "null pointer");
    MG_CHECK_ARG(L >= 16 && L % 16 == 0, "L must be a multiple of 16");
    std::unique_ptr<mgmlmc_hier> h(new mgmlmc_hier);
    h->ctx = ctx;
    h->stream = ctx->stream;
    h->L = L;
    h->m0 = m0;
    if (params)
      h->prm = *params;
    else
      mg_params_default(&h->prm);
    build_hierarchy(ctx, h.get(), (const double2*)U);
    if (h->prm.autotune) autotune(h.get(), {8, 16, 32, 64, 128, 256}, false);
    *out = h.release();
  });
}

void mg_destroy(mgmlmc_hier* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  delete h;
}

int mg_num_levels(const mgmlmc_hier* h) { return h ? h->nlev : MGMLMC_ERR_INVALID_ARG; }

int mg_level_info(const mgmlmc_hier* h, int level, int* side, int* dof, int64_t* n) {
  if (!h || level < 0 || level >= h->nlev) return MGMLMC_ERR_INVALID_ARG;
  if (side) *side = h->lv[level].side;
  if (dof) *dof = h->lv[level].dof;
  if (n) *n = h->lv[level].n;
  return MGMLMC_OK;
}

int mg_coarsest_trace(const mgmlmc_hier* h, double* tau_L) {
  if (!h || !tau_L) return MGMLMC_ERR_INVALID_ARG;
  tau_L[0] = h->lv[h->nlev - 1].trace.x;
  tau_L[1] = h->lv[h->nlev - 1].trace.y;
  return MGMLMC_OK;
}

// image format of a tensor-core precision: 0 TF32, 1 BF16, 2 FP16
static int tc_format_of(int prec) { return prec == MGMLMC_BF16 ? 1 : prec == MGMLMC_FP16 ? 2 : 0; }

int mg_apply(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* x, void* y, int nrhs, int prec) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && x && y && x != y, "null or aliased pointer");
    const_cast<mgmlmc_hier*>(h)->ctx = ctx;
    MG_CHECK_ARG(level >= 0 && level < h->nlev, "level out of range");
    const bool tc = prec == MGMLMC_TF32 || prec == MGMLMC_BF16 || prec == MGMLMC_FP16;
    MG_CHECK_ARG(!tc || (h->use_tc(level) && h->lv[level].tc_bf == tc_format_of(prec)),
                 "tensor-core apply needs a coarse level with 16 dof whose images have this format "
                 "(mg_params.tensor_cores: 1 BF16, 2 TF32, 3 FP16)");
    if (!tc) check_prec(prec);
    if (nrhs <= 0) return;
    if (tc) {
      const LevelData& L = h->lv[level];
      void* x16 = nullptr;
      if (tc_block_selected(L.tc_bf, L.side, nrhs)) {  // the block stencil reads a 16-bit copy of x
        x16 = h->work("ap_x16", level, sizeof(uint32_t) * L.n * nrhs);
        tc_round16(ctx->stream, L.tc_bf, (const float2*)x, x16, L.side * L.side, nrhs);
      }
      tc_stencil_apply(ctx->stream, L.tcW.p, L.tc_bf, L.side, (const float2*)x, x16, (float2*)y, nullptr, nrhs,
                       nullptr, h->tc_err.as<int>());
    }
    else if (prec == MGMLMC_FP32)
      op_apply<float>(h, level, (const float2*)x, (float2*)y, nullptr, nrhs, nullptr);
    else
      op_apply<double>(h, level, (const double2*)x, (double2*)y, nullptr, nrhs, nullptr);
  });
}

int mg_smooth(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* f, void* x, int nrhs, int prec, int sweeps) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && f && x && f != x, "null or aliased pointer");
    h->ctx = ctx;
    MG_CHECK_ARG(level >= 0 && level + 1 < h->nlev, "the coarsest level has no smoother");
    const bool tc = prec == MGMLMC_TF32 || prec == MGMLMC_BF16 || prec == MGMLMC_FP16;
    MG_CHECK_ARG(prec == MGMLMC_FP64 || prec == MGMLMC_FP32 || tc, "FP64, FP32, TF32, BF16 or FP16");
    MG_CHECK_ARG(!tc || (h->use_tc(level) && h->lv[level].tcInv[0].p && h->lv[level].tc_bf == tc_format_of(prec)),
                 "tensor-core smoothing needs a coarse level with 16 dof, 2x2 SAP blocks and images of this format");
    MG_CHECK_ARG(sweeps >= 0, "sweeps must be >= 0");
    if (nrhs <= 0) return;
    const int saved = h->prm.tensor_cores;
    h->prm.tensor_cores = tc ? saved : 0;
    try {
      for (int s = 0; s < sweeps; ++s) {
        if (prec == MGMLMC_FP64)
          sap_sweep<double>(h, level, (const double2*)f, (double2*)x, nrhs, nullptr);
        else
          sap_sweep<float>(h, level, (const float2*)f, (float2*)x, nrhs, nullptr);
      }
    } catch (...) {
      h->prm.tensor_cores = saved;
      throw;
    }
    h->prm.tensor_cores = saved;
  });
}

int mg_autotune(mgmlmc_ctx* ctx, mgmlmc_hier* h, const int* nrhs_list, int count, int force) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && nrhs_list && count > 0, "null pointer or empty list");
    h->ctx = ctx;
    std::vector<int> v(nrhs_list, nrhs_list + count);
    for (int n : v) MG_CHECK_ARG(n >= 1, "batch sizes must be positive");
    autotune(h, v, force != 0);
  });
}

int mgmlmc_tune_report(char* buf, int64_t len) {
  if (!buf || len <= 0) return MGMLMC_ERR_INVALID_ARG;
  const std::string t = tune_table_text();
  if ((int64_t)t.size() >= len) return MGMLMC_ERR_INVALID_ARG;
  std::memcpy(buf, t.c_str(), t.size() + 1);
  return MGMLMC_OK;
}

int mgmlmc_tune_set(int kind, int side, int bucket, int format, int variant) {
  if (kind < 0 || kind > 2 || side < 1 || bucket < 8 || bucket > 256 || (bucket & (bucket - 1)) || format < 0 ||
      format > 2 || variant < 0 || variant > 31)
    return MGMLMC_ERR_INVALID_ARG;
  if (kind == TUNE_WILSON32 && variant != 1 && variant != 2 && variant != 4) return MGMLMC_ERR_INVALID_ARG;
  // bit 4 (the 2x2-block stencil) exists for the 16-bit formats on sides divisible by 4 only
  if ((variant & 16) && (kind != TUNE_TC0 || format == 0 || side % 4)) return MGMLMC_ERR_INVALID_ARG;
  if (kind != TUNE_TC0 && variant > 15) return MGMLMC_ERR_INVALID_ARG;
  tune_store(kind, side, bucket, format, variant, 0.f);
  return MGMLMC_OK;
}

int mgmlmc_tune_clear(void) {
  tune_clear();
  return MGMLMC_OK;
}

int mg_tc_status(mgmlmc_ctx* ctx, mgmlmc_hier* h) {
  int flag = 0;
  int rc = guarded(ctx, [&] {
    MG_CHECK_ARG(h, "null hierarchy");
    MG_CUDA(cudaMemcpyAsync(&flag, h->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
  return rc != MGMLMC_OK ? rc : (flag ? MGMLMC_ERR_TIMEOUT : MGMLMC_OK);
}

int mg_restrict(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* xf, void* xc, int nrhs, int prec) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && xf && xc, "null pointer");
    const_cast<mgmlmc_hier*>(h)->ctx = ctx;
    MG_CHECK_ARG(level >= 0 && level + 1 < h->nlev, "level out of range");
    check_prec(prec);
    if (nrhs <= 0) return;
    if (prec == MGMLMC_FP32)
      restrict_level<float>(h, level, (const float2*)xf, (float2*)xc, nrhs);
    else
      restrict_level<double>(h, level, (const double2*)xf, (double2*)xc, nrhs);
  });
}

int mg_prolong(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* xc, void* xf, int nrhs, int prec) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && xf && xc, "null pointer");
    const_cast<mgmlmc_hier*>(h)->ctx = ctx;
    MG_CHECK_ARG(level >= 0 && level + 1 < h->nlev, "level out of range");
    check_prec(prec);
    if (nrhs <= 0) return;
    if (prec == MGMLMC_FP32)
      prolong_level<float>(h, level, (const float2*)xc, (float2*)xf, nrhs);
    else
      prolong_level<double>(h, level, (const double2*)xc, (double2*)xf, nrhs);
  });
}

int mg_get_prolongator(mgmlmc_ctx* ctx, const mgmlmc_hier* h, int level, double* host_out) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && host_out, "null pointer");
    MG_CHECK_ARG(level >= 0 && level + 1 < h->nlev, "level out of range");
    const LevelData& L = h->lv[level];
    MG_CUDA(cudaMemcpyAsync(host_out, L.P64.p, L.P64.bytes, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

int mg_get_stencil(mgmlmc_ctx* ctx, const mgmlmc_hier* h, int level, double* host_out) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && host_out, "null pointer");
    MG_CHECK_ARG(level >= 1 && level < h->nlev, "level out of range");
    const LevelData& L = h->lv[level];
    MG_CUDA(cudaMemcpyAsync(host_out, L.st64.p, L.st64.bytes, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

int mg_dense_inverse(mgmlmc_ctx* ctx, void* A, int n, int prec, int64_t barrier_polls) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(A, "null pointer");
    MG_CHECK_ARG(n >= 1 && n <= 8192, "n must be 1..8192");
    MG_CHECK_ARG(prec == MGMLMC_FP64 || prec == MGMLMC_FP32, "FP64 or FP32");
    cudaStream_t st = ctx->stream;
    DBuf piv(sizeof(int) * n, st), work(invert_large_work_bytes(n), st), flags(2 * sizeof(int), st);
    MG_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int), st));
    int* f = flags.as<int>();
    if (prec == MGMLMC_FP64)
      invert_large<double2>(st, (double2*)A, n, piv.as<int>(), work.p, f, f + 1, (long)barrier_polls);
    else
      invert_large<float2>(st, (float2*)A, n, piv.as<int>(), work.p, f, f + 1, (long)barrier_polls);
    int hf[2];
    MG_CUDA(cudaMemcpyAsync(hf, f, sizeof(hf), cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    if (hf[1]) throw Error(MGMLMC_ERR_TIMEOUT, "dense inverse: a grid-barrier wait ran out");
    if (hf[0]) throw Error(MGMLMC_ERR_NAN, "dense inverse: zero pivot (singular matrix)");
  });
}

int mg_vcycle(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* b, void* x, int nrhs, int prec) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && b && x && b != x, "null or aliased pointer");
    const_cast<mgmlmc_hier*>(h)->ctx = ctx;
    MG_CHECK_ARG(level >= 0 && level < h->nlev, "level out of range");
    MG_CHECK_ARG(prec == MGMLMC_FP64 || prec == MGMLMC_FP32, "V-cycle precision is FP64 or FP32");
    if (nrhs <= 0) return;
    if (prec == MGMLMC_FP32)
      vcycle<float>(h, level, (const float2*)b, (float2*)x, nrhs, nullptr);
    else
      vcycle<double>(h, level, (const double2*)b, (double2*)x, nrhs, nullptr);
  });
}

int solve_params_default(solve_params* p) {
  if (!p) return MGMLMC_ERR_INVALID_ARG;
  p->m = 16;
  p->tol = 1e-10;
  p->maxit = 2000;
  p->precond = 1;
  p->prec = MGMLMC_MIXED;
  p->inner_tol = 1e-5;
  return MGMLMC_OK;
}

static void fill_stats(const SolveOut& o, solve_stats* st) {
  if (!st) return;
  st->iters = o.iters;
  st->outer = o.outer;
  st->max_relres = o.max_relres;
  st->converged = o.converged;
  st->total_iters = o.total_iters;
}

int fgmres_batched(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const void* b, void* x, int nrhs,
                   const solve_params* sp, solve_stats* st, int* iters_out) {
  int nc = 0;
  int rc = guarded(ctx, [&] {
    MG_CHECK_ARG(h && b && x && sp && b != x, "null or aliased pointer");
    const_cast<mgmlmc_hier*>(h)->ctx = ctx;
    MG_CHECK_ARG(level >= 0 && level < h->nlev, "level out of range");
    MG_CHECK_ARG(sp->tol > 0 && sp->maxit > 0, "tol and maxit must be positive");
    check_prec(sp->prec);
    if (nrhs <= 0) return;
    SolveOut o = solve(h, level, b, x, nrhs, *sp);
    fill_stats(o, st);
    if (iters_out) std::memcpy(iters_out, o.its.data(), sizeof(int) * nrhs);
    nc = !o.converged;
  });
  if (rc == MGMLMC_OK && nc) {
    ctx->err = "fgmres_batched: not every right-hand side reached tol";
    return MGMLMC_ERR_NOT_CONVERGED;
  }
  return rc;
}

int mlmc_level_sample(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, int form, const double* zeta, double* y, int nrhs,
                      const solve_params* sp, solve_stats* st) {
  int nc = 0;
  int rc = guarded(ctx, [&] {
    MG_CHECK_ARG(h && zeta && y && sp && (const void*)zeta != (void*)y, "null or aliased pointer");
    const_cast<mgmlmc_hier*>(h)->ctx = ctx;
    MG_CHECK_ARG(level >= 0 && level + 1 < h->nlev, "level difference out of range");
    MG_CHECK_ARG(form == MGMLMC_ACCUMULATED || form == MGMLMC_REDUCED, "unknown form");
    if (nrhs <= 0) return;
    SolveOut o = form == MGMLMC_ACCUMULATED
                     ? level_sample_accumulated(h, level, (const double2*)zeta, (double2*)y, nrhs, *sp)
                     : level_sample(h, level, (const double2*)zeta, (double2*)y, nrhs, *sp);
    fill_stats(o, st);
    nc = !o.converged;
  });
  if (rc == MGMLMC_OK && nc) {
    ctx->err = "mlmc_level_sample: a solve did not reach tol";
    return MGMLMC_ERR_NOT_CONVERGED;
  }
  return rc;
}

int mg_restrict_to_level(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, const double* zeta_fine, double* out, int nrhs) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && zeta_fine && out, "null pointer");
    const_cast<mgmlmc_hier*>(h)->ctx = ctx;
    MG_CHECK_ARG(level >= 0 && level < h->nlev, "level out of range");
    if (nrhs <= 0) return;
    restrict_to_level(h, level, (const double2*)zeta_fine, (double2*)out, nrhs);
  });
}

int hutchpp_sketch_qr(mgmlmc_ctx* ctx, mgmlmc_hier* h, int level, int d, int k, uint64_t seed, int form,
                      const solve_params* sp, mgmlmc_sketch** out, double* tau_lr) {
  if (out) *out = nullptr;
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && sp && out && tau_lr, "null pointer");
    const_cast<mgmlmc_hier*>(h)->ctx = ctx;
    MG_CHECK_ARG(level >= 0 && level + 1 < h->nlev, "level difference out of range");
    MG_CHECK_ARG(form == MGMLMC_ACCUMULATED || form == MGMLMC_REDUCED, "unknown form");
    double2 t;
    *out = sketch_qr(h, level, d, k, seed, form, *sp, &t);
    tau_lr[0] = t.x;
    tau_lr[1] = t.y;
  });
}

void hutchpp_sketch_destroy(mgmlmc_sketch* s) {
  if (!s) return;
  cudaStreamSynchronize(s->st);
  delete s;
}

int hutchpp_cholqr2(mgmlmc_ctx* ctx, double* Y, int d, int64_t n) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(Y, "null pointer");
    MG_CHECK_ARG(d >= 1 && d <= SK_MAXD, "d must be 1..64");
    MG_CHECK_ARG(n >= d, "need n >= d");
    cholesky_qr2(ctx, (double2*)Y, d, (long)n);
  });
}

int hutchpp_sketch_get_q(mgmlmc_ctx* ctx, const mgmlmc_sketch* s, double* q_dev, int* d, int64_t* n) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(s, "null sketch");
    if (d) *d = s->d;
    if (n) *n = s->n;
    if (q_dev)
      MG_CUDA(cudaMemcpyAsync(q_dev, s->Q.p, sizeof(double2) * s->n * s->d, cudaMemcpyDeviceToDevice, ctx->stream));
  });
}

int hutchpp_project(mgmlmc_ctx* ctx, const mgmlmc_sketch* s, const double* zeta, const double* y, int64_t n, int nrhs,
                    double* tau_out) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(zeta && y && tau_out, "null pointer");
    MG_CHECK_ARG(n > 0, "n must be positive");
    if (nrhs <= 0) return;
    std::vector<double2> t(nrhs);
    project(ctx, s, (const double2*)zeta, (const double2*)y, (long)n, nrhs, t.data());
    std::memcpy(tau_out, t.data(), sizeof(double2) * nrhs);
  });
}

int est_params_default(est_params* p) {
  if (!p) return MGMLMC_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->eps = 1e-3;
  for (int l = 0; l < MGMLMC_MAX_LEVELS; ++l) {
    p->d[l] = 32;
    p->cost[l] = 1.0;
  }
  p->k = 2;
  p->nrhs_max = 256;
  p->nrhs_first = 32;
  p->policy = MGMLMC_OPTIMAL;
  p->form = MGMLMC_ACCUMULATED;
  p->seed = 0;
  p->cost_mode = 0;
  p->min_samples = 2;
  p->max_samples = 1 << 20;
  solve_params_default(&p->solve);
  p->noise = MGMLMC_NOISE_RADEMACHER;
  p->weight = MGMLMC_TRACE_PLAIN;
  return MGMLMC_OK;
}

int hutch_params_default(hutch_params* p) {
  if (!p) return MGMLMC_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->eps = 1e-2;
  p->nrhs_first = 32;
  p->nrhs_max = 256;
  p->noise = MGMLMC_NOISE_RADEMACHER;
  p->weight = MGMLMC_TRACE_PLAIN;
  p->min_samples = 2;
  p->max_samples = 1 << 20;
  solve_params_default(&p->solve);
  return MGMLMC_OK;
}

int deflation_basis(mgmlmc_ctx* ctx, mgmlmc_hier* h, int k, int sweeps, uint64_t seed, const solve_params* sp,
                    mgmlmc_sketch** out, double* tau_defl, double* residual) {
  if (out) *out = nullptr;
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && sp && out && tau_defl, "null pointer");
    h->ctx = ctx;
    MG_CHECK_ARG(sp->tol > 0 && sp->maxit > 0, "tol and maxit must be positive");
    check_prec(sp->prec);
    mgmlmc_sketch* s = deflation_basis(h, k, sweeps, seed, *sp, residual, nullptr);
    tau_defl[0] = s->tau.x;
    tau_defl[1] = s->tau.y;
    *out = s;
  });
}

int hutchinson_estimate(mgmlmc_ctx* ctx, mgmlmc_hier* h, const hutch_params* p, hutch_result* r) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && p && r, "null pointer");
    h->ctx = ctx;
    MG_CHECK_ARG(p->solve.tol > 0 && p->solve.maxit > 0, "tol and maxit must be positive");
    check_prec(p->solve.prec);
    hutchinson(h, *p, r);
  });
}

int trace_estimate(mgmlmc_ctx* ctx, mgmlmc_hier* h, const est_params* p, est_result* r) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && p && r, "null pointer");
    const_cast<mgmlmc_hier*>(h)->ctx = ctx;
    MG_CHECK_ARG(p->form == MGMLMC_ACCUMULATED || p->form == MGMLMC_REDUCED, "unknown form");
    estimate(h, *p, r);
  });
}

}  // extern "C"

struct mgmlmc_nn {
  mg::NNet net;
};

extern "C" {

int nn_create(mgmlmc_ctx* ctx, const double* U, int L, int layers, int channels, uint64_t seed, mgmlmc_nn** out) {
  if (out) *out = nullptr;
  return guarded(ctx, [&] {
    MG_CHECK_ARG(U && out, "null pointer");
    std::unique_ptr<mgmlmc_nn> nn(new mgmlmc_nn);
    nn_init(&nn->net, (const double2*)U, L, layers, channels, seed, ctx->stream);
    *out = nn.release();
  });
}

void nn_destroy(mgmlmc_nn* nn) {
  if (!nn) return;
  cudaStreamSynchronize(nn->net.st);
  delete nn;
}

int64_t nn_num_params(const mgmlmc_nn* nn) { return nn ? (int64_t)nn->net.nparams : MGMLMC_ERR_INVALID_ARG; }

int nn_set_params(mgmlmc_ctx* ctx, mgmlmc_nn* nn, const float* host) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(nn && host, "null pointer");
    MG_CUDA(cudaMemcpyAsync(nn->net.params.p, host, sizeof(float) * nn->net.nparams, cudaMemcpyHostToDevice,
                            ctx->stream));
    MG_CUDA(cudaMemsetAsync(nn->net.m.p, 0, sizeof(float) * nn->net.nparams, ctx->stream));
    MG_CUDA(cudaMemsetAsync(nn->net.v.p, 0, sizeof(float) * nn->net.nparams, ctx->stream));
    nn->net.step = 0;
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

int nn_get_params(mgmlmc_ctx* ctx, const mgmlmc_nn* nn, float* host) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(nn && host, "null pointer");
    MG_CUDA(cudaMemcpyAsync(host, nn->net.params.p, sizeof(float) * nn->net.nparams, cudaMemcpyDeviceToHost,
                            ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

int nn_forward(mgmlmc_ctx* ctx, mgmlmc_nn* nn, const void* r, void* y, int nrhs) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(nn && r && y && r != y, "null or aliased pointer");
    if (nrhs <= 0) return;
    mg::nn_forward(&nn->net, (const float2*)r, (float2*)y, nrhs, false, ctx->stream);
    if (nn->net.tc) mg::nn_check(&nn->net, ctx->stream);
  });
}

int nn_set_format(mgmlmc_ctx* ctx, mgmlmc_nn* nn, int format) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(nn, "null pointer");
    MG_CHECK_ARG(format == 0 || format == 1, "format: 0 FP32 CUDA cores, 1 BF16 tensor cores");
    MG_CHECK_ARG(format == 0 || mg::nn_tc_supported(nn->net.L), "tensor-core layers need L a multiple of 16");
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    nn->net.tc = format;
  });
}

int nn_get_format(const mgmlmc_nn* nn) { return nn ? nn->net.tc : MGMLMC_ERR_INVALID_ARG; }

int nn_set_field(mgmlmc_ctx* ctx, mgmlmc_nn* nn, const double* U, int L) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(nn && U, "null pointer");
    mg::nn_bind_field(&nn->net, (const double2*)U, L, ctx->stream);
  });
}

int nn_harvest_pairs(mgmlmc_ctx* ctx, mgmlmc_hier* h, uint64_t seed, int64_t sample0, int count, double tol,
                     void* R, void* E) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h && R && E && R != E, "null or aliased pointer");
    MG_CHECK_ARG(count >= 0 && sample0 >= 0, "negative count or sample index");
    MG_CHECK_ARG(tol > 0 && tol < 1, "tol must lie in (0, 1)");
    h->ctx = ctx;
    if (count == 0) return;
    cudaStream_t st = ctx->stream;
    const long n = h->lv[0].n;
    const int B = std::min(count, 64);
    DBuf z64(sizeof(double2) * n * B, st), z(sizeof(float2) * n * B, st), v(sizeof(float2) * n * B, st),
        x(sizeof(float2) * n * B, st), nrm(sizeof(double) * B, st), red(reduce_work_bytes(n, B, 1), st);
    solve_params sp;
    solve_params_default(&sp);
    sp.prec = MGMLMC_FP32;
    sp.tol = tol;
    sp.precond = 1;
    for (int s0 = 0; s0 < count; s0 += B) {
      const int nb = std::min(B, count - s0);
      float2* Rb = (float2*)R + (size_t)s0 * n;
      float2* Eb = (float2*)E + (size_t)s0 * n;
      rademacher_fill(st, seed, 0, MGMLMC_PHASE_HARVEST, sample0 + s0, n, nb, z64.as<double2>());
      vconvert<float2, double2>(st, z64.as<double2>(), z.as<float2>(), n, nb, nullptr, nullptr);
      vcycle<float>(h, 0, z.as<float2>(), v.as<float2>(), nb, nullptr);           // v = V(zeta)
      op_apply<float>(h, 0, v.as<float2>(), Rb, z.as<float2>(), nb, nullptr);    // r = zeta - D v
      solve(h, 0, z.p, x.p, nb, sp);                                              // x = D^{-1} zeta (FP32, tol)
      vnorm2<float2>(st, Rb, n, nb, nrm.as<double>(), red.p, nullptr);
      sqrt_inplace(st, nrm.as<double>(), nb);
      mg::nn_pair_finish(st, Rb, Eb, x.as<float2>(), v.as<float2>(), nrm.as<double>(), n, nb);
    }
    MG_CUDA(cudaStreamSynchronize(st));
  });
}

int nn_loss_grad(mgmlmc_ctx* ctx, mgmlmc_nn* nn, const void* r, const void* e, int nrhs, double* loss,
                 float* host_grad) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(nn && r && e && loss && nrhs > 0, "null pointer or empty batch");
    *loss = mg::nn_backward(&nn->net, (const float2*)r, (const float2*)e, nrhs, ctx->stream, ctx->pinned);
    if (nn->net.tc) mg::nn_check(&nn->net, ctx->stream);
    if (host_grad) {
      MG_CUDA(cudaMemcpyAsync(host_grad, nn->net.grad.p, sizeof(float) * nn->net.nparams, cudaMemcpyDeviceToHost,
                              ctx->stream));
      MG_CUDA(cudaStreamSynchronize(ctx->stream));
    }
  });
}

int nn_train_step(mgmlmc_ctx* ctx, mgmlmc_nn* nn, const void* r, const void* e, int nrhs, double lr, double* loss) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(nn && r && e && loss && nrhs > 0 && lr > 0, "bad arguments");
    *loss = mg::nn_backward(&nn->net, (const float2*)r, (const float2*)e, nrhs, ctx->stream, ctx->pinned);
    if (nn->net.tc) mg::nn_check(&nn->net, ctx->stream);
    mg::nn_adam(&nn->net, lr, ctx->stream);
  });
}

int mg_attach_nn(mgmlmc_ctx* ctx, mgmlmc_hier* h, mgmlmc_nn* nn) {
  return guarded(ctx, [&] {
    MG_CHECK_ARG(h, "null hierarchy");
    MG_CHECK_ARG(!nn || nn->net.L == h->L, "network and hierarchy lattices differ");
    h->nn = nn ? &nn->net : nullptr;
  });
}

int mlmc_update_active(int nd, int* active, const double* V, const int64_t* N, const double* C, double eps,
                       double tau_abs, int policy, int min_samples) {
  if (nd <= 0 || nd > MGMLMC_MAX_LEVELS || !active || !V || !N || !C) return MGMLMC_ERR_INVALID_ARG;
  update_active(nd, active, V, N, C, eps, tau_abs, policy, min_samples);
  return MGMLMC_OK;
}

}  // extern "C"
