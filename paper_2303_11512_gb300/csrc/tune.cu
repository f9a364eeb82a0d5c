// Launch-shape autotuner.  Some kernels have several launch variants that compute the same result (the
// tensor-core coarse operators: MMA tile rows and pipeline depth; the fine stencil: right-hand sides per
// thread).  Which one is fastest depends on the level's shape and the batch size, so the library keeps a
// process-wide table  (device, kernel, lattice side, batch bucket, weight format) -> variant  that every launch
// consults (unknown keys take the default variant), and mg_autotune fills it by timing every variant with CUDA
// events on scratch vectors.  Entries persist for the life of the process, so later hierarchies of the same
// shape (an ensemble of fields) reuse them; tune_report / tune_set export and import the table.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "engine.cuh"

namespace mg {
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, std::pair<int, float>> g_tune;  // -> (variant, microseconds)
}  // namespace

int tune_bucket(int nrhs) {
  int b = 8;
  while (b < nrhs && b < 256) b <<= 1;
  return b;
}

int tune_lookup(int kind, int shape, int nrhs, int fmt, int dflt) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(dev, kind, shape, tune_bucket(nrhs), fmt));
  return it == g_tune.end() ? dflt : it->second.first;
}

void tune_store(int kind, int shape, int bucket, int fmt, int variant, float us) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[std::make_tuple(dev, kind, shape, bucket, fmt)] = std::make_pair(variant, us);
}

bool tune_known(int kind, int shape, int bucket, int fmt) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return g_tune.count(std::make_tuple(dev, kind, shape, bucket, fmt)) != 0;
}

void tune_clear() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto it = g_tune.begin(); it != g_tune.end();) it = std::get<0>(it->first) == dev ? g_tune.erase(it) : ++it;
}

std::string tune_table_text() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  std::string out;
  char line[160];
  for (auto& kv : g_tune) {
    std::snprintf(line, sizeof(line), "%d\t%d\t%d\t%d\t%d\t%d\t%.3f\n", std::get<0>(kv.first), std::get<1>(kv.first),
                  std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first), kv.second.first,
                  kv.second.second);
    out += line;
  }
  return out;
}

// time fn() (median of `reps` after one warm-up call), microseconds
template <typename F>
static float time_us(cudaStream_t st, F&& fn, int reps = 5) {
  cudaEvent_t a, b;
  MG_CUDA(cudaEventCreate(&a));
  MG_CUDA(cudaEventCreate(&b));
  fn();
  std::vector<float> t;
  for (int r = 0; r < reps; ++r) {
    MG_CUDA(cudaEventRecord(a, st));
    fn();
    MG_CUDA(cudaEventRecord(b, st));
    MG_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    MG_CUDA(cudaEventElapsedTime(&ms, a, b));
    t.push_back(ms * 1e3f);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

// Tune every tunable launch of hierarchy h for the given batch sizes: the fine FP32 stencil (level 0) and, on
// coarse levels with tensor-core images, the stencil apply (MODE 0) and the SAP block-inverse update (MODE 1).
// Keys already in the table are kept unless `force`.
void autotune(mgmlmc_hier* h, const std::vector<int>& nrhs_list, bool force) {
  cudaStream_t st = h->ctx->stream;
  int* err = h->tc_err.as<int>();
  for (int nr : nrhs_list) {
    const int bucket = tune_bucket(nr);
    // fine stencil
    {
      const LevelData& L0 = h->lv[0];
      if (force || !tune_known(TUNE_WILSON32, L0.side, bucket, 0)) {
        DBuf x(sizeof(float2) * L0.n * bucket, st), y(sizeof(float2) * L0.n * bucket, st);
        vzero<float2>(st, x.as<float2>(), L0.n, bucket);
        int best = 1;
        float tbest = 1e30f;
        for (int v : {1, 2, 4}) {
          tune_store(TUNE_WILSON32, L0.side, bucket, 0, v, 0.f);
          const float t = time_us(st, [&] {
            wilson_apply<float>(st, L0.links32.as<float2>(), (float)L0.diag, L0.side, x.as<float2>(), y.as<float2>(),
                                nullptr, bucket, nullptr);
          });
          if (t < tbest) { tbest = t; best = v; }
        }
        tune_store(TUNE_WILSON32, L0.side, bucket, 0, best, tbest);
      }
    }
    for (int l = 1; l < h->nlev - 1; ++l) {
      LevelData& L = h->lv[l];
      if (!h->use_tc(l) || !L.tcInv[0].p) continue;
      const int fmt = L.tc_bf;
      DBuf x(sizeof(float2) * L.n * bucket, st), y(sizeof(float2) * L.n * bucket, st),
          f(sizeof(float2) * L.n * bucket, st), x16(fmt ? sizeof(uint32_t) * L.n * bucket : 16, st);
      vzero<float2>(st, x.as<float2>(), L.n, bucket);
      vzero<float2>(st, f.as<float2>(), L.n, bucket);
      if (fmt) MG_CUDA(cudaMemsetAsync(x16.p, 0, sizeof(uint32_t) * L.n * bucket, st));
      if (force || !tune_known(TUNE_TC0, L.side, bucket, fmt)) {
        int best = 0;
        float tbest = 1e30f;
        std::vector<int> vars;
        for (int m128 : {0, 1})
          for (int cap : {0, 2, 3, 4}) vars.push_back(m128 | (cap << 1));
        if (fmt && L.side % 4 == 0) vars.push_back(16);  // 16-bit formats: the 2x2-block kernel
        for (int v : vars) {
          tune_store(TUNE_TC0, L.side, bucket, fmt, v, 0.f);
          const float t = time_us(st, [&] {
            tc_stencil_apply(st, L.tcW.p, fmt, L.side, x.as<float2>(), x16.p, y.as<float2>(), f.as<float2>(),
                             bucket, nullptr, err);
          });
          if (t < tbest) { tbest = t; best = v; }
        }
        tune_store(TUNE_TC0, L.side, bucket, fmt, best, tbest);
      }
      if (force || !tune_known(TUNE_TC1, L.side, bucket, fmt)) {
        int best = 0;
        float tbest = 1e30f;
        for (int cap : {0, 1, 2, 4}) {
          tune_store(TUNE_TC1, L.side, bucket, fmt, cap, 0.f);
          const float t = time_us(st, [&] {
            tc_sap_half(st, L.tcW.p, L.tcInv[0].p, fmt, L.side, f.as<float2>(), x.as<float2>(), fmt ? x16.p : nullptr,
                        y.as<float2>(), 0, bucket, nullptr, err);
          });
          if (t < tbest) { tbest = t; best = cap; }
        }
        tune_store(TUNE_TC1, L.side, bucket, fmt, best, tbest);
      }
    }
  }
  MG_CUDA(cudaStreamSynchronize(st));
}

// ---- measured ALU peaks -------------------------------------------------------------------------------------
// Eight independent FMA chains per thread, a full grid of resident warps: the CUDA-core FMA throughput that the
// roofline of ALU-bound kernels (FP64 refinement residual, Galerkin products) is taken against.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + 1) * (T)(j + 1) * (T)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == (T)12345.678) out[blockIdx.x] = s;  // never true: keeps the chains from being removed
}

double alu_peak_tflops(cudaStream_t st, bool fp64) {
  int dev = 0, nsm = 152;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int grid = nsm * 8, iters = fp64 ? 2048 : 65536;
  DBuf out(sizeof(double) * grid, st);
  auto launch = [&] {
    if (fp64)
      MG_LAUNCH(k_fma_peak<double>, grid, 256, 0, st, out.as<double>(), iters, 0.999, 0.001);
    else
      MG_LAUNCH(k_fma_peak<float>, grid, 256, 0, st, out.as<float>(), iters, 0.999f, 0.001f);
  };
  launch();
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) best = std::min(best, time_us(st, launch, 1));
  return 2.0 * 8.0 * iters * (double)grid * 256 / (best * 1e-6) / 1e12;
}

}  // namespace mg
