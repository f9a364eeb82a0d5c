// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mgmlmc.h"

namespace mg {

// ---------------------------------------------------------------- errors
struct Error : public std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define MG_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      throw ::mg::Error(e_ == cudaErrorMemoryAllocation ? MGMLMC_ERR_OOM            \
                                                          : MGMLMC_ERR_CUDA,       \
                        std::string(#call) + ": " + cudaGetErrorString(e_));       \
    }                                                                              \
  } while (0)

// Raise a kernel's dynamic shared-memory limit once per (kernel, device, size): the attribute belongs to the
// device's context, so a process that drives several GPUs needs it set on each.
inline void ensure_max_smem(const void* kernel, int bytes) {
  static std::mutex mu;
  static std::set<std::tuple<const void*, int, int>> done;
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(std::make_tuple(kernel, dev, bytes))) return;
  MG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert(std::make_tuple(kernel, dev, bytes));
}

#define MG_CHECK_ARG(cond, msg)                                                    \
  do {                                                                             \
    if (!(cond)) throw ::mg::Error(MGMLMC_ERR_INVALID_ARG, msg);                   \
  } while (0)

// launch bookkeeping: every kernel launch of the library goes through MG_LAUNCH
// (counted per context) or MG_LAUNCH_W, which also carries the launch's
// algorithmic bytes and flops for the optional per-kernel event timer.
extern thread_local int64_t* g_launch_counter;
// Per-kernel CUDA-event timer (enabled per context for kernels whose name
// contains a filter string); records are resolved when the report is read.
struct KTimer {
  bool on = false;
  std::string filter;
  struct Rec {
    const char* name;
    const char* where;  // launching function (its template arguments name the precision)
    double bytes, flops;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    MG_CUDA(cudaEventCreate(&e));
    return e;
  }
  bool want(const char* name) const { return on && (filter.empty() || std::strstr(name, filter.c_str())); }
};
extern thread_local KTimer* g_timer;
// number of right-hand sides still iterating (host hint for byte accounting), -1 = all
extern thread_local int g_nact_hint;
inline double act_rhs(int nrhs) { return (g_nact_hint >= 0 && g_nact_hint < nrhs) ? g_nact_hint : nrhs; }

#define MG_LAUNCH_W(bytes, flops, kernel, grid, block, smem, stream, ...)          \
  do {                                                                             \
    ::mg::KTimer* t_ = ::mg::g_timer;                                              \
    if (t_ && t_->want(#kernel)) {                                                 \
      cudaEvent_t a_ = t_->get(), b_ = t_->get();                                  \
      MG_CUDA(cudaEventRecord(a_, (stream)));                                      \
      kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                  \
      MG_CUDA(cudaGetLastError());                                                 \
      MG_CUDA(cudaEventRecord(b_, (stream)));                                      \
      t_->recs.push_back({#kernel, __PRETTY_FUNCTION__, (double)(bytes), (double)(flops), a_, b_}); \
    } else {                                                                       \
      kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                  \
      MG_CUDA(cudaGetLastError());                                                 \
    }                                                                              \
    if (::mg::g_launch_counter) ++*::mg::g_launch_counter;                         \
  } while (0)
#define MG_LAUNCH(kernel, grid, block, smem, stream, ...) \
  MG_LAUNCH_W(0, 0, kernel, grid, block, smem, stream, __VA_ARGS__)

// ---------------------------------------------------------------- complex
template <typename R> struct CT;
template <> struct CT<float> { typedef float2 T; };
template <> struct CT<double> { typedef double2 T; };

__host__ __device__ __forceinline__ float2 cmake(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 cmake(double a, double b) { return make_double2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cneg(C a) { a.x = -a.x; a.y = -a.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
// acc + a * b
template <typename C> __host__ __device__ __forceinline__ C cfma(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc + conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cfmac(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
// i * a and -i * a
template <typename C> __host__ __device__ __forceinline__ C cmuli(C a) { C r; r.x = -a.y; r.y = a.x; return r; }
template <typename C> __host__ __device__ __forceinline__ C cmulmi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

template <typename Cdst, typename Csrc> __host__ __device__ __forceinline__ Cdst cconv(Csrc a) {
  Cdst r; r.x = a.x; r.y = a.y; return r;
}

// ---------------------------------------------------------------- RNG
// SplitMix64 output finaliser (Steele, Lea & Flood 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27; z *= 0x94D049BB133111EBull;
  z ^= z >> 31; return z;
}
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, int level, int phase, uint64_t sample) {
  uint64_t ctr = ((uint64_t)level << 56) | ((uint64_t)phase << 48) | sample;
  return mix64(seed ^ mix64(ctr));
}
__host__ __device__ __forceinline__ double rad_sign(uint64_t key, uint64_t i) {
  return (mix64(key + 0x9E3779B97F4A7C15ull * (i + 1)) >> 63) ? -1.0 : 1.0;
}

// ---------------------------------------------------------------- device memory
// RAII device buffer (stream-ordered allocation).
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = 0;
  DBuf() {}
  DBuf(size_t b, cudaStream_t s) { alloc(b, s); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { p = o.p; bytes = o.bytes; st = o.st; o.p = nullptr; o.bytes = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; st = o.st; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  void alloc(size_t b, cudaStream_t s) {
    release();
    st = s;
    bytes = b;
    if (b) MG_CUDA(cudaMallocAsync(&p, b, s));
  }
  void ensure(size_t b, cudaStream_t s) { if (b > bytes) alloc(b, s); }
  void release() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    bytes = 0;
  }
  ~DBuf() { release(); }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

inline unsigned cdiv(long a, long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace mg
