// Allocation-free variant of the projected-sample computation of hutchpp_project.
//
// Some callers cannot allocate device memory at the point where they need the
// projected samples: a host framework that reserved the whole GPU for its own
// caching allocator (so cudaMalloc would fail or fragment its pool), or a
// latency-critical serving loop that forbids cudaMalloc/cudaFree after start-up
// because they synchronise the device and have unpredictable cost.  For them
// this file offers one entry point that only launches kernels: its partial sums
// live in a fixed file-scope device array instead of memory allocated per call.
//
// The array is a static __device__ object, so every GPU that loads this library
// holds it (NA_SCRATCH_BYTES, about 4.3 MB) until the process exits.  Host code
// cannot use the array's name as a device address (it names a host-side stand-in),
// so the first call on each device resolves the real address with
// cudaGetSymbolAddress while that device is current and caches it together with
// the CUDA context it belongs to; a call that finds another context current (after
// cudaDeviceReset, say, the module and its array are loaded anew) looks it up again.
#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr int NA_MAX_RHS = 256;  // largest nrhs accepted
constexpr int NA_MAX_D = 32;     // largest sketch size accepted
constexpr int NA_CHUNKS = 16;    // row chunks reduced in the second pass
constexpr int NA_PCH = 64;       // rows staged in shared memory at a time
constexpr int NA_RG = 8;         // rhs per block
// layout (double2): a[chunk][rhs], then c[chunk][i][rhs], then g[chunk][i][rhs]
constexpr size_t NA_A = (size_t)NA_CHUNKS * NA_MAX_RHS;
constexpr size_t NA_C = (size_t)NA_CHUNKS * NA_MAX_D * NA_MAX_RHS;
constexpr size_t NA_SCRATCH = NA_A + 2 * NA_C;

static __device__ __align__(256) double2 g_na_scratch[NA_SCRATCH];

std::mutex g_na_mu;
constexpr int NA_MAX_DEVICES = 64;
struct NaSlot {
  CUcontext ctx = nullptr;  // context the cached address belongs to
  double2* ptr = nullptr;
};
NaSlot g_na_slot[NA_MAX_DEVICES];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

// cuCtxGetCurrent from the driver (through the runtime's entry-point query, so nothing links libcuda)
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Partial sums over row chunk blockIdx.x for the rhs group blockIdx.y:
// a = zeta^H y, c_i = q_i^H zeta, g_i = q_i^H y.  Every slot a launch later reads
// is written here, so nothing carried over from an earlier call is ever used.
__global__ void __launch_bounds__(256) k_na_partial(const double2* __restrict__ Q, int d,
                                                    const double2* __restrict__ z,
                                                    const double2* __restrict__ y, long n, int nrhs,
                                                    double2* __restrict__ scratch) {
  __shared__ double2 Qs[NA_PCH * (NA_MAX_D + 1)];
  __shared__ double2 Zs[NA_RG * NA_PCH];
  __shared__ double2 Ys[NA_RG * NA_PCH];
  const int tid = threadIdx.x, i = tid % 32, g = tid / 32;
  const int r0 = blockIdx.y * NA_RG;
  const long per = (n + NA_CHUNKS - 1) / NA_CHUNKS;
  const long lo = (long)blockIdx.x * per, hi = min(n, lo + per);
  double2 ac = make_double2(0, 0), ag = make_double2(0, 0), aa = make_double2(0, 0);
  for (long e0 = lo; e0 < hi; e0 += NA_PCH) {
    __syncthreads();
    for (int q = tid; q < d * NA_PCH; q += blockDim.x) {
      const int c = q / NA_PCH, e = q % NA_PCH;
      Qs[e * (NA_MAX_D + 1) + c] = (e0 + e < hi) ? Q[(size_t)c * n + e0 + e] : make_double2(0, 0);
    }
    for (int q = tid; q < NA_RG * NA_PCH; q += blockDim.x) {
      const int rr = q / NA_PCH, e = q % NA_PCH;
      const bool in = r0 + rr < nrhs && e0 + e < hi;
      Zs[q] = in ? z[(size_t)(r0 + rr) * n + e0 + e] : make_double2(0, 0);
      Ys[q] = in ? y[(size_t)(r0 + rr) * n + e0 + e] : make_double2(0, 0);
    }
    __syncthreads();
    if (i < d)
      for (int e = 0; e < NA_PCH; ++e) {
        const double2 qv = Qs[e * (NA_MAX_D + 1) + i];
        ac = mg::cfmac(qv, Zs[g * NA_PCH + e], ac);
        ag = mg::cfmac(qv, Ys[g * NA_PCH + e], ag);
      }
    for (int e = i; e < NA_PCH; e += 32) aa = mg::cfmac(Zs[g * NA_PCH + e], Ys[g * NA_PCH + e], aa);
  }
  for (int o = 16; o; o >>= 1) {
    aa.x += __shfl_xor_sync(0xffffffff, aa.x, o);
    aa.y += __shfl_xor_sync(0xffffffff, aa.y, o);
  }
  const int r = r0 + g;
  if (r < nrhs) {
    if (i == 0) scratch[(size_t)blockIdx.x * NA_MAX_RHS + r] = aa;
    if (i < d) {
      scratch[NA_A + ((size_t)blockIdx.x * NA_MAX_D + i) * NA_MAX_RHS + r] = ac;
      scratch[NA_A + NA_C + ((size_t)blockIdx.x * NA_MAX_D + i) * NA_MAX_RHS + r] = ag;
    }
  }
}

// tau_r = a_r - sum_i conj(c_ir) g_ir, chunks summed in a fixed order.
__global__ void k_na_final(int d, int nrhs, const double2* __restrict__ scratch, double2* __restrict__ tau) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  double2 a = make_double2(0, 0);
  for (int k = 0; k < NA_CHUNKS; ++k) a = mg::cadd(a, scratch[(size_t)k * NA_MAX_RHS + r]);
  for (int i = 0; i < d; ++i) {
    double2 c = make_double2(0, 0), g = make_double2(0, 0);
    for (int k = 0; k < NA_CHUNKS; ++k) {
      c = mg::cadd(c, scratch[NA_A + ((size_t)k * NA_MAX_D + i) * NA_MAX_RHS + r]);
      g = mg::cadd(g, scratch[NA_A + NA_C + ((size_t)k * NA_MAX_D + i) * NA_MAX_RHS + r]);
    }
    a = mg::csub(a, mg::cmulc(c, g));
  }
  tau[r] = a;
}

// Device address of the scratch array for the current device and context: looked up once per (device,
// context) with that device current, then cached.
int na_scratch_ptr(double2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MGMLMC_ERR_CUDA;
  }
  if (dev < 0 || dev >= NA_MAX_DEVICES) return MGMLMC_ERR_INVALID_ARG;
  CUcontext cur = nullptr;
  CtxGetCurrentFn get = ctx_get_current();
  const bool known_ctx = get && get(&cur) == CUDA_SUCCESS && cur;
  std::lock_guard<std::mutex> lock(g_na_mu);
  NaSlot& slot = g_na_slot[dev];
  if (!slot.ptr || !known_ctx || slot.ctx != cur) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return MGMLMC_ERR_CUDA;
    }
    slot.ptr = static_cast<double2*>(p);
    slot.ctx = known_ctx ? cur : nullptr;  // without a context handle the lookup repeats on every call
  }
  *out = slot.ptr;
  return MGMLMC_OK;
}

}  // namespace

extern "C" int hutchpp_project_noalloc(void* stream, const double* Q, int d, const double* zeta, const double* y,
                                       int64_t n, int nrhs, double* tau_out) {
  if (nrhs < 0 || d < 0 || n < 0) return MGMLMC_ERR_INVALID_ARG;
  if (nrhs > NA_MAX_RHS || d > NA_MAX_D) return MGMLMC_ERR_INVALID_ARG;  // beyond the fixed scratch
  if (nrhs == 0) return MGMLMC_OK;
  if (n == 0 || !zeta || !y || !tau_out || (d > 0 && !Q)) return MGMLMC_ERR_INVALID_ARG;
  double2* scratch = nullptr;
  const int rc = na_scratch_ptr(&scratch);
  if (rc != MGMLMC_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 grid(NA_CHUNKS, (nrhs + NA_RG - 1) / NA_RG);
  // Each launch is checked right after it is issued.  cudaGetLastError also returns (and clears) an error left
  // pending by earlier, unrelated work on this thread, which is then reported here as MGMLMC_ERR_CUDA.
  k_na_partial<<<grid, 256, 0, st>>>(reinterpret_cast<const double2*>(Q), d, reinterpret_cast<const double2*>(zeta),
                                     reinterpret_cast<const double2*>(y), (long)n, nrhs, scratch);
  if (cudaGetLastError() != cudaSuccess) return MGMLMC_ERR_CUDA;
  k_na_final<<<(nrhs + 63) / 64, 64, 0, st>>>(d, nrhs, scratch, reinterpret_cast<double2*>(tau_out));
  if (cudaGetLastError() != cudaSuccess) return MGMLMC_ERR_CUDA;
  return MGMLMC_OK;
}
