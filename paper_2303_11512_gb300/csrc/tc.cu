// Coarse-level block operators on the 5th-generation tensor cores (tcgen05).
//
// On a coarse level every site carries d = 16 complex dof and the operator
// (Galerkin stencil, SAP block inverse) is a small dense complex matrix per
// site or block applied to all right-hand sides at once: with the rhs on the
// M dimension that is a batched GEMM  Y^T[rhs, n] = sum_k X^T[rhs, k] E[n, k]
// with the complex matrix embedded as a real one (output rows Re y_i = [Re w_ij, -Im w_ij],
// Im y_i = [Im w_ij, Re w_ij] over k = 2j + {0, 1}), and FP32 data read directly as TF32.
//
//   mode 0 (stencil):   per site s, K = 5 chunks (x at s, s+x, s-x, s+t, s-t),
//                       N = 32:   y = D x   or   y = b - D x
//   mode 1 (SAP block): per 2x2 block B of one colour, K = 4 chunks (its sites),
//                       N = 128:  x_B += inv_B r_B
//
// Data movement: the rhs x 32-float slab of one site is one TMA box (the launch's
// rhs count rounded up to 8, at most 128 rows, x 128 B, 128-byte swizzle) straight
// from the canonical [rhs][site][dof] vector; MMA rows beyond the box are never
// stored.  Weights are stored pre-swizzled, Re rows only (half the real embedding),
// fetched with one bulk copy per chunk; two expander warps derive the Im rows in
// shared memory.  One thread issues the MMAs (M = 128, K = 8 per instruction) into
// TMEM accumulators; epilogue warps read them back with tcgen05.ld (row = rhs =
// lane).  Warp-specialised: a producer warp streams items through S shared-memory
// stages (lane k issuing the copies of chunk k), the expander completes each
// stage's weights, one thread issues the MMAs into four rotating TMEM
// accumulators, and eight epilogue warps (two per TMEM lane quarter, alternating
// items, the additive input fetched a few steps ahead) drain them.  Every wait on
// an mbarrier is bounded: on expiry the kernel records an error code, stops, waits
// (bounded) for its own copies and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ops.cuh"
#include "tcgen05.cuh"

namespace mg {
namespace {

constexpr int TC_M = 128;          // rhs per tile (MMA M)
constexpr int TC_CHUNK = 32;       // floats per site slab (16 complex)

__device__ __forceinline__ int nbr_site_tc(int s, int dir, int Ls) {
  const int t = s / Ls, x = s - t * Ls;
  switch (dir) {
    case 1: return t * Ls + (x + 1 == Ls ? 0 : x + 1);
    case 2: return t * Ls + (x == 0 ? Ls - 1 : x - 1);
    case 3: return (t + 1 == Ls ? 0 : t + 1) * Ls + x;
    case 4: return (t == 0 ? Ls - 1 : t - 1) * Ls + x;
    default: return s;
  }
}
// site of local index j (0..3) of the k-th 2x2 block of colour `color`
__device__ __forceinline__ int block_site(int k, int j, int Ls, int color) {
  const int nbx = Ls / 2, half = nbx / 2;
  const int BT = k / half;
  const int BX = 2 * (k % half) + ((BT + color) & 1);
  return (2 * BT + (j >> 1)) * Ls + 2 * BX + (j & 1);
}

// MODE 0: KC = 5 site slabs; the vectors are the A operand (rows = rhs, M = 64), the weights B (N = 32).
// MODE 1: KC = 4 site slabs; the block inverse is the A operand (M = 128 outputs), the residual slabs B
//         (rows = rhs, N = the launch's rhs count rounded up to 16): the transposed product, so a small batch
//         is not padded to 128 MMA rows.
// BF = 0: TF32 operands (kind::tf32, K = 8 per instruction); the FP32 vector slabs that TMA brings in are the
//         MMA operand directly (128-byte rows, 128-byte swizzle).
// BF = 1 / 2: BF16 / FP16 operands (kind::f16, K = 16 per instruction, FP32 accumulation): half the weight bytes and half
//         the MMA instructions; converter warps turn each staged FP32 slab into a BF16 operand tile
//         (64-byte rows, 64-byte swizzle) before the MMA reads it.
template <int MODE>
struct TcCfg;
template <>
struct TcCfg<0> {
  static constexpr int KC = 5, NW = 32;  // NW: weight rows per chunk (outputs of one site, real embedding)
};
template <>
struct TcCfg<1> {
  static constexpr int KC = 4, NW = 128;  // outputs of the 4 block sites
};
constexpr int TC_MAX_STAGES = 8;
constexpr int TC_PROD_WARPS = 5;  // one producer warp per chunk: the copies of an item are issued in parallel
constexpr int TC_MMA_WARPS = 1;   // one MMA-issuing thread (two issuing warps faulted the GPU)
constexpr int TC_EPI_WARPS = 8;   // two epilogue warps per TMEM lane quarter, alternating items
constexpr int TC_EXP_WARPS = 4;   // expander/converter warps: Im rows of the weight tiles (and BF16 vector tiles)
constexpr int TC_MMA_WARP0 = TC_PROD_WARPS;
constexpr int TC_EPI_WARP0 = TC_MMA_WARP0 + TC_MMA_WARPS;
constexpr int TC_EXP_WARP0 = TC_EPI_WARP0 + TC_EPI_WARPS;
// producer warps, MMA warp, epilogue warps, expander warps
constexpr int TC_THREADS = 32 * (TC_EXP_WARP0 + TC_EXP_WARPS);
constexpr int TC_NACC = 4;       // TMEM accumulators in flight

// Shared-memory layout of one pipeline stage (every tile base 1024-byte aligned):
//   TF32: KC FP32 vector slabs (vrows rows x 128 B, the MMA operand), KC weight tiles (NW rows x 128 B);
//   BF16: KC FP32 staging slabs (vrows x 128 B, TMA), KC BF16 vector tiles (vt rows x 64 B), KC weight tiles
//         (NW rows x 64 B); vt = mm in MODE 0 (the MMA reads M = mm rows), vrows in MODE 1.
// In MODE 0 the MMA reads mm A rows from a vector tile of `vrows` rows (TF32) or from an mm-row BF16 tile; rows
// past the converted/loaded ones only feed accumulator rows that are never stored.
__host__ __device__ constexpr int tc_vt(int MODE, int vrows, int mm) { return MODE == 0 ? mm : vrows; }
__host__ __device__ constexpr int tc_stage_bytes(int MODE, int BF, int KC, int NW, int vrows, int mm) {
  return BF ? KC * (vrows * 128 + tc_vt(MODE, vrows, mm) * 64 + NW * 64) : KC * (vrows + NW) * 128;
}

// items: MODE 0 with bmode = 0: every site; bmode = 1: the 4 sites of every colour-`color` 2x2 block.
//        MODE 1: every colour-`color` 2x2 block.
// vrows: rows of a vector slab (MODE 0: rhs of the mm-rhs tile rounded up to 8; MODE 1: up to 16, the MMA N);
// mm: MMA M of MODE 0 (64 or 128, also the rhs covered by one blockIdx.y; a tuned launch variant).
// Warp-specialised pipeline: the producers keep up to `stages` items in flight in shared memory (full/empty
// mbarriers), the expander/converter warps complete each stage (xfull), the MMA thread rotates over TC_NACC
// TMEM accumulators (tmem_full/tmem_empty mbarriers), the epilogue warps drain one accumulator while the next
// item is multiplied.
template <int MODE, int BF>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc(const __grid_constant__ CUtensorMap amap, const void* __restrict__ Wv, float* __restrict__ out,
         const float* __restrict__ bvec, int Ls, int nitems, int bmode, int color, int nrhs, int vrows, int mm,
         int stages, const int* __restrict__ active, int* err) {
  typedef TcCfg<MODE> CF;
  constexpr int KC = CF::KC, NW = CF::NW;
  const int MM = MODE == 0 ? mm : TC_M;           // MMA M
  constexpr int WROW = BF ? 64 : 128;             // bytes of one weight / operand row
  const int acc_cols = MODE == 0 ? NW : vrows;    // TMEM columns of one accumulator
  const int vt = tc_vt(MODE, vrows, MM);
  const int NI = MODE == 0 ? NW : vrows;  // MMA N
  const uint32_t idesc = BF == 2 ? idesc_f16(MM, NI) : BF == 1 ? idesc_bf16(MM, NI) : idesc_tf32(MM, NI);
  uint32_t ncol = 32;
  while (ncol < (uint32_t)(TC_NACC * acc_cols)) ncol <<= 1;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[TC_MAX_STAGES], empty_bar[TC_MAX_STAGES], xfull_bar[TC_MAX_STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[TC_NACC], tempty_bar[TC_NACC];
  __shared__ uint32_t s_taddr;
  __shared__ int s_skip;
  __shared__ volatile int s_bad;
  __shared__ unsigned char s_live[TC_M];  // MODE 1: rhs rhs0 + c exists and is active
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rhs0 = blockIdx.y * (MODE == 0 ? MM : TC_M);
  if (tid == 0) s_skip = *(volatile int*)err;  // an earlier launch gave up: do nothing until the host sees it
  if (MODE == 1 && tid < TC_M) {
    const int r = rhs0 + tid;
    s_live[tid] = r < nrhs && !(active && !active[r]);
  }
  __syncthreads();
  if (s_skip) return;
  const long ncf = (long)Ls * Ls * TC_CHUNK;  // floats per rhs row
  const int sbytes = tc_stage_bytes(MODE, BF, KC, NW, vrows, MM);
  const uint32_t chunk_tx = (uint32_t)(vrows * 128 + (NW / 2) * WROW);  // one vector slab + one stored weight half
  // staged FP32 slab, MMA vector operand and weight tile of chunk kc in stage st
  auto sS = [&](int st, int kc) { return base + st * sbytes + kc * vrows * 128; };
  auto sV = [&](int st, int kc) { return BF ? base + st * sbytes + KC * vrows * 128 + kc * vt * 64 : sS(st, kc); };
  auto sW = [&](int st, int kc) {
    return base + st * sbytes + KC * vrows * 128 + (BF ? KC * vt * 64 : 0) + kc * NW * WROW;
  };
  auto center = [&](int item) -> int { return bmode ? block_site(item >> 2, item & 3, Ls, color) : item; };
  auto site_of = [&](int item, int kc) -> int {
    if (MODE == 1) return block_site(item, kc, Ls, color);
    return nbr_site_tc(center(item), kc, Ls);
  };
  auto w_of = [&](int item, int kc) -> const unsigned char* {
    const size_t wi = MODE == 1 ? (size_t)item * KC + kc : (size_t)center(item) * KC + kc;
    return reinterpret_cast<const unsigned char*>(Wv) + wi * (NW / 2) * WROW;
  };

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full_bar[s], KC);  // one arrive.expect_tx per producer warp
      mbar_init(&empty_bar[s], 1);
      mbar_init(&xfull_bar[s], TC_EXP_WARPS);
    }
    for (int a = 0; a < TC_NACC; ++a) {
      mbar_init(&tfull_bar[a], 1);
      mbar_init(&tempty_bar[a], 4);  // the four lane-quarter warps of the item's parity
    }
    s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                 "r"(ncol)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  int n_my = 0;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) ++n_my;

  if (warp < TC_PROD_WARPS) {
    // ---------------- producers: warp kc (< KC) issues chunk kc of every item, lane 0 the vector slab (TMA),
    // lane 1 the stored weight half; the stage's full barrier completes once all KC warps arrived and every
    // announced byte landed
    const int kc = warp;
    if (kc < KC) {
      int issued = 0;
      for (int i = 0; i < n_my; ++i) {
        const int s = i % stages;
        int ok = lane == 0 ? !s_bad : 0;
        if (lane == 0 && ok && i >= stages && !mbar_wait(&empty_bar[s], (uint32_t)((i / stages) - 1) & 1u)) {
          atomicExch(err, 1);
          s_bad = 1;
          ok = 0;
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) break;
        const int item = blockIdx.x + i * gridDim.x;
        // the warp posts its own bytes before either of its copies is issued, so the stage's transaction
        // count never runs ahead of the bytes announced for it
        if (lane == 0) mbar_expect_tx(&full_bar[s], chunk_tx);
        __syncwarp();
        if (lane == 0)
          tma_load_2d(sS(s, kc), &amap, site_of(item, kc) * TC_CHUNK, rhs0, &full_bar[s]);
        else if (lane == 1)
          bulk_load(sW(s, kc), w_of(item, kc), (NW / 2) * WROW, &full_bar[s]);
        issued = i + 1;
      }
      // let the last loads (of every producer warp) land before the CTA can exit (bounded)
      if (kc == 0 && lane == 0)
        for (int i = std::max(0, issued - stages); i < issued; ++i)
          mbar_wait(&full_bar[i % stages], (uint32_t)(i / stages) & 1u);
    }
  } else if (warp < TC_EPI_WARP0) {
    // ---------------- MMA issuer
    const uint64_t vdesc0 = BF ? sw64_desc(smem_u32(sV(0, 0))) : sw128_desc(smem_u32(sV(0, 0)));
    const uint64_t wdesc0 = BF ? sw64_desc(smem_u32(sW(0, 0))) : sw128_desc(smem_u32(sW(0, 0)));
    const uint32_t stage16 = (uint32_t)sbytes >> 4;
    const uint32_t vstep16 = (uint32_t)(BF ? vt * 64 : vrows * 128) >> 4, wstep16 = (uint32_t)(NW * WROW) >> 4;
    if (lane == 0) {
      for (int i = 0; i < n_my && !s_bad; ++i) {
        const int s = i % stages, a = i % TC_NACC;
        if (!mbar_wait(&xfull_bar[s], (uint32_t)(i / stages) & 1u)) {
          atomicExch(err, 2);
          s_bad = 1;
          break;
        }
        if (i >= TC_NACC && !mbar_wait(&tempty_bar[a], (uint32_t)((i / TC_NACC) - 1) & 1u)) {
          atomicExch(err, 3);
          s_bad = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = taddr + (uint32_t)(a * acc_cols);
        // descriptors of this stage: the first chunk's plus fixed steps (address field in 16-byte units)
        const uint64_t vds = vdesc0 + (uint64_t)(s * stage16), wds = wdesc0 + (uint64_t)(s * stage16);
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) {
          const uint64_t vd = vds + (uint64_t)(kc * vstep16), wd = wds + (uint64_t)(kc * wstep16);
          const uint64_t ad = MODE == 0 ? vd : wd, bd = MODE == 0 ? wd : vd;
          if (BF) {
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2)  // K = 16 bf16 = 32 B per instruction
              mma_bf16(d, ad + 2 * k2, bd + 2 * k2, idesc, (kc | k2) != 0);
          } else {
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4)  // K = 8 tf32 = 32 B per instruction
              mma_tf32(d, ad + 2 * k4, bd + 2 * k4, idesc, (kc | k4) != 0);
          }
        }
        mma_commit(&empty_bar[s]);  // smem stage free once these MMAs completed
        mma_commit(&tfull_bar[a]);  // accumulator a ready for the epilogue
      }
    }
  } else if (warp >= TC_EXP_WARP0) {
    // ---------------- expander / converter.  Weight tiles: the Im rows from the stored Re rows; row n + NW/2
    // has the swizzle phase of row n.  TF32: (a, b) -> (-b, a) per complex pair, each 16-byte chunk keeps its
    // position.  16-bit (planar K): logical chunk c of the Im row is chunk c ^ 2 of the Re row, negated for
    // c < 2 (the -Im half becomes the leading Im half).  16-bit formats: every staged FP32 slab (128-byte
    // swizzle, interleaved Re/Im) becomes a planar operand tile (64-byte swizzle, round to nearest even).
    const int et = (warp - TC_EXP_WARP0) * 32 + lane;
    constexpr int NT = 32 * TC_EXP_WARPS;
    constexpr int CPR = WROW / 16;           // 16-byte chunks per row
    constexpr int HALF = (NW / 2) * CPR;     // chunks per stored half tile
    constexpr int TILE = NW * CPR;           // chunks per full tile
    for (int i = 0; i < n_my; ++i) {
      const int s = i % stages;
      if (s_bad || !mbar_wait(&full_bar[s], (uint32_t)(i / stages) & 1u)) {
        if (!s_bad) atomicExch(err, 5);
        s_bad = 1;
        break;
      }
      // weight tiles: the KC chunks of one (row, 16-byte chunk) position are independent, so each thread handles
      // a position of all KC tiles at once (KC loads in flight, no index division)
      uint4* w0 = reinterpret_cast<uint4*>(sW(s, 0));
      for (int e = et; e < HALF; e += NT) {
        // 16-bit: position e ^ 2 holds logical chunk c ^ 2; the sign flips where the Im row's logical chunk < 2
        const uint32_t neg = BF && !(((e & 3) ^ ((e >> 3) & 3)) & 2) ? 0x80008000u : 0u;
        uint4 v[KC];
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) v[kc] = w0[kc * TILE + (BF ? e ^ 2 : e)];
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) {
          uint4 r;
          if (BF) {
            r = make_uint4(v[kc].x ^ neg, v[kc].y ^ neg, v[kc].z ^ neg, v[kc].w ^ neg);
          } else {  // two fp32 pairs (a, b) -> (-b, a)
            r.x = v[kc].y ^ 0x80000000u;
            r.y = v[kc].x;
            r.z = v[kc].w ^ 0x80000000u;
            r.w = v[kc].z;
          }
          w0[kc * TILE + e + HALF] = r;
        }
      }
      if (BF) {
        // unit (row, c): complex dofs 4c .. 4c+3 = FP32 chunks 2c and 2c+1 of the staged row; their Re parts go
        // to half c & 1 of logical output chunk c >> 1, their Im parts to the same half of chunk 2 + (c >> 1).
        // A thread converts position (row, c) of all KC slabs.
        for (int u = et; u < vrows * 4; u += NT) {
          const int row = u >> 2, c = u & 3, ph = (row >> 1) & 3;
          float4 f[KC][2];
#pragma unroll
          for (int kc = 0; kc < KC; ++kc) {
            const float4* src = reinterpret_cast<const float4*>(sS(s, kc)) + row * 8;
            f[kc][0] = src[(2 * c) ^ (row & 7)];
            f[kc][1] = src[(2 * c + 1) ^ (row & 7)];
          }
          const int ore = row * 8 + ((((c >> 1)) ^ ph) << 1) + (c & 1);      // uint2 index of the Re half
          const int oim = row * 8 + (((2 + (c >> 1)) ^ ph) << 1) + (c & 1);  // uint2 index of the Im half
#pragma unroll
          for (int kc = 0; kc < KC; ++kc) {
            uint2 re, im;
            if (BF == 2) {
              re = make_uint2(f16x2_rn(f[kc][0].x, f[kc][0].z), f16x2_rn(f[kc][1].x, f[kc][1].z));
              im = make_uint2(f16x2_rn(f[kc][0].y, f[kc][0].w), f16x2_rn(f[kc][1].y, f[kc][1].w));
            } else {
              re = make_uint2(bf16x2_rn(f[kc][0].x, f[kc][0].z), bf16x2_rn(f[kc][1].x, f[kc][1].z));
              im = make_uint2(bf16x2_rn(f[kc][0].y, f[kc][0].w), bf16x2_rn(f[kc][1].y, f[kc][1].w));
            }
            reinterpret_cast<uint2*>(sV(s, kc))[ore] = re;
            reinterpret_cast<uint2*>(sV(s, kc))[oim] = im;
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> MMA reads
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&xfull_bar[s])) : "memory");
    }
  } else if (MODE == 0) {
    // ---------------- epilogue (rows = rhs): warp w owns TMEM lane quarter w % 4 and the items of parity
    // (w - first epilogue warp) / 4.  With M = 128 accumulator row r sits in lane r; with M = 64 in lane
    // 32 (r / 16) + r % 16, so lanes 16..31 of each quarter are unused.
    const int q = warp & 3, par = (warp - TC_EPI_WARP0) >> 2;
    const int qrows = MM == 128 ? 32 : 16;
    const int row = q * qrows + lane;
    const int rhs = rhs0 + row;
    const bool live = lane < qrows && rhs < nrhs && !(active && !active[rhs]);
    const bool quarter_live = rhs0 + q * qrows < nrhs;  // warp-uniform
    // with bvec the output is b - D x; the work of an item is split in steps of 8 complex outputs (half a site
    // slab); the additive input of step t + RD is fetched at step t.
    const float* in = bvec;
    constexpr int NSTEP = NW / 16, RD = NSTEP < 4 ? NSTEP : 4;
    static_assert(NSTEP % RD == 0, "prefetch ring must divide the steps of an item");
    auto step_ptr = [&](const float* v, int i, int t) -> const float* {
      const int item = blockIdx.x + i * gridDim.x;
      return v + (size_t)rhs * ncf + (size_t)center(item) * TC_CHUNK + 16 * (t & 1);
    };
    float4 ring[RD][4];
    auto prefetch = [&](float4 (&dst)[4], int i, int t) {
      if (in && live && i < n_my) {
        const float4* src = reinterpret_cast<const float4*>(step_ptr(in, i, t));
#pragma unroll
        for (int u = 0; u < 4; ++u) dst[u] = src[u];
      }
    };
#pragma unroll
    for (int g = 0; g < RD; ++g) prefetch(ring[g], par + 2 * (g / NSTEP), g % NSTEP);
    for (int i = par; i < n_my; i += 2) {
      const int a = i % TC_NACC;
      if (s_bad || !mbar_wait(&tfull_bar[a], (uint32_t)(i / TC_NACC) & 1u)) {
        if (!s_bad) atomicExch(err, 4);
        s_bad = 1;
        break;
      }
      tc_fence_after();
      const uint32_t tq = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * acc_cols);
#pragma unroll
      for (int t = 0; t < NSTEP; ++t) {
        float4 cur[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cur[u] = ring[t % RD][u];
        prefetch(ring[t % RD], i + 2 * ((t + RD) / NSTEP), (t + RD) % NSTEP);
        if (!quarter_live) continue;
        // v[0..7] = Re, v[8..15] = Im of complex outputs 8t .. 8t + 7
        float v[16];
        tmem_ld8x2(tq + 8 * t, tq + NW / 2 + 8 * t, v);
        if (live) {
          float4* o = reinterpret_cast<float4*>(const_cast<float*>(step_ptr(out, i, t)));
          if (bvec) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              o[u] = make_float4(cur[u].x - v[2 * u], cur[u].y - v[8 + 2 * u], cur[u].z - v[2 * u + 1],
                                 cur[u].w - v[9 + 2 * u]);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) o[u] = make_float4(v[2 * u], v[8 + 2 * u], v[2 * u + 1], v[9 + 2 * u]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty_bar[a])) : "memory");
    }
  } else {
    // ---------------- epilogue (rows = block outputs, columns = rhs): lane r of the accumulator holds output
    // row r of the weight image (r < 64: Re y_r, r >= 64: Im y_{r-64}; y_i is dof i % 16 of block site i / 16).
    // Warp w owns lane quarter q = w % 4 and the items of parity (w - 2) / 4; x_B += inv_B r_B in 16-rhs steps.
    const int q = warp & 3, par = (warp - TC_EPI_WARP0) >> 2;
    const int oi = (q & 1) * 32 + lane;                 // complex output index of this thread
    const int bj = oi >> 4, fo = 2 * (oi & 15) + (q >> 1);  // block site, float within its 32-float slab
    const int nstep = vrows / 16;
    // this thread's float of block site bj in the rhs-rhs0 row of item i's block
    auto base_of = [&](int i) -> float* {
      const int item = blockIdx.x + i * gridDim.x;
      return out + (size_t)rhs0 * ncf + (size_t)block_site(item, bj, Ls, color) * TC_CHUNK + fo;
    };
    float cur[16];
    float* pcur = nullptr;
    auto fetch = [&](float* p, int t) {
#pragma unroll
      for (int u = 0; u < 16; ++u) cur[u] = s_live[16 * t + u] ? p[(size_t)(16 * t + u) * ncf] : 0.f;
    };
    if (par < n_my) {
      pcur = base_of(par);
      fetch(pcur, 0);
    }
    for (int i = par; i < n_my; i += 2) {
      const int a = i % TC_NACC;
      if (s_bad || !mbar_wait(&tfull_bar[a], (uint32_t)(i / TC_NACC) & 1u)) {
        if (!s_bad) atomicExch(err, 4);
        s_bad = 1;
        break;
      }
      tc_fence_after();
      const uint32_t tq = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * acc_cols);
      float* pnext = i + 2 < n_my ? base_of(i + 2) : nullptr;
      for (int t = 0; t < nstep; ++t) {
        float v[16];
        tmem_ld8x2(tq + 16 * t, tq + 16 * t + 8, v);
        float nx[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) nx[u] = cur[u] + v[u];
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (s_live[16 * t + u]) pcur[(size_t)(16 * t + u) * ncf] = nx[u];
        if (t + 1 < nstep)
          fetch(pcur, t + 1);
        else if (pnext)
          fetch(pnext, 0);
      }
      pcur = pnext;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty_bar[a])) : "memory");
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncol) : "memory");
  }
}

// Weight images.  The real embedding of a complex output row i is the pair of rows
//   TF32 (k = 2j + b, the interleaved order of the FP32 vectors):
//     Re y_i:  (Re w_ij, -Im w_ij)        Im y_i:  (Im w_ij, Re w_ij)
//   16-bit (k = 16b + j, planar: the 16-bit operand tiles hold the 16 Re parts of a site, then the 16 Im parts):
//     Re y_i:  [Re w_i. | -Im w_i.]       Im y_i:  [Im w_i. | Re w_i.]
// the second a fixed rearrangement of the first.  Only the Re rows are stored (NW/2 rows per K chunk of 32
// reals), pre-swizzled K-major: TF32 element (n, k) at n * 32 + (((k >> 2) ^ (n & 7)) << 2) + (k & 3) (128-byte
// rows), 16-bit element (n, k) at n * 32 + (((k >> 3) ^ ((n >> 1) & 3)) << 3) + (k & 7) (64-byte rows); the
// kernel's expander warps build the Im rows in shared memory, so accumulator columns (MODE 0) or lanes
// (MODE 1) [0, NW/2) hold Re y and [NW/2, NW) Im y.
__device__ __forceinline__ int sw_index(int n, int k) { return n * 32 + ((((k >> 2) ^ (n & 7)) << 2) | (k & 3)); }
__device__ __forceinline__ int sw64_index(int n, int k) {
  return n * 32 + ((((k >> 3) ^ ((n >> 1) & 3)) << 3) | (k & 7));
}
template <int BF>
__device__ __forceinline__ void put_w(void* W, size_t tile, int rows, int n, int k, float v) {
  if (BF == 2)
    reinterpret_cast<__half*>(W)[tile * rows * 32 + sw64_index(n, k)] = __float2half_rn(v);
  else if (BF == 1)
    reinterpret_cast<__nv_bfloat16*>(W)[tile * rows * 32 + sw64_index(n, k)] = __float2bfloat16_rn(v);
  else
    reinterpret_cast<float*>(W)[tile * rows * 32 + sw_index(n, k)] = v;
}

template <int BF>
__global__ void k_tc_stencil_weights(const float2* __restrict__ st, int nsite, void* __restrict__ W) {
  // st[site][dir][16][16] complex -> W[site][dir][16 stored rows x 32]
  const size_t total = (size_t)nsite * 5 * 16 * 32;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int k = e % 32, i = (e / 32) % 16;
    const size_t sd = e / 512;  // site * 5 + dir
    const int j = k >> 1, b = k & 1;
    const float2 z = st[sd * 256 + i * 16 + j];
    put_w<BF>(W, sd, 16, i, BF ? 16 * b + j : k, b ? -z.y : z.x);
  }
}

template <int BF>
__global__ void k_tc_blockinv_weights(const float2* __restrict__ inv, int Ls, int color, int nblk, void* __restrict__ W) {
  // colour-`color` blocks only, in their item order: inv[block][64][64] -> W[item][kc 4][64 stored rows x 32]
  const size_t total = (size_t)nblk * 4 * 64 * 32;
  const int nbx = Ls / 2, half = nbx / 2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int kk = e % 32, i = (e / 32) % 64, kc = (e / 2048) % 4;
    const int item = (int)(e / 8192);
    const int BT = item / half, BX = 2 * (item % half) + ((BT + color) & 1);
    const int blk = BT * nbx + BX;
    const int kg = kc * 32 + kk;  // real input index 2 * (16 * site_j + dof) + b
    const int j = kg >> 1, b = kg & 1;
    const float2 z = inv[(size_t)blk * 4096 + i * 64 + j];
    put_w<BF>(W, (size_t)item * 4 + kc, 64, i, BF ? 16 * b + (kk >> 1) : kk, b ? -z.y : z.x);
  }
}

// 2D view [nrhs rows][nsite * 32 floats] of a coarse FP32 vector; box 32 floats x `rows` rows (rows past
// nrhs are filled with zeros by the copy engine)
CUtensorMap make_map(const float2* v, int nsite, int nrhs, int rows) {
  MG_CHECK_ARG(((uintptr_t)v & 15) == 0, "tensor-core operand must be 16-byte aligned");
  MG_CHECK_ARG(rows >= 8 && rows <= TC_M && rows % 8 == 0, "tensor-core box rows");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)nsite * TC_CHUNK, (cuuint64_t)nrhs};
  cuuint64_t strides[1] = {(cuuint64_t)nsite * TC_CHUNK * 4};
  cuuint32_t box[2] = {TC_CHUNK, (cuuint32_t)rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)v, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(MGMLMC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

// Launch shape of one tensor-core launch over nrhs right-hand sides:
//   MODE 0: MMA M = 64 and 64 rhs per blockIdx.y (half the shared-memory operand reads of M = 128 and
//           stages small enough for a deep pipeline); slab rows = rhs rounded up to 8 (at most 64).
//   MODE 1: 128 rhs per blockIdx.y, slab rows = MMA N = rhs rounded up to 16 (at most 128).
template <int MODE, int BF>
void launch_tc(cudaStream_t st, const float2* vin, const void* W, float* out, const float* b, int Ls, int nitems,
               int bmode, int color, int nrhs, const int* active, int* err, double bytes, double flops) {
  typedef TcCfg<MODE> CF;
  constexpr int SMEM_BUDGET = 225 * 1024;  // dynamic shared memory per CTA (one CTA per SM)
  auto* k_tc_kernel = &k_tc<MODE, BF>;
  ensure_max_smem((const void*)k_tc_kernel, SMEM_BUDGET);
  // tuned variant: MODE 0 bit 0 = MMA M 128 (else 64), bits 1.. = pipeline-depth cap (0 = as deep as fits);
  // MODE 1: the depth cap
  const int var = tune_lookup(MODE == 0 ? TUNE_TC0 : TUNE_TC1, Ls, nrhs, BF, 0) & (MODE == 0 ? 15 : ~0);
  const int mm = MODE == 0 ? ((var & 1) ? TC_M : 64) : TC_M;
  const int cap = MODE == 0 ? (var >> 1) : var;
  const int tile = mm;
  const int vrows = MODE == 0 ? std::min(mm, ((nrhs + 7) / 8) * 8) : std::min(TC_M, ((nrhs + 15) / 16) * 16);
  const CUtensorMap m = make_map(vin, Ls * Ls, nrhs, vrows);
  const int sbytes = tc_stage_bytes(MODE, BF, CF::KC, CF::NW, vrows, mm);
  const int stages = std::max(1, std::min(cap > 0 ? cap : TC_MAX_STAGES, (SMEM_BUDGET - 1024) / sbytes));
  const int sm = stages * sbytes + 1024;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = (nrhs + tile - 1) / tile;
  const int gx = std::max(1, std::min(nitems, (nsm + tiles - 1) / tiles));
  dim3 grid(gx, tiles);
  MG_LAUNCH_W(bytes, flops, k_tc_kernel, grid, TC_THREADS, sm, st, m, W, out, b, Ls, nitems, bmode, color, nrhs,
              vrows, mm, stages, active, err);
}

template <int MODE>
void launch_tc_fmt(int bf, cudaStream_t st, const float2* vin, const void* W, float* out, const float* b, int Ls,
                   int nitems, int bmode, int color, int nrhs, const int* active, int* err, double bytes,
                   double flops) {
  if (bf == 2)
    launch_tc<MODE, 2>(st, vin, W, out, b, Ls, nitems, bmode, color, nrhs, active, err, bytes, flops);
  else if (bf == 1)
    launch_tc<MODE, 1>(st, vin, W, out, b, Ls, nitems, bmode, color, nrhs, active, err, bytes, flops);
  else
    launch_tc<MODE, 0>(st, vin, W, out, b, Ls, nitems, bmode, color, nrhs, active, err, bytes, flops);
}

// FP32 coarse vectors [rhs][site][16 complex] -> the planar 16-bit copy [rhs][site][16 Re | 16 Im] (round to
// nearest even); one thread per 4 complex dofs
template <int BF>
__global__ void k_round16(const float4* __restrict__ x, uint2* __restrict__ x16, size_t nquad) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nquad; e += (size_t)gridDim.x * blockDim.x) {
    const float4 a = x[2 * e], b = x[2 * e + 1];
    const size_t site = e >> 2;  // 4 quads per site
    const int c = (int)(e & 3);
    uint2 re, im;
    if (BF == 2) {
      re = make_uint2(f16x2_rn(a.x, a.z), f16x2_rn(b.x, b.z));
      im = make_uint2(f16x2_rn(a.y, a.w), f16x2_rn(b.y, b.w));
    } else {
      re = make_uint2(bf16x2_rn(a.x, a.z), bf16x2_rn(b.x, b.z));
      im = make_uint2(bf16x2_rn(a.y, a.w), bf16x2_rn(b.y, b.w));
    }
    x16[site * 8 + c] = re;      // uint2 units: Re dofs 4c .. 4c+3
    x16[site * 8 + 4 + c] = im;  // Im dofs 4c .. 4c+3
  }
}

}  // namespace

// stored weight bytes: stencil 5 dirs x 16 Re rows x 32 reals per site; block inverses 4 chunks x 64 Re rows x
// 32 reals per 2x2 block, for the (Ls/2)^2 / 2 blocks of one colour
size_t tc_stencil_weight_bytes(int nsite, int bf) { return (size_t)nsite * 5 * 16 * 32 * (bf ? 2 : 4); }
size_t tc_blockinv_weight_bytes(int Ls, int bf) { return (size_t)(Ls / 2) * (Ls / 2) / 2 * 4 * 64 * 32 * (bf ? 2 : 4); }

void tc_stencil_weights(cudaStream_t st, const float2* st32, int nsite, void* W, int bf) {
  if (bf == 2)
    MG_LAUNCH(k_tc_stencil_weights<2>, 1024, 256, 0, st, st32, nsite, W);
  else if (bf == 1)
    MG_LAUNCH(k_tc_stencil_weights<1>, 1024, 256, 0, st, st32, nsite, W);
  else
    MG_LAUNCH(k_tc_stencil_weights<0>, 1024, 256, 0, st, st32, nsite, W);
}
void tc_blockinv_weights(cudaStream_t st, const float2* inv32, int Ls, int color, void* W, int bf) {
  const int nblk = (Ls / 2) * (Ls / 2) / 2;
  if (bf == 2)
    MG_LAUNCH(k_tc_blockinv_weights<2>, 1024, 256, 0, st, inv32, Ls, color, nblk, W);
  else if (bf == 1)
    MG_LAUNCH(k_tc_blockinv_weights<1>, 1024, 256, 0, st, inv32, Ls, color, nblk, W);
  else
    MG_LAUNCH(k_tc_blockinv_weights<0>, 1024, 256, 0, st, inv32, Ls, color, nblk, W);
}

// 16-bit formats: the 2x2-block kernel (tc_block.cu) or the per-site kernel; a tuned variant of the stencil
// (TUNE_TC0) with bit 4 set selects the block kernel, untuned launches take it for batches of at most 32 rhs (it
// issues fewer MMAs per site; at larger batches the per-site kernel's TMA staging keeps more loads in flight)
bool tc_block_selected(int bf, int Ls, int nrhs) {
  if (!bf || Ls % 4) return false;
  const int var = tune_lookup(TUNE_TC0, Ls, nrhs, bf, -1);
  return var < 0 ? nrhs <= 32 : (var & 16) != 0;
}

void tc_round16(cudaStream_t st, int bf, const float2* x, void* x16, int nsite, int nrhs) {
  MG_CHECK_ARG(bf == 1 || bf == 2, "16-bit copy of a coarse vector needs a 16-bit format");
  if (nrhs <= 0) return;
  const size_t nquad = (size_t)nsite * 4 * nrhs;
  const double bytes = (double)nquad * 48.0;
  const unsigned grid = (unsigned)std::min<size_t>((nquad + 255) / 256, 152 * 16);
  if (bf == 2)
    MG_LAUNCH_W(bytes, 0, k_round16<2>, grid, 256, 0, st, (const float4*)x, (uint2*)x16, nquad);
  else
    MG_LAUNCH_W(bytes, 0, k_round16<1>, grid, 256, 0, st, (const float4*)x, (uint2*)x16, nquad);
}

void tc_stencil_apply(cudaStream_t st, const void* W, int bf, int Ls, const float2* x, const void* x16, float2* y,
                      const float2* b, int nrhs, const int* active, int* err) {
  if (nrhs <= 0) return;
  const int ns = Ls * Ls;
  const double ar = act_rhs(nrhs);
  const double flops = ar * ns * 2.0 * 32 * 160;
  if (tc_block_selected(bf, Ls, nrhs)) {  // 16-bit operands: 2x2-site items sharing slabs (tc_block.cu)
    MG_CHECK_ARG(x16, "the 2x2-block stencil reads the 16-bit copy of x");
    const double bytes = ar * ns * (64.0 + 128.0 * (b ? 2 : 1)) + (double)tc_stencil_weight_bytes(ns, bf);
    tc_block_stencil(st, bf, W, Ls, x16, y, 0, b, 0, 0, nrhs, active, err, bytes, flops);
  } else {
    const double bytes = ar * ns * 128.0 * (b ? 3 : 2) + (double)tc_stencil_weight_bytes(ns, bf);
    launch_tc_fmt<0>(bf, st, x, W, (float*)y, (const float*)b, Ls, ns, 0, 0, nrhs, active, err, bytes, flops);
  }
}

// zero the sites of every colour-`color` 2x2 block of res ([rhs][site][16 complex])
__global__ void k_zero_colour_blocks(float2* __restrict__ res, int Ls, int color, int nrhs, const int* active) {
  const int nblk = Ls * Ls / 8;  // blocks of one colour
  const size_t per_rhs = (size_t)nblk * 4 * 8;  // float4 per rhs: 4 sites x 16 complex = 8 float4 each
  const size_t total = per_rhs * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int rhs = (int)(e / per_rhs);
    if (active && !active[rhs]) continue;
    const size_t r = e - (size_t)rhs * per_rhs;
    const int item = (int)(r / 32), j = (int)(r % 32) >> 3, u = (int)(r & 7);
    const int s = block_site(item, j, Ls, color);
    reinterpret_cast<float4*>(res + ((size_t)rhs * Ls * Ls + s) * 16)[u] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// res = f - D x on the sites of the colour-0 blocks and 0 on the colour-1 blocks: the V-cycle residual after
// a SAP sweep whose last half sweep solved the colour-1 blocks.  The blocks of one colour do not couple to each
// other, so with exact block solves f - D x would vanish on them; here the block inverses, the residual feeding
// them and the stored x are TF32/BF16/FP16-accurate, so the residual that is set to zero is of the order of that
// format's rounding times |f - D x|.  Dropping it perturbs the preconditioner only: the outer flexible Krylov
// iteration and the FP64 true-residual refinement still converge to the requested residual.
void tc_residual_after_sap(cudaStream_t st, const void* Wst, int bf, int Ls, const float2* x, const void* x16,
                           float2* res, const float2* f, int nrhs, const int* active, int* err) {
  if (nrhs <= 0) return;
  const int ns = Ls * Ls;
  const double ar = act_rhs(nrhs);
  const double flops = ar * (ns / 2) * 2.0 * 32 * 160;
  if (tc_block_selected(bf, Ls, nrhs)) {
    MG_CHECK_ARG(x16, "the 2x2-block stencil reads the 16-bit copy of x");
    const double bytes = ar * (ns / 2) * (64.0 + 128.0 * 2) + (double)tc_stencil_weight_bytes(ns / 2, bf);
    tc_block_stencil(st, bf, Wst, Ls, x16, res, 0, f, 1, 0, nrhs, active, err, bytes, flops);
  } else {
    const double bytes = ar * (ns / 2) * 128.0 * 3 + (double)tc_stencil_weight_bytes(ns / 2, bf);
    launch_tc_fmt<0>(bf, st, x, Wst, (float*)res, (const float*)f, Ls, ns / 2, 1, 0, nrhs, active, err, bytes,
                     flops);
  }
  MG_LAUNCH_W(ar * (ns / 2) * 128.0, 0, k_zero_colour_blocks, 1024, 256, 0, st, res, Ls, 1, nrhs, active);
}

void tc_sap_half(cudaStream_t st, const void* Wst, const void* Winv, int bf, int Ls, const float2* f, float2* x,
                 void* x16, float2* res, int color, int nrhs, const int* active, int* err) {
  if (nrhs <= 0) return;
  const int ns = Ls * Ls, nblk = ns / 8;
  const double ar = act_rhs(nrhs);
  const double sflops = ar * (ns / 2) * 2.0 * 32 * 160, uflops = ar * nblk * 2.0 * 128 * 128;
  if (tc_block_selected(bf, Ls, nrhs)) {
    // 16-bit path: the block stencil writes r = f - D x of the colour's sites as planar 16-bit tiles (into res's
    // memory), the rhs-on-M block update reads them by TMA and updates x and its 16-bit copy
    MG_CHECK_ARG(x16, "the 2x2-block stencil reads the 16-bit copy of x");
    tc_block_stencil(st, bf, Wst, Ls, x16, res, 1, f, 1, color, nrhs, active, err,
                     ar * (ns / 2) * (64.0 + 128.0 + 64.0) + (double)tc_stencil_weight_bytes(ns / 2, bf), sflops);
    tc_block_update(st, bf, Winv, Ls, res, x, x16, color, nrhs, active, err,
                    ar * (ns / 2) * (64.0 + 128.0 * 2 + 64.0) + (double)tc_blockinv_weight_bytes(Ls, bf), uflops);
    return;
  }
  launch_tc_fmt<0>(bf, st, x, Wst, (float*)res, (const float*)f, Ls, ns / 2, 1, color, nrhs, active, err,
                   ar * (ns / 2) * 128.0 * 3 + (double)tc_stencil_weight_bytes(ns / 2, bf), sflops);
  launch_tc_fmt<1>(bf, st, res, Winv, (float*)x, nullptr, Ls, nblk, 0, color, nrhs, active, err,
                   ar * (ns / 2) * 128.0 * 3 + (double)tc_blockinv_weight_bytes(Ls, bf), uflops);
}

}  // namespace mg
