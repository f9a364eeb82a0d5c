// Tensor-core form of the learned preconditioner's layers (tcgen05, BF16 operands, FP32 accumulation).
//
// Forward layer.  The transporter T_d(x) is a complex scalar per site and offset, so it commutes with the
// channel mixing:
//   z(x) = sum_d W_d T_d(x) a(x + d) = sum_d T_d(x) [W_d a(x + d)].
// For a tile of 128 consecutive sites (one rhs) every offset d is one GEMM  P_d[128, CO] = A_d[128, CI] W_d^T
// whose A operand is the gathered input rows a(x + d) (BF16, as stored by the previous layer); the MMA
// accumulates P_d in TMEM, and the epilogue adds T_d(x) P_d(x) over the 9 offsets in FP32, then applies the
// activation (hidden layers, the BF16 result is the next layer's input) or stores the FP32 output.
//
// Input gradient.  With the reversed-path identity conj(T_d(y - d)) = T_(-d)(y) the adjoint of the forward
// scatter becomes the same gathered form:
//   g_a(y) = sum_e T_e(y) [conj(W_(-e))^T g_z(y + e)],
// so the same kernel runs with the conjugate-transposed weight image and BF16 output gradients as input.
//
// Weight gradient.  g_W[d] = sum_x g_z(x) conj(u_d(x)), u_d(x) = T_d(x) a(x + d): a GEMM whose K dimension is
// the sites.  Converter warps stage, per chunk of 64 sites, g_z (rows: Re/Im parts of the outputs) and the
// transported inputs u_d (rows: offset x input channel, rounded to BF16) K-major in shared memory, and one
// thread accumulates the whole CTA's sum of chunks in TMEM; partial sums per CTA are reduced in a fixed order.
//
// Complex products use the real embedding: an input pair (re, im) on K, output rows
// Re = [w_re, -w_im], Im = [w_im, w_re] on N.  All mbarrier waits are bounded (error code, then return).
#include <cstring>

#include "nn.cuh"
#include "tcgen05.cuh"

namespace mg {
namespace {

constexpr int NM_M = 128;        // sites per tile (MMA M = TMEM lanes)
constexpr int NM_TAPS = 9;
constexpr int NM_GROUP = 3;      // offsets per TMEM accumulator group: one commit (an expensive issue) per group
constexpr int NM_STAGES = 2;
constexpr int NM_PROD_WARPS = 4;
constexpr int NM_EPI_WARPS = 16;  // four per TMEM lane quarter: each takes 4 of the output channels
constexpr int NM_MMA_WARP = NM_PROD_WARPS;
constexpr int NM_EPI_WARP0 = NM_MMA_WARP + 1;
constexpr int NM_THREADS = 32 * (NM_EPI_WARP0 + NM_EPI_WARPS);
constexpr int NM_ROW = 64;                     // bytes per operand row: 32 BF16 (two MMA K steps), 64-byte swizzle
constexpr int NM_TILE = NM_M * NM_ROW;         // one offset's A tile
constexpr int NM_STAGE = NM_TAPS * NM_TILE;    // the 9 gathered tiles of one site tile
constexpr uint32_t NM_TMEM_COLS = 512;

// Row-segment staging (lattice side a multiple of 128, CI >= 4): a tile of 128 sites is one stretch of a
// lattice row, so the 9 gathered tiles are row windows (shifted by dx = -1, 0, 1) of three segments, the
// lattice rows t - 1, t, t + 1 from x0 - 1 to x0 + 128.  A segment is stored as K planes of 16 bytes (8 BF16)
// per site without swizzle, 130 sites 16 bytes apart, so the MMA descriptor of a window just starts dx + 1 rows
// later; TMA brings the 128 interior sites of each plane (a box of 8 elements x 128 rows) and the producer
// warp the two wrapped halo sites.
constexpr int NS_PLANE = 2304;      // bytes per plane: halo site at +112, interior sites from +128 (TMA aligned)
constexpr int NS_ROW0 = 112;        // offset of the first (halo) site of a plane
constexpr int NS_STAGES = 4;

__host__ __device__ constexpr int nm_nc(int co) { return co < 8 ? 8 : co; }  // TMEM columns per Re / Im half
__host__ __device__ constexpr int nm_n(int co) { return 2 * nm_nc(co); }     // MMA N
__host__ __device__ constexpr int nm_wbytes(int co) { return NM_TAPS * nm_n(co) * NM_ROW; }
__host__ __device__ constexpr int nm_ks(int ci) { return (2 * ci + 15) / 16; }  // MMA K steps per offset
__host__ __device__ constexpr int ns_stage(int ci) { return 3 * 2 * nm_ks(ci) * NS_PLANE; }
__host__ __device__ constexpr int nm_stage_bytes(int ci, bool seg) { return seg ? ns_stage(ci) : NM_STAGE; }
__host__ __device__ constexpr int nm_nstages(bool seg) { return seg ? NS_STAGES : NM_STAGES; }
// tail pad: every address an operand descriptor of the segment layout can form, under either assignment of its
// two strides, stays inside the allocation
constexpr int NS_TAIL = 40 * 1024;
inline int nm_smem(int ci, int co, bool seg) {
  return 1024 + nm_nstages(seg) * nm_stage_bytes(ci, seg) + nm_wbytes(co) + (seg ? NS_TAIL : 0);
}

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return (unsigned char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}
// site index of (t + dt, x + dx) for offset e = 3 (dt + 1) + (dx + 1), periodic
__device__ __forceinline__ int nm_nbr(int t, int x, int e, int L) {
  int xx = x + e % 3 - 1, tt = t + e / 3 - 1;
  xx = xx < 0 ? xx + L : (xx >= L ? xx - L : xx);
  tt = tt < 0 ? tt + L : (tt >= L ? tt - L : tt);
  return tt * L + xx;
}
__device__ __forceinline__ float2 bf16x2_to_f2(uint32_t v) {
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xFFFF0000u));
}

// EPI 0: out32 = sum_d T_d P_d (FP32).  EPI 1 (hidden layer): z = sum_d T_d P_d stored to out32 when given,
// a = z max(0, |z| + b)/|z| stored to out16 as BF16 pairs.
// in16: [rows][CI] complex BF16 (pairs), T: [site][9], wimg: [9][N rows][32] BF16 (64-byte swizzle).
template <int CI, int CO, int EPI, bool SEG>
__global__ void __launch_bounds__(NM_THREADS, 1)
    k_nn_mix(const __grid_constant__ CUtensorMap amap, const unsigned char* __restrict__ in16,
             const float2* __restrict__ T, const uint4* __restrict__ wimg, const float* __restrict__ bias,
             float2* __restrict__ out32, uint32_t* __restrict__ out16, int L, int ntiles, int* err) {
  constexpr int NC = nm_nc(CO), N = nm_n(CO);
  constexpr int GCOLS = NM_GROUP * N;                 // TMEM columns of one group of offsets
  constexpr int NSLOT = (int)NM_TMEM_COLS / GCOLS;    // groups in flight (3 per tile)
  constexpr int KS = nm_ks(CI);                 // MMA K steps of one offset (16 BF16 each)
  constexpr int IB = 4 * CI;                    // bytes of one input row
  constexpr int CH = IB >= 16 ? IB / 16 : 1;    // 16-byte chunks of a row (CI = 2: one half chunk)
  constexpr int NSTG = nm_nstages(SEG), STG = nm_stage_bytes(CI, SEG);
  constexpr int KP = 2 * KS;                    // planes per segment (those past the input's K stay zero)
  constexpr uint32_t IDESC = idesc_bf16(NM_M, N);
  static_assert(!SEG || CI >= 4, "row segments need 16-byte planes");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = align1024(smem_raw);
  unsigned char* sW = base + NSTG * STG;
  __shared__ __align__(8) uint64_t full_bar[NSTG], empty_bar[NSTG], tfull[NSLOT], tempty[NSLOT];
  __shared__ uint32_t s_taddr;
  __shared__ int s_skip;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) s_skip = *(volatile int*)err;  // an earlier launch gave up: do nothing until the host sees it
  __syncthreads();
  if (s_skip) return;
  // zero the operand stages (the K padding of narrow inputs must read as zero) and stage the weight image
  for (int i = tid; i < NSTG * STG / 16; i += NM_THREADS) reinterpret_cast<uint4*>(base)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < nm_wbytes(CO) / 16; i += NM_THREADS) reinterpret_cast<uint4*>(sW)[i] = wimg[i];
  if (tid == 0) {
    for (int s = 0; s < NSTG; ++s) {
      mbar_init(&full_bar[s], SEG ? 1 : NM_PROD_WARPS);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < NSLOT; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], NM_EPI_WARPS);
    }
    s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // zeroed stages and weights -> MMA reads
  if (warp == 0) tmem_alloc(&s_taddr, NM_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  const int V = L * L;
  int n_my = 0;
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) ++n_my;

  // plane p of segment g (lattice row t + g - 1) in stage s
  auto plane = [&](int s, int g, int p) { return base + s * STG + (g * KP + p) * NS_PLANE; };
  if (SEG && warp < NM_PROD_WARPS) {
    // ---------------- producer (one warp): TMA for the interior of the 3 x KP planes, lanes for the halo sites
    if (warp == 0) {
      constexpr int KPI = IB >= 16 ? IB / 16 : 1;  // planes that hold input
      for (int i = 0; i < n_my; ++i) {
        const int s = i % NSTG;
        int ok = !s_bad;
        if (i >= NSTG && lane == 0 && ok && !mbar_wait(&empty_bar[s], (uint32_t)((i / NSTG) - 1) & 1u)) {
          atomicExch(err, 15);
          s_bad = 1;
          ok = 0;
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) break;
        const long R0 = (long)(blockIdx.x + (long)i * gridDim.x) * NM_M;
        const long rr = R0 / V;
        const int s0 = (int)(R0 - rr * V), t0 = s0 / L, x0 = s0 - t0 * L;
        if (lane < 3 * 2 * KPI) {  // halo site (x0 - 1 or x0 + 128 of lattice row t0 + g - 1), plane p
          const int g = lane / (2 * KPI), side = (lane / KPI) & 1, p = lane % KPI;
          int tt = t0 + g - 1;
          tt = tt < 0 ? tt + L : (tt >= L ? tt - L : tt);
          const int xx = side ? (x0 + NM_M == L ? 0 : x0 + NM_M) : (x0 == 0 ? L - 1 : x0 - 1);
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(in16 + ((size_t)rr * V + (size_t)tt * L + xx) * IB) + p);
          *reinterpret_cast<uint4*>(plane(s, g, p) + NS_ROW0 + 16 * (side ? NM_M + 1 : 0)) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_expect_tx(&full_bar[s], (uint32_t)(3 * KPI * NM_M * 16));
          for (int g = 0; g < 3; ++g) {
            int tt = t0 + g - 1;
            tt = tt < 0 ? tt + L : (tt >= L ? tt - L : tt);
            const int row = (int)(rr * V + (long)tt * L + x0);
            for (int p = 0; p < KPI; ++p) tma_load_2d(plane(s, g, p) + NS_ROW0 + 16, &amap, 8 * p, row, &full_bar[s]);
          }
        }
      }
      // let the last copies land before the CTA can exit (bounded)
      if (lane == 0)
        for (int i = std::max(0, n_my - NSTG); i < n_my && !s_bad; ++i)
          mbar_wait(&full_bar[i % NSTG], (uint32_t)(i / NSTG) & 1u);
    }
  } else if (warp < NM_PROD_WARPS) {
    // ---------------- producers: gather the 9 offset tiles of every site tile (row m of tap e = input row of
    // site (t, x) + e), 16-byte chunks into the 64-byte-swizzled K-major layout
    for (int i = 0; i < n_my; ++i) {
      const int s = i % NM_STAGES;
      int ok = !s_bad;
      if (i >= NM_STAGES && lane == 0 && ok && !mbar_wait(&empty_bar[s], (uint32_t)((i / NM_STAGES) - 1) & 1u)) {
        atomicExch(err, 11);
        s_bad = 1;
        ok = 0;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      const long R0 = (long)(blockIdx.x + (long)i * gridDim.x) * NM_M;
      const long rr = R0 / V;
      const int s0 = (int)(R0 - rr * V);
      const unsigned char* src = in16 + (size_t)rr * V * IB;
      unsigned char* dst = base + s * NM_STAGE;
      for (int u = tid; u < NM_M * CH; u += NM_PROD_WARPS * 32) {
        const int m = u / CH, q = u - m * CH;
        const int site = s0 + m, t = site / L, x = site - t * L;
        const int off = m * NM_ROW + ((q ^ ((m >> 1) & 3)) << 4);
        if constexpr (IB >= 16) {
          uint4 v[NM_TAPS];
#pragma unroll
          for (int e = 0; e < NM_TAPS; ++e)
            v[e] = __ldg(reinterpret_cast<const uint4*>(src + (size_t)nm_nbr(t, x, e, L) * IB) + q);
#pragma unroll
          for (int e = 0; e < NM_TAPS; ++e) *reinterpret_cast<uint4*>(dst + e * NM_TILE + off) = v[e];
        } else {
          uint2 v[NM_TAPS];
#pragma unroll
          for (int e = 0; e < NM_TAPS; ++e)
            v[e] = __ldg(reinterpret_cast<const uint2*>(src + (size_t)nm_nbr(t, x, e, L) * IB));
#pragma unroll
          for (int e = 0; e < NM_TAPS; ++e) *reinterpret_cast<uint2*>(dst + e * NM_TILE + off) = v[e];
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> MMA reads
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_bar[s]);
    }
  } else if (warp == NM_MMA_WARP) {
    // ---------------- MMA issuer: offsets 3 gi .. 3 gi + 2 of tile i into accumulator group slot (3 i + gi) mod
    // NSLOT, one commit per group; the stage is released by the epilogue once the tile's last group completed
    if (lane == 0) {
      int g = 0;
      for (int i = 0; i < n_my && !s_bad; ++i) {
        const int s = i % NSTG;
        if (!mbar_wait(&full_bar[s], (uint32_t)(i / NSTG) & 1u)) {
          atomicExch(err, 12);
          s_bad = 1;
          break;
        }
        tc_fence_after();
        bool bad = false;
        for (int gi = 0; gi < NM_TAPS / NM_GROUP; ++gi, ++g) {
          const int sl = g % NSLOT;
          if (g >= NSLOT && !mbar_wait(&tempty[sl], (uint32_t)((g / NSLOT) - 1) & 1u)) {
            atomicExch(err, 13);
            s_bad = 1;
            bad = true;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int j = 0; j < NM_GROUP; ++j) {
            const int e = NM_GROUP * gi + j;
            const uint32_t d = taddr + (uint32_t)(sl * GCOLS + j * N);
            const uint64_t bd = sw64_desc(smem_u32(sW + e * N * NM_ROW));
            if (SEG) {  // window of segment dt + 1 starting dx + 1 sites in; a K step spans two planes
              const uint64_t ad = nosw_desc(smem_u32(plane(s, e / 3, 0) + NS_ROW0 + 16 * (e % 3)), NS_PLANE, 128);
#pragma unroll
              for (int k = 0; k < KS; ++k)
                mma_bf16(d, ad + (uint64_t)((2 * k * NS_PLANE) >> 4), bd + 2 * k, IDESC, k != 0);
            } else {
              const uint64_t ad = sw64_desc(smem_u32(base + s * NM_STAGE + e * NM_TILE));
#pragma unroll
              for (int k = 0; k < KS; ++k) mma_bf16(d, ad + 2 * k, bd + 2 * k, IDESC, k != 0);
            }
          }
          mma_commit(&tfull[sl]);
        }
        if (bad) break;
      }
    }
  } else {
    // ---------------- epilogue: warp w owns TMEM lane quarter w % 4 (row m = 32 (w % 4) + lane of the tile)
    // and a group of 4 complex outputs (the four warps of a quarter cover 16 outputs; with CO < 16 the groups
    // past CO only keep the barrier protocol).  The offsets of a tile are unrolled so that each transporter
    // stays in a register.
    const int ew = warp - NM_EPI_WARP0, q = warp & 3, h = ew >> 2;
    const int m = q * 32 + lane;
    constexpr int KH = CO < 4 ? CO : 4;
    const int k0 = 4 * h;
    const bool act = k0 < CO;  // warp-uniform
    float bb[KH];
#pragma unroll
    for (int j = 0; j < KH; ++j) bb[j] = (EPI == 1 && act) ? bias[k0 + j] : 0.f;
    int g = 0;
    bool bad = false;
    for (int i = 0; i < n_my && !bad; ++i) {
      const long R = (long)(blockIdx.x + (long)i * gridDim.x) * NM_M + m;
      const int site = (int)(R % V);
      float2 tr[NM_TAPS];
#pragma unroll
      for (int e = 0; e < NM_TAPS; ++e) tr[e] = act ? __ldg(T + (size_t)site * NM_TAPS + e) : make_float2(0.f, 0.f);
      float are[KH], aim[KH];
#pragma unroll
      for (int j = 0; j < KH; ++j) are[j] = aim[j] = 0.f;
#pragma unroll
      for (int gi = 0; gi < NM_TAPS / NM_GROUP; ++gi) {
        const int sl = (g + gi) % NSLOT;
        if (s_bad || !mbar_wait(&tfull[sl], (uint32_t)((g + gi) / NSLOT) & 1u)) {
          if (!s_bad) atomicExch(err, 14);
          s_bad = 1;
          bad = true;
          break;
        }
        tc_fence_after();
        __syncwarp();
        if (gi == NM_TAPS / NM_GROUP - 1 && ew == 0 && lane == 0)
          mbar_arrive(&empty_bar[i % NSTG]);  // every MMA of the tile has completed: its stage is free
        if (act) {
#pragma unroll
          for (int j = 0; j < NM_GROUP; ++j) {
            const int e = NM_GROUP * gi + j;
            float v[8];  // Re of outputs k0 .. k0 + 3, then Im
            const uint32_t ta = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(sl * GCOLS + j * N);
            tmem_ld4x2(ta + k0, ta + NC + k0, v);
#pragma unroll
            for (int u = 0; u < KH; ++u) {
              are[u] = fmaf(tr[e].x, v[u], fmaf(-tr[e].y, v[4 + u], are[u]));
              aim[u] = fmaf(tr[e].x, v[4 + u], fmaf(tr[e].y, v[u], aim[u]));
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[sl]);
      }
      g += NM_TAPS / NM_GROUP;
      if (bad || !act) continue;
      if (EPI == 0 || out32) {
        float2* o = out32 + (size_t)R * CO + k0;
#pragma unroll
        for (int j = 0; j < KH; ++j) o[j] = make_float2(are[j], aim[j]);
      }
      if (EPI == 1) {
        uint32_t w[KH];
#pragma unroll
        for (int j = 0; j < KH; ++j) {
          const float mg = sqrtf(are[j] * are[j] + aim[j] * aim[j]);
          const float f = mg > 0.f ? fmaxf(0.f, mg + bb[j]) / mg : 0.f;
          w[j] = bf16x2_rn(are[j] * f, aim[j] * f);
        }
        uint32_t* o = out16 + (size_t)R * CO + k0;
        if constexpr (KH == 4)
          *reinterpret_cast<uint4*>(o) = make_uint4(w[0], w[1], w[2], w[3]);
        else
#pragma unroll
          for (int j = 0; j < KH; ++j) o[j] = w[j];
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, NM_TMEM_COLS);
  }
}

// ---- weight gradient ------------------------------------------------------------------------------------
constexpr int NW_X = 64;          // sites per chunk: K = 128 (Re, Im of 64 sites), two 128-byte K halves
constexpr int NW_STAGES = 3;
constexpr int NW_CONV_WARPS = 8;
constexpr int NW_MMA_WARP = NW_CONV_WARPS;
constexpr int NW_THREADS = 32 * (NW_CONV_WARPS + 1);
constexpr int NW_AROWS = 64;      // MMA M: rows [0, CO) Re, [CO, 2 CO) Im of the outputs, the rest zero
__host__ __device__ constexpr int nw_nb(int ci) { return (9 * ci + 7) / 8 * 8; }  // MMA N (offset x channel)
__host__ __device__ constexpr int nw_stage(int ci) { return 2 * NW_AROWS * 128 + 2 * nw_nb(ci) * 128; }
inline int nw_smem(int ci) { return 1024 + NW_STAGES * nw_stage(ci); }
__host__ __device__ constexpr uint32_t nw_cols(int ci) {
  return nw_nb(ci) <= 32 ? 32u : nw_nb(ci) <= 64 ? 64u : nw_nb(ci) <= 128 ? 128u : 256u;
}

// part[cta][2 CO][9 CI]: this CTA's sums over its chunks of Re / Im (g_z conj(u_d)) for (k, d, c)
template <int CI, int CO>
__global__ void __launch_bounds__(NW_THREADS, 1)
    k_nn_wgrad(const uint32_t* __restrict__ a16, const uint32_t* __restrict__ gz16, const float2* __restrict__ T,
               int L, int nchunks, float* __restrict__ part, int* err) {
  constexpr int NB = nw_nb(CI), SB = nw_stage(CI);
  constexpr uint32_t NCOL = nw_cols(CI);
  constexpr uint32_t IDESC = idesc_bf16(NW_AROWS, NB);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = align1024(smem_raw);
  __shared__ __align__(8) uint64_t full_bar[NW_STAGES], empty_bar[NW_STAGES], done_bar;
  __shared__ uint32_t s_taddr;
  __shared__ int s_skip;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) s_skip = *(volatile int*)err;
  __syncthreads();
  if (s_skip) return;
  for (int i = tid; i < NW_STAGES * SB / 16; i += NW_THREADS) reinterpret_cast<uint4*>(base)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < NW_STAGES; ++s) {
      mbar_init(&full_bar[s], NW_CONV_WARPS);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) tmem_alloc(&s_taddr, NCOL);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  const int V = L * L;
  int n_my = 0;
  for (int it = blockIdx.x; it < nchunks; it += gridDim.x) ++n_my;
  // A tile: K half hf at base + hf * 8 KB (64 rows x 128 B); B tile: K half hf after the A halves (NB rows)
  auto sA = [&](int s, int hf) { return base + s * SB + hf * NW_AROWS * 128; };
  auto sB = [&](int s, int hf) { return base + s * SB + 2 * NW_AROWS * 128 + hf * NB * 128; };
  // 4-byte word of (row n, site xl) in a 128-byte-swizzled K-major tile: K elements 2 xl, 2 xl + 1
  auto word = [](int n, int xl) { return n * 32 + ((((xl & 31) >> 2) ^ (n & 7)) << 2) + (xl & 3); };

  if (warp < NW_CONV_WARPS) {
    for (int i = 0; i < n_my; ++i) {
      const int s = i % NW_STAGES;
      int ok = !s_bad;
      if (i >= NW_STAGES && lane == 0 && ok && !mbar_wait(&empty_bar[s], (uint32_t)((i / NW_STAGES) - 1) & 1u)) {
        atomicExch(err, 21);
        s_bad = 1;
        ok = 0;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      const long R0 = (long)(blockIdx.x + (long)i * gridDim.x) * NW_X;
      const long rr = R0 / V;
      const int s0 = (int)(R0 - rr * V);
      // A: g_z rows (Re: (g_re, g_im), Im: (g_im, -g_re) on the site's K pair)
      for (int u = tid; u < NW_X * CO; u += NW_CONV_WARPS * 32) {
        const int xl = u / CO, k = u - xl * CO;
        const uint32_t v = __ldg(gz16 + (size_t)(R0 + xl) * CO + k);
        uint32_t* A = reinterpret_cast<uint32_t*>(sA(s, xl >> 5));
        A[word(k, xl)] = v;
        A[word(CO + k, xl)] = (v >> 16) | (((v & 0xFFFFu) ^ 0x8000u) << 16);
      }
      // B: transported inputs u_d(x)_c = T_d(x) a(x + d)_c, rows d * CI + c
      for (int u = tid; u < NW_X * NM_TAPS; u += NW_CONV_WARPS * 32) {
        const int xl = u / NM_TAPS, e = u - xl * NM_TAPS;
        const int site = s0 + xl, t = site / L, x = site - t * L;
        const float2 te = __ldg(T + (size_t)site * NM_TAPS + e);
        const uint32_t* ar = a16 + ((size_t)rr * V + nm_nbr(t, x, e, L)) * CI;
        uint32_t* B = reinterpret_cast<uint32_t*>(sB(s, xl >> 5));
#pragma unroll
        for (int c = 0; c < CI; ++c) {
          const float2 av = bf16x2_to_f2(__ldg(ar + c));
          B[word(e * CI + c, xl)] = bf16x2_rn(te.x * av.x - te.y * av.y, te.x * av.y + te.y * av.x);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_bar[s]);
    }
  } else if (lane == 0) {
    // ---------------- MMA issuer: the CTA's chunks accumulate into one TMEM tile [64 rows, NB]
    bool ok = true;
    for (int i = 0; i < n_my && ok && !s_bad; ++i) {
      const int s = i % NW_STAGES;
      if (!mbar_wait(&full_bar[s], (uint32_t)(i / NW_STAGES) & 1u)) {
        atomicExch(err, 22);
        s_bad = 1;
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int t = 0; t < 8; ++t) {  // K steps of 16 BF16 (8 sites): 4 per 128-byte half
        const uint64_t ad = sw128_desc(smem_u32(sA(s, t >> 2))) + 2 * (t & 3);
        const uint64_t bd = sw128_desc(smem_u32(sB(s, t >> 2))) + 2 * (t & 3);
        mma_bf16(taddr, ad, bd, IDESC, (i | t) != 0);
      }
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&done_bar);  // completes once every MMA issued above has (an empty issue completes at once)
  }
  // ---------------- partial sums: with M = 64, accumulator row r sits in TMEM lane 32 (r / 16) + r % 16, so
  // rows 0..15 belong to warp 0 and rows 16..31 to warp 1 (lanes 0..15)
  if (warp < 2) {
    const bool ok = !s_bad && mbar_wait(&done_bar, 0);
    if (!ok && lane == 0) atomicExch(err, 23);
    if (__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
      tc_fence_after();
      const int r = 16 * warp + lane;
      float* P = part + (size_t)blockIdx.x * 2 * CO * 9 * CI;
      for (int j = 0; j < NB / 8; ++j) {
        float v[8];
        tmem_ld8(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)(8 * j), v);
        if (lane < 16 && r < 2 * CO) {
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (8 * j + u < 9 * CI) P[(size_t)r * 9 * CI + 8 * j + u] = v[u];
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, NCOL);
  }
}

// grad[2 ((d CO + k) CI + c) + {0, 1}] = sums over the CTAs (fixed order) of the Re / Im partials
__global__ void k_nn_wgrad_reduce(const float* __restrict__ part, int nblk, int ci, int co, float* __restrict__ grad) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;  // (d, k, c)
  if (w >= 9 * co * ci) return;
  const int d = w / (co * ci), k = (w / ci) % co, c = w % ci;
  const size_t stride = (size_t)2 * co * 9 * ci;
  const size_t ore = (size_t)k * 9 * ci + d * ci + c, oim = (size_t)(co + k) * 9 * ci + d * ci + c;
  double re = 0, im = 0;
  for (int b = 0; b < nblk; ++b) {
    re += part[b * stride + ore];
    im += part[b * stride + oim];
  }
  grad[2 * w] = (float)re;
  grad[2 * w + 1] = (float)im;
}

// weight image of one layer: forward B_d = W_d (rows = outputs co), or backward B_e = conj(W_(8-e))^T (rows =
// inputs ci); rows [0, NC) Re, [NC, 2 NC) Im, K element j = 2 c + part; BF16 in the 64-byte swizzle
__global__ void k_nn_wimg(const float* __restrict__ p, int ci, int co, int bwd, __nv_bfloat16* __restrict__ img) {
  const int nout = bwd ? ci : co, nin = bwd ? co : ci;
  const int NC = nout < 8 ? 8 : nout, N = 2 * NC;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (e, n, j)
  if (i >= NM_TAPS * N * 32) return;
  const int e = i / (N * 32), n = (i / 32) % N, j = i % 32;
  const int o = n < NC ? n : n - NC, c = j >> 1, part = j & 1;
  float v = 0.f;
  if (o < nout && c < nin) {
    // w = W[d][k][c'] (FP32 master, interleaved complex)
    const int d = bwd ? 8 - e : e, k = bwd ? c : o, cc = bwd ? o : c;
    const float wr = p[2 * ((d * co + k) * ci + cc)], wi = p[2 * ((d * co + k) * ci + cc) + 1];
    const float br = wr, bi = bwd ? -wi : wi;  // the complex entry b of this GEMM
    if (n < NC)
      v = part ? -bi : br;  // Re row: [b_re, -b_im]
    else
      v = part ? br : bi;   // Im row: [b_im, b_re]
  }
  img[(size_t)e * N * 32 + n * 32 + ((((j >> 3) ^ ((n >> 1) & 3)) << 3) | (j & 7))] = __float2bfloat16_rn(v);
}

// complex FP32 -> BF16 pairs, optionally scaled per rhs by 1 / s[rhs] (s = null: 1)
__global__ void k_nn_to_bf16(const float2* __restrict__ x, long n, const double* __restrict__ s,
                             uint32_t* __restrict__ y) {
  const int rhs = blockIdx.y;
  const float f = s ? (s[rhs] > 0 ? (float)(1.0 / s[rhs]) : 0.f) : 1.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float2 v = x[(size_t)rhs * n + i];
    y[(size_t)rhs * n + i] = bf16x2_rn(v.x * f, v.y * f);
  }
}

// activation backward: g (w.r.t. the activation output, FP32) and the pre-activation z -> g_z as BF16 pairs;
// bias partial sums per block
template <int CO>
__global__ void __launch_bounds__(128) k_nn_act_bwd16(const float2* __restrict__ z, const float* __restrict__ b,
                                                      const float2* __restrict__ g, long rows,
                                                      uint32_t* __restrict__ gz, float* __restrict__ bpart) {
  __shared__ float red[4][CO];
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  float rb[CO];
#pragma unroll
  for (int k = 0; k < CO; ++k) rb[k] = 0.f;
  if (i < rows) {
#pragma unroll
    for (int k = 0; k < CO; ++k) {
      const float2 zz = z[i * CO + k];
      const float2 gg = g[i * CO + k];
      const float mg = sqrtf(zz.x * zz.x + zz.y * zz.y);
      float2 o = make_float2(0.f, 0.f);
      if (mg > 0.f && mg + b[k] > 0.f) {
        const float2 ph = make_float2(zz.x / mg, zz.y / mg);
        const float rad = ph.x * gg.x + ph.y * gg.y;
        const float sc = (mg + b[k]) / mg;
        o = make_float2(rad * ph.x + sc * (gg.x - rad * ph.x), rad * ph.y + sc * (gg.y - rad * ph.y));
        rb[k] = rad;
      }
      gz[i * CO + k] = bf16x2_rn(o.x, o.y);
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < CO; ++k) {
    float v = rb[k];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
    if (l == 0) red[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < CO)
    bpart[(size_t)blockIdx.x * CO + threadIdx.x] =
        red[0][threadIdx.x] + red[1][threadIdx.x] + red[2][threadIdx.x] + red[3][threadIdx.x];
}

__global__ void k_nn_reduce_bias(const float* __restrict__ part, int nblk, int count, float* __restrict__ grad) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= count) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * count + w];
  grad[w] = (float)s;
}

template <typename F>
void with_dims_tc(int ci, int co, F&& f) {
#define MG_NNT_CASE(A, B) \
  if (ci == A && co == B) return f(std::integral_constant<int, A>(), std::integral_constant<int, B>());
  MG_NNT_CASE(2, 4) MG_NNT_CASE(4, 4) MG_NNT_CASE(4, 2)
  MG_NNT_CASE(2, 8) MG_NNT_CASE(8, 8) MG_NNT_CASE(8, 2)
  MG_NNT_CASE(2, 16) MG_NNT_CASE(16, 16) MG_NNT_CASE(16, 2)
#undef MG_NNT_CASE
  throw Error(MGMLMC_ERR_INVALID_ARG, "unsupported channel count (4, 8 or 16)");
}

// 2D view [rows][2 ci BF16] of a layer input; box 8 elements (one 16-byte plane) x 128 rows, no swizzle
CUtensorMap act_map(const void* in16, long rows, int ci) {
  MG_CHECK_ARG(((uintptr_t)in16 & 15) == 0, "layer input must be 16-byte aligned");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)(2 * ci), (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(4 * ci)};
  cuuint32_t box[2] = {8, (cuuint32_t)NM_M};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(in16), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(MGMLMC_ERR_CUDA, "cuTensorMapEncodeTiled failed (layer input)");
  return m;
}

int nsm_count() {
  int dev = 0, nsm = 152;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  return nsm;
}

// one gathered-mixing launch: in16 [rows][ci], EPI 0 -> out32 [rows][co]; EPI 1 -> out16 (+ out32 = z)
void mix_launch(cudaStream_t st, const NNet* net, int ci, int co, bool act, const void* in16, const void* wimg,
                const float* bias, float2* out32, uint32_t* out16, int nrhs, int* err) {
  const int L = net->L;
  const long rows = (long)nrhs * L * L;
  const int ntiles = (int)(rows / NM_M);
  const int grid = std::max(1, std::min(ntiles, nsm_count()));
  const double flops = 8.0 * NM_TAPS * ci * co * rows;
  const double bytes = (double)rows * (4.0 * ci + (act ? 4.0 * co + (out32 ? 8.0 * co : 0) : 8.0 * co));
  const bool seg = L % NM_M == 0 && ci >= 4;
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  if (seg) m = act_map(in16, rows, ci);
  with_dims_tc(ci, co, [&](auto CI, auto CO) {
    auto go = [&](auto* k_nn_mix_kernel, bool sg) {
      const int sm = nm_smem(CI.value, CO.value, sg);
      ensure_max_smem((const void*)k_nn_mix_kernel, sm);
      MG_LAUNCH_W(bytes, flops, k_nn_mix_kernel, grid, NM_THREADS, sm, st, m, (const unsigned char*)in16,
                  net->T.as<float2>(), (const uint4*)wimg, bias, out32, out16, L, ntiles, err);
    };
    if constexpr (CI.value >= 4) {
      if (seg) {
        if (act) go(&k_nn_mix<CI.value, CO.value, 1, true>, true);
        else go(&k_nn_mix<CI.value, CO.value, 0, true>, true);
        return;
      }
    }
    if (act) go(&k_nn_mix<CI.value, CO.value, 1, false>, false);
    else go(&k_nn_mix<CI.value, CO.value, 0, false>, false);
  });
}

__global__ void k_nn_pair(float2* __restrict__ R, float2* __restrict__ E, const float2* __restrict__ x,
                          const float2* __restrict__ v, const double* __restrict__ s, long n) {
  const int rhs = blockIdx.y;
  const float f = s[rhs] > 0 ? (float)(1.0 / s[rhs]) : 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const size_t o = (size_t)rhs * n + i;
    R[o] = make_float2(R[o].x * f, R[o].y * f);
    E[o] = make_float2((x[o].x - v[o].x) * f, (x[o].y - v[o].y) * f);
  }
}

}  // namespace

void nn_pair_finish(cudaStream_t st, float2* R, float2* E, const float2* x, const float2* v, const double* s, long n,
                    int nrhs) {
  MG_LAUNCH(k_nn_pair, dim3((unsigned)std::min<long>(cdiv(n, 256), 1024), nrhs), 256, 0, st, R, E, x, v, s, n);
}

size_t nn_tc_wimg_bytes(int co) { return (size_t)nm_wbytes(co); }

bool nn_tc_supported(int L) { return L >= 16 && L % 16 == 0; }

void nn_tc_weights(NNet* net, cudaStream_t st) {
  net->wimg.resize(2 * net->layers);
  for (int l = 0; l < net->layers; ++l) {
    const int ci = net->dim(l), co = net->dim(l + 1);
    for (int bwd = 0; bwd < 2; ++bwd) {
      const int nout = bwd ? ci : co;
      DBuf& img = net->wimg[2 * l + bwd];
      img.ensure(nn_tc_wimg_bytes(nout), st);
      const int cnt = NM_TAPS * nm_n(nout) * 32;
      MG_LAUNCH(k_nn_wimg, cdiv(cnt, 256), 256, 0, st, net->params.as<float>() + net->w_offset(l), ci, co, bwd,
                img.as<__nv_bfloat16>());
    }
  }
}

void nn_tc_forward(NNet* net, const float2* r, const double* rscale, float2* y, int nrhs, bool tape, int* err,
                   cudaStream_t st) {
  const int L = net->L, V = L * L;
  const long n = 2L * V;
  nn_tc_weights(net, st);
  const int nl = net->layers;
  net->acts16.resize(nl);
  if (tape) net->zs.resize(nl);
  // layer inputs: BF16 [nrhs][site][dim]; without a tape two ping-pong buffers suffice
  auto in_buf = [&](int l) -> DBuf& { return tape ? net->acts16[l] : net->acts16[l & 1]; };
  in_buf(0).ensure(sizeof(uint32_t) * n * nrhs, st);
  MG_LAUNCH(k_nn_to_bf16, dim3((unsigned)std::min<long>(cdiv(n, 256), 1024), nrhs), 256, 0, st, r, n, rscale,
            in_buf(0).as<uint32_t>());
  for (int l = 0; l < nl; ++l) {
    const int ci = net->dim(l), co = net->dim(l + 1);
    const bool last = l == nl - 1;
    const float* bias = last ? nullptr : net->params.as<float>() + net->w_offset(l) + 2 * 9 * co * ci;
    if (last) {
      mix_launch(st, net, ci, co, false, in_buf(l).p, net->wimg[2 * l].p, nullptr, y, nullptr, nrhs, err);
    } else {
      DBuf& nx = in_buf(l + 1);
      nx.ensure(sizeof(uint32_t) * (size_t)nrhs * V * co, st);
      float2* z = nullptr;
      if (tape) {
        net->zs[l].ensure(sizeof(float2) * (size_t)nrhs * V * co, st);
        z = net->zs[l].as<float2>();
      }
      mix_launch(st, net, ci, co, true, in_buf(l).p, net->wimg[2 * l].p, bias, z, nx.as<uint32_t>(), nrhs, err);
    }
  }
}

// gradient of the loss w.r.t. the BF16-rounded weights and the biases into net->grad, given the FP32 gradient
// g (w.r.t. the output, overwritten) of a forward with tape
void nn_tc_backward(NNet* net, float2* g, int nrhs, int* err, cudaStream_t st) {
  const int L = net->L, V = L * L;
  const long rows = (long)nrhs * V;
  const int nl = net->layers;
  DBuf gz16(sizeof(uint32_t) * rows * 16, st), ga(sizeof(float2) * rows * 16, st);
  MG_LAUNCH(k_nn_to_bf16, dim3((unsigned)std::min<long>(cdiv(2L * V, 256), 1024), nrhs), 256, 0, st, g, 2L * V,
            nullptr, gz16.as<uint32_t>());
  const int nsm = nsm_count();
  for (int l = nl - 1; l >= 0; --l) {
    const int ci = net->dim(l), co = net->dim(l + 1);
    const size_t woff = net->w_offset(l);
    if (l < nl - 1) {  // activation backward: ga (w.r.t. this layer's output) -> gz16, bias gradient
      const int nb = (int)cdiv(rows, 128);
      DBuf bpart(sizeof(float) * nb * co, st);
      const float* b = net->params.as<float>() + woff + 2 * 9 * co * ci;
      switch (co) {
        case 4: MG_LAUNCH((k_nn_act_bwd16<4>), nb, 128, 0, st, net->zs[l].as<float2>(), b, ga.as<float2>(), rows, gz16.as<uint32_t>(), bpart.as<float>()); break;
        case 8: MG_LAUNCH((k_nn_act_bwd16<8>), nb, 128, 0, st, net->zs[l].as<float2>(), b, ga.as<float2>(), rows, gz16.as<uint32_t>(), bpart.as<float>()); break;
        case 16: MG_LAUNCH((k_nn_act_bwd16<16>), nb, 128, 0, st, net->zs[l].as<float2>(), b, ga.as<float2>(), rows, gz16.as<uint32_t>(), bpart.as<float>()); break;
        default: throw Error(MGMLMC_ERR_INVALID_ARG, "unsupported hidden channel count");
      }
      MG_LAUNCH(k_nn_reduce_bias, cdiv(co, 64), 64, 0, st, bpart.as<float>(), nb, co,
                net->grad.as<float>() + woff + 2 * 9 * co * ci);
    }
    // weight gradient
    const int nchunks = (int)(rows / NW_X);
    const int grid = std::max(1, std::min(nchunks, nsm));
    DBuf part(sizeof(float) * (size_t)grid * 2 * co * 9 * ci, st);
    with_dims_tc(ci, co, [&](auto CI, auto CO) {
      auto* k = &k_nn_wgrad<CI.value, CO.value>;
      const int sm = nw_smem(CI.value);
      ensure_max_smem((const void*)k, sm);
      MG_LAUNCH_W(rows * (4.0 * co + 9 * 4.0 * ci), 8.0 * 9 * ci * co * rows, k, grid, NW_THREADS, sm, st,
                  net->acts16[l].as<uint32_t>(), gz16.as<uint32_t>(), net->T.as<float2>(), L, nchunks,
                  part.as<float>(), err);
    });
    MG_LAUNCH(k_nn_wgrad_reduce, cdiv(9 * co * ci, 128), 128, 0, st, part.as<float>(), grid, ci, co,
              net->grad.as<float>() + woff);
    // input gradient (the gathered mixing with the conjugate-transposed weights), FP32
    if (l > 0) mix_launch(st, net, co, ci, false, gz16.p, net->wimg[2 * l + 1].p, nullptr, ga.as<float2>(), nullptr, nrhs, err);
  }
}

}  // namespace mg
