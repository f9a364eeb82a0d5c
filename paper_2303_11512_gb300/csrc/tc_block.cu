// Coarse stencil on the tensor cores, one 2x2 block of sites per item (16-bit operands: BF16 or FP16).
//
// y_s = sum_f W_(s,f) x_(s+f) over f in {self, +x, -x, +t, -t}.  With the rhs on M, the per-site form issues one
// N = 32 MMA chain per (site, slab): 20 MMAs of K = 8 (TF32) or 10 of K = 16 per site, and a tcgen05.mma costs its
// issuing thread about the same time for N = 32 as for N = 96 or 128.  Here an item is a 2x2 block of sites
// (s00, s01, s10, s11 = (t, x), (t, x+1), (t+1, x), (t+1, x+1)): each block site's slab feeds three sites of the
// block (itself and its two block neighbours), so one MMA with the three sites' weights stacked on N (a window of
// the item's 4 x 32 accumulator columns) replaces three; the 8 halo slabs feed one site each.  12 slabs x 2 K
// steps = 24 MMAs per block, 6 per site.
//
// Shared memory of a stage: 12 vector tiles (64 rhs rows x 32 16-bit values, 64-byte swizzle) converted from the
// FP32 vectors by converter warps, and the weight windows: 22 sub-tiles of 32 rows (Re rows from the per-site
// weight image by bulk copies, Im rows derived), two of them zero, arranged so that every slab's targets are
// consecutive rows:
//   slab s00: [W(s00,self) W(s01,-x) W(s10,-t)]            N =  96, columns  0..95
//   slab s01: [W(s00,+x) W(s01,self) 0 W(s11,-t)]          N = 128, columns  0..127
//   slab s10: [W(s00,+t) 0 W(s10,self) W(s11,-x)]          N = 128, columns  0..127
//   slab s11: [W(s01,+t) W(s10,+x) W(s11,self)]            N =  96, columns 32..127
//   halos:    W(s00,-x) W(s00,-t) W(s01,+x) W(s01,-t) W(s10,-x) W(s10,+t) W(s11,+x) W(s11,+t), N = 32 each.
// The halo MMAs run first (the first of each site overwrites its columns), so the zero rows of the two N = 128
// windows only add zero.  Warp roles and bounded waits as in the per-site kernel.
#include "ops.cuh"
#include "tcgen05.cuh"

namespace mg {
namespace {

constexpr int TB_MM = 64;                   // rhs per tile (MMA M)
constexpr int TB_SLABS = 12;
constexpr int TB_BROWS = 704;               // weight rows per stage (22 sub-tiles of 32)
constexpr int TB_VTILE = TB_MM * 64;        // bytes of one vector tile
constexpr int TB_STAGE = TB_SLABS * TB_VTILE + TB_BROWS * 64;
constexpr int TB_STAGES = 2;
constexpr int TB_NACC = 4;                  // accumulators (128 columns each)
constexpr int TB_PROD_WARP = 0, TB_MMA_WARP = 1, TB_EPI_WARP0 = 2, TB_EPI_WARPS = 8, TB_CONV_WARP0 = 10,
              TB_CONV_WARPS = 8;
constexpr int TB_THREADS = 32 * (TB_CONV_WARP0 + TB_CONV_WARPS);
static_assert(TB_CONV_WARP0 == TB_EPI_WARP0 + TB_EPI_WARPS, "warp roles: producer, MMA, epilogue, converters");
constexpr int TB_SMEM = 1024 + TB_STAGES * TB_STAGE;

// weight sub-tile row of (block site j, direction f), f: 0 self, 1 +x, 2 -x, 3 +t, 4 -t
__constant__ short c_rowpos[4][5] = {{0, 96, 448, 224, 480},
                                     {128, 512, 32, 352, 544},
                                     {288, 384, 576, 608, 64},
                                     {416, 640, 320, 672, 192}};
// slab q: weight window start row, N, first accumulator column
__constant__ short c_brow[TB_SLABS] = {0, 96, 224, 352, 448, 480, 512, 544, 576, 608, 640, 672};
__constant__ short c_ncol[TB_SLABS] = {96, 128, 128, 96, 32, 32, 32, 32, 32, 32, 32, 32};
__constant__ short c_col0[TB_SLABS] = {0, 0, 0, 32, 0, 0, 32, 32, 64, 64, 96, 96};
// slab q's site as (dt, dx) from the block's corner (t0, x0)
__constant__ signed char c_sdt[TB_SLABS] = {0, 0, 1, 1, 0, -1, 0, -1, 1, 2, 1, 2};
__constant__ signed char c_sdx[TB_SLABS] = {0, 1, 0, 1, -1, 0, 2, 1, -1, 0, 2, 1};
// MMA order: the first halo of each site first (they overwrite), then the others
__constant__ signed char c_order[TB_SLABS] = {4, 6, 8, 10, 5, 7, 9, 11, 0, 1, 2, 3};

__device__ __forceinline__ int tb_wrap(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// corner (t0, x0) of item k: all blocks (bmode 0, colour-0 blocks then colour-1 blocks) or the blocks of colour
// `color` (bmode 1), in the block order of the SAP sweeps
__device__ __forceinline__ void tb_corner(int k, int Ls, int bmode, int color, int& t0, int& x0) {
  const int nbx = Ls / 2, half = nbx / 2, nblk = nbx * nbx / 2;
  int c = color;
  if (!bmode && k >= nblk) {
    k -= nblk;
    c = 1;
  } else if (!bmode) {
    c = 0;
  }
  const int BT = k / half;
  const int BX = 2 * (k % half) + ((BT + c) & 1);
  t0 = 2 * BT;
  x0 = 2 * BX;
}

template <int BF>
__device__ __forceinline__ uint32_t tb_pack(float a, float b) {
  return BF == 2 ? f16x2_rn(a, b) : bf16x2_rn(a, b);
}

template <int BF>
__global__ void __launch_bounds__(TB_THREADS, 1)
    k_tcb(const float* __restrict__ xin, const unsigned char* __restrict__ W, float* __restrict__ out,
          const float* __restrict__ bvec, int Ls, int nitems, int bmode, int color, int nrhs,
          const int* __restrict__ active, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[TB_STAGES], empty_bar[TB_STAGES], xfull_bar[TB_STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[TB_NACC], tempty_bar[TB_NACC];
  __shared__ uint32_t s_taddr;
  __shared__ int s_skip;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rhs0 = blockIdx.y * TB_MM;
  const int vrows = min(TB_MM, ((nrhs - rhs0 + 7) / 8) * 8);  // vector rows converted per tile
  const long ncf = (long)Ls * Ls * 32;                          // floats per rhs row
  if (tid == 0) s_skip = *(volatile int*)err;
  __syncthreads();
  if (s_skip) return;
  // zero both stages (the two zero weight sub-tiles are never written afterwards)
  for (int i = tid; i < TB_STAGES * TB_STAGE / 16; i += TB_THREADS)
    reinterpret_cast<uint4*>(base)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < TB_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
      mbar_init(&xfull_bar[s], TB_CONV_WARPS);
    }
    for (int a = 0; a < TB_NACC; ++a) {
      mbar_init(&tfull_bar[a], 1);
      mbar_init(&tempty_bar[a], 4);  // the four lane-quarter warps of the item's parity
    }
    s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) tmem_alloc(&s_taddr, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  int n_my = 0;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) ++n_my;
  auto sV = [&](int s, int q) { return base + s * TB_STAGE + q * TB_VTILE; };
  auto sB = [&](int s) { return base + s * TB_STAGE + TB_SLABS * TB_VTILE; };

  if (warp == TB_PROD_WARP) {
    // ---------------- producer: the 20 stored weight halves of the block (lane k issues copy k)
    for (int i = 0; i < n_my; ++i) {
      const int s = i % TB_STAGES;
      int ok = lane == 0 ? !s_bad : 0;
      if (lane == 0 && ok && i >= TB_STAGES &&
          !mbar_wait(&empty_bar[s], (uint32_t)((i / TB_STAGES) - 1) & 1u)) {
        atomicExch(err, 31);
        s_bad = 1;
        ok = 0;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      if (lane == 0) mbar_expect_tx(&full_bar[s], 20u * 1024u);
      __syncwarp();
      if (lane < 20) {
        int t0, x0;
        tb_corner(blockIdx.x + i * gridDim.x, Ls, bmode, color, t0, x0);
        const int j = lane / 5, f = lane % 5;
        const int site = (t0 + (j >> 1)) * Ls + x0 + (j & 1);
        bulk_load(sB(s) + c_rowpos[j][f] * 64, W + ((size_t)site * 5 + f) * 1024, 1024, &full_bar[s]);
      }
    }
    // the last copies land before the CTA can exit (bounded)
    if (lane == 0)
      for (int i = max(0, n_my - TB_STAGES); i < n_my && !s_bad; ++i)
        mbar_wait(&full_bar[i % TB_STAGES], (uint32_t)(i / TB_STAGES) & 1u);
  } else if (warp == TB_MMA_WARP) {
    // ---------------- MMA issuer
    if (lane == 0) {
      for (int i = 0; i < n_my && !s_bad; ++i) {
        const int s = i % TB_STAGES, a = i % TB_NACC;
        if (!mbar_wait(&xfull_bar[s], (uint32_t)(i / TB_STAGES) & 1u)) {
          atomicExch(err, 32);
          s_bad = 1;
          break;
        }
        if (i >= TB_NACC && !mbar_wait(&tempty_bar[a], (uint32_t)((i / TB_NACC) - 1) & 1u)) {
          atomicExch(err, 33);
          s_bad = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d0 = taddr + (uint32_t)(a * 128);
        const uint64_t vd0 = sw64_desc(smem_u32(sV(s, 0))), bd0 = sw64_desc(smem_u32(sB(s)));
#pragma unroll
        for (int o = 0; o < TB_SLABS; ++o) {
          const int q = c_order[o];
          const int nn = c_ncol[q];
          const uint32_t idesc = BF == 2 ? idesc_f16(TB_MM, nn) : idesc_bf16(TB_MM, nn);
          const uint64_t ad = vd0 + (uint64_t)((q * TB_VTILE) >> 4), bd = bd0 + (uint64_t)((c_brow[q] * 64) >> 4);
          const uint32_t d = d0 + (uint32_t)c_col0[q];
#pragma unroll
          for (int k2 = 0; k2 < 2; ++k2) mma_bf16(d, ad + 2 * k2, bd + 2 * k2, idesc, (o >= 4 || k2 > 0) ? 1u : 0u);
        }
        mma_commit(&empty_bar[s]);  // the stage is free once these MMAs completed
        mma_commit(&tfull_bar[a]);  // accumulator a is ready for the epilogue
      }
    }
  } else if (warp >= TB_CONV_WARP0) {
    // ---------------- converters: Im rows of the weight sub-tiles; FP32 vector rows -> 16-bit operand tiles
    const int ct = (warp - TB_CONV_WARP0) * 32 + lane;
    constexpr int NT = 32 * TB_CONV_WARPS;
    for (int i = 0; i < n_my; ++i) {
      const int s = i % TB_STAGES;
      if (s_bad || !mbar_wait(&full_bar[s], (uint32_t)(i / TB_STAGES) & 1u)) {
        if (!s_bad) atomicExch(err, 35);
        s_bad = 1;
        break;
      }
      // Im rows: 20 sub-tiles x 16 rows x 4 chunks; (a, b) -> (-b, a) per 16-bit pair, same swizzle phase
      uint4* wb = reinterpret_cast<uint4*>(sB(s));
      for (int e = ct; e < 20 * 64; e += NT) {
        const int t = e >> 6, r = e & 63;
        const int row0 = c_rowpos[t / 5][t % 5];
        const uint4 v = wb[row0 * 4 + r];
        uint4 o;
        o.x = ((v.x & 0xFFFFu) << 16) | ((v.x >> 16) ^ 0x8000u);
        o.y = ((v.y & 0xFFFFu) << 16) | ((v.y >> 16) ^ 0x8000u);
        o.z = ((v.z & 0xFFFFu) << 16) | ((v.z >> 16) ^ 0x8000u);
        o.w = ((v.w & 0xFFFFu) << 16) | ((v.w >> 16) ^ 0x8000u);
        wb[(row0 + 16) * 4 + r] = o;
      }
      // vector tiles: unit (slab q, row r, 16-byte output chunk c) from two float4 of the FP32 vector
      int t0, x0;
      tb_corner(blockIdx.x + i * gridDim.x, Ls, bmode, color, t0, x0);
      const int units = TB_SLABS * vrows * 4;
      // batches of UB units per thread: 2 UB global loads in flight (the loads come mostly from L2, so the
      // converters are latency bound without them)
      constexpr int UB = 6;
      for (int u0 = ct; u0 < units; u0 += UB * NT) {
        float4 f[UB][2];
        int q2[UB], r2[UB], c2[UB];
#pragma unroll
        for (int h = 0; h < UB; ++h) {
          const int u = u0 + h * NT;
          const bool ok = u < units;
          const int q = ok ? u / (vrows * 4) : 0, rem = u - q * vrows * 4;
          const int r = rem >> 2, c = rem & 3;
          q2[h] = ok ? q : -1;
          r2[h] = r;
          c2[h] = c;
          const int rhs = rhs0 + r;
          if (ok && rhs < nrhs) {
            const int site = tb_wrap(t0 + c_sdt[q], Ls) * Ls + tb_wrap(x0 + c_sdx[q], Ls);
            const float4* src = reinterpret_cast<const float4*>(xin + (size_t)rhs * ncf + (size_t)site * 32) + 2 * c;
            f[h][0] = __ldg(src);
            f[h][1] = __ldg(src + 1);
          } else {
            f[h][0] = f[h][1] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int h = 0; h < UB; ++h) {
          if (q2[h] < 0) continue;
          uint4 o;
          o.x = tb_pack<BF>(f[h][0].x, f[h][0].y);
          o.y = tb_pack<BF>(f[h][0].z, f[h][0].w);
          o.z = tb_pack<BF>(f[h][1].x, f[h][1].y);
          o.w = tb_pack<BF>(f[h][1].z, f[h][1].w);
          const int r = r2[h];
          reinterpret_cast<uint4*>(sV(s, q2[h]))[r * 4 + (c2[h] ^ ((r >> 1) & 3))] = o;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> MMA reads
      __syncwarp();
      if (lane == 0) mbar_arrive(&xfull_bar[s]);
    }
  } else {
    // ---------------- epilogue: warp w owns TMEM lane quarter w % 4 (M = 64: rhs row r of the tile in lane
    // 32 (r / 16) + r % 16) and the items of parity (w - first epilogue warp) / 4; per site, two steps of 8
    // complex outputs (Re in columns 32 j + [0, 16), Im in 32 j + [16, 32))
    const int q = warp & 3, par = (warp - TB_EPI_WARP0) >> 2;
    const int row = q * 16 + lane;
    const int rhs = rhs0 + row;
    const bool live = lane < 16 && rhs < nrhs && !(active && !active[rhs]);
    const bool quarter_live = rhs0 + q * 16 < nrhs;  // warp-uniform
    for (int i = par; i < n_my; i += 2) {
      const int a = i % TB_NACC;
      if (s_bad || !mbar_wait(&tfull_bar[a], (uint32_t)(i / TB_NACC) & 1u)) {
        if (!s_bad) atomicExch(err, 34);
        s_bad = 1;
        break;
      }
      tc_fence_after();
      __syncwarp();
      int t0, x0;
      tb_corner(blockIdx.x + i * gridDim.x, Ls, bmode, color, t0, x0);
      const uint32_t tq = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * 128);
      if (quarter_live) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int site = (t0 + (j >> 1)) * Ls + x0 + (j & 1);
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            float v[16];  // v[0..7] Re, v[8..15] Im of complex outputs 8t .. 8t + 7
            tmem_ld8x2(tq + 32 * j + 8 * t, tq + 32 * j + 16 + 8 * t, v);
            if (live) {
              const size_t off = (size_t)rhs * ncf + (size_t)site * 32 + 16 * t;
              float4* o = reinterpret_cast<float4*>(out + off);
              if (bvec) {
                const float4* bb = reinterpret_cast<const float4*>(bvec + off);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const float4 c = bb[u];
                  o[u] = make_float4(c.x - v[2 * u], c.y - v[8 + 2 * u], c.z - v[2 * u + 1], c.w - v[9 + 2 * u]);
                }
              } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) o[u] = make_float4(v[2 * u], v[8 + 2 * u], v[2 * u + 1], v[9 + 2 * u]);
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar[a]);
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, 512);
  }
}

}  // namespace

void tc_block_stencil(cudaStream_t st, int bf, const void* W, int Ls, const float2* x, float2* y, const float2* b,
                      int bmode, int color, int nrhs, const int* active, int* err, double bytes, double flops) {
  MG_CHECK_ARG(bf == 1 || bf == 2, "the block stencil kernel takes 16-bit operands");
  MG_CHECK_ARG(Ls >= 4 && Ls % 4 == 0, "the block stencil kernel needs a lattice side that is a multiple of 4");
  const int nitems = bmode ? Ls * Ls / 8 : Ls * Ls / 4;
  int dev = 0, nsm = 152;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int tiles = (nrhs + TB_MM - 1) / TB_MM;
  const int gx = std::max(1, std::min(nitems, (nsm + tiles - 1) / tiles));
  dim3 grid(gx, tiles);
  auto go = [&](auto* k_tcb_kernel) {
    ensure_max_smem((const void*)k_tcb_kernel, TB_SMEM);
    MG_LAUNCH_W(bytes, flops, k_tcb_kernel, grid, TB_THREADS, TB_SMEM, st, (const float*)x,
                (const unsigned char*)W, (float*)y, (const float*)b, Ls, nitems, bmode, color, nrhs, active, err);
  };
  if (bf == 2)
    go(&k_tcb<2>);
  else
    go(&k_tcb<1>);
}

}  // namespace mg
