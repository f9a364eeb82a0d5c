// The 16-bit (BF16 or FP16) coarse-level kernels on 2x2 blocks of sites: the stencil / SAP residual k_tcb and the
// SAP block update k_tcs (at the end of the file).
//
// Coarse stencil on the tensor cores, one 2x2 block of sites per item.
//
// y_s = sum_f W_(s,f) x_(s+f) over f in {self, +x, -x, +t, -t}.  With the rhs on M, the per-site form issues one
// N = 32 MMA chain per (site, slab): 20 MMAs of K = 8 (TF32) or 10 of K = 16 per site, and a tcgen05.mma costs its
// issuing thread about the same time for N = 32 as for N = 96 or 128.  Here an item is a 2x2 block of sites
// (s00, s01, s10, s11 = (t, x), (t, x+1), (t+1, x), (t+1, x+1)): each block site's slab feeds three sites of the
// block (itself and its two block neighbours), so one MMA with the three sites' weights stacked on N (a window of
// the item's 4 x 32 accumulator columns) replaces three; the 8 halo slabs feed one site each.  12 slabs x 2 K
// steps = 24 MMAs per block, 6 per site.
//
// Shared memory of a stage: 12 vector tiles (64 rhs rows, or 32 for launches of at most 32 rhs, x 32 16-bit
// values, 64-byte swizzle), each one TMA box of the planar 16-bit copy of x ([rhs][site][16 Re | 16 Im], kept up
// to date by the kernels that write x, rows past nrhs filled with zeros by the copy engine), and the weight
// windows: 22 sub-tiles of 32 rows (Re rows from the per-site weight image by bulk copies, Im rows derived by
// converter warps), two of them zero, arranged so that every slab's targets are consecutive rows:
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
// a vector tile holds vrows_t = 64 rhs rows (32 where the launch has at most 32 rhs: the M = 64 MMA then also reads
// the next 2 KB as rows 32..63, whose accumulator rows are never stored), so a stage is 92 KB or 68 KB and the
// pipeline 2 or 3 stages deep
constexpr int TB_MAXST = 3;
__host__ __device__ constexpr int tb_stage_bytes(int vrows_t) { return TB_SLABS * vrows_t * 64 + TB_BROWS * 64; }
__host__ __device__ constexpr int tb_stages(int vrows_t) { return vrows_t == 32 ? 3 : 2; }
constexpr int TB_NACC = 4;                  // accumulators (128 columns each)
constexpr int TB_PROD_WARP = 0, TB_MMA_WARP = 1, TB_EPI_WARP0 = 2, TB_EPI_WARPS = 8, TB_CONV_WARP0 = 10,
              TB_CONV_WARPS = 4;

constexpr int TB_THREADS = 32 * (TB_CONV_WARP0 + TB_CONV_WARPS);
static_assert(TB_CONV_WARP0 == TB_EPI_WARP0 + TB_EPI_WARPS, "warp roles: producer, MMA, epilogue, converters");
constexpr int TB_EBUF = 2048;  // per epilogue warp and slot: one site of its 16 rhs rows (b in, the output out)
// epilogue buffers: two slots for each warp whose lane quarter can hold rhs (all 8 warps, or the 4 of quarters
// 0 and 1 with 32-row tiles)
__host__ __device__ constexpr int tb_smem_bytes(int vrows_t) {
  return 1024 + tb_stages(vrows_t) * tb_stage_bytes(vrows_t) + (vrows_t == 32 ? 4 : 8) * 2 * TB_EBUF;
}
static_assert(tb_smem_bytes(32) <= 227 * 1024 && tb_smem_bytes(64) <= 227 * 1024, "shared memory per CTA");

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

template <int BF>
__device__ __forceinline__ uint32_t tb_pack(float a, float b) {
  return BF == 2 ? f16x2_rn(a, b) : bf16x2_rn(a, b);
}

// 16-byte global -> shared copy without a register round trip (completion by commit / wait groups)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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

// O16 = 0: y (FP32, [rhs][site][16 complex]); O16 = 1: y as a planar 16-bit tile ([rhs][site][16 Re | 16 Im],
// the A operand of the SAP block update k_tcs)
template <int BF, int O16>
__global__ void __launch_bounds__(TB_THREADS, 1)
    k_tcb(const __grid_constant__ CUtensorMap xmap, const unsigned char* __restrict__ W, void* __restrict__ out,
          const float* __restrict__ bvec, int Ls, int nitems, int bmode, int color, int nrhs, int vrows_t,
          const int* __restrict__ active, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[TB_MAXST], empty_bar[TB_MAXST], xfull_bar[TB_MAXST];
  __shared__ __align__(8) uint64_t tfull_bar[TB_NACC], tempty_bar[TB_NACC];
  __shared__ uint32_t s_taddr;
  __shared__ int s_skip;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rhs0 = blockIdx.y * TB_MM;
  const int vtile = vrows_t * 64, stage = tb_stage_bytes(vrows_t), nst = tb_stages(vrows_t);
  const uint32_t tx = 20u * 1024u + (uint32_t)(TB_SLABS * vtile);  // bytes landing in a stage per item
  const long ncf = (long)Ls * Ls * 32;  // floats per rhs row
  if (tid == 0) s_skip = *(volatile int*)err;
  __syncthreads();
  if (s_skip) return;
  // the two zero weight sub-tiles (rows 160..191 and 256..287 of every stage's weight windows) are never written
  // by the pipeline: clear them once
  for (int i = tid; i < nst * 2 * 32 * 4; i += TB_THREADS) {
    const int st = i / 256, z = (i >> 7) & 1, e = i & 127;
    reinterpret_cast<uint4*>(base + st * stage + TB_SLABS * vtile + (z ? 256 : 160) * 64)[e] =
        make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
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
  auto sV = [&](int s, int q) { return base + s * stage + q * vtile; };
  auto sB = [&](int s) { return base + s * stage + TB_SLABS * vtile; };

  if (warp == TB_PROD_WARP) {
    // ---------------- producer: lanes 0..19 the 20 stored weight halves of the block (lane 5 j + f: site j,
    // direction f), lanes 20..31 the 12 vector slabs (TMA boxes of the 16-bit copy)
    for (int i = 0; i < n_my; ++i) {
      const int s = i % nst;
      int ok = lane == 0 ? !s_bad : 0;
      if (lane == 0 && ok && i >= nst && !mbar_wait(&empty_bar[s], (uint32_t)((i / nst) - 1) & 1u)) {
        atomicExch(err, 31);
        s_bad = 1;
        ok = 0;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      if (lane == 0) mbar_expect_tx(&full_bar[s], tx);
      __syncwarp();
      int t0, x0;
      tb_corner(blockIdx.x + i * gridDim.x, Ls, bmode, color, t0, x0);
      if (lane < 20) {
        const int j = lane / 5, f = lane % 5;
        const int site = (t0 + (j >> 1)) * Ls + x0 + (j & 1);
        bulk_load(sB(s) + c_rowpos[j][f] * 64, W + ((size_t)site * 5 + f) * 1024, 1024, &full_bar[s]);
      } else {
        const int q = lane - 20;
        const int site = tb_wrap(t0 + c_sdt[q], Ls) * Ls + tb_wrap(x0 + c_sdx[q], Ls);
        tma_load_2d(sV(s, q), &xmap, site * 32, rhs0, &full_bar[s]);
      }
    }
    // the last copies land before the CTA can exit (bounded)
    if (lane == 0)
      for (int i = max(0, n_my - nst); i < n_my && !s_bad; ++i) mbar_wait(&full_bar[i % nst], (uint32_t)(i / nst) & 1u);
  } else if (warp == TB_MMA_WARP) {
    // ---------------- MMA issuer
    if (lane == 0) {
      for (int i = 0; i < n_my && !s_bad; ++i) {
        const int s = i % nst, a = i % TB_NACC;
        if (!mbar_wait(&xfull_bar[s], (uint32_t)(i / nst) & 1u)) {
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
          const uint64_t ad = vd0 + (uint64_t)((q * vtile) >> 4), bd = bd0 + (uint64_t)((c_brow[q] * 64) >> 4);
          const uint32_t d = d0 + (uint32_t)c_col0[q];
#pragma unroll
          for (int k2 = 0; k2 < 2; ++k2) mma_bf16(d, ad + 2 * k2, bd + 2 * k2, idesc, (o >= 4 || k2 > 0) ? 1u : 0u);
        }
        mma_commit(&empty_bar[s]);  // the stage is free once these MMAs completed
        mma_commit(&tfull_bar[a]);  // accumulator a is ready for the epilogue
      }
    }
  } else if (warp >= TB_CONV_WARP0) {
    // ---------------- converters: the Im rows of the weight sub-tiles (planar K: logical chunk c of an Im row
    // is chunk c ^ 2 of its Re row, negated for c < 2; rows n and n + 16 share the swizzle phase)
    const int ct = (warp - TB_CONV_WARP0) * 32 + lane;
    constexpr int NT = 32 * TB_CONV_WARPS;
    for (int i = 0; i < n_my; ++i) {
      const int s = i % nst;
      if (s_bad || !mbar_wait(&full_bar[s], (uint32_t)(i / nst) & 1u)) {
        if (!s_bad) atomicExch(err, 35);
        s_bad = 1;
        break;
      }
      uint4* wb = reinterpret_cast<uint4*>(sB(s));
#pragma unroll 2
      for (int e = ct; e < 20 * 64; e += NT) {
        const int t = e >> 6, r = e & 63;
        const int c0 = c_rowpos[t / 5][t % 5] * 4 + r;  // chunk index of the Re row position
        const uint32_t neg = (((c0 & 3) ^ ((c0 >> 3) & 3)) & 2) ? 0u : 0x80008000u;
        const uint4 v = wb[c0 ^ 2];
        wb[c0 + 64] = make_uint4(v.x ^ neg, v.y ^ neg, v.z ^ neg, v.w ^ neg);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> MMA reads
      __syncwarp();
      if (lane == 0) mbar_arrive(&xfull_bar[s]);
    }
  } else {
    // ---------------- epilogue: warp w owns TMEM lane quarter w % 4 (M = 64: rhs row r of the tile in lane
    // 32 (r / 16) + r % 16) and the items of parity (w - first epilogue warp) / 4; per site j, Re outputs in
    // columns 32 j + [0, 16), Im in 32 j + [16, 32).  Memory traffic goes through two per-warp slots of one site
    // x 16 rows: the additive input b of the next site is copied in (cp.async, each instruction 4 whole 128-byte
    // rows) while the current one is used, and the outputs are staged in the slot just read and stored with
    // each instruction covering whole row segments, instead of 16-byte pieces of 16 rows.
    const int q = warp & 3, ew = warp - TB_EPI_WARP0, par = ew >> 2;
    const int row = q * 16 + lane;
    const int rhs = rhs0 + row;
    const bool live = lane < 16 && rhs < nrhs && !(active && !active[rhs]);
    const bool quarter_live = rhs0 + q * 16 < nrhs;  // warp-uniform
    const unsigned live_mask = __ballot_sync(0xffffffffu, live);  // bit r: row r of the quarter is stored
    const int rows_here = min(16, max(0, nrhs - (rhs0 + q * 16)));
    unsigned char* ebuf = base + nst * stage + (vrows_t == 32 ? 2 * par + (q & 1) : ew) * 2 * TB_EBUF;
    // the warp's site sequence g = 4 (k-th item of the parity) + j
    const int n_par = n_my > par ? (n_my - par + 1) / 2 : 0;
    auto site_g = [&](int g) -> int {
      int t0, x0;
      tb_corner(blockIdx.x + (par + 2 * (g >> 2)) * gridDim.x, Ls, bmode, color, t0, x0);
      const int j = g & 3;
      return (t0 + (j >> 1)) * Ls + x0 + (j & 1);
    };
    auto fetch_b = [&](int g) {  // rows 4k + lane / 8, 16-byte chunk lane % 8 (swizzled by the row)
      if (bvec && quarter_live && g < 4 * n_par) {
        const int site = site_g(g);
        unsigned char* slot = ebuf + (g & 1) * TB_EBUF;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int r = 4 * k + (lane >> 3), c = lane & 7;
          if (r < rows_here)
            cp_async16(slot + r * 128 + ((c ^ (r & 7)) << 4),
                       bvec + (size_t)(rhs0 + q * 16 + r) * ncf + (size_t)site * 32 + 4 * c);
        }
      }
      cp_async_commit();
    };
    fetch_b(0);
    for (int ii = 0; ii < n_par; ++ii) {
      const int i = par + 2 * ii;
      const int a = i % TB_NACC;
      if (s_bad || !mbar_wait(&tfull_bar[a], (uint32_t)(i / TB_NACC) & 1u)) {
        if (!s_bad) atomicExch(err, 34);
        s_bad = 1;
        break;
      }
      tc_fence_after();
      __syncwarp();
      const uint32_t tq = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * 128);
#pragma unroll 1
      for (int j = 0; j < 4; ++j) {
        const int g = 4 * ii + j;
        fetch_b(g + 1);  // into the other slot, read two sites ago
        cp_async_wait1();
        __syncwarp();
        if (!quarter_live) continue;
        unsigned char* slot = ebuf + (g & 1) * TB_EBUF;
        float vs[32];  // vs[0..15] Re, vs[16..31] Im of the site's 16 complex outputs, this lane's row
        tmem_ld16x2(tq + 32 * j, tq + 32 * j + 16, vs);
        if (bvec && lane < 16) {  // y = b - D x; b's complex k at floats 2k, 2k + 1 of the row
          const float4* bs = reinterpret_cast<const float4*>(slot + lane * 128);
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 bb = bs[c ^ (lane & 7)];
            vs[2 * c] = bb.x - vs[2 * c];
            vs[16 + 2 * c] = bb.y - vs[16 + 2 * c];
            vs[2 * c + 1] = bb.z - vs[2 * c + 1];
            vs[17 + 2 * c] = bb.w - vs[17 + 2 * c];
          }
        }
        __syncwarp();  // the slot's b is read: stage the outputs in it
        if (lane < 16) {
          if (O16) {  // 64-byte row: chunks Re 0..7, Re 8..15, Im 0..7, Im 8..15
            uint4* os = reinterpret_cast<uint4*>(slot + lane * 64);
            const int sw = (lane >> 1) & 3;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const float* h = vs + (c >> 1) * 16 + (c & 1) * 8;
              os[c ^ sw] = make_uint4(tb_pack<BF>(h[0], h[1]), tb_pack<BF>(h[2], h[3]), tb_pack<BF>(h[4], h[5]),
                                      tb_pack<BF>(h[6], h[7]));
            }
          } else {  // 128-byte row, interleaved (Re, Im)
            float4* os = reinterpret_cast<float4*>(slot + lane * 128);
#pragma unroll
            for (int c = 0; c < 8; ++c)
              os[c ^ (lane & 7)] = make_float4(vs[2 * c], vs[16 + 2 * c], vs[2 * c + 1], vs[17 + 2 * c]);
          }
        }
        __syncwarp();
        const int site = site_g(g);
        if (O16) {  // 2 instructions of 8 rows x 64 bytes
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int r = 8 * k + (lane >> 2), c = lane & 3;
            if ((live_mask >> r) & 1u) {
              const uint4 v = reinterpret_cast<const uint4*>(slot + r * 64)[c ^ ((r >> 1) & 3)];
              *reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(out) + (size_t)(rhs0 + q * 16 + r) * ncf +
                                        (size_t)site * 32 + 8 * c) = v;
            }
          }
        } else {  // 4 instructions of 4 rows x 128 bytes
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int r = 4 * k + (lane >> 3), c = lane & 7;
            if ((live_mask >> r) & 1u) {
              const float4 v = reinterpret_cast<const float4*>(slot + r * 128)[c ^ (r & 7)];
              *reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + (size_t)(rhs0 + q * 16 + r) * ncf +
                                         (size_t)site * 32 + 4 * c) = v;
            }
          }
        }
        __syncwarp();  // the slot is refilled two sites later
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar[a]);
    }
    cp_async_wait0();
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, 512);
  }
}

// ---------------------------------------------------------------------------------------------------------------
// SAP block update x_B += inv_B r_B for the 2x2 blocks of one colour, rhs on M: per block the A operand is the
// block's 4 residual slabs (the planar 16-bit tiles that k_tcb<BF, 1> wrote, TMA boxes of 64 rhs rows x 32
// values), the B operand the block inverse image (4 K chunks of 64 stored Re rows x 32 values, Im rows derived),
// N = 128 outputs (accumulator columns 16 j + i: Re of dof i of block site j, 64 + 16 j + i: its Im part), 8 MMAs
// of K = 16.  The old x of the block's sites comes by TMA too (FP32 boxes of 64 rhs rows x 32 floats, 128-byte
// swizzle) into one shared-memory slot per epilogue parity, issued by a warp of its own as soon as the slot is
// free; the epilogue adds the product in place (rows of inactive rhs keep their values) and one thread of the
// parity writes the slot back with TMA stores (whole 128-byte rows, instead of 16-byte pieces of 16 rows per
// warp instruction); the updated sites' planar 16-bit copy is stored from registers.
constexpr int TS_STAGES = 3;
constexpr int TS_ATILE = TB_MM * 64;                   // one residual slab
constexpr int TS_BTILE = 128 * 64;                     // one K chunk of the inverse image (Re and Im rows)
constexpr int TS_STAGE = 4 * TS_ATILE + 4 * TS_BTILE;  // 48 KB
constexpr int TS_XBYTES = 2 * 4 * TB_MM * 128;         // old-x slots: 2 of 64 rows or 4 of 32 rows x 4 sites
constexpr uint32_t TS_TX = 4u * TS_ATILE + 4u * 64u * 64u;
constexpr int TS_XPROD_WARP = TB_CONV_WARP0 + TB_CONV_WARPS;
constexpr int TS_THREADS = 32 * (TS_XPROD_WARP + 1);
constexpr int TS_SMEM = 1024 + TS_STAGES * TS_STAGE + TS_XBYTES;

template <int BF>
__global__ void __launch_bounds__(TS_THREADS, 1)
    k_tcs(const __grid_constant__ CUtensorMap rmap, const __grid_constant__ CUtensorMap xmap,
          const unsigned char* __restrict__ Winv, float* __restrict__ x, uint16_t* __restrict__ x16, int Ls, int nitems,
          int color, int nrhs, int xrows, const int* __restrict__ active, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[TS_STAGES], empty_bar[TS_STAGES], xfull_bar[TS_STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[TB_NACC], tempty_bar[TB_NACC];
  __shared__ __align__(8) uint64_t oxfull_bar[4], oxempty_bar[4];  // old-x slots (items i, i + nxs, ... share one)
  __shared__ __align__(8) uint64_t edone_bar[4];                    // the parity's warps finished the slot
  __shared__ uint32_t s_taddr;
  __shared__ int s_skip;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rhs0 = blockIdx.y * TB_MM;
  const long ncf = (long)Ls * Ls * 32;  // floats (and 16-bit values) per rhs row
  if (tid == 0) s_skip = *(volatile int*)err;
  __syncthreads();
  if (s_skip) return;
  if (tid == 0) {
    for (int s = 0; s < TS_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
      mbar_init(&xfull_bar[s], TB_CONV_WARPS);
    }
    for (int a = 0; a < TB_NACC; ++a) {
      mbar_init(&tfull_bar[a], 1);
      mbar_init(&tempty_bar[a], 4);
    }
    for (int p = 0; p < 4; ++p) {
      mbar_init(&oxfull_bar[p], 1);
      mbar_init(&oxempty_bar[p], 1);  // the storing thread of the parity, once its stores have read the slot
      mbar_init(&edone_bar[p], 4);    // the four lane-quarter warps of the parity
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
  auto sA = [&](int s, int kc) { return base + s * TS_STAGE + kc * TS_ATILE; };
  auto sB = [&](int s, int kc) { return base + s * TS_STAGE + 4 * TS_ATILE + kc * TS_BTILE; };
  // old-x slots: xrows rows per site slab (64, or 32 where the launch has at most 32 rhs: then 4 slots), the slot
  // of item i is i % nxs, so each epilogue parity owns nxs / 2 of them
  const int nxs = xrows == 32 ? 4 : 2, xtile = xrows * 128;
  auto sX = [&](int sl, int j) { return base + TS_STAGES * TS_STAGE + (sl * 4 + j) * xtile; };
  auto site_of = [&](int i, int j) -> int {
    int t0, x0;
    tb_corner(blockIdx.x + i * gridDim.x, Ls, 1, color, t0, x0);
    return (t0 + (j >> 1)) * Ls + x0 + (j & 1);
  };

  if (warp == TB_PROD_WARP) {
    // ---------------- producer: lanes 0..3 the stored Re rows of K chunk kc, lanes 4..7 the residual slab of
    // block site kc
    for (int i = 0; i < n_my; ++i) {
      const int s = i % TS_STAGES;
      int ok = lane == 0 ? !s_bad : 0;
      if (lane == 0 && ok && i >= TS_STAGES &&
          !mbar_wait(&empty_bar[s], (uint32_t)((i / TS_STAGES) - 1) & 1u)) {
        atomicExch(err, 41);
        s_bad = 1;
        ok = 0;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      if (lane == 0) mbar_expect_tx(&full_bar[s], TS_TX);
      __syncwarp();
      const int item = blockIdx.x + i * gridDim.x;
      if (lane < 4)
        bulk_load(sB(s, lane), Winv + ((size_t)item * 4 + lane) * 4096, 4096, &full_bar[s]);
      else if (lane < 8)
        tma_load_2d(sA(s, lane - 4), &rmap, site_of(i, lane - 4) * 32, rhs0, &full_bar[s]);
    }
    if (lane == 0)
      for (int i = max(0, n_my - TS_STAGES); i < n_my && !s_bad; ++i)
        mbar_wait(&full_bar[i % TS_STAGES], (uint32_t)(i / TS_STAGES) & 1u);
  } else if (warp == TS_XPROD_WARP) {
    // ---------------- old-x producer: item i's 4 site slabs into slot i % nxs once the epilogue warps released
    // it (lane j issues site j)
    for (int i = 0; i < n_my; ++i) {
      const int sl = i % nxs;
      int ok = lane == 0 ? !s_bad : 0;
      if (lane == 0 && ok && i >= nxs && !mbar_wait(&oxempty_bar[sl], (uint32_t)((i / nxs) - 1) & 1u)) {
        atomicExch(err, 46);
        s_bad = 1;
        ok = 0;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      if (lane == 0) mbar_expect_tx(&oxfull_bar[sl], (uint32_t)(4 * xtile));
      __syncwarp();
      if (lane < 4) tma_load_2d(sX(sl, lane), &xmap, site_of(i, lane) * 32, rhs0, &oxfull_bar[sl]);
    }
    if (lane == 0)
      for (int i = max(0, n_my - nxs); i < n_my && !s_bad; ++i)
        mbar_wait(&oxfull_bar[i % nxs], (uint32_t)(i / nxs) & 1u);
  } else if (warp == TB_MMA_WARP) {
    // ---------------- MMA issuer: D[rhs][n] = sum_k r[rhs][k] inv[n][k], K chunk kc = block site kc
    if (lane == 0) {
      const uint32_t idesc = BF == 2 ? idesc_f16(TB_MM, 128) : idesc_bf16(TB_MM, 128);
      const uint64_t ad0 = sw64_desc(smem_u32(sA(0, 0))), bd0 = sw64_desc(smem_u32(sB(0, 0)));
      for (int i = 0; i < n_my && !s_bad; ++i) {
        const int s = i % TS_STAGES, a = i % TB_NACC;
        if (!mbar_wait(&xfull_bar[s], (uint32_t)(i / TS_STAGES) & 1u)) {
          atomicExch(err, 42);
          s_bad = 1;
          break;
        }
        if (i >= TB_NACC && !mbar_wait(&tempty_bar[a], (uint32_t)((i / TB_NACC) - 1) & 1u)) {
          atomicExch(err, 43);
          s_bad = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = taddr + (uint32_t)(a * 128);
        const uint64_t ads = ad0 + (uint64_t)((s * TS_STAGE) >> 4), bds = bd0 + (uint64_t)((s * TS_STAGE) >> 4);
#pragma unroll
        for (int kc = 0; kc < 4; ++kc)
#pragma unroll
          for (int k2 = 0; k2 < 2; ++k2)
            mma_bf16(d, ads + (uint64_t)((kc * TS_ATILE) >> 4) + 2 * k2, bds + (uint64_t)((kc * TS_BTILE) >> 4) + 2 * k2,
                     idesc, (kc | k2) ? 1u : 0u);
        mma_commit(&empty_bar[s]);
        mma_commit(&tfull_bar[a]);
      }
    }
  } else if (warp >= TB_CONV_WARP0) {
    // ---------------- converters: Im rows 64 + n of every K chunk from its stored Re row n (planar K: logical
    // chunk c of the Im row is chunk c ^ 2 of the Re row, negated for c < 2; rows n and n + 64 share the phase)
    const int ct = (warp - TB_CONV_WARP0) * 32 + lane;
    constexpr int NT = 32 * TB_CONV_WARPS;
    for (int i = 0; i < n_my; ++i) {
      const int s = i % TS_STAGES;
      if (s_bad || !mbar_wait(&full_bar[s], (uint32_t)(i / TS_STAGES) & 1u)) {
        if (!s_bad) atomicExch(err, 45);
        s_bad = 1;
        break;
      }
#pragma unroll 2
      for (int e = ct; e < 4 * 256; e += NT) {
        uint4* wb = reinterpret_cast<uint4*>(sB(s, e >> 8));
        const int c0 = e & 255;  // chunk index within the stored Re rows (64 rows x 4 chunks)
        const uint32_t neg = (((c0 & 3) ^ ((c0 >> 3) & 3)) & 2) ? 0u : 0x80008000u;
        const uint4 v = wb[c0 ^ 2];
        wb[c0 + 256] = make_uint4(v.x ^ neg, v.y ^ neg, v.z ^ neg, v.w ^ neg);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&xfull_bar[s]);
    }
  } else {
    // ---------------- epilogue: warp w owns TMEM lane quarter w % 4 (rhs row r in lane 32 (r / 16) + r % 16)
    // and the items of parity p = (w - first epilogue warp) / 4 (item i's old x in slot i % nxs); step k =
    // (block site j = k / 2, complex dofs 8 (k % 2) .. + 7): x += product
    const int q = warp & 3, par = (warp - TB_EPI_WARP0) >> 2;
    const int row = q * 16 + lane;
    const int rhs = rhs0 + row;
    const bool exists = lane < 16 && rhs < nrhs;
    const bool live = exists && !(active && !active[rhs]);
    const bool quarter_live = rhs0 + q * 16 < nrhs;
    const bool storer = q == 0 && lane == 0;
    for (int i = par; i < n_my; i += 2) {
      const int a = i % TB_NACC;
      if (s_bad || !mbar_wait(&tfull_bar[a], (uint32_t)(i / TB_NACC) & 1u) ||
          !mbar_wait(&oxfull_bar[i % nxs], (uint32_t)(i / nxs) & 1u)) {
        if (!s_bad) atomicExch(err, 44);
        s_bad = 1;
        break;
      }
      tc_fence_after();
      __syncwarp();
      const uint32_t tq = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * 128);
      float vs[32];  // site j's product: vs[0..15] Re, vs[16..31] Im of dofs 0 .. 15
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int j = k >> 1, t = k & 1;
        if (!quarter_live) continue;
        if (t == 0) tmem_ld16x2(tq + 16 * j, tq + 64 + 16 * j, vs);  // one TMEM wait per site
        float v[16];  // v[0..7] Re, v[8..15] Im of dofs 8t .. 8t + 7 of block site j
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          v[e] = vs[8 * t + e];
          v[8 + e] = vs[16 + 8 * t + e];
        }
        if (exists) {
          // old x: FP32 chunks 4t .. 4t+3 of this row of site j's slab (128-byte swizzle: chunk c at c ^ (row & 7)),
          // updated in place
          float4* xs = reinterpret_cast<float4*>(sX(i % nxs, j)) + row * 8;
          float4 cur[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) cur[u] = xs[(4 * t + u) ^ (row & 7)];
#pragma unroll
          for (int u = 0; u < 4; ++u) {  // inactive rhs: x unchanged (their product rows may hold anything)
            v[2 * u] = live ? v[2 * u] + cur[u].x : cur[u].x;
            v[8 + 2 * u] = live ? v[8 + 2 * u] + cur[u].y : cur[u].y;
            v[2 * u + 1] = live ? v[2 * u + 1] + cur[u].z : cur[u].z;
            v[9 + 2 * u] = live ? v[9 + 2 * u] + cur[u].w : cur[u].w;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            xs[(4 * t + u) ^ (row & 7)] = make_float4(v[2 * u], v[8 + 2 * u], v[2 * u + 1], v[9 + 2 * u]);
          const int site = site_of(i, j);
          uint16_t* o16 = x16 + (size_t)rhs * ncf + (size_t)site * 32 + 8 * t;
          uint4 re, im;
          re.x = tb_pack<BF>(v[0], v[1]), re.y = tb_pack<BF>(v[2], v[3]);
          re.z = tb_pack<BF>(v[4], v[5]), re.w = tb_pack<BF>(v[6], v[7]);
          im.x = tb_pack<BF>(v[8], v[9]), im.y = tb_pack<BF>(v[10], v[11]);
          im.z = tb_pack<BF>(v[12], v[13]), im.w = tb_pack<BF>(v[14], v[15]);
          *reinterpret_cast<uint4*>(o16) = re;
          *reinterpret_cast<uint4*>(o16 + 16) = im;
        }
      }
      tc_fence_before();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // slot writes -> TMA store reads
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&tempty_bar[a]);
        mbar_arrive(&edone_bar[i % nxs]);
      }
      if (q == 0) {  // the storing warp (warp-uniform wait; lane 0 issues the stores)
        if (!mbar_wait(&edone_bar[i % nxs], (uint32_t)(i / nxs) & 1u)) {
          if (lane == 0) atomicExch(err, 47);
          s_bad = 1;
          break;
        }
        if (storer) {
          for (int j = 0; j < 4; ++j) tma_store_2d(&xmap, sX(i % nxs, j), site_of(i, j) * 32, rhs0);
          bulk_commit();
          bulk_wait_read0();  // the slot may be refilled once the stores have read it
          mbar_arrive(&oxempty_bar[i % nxs]);
        }
        __syncwarp();
      }
    }
    if (storer) bulk_wait0();  // the stores have landed before the CTA exits
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, 512);
  }
}

// 2D view [nrhs rows][ns x 32 16-bit values]; box 32 values (one site, 64 B) x `rows` rows, 64-byte swizzle (rows
// past nrhs are filled with zeros by the copy engine)
CUtensorMap map16(const void* v, int ns, int nrhs, int rows) {
  MG_CHECK_ARG(v && ((uintptr_t)v & 15) == 0, "16-bit coarse vector: 16-byte aligned device pointer");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)ns * 32, (cuuint64_t)nrhs};
  cuuint64_t strides[1] = {(cuuint64_t)ns * 64};
  cuuint32_t box[2] = {32, (cuuint32_t)rows};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(v), dims, strides, box, es,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(MGMLMC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

dim3 grid_of(int nitems, int nrhs) {
  int dev = 0, nsm = 152;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int tiles = (nrhs + TB_MM - 1) / TB_MM;
  return dim3(std::max(1, std::min(nitems, (nsm + tiles - 1) / tiles)), tiles);
}

}  // namespace

void tc_block_stencil(cudaStream_t st, int bf, const void* W, int Ls, const void* x16, void* y, int y16,
                      const float2* b, int bmode, int color, int nrhs, const int* active, int* err, double bytes,
                      double flops) {
  MG_CHECK_ARG(bf == 1 || bf == 2, "the block stencil kernel takes 16-bit operands");
  MG_CHECK_ARG(Ls >= 4 && Ls % 4 == 0, "the block stencil kernel needs a lattice side that is a multiple of 4");
  MG_CHECK_ARG(!y16 || bmode, "16-bit output: colour blocks only");
  const int vrows_t = nrhs <= 32 ? 32 : TB_MM;
  const CUtensorMap xmap = map16(x16, Ls * Ls, nrhs, vrows_t);
  const int nitems = bmode ? Ls * Ls / 8 : Ls * Ls / 4;
  const dim3 grid = grid_of(nitems, nrhs);
  const int smem = tb_smem_bytes(vrows_t);
  auto go = [&](auto* k_tcb_kernel) {
    ensure_max_smem((const void*)k_tcb_kernel, tb_smem_bytes(32) > tb_smem_bytes(64) ? tb_smem_bytes(32)
                                                                                      : tb_smem_bytes(64));
    MG_LAUNCH_W(bytes, flops, k_tcb_kernel, grid, TB_THREADS, smem, st, xmap, (const unsigned char*)W, y,
                (const float*)b, Ls, nitems, bmode, color, nrhs, vrows_t, active, err);
  };
  if (bf == 2)
    y16 ? go(&k_tcb<2, 1>) : go(&k_tcb<2, 0>);
  else
    y16 ? go(&k_tcb<1, 1>) : go(&k_tcb<1, 0>);
}

void tc_block_update(cudaStream_t st, int bf, const void* Winv, int Ls, const void* r16, float2* x, void* x16,
                     int color, int nrhs, const int* active, int* err, double bytes, double flops) {
  MG_CHECK_ARG(bf == 1 || bf == 2, "the block update kernel takes 16-bit operands");
  MG_CHECK_ARG(Ls >= 4 && Ls % 4 == 0, "the block update kernel needs a lattice side that is a multiple of 4");
  MG_CHECK_ARG(x && x16, "block update: x and its 16-bit copy");
  const CUtensorMap rmap = map16(r16, Ls * Ls, nrhs, TB_MM);
  MG_CHECK_ARG(((uintptr_t)x & 15) == 0, "x: 16-byte aligned device pointer");
  // 2D view [nrhs rows][Ls^2 x 32 floats] of x; box 32 floats (one site) x xrows rows, 128-byte swizzle
  const int xrows = nrhs <= 32 ? 32 : TB_MM;
  CUtensorMap xmap;
  {
    const int ns = Ls * Ls;
    cuuint64_t dims[2] = {(cuuint64_t)ns * 32, (cuuint64_t)nrhs};
    cuuint64_t strides[1] = {(cuuint64_t)ns * 128};
    cuuint32_t box[2] = {32, (cuuint32_t)xrows};
    cuuint32_t es[2] = {1, 1};
    const CUresult r = encode_fn()(&xmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)x, dims, strides, box, es,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(MGMLMC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  }
  const int nitems = Ls * Ls / 8;
  const dim3 grid = grid_of(nitems, nrhs);
  auto go = [&](auto* k_tcs_kernel) {
    ensure_max_smem((const void*)k_tcs_kernel, TS_SMEM);
    MG_LAUNCH_W(bytes, flops, k_tcs_kernel, grid, TS_THREADS, TS_SMEM, st, rmap, xmap, (const unsigned char*)Winv,
                (float*)x, (uint16_t*)x16, Ls, nitems, color, nrhs, xrows, active, err);
  };
  if (bf == 2)
    go(&k_tcs<2>);
  else
    go(&k_tcs<1>);
}

}  // namespace mg
