// svdup_mixed.cu -- the product X * Ctilde (RankOneUpdate STEPs 3-7, Sec. 6.2; Eq.
// UCTildeProduct) in split BF16 on the fifth-generation tensor cores (tcgen05).
//
// The contractions are those of the FP64 path (svdup_product.cu): the Chebyshev far
// field of App. D read with a flat partition into leaves,
//     Phi = X_leaf S_leaf    (P2M),   Psi = Phi T    (M2L),
//     Y_b = Psi_b L_b + X_near(b) C_near(b)    (L2P + near field),
// with P = 16 Chebyshev nodes.  Every operand value x is split as x = hi + mid + lo
// (three BF16 numbers, 24 significant bits together) and each product A B is formed
// from the six partial products hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid with FP32
// accumulation in tensor memory: FP32-level accuracy from BF16 multiplies.
//
// The FP64 operator values (S, T, L from the FP64 set-up kernels, the near-field Cauchy
// entries zhat_t inv_j / delta_tj from the root offsets delta_tj = (d_t - d_org(j)) -
// tau_j) are computed once per product and stored as split tiles; only the split, not
// the arithmetic, is in BF16.  The near-field entries are generated once per product
// rather than once per row tile: on this part an FP64 operation costs as much as ~64
// FP32 ones, and every row tile shares the same entries.
//
// Tiles: every operand is stored in HBM pre-tiled, each tile's three planes back to
// back, each plane in the canonical K-major no-swizzle layout of the tcgen05 shared
// memory descriptor: element (r, k) of an R x KB plane is at byte
//     (r / 8) * (KB * 16) + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// i.e. 8 x 8 core matrices of 128 contiguous bytes, K-adjacent core matrices 128 B
// apart (leading byte offset) and 8-row groups KB * 16 B apart (stride byte offset).
// A tile is therefore one contiguous bulk copy (cp.async.bulk) into shared memory.
//
// GEMM kernel: one CTA per 128-row output tile; 6 warps.  Warp 4 issues the bulk
// copies into a two-stage shared-memory ring, warp 5 allocates tensor memory and one of
// its threads issues the MMAs (M = 128, N = 16..128, K = 16 per instruction), warps 0-3
// read the FP32 accumulator back (tcgen05.ld) and write the stage's output.  Every wait
// on an mbarrier gives up after about one second of global time, latches
// SVDUP_ETIMEOUT and lets the CTA finish.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>
#include <string.h>

#include "svdup_df.cuh"
#include "svdup_internal.cuh"

namespace svdup {

namespace {

// ---------------------------------------------------------------------------
// Tile geometry
// ---------------------------------------------------------------------------
constexpr int kTM = 128;                      // rows per A tile / MMA M
constexpr int kKB = 64;                       // K per tile (X, Phi, T, C)
constexpr uint32_t kTileA = 3 * kTM * kKB * 2;       // 49152
constexpr uint32_t kTilePsi = 3 * kTM * kMixP * 2;   // 12288 (128 x 16)
constexpr uint32_t kPlanePsi = kTM * kMixP * 2;      // 4096
constexpr uint32_t kTileS = 3 * kMixP * kKB * 2;     // 6144 (16 x 64)
constexpr int kStages = 2;                           // ring stages
constexpr int kHalvesPerStep = 4 / kStages;          // K halves of a 64-K tile per stage
constexpr uint32_t kStepMax = kTileA / 2 * kHalvesPerStep;  // A (or B) bytes of one step
constexpr uint32_t kStageBytes = 2 * kStepMax;       // A + B region per ring stage
constexpr uint32_t kRingBytes = kStages * kStageBytes;
constexpr uint32_t kSmemBytes = kRingBytes + 256 + 1024;  // + barriers, + alignment slack

__host__ __device__ constexpr uint32_t tile_L_bytes(int s) { return 3u * s * kMixP * 2; }
__host__ __device__ constexpr uint32_t tile_C_bytes(int s) { return 3u * s * kKB * 2; }

// byte offset of element (r, k) in a canonical K-major plane with K extent KB
__device__ __forceinline__ uint32_t cl_off(int r, int k, int KB) {
  return (uint32_t)((r >> 3) * (KB * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// A 64-K tile of R rows is stored as its two K halves one after the other, each half
// three planes (hi, mid, lo) of R x 32 in the canonical layout, half_plane(R) bytes
// apart, so that one ring stage takes one contiguous half.
__host__ __device__ constexpr uint32_t half_plane(int R) { return (uint32_t)R * 64u; }
__device__ __forceinline__ uint32_t t64_off(int r, int k, int R) {
  return (uint32_t)(k >> 5) * 3u * half_plane(R) + cl_off(r, k & 31, 32);
}

// ---------------------------------------------------------------------------
// Splits: x = hi + mid + lo in BF16 (round to nearest at each step; each remainder is
// exact in the wider type).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split3f(float x, uint16_t& h, uint16_t& m, uint16_t& l) {
  __nv_bfloat16 bh = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(bh);
  __nv_bfloat16 bm = __float2bfloat16_rn(r);
  r = r - __bfloat162float(bm);
  __nv_bfloat16 bl = __float2bfloat16_rn(r);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}



__device__ __forceinline__ uint4 pack8(const uint16_t* v) {
  uint4 o;
  o.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
  o.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
  o.z = (uint32_t)v[4] | ((uint32_t)v[5] << 16);
  o.w = (uint32_t)v[6] | ((uint32_t)v[7] << 16);
  return o;
}

// Writes 8 consecutive K values of one row into the three planes of a tile.
__device__ __forceinline__ void store_split8(unsigned char* tile, uint32_t plane, uint32_t off,
                                             const uint16_t* h, const uint16_t* m,
                                             const uint16_t* l) {
  *(uint4*)(tile + off) = pack8(h);
  *(uint4*)(tile + plane + off) = pack8(m);
  *(uint4*)(tile + 2 * plane + off) = pack8(l);
}

// Three BF16 terms of the double-float value hi + lo (24 significant bits).
__device__ __forceinline__ void split3ff(float hi, float lo, uint16_t& h, uint16_t& m,
                                         uint16_t& l) {
  __nv_bfloat16 bh = __float2bfloat16_rn(hi);
  float r = (hi - __bfloat162float(bh)) + lo;
  __nv_bfloat16 bm = __float2bfloat16_rn(r);
  r = r - __bfloat162float(bm);
  __nv_bfloat16 bl = __float2bfloat16_rn(r);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}

__device__ __forceinline__ void store_split8_ff(unsigned char* tile, uint32_t plane, uint32_t off,
                                                const float* hi, const float* lo) {
  uint16_t h[8], m[8], l[8];
#pragma unroll
  for (int c = 0; c < 8; c++) split3ff(hi[c], lo[c], h[c], m[c], l[c]);
  store_split8(tile, plane, off, h, m, l);
}

// An FP64 value reaches its three BF16 terms through an FP32 pair (bit fields, no FP64
// operation): the pair carries 47 bits, the split keeps the top 24.
__device__ __forceinline__ void store_split8_d(unsigned char* tile, uint32_t plane, uint32_t off,
                                               const double* v) {
  float hi[8], lo[8];
#pragma unroll
  for (int c = 0; c < 8; c++) {
    const Df p = df_from_f64(v[c], 0);
    hi[c] = p.hi;
    lo[c] = p.lo;
  }
  store_split8_ff(tile, plane, off, hi, lo);
}

__device__ __forceinline__ void store_split8_f(unsigned char* tile, uint32_t plane, uint32_t off,
                                               const float* v) {
  uint16_t h[8], m[8], l[8];
#pragma unroll
  for (int c = 0; c < 8; c++) split3f(v[c], h[c], m[c], l[c]);
  store_split8(tile, plane, off, h, m, l);
}


// ---------------------------------------------------------------------------
// FP16 2-term split (SVDUP_MIXED_FP16X2): a tile's values v are stored as
// v 2^sc = hi + lo, two FP16 numbers (round to nearest; the first remainder is exact in
// FP32), with one power of two 2^sc per tile that puts the tile's largest magnitude in
// [2^14, 2^15).  hi + lo carries 22 significant bits down to 2^-3 of that magnitude and
// an absolute error below 2^-39 of it beyond.  Values are collected as FP32 in shared
// memory (row r, K position k at r * KB + k), then the block finds the scale and writes
// the two planes.
// ---------------------------------------------------------------------------
constexpr int kScMax = 100;  // scales are clamped to [-100, 100] (one signed byte)

__device__ __forceinline__ void split2h(float x, uint16_t& h, uint16_t& l) {
  const __half bh = __float2half_rn(x);
  const float r = x - __half2float(bh);
  h = __half_as_ushort(bh);
  l = __half_as_ushort(__float2half_rn(r));
}

// Largest |v| over the block (every thread passes its partial maximum).
__device__ float block_max(float v) {
  __shared__ float wmax[32];
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) wmax[w] = v;
  __syncthreads();
  float m = 0.0f;
  for (int i = 0; i < nw; i++) m = fmaxf(m, wmax[i]);
  return m;
}

// The scale of a tile whose largest magnitude is m (0 for an empty or non-finite tile).
__device__ __forceinline__ int fp16_scale(float m) {
  if (!(m > 0.0f) || !isfinite(m)) return 0;
  const int e = ((__float_as_int(m) >> 23) & 0xff) - 127;  // m in [2^e, 2^(e+1))
  return max(-kScMax, min(kScMax, 14 - e));
}

// Tile layouts: a 64-K tile (two K halves of three planes each, t64_off) or a 16-K tile
// (three planes of R x 16, cl_off).
enum { TL_K64 = 0, TL_K16 = 1 };

// Splits the R x KB FP32 values in shared memory `v` into the FP16 planes of `tile` and
// stores the tile's scale; every thread of the block calls it.
__device__ void finish_tile16(unsigned char* tile, const float* v, int R, int KB, int layout,
                              signed char* sc_out) {
  float m = 0.0f;
  for (int i = threadIdx.x; i < R * KB; i += blockDim.x) m = fmaxf(m, fabsf(v[i]));
  const int sc = fp16_scale(block_max(m));
  const float f = pow2f(sc);
  if (threadIdx.x == 0) *sc_out = (signed char)sc;
  const uint32_t plane = layout == TL_K64 ? half_plane(R) : (uint32_t)R * KB * 2;
  for (int it = threadIdx.x; it < R * (KB / 8); it += blockDim.x) {
    const int r = it % R, k8 = (it / R) * 8;
    uint16_t h[8], l[8];
#pragma unroll
    for (int c = 0; c < 8; c++) split2h(v[r * KB + k8 + c] * f, h[c], l[c]);
    const uint32_t off = layout == TL_K64 ? t64_off(r, k8, R) : cl_off(r, k8, KB);
    *(uint4*)(tile + off) = pack8(h);
    *(uint4*)(tile + plane + off) = pack8(l);
  }
}

// The same for a tile whose FP32 values the tensor-core epilogue left in the tile's own
// memory, row-major (P2M's Phi, M2L's Psi): read into shared memory first.
__global__ void __launch_bounds__(256) k_split16_inplace(unsigned char* base, size_t tile_bytes,
                                                        int R, int KB, int layout,
                                                        signed char* scales, int tiles_per_row,
                                                        const int* fL, int which) {
  extern __shared__ float sv16[];
  // only the tiles the stage wrote: P2M, K tiles below ceil(Ls / 4); M2L, leaves below Lt
  const int row_tile_pos = blockIdx.x % tiles_per_row;
  const int lim = which == 0 ? (fL[0] + 3) / 4 : fL[1];
  if (row_tile_pos >= lim) return;
  unsigned char* tile = base + (size_t)blockIdx.x * tile_bytes;
  const float* src = (const float*)tile;
  for (int i = threadIdx.x; i < R * KB; i += blockDim.x) sv16[i] = src[i];
  __syncthreads();
  finish_tile16(tile, sv16, R, KB, layout, scales + blockIdx.x);
}

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier, bulk copy, tcgen05
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // one second

// Waits for the phase of `bar` with the given parity to complete.  Gives up (returns
// false) after `limit` ns of global time or once another role of the CTA has raised
// *abort.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, uint64_t limit) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*abort) return false;
      uint64_t t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > limit) return false;
    }
  }
}

// The same wait bounded by time only (used for the final drains of issued MMAs and
// bulk copies, which must complete even after another role gave up).
__device__ bool mbar_wait_timed(uint32_t bar, uint32_t parity, uint64_t limit) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      uint64_t t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > limit) return false;
    }
  }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared memory matrix descriptor (tcgen05): start address, leading and stride byte
// offsets (all >> 4), descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// X -> split A tiles.  Tile (rt, kt): rows rt*128.., sorted columns t = kt*64 + c
// (column perm[idx[t]] of X for t < k, zero beyond; zero rows beyond `rows`).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float as_f32(double x) { return narrow_rn(x); }
__device__ __forceinline__ float as_f32(float x) { return x; }

template <typename T>
__global__ void __launch_bounds__(256) k_mix_gather(Eig e, const T* __restrict__ X,
                                                    long long ldx, int rows, MixPlan mp) {
  extern __shared__ float stage16[];  // FP16 mode: the tile's values (kTM x kKB)
  __shared__ long long scol[kKB];
  const int rt = blockIdx.x, kt = blockIdx.y;
  const int k = e.kp[0];
  if (threadIdx.x < kKB) {  // K position kt 64 + c holds sorted pole kt 64 + c - P
    const int t = kt * kKB + threadIdx.x - mp.fL[2];
    scol[threadIdx.x] = (t >= 0 && t < k) ? (long long)e.perm[e.idx[t]] * ldx : -1;
  }
  __syncthreads();
  unsigned char* tile = mp.Xp + ((size_t)rt * mp.kx + kt) * kTileA;
  for (int it = threadIdx.x; it < kTM * (kKB / 8); it += blockDim.x) {
    const int r = it & (kTM - 1), ch = it >> 7;
    const long long row = (long long)rt * kTM + r;
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
      long long col = scol[ch * 8 + c];
      v[c] = (col >= 0 && row < rows) ? as_f32(X[row + col]) : 0.0f;
    }
    if (mp.fp16) {
#pragma unroll
      for (int c = 0; c < 8; c++) stage16[r * kKB + ch * 8 + c] = v[c];
    } else {
      store_split8_f(tile, half_plane(kTM), t64_off(r, ch * 8, kTM), v);
    }
  }
  if (mp.fp16) {
    __syncthreads();
    finish_tile16(tile, stage16, kTM, kKB, TL_K64, mp.scX + (size_t)rt * mp.kx + kt);
  }
}

__device__ __forceinline__ long long out_col_m(const OutMap& om, int q) {
  return om.out_rev ? (long long)(om.out_n - 1 - q) : (long long)q;
}

// Deflated columns are eigenvectors already: straight to their output column.
template <typename T>
__global__ void k_mix_defl(Eig e, const T* __restrict__ X, long long ldx, int rows,
                           OutMap om) {
  const int k = e.kp[0];
  const int c = k + blockIdx.x;
  if (c >= e.N) return;
  int s = e.didx[c - k];
  if (e.defl[s] == 2) return;  // deflated by a rotation: the rotation kernel wrote it
  int q = e.rank_defl[s];
  const T* src = X + (long long)e.perm[s] * ldx;
  const long long o = out_col_m(om, q) * om.ldy;
  if (om.Yf) {
    for (int r = threadIdx.x; r < rows; r += blockDim.x) om.Yf[o + r] = as_f32(src[r]);
  } else {
    for (int r = threadIdx.x; r < rows; r += blockDim.x) om.Y[o + r] = (double)src[r];
  }
}

// ---------------------------------------------------------------------------
// Set-up: near lists (dense: every source leaf), their offsets into the pool, and the
// split operator tiles.
// ---------------------------------------------------------------------------
__global__ void k_mix_near(FmmPlan f, MixPlan mp, int dense) {
  const int Ls = f.L[0], Lt = f.L[1];
  for (int b = threadIdx.x; b < Lt; b += blockDim.x) {
    int n = dense ? Ls : f.nnear[b];
    mp.nnear[b] = n;
    for (int i = 0; i < n; i++)
      mp.near[(long long)b * mp.Lmax + i] = dense ? i : f.near[(long long)b * f.Lmax + i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = 0; b < Lt; b++) {
      mp.noff[b] = acc;
      acc += mp.nnear[b];
    }
    mp.noff[Lt] = acc;
  }
  // Output jobs by descending near count (ties by leaf): the longest CTAs start first
  // instead of trailing the grid.
  for (int b = threadIdx.x; b < Lt; b += blockDim.x) {
    const int nb = mp.nnear[b];
    int rank = 0;
    for (int c = 0; c < Lt; c++) {
      const int nc = mp.nnear[c];
      rank += (nc > nb || (nc == nb && c < b)) ? 1 : 0;
    }
    mp.order[rank] = b;
  }
}

// S tile (a, h): B[alpha][kk] = S_a(tl = 64 h + kk, alpha) (16 x 64).
__global__ void k_mix_pack_S(Eig e, FmmPlan f, MixPlan mp) {
  extern __shared__ float stage16[];
  const int hs = mp.s / kKB;
  const int a = blockIdx.x / hs, h = blockIdx.x % hs;
  if (a >= f.L[0]) return;
  unsigned char* tile = mp.Sp + (size_t)blockIdx.x * kTileS;
  for (int it = threadIdx.x; it < kMixP * (kKB / 8); it += blockDim.x) {
    const int al = it % kMixP, ch = it / kMixP;
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
      int tl = h * kKB + ch * 8 + c;
      v[c] = f.S[(size_t)a * f.s * f.p + (size_t)al * f.s + tl];
    }
    if (mp.fp16) {
#pragma unroll
      for (int c = 0; c < 8; c++) stage16[al * kKB + ch * 8 + c] = narrow_rn(v[c]);
    } else {
      store_split8_d(tile, half_plane(kMixP), t64_off(al, ch * 8, kMixP), v);
    }
  }
  if (mp.fp16) {
    __syncthreads();
    finish_tile16(tile, stage16, kMixP, kKB, TL_K64, mp.scS + blockIdx.x);
  }
}

// T tile (nt, kt): B[n][kk] = T(row = 64 kt + kk, col = 128 nt + n), zero outside
// (Ls P) x (Lt P).
__global__ void k_mix_pack_T(FmmPlan f, MixPlan mp) {
  extern __shared__ float stage16[];
  const int nt = blockIdx.x, kt = blockIdx.y;
  const int Ls = f.L[0], Lt = f.L[1];
  const long long ldT = (long long)f.Lmax * f.p;
  unsigned char* tile = mp.Tp + ((size_t)nt * mp.kphi + kt) * kTileA;
  for (int it = threadIdx.x; it < kTM * (kKB / 8); it += blockDim.x) {
    const int n = it & (kTM - 1), ch = it >> 7;
    const int col = nt * kTM + n;
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
      int row = kt * kKB + ch * 8 + c;
      v[c] = (col < Lt * kMixP && row < Ls * kMixP) ? f.T[row + col * ldT] : 0.0;
    }
    if (mp.fp16) {
#pragma unroll
      for (int c = 0; c < 8; c++) stage16[n * kKB + ch * 8 + c] = narrow_rn(v[c]);
    } else {
      store_split8_d(tile, half_plane(kTM), t64_off(n, ch * 8, kTM), v);
    }
  }
  if (mp.fp16) {
    __syncthreads();
    finish_tile16(tile, stage16, kTM, kKB, TL_K64, mp.scT + (size_t)nt * mp.kphi + kt);
  }
}

// L tile b: B[jl][beta] = L_b(beta, jl) (s x 16).
__global__ void k_mix_pack_L(FmmPlan f, MixPlan mp) {
  extern __shared__ float stage16[];
  const int b = blockIdx.x;
  if (b >= f.L[1]) return;
  const int s = mp.s;
  unsigned char* tile = mp.Lp + (size_t)b * tile_L_bytes(s);
  const uint32_t plane = (uint32_t)s * kMixP * 2;
  for (int it = threadIdx.x; it < s * (kMixP / 8); it += blockDim.x) {
    const int jl = it % s, ch = it / s;
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; c++)
      v[c] = f.Lop[(size_t)b * f.s * f.p + (size_t)jl * f.p + ch * 8 + c];
    if (mp.fp16) {
#pragma unroll
      for (int c = 0; c < 8; c++) stage16[jl * kMixP + ch * 8 + c] = narrow_rn(v[c]);
    } else {
      store_split8_d(tile, plane, cl_off(jl, ch * 8, kMixP), v);
    }
  }
  if (mp.fp16) {
    __syncthreads();
    finish_tile16(tile, stage16, s, kMixP, TL_K16, mp.scL + b);
  }
}

// Near-field tile (b, i, h): source leaf a = near[b][i], K half h:
//   B[jl][kk] = zhat_t inv_j / delta_tj,  t = a s + 64 h + kk,  j = tj0[b] + jl,
//   delta_tj = (dk_t - d_org(j)) - tau_j   (the offsets of the FP64 root solve),
// zero for t >= k or j >= tj1[b].  One FP64 operation per entry, the pole difference
// (exact when the poles are close, by Sterbenz's lemma); tau_j is subtracted, and the
// reciprocal and products formed, on FP32 pairs at a common power-of-two scale (a
// pair carries about 46 bits, the split keeps 24).  For a pole t outside root j's
// bracket the subtraction cancels at most a factor 3 (|tau_j| is at most half the
// bracket); at the bracketing poles it is exact or cancels at most a factor 2.
__device__ __forceinline__ Df df_scaled_pow2(Df v, int sh) {  // v 2^sh, in two exact steps
  const float a = pow2f(max(sh, -126)), b = pow2f(min(0, sh + 126));
  return Df{(v.hi * a) * b, (v.lo * a) * b};
}

__global__ void k_mix_pack_C(Eig e, FmmPlan f, MixPlan mp) {
  extern __shared__ float stage16[];
  const int b = blockIdx.x, i = blockIdx.y, h = blockIdx.z;
  if (b >= f.L[1] || i >= mp.nnear[b]) return;
  const int k = e.kp[0];
  const int s = mp.s, hs = s / kKB;
  const int a = mp.near[(long long)b * mp.Lmax + i];
  const int j0 = f.tj0[b], j1 = f.tj1[b];
  const int P = f.L[2];  // source leaf a holds poles [a s - P, a s + s - P)
  unsigned char* tile = mp.Cp + ((size_t)(mp.noff[b] + i) * hs + h) * tile_C_bytes(s);
  for (int it = threadIdx.x; it < s * (kKB / 8); it += blockDim.x) {
    const int jl = it % s, ch = it / s;
    const int j = j0 + jl;
    float hi[8], lo[8];
#pragma unroll
    for (int c = 0; c < 8; c++) { hi[c] = 0.f; lo[c] = 0.f; }
    if (j < j1) {
      const double dO = e.dorg[j], tj = e.tau[j], inv = e.inv[j];
      const int eT = exp2_of(tj), eI = exp2_of(inv);
      const Df ij = df_from_f64(inv, eI);
#pragma unroll
      for (int c = 0; c < 8; c++) {
        const int t = a * s + h * kKB + ch * 8 + c - P;
        if (t < 0 || t >= k) continue;
        const double zt = e.zhat[t];
        const double d1 = e.dk[t] - dO;
        const int eD = max(exp2_of(d1), eT), eZ = exp2_of(zt);
        if (zt == 0.0 || eZ < -1000 || eI < -1000 || eD < -1000) {  // zero or subnormal
          const double v = zt * inv * rcp64(d1 - tj);
          const Df p = df_from_f64(v, 0);
          hi[c] = p.hi;
          lo[c] = p.lo;
          continue;
        }
        const Df del = df_add(df_from_f64(d1, eD), df_neg(df_from_f64(tj, eD)));
        const Df v = df_mul(df_mul(df_from_f64(zt, eZ), ij), df_rcp(del));
        const Df w = df_scaled_pow2(v, eZ + eI - eD);
        hi[c] = w.hi;
        lo[c] = w.lo;
      }
    }
    if (mp.fp16) {
#pragma unroll
      for (int c = 0; c < 8; c++) stage16[jl * kKB + ch * 8 + c] = hi[c] + lo[c];
    } else {
      store_split8_ff(tile, half_plane(s), t64_off(jl, ch * 8, s), hi, lo);
    }
  }
  if (mp.fp16) {
    __syncthreads();
    finish_tile16(tile, stage16, s, kKB, TL_K64, mp.scC + ((size_t)(mp.noff[b] + i) * hs + h));
  }
}

// ---------------------------------------------------------------------------
// The tcgen05 GEMM.  A K tile is a pair (A tile, B tile) of split operands; the CTA
// accumulates sum over its K tiles of A B^T (B stored N x K) into tensor memory.
// ---------------------------------------------------------------------------
enum { MS_P2M = 0, MS_M2L = 1, MS_OUT = 2, MS_GRAM = 3, MS_CORR = 4 };

struct KTile {
  const unsigned char* a;
  const unsigned char* b;
  uint32_t astep, bstep;    // bytes per step: a K half of a 64-K tile, or a 16-K tile whole
  uint32_t aplane, bplane;  // plane strides within a step
  int kstep;                // K per step (32 or 16)
  int nsteps;               // steps (ring stages) of the tile: 2 or 1
  int n;                    // MMA N
  int col;                  // accumulator column offset
  int first;                // first K tile of its accumulator
};

struct Job {
  int rt, job;
  int k, Ls, Lt;
  int ntiles;
};

template <int STAGE>
__device__ __forceinline__ int job_tiles(const Job& J, const FmmPlan& f, const MixPlan& mp,
                                         int dense) {
  if (STAGE == MS_GRAM) return mp.kr;  // K: the rows of X
  if (STAGE == MS_CORR) return mp.kx;  // K: the columns of X
  const int hs = mp.s / kKB;
  if (STAGE == MS_P2M) return (min(4 * J.job + 4, J.Ls) - 4 * J.job) * hs;
  if (STAGE == MS_M2L) return (J.Ls + 3) / 4;
  return (dense ? 0 : 1) + mp.nnear[J.job] * hs;
}

// a 64-K tile of rows R at p, in steps of kHalvesPerStep K halves
__device__ __forceinline__ void half_steps_a(KTile& t, const unsigned char* p, int R) {
  t.a = p; t.astep = 3u * half_plane(R) * kHalvesPerStep; t.aplane = half_plane(R);
}
__device__ __forceinline__ void half_steps_b(KTile& t, const unsigned char* p, int R) {
  t.b = p; t.bstep = 3u * half_plane(R) * kHalvesPerStep; t.bplane = half_plane(R);
}

template <int STAGE>
__device__ __forceinline__ KTile ktile(int i, const Job& J, const FmmPlan& f, const MixPlan& mp,
                                       int dense) {
  KTile t;
  const int hs = mp.s / kKB;
  t.kstep = kKB / 2 * kHalvesPerStep;
  t.nsteps = 2 / kHalvesPerStep;
  if (STAGE == MS_GRAM) {  // (X^T X) tile (J.rt, J.job): both operands are X^T tiles
    half_steps_a(t, mp.Xt + ((size_t)J.rt * mp.kr + i) * kTileA, kTM);
    half_steps_b(t, mp.Xt + ((size_t)J.job * mp.kr + i) * kTileA, kTM);
    t.n = kTM; t.col = 0; t.first = (i == 0);
  } else if (STAGE == MS_CORR) {  // (X E) tile (J.rt, J.job)
    half_steps_a(t, mp.Xp + ((size_t)J.rt * mp.kx + i) * kTileA, kTM);
    half_steps_b(t, mp.Et + ((size_t)J.job * mp.kx + i) * kTileA, kTM);
    t.n = kTM; t.col = 0; t.first = (i == 0);
  } else if (STAGE == MS_P2M) {
    const int a = 4 * J.job + i / hs, h = i % hs;
    half_steps_a(t, mp.Xp + ((size_t)J.rt * mp.kx + (size_t)a * hs + h) * kTileA, kTM);
    half_steps_b(t, mp.Sp + ((size_t)a * hs + h) * kTileS, kMixP);
    t.n = kMixP; t.col = (a - 4 * J.job) * kMixP; t.first = (h == 0);
  } else if (STAGE == MS_M2L) {
    half_steps_a(t, mp.Phip + ((size_t)J.rt * mp.kphi + i) * kTileA, kTM);
    half_steps_b(t, mp.Tp + ((size_t)J.job * mp.kphi + i) * kTileA, kTM);
    t.n = kTM; t.col = 0; t.first = (i == 0);
  } else {
    const int s = mp.s;
    const int b = J.job;
    if (!dense && i == 0) {
      t.a = mp.Psip + ((size_t)J.rt * (mp.Lmax + 1) + b) * kTilePsi;
      t.b = mp.Lp + (size_t)b * tile_L_bytes(s);
      t.astep = kTilePsi; t.aplane = kPlanePsi;
      t.bstep = tile_L_bytes(s); t.bplane = (uint32_t)s * kMixP * 2;
      t.kstep = kMixP; t.nsteps = 1; t.n = s; t.col = 0; t.first = 1;
    } else {
      const int q = i - (dense ? 0 : 1);
      const int ni = q / hs, h = q % hs;
      const int a = mp.near[(long long)b * mp.Lmax + ni];
      half_steps_a(t, mp.Xp + ((size_t)J.rt * mp.kx + (size_t)a * hs + h) * kTileA, kTM);
      half_steps_b(t, mp.Cp + ((size_t)(mp.noff[b] + ni) * hs + h) * tile_C_bytes(s), s);
      t.n = s; t.col = 0;
      t.first = dense && q == 0;  // with the far field, tile 0 (Psi L) opened the sum
    }
  }
  return t;
}

// FP16 mode: the sum of the two operand tiles' scales of K tile i (the drain multiplies
// the tile's accumulator by 2^-scale).
template <int STAGE>
__device__ __forceinline__ int tile_scale(int i, const Job& J, const FmmPlan& f, const MixPlan& mp,
                                          int dense) {
  const int hs = mp.s / kKB;
  if (STAGE == MS_P2M) {
    const int a = 4 * J.job + i / hs, h = i % hs;
    return mp.scX[(size_t)J.rt * mp.kx + (size_t)a * hs + h] + mp.scS[(size_t)a * hs + h];
  }
  if (STAGE == MS_M2L)
    return mp.scPhi[(size_t)J.rt * mp.kphi + i] + mp.scT[(size_t)J.job * mp.kphi + i];
  const int b = J.job;
  if (!dense && i == 0) return mp.scPsi[(size_t)J.rt * (mp.Lmax + 1) + b] + mp.scL[b];
  const int q = i - (dense ? 0 : 1);
  const int ni = q / hs, h = q % hs;
  const int a = mp.near[(long long)b * mp.Lmax + ni];
  return mp.scX[(size_t)J.rt * mp.kx + (size_t)a * hs + h] + mp.scC[(size_t)(mp.noff[b] + ni) * hs + h];
}

// 2^-sc in two steps (sc up to 2 kScMax in magnitude), exact unless the result is
// subnormal.
__device__ __forceinline__ float unscale(float v, int sc) {
  const int s1 = sc / 2;
  return (v * pow2f(-s1)) * pow2f(s1 - sc);
}

// Instruction descriptor, kind::f16 with FP16 operands (A and B type fields 0).
__device__ __forceinline__ uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The six partial products of the 3-term split, (A plane, B plane): (hi, hi) accumulates
// in its own tensor-memory region; (hi, mid) (mid, hi) (hi, lo) (lo, hi) (mid, mid),
// smaller by 2^-8 or more, share a second region.

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// (hi, lo) += x with Knuth's TwoSum in FP32: hi + lo carries about 48 significant bits.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += err;
}



// Roles: warps 0-7 drain the accumulators (warp w reads TMEM lanes 32 (w % 4) .., i.e.
// output rows, and the column half w / 4 of the W accumulator columns), warp 8 issues
// the bulk copies, warp 9 owns tensor memory and issues the MMAs.
// Tensor memory (512 columns): three hi.hi accumulators that K tiles take in turn, and
// one accumulator for the five cross products of the whole item.  Every K tile's hi.hi
// sum is drained into double-float registers while the next ones are multiplied, so FP32
// rounding of the leading products covers at most one K tile (64 or 16 products); the
// cross products, 2^-8 of them and below, accumulate in FP32 over the item and are
// drained once.  With three hi.hi regions the MMAs run up to three K tiles ahead of the
// drains, which covers the epilogue's output stores at the end of an item.
constexpr int kEpiWarps = 16;  // four per quarter of the TMEM lanes (rows), each a quarter of the columns
constexpr int kUmmaThreads = (kEpiWarps + 2) * 32;
constexpr uint32_t kTmemCols = 512;
constexpr int kHiRegions = 3;          // hi.hi accumulators, columns [128 r, 128 r + 128)
constexpr uint32_t kCrossCol = 384;    // the cross-product accumulator, columns [384, 512)

// Work items: (row tile rt, job).  Jobs per row tile: P2M one per 4 source leaves, M2L
// one per 128 local-expansion columns (8 target leaves), OUT one per target leaf (in
// descending near count).  Items run row-tile major, so the CTAs running at one time
// share a few row tiles of X: the X tiles that neighbouring target leaves both read
// stay in L2 between their uses.
template <int STAGE>
__device__ __forceinline__ int stage_jobs(const Job& J, const MixPlan& mp) {
  if (STAGE == MS_GRAM || STAGE == MS_CORR) return mp.ct;  // 128-column tiles of the output
  if (STAGE == MS_P2M) return (J.Ls + 3) / 4;
  if (STAGE == MS_M2L) return (J.Lt + kTM / kMixP - 1) / (kTM / kMixP);
  return J.Lt;
}

template <int STAGE>
__device__ __forceinline__ void set_item(Job& J, int x, int njobs, const FmmPlan& f,
                                         const MixPlan& mp, int dense) {
  J.rt = x / njobs;
  const int jo = x - J.rt * njobs;
  J.job = (STAGE == MS_OUT) ? mp.order[jo] : jo;
  J.ntiles = job_tiles<STAGE>(J, f, mp, dense);
}

// Persistent: one CTA per SM loops over the work items (x = blockIdx.x, += gridDim.x).
// The producer and MMA warps run ahead into the next item while the epilogue warps
// finish the previous one; every role counts what it has handled across items (ring
// steps, K tiles, items), which fixes the slot or region (count mod their number) and
// the barrier phase (count / their number, mod 2).
template <int STAGE, int W>
__global__ void __launch_bounds__(kUmmaThreads, 1) k_umma(Eig e, FmmPlan f, MixPlan mp, OutMap om,
                                                          int dense, int* status) {
  constexpr int QW = W / (kEpiWarps / 4);  // columns per epilogue warp
  constexpr int NCH = QW / 16;     // 16-column chunks per epilogue warp
  extern __shared__ unsigned char smem_raw[];
  constexpr bool kRef = (STAGE == MS_GRAM || STAGE == MS_CORR);  // no eigen-system, no plan
  Job J;
  J.k = kRef ? 0 : e.kp[0];
  J.Ls = kRef ? 0 : f.L[0];
  J.Lt = kRef ? 0 : f.L[1];
  const int njobs = stage_jobs<STAGE>(J, mp);
  const int nitems = (STAGE == MS_GRAM ? mp.ct : mp.rt) * njobs;

  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t s_base = smem_u32(sm);
  // barriers: full[S] empty[S] (ring), tfull[3] tempty[3] (hi.hi regions), xfull xempty
  // (cross region), done
  uint64_t* bars = (uint64_t*)(sm + kRingBytes);
  const uint32_t bar0 = smem_u32(bars);
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(sm + kRingBytes + 128);
  volatile int* abort_flag = (volatile int*)(sm + kRingBytes + 192);
  auto bar_full = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  auto bar_empty = [&](int i) { return bar0 + 8u * (uint32_t)(kStages + i); };
  auto bar_tfull = [&](int i) { return bar0 + 8u * (uint32_t)(2 * kStages + i); };
  auto bar_tempty = [&](int i) { return bar0 + 8u * (uint32_t)(2 * kStages + 3 + i); };
  const uint32_t bar_xfull = bar0 + 8u * (uint32_t)(2 * kStages + 6);
  const uint32_t bar_xempty = bar0 + 8u * (uint32_t)(2 * kStages + 7);
  const uint32_t bar_done = bar0 + 8u * (uint32_t)(2 * kStages + 8);
  if ((int)blockIdx.x >= nitems) return;  // uniform per CTA, before any barrier or TMEM use
  if (kRef && *mp.gate == 0) return;  // refinement not due
  const uint64_t wlim = mp.wait_ns ? (uint64_t)mp.wait_ns : kWaitLimitNs;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == kEpiWarps + 1) {
    tmem_alloc(smem_u32((const void*)tmem_slot), kTmemCols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; i++) {
      mbar_init(bar_full(i), 1);
      mbar_init(bar_empty(i), 1);
    }
    for (int i = 0; i < kHiRegions; i++) {
      mbar_init(bar_tfull(i), 1);
      mbar_init(bar_tempty(i), kEpiWarps * 32);
    }
    mbar_init(bar_xfull, 1);
    mbar_init(bar_xempty, kEpiWarps * 32);
    mbar_init(bar_done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kEpiWarps) {
    if (lane == 0) {  // producer: bulk copies into the shared-memory ring, a step per stage
      uint32_t g = 0;  // steps issued
      bool alive = true;
      for (int x = blockIdx.x; x < nitems && alive; x += gridDim.x) {
        set_item<STAGE>(J, x, njobs, f, mp, dense);
        for (int i = 0; i < J.ntiles && alive; i++) {
          KTile t = ktile<STAGE>(i, J, f, mp, dense);
          for (int q = 0; q < t.nsteps; q++, g++) {
            const int st = (int)(g % kStages);
            if (g >= (uint32_t)kStages &&
                !mbar_wait(bar_empty(st), ((g / kStages) & 1u) ^ 1u, abort_flag, wlim)) {
              *abort_flag = 1;
              latch(status, SVDUP_ETIMEOUT);
              alive = false;
              break;
            }
            const uint32_t sa = s_base + (uint32_t)st * kStageBytes, sb = sa + kStepMax;
            if (!mp.fp16) {
              mbar_expect_tx(bar_full(st), t.astep + t.bstep);
              bulk_g2s(sa, t.a + (size_t)q * t.astep, t.astep, bar_full(st));
              bulk_g2s(sb, t.b + (size_t)q * t.bstep, t.bstep, bar_full(st));
            } else {
              // FP16 planes (hi, lo) only: each K half's first two planes, packed
              const int nh = t.kstep / 32;  // K halves in the step (0: one 16-K tile)
              const uint32_t ab = 2u * t.aplane, bb = 2u * t.bplane;
              mbar_expect_tx(bar_full(st), (ab + bb) * (uint32_t)max(nh, 1));
              if (nh == 0) {
                bulk_g2s(sa, t.a + (size_t)q * t.astep, ab, bar_full(st));
                bulk_g2s(sb, t.b + (size_t)q * t.bstep, bb, bar_full(st));
              } else {
                for (int hh = 0; hh < nh; hh++) {
                  bulk_g2s(sa + hh * ab, t.a + (size_t)q * t.astep + (size_t)hh * 3u * t.aplane, ab,
                           bar_full(st));
                  bulk_g2s(sb + hh * bb, t.b + (size_t)q * t.bstep + (size_t)hh * 3u * t.bplane, bb,
                           bar_full(st));
                }
              }
            }
          }
        }
      }
      // Every bulk copy issued has landed before the CTA may exit: wait on the last use
      // of each ring stage (at once in a normal run, where the MMA issuer consumed them;
      // after an abort, the copies still in flight).
      const uint32_t g0 = g >= (uint32_t)kStages ? g - (uint32_t)kStages : 0u;
      for (uint32_t s2 = g0; s2 < g; s2++)
        if (!mbar_wait_timed(bar_full((int)(s2 % kStages)), (s2 / kStages) & 1u, wlim))
          latch(status, SVDUP_ETIMEOUT);
    }
  } else if (warp == kEpiWarps + 1) {
    if (lane == 0) {  // MMA issuer
      uint32_t g = 0;   // K tiles (hi.hi regions rotate per K tile)
      uint32_t gs = 0;  // ring steps
      uint32_t y = 0;   // items (the cross region is drained once per item)
      bool alive = true;
      for (int x = blockIdx.x; x < nitems && alive; x += gridDim.x, y++) {
        set_item<STAGE>(J, x, njobs, f, mp, dense);
        if (y >= 1 && !mbar_wait(bar_xempty, (y - 1) & 1u, abort_flag, wlim)) {
          *abort_flag = 1;
          latch(status, SVDUP_ETIMEOUT);
          break;
        }
        for (int i = 0; i < J.ntiles && alive; i++, g++) {
          const int rg = (int)(g % kHiRegions);
          if (g >= (uint32_t)kHiRegions &&
              !mbar_wait(bar_tempty(rg), ((g / kHiRegions) & 1u) ^ 1u, abort_flag, wlim)) {
            *abort_flag = 1;
            latch(status, SVDUP_ETIMEOUT);
            alive = false;
            break;
          }
          KTile t = ktile<STAGE>(i, J, f, mp, dense);
          const uint32_t dA = tmem + (uint32_t)rg * 128u + (uint32_t)t.col;
          const uint32_t dX = tmem + kCrossCol + (uint32_t)t.col;
          const uint32_t idesc = mp.fp16 ? idesc_f16(kTM, t.n) : idesc_bf16(kTM, t.n);
          const uint32_t sbo = (uint32_t)min(t.kstep, 32) * 16;  // a K half holds 32
          for (int q = 0; q < t.nsteps; q++, gs++) {
            const int st = (int)(gs % kStages);
            if (!mbar_wait(bar_full(st), (gs / kStages) & 1u, abort_flag, wlim)) {
              *abort_flag = 1;
              latch(status, SVDUP_ETIMEOUT);
              alive = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = s_base + (uint32_t)st * kStageBytes, sb = sa + kStepMax;
            // Descriptors differ only in their start-address field (bytes >> 4, below
            // 2^14 for any shared-memory address), so planes and K steps are additions.
            const uint64_t a0 = sdesc(sa, 128, sbo), b0 = sdesc(sb, 128, sbo);
            const uint64_t ap = t.aplane >> 4, bp = t.bplane >> 4;
            if (mp.fp16 && STAGE != MS_CORR) {
              // FP16 2-term split: (hi, lo) and (lo, hi) of every K step first, while the
              // accumulator holds only their own sums, then (hi, hi), all in the K tile's
              // accumulator (the tiles' scales differ, so every K tile is drained)
              const int nks = t.kstep / 16;
              for (int pass = 0; pass < 2; pass++)
                for (int ks = 0; ks < nks; ks++) {
                  const uint32_t acc = (q > 0 || pass > 0 || ks > 0) ? 1u : 0u;
                  const uint64_t ka = a0 + (uint64_t)((ks >> 1) * 2) * ap + (uint64_t)((ks & 1) * 16);
                  const uint64_t kb = b0 + (uint64_t)((ks >> 1) * 2) * bp + (uint64_t)((ks & 1) * 16);
                  if (pass == 0) {
                    umma_bf16(dA, ka, kb + bp, idesc, acc);
                    umma_bf16(dA, ka + ap, kb, idesc, 1u);
                  } else {
                    umma_bf16(dA, ka, kb, idesc, acc);
                  }
                }
            } else
            for (int ks = 0; ks < t.kstep / 16; ks++) {
              const uint32_t acc = (q > 0 || ks > 0) ? 1u : 0u;
              const uint32_t xacc = (t.first && q == 0 && ks == 0) ? 0u : 1u;
              // K step ks: half ks / 2 (three planes further on), core matrices 2 (ks % 2)
              // (FP16: the halves hold two planes each in shared memory)
              const int hp = mp.fp16 ? 2 : 3;
              const uint64_t ko = (uint64_t)((ks >> 1) * hp) * ap + (uint64_t)((ks & 1) * 16);
              const uint64_t kob = (uint64_t)((ks >> 1) * hp) * bp + (uint64_t)((ks & 1) * 16);
              const uint64_t ka = a0 + ko, kb = b0 + kob;
              if (STAGE == MS_CORR) {
                // the correction X E / 2 is about |E| of X: one BF16 product (hi, hi)
                // leaves an error of 2^-8 |E|
                umma_bf16(dA, ka, kb, idesc, acc);
              } else {
                // (A plane, B plane): hi.hi alone, then (hi, mid) (mid, hi) (hi, lo) (lo, hi)
                // (mid, mid)
                umma_bf16(dA, ka, kb, idesc, acc);
                umma_bf16(dX, ka, kb + bp, idesc, xacc);
                umma_bf16(dX, ka + ap, kb, idesc, 1u);
                umma_bf16(dX, ka, kb + 2 * bp, idesc, 1u);
                umma_bf16(dX, ka + 2 * ap, kb, idesc, 1u);
                umma_bf16(dX, ka + ap, kb + bp, idesc, 1u);
              }
            }
            umma_commit(bar_empty(st));  // frees the ring stage once these MMAs have read it
          }
          if (!alive) break;
          umma_commit(bar_tfull(rg));  // hands the hi.hi accumulator to the epilogue
        }
        if (!alive) break;
        umma_commit(bar_xfull);  // the item's cross products are complete
      }
      // every MMA this thread issued has completed before tensor memory is released
      umma_commit(bar_done);
      if (!mbar_wait_timed(bar_done, 0, wlim)) latch(status, SVDUP_ETIMEOUT);
    }
  } else {
    // epilogue: drain every K tile's hi.hi products into (hi, lo) pairs and the item's
    // cross products once, then write the item's output
    const int quad = warp & 3, qc = warp >> 2;
    const int r = quad * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    uint32_t g = 0, y = 0;
    bool ok = true;
    for (int x = blockIdx.x; x < nitems && ok; x += gridDim.x, y++) {
      set_item<STAGE>(J, x, njobs, f, mp, dense);
      // the output columns of this warp's 64 (or 32) accumulator columns, one or two per
      // lane, loaded now (their latency hides behind the drains), shuffled at the end
      int cm0 = -1, cm1 = -1;
      if (STAGE == MS_OUT) {
        const int j0 = f.tj0[J.job], nb = f.tj1[J.job] - j0;
        const int c0 = qc * QW + lane;
        if (c0 < nb) cm0 = (int)out_col_m(om, e.rank_root[j0 + c0]);
        if (QW > 32 && c0 + 32 < nb) cm1 = (int)out_col_m(om, e.rank_root[j0 + c0 + 32]);
      }
      float hi[QW], lo[QW];
#pragma unroll
      for (int c = 0; c < QW; c++) { hi[c] = 0.0f; lo[c] = 0.0f; }
      for (int i = 0; i < J.ntiles; i++, g++) {
        const int rg = (int)(g % kHiRegions);
        if (!mbar_wait(bar_tfull(rg), (g / kHiRegions) & 1u, abort_flag, wlim)) {
          ok = false;
          break;
        }
        tc_fence_after();
        KTile t = ktile<STAGE>(i, J, f, mp, dense);
        const int tsc = mp.fp16 ? tile_scale<STAGE>(i, J, f, mp, dense) : 0;
#pragma unroll
        for (int ch = 0; ch < NCH; ch++) {
          const int col = qc * QW + ch * 16;
          if (col >= t.col && col < t.col + t.n) {
            float v[16];
            tmem_ld16(lane_base + (uint32_t)rg * 128u + (uint32_t)col, v);
            if (mp.fp16) {
#pragma unroll
              for (int c = 0; c < 16; c++) v[c] = unscale(v[c], tsc);
            }
#pragma unroll
            for (int c = 0; c < 16; c++) two_sum_acc(hi[ch * 16 + c], lo[ch * 16 + c], v[c]);
          }
        }
        tc_fence_before();
        if (!mp.stall) mbar_arrive(bar_tempty(rg));
      }
      if (!ok || !mbar_wait(bar_xfull, y & 1u, abort_flag, wlim)) {
        ok = false;
        break;
      }
      tc_fence_after();
      if (!mp.fp16 && STAGE != MS_CORR) {
#pragma unroll
        for (int ch = 0; ch < NCH; ch++) {  // cross terms: 2^-8 of hi.hi and below
          float v[16];
          tmem_ld16(lane_base + kCrossCol + (uint32_t)(qc * QW + ch * 16), v);
#pragma unroll
          for (int c = 0; c < 16; c++) lo[ch * 16 + c] += v[c];
        }
      }
      tc_fence_before();
      mbar_arrive(bar_xempty);
      if (!ok || *abort_flag) break;
      if (STAGE == MS_GRAM) {
        // E = X^T X - I, stored as the B operand of the correction: E is symmetric, so
        // row i of this tile (the lane's row) is written as B row n = i with K = j.
        const int i = J.rt * kTM + r;
        const int kt = 2 * J.job + (qc >> 1), k0 = (qc & 1) * 32;
        unsigned char* tile = mp.Et + ((size_t)J.rt * mp.kx + kt) * kTileA;
#pragma unroll
        for (int c = 0; c < QW; c++) {
          const int j = J.job * kTM + qc * QW + c;
          if (i >= mp.cols || j >= mp.cols) {
            hi[c] = 0.0f; lo[c] = 0.0f;
            continue;
          }
          if (i == j) two_sum_acc(hi[c], lo[c], -1.0f);  // (hi + lo) - 1
          // The pair's two halves may nearly cancel (lo carries the cross products,
          // 2^-8 of hi.hi); renormalise it (TwoSum) so that hi is E rounded to FP32: the
          // correction product uses E's leading BF16 term only.
          const float sum = hi[c] + lo[c];
          const float bb = sum - hi[c];
          const float err = (hi[c] - (sum - bb)) + (lo[c] - bb);
          hi[c] = sum;
          lo[c] = err;
        }
        if (kt < mp.kx) {  // (a K tile past the last column holds nothing)
#pragma unroll
          for (int c8 = 0; c8 < QW; c8 += 8)
            store_split8_ff(tile, half_plane(kTM), t64_off(r, k0 + c8, kTM), hi + c8, lo + c8);
        }
      } else if (STAGE == MS_CORR) {
        // X <- X - (X E) / 2 in FP64 (lanes: consecutive rows of one column)
        const long long row = (long long)J.rt * kTM + r;
#pragma unroll
        for (int c = 0; c < QW; c++) {
          const int j = J.job * kTM + qc * QW + c;
          if (row < mp.rows && j < mp.cols) {
            double* x = mp.Xr + (long long)j * mp.ldxr + row;
            *x -= 0.5 * ((double)hi[c] + (double)lo[c]);
          }
        }
      } else if (STAGE == MS_P2M) {
        // column group qc = leaves 4 job + (QW / 16) qc + u: columns QW qc .. of the Phi tile
        unsigned char* tile = mp.Phip + ((size_t)J.rt * mp.kphi + J.job) * kTileA;
#pragma unroll
        for (int u = 0; u < QW / kMixP; u++) {
          if (4 * J.job + qc * (QW / kMixP) + u >= J.Ls)  // past the last leaf: zeros
#pragma unroll
            for (int c = 0; c < kMixP; c++) { hi[u * kMixP + c] = 0.0f; lo[u * kMixP + c] = 0.0f; }
        }
        if (mp.fp16) {  // FP32 values, row-major in the tile; k_split16_inplace splits them
          float* out = (float*)tile + (size_t)r * kKB + qc * QW;
#pragma unroll
          for (int c = 0; c < QW; c++) out[c] = hi[c] + lo[c];
        } else {
#pragma unroll
          for (int c8 = 0; c8 < QW; c8 += 8)
            store_split8_ff(tile, half_plane(kTM), t64_off(r, qc * QW + c8, kTM), hi + c8, lo + c8);
        }
      } else if (STAGE == MS_M2L) {
#pragma unroll
        for (int u = 0; u < QW / kMixP; u++) {
          const int b = J.job * (kTM / kMixP) + qc * (QW / kMixP) + u;
          if (b < J.Lt) {
            unsigned char* tile = mp.Psip + ((size_t)J.rt * (mp.Lmax + 1) + b) * kTilePsi;
            if (mp.fp16) {
              float* out = (float*)tile + (size_t)r * kMixP;
#pragma unroll
              for (int c = 0; c < kMixP; c++) out[c] = hi[u * 16 + c] + lo[u * 16 + c];
            } else {
              store_split8_ff(tile, kPlanePsi, cl_off(r, 0, kMixP), hi + u * 16, lo + u * 16);
              store_split8_ff(tile, kPlanePsi, cl_off(r, 8, kMixP), hi + u * 16 + 8,
                              lo + u * 16 + 8);
            }
          }
        }
      } else {
        // The operands carry 24 significant bits, so the output is rounded to FP32
        // (hi + lo) and widened exactly.  Each store of a warp covers 32 consecutive
        // rows of one column.
        const long long row = (long long)J.rt * kTM + r;
#pragma unroll
        for (int c = 0; c < QW; c++) {
          const int oc = __shfl_sync(0xffffffffu, c < 32 ? cm0 : cm1, c & 31);
          if (oc >= 0 && row < mp.rows) {
            const float v = hi[c] + lo[c];
            if (om.Yf) om.Yf[(long long)oc * om.ldy + row] = v;  // the FP32 intermediate
            else om.Y[(long long)oc * om.ldy + row] = widen_f32(v);
          }
        }
      }
    }
    if (!ok) {
      *abort_flag = 1;
      latch(status, SVDUP_ETIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kEpiWarps + 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

template <int STAGE, int W>
void launch_umma(cudaStream_t st, int items_max, Eig e, FmmPlan f, MixPlan mp, OutMap om,
                 int dense, int* status) {
  cudaFuncSetAttribute(k_umma<STAGE, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kSmemBytes);
  const int grid = std::max(1, std::min(items_max, device_sm_count()));  // persistent
  k_umma<STAGE, W><<<grid, kUmmaThreads, kSmemBytes, st>>>(e, f, mp, om, dense, status);
  SVDUP_COUNT_LAUNCH();
}

// ---------------------------------------------------------------------------
// The orthogonalising refinement: operand gathers and the probe check.
// ---------------------------------------------------------------------------
// X^T tile (ct, kt): B-style rows n = columns ct*128 + n of X, K = rows kt*64 + k.  A
// thread takes 8 consecutive rows of one column (contiguous in X).
__global__ void __launch_bounds__(256) k_ref_gather_t(const double* __restrict__ X, long long ldx,
                                                      int rows, int cols, MixPlan mp) {
  if (*mp.gate == 0) return;
  const int ct = blockIdx.x, kt = blockIdx.y;
  unsigned char* tile = mp.Xt + ((size_t)ct * mp.kr + kt) * kTileA;
  for (int it = threadIdx.x; it < kTM * (kKB / 8); it += blockDim.x) {
    const int n = it >> 3, k8 = (it & 7) * 8;
    const int col = ct * kTM + n;
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
      const int row = kt * kKB + k8 + c;
      v[c] = (col < cols && row < rows) ? X[(long long)col * ldx + row] : 0.0;
    }
    store_split8_d(tile, half_plane(kTM), t64_off(n, k8, kTM), v);
  }
}

// X tile (rt, kt): rows rt*128 + r, K = columns kt*64 + k (lanes: consecutive rows).
__global__ void __launch_bounds__(256) k_ref_gather(const double* __restrict__ X, long long ldx,
                                                    int rows, int cols, MixPlan mp) {
  if (*mp.gate == 0) return;
  const int rt = blockIdx.x, kt = blockIdx.y;
  unsigned char* tile = mp.Xp + ((size_t)rt * mp.kx + kt) * kTileA;
  for (int it = threadIdx.x; it < kTM * (kKB / 8); it += blockDim.x) {
    const int r = it & (kTM - 1), ch = it >> 7;
    const long long row = (long long)rt * kTM + r;
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
      const int col = kt * kKB + ch * 8 + c;
      v[c] = (col < cols && row < rows) ? X[(long long)col * ldx + row] : 0.0;
    }
    store_split8_d(tile, half_plane(kTM), t64_off(r, ch * 8, kTM), v);
  }
}

// Probe vectors: entry c of probe q is +-1 by the parity of a SplitMix64 hash of (q, c).
__device__ __forceinline__ double probe_sign(int q, int c) {
  unsigned long long x = 0x9E3779B97F4A7C15ull * (unsigned long long)(4 * (long long)c + q + 1);
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (x & 1ull) ? -1.0 : 1.0;
}

constexpr int kProbeChunk = 512;  // columns per block of the first probe product

// y = X w for the four probes: a thread per row, the columns in chunks over blocks
// (FP64 atomic sums into y, zeroed by the caller).
__global__ void __launch_bounds__(256) k_ref_probe1(const double* __restrict__ X, long long ldx,
                                                    int rows, int cols, double* y) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int c0 = blockIdx.y * kProbeChunk, c1 = min(cols, c0 + kProbeChunk);
  if (r >= rows) return;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  for (int c = c0; c < c1; c++) {
    const double x = X[(long long)c * ldx + r];
    a0 = fma(x, probe_sign(0, c), a0);
    a1 = fma(x, probe_sign(1, c), a1);
    a2 = fma(x, probe_sign(2, c), a2);
    a3 = fma(x, probe_sign(3, c), a3);
  }
  atomicAdd(y + r, a0);
  atomicAdd(y + rows + r, a1);
  atomicAdd(y + 2 * rows + r, a2);
  atomicAdd(y + 3 * rows + r, a3);
}

// v = X^T y - w for the four probes: a block per column.
__global__ void __launch_bounds__(256) k_ref_probe2(const double* __restrict__ X, long long ldx,
                                                    int rows, int cols, const double* __restrict__ y,
                                                    double* v) {
  __shared__ double part[4][8];
  const int c = blockIdx.x;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    const double x = X[(long long)c * ldx + r];
#pragma unroll
    for (int q = 0; q < 4; q++) a[q] = fma(x, y[(long long)q * rows + r], a[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; q++) {
    double t = a[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) part[q][threadIdx.x >> 5] = t;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[threadIdx.x][w];
    v[(long long)threadIdx.x * cols + c] = t - probe_sign(threadIdx.x, c);
  }
}

// residual = max over the probes of ||X^T X w - w|| / ||w|| (||w||^2 = cols); the gate
// opens when it exceeds tol.
__global__ void __launch_bounds__(256) k_ref_gate(const double* __restrict__ v, int cols, double tol,
                                                  double* res, int* gate, int* status) {
  __shared__ double part[4][8];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c = threadIdx.x; c < cols; c += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const double t = v[(long long)q * cols + c];
      a[q] = fma(t, t, a[q]);
    }
#pragma unroll
  for (int q = 0; q < 4; q++) {
    double t = a[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) part[q][threadIdx.x >> 5] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int q = 0; q < 4; q++) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[q][w];
      m = fmax(m, sqrt(t / (double)cols));
    }
    *res = m;
    if (!isfinite(m)) latch(status, SVDUP_ENONFINITE);
    *gate = (tol <= 0.0 || m > tol) && isfinite(m) ? 1 : 0;
  }
}

// Executed tensor-core flops: 2 M N K per split product, six split products (three in
// the FP16 mode).
__global__ void k_mix_flops(Eig e, FmmPlan f, MixPlan mp, int dense, double* acc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double parts = mp.fp16 ? 3.0 : 6.0;
  const double M = (double)mp.rt * kTM, s = (double)mp.s;
  const int Ls = f.L[0], Lt = f.L[1];
  if (Ls == 0) return;
  double p2m = 0.0, m2l = 0.0, out = 0.0;
  if (!dense) {
    p2m = parts * 2.0 * M * kMixP * (double)Ls * s;
    m2l = parts * 2.0 * M * (double)((Lt * kMixP + kTM - 1) / kTM) * kTM *
          (double)((Ls + 3) / 4) * kKB;
  }
  for (int b = 0; b < Lt; b++)
    out += parts * 2.0 * M * s * ((dense ? 0.0 : (double)kMixP) + (double)mp.nnear[b] * s);
  acc[0] += p2m;
  acc[1] += m2l;
  acc[2] += out;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_mix_gather(cudaStream_t st, Eig e, const void* X, bool xf32, long long ldx, int rows,
                       MixPlan mp, OutMap om) {
  dim3 g(mp.rt, mp.kx);
  const size_t sm16 = mp.fp16 ? (size_t)kTM * kKB * sizeof(float) : 0;
  if (xf32) {
    k_mix_gather<float><<<g, 256, sm16, st>>>(e, (const float*)X, ldx, rows, mp);
    SVDUP_COUNT_LAUNCH();
    k_mix_defl<float><<<e.N, 256, 0, st>>>(e, (const float*)X, ldx, rows, om);
  } else {
    k_mix_gather<double><<<g, 256, sm16, st>>>(e, (const double*)X, ldx, rows, mp);
    SVDUP_COUNT_LAUNCH();
    k_mix_defl<double><<<e.N, 256, 0, st>>>(e, (const double*)X, ldx, rows, om);
  }
  SVDUP_COUNT_LAUNCH();
}

void launch_mix_setup(cudaStream_t st, Eig e, FmmPlan f, MixPlan mp, int dense) {
  k_mix_near<<<1, 256, 0, st>>>(f, mp, dense);
  SVDUP_COUNT_LAUNCH();
  const int hs = mp.s / kKB;
  // FP16 mode: each block collects its tile's FP32 values in shared memory
  const size_t f4 = mp.fp16 ? sizeof(float) : 0;
  if (!dense) {
    k_mix_pack_S<<<mp.Lmax * hs, 128, f4 * kMixP * kKB, st>>>(e, f, mp);
    SVDUP_COUNT_LAUNCH();
    k_mix_pack_T<<<dim3(mp.ntT, mp.kphi), 256, f4 * kTM * kKB, st>>>(f, mp);
    SVDUP_COUNT_LAUNCH();
    k_mix_pack_L<<<mp.Lmax + 1, 256, f4 * mp.s * kMixP, st>>>(f, mp);
    SVDUP_COUNT_LAUNCH();
  }
  k_mix_pack_C<<<dim3(mp.Lmax + 1, mp.Lmax, hs), 256, f4 * mp.s * kKB, st>>>(e, f, mp);
  SVDUP_COUNT_LAUNCH();
}

void launch_mix_stage(cudaStream_t st, int stage, Eig e, FmmPlan f, MixPlan mp, OutMap om,
                      int dense, int* status) {
  if (stage == 0) {
    if (dense) return;
    launch_umma<MS_P2M, 64>(st, mp.rt * mp.kphi, e, f, mp, om, dense, status);
    if (mp.fp16) {  // Phi: FP32 values to FP16 planes
      k_split16_inplace<<<mp.rt * mp.kphi, 256, kTM * kKB * sizeof(float), st>>>(
          mp.Phip, kTileA, kTM, kKB, TL_K64, mp.scPhi, mp.kphi, mp.fL, 0);
      SVDUP_COUNT_LAUNCH();
    }
  } else if (stage == 1) {
    if (dense) return;
    launch_umma<MS_M2L, 128>(st, mp.rt * mp.ntT, e, f, mp, om, dense, status);
    if (mp.fp16) {  // Psi: FP32 values to FP16 planes
      k_split16_inplace<<<mp.rt * (mp.Lmax + 1), 256, kTM * kMixP * sizeof(float), st>>>(
          mp.Psip, kTilePsi, kTM, kMixP, TL_K16, mp.scPsi, mp.Lmax + 1, mp.fL, 1);
      SVDUP_COUNT_LAUNCH();
    }
  } else if (mp.s == 64) {
    launch_umma<MS_OUT, 64>(st, mp.rt * (mp.Lmax + 1), e, f, mp, om, dense, status);
  } else {
    launch_umma<MS_OUT, 128>(st, mp.rt * (mp.Lmax + 1), e, f, mp, om, dense, status);
  }
}

void launch_mix_flop_count(cudaStream_t st, Eig e, FmmPlan f, MixPlan mp, int dense,
                           double* acc) {
  k_mix_flops<<<1, 32, 0, st>>>(e, f, mp, dense, acc);
  SVDUP_COUNT_LAUNCH();
}

// ---------------------------------------------------------------------------
// The refinement's scratch and launch sequence.
// ---------------------------------------------------------------------------
namespace {
struct RefLayout {
  size_t off_probe, off_res, off_gate, off_xt, off_et, off_xp, total;
};

RefLayout ref_layout(int rows, int cols) {
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t ct = (cols + kTM - 1) / kTM, rt = (rows + kTM - 1) / kTM;
  const size_t kr = (rows + kKB - 1) / kKB, kx = (cols + kKB - 1) / kKB;
  RefLayout L;
  size_t o = 0;
  L.off_probe = o; o += up(sizeof(double) * (4 * (size_t)rows + 8 * (size_t)cols));
  L.off_res = o; o += up(sizeof(double));
  L.off_gate = o; o += up(sizeof(int));
  L.off_xt = o; o += up(ct * kr * kTileA);
  L.off_et = o; o += up(ct * kx * kTileA);
  L.off_xp = o; o += up(rt * kx * kTileA);
  L.total = o;
  return L;
}
}  // namespace

size_t refine_ws_bytes(int rows, int cols) { return ref_layout(rows, cols).total; }

RefWs refine_ws_carve(void* base, int rows, int cols) {
  const RefLayout L = ref_layout(rows, cols);
  char* b = (char*)base;
  RefWs w;
  memset(&w, 0, sizeof(w));
  w.probe = (double*)(b + L.off_probe);
  w.res = (double*)(b + L.off_res);
  w.gate = (int*)(b + L.off_gate);
  MixPlan& mp = w.mp;
  mp.rows = rows;
  mp.rt = (rows + kTM - 1) / kTM;
  mp.cols = cols;
  mp.ct = (cols + kTM - 1) / kTM;
  mp.kr = (rows + kKB - 1) / kKB;
  mp.kx = (cols + kKB - 1) / kKB;
  mp.Xt = (unsigned char*)(b + L.off_xt);
  mp.Et = (unsigned char*)(b + L.off_et);
  mp.Xp = (unsigned char*)(b + L.off_xp);
  mp.gate = w.gate;
  mp.s = kKB;
  return w;
}

void launch_refine(cudaStream_t st, double* X, long long ldx, int rows, int cols, RefWs ws,
                   double tol, int* status) {
  MixPlan mp = ws.mp;
  mp.Xr = X;
  mp.ldxr = ldx;
  double* w = ws.probe;  // y (4 rows), then v (4 cols)
  cudaMemsetAsync(w, 0, sizeof(double) * 4 * (size_t)rows, st);
  k_ref_probe1<<<dim3((rows + 255) / 256, (cols + kProbeChunk - 1) / kProbeChunk), 256, 0, st>>>(
      X, ldx, rows, cols, w);
  SVDUP_COUNT_LAUNCH();
  k_ref_probe2<<<cols, 256, 0, st>>>(X, ldx, rows, cols, w, w + 4 * (size_t)rows);
  SVDUP_COUNT_LAUNCH();
  k_ref_gate<<<1, 256, 0, st>>>(w + 4 * (size_t)rows, cols, tol, ws.res, ws.gate, status);
  SVDUP_COUNT_LAUNCH();
  // (every kernel below returns at once unless the gate opened)
  k_ref_gather_t<<<dim3(mp.ct, mp.kr), 256, 0, st>>>(X, ldx, rows, cols, mp);
  SVDUP_COUNT_LAUNCH();
  k_ref_gather<<<dim3(mp.rt, mp.kx), 256, 0, st>>>(X, ldx, rows, cols, mp);
  SVDUP_COUNT_LAUNCH();
  Eig e;
  memset(&e, 0, sizeof(e));
  FmmPlan f;
  memset(&f, 0, sizeof(f));
  OutMap om;
  memset(&om, 0, sizeof(om));
  launch_umma<MS_GRAM, 128>(st, mp.ct * mp.ct, e, f, mp, om, 0, status);
  launch_umma<MS_CORR, 128>(st, mp.rt * mp.ct, e, f, mp, om, 0, status);
}

}  // namespace svdup
