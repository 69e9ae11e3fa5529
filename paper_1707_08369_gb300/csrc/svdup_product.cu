// svdup_product.cu -- the product X * Ctilde (RankOneUpdate STEPs 3-7, Sec. 6.2;
// Eq. U1CTrummers / UCTildeProduct) in FP64:
//   Ctilde_tj = zhat_t / (d_t - mu_j) * (1 / ||c_j||)
// evaluated for all rows of X at once by a Chebyshev far-field / direct near-field
// split of the Cauchy matrix (Sec. 5 and App. D, Dutt-Gu-Rokhlin), or densely.
//
// Far field (App. D, read with a flat, single-level partition): the k sorted poles are
// cut into leaves of s consecutive poles, and target leaf b holds roots [b s, b s + s)
// (roots interlace the poles).  For a source leaf a and target leaf b that are well
// separated, 1/(x - y) is interpolated in both variables on p Chebyshev nodes
// t_alpha = cos((2 alpha - 1) pi / (2p)) (App. D STEP 3) with the Lagrange basis
// u_alpha (STEP 4):
//     1/(x - y) ~= sum_alpha sum_beta u_alpha(x^) [1 / (xbar_alpha - ybar_beta)] u_beta(y^),
// which turns the product into three GEMMs over all rows:
//     Phi = X_leaf * S_leaf           (P2M, far-field expansions, STEP 5)
//     Psi = Phi * T                   (M2L, expansions translated to targets, STEP 8)
//     Y   = Psi_leaf * L_leaf + X_near * C_near    (L2P, STEP 9, and P2P, STEP 10)
// The near-field block C_near is generated on the fly from the offsets (never stored).
// Separation: leaves a, b are admissible when |a - b| >= 2 and the gap between their
// intervals is at least max(r_a, r_b); the near range of b is the smallest run of
// source leaves containing b-1..b+1 and every non-admissible leaf.
#include <cuda_runtime.h>

#include "svdup_df.cuh"
#include "svdup_internal.cuh"

namespace svdup {


// ---------------------------------------------------------------------------
// Deflation rotations applied to the columns of X (in place): X <- X G_1^T ... G_r^T,
// i.e. each row of X transforms like z^T.  Rotation i acts on columns (a_i, b_i) with
// (cos, sin) = (c_i, s_i); the deflation walk makes each rotation either open a run
// (a_i untouched so far) or continue the previous one (a_i = b_{i-1}, the run's
// carrier), and different runs touch disjoint columns.  Per row, with x the ORIGINAL
// column values, the carrier follows the affine recurrence
//     v_i = s_i u_i + c_i x_{b_i},   u_i = chained ? v_{i-1} : x_{a_i},
// and the outputs are  X[a_i] = c_i u_i - s_i x_{b_i}  and, at a run's end, X[b_i] = v_i.
// One run can hold thousands of rotations (a graded spectrum merges most of its small
// poles), so the list is cut into chunks of kRotChunk and scanned:
//   prep     per chunk, the row-independent factor A = prod s_i of the map
//            v_out = A v_in + B (A = 0 when a run starts inside the chunk);
//   compose  per (row, chunk), the offset B, and the chunk's last original x_b;
//   carry    per row, the carrier entering every chunk (B is overwritten with it);
//   apply    per (row, chunk), the replay from that carrier, writing X.
// The only column two chunks share is the last b of a chunk that the next chunk
// overwrites as its first a; compose saves its original value, so apply never reads it
// back.  Scratch is chunk-major ([chunk][row]), so the row threads of a block read and
// write it coalesced.  FP64 form: 6 FP64 operations per row and rotation.  The mixed
// form rounds every loaded value once to FP32 and carries unevaluated pairs of FP32
// numbers (about 48 bits), so errors do not grow along long runs; its outputs are
// FP32-accurate, as the split operands that follow.
// ---------------------------------------------------------------------------
constexpr int kRotChunk = 64;
constexpr int kRotBatch = 8;

struct RotScratch {  // carved from the plan's rotation scratch (see launch_rotate_columns)
  double* A;         // [nch] chunk factors
  float4* rotf;      // [N] (c_hi, c_lo, s_hi, s_lo)
  double* Bw;        // [nch][rows] offsets, then carries (the mixed form stores a float2)
  double* Xw;        // [nch][rows] the chunk's last original x_b
};

__global__ void __launch_bounds__(1024) k_rot_prep(Eig e, RotScratch w) {
  const int nr = e.nrot[0];
  const int nch = (nr + kRotChunk - 1) / kRotChunk;
  for (int ch = threadIdx.x; ch < nch; ch += blockDim.x) {
    const int c0 = ch * kRotChunk, c1 = min(nr, c0 + kRotChunk);
    double A = 1.0;
    for (int g = c0; g < c1; g++) {
      const bool chained = g > 0 && e.rj[g] == e.ri[g - 1];
      A = chained ? A * e.rs[g] : 0.0;
    }
    w.A[ch] = A;
  }
  for (int g = threadIdx.x; g < nr; g += blockDim.x) {
    const double c = e.rc[g], sn = e.rs[g];
    const float ch = (float)c, sh = (float)sn;
    w.rotf[g] = make_float4(ch, (float)(c - (double)ch), sh, (float)(sn - (double)sh));
  }
}

// The chunk's rotations, staged once per block.
struct RotChunkSm {
  long long a[kRotChunk], b[kRotChunk];
  long long ya[kRotChunk];  // output column of the deflated a (the product's OutMap)
  float4 cs[kRotChunk];
  double c[kRotChunk], s[kRotChunk];
  unsigned char chained[kRotChunk], ends[kRotChunk];
};

__device__ __forceinline__ int stage_chunk(Eig e, long long ldx, const float4* rotf, int c0,
                                           int nr, RotChunkSm& sm, const OutMap* om) {
  const int cn = min(kRotChunk, nr - c0);
  for (int i = threadIdx.x; i < cn; i += blockDim.x) {
    const int g = c0 + i;
    sm.a[i] = (long long)e.perm[e.rj[g]] * ldx;
    sm.b[i] = (long long)e.perm[e.ri[g]] * ldx;
    if (om) {  // the deflated column goes straight to its output column
      const int q = e.rank_defl[e.rj[g]];
      sm.ya[i] = (om->out_rev ? (long long)(om->out_n - 1 - q) : (long long)q) * om->ldy;
    }
    sm.c[i] = e.rc[g];
    sm.s[i] = e.rs[g];
    sm.cs[i] = rotf[g];
    sm.chained[i] = (g > 0 && e.rj[g] == e.ri[g - 1]) ? 1 : 0;
    sm.ends[i] = (g + 1 >= nr || e.rj[g + 1] != e.ri[g]) ? 1 : 0;
  }
  __syncthreads();
  return cn;
}

// Columns of X are FP64, or FP32 for an intermediate of the mixed form (the first
// product's output, FP32-accurate by construction).
__device__ __forceinline__ float to_f32(double x) { return narrow_rn(x); }
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ void store_from_f32(double* p, float v) { *p = widen_f32(v); }
__device__ __forceinline__ void store_from_f32(float* p, float v) { *p = v; }

// A batch of the chunk's original column values (xb for every rotation, xa where a run
// starts) for row r; i >= cn loads nothing.  xlast replaces the chunk's last b when set.
template <typename T>
__device__ __forceinline__ void rot_load(const T* __restrict__ X, const RotChunkSm& sm,
                                         long long r, int i0, int cn, bool use_last,
                                         double xlast, T (&xb)[kRotBatch], T (&xa)[kRotBatch]) {
#pragma unroll
  for (int u = 0; u < kRotBatch; u++) {
    const int i = i0 + u;
    xb[u] = i < cn ? ((use_last && i == cn - 1) ? (T)xlast : X[r + sm.b[i]]) : (T)0;
    xa[u] = (i < cn && !sm.chained[i]) ? X[r + sm.a[i]] : (T)0;
  }
}

template <bool MIXED, typename T>
__global__ void __launch_bounds__(128) k_rot_compose(Eig e, const T* __restrict__ X,
                                                     long long ldx, int rows, RotScratch w) {
  __shared__ RotChunkSm sm;
  const int nr = e.nrot[0];
  const int ch = blockIdx.y, c0 = ch * kRotChunk;
  if (c0 >= nr) return;
  const int cn = stage_chunk(e, ldx, w.rotf, c0, nr, sm, nullptr);
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double B = 0.0, xlast = 0.0;
  Df Bf = {0.f, 0.f};
  // (no prefetch of the next batch here: this kernel is bound by its arithmetic issue
  // rate, and the extra registers would cost occupancy)
  for (int i0 = 0; i0 < cn; i0 += kRotBatch) {
    T xb[kRotBatch], xa[kRotBatch];
    rot_load<T>(X, sm, r, i0, cn, false, 0.0, xb, xa);
#pragma unroll
    for (int u = 0; u < kRotBatch; u++) {
      const int i = i0 + u;
      if (i < cn) {
        if (!MIXED) {
          B = fma(sm.s[i], sm.chained[i] ? B : xa[u], sm.c[i] * xb[u]);
        } else {
          const float4 q = sm.cs[i];
          const Df uu = sm.chained[i] ? Bf : Df{to_f32(xa[u]), 0.f};
          Bf = df_add(df_mul(Df{q.z, q.w}, uu), df_mul(Df{q.x, q.y}, Df{to_f32(xb[u]), 0.f}));
        }
        xlast = (double)xb[u];
      }
    }
  }
  const size_t o = (size_t)ch * rows + r;
  if (MIXED) {
    float2 t = make_float2(Bf.hi, Bf.lo);
    w.Bw[o] = *reinterpret_cast<double*>(&t);
  } else {
    w.Bw[o] = B;
  }
  w.Xw[o] = xlast;
}

template <bool MIXED>
__global__ void k_rot_carry(Eig e, int rows, RotScratch w) {
  const int nr = e.nrot[0];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows || nr == 0) return;
  const int nch = (nr + kRotChunk - 1) / kRotChunk;
  double v = 0.0;
  Df vf = {0.f, 0.f};
  for (int ch = 0; ch < nch; ch++) {
    const size_t o = (size_t)ch * rows + r;
    const double B = w.Bw[o], A = w.A[ch];
    if (!MIXED) {
      w.Bw[o] = v;  // the carrier entering this chunk
      v = fma(A, v, B);
    } else {
      float2 t;
      *reinterpret_cast<double*>(&t) = B;
      float2 cur = make_float2(vf.hi, vf.lo);
      w.Bw[o] = *reinterpret_cast<double*>(&cur);
      vf = df_add(df_mul(df_from_f64(A, 0), vf), Df{t.x, t.y});
    }
  }
}

template <bool MIXED, typename T>
__global__ void __launch_bounds__(128) k_rot_apply(Eig e, T* X, long long ldx, int rows,
                                                   RotScratch w, OutMap om) {
  __shared__ RotChunkSm sm;
  const int nr = e.nrot[0];
  const int ch = blockIdx.y, c0 = ch * kRotChunk;
  if (c0 >= nr) return;
  const int cn = stage_chunk(e, ldx, w.rotf, c0, nr, sm, &om);
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const size_t o = (size_t)ch * rows + r;
  const double xlast = w.Xw[o];
  double v = w.Bw[o];
  Df vf;
  if (MIXED) {
    float2 t;
    *reinterpret_cast<double*>(&t) = v;
    vf = Df{t.x, t.y};
  }
  // Loads run a batch ahead of the arithmetic.  Within a chunk, column b_i is written
  // only at rotation i (a run's end, and no later rotation reads it) and a run-start
  // column a_i is never written (its output goes to Y), so no value loaded early has
  // been written yet; the chunk's last b comes from compose (the next chunk may write it).
  T xb[kRotBatch], xa[kRotBatch], nb[kRotBatch], na[kRotBatch];
  rot_load<T>(X, sm, r, 0, cn, true, xlast, xb, xa);
  for (int i0 = 0; i0 < cn; i0 += kRotBatch) {
    if (i0 + kRotBatch < cn) rot_load<T>(X, sm, r, i0 + kRotBatch, cn, true, xlast, nb, na);
#pragma unroll
    for (int u = 0; u < kRotBatch; u++) {
      const int i = i0 + u;
      if (i < cn) {
        if (!MIXED) {
          const double uu = sm.chained[i] ? v : (double)xa[u];
          om.Y[r + sm.ya[i]] = fma(sm.c[i], uu, -sm.s[i] * (double)xb[u]);
          v = fma(sm.s[i], uu, sm.c[i] * (double)xb[u]);
          if (sm.ends[i]) X[r + sm.b[i]] = (T)v;
        } else {
          // the carrier stays a pair (runs are long); the deflated output is a rotation
          // of two unit-scale values and needs FP32 accuracy only
          const float4 q = sm.cs[i];
          const Df cc = {q.x, q.y}, ss = {q.z, q.w};
          const float xx = to_f32(xb[u]);
          const Df uu = sm.chained[i] ? vf : Df{to_f32(xa[u]), 0.f};
          float t = fmaf(cc.lo, uu.hi, -ss.lo * xx);
          t = fmaf(cc.hi, uu.lo, t);
          t = fmaf(-ss.hi, xx, t);
          const float ov = fmaf(cc.hi, uu.hi, t);
          if (om.Yf) om.Yf[r + sm.ya[i]] = ov;
          else om.Y[r + sm.ya[i]] = widen_f32(ov);
          vf = df_add(df_mul(ss, uu), df_mul(cc, Df{xx, 0.f}));
          if (sm.ends[i]) store_from_f32(&X[r + sm.b[i]], vf.hi + vf.lo);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kRotBatch; u++) {
      xb[u] = nb[u];
      xa[u] = na[u];
    }
  }
}

size_t rotate_scratch_bytes(int N, int rows) {
  const size_t nch = ((size_t)N + kRotChunk - 1) / kRotChunk;
  const size_t rr = (size_t)(rows > 0 ? rows : 1);
  return nch * 8 + (size_t)N * 16 + 2 * nch * rr * 8 + 256;
}

static RotScratch rot_scratch(Eig e, int rows, void* scratch) {
  const int nch = (e.N + kRotChunk - 1) / kRotChunk;
  const size_t rr = (size_t)(rows > 0 ? rows : 1);
  RotScratch w;
  unsigned char* p = (unsigned char*)scratch;
  w.A = (double*)p;
  p += ((size_t)nch * 8 + 15) & ~(size_t)15;
  w.rotf = (float4*)p;
  p += (size_t)e.N * 16;
  w.Bw = (double*)p;
  w.Xw = w.Bw + (size_t)nch * rr;
  return w;
}

// The scan's first half (chunk factors, offsets, carries): needs the deflation only.
// X is FP64, or FP32 when xf32 (mixed only).
void launch_rotate_prepare(cudaStream_t st, Eig e, const void* X, long long ldx, int rows,
                           void* scratch, bool mixed, bool xf32) {
  const int nch = (e.N + kRotChunk - 1) / kRotChunk;
  if (rows <= 0 || nch == 0) return;
  const RotScratch w = rot_scratch(e, rows, scratch);
  k_rot_prep<<<1, 1024, 0, st>>>(e, w);
  SVDUP_COUNT_LAUNCH();
  dim3 g((rows + 127) / 128, nch);
  if (mixed && xf32) k_rot_compose<true, float><<<g, 128, 0, st>>>(e, (const float*)X, ldx, rows, w);
  else if (mixed) k_rot_compose<true, double><<<g, 128, 0, st>>>(e, (const double*)X, ldx, rows, w);
  else k_rot_compose<false, double><<<g, 128, 0, st>>>(e, (const double*)X, ldx, rows, w);
  SVDUP_COUNT_LAUNCH();
  if (mixed) k_rot_carry<true><<<(rows + 127) / 128, 128, 0, st>>>(e, rows, w);
  else k_rot_carry<false><<<(rows + 127) / 128, 128, 0, st>>>(e, rows, w);
  SVDUP_COUNT_LAUNCH();
}

// The replay: deflated columns go to their output columns, which needs the final order
// of the eigenvalues (after the roots and their merge with the deflated values).
void launch_rotate_apply(cudaStream_t st, Eig e, void* X, long long ldx, int rows,
                         void* scratch, bool mixed, OutMap om, bool xf32) {
  const int nch = (e.N + kRotChunk - 1) / kRotChunk;
  if (rows <= 0 || nch == 0) return;
  const RotScratch w = rot_scratch(e, rows, scratch);
  dim3 g((rows + 127) / 128, nch);
  if (mixed && xf32) k_rot_apply<true, float><<<g, 128, 0, st>>>(e, (float*)X, ldx, rows, w, om);
  else if (mixed) k_rot_apply<true, double><<<g, 128, 0, st>>>(e, (double*)X, ldx, rows, w, om);
  else k_rot_apply<false, double><<<g, 128, 0, st>>>(e, (double*)X, ldx, rows, w, om);
  SVDUP_COUNT_LAUNCH();
}

void launch_rotate_columns(cudaStream_t st, Eig e, double* X, long long ldx, int rows,
                           void* scratch, bool mixed, OutMap om) {
  launch_rotate_prepare(st, e, X, ldx, rows, scratch, mixed, false);
  launch_rotate_apply(st, e, X, ldx, rows, scratch, mixed, om, false);
}

__device__ __forceinline__ long long out_col(const OutMap& om, int q) {
  return om.out_rev ? (long long)(om.out_n - 1 - q) : (long long)q;
}

// Non-deflated columns gathered into sorted order (Xs[:, t] = X[:, perm[idx[t]]]);
// deflated columns are eigenvectors already and go straight to their output column.
// One block per column.
__global__ void k_gather_columns(Eig e, const double* __restrict__ X, long long ldx, int rows,
                                 double* Xs, long long ldxs, OutMap om) {
  const int k = e.kp[0];
  const int c = blockIdx.x;
  if (c < k) {
    const double* src = X + (long long)e.perm[e.idx[c]] * ldx;
    double* dst = Xs + (long long)c * ldxs;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) dst[r] = src[r];
  } else if (c < e.N) {
    int s = e.didx[c - k];
    if (e.defl[s] == 2) return;  // written by the rotation kernel
    int q = e.rank_defl[s];
    const double* src = X + (long long)e.perm[s] * ldx;
    double* dst = om.Y + out_col(om, q) * om.ldy;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) dst[r] = src[r];
  }
}

void launch_gather_columns(cudaStream_t st, Eig e, const double* X, long long ldx, int rows,
                           double* Xs, long long ldxs, OutMap om) {
  k_gather_columns<<<e.N, 256, 0, st>>>(e, X, ldx, rows, Xs, ldxs, om);
  SVDUP_COUNT_LAUNCH();
}

// ---------------------------------------------------------------------------
// FMM set-up: leaves, boxes, near ranges, and the operator matrices.
// ---------------------------------------------------------------------------
// Leaves and boxes.  The largest poles of a solve may stand far above the rest (the
// large eigenvalues that earlier updates added); a leaf holding them and ordinary poles
// would reach over the whole spectrum and be near every target.  So the partition is
// shifted to start a leaf at that group: with g the first pole above a gap wider than
// half the span of the top s + 1 poles (at most kMaxTop poles above it; g = k when
// there is none), source leaf a holds the sorted poles [a s - P, a s + s - P) with
// P = (-g) mod s, and target leaf b < Lt - 1 the roots [b s - Pt, b s + s - Pt) that lie
// between poles, with Pt = (-gt) mod s for gt the root in the gap (g - 1 when rho > 0,
// g when rho < 0), so that the root in the gap and the roots above it share a leaf.  The
// last target leaf holds the root beyond all poles.  Dense mode: one source leaf with
// every pole, one target leaf with every root.
constexpr int kMaxTop = 16;

__device__ int top_group(const double* __restrict__ dk, int k, int s) {
  if (k < 2 * s + 2) return k;
  const double span = dk[k - 1] - dk[k - 1 - s];
  double gmax = -1.0;
  int g = k;
  for (int j = k - 2; j >= k - 1 - s; j--) {
    const double gap = dk[j + 1] - dk[j];
    if (gap > gmax) { gmax = gap; g = j + 1; }
  }
  return (gmax > 0.5 * span && k - g <= kMaxTop) ? g : k;
}

__global__ void k_fmm_boxes(Eig e, FmmPlan f, int dense) {
  const int k = e.kp[0];
  const double rho = e.rhop[0];
  const int rlo = rho > 0.0 ? 0 : 1, rhi = rho > 0.0 ? k - 1 : k;  // roots between poles
  int Ls, Lt, P = 0, Pt = 0;
  if (k == 0) { Ls = 0; Lt = 0; }
  else if (dense) { Ls = 1; Lt = 1; }
  else {
    const int g = top_group(e.dk, k, f.s);
    if (g < k) {
      const int gt = rho > 0.0 ? g - 1 : g;
      P = (f.s - g % f.s) % f.s;
      Pt = (f.s - gt % f.s) % f.s;
    }
    Ls = (k + P + f.s - 1) / f.s;
    Lt = (rhi > rlo ? (rhi - 1 + Pt) / f.s + 1 : 1) + 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    f.L[0] = Ls;
    f.L[1] = Lt;
    f.L[2] = P;
    f.L[3] = Pt;
  }
  const int s = dense ? max(k, 1) : f.s;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < Lt; a += gridDim.x * blockDim.x) {
    if (a < Ls) {
      const int t0 = max(0, a * s - P), t1 = min(k, a * s + s - P) - 1;
      const double lo = e.dk[t0], hi = e.dk[t1];
      f.sbox_c[a] = 0.5 * (lo + hi);
      f.sbox_r[a] = box_radius(lo, hi);
    }
    int j0, j1;
    if (dense) { j0 = 0; j1 = k; }
    else if (a < Lt - 1) {
      j0 = max(a * s - Pt, rlo);
      j1 = min(a * s + s - Pt, rhi);
      if (j1 < j0) j1 = j0;
    } else {
      j0 = rho > 0.0 ? k - 1 : 0;
      j1 = j0 + 1;
    }
    f.tj0[a] = j0;
    f.tj1[a] = j1;
    if (j1 > j0) {
      double lo = e.dorg[j0] + e.tau[j0], hi = e.dorg[j1 - 1] + e.tau[j1 - 1];
      f.tbox_c[a] = 0.5 * (lo + hi);
      f.tbox_r[a] = box_radius(lo, hi);
    } else {
      f.tbox_c[a] = 0.0;
      f.tbox_r[a] = 1.0;
    }
  }
}

// Near list of target leaf b: the source leaves b-1..b+1 (for b < Lt - 1) and every source
// leaf a not admissible with b, i.e. with |c_a - c_b| - r_a - r_b < max(r_a, r_b).
// Everything else is far field.
__global__ void k_fmm_near(Eig e, FmmPlan f, int dense) {
  const int Ls = f.L[0], Lt = f.L[1];
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < Lt; b += gridDim.x * blockDim.x) {
    int* lst = f.near + (long long)b * f.Lmax;
    if (dense) { lst[0] = 0; f.nnear[b] = 1; continue; }
    int cnt = 0;
    const bool has = f.tj1[b] > f.tj0[b];
    const double cb = f.tbox_c[b], rb = f.tbox_r[b];
    for (int a = 0; a < Ls; a++) {
      bool nr = (b < Lt - 1 && a >= b - 1 && a <= b + 1);
      if (!nr && has) {
        double ca = f.sbox_c[a], ra = f.sbox_r[a];
        double gap = fabs(ca - cb) - ra - rb;
        nr = !(gap >= fmax(ra, rb));
      }
      if (nr) lst[cnt++] = a;
    }
    f.nnear[b] = cnt;
  }
}

__device__ __forceinline__ bool is_near(const FmmPlan& f, int b, int a) {
  const int* lst = f.near + (long long)b * f.Lmax;
  const int n = f.nnear[b];
  for (int i = 0; i < n; i++) {
    if (lst[i] == a) return true;
    if (lst[i] > a) return false;
  }
  return false;
}

// P2M operator of source leaf a: S[a][alpha][tl] = zhat_t u_alpha((d_t - c_a) / r_a)
// (App. D STEP 5 with the far-field variable mapped to [-1, 1]); one thread per pole.
__global__ void k_fmm_S(Eig e, FmmPlan f) {
  __shared__ double st[32], sw[32];
  cheb_tables(f.p, st, sw);
  const int k = e.kp[0], L = f.L[0], p = f.p, s = f.s, P = f.L[2];
  const long long total = (long long)L * s;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(x / s), tl = (int)(x - (long long)a * s);
    const int t = a * s + tl - P;
    double* col = f.S + (size_t)a * s * p + tl;
    if (t >= 0 && t < k) {
      double u[32];
      lagrange_all(p, box_coord(e.dk[t] - f.sbox_c[a], f.sbox_r[a]), st, sw, u);
      const double zt = e.zhat[t];
      for (int alpha = 0; alpha < p; alpha++) col[(size_t)alpha * s] = zt * u[alpha];
    } else {
      for (int alpha = 0; alpha < p; alpha++) col[(size_t)alpha * s] = 0.0;
    }
  }
}

// M2L operator: T[(a, alpha), (b, beta)] = 1 / (xbar_{a,alpha} - ybar_{b,beta}) for
// admissible pairs, 0 otherwise (App. D STEP 8, with the kernel evaluated at the two
// boxes' Chebyshev nodes).  Col-major with leading dimension Lmax p.
__global__ void k_fmm_T(FmmPlan f) {
  const int Ls = f.L[0], Lt = f.L[1], p = f.p;
  const long long ldT = (long long)f.Lmax * p;
  const long long nr = (long long)Ls * p, nc = (long long)Lt * p;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < nr * nc;
       x += (long long)gridDim.x * blockDim.x) {
    int col = (int)(x / nr), row = (int)(x - (long long)col * nr);
    int a = row / p, alpha = row - a * p;
    int b = col / p, beta = col - b * p;
    double v = 0.0;
    if (!is_near(f, b, a)) {
      double xa = (f.sbox_c[a] - f.tbox_c[b]) + f.sbox_r[a] * cheb_node(alpha, p) -
                  f.tbox_r[b] * cheb_node(beta, p);
      v = 1.0 / xa;
    }
    f.T[row + col * ldT] = v;
  }
}

// L2P operator of target leaf b: Lop[b][jl][beta] = u_beta((mu_j - c_b) / r_b) inv_j
// (App. D STEP 9), j = tj0[b] + jl; one thread per root.
__global__ void k_fmm_L(Eig e, FmmPlan f) {
  __shared__ double st[32], sw[32];
  cheb_tables(f.p, st, sw);
  const int Lt = f.L[1], p = f.p, s = f.s;
  const long long total = (long long)Lt * s;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(x / s), jl = (int)(x - (long long)b * s);
    const int j = f.tj0[b] + jl;
    double* out = f.Lop + (size_t)b * s * p + (size_t)jl * p;
    if (j < f.tj1[b]) {
      double u[32];
      lagrange_all(p, box_coord((e.dorg[j] - f.tbox_c[b]) + e.tau[j], f.tbox_r[b]), st, sw, u);
      const double inv = e.inv[j];
      for (int beta = 0; beta < p; beta++) out[beta] = u[beta] * inv;
    } else {
      for (int beta = 0; beta < p; beta++) out[beta] = 0.0;
    }
  }
}

// Leaves and their boxes: the poles (and the leaf offset at an isolated top group) and the
// roots; no zhat or norms.
void launch_fmm_boxes(cudaStream_t st, Eig e, FmmPlan f, int dense) {
  k_fmm_boxes<<<(f.Lmax + 128) / 128, 128, 0, st>>>(e, f, dense);
  SVDUP_COUNT_LAUNCH();
}

// Near lists and the far-field operators (S carries zhat, L the column norms).
void launch_fmm_ops(cudaStream_t st, Eig e, FmmPlan f, int dense) {
  k_fmm_near<<<(f.Lmax + 128) / 128, 128, 0, st>>>(e, f, dense);
  SVDUP_COUNT_LAUNCH();
  if (dense) return;
  long long sp = (long long)(f.Lmax + 1) * f.s;
  int blocks = (int)((sp + 127) / 128);
  k_fmm_S<<<blocks, 128, 0, st>>>(e, f);
  SVDUP_COUNT_LAUNCH();
  k_fmm_L<<<blocks, 128, 0, st>>>(e, f);
  SVDUP_COUNT_LAUNCH();
  if (f.tree) return;  // the hierarchy forms its translations in its GEMMs
  long long nt = (long long)f.Lmax * f.p * (long long)(f.Lmax + 1) * f.p;
  int tb = (int)((nt + 255) / 256);
  k_fmm_T<<<tb, 256, 0, st>>>(f);
  SVDUP_COUNT_LAUNCH();
}

void launch_fmm_setup(cudaStream_t st, Eig e, FmmPlan f, int dense) {
  launch_fmm_boxes(st, e, f, dense);
  launch_fmm_ops(st, e, f, dense);
}

// ---------------------------------------------------------------------------
// FP64 GEMM tiles for the three stages.  Tile 64 rows x 32 columns, K in steps of 16,
// 128 threads, 4 x 4 outputs per thread.  (FP64 on this part issues roughly two DFMA
// per SM per clock, so the tile only has to keep the FP64 pipe fed.)
// ---------------------------------------------------------------------------
constexpr int BM = 64, BN = 32, BK = 16;

enum { ST_P2M = 0, ST_M2L = 1, ST_OUT = 2 };

template <int STAGE>
__global__ void __launch_bounds__(128) k_gemm_f64(Eig e, FmmPlan f, int rows,
                                                  const double* __restrict__ Xs, long long ldxs,
                                                  OutMap om, int dense) {
  __shared__ double As[BK][BM];
  __shared__ double Bs[BK][BN + 1];
  const int k = e.kp[0];
  const int Ls = f.L[0], Lt = f.L[1];
  const int p = f.p;
  const int s = dense ? max(k, 1) : f.s;
  const int P = dense ? 0 : f.L[2];  // K positions g are poles g - P (leaf offset)
  const int leaf = blockIdx.y;
  if (leaf >= (STAGE == ST_P2M ? Ls : Lt)) return;
  const int r0 = blockIdx.x * BM;
  const int c0 = blockIdx.z * BN;  // column chunk within the block's output range
  int ncols, j0 = 0;
  if (STAGE == ST_P2M || STAGE == ST_M2L) ncols = p;
  else { j0 = f.tj0[leaf]; ncols = f.tj1[leaf] - j0; }
  if (c0 >= ncols) return;
  const int tid = threadIdx.x;
  const int tx = tid & 7, ty = tid >> 3;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

  // K segments.  P2M: the leaf's poles.  M2L: every source expansion (T is zero on
  // near pairs).  Output: the leaf's local expansion (L2P), then each near source leaf.
  int nseg;
  if (STAGE == ST_P2M || STAGE == ST_M2L) nseg = 1;
  else nseg = dense ? 2 : 1 + f.nnear[leaf];
  for (int sg = 0; sg < nseg; sg++) {
    int g0, g1;
    if (STAGE == ST_P2M) { g0 = leaf * f.s; g1 = min(k + P, g0 + f.s); }
    else if (STAGE == ST_M2L) { g0 = 0; g1 = Ls * p; }
    else if (dense) { g0 = 0; g1 = (sg == 0) ? 0 : k; }
    else if (sg == 0) { g0 = 0; g1 = p; }
    else {
      int a = f.near[(long long)leaf * f.Lmax + sg - 1];
      g0 = a * f.s;
      g1 = min(k + P, g0 + f.s);
    }
    const bool poles = STAGE == ST_P2M || (STAGE == ST_OUT && sg > 0);
    for (int kb = g0; kb < g1; kb += BK) {
      // A tile: BK columns x BM rows
      for (int x = tid; x < BK * BM; x += 128) {
        int kk = x / BM, r = x - kk * BM;
        int g = kb + kk;
        double v = 0.0;
        if (g < g1 && r0 + r < rows && !(poles && g < P)) {
          const double* col;
          if (STAGE == ST_P2M) col = Xs + (long long)(g - P) * ldxs;
          else if (STAGE == ST_M2L) col = f.Phi + (long long)g * f.ldphi;
          else col = (sg == 0) ? f.Psi + (long long)(leaf * p + g) * f.ldphi
                               : Xs + (long long)(g - P) * ldxs;
          v = col[r0 + r];
        }
        As[kk][r] = v;
      }
      // B tile: BK x BN
      for (int x = tid; x < BK * BN; x += 128) {
        int kk = x / BN, c = x - kk * BN;
        int g = kb + kk;
        int cc = c0 + c;
        double v = 0.0;
        if (g < g1 && cc < ncols) {
          if (STAGE == ST_P2M) {
            v = f.S[(long long)leaf * f.s * p + (long long)cc * f.s + (g - leaf * f.s)];
          } else if (STAGE == ST_M2L) {
            v = f.T[(long long)g + (long long)(leaf * p + cc) * ((long long)f.Lmax * p)];
          } else if (sg == 0) {
            v = f.Lop[(long long)leaf * f.s * p + (long long)cc * p + g];
          } else if (g >= P) {
            const int j = j0 + cc, t = g - P;
            double del = (e.dk[t] - e.dorg[j]) - e.tau[j];
            v = e.zhat[t] * e.inv[j] * rcp64(del);
          }
        }
        Bs[kk][c] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; kk++) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
          for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  // epilogue
#pragma unroll
  for (int j = 0; j < 4; j++) {
    int cc = c0 + tx * 4 + j;
    if (cc >= ncols) continue;
    double* col;
    if (STAGE == ST_P2M) col = f.Phi + (long long)(leaf * p + cc) * f.ldphi;
    else if (STAGE == ST_M2L) col = f.Psi + (long long)(leaf * p + cc) * f.ldphi;
    else col = om.Y + out_col(om, e.rank_root[j0 + cc]) * om.ldy;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      int r = r0 + ty * 4 + i;
      if (r < rows) col[r] = acc[i][j];
    }
  }
}

// Useful flops of the three product stages (2 per multiply-add), from the device-side
// plan: P2M 2 rows k p; M2L 2 rows p^2 per admissible leaf pair; output 2 rows s_b
// (p + near sources of b) per target leaf (dense: 2 rows k^2).
__global__ void k_flop_count(Eig e, FmmPlan f, int rows, int dense, double* acc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = e.kp[0];
  const double R = (double)rows;
  if (dense) {
    acc[2] += 2.0 * R * (double)k * (double)k;
    acc[8] += 2.0 * R * (double)k * (double)k;
    return;
  }
  const int Ls = f.L[0], Lt = f.L[1], p = f.p, s = f.s, P = f.L[2];
  double p2m = 2.0 * R * (double)k * p, m2l = 0.0, out = 0.0;
  for (int b = 0; b < Lt; b++) {
    int nb = f.tj1[b] - f.tj0[b];
    if (nb <= 0) continue;
    int near_src = 0;
    for (int i = 0; i < f.nnear[b]; i++) {
      int a = f.near[(long long)b * f.Lmax + i];
      near_src += min(k, a * s + s - P) - max(0, a * s - P);
    }
    if (!f.tree) m2l += 2.0 * R * (double)p * p * (double)(Ls - f.nnear[b]);
    out += 2.0 * R * (double)nb * (double)(p + near_src);
  }
  acc[0] += p2m;
  acc[1] += m2l;
  acc[2] += out;
  // App. D's operation count for N = k points with leaves of s = 2p: STEPs 5-6 (the
  // far-field expansions and their bottom-up shifts) 2 N p multiply-adds, STEPs 7-8 (the
  // local expansions and translations) 5 N p, STEPs 9-10 (evaluation and the near field)
  // 7 N p; 14 N p in all, for each of the `rows` right-hand sides.
  const double np = R * (double)k * p;
  acc[6] += 4.0 * np;
  acc[7] += 10.0 * np;
  acc[8] += 14.0 * np;
}

void launch_flop_count(cudaStream_t st, Eig e, FmmPlan f, int rows, int dense, double* acc) {
  k_flop_count<<<1, 32, 0, st>>>(e, f, rows, dense, acc);
  SVDUP_COUNT_LAUNCH();
}

void launch_product_f64_stage(cudaStream_t st, int stage, Eig e, FmmPlan f, int rows,
                              const double* Xs, long long ldxs, OutMap om, int dense) {
  int rt = (rows + BM - 1) / BM;
  if (dense) {
    if (stage != 2) return;
    dim3 g3(rt, 1, (e.N + BN - 1) / BN);
    k_gemm_f64<ST_OUT><<<g3, 128, 0, st>>>(e, f, rows, Xs, ldxs, om, dense);
    SVDUP_COUNT_LAUNCH();
    return;
  }
  int pc = (f.p + BN - 1) / BN;
  if (stage == 0) {
    dim3 g1(rt, f.Lmax, pc);
    k_gemm_f64<ST_P2M><<<g1, 128, 0, st>>>(e, f, rows, Xs, ldxs, om, dense);
  } else if (stage == 1) {
    dim3 g1(rt, f.Lmax + 1, pc);
    k_gemm_f64<ST_M2L><<<g1, 128, 0, st>>>(e, f, rows, Xs, ldxs, om, dense);
  } else {
    dim3 g3(rt, f.Lmax + 1, (f.s + BN - 1) / BN);
    k_gemm_f64<ST_OUT><<<g3, 128, 0, st>>>(e, f, rows, Xs, ldxs, om, dense);
  }
  SVDUP_COUNT_LAUNCH();
}

}  // namespace svdup
