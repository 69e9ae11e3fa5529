// svdup_solve.cu -- the scalar (FP64) stages of the rank-one SVD update:
//   the projections p = U^T a, q = V^T b (Alg. 6.1 STEP 1, rewritten, see below),
//   the 2x2 Schur splits and z vectors (STEPs 2-3, App. A),
//   sorting and deflation (Sec. 3.1),
//   the secular-equation roots (Sec. 3.1, RankOneUpdate STEP 2),
//   z recomputed from the roots and the column norms of the Cauchy-like
//   eigenvector matrix (Sec. 3.2, Eq. CTildeFinalForm1; RankOneUpdate STEP 7),
//   Cauchy matrix-vector products with those matrices (the second z, the sign
//   probe that pairs left and right vectors), and Shat = sqrt(D_n) (STEP 8).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "svdup_df.cuh"
#include "svdup_internal.cuh"

namespace svdup {


// ---------------------------------------------------------------------------
// Alg. 6.1 STEP 1.  The paper forms btilde = U S V^T b and atilde = V S^T U^T a and
// then, inside RankOneUpdate STEP 1, abar = U^T a1.  With U, V orthogonal (App. A)
// U^T btilde = S (V^T b) and V^T atilde = S^T (U^T a), so every z vector follows from
// p = U^T a and q = V^T b: one pass over U and one over V.
// The pass is bound by reading U and V (8 (m^2 + n^2) bytes), so the dot products run
// on FP32 pairs (svdup_df.cuh) rather than on the FP64 pipe, which would take twice the
// time of the reads: every entry of U (|u| <= 1) and of a 2^-Ea is truncated to a pair
// (47 bits), their product formed exactly but for the lo.lo term, and the sum kept as a
// pair.  Each term carries about 2^-46 relative error, so the result's error is about
// 2^-46 sum |u_r a_r|, the size of an FP64 dot product's typical rounding (sqrt(m) u).
// k_gemv_prep (one block): Ea, Eb (exponents of max|a|, max|b|), the pairs of
// a 2^-Ea and b 2^-Eb, and alpha = a^T a, beta = b^T b in FP64.
// k_gemv_pq: one block per column, [0, m) of U and [m, m + n) of V.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_gemv_prep(int m, int n, const double* __restrict__ a,
                                                    const double* __restrict__ b, float2* abf,
                                                    int* abe, double* ab) {
  __shared__ double red[2][32];
  __shared__ int sx[2];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nt = blockDim.x;
  if (tid < 2) sx[tid] = -1100;
  __syncthreads();
  double s0 = 0.0, s1 = 0.0;
  int ea = -1100, eb = -1100;
  for (int r = tid; r < m; r += nt) {
    const double x = a[r];
    s0 = fma(x, x, s0);
    ea = max(ea, exp2_of(x));
  }
  for (int r = tid; r < n; r += nt) {
    const double x = b[r];
    s1 = fma(x, x, s1);
    eb = max(eb, exp2_of(x));
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, o));
    eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, o));
  }
  if (lane == 0) {
    red[0][w] = s0;
    red[1][w] = s1;
    atomicMax(&sx[0], ea);
    atomicMax(&sx[1], eb);
  }
  __syncthreads();
  if (w == 0) {
    const int nw = nt >> 5;
    s0 = lane < nw ? red[0][lane] : 0.0;
    s1 = lane < nw ? red[1][lane] : 0.0;
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (lane == 0) {
      ab[0] = s0;
      ab[1] = s1;
    }
  }
  const int Ea = sx[0] < -1000 ? 0 : sx[0], Eb = sx[1] < -1000 ? 0 : sx[1];
  if (tid == 0) {
    abe[0] = Ea;
    abe[1] = Eb;
  }
  for (int r = tid; r < m; r += nt) {
    const Df v = df_from_f64(a[r], Ea);
    abf[r] = make_float2(v.hi, v.lo);
  }
  for (int r = tid; r < n; r += nt) {
    const Df v = df_from_f64(b[r], Eb);
    abf[m + r] = make_float2(v.hi, v.lo);
  }
}

__global__ void __launch_bounds__(256) k_gemv_pq(int m, int n, const double* __restrict__ U,
                                                 long long ldu, const double* __restrict__ V,
                                                 long long ldv, const float2* __restrict__ abf,
                                                 const int* __restrict__ abe, double* p, double* q) {
  __shared__ float2 red[8];
  const int c = blockIdx.x;
  const bool left = c < m;
  const double* col = left ? U + (long long)c * ldu : V + (long long)(c - m) * ldv;
  const float2* vec = left ? abf : abf + m;
  const int len = left ? m : n;
  // four rows per thread and step, their loads issued together (the pass is bound by
  // the loads in flight), summed into two chains
  Df acc = {0.0f, 0.0f}, acc2 = {0.0f, 0.0f};
  const int bd = blockDim.x;
  int r = threadIdx.x;
  for (; r + 3 * bd < len; r += 4 * bd) {
    const double u0 = col[r], u1 = col[r + bd], u2 = col[r + 2 * bd], u3 = col[r + 3 * bd];
    const float2 v0 = vec[r], v1 = vec[r + bd], v2 = vec[r + 2 * bd], v3 = vec[r + 3 * bd];
    acc = df_add(acc, df_mul(df_from_f64(u0, 0), Df{v0.x, v0.y}));
    acc2 = df_add(acc2, df_mul(df_from_f64(u1, 0), Df{v1.x, v1.y}));
    acc = df_add(acc, df_mul(df_from_f64(u2, 0), Df{v2.x, v2.y}));
    acc2 = df_add(acc2, df_mul(df_from_f64(u3, 0), Df{v3.x, v3.y}));
  }
  for (; r < len; r += bd) {
    const float2 v = vec[r];
    acc = df_add(acc, df_mul(df_from_f64(col[r], 0), Df{v.x, v.y}));
  }
  acc = df_warp_sum(df_add(acc, acc2));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = make_float2(acc.hi, acc.lo);
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    const float2 t = l < nw ? red[l] : make_float2(0.0f, 0.0f);
    acc = df_warp_sum(Df{t.x, t.y});
    if (l == 0) {
      const double r = df_to_f64(acc, left ? abe[0] : abe[1]);
      if (left) p[c] = r;
      else q[c - m] = r;
    }
  }
}

void launch_gemv_pq(cudaStream_t st, int m, int n, const double* U, long long ldu, const double* V,
                    long long ldv, const double* a, const double* b, double* p, double* q,
                    double* ab, float2* abf, int* abe) {
  k_gemv_prep<<<1, 1024, 0, st>>>(m, n, a, b, abf, abe, ab);
  SVDUP_COUNT_LAUNCH();
  k_gemv_pq<<<m + n, 256, 0, st>>>(m, n, U, ldu, V, ldv, abf, abe, p, q);
  SVDUP_COUNT_LAUNCH();
}

// 2x2 Schur form of [[g, 1], [1, 0]] (Alg. 6.1 STEPs 2-3): eigenvalues r1 >= r2 with
// r1 r2 = -1 (the determinant), so the smaller-magnitude one is -1/(larger) and no
// cancellation occurs; eigenvector k is (r_k, 1) / sqrt(r_k^2 + 1).
__device__ void schur2(double g, double* r1, double* r2, double* q11, double* q21, double* q12,
                       double* q22) {
  double s = sqrt(g * g + 4.0);
  double a, b;
  if (g >= 0.0) { a = 0.5 * (g + s); b = -1.0 / a; }
  else { b = 0.5 * (g - s); a = -1.0 / b; }
  double na = sqrt(a * a + 1.0), nb = sqrt(b * b + 1.0);
  *r1 = a; *r2 = b;
  *q11 = a / na; *q21 = 1.0 / na;
  *q12 = b / nb; *q22 = 1.0 / nb;
}

// Left problem (STEPs 2, 4): poles D = S^2 in ascending order (sorted position s is
// physical column m-1-s since S is descending); z1 = Q11 p + Q21 (S .* q[:m]) and the
// second direction z2' = Q12 p + Q22 (S .* q[:m]) (kept in physical order).
// rho1 = r1 >= 0 goes first (the intermediate problem stays positive semidefinite);
// rho2 = r2 < 0 is stored for the second solve.
__global__ void k_fill_left(Eig e, int m, const double* __restrict__ S, const double* __restrict__ p,
                            const double* __restrict__ q, const double* __restrict__ ab,
                            double* z2p, double* rho2, int* status) {
  double r1, r2, q11, q21, q12, q22;
  schur2(ab[1], &r1, &r2, &q11, &q21, &q12, &q22);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    e.rhop[0] = r1;
    rho2[0] = r2;
    if (!isfinite(ab[0]) || !isfinite(ab[1])) latch(status, SVDUP_ENONFINITE);
  }
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m; s += gridDim.x * blockDim.x) {
    int c = m - 1 - s;
    double sc = S[c];
    if (c + 1 < m && S[c + 1] > sc) latch(status, SVDUP_EORDER);
    double sq = sc * q[c];
    double z1 = q11 * p[c] + q21 * sq;
    double z2 = q12 * p[c] + q22 * sq;
    if (!isfinite(z1) || !isfinite(z2) || !isfinite(sc)) latch(status, SVDUP_ENONFINITE);
    e.ds[s] = sc * sc;
    e.zs[s] = z1;
    e.perm[s] = c;
    z2p[c] = z2;
  }
}

void launch_fill_left(cudaStream_t st, Eig e, int m, const double* S, const double* p,
                      const double* q, const double* ab, double* z2p, double* rho2, int* status) {
  int blocks = (m + 255) / 256;
  k_fill_left<<<blocks, 256, 0, st>>>(e, m, S, p, q, ab, z2p, rho2, status);
  SVDUP_COUNT_LAUNCH();
}

// Right problem (STEPs 3, 6): D_v = S^T S = diag(S^2, 0_{n-m}) (App. A).  Sorted order:
// the n-m zero poles first (physical columns m..n-1), then S^2 ascending.
// z3 = Q11 q + Q21 [S .* p; 0] and z4' = Q12 q + Q22 [S .* p; 0] with Q from
// [[alpha, 1], [1, 0]].
__global__ void k_fill_right(Eig e, int m, int n, const double* __restrict__ S,
                             const double* __restrict__ p, const double* __restrict__ q,
                             const double* __restrict__ ab, double* z4p, double* rho4,
                             int* status) {
  double r1, r2, q11, q21, q12, q22;
  schur2(ab[0], &r1, &r2, &q11, &q21, &q12, &q22);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    e.rhop[0] = r1;
    rho4[0] = r2;
  }
  int nm = n - m;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    int c;
    double sc, sp;
    if (s < nm) { c = m + s; sc = 0.0; sp = 0.0; }
    else { c = m - 1 - (s - nm); sc = S[c]; sp = sc * p[c]; }
    double z3 = q11 * q[c] + q21 * sp;
    double z4 = q12 * q[c] + q22 * sp;
    if (!isfinite(z3) || !isfinite(z4)) latch(status, SVDUP_ENONFINITE);
    e.ds[s] = sc * sc;
    e.zs[s] = z3;
    e.perm[s] = c;
    z4p[c] = z4;
  }
}

void launch_fill_right(cudaStream_t st, Eig e, int m, int n, const double* S, const double* p,
                       const double* q, const double* ab, double* z4p, double* rho4, int* status) {
  int blocks = (n + 255) / 256;
  k_fill_right<<<blocks, 256, 0, st>>>(e, m, n, S, p, q, ab, z4p, rho4, status);
  SVDUP_COUNT_LAUNCH();
}

// Second solve of a side (STEPs 5, 7): the poles are the first solve's eigenvalues
// (already ascending, physical column = final index of the first solve).
__global__ void k_fill_second(Eig e, const double* __restrict__ lam_prev,
                              const double* __restrict__ zsec) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < e.N; s += gridDim.x * blockDim.x) {
    e.ds[s] = lam_prev[s];
    e.zs[s] = zsec[s];
    e.perm[s] = s;
  }
}

void launch_fill_second(cudaStream_t st, Eig e, const double* lam_prev, const double* zsec) {
  k_fill_second<<<(e.N + 255) / 256, 256, 0, st>>>(e, lam_prev, zsec);
  SVDUP_COUNT_LAUNCH();
}

// Arbitrary pole order (the stand-alone eigen-update entry point): the sorted position
// of pole i is its rank under (d_i, i), found by counting.
__global__ void k_fill_generic(Eig e, const double* __restrict__ d, const double* __restrict__ z,
                               const double* rho, int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) e.rhop[0] = rho[0];
  if (i >= e.N) return;
  double di = d[i];
  if (!isfinite(di) || !isfinite(z[i])) latch(status, SVDUP_ENONFINITE);
  int r = 0;
  for (int j = 0; j < e.N; j++) {
    double dj = d[j];
    r += (dj < di) || (dj == di && j < i);
  }
  e.ds[r] = di;
  e.zs[r] = z[i];
  e.perm[r] = i;
}

void launch_fill_generic(cudaStream_t st, Eig e, const double* d, const double* z,
                         const double* rho, int* status) {
  k_fill_generic<<<(e.N + 255) / 256, 256, 0, st>>>(e, d, z, rho, status);
  SVDUP_COUNT_LAUNCH();
}

// ---------------------------------------------------------------------------
// Deflation (Sec. 3.1; Bunch, Nielsen and Sorensen):
//  case (1) a negligible coupling |rho| ||z|| |z_s| <= tol removes pole s (its
//           eigenpair is (d_s, e_s));
//  case (3) two (numerically) equal poles: a Givens rotation in the plane of the
//           previous kept pole j and pole s moves all of z's weight onto s; j is
//           removed when the dropped coupling |(d_s - d_j) c s| <= tol.
//  (The paper's case (2), |abar| = 1, is the special case of (1) where z is a unit
//  coordinate vector.)  tol = 8 u max(max|d|, |rho| ||z||^2).
// Case (3) runs on consecutive survivors of case (1) (i-1, i): a rotation merges
// survivor i-1 into i, and the next pair (i, i+1) sees the merged values.  Along a run
// of merges starting at i0 the carrier after i holds
//     z~_i^2 = sum_{t=i0..i} z_t^2   and   d~_i = sum z_t^2 d_t / z~_i^2
// (each Givens step is a z^2-weighted mean), so the sequential test reduces to
//     |d_i - d~_{i-1}| |z_i| z~_{i-1} <= tol (z~_{i-1}^2 + z_i^2).
// Five launches.  An FP64 instruction costs as much as about 60 FP32 ones on this GPU,
// so per-pole FP64 work runs on many SMs and the single-block steps do integer work:
//  pre   (one block)  reductions, tol, case (1), the survivors' positions;
//  bits  (many)       scaled survivors and the candidate bitmask: the pairs that pass
//                     with the original values, the only places a run can start;
//  walk  (many)       the run boundaries: warp w walks the chains (maximal sequences
//                     of candidate pairs) whose first pair lies in its range of
//                     survivors, in order, as the sequential walk does;
//  fix   (one block)  a run that the previous range's walk carried into a range's
//                     first chain is resumed there, until the resumed walk starts a
//                     run where the range's own walk started one; then the rotation
//                     and kept indices and the compaction;
//  rec   (many)       the rotation records and merged values, from segmented sums of
//                     z^2 and z^2 d over the runs.
// The run boundaries are those of the sequential walk (in this arithmetic); only the
// rounding of the merged values differs from applying the rotations one at a time.
// ---------------------------------------------------------------------------
constexpr int kDeflateThreads = 1024;
constexpr int kDeflRecThreads = 256;
constexpr int kDeflRange = 128;  // survivors per walking warp (at least; see defl_range)

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  return v;
}

// The merge test of survivor i against the carrier (W = z~^2, M = W d~) of the run
// through i - 1, squared so that it needs no division or root:
//   (d_i W - M)^2 z_i^2 <= tol^2 W (W + z_i^2)^2   <=>   |d_i - d~| |z_i| z~ <= tol (z~^2 + z_i^2).
// It is homogeneous in d (with tol) and in z; the caller scales both by powers of two.
__device__ __forceinline__ bool merges(double di, double zi, double W, double M, double tol2) {
  const double zi2 = zi * zi;
  const double g = fma(di, W, -M);
  const double s = W + zi2;
  return g * g * zi2 <= tol2 * W * s * s;
}

// The sequential walk over the survivors (scaled d and z, the candidate bitmask, the
// run-start flags); every member is warp-collective.
struct DeflWalk {
  const double* kd;
  const double* kz;
  const unsigned* cm;   // bit i: pair (i-1, i) passes with the original values
  unsigned char* brk;   // 1: survivor i starts a run
  int nk;
  double itol;          // 1 / tol (tol in the scaled units of kd)

  // first i >= from with bit i set (nk if none)
  __device__ int next_set(int from, int lane) const {
    const int nw = (nk + 31) >> 5;
    for (int w0 = from >> 5; w0 < nw && from < nk; w0 += 32) {
      const int w = w0 + lane;
      unsigned m = 0u;
      if (w < nw) {
        m = cm[w];
        if (w == (from >> 5)) m &= 0xffffffffu << (from & 31);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, m != 0u);
      if (bal) {
        const int src = __ffs(bal) - 1;
        const unsigned mm = __shfl_sync(0xffffffffu, m, src);
        return min(nk, ((w0 + src) << 5) + __ffs(mm) - 1);
      }
    }
    return nk;
  }
  // first chain head h >= from (bit h set, bit h - 1 clear); nk if none
  __device__ int first_head(int from, int lane) const {
    const int nw = (nk + 31) >> 5;
    for (int w0 = from >> 5; w0 < nw && from < nk; w0 += 32) {
      const int w = w0 + lane;
      unsigned hm = 0u;
      if (w < nw) {
        const unsigned m = cm[w];
        const unsigned prev = w > 0 ? cm[w - 1] : 0u;
        hm = m & ~((m << 1) | (prev >> 31));
        if (w == (from >> 5)) hm &= 0xffffffffu << (from & 31);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, hm != 0u);
      if (bal) {
        const int src = __ffs(bal) - 1;
        const unsigned mm = __shfl_sync(0xffffffffu, hm, src);
        return min(nk, ((w0 + src) << 5) + __ffs(mm) - 1);
      }
    }
    return nk;
  }
  // resumed walk: the first q in [a, b) whose flag is set (b if none); flags a .. that q
  // (or b - 1) are set, since those survivors now start runs of one
  __device__ int restart_span(int a, int b, int lane) const {
    for (int x0 = a; x0 < b; x0 += 32) {
      const int x = x0 + lane;
      const bool was = x < b && brk[x] != 0;
      const unsigned bal = __ballot_sync(0xffffffffu, was);
      const int q = bal ? x0 + __ffs(bal) - 1 : b;
      if (x < b && x < q) brk[x] = 1;
      if (bal) return q;
    }
    return b;
  }

  // The merge test in the units of a run, on FP32 pairs (svdup_df.cuh): d is measured
  // from the run's first pole (ref) in multiples of tol, dh_i = (d_i - ref) / tol (one
  // FP64 subtraction, exact for close poles, and one product), W = sum z^2 and
  // M = sum z^2 dh over the run so far; survivor i merges when
  //   (dh_i W - M)^2 z_i^2 <= W (W + z_i^2)^2        (merges(), with tol = 1).
  // Both sides are homogeneous of degree 6 in z, so W, M and z_i^2 are first scaled by
  // the power of two that brings W + z_i^2 into [1, 2).  Then nothing overflows
  // (|dh| < 2^52), and the right side stays above 2^-90 unless the carrier is that much
  // lighter than z_i^2; there the test is taken in FP64.  The measured differences
  // stay small along a run, so the pairs' 2^-46 leave the decisions those of exact
  // arithmetic but for margins below about 2^-40.
  __device__ bool merge_df(Df W, Df M, Df z2, Df dh, double dhd) const {
    const Df s = df_add(W, z2);
    const float sc = pow2f(127 - ((__float_as_int(s.hi) >> 23) & 0xff));
    const Df Ws = {W.hi * sc, W.lo * sc}, Ms = {M.hi * sc, M.lo * sc};
    const Df z2s = {z2.hi * sc, z2.lo * sc}, ss = {s.hi * sc, s.lo * sc};
    const Df g = df_add(df_mul(dh, Ws), df_neg(Ms));
    const Df lhs = df_mul(df_sqr(g), z2s);
    const Df rhs = df_mul(Ws, df_sqr(ss));
    if (!(rhs.hi >= 0x1p-90f)) {
      const double Wd = df_to_f64(W, 0), Md = df_to_f64(M, 0), z2d = df_to_f64(z2, 0);
      const double gd = fma(dhd, Wd, -Md), sd = Wd + z2d;
      return gd * gd * z2d <= Wd * sd * sd;
    }
    return df_add(rhs, df_neg(lhs)).hi >= 0.0f;
  }

  // The sequential rule from survivor pos (pos <= lim): a run in progress merges survivor
  // i when the test passes against its carrier, else i starts a new run; a run of one
  // at i - 1 can grow only where bit i is set (and the test passes), so stretches without
  // bits are skipped.  The carrier of the run through pos - 1 is (W, M) with first pole
  // ref, or with fresh the run is survivor pos - 1 alone.  A run of one at p has the
  // carrier (z_p^2, 0) and ref = d_p whichever way the walk reaches it, so the rule is a
  // function of the state alone.
  // One step tests a window of 32 survivors (pos's aligned window): lane l against the
  // carrier that exists if every earlier lane merged (the carrier plus the lanes'
  // exclusive prefix sums of z^2 and z^2 dh), which is the sequential carrier up to the
  // first lane that fails; a failing lane starts a run, and the rest of the window is
  // tested again from it without reloading.
  // Plain walk (RESUME false): stops at survivor lim; returns lim + 1 when the run merged
  // lim (its carrier in oW, oM, oref: it continues into the next range), else -1.
  // RESUME: lim = nk - 1; flags are rewritten, and the walk stops at the first survivor
  // where it starts a run whose flag was already set (there it agrees with the plain
  // walk that wrote the flags); returns that survivor, or nk.
  template <bool RESUME>
  __device__ int walk(int pos, bool fresh, Df W, Df M, double ref, int lim, int lane, Df& oW,
                      Df& oM, double& oref) const {
    // the next two windows load while this one is tested (a long run takes them in turn)
    int pw1 = -1, pw2 = -1;
    double pz1 = 0.0, pd1 = 0.0, pz2 = 0.0, pd2 = 0.0;
    unsigned pword1 = 0u, pword2 = 0u;
    const Df zero = {0.0f, 0.0f};
    while (true) {
      const int w0 = pos & ~31;
      double zi, di;
      unsigned word;
      if (pw1 == w0) {
        zi = pz1;
        di = pd1;
        word = pword1;
        pw1 = pw2;
        pz1 = pz2;
        pd1 = pd2;
        pword1 = pword2;
      } else {
        const int i = w0 + lane;
        zi = i < nk ? kz[i] : 0.0;
        di = i < nk ? kd[i] : 0.0;
        word = cm[w0 >> 5];
        pw1 = w0 + 32;
        if (pw1 < nk) {
          const int j = pw1 + lane;
          pz1 = j < nk ? kz[j] : 0.0;
          pd1 = j < nk ? kd[j] : 0.0;
          pword1 = cm[pw1 >> 5];
        }
      }
      pw2 = w0 + 64;
      if (pw2 < nk) {
        const int j = pw2 + lane;
        pz2 = j < nk ? kz[j] : 0.0;
        pd2 = j < nk ? kd[j] : 0.0;
        pword2 = cm[pw2 >> 5];
      }
      const Df z2 = df_sqr(df_from_f64(zi, 0));
      int start = pos - w0;  // lanes >= start are tested
      int src = start;       // lanes >= src are in the run, after the carrier (Wb, Mb)
      Df Wb = W, Mb = M;
      if (fresh) {  // the run is survivor pos - 1 alone, which lies in this window
        src = start - 1;
        ref = __shfl_sync(0xffffffffu, di, src);
        Wb = zero;
        Mb = zero;
      }
      double dhd = (di - ref) * itol;
      Df dh = df_from_f64(dhd, 0);
      Df dz = df_mul(z2, dh);
      const int last = min(31, lim - w0);
      while (true) {
        Df v2 = lane >= src ? z2 : zero, vd = lane >= src ? dz : zero;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const Df a2 = {__shfl_up_sync(0xffffffffu, v2.hi, o), __shfl_up_sync(0xffffffffu, v2.lo, o)};
          const Df ad = {__shfl_up_sync(0xffffffffu, vd.hi, o), __shfl_up_sync(0xffffffffu, vd.lo, o)};
          if (lane >= o) {
            v2 = df_add(v2, a2);
            vd = df_add(vd, ad);
          }
        }
        Df e2 = {__shfl_up_sync(0xffffffffu, v2.hi, 1), __shfl_up_sync(0xffffffffu, v2.lo, 1)};
        Df ed = {__shfl_up_sync(0xffffffffu, vd.hi, 1), __shfl_up_sync(0xffffffffu, vd.lo, 1)};
        if (lane == 0) { e2 = zero; ed = zero; }
        const bool act = lane >= start && lane <= last;
        const bool ok = act && merge_df(df_add(Wb, e2), df_add(Mb, ed), z2, dh, dhd);
        const unsigned fail = __ballot_sync(0xffffffffu, act && !ok);
        const int f = fail ? __ffs(fail) - 1 : last + 1;
        if (lane >= start && lane < f) brk[w0 + lane] = 0;
        if (!fail) {  // every tested lane merged
          const Df Wn = df_add(Wb, Df{__shfl_sync(0xffffffffu, v2.hi, last),
                                      __shfl_sync(0xffffffffu, v2.lo, last)});
          const Df Mn = df_add(Mb, Df{__shfl_sync(0xffffffffu, vd.hi, last),
                                      __shfl_sync(0xffffffffu, vd.lo, last)});
          if (w0 + last >= lim) {
            if (RESUME) return nk;
            oW = Wn;
            oM = Mn;
            oref = ref;
            return lim + 1 < nk ? lim + 1 : -1;
          }
          W = Wn;
          M = Mn;
          fresh = false;
          pos = w0 + 32;
          break;
        }
        const int p = w0 + f;  // survivor p starts a run
        if (RESUME) {
          if (brk[p]) return p;
          __syncwarp();
          if (lane == 0) brk[p] = 1;
        }
        if (p >= lim) return RESUME ? nk : -1;
        const unsigned above = f < 31 ? (word >> (f + 1)) : 0u;
        const int h = above ? p + __ffs(above) : next_set(w0 + 32, lane);  // the next bit
        if (RESUME && h > p + 1) {
          const int q = restart_span(p + 1, h, lane);
          if (q < h) return q;
        }
        if (h > lim) return RESUME ? nk : -1;
        if (h < w0 + 32) {  // a run of one at h - 1 in this window: measure from it
          src = h - 1 - w0;
          start = h - w0;
          Wb = zero;
          Mb = zero;
          ref = __shfl_sync(0xffffffffu, di, src);
          dhd = (di - ref) * itol;
          dh = df_from_f64(dhd, 0);
          dz = df_mul(z2, dh);
          continue;
        }
        pos = h;
        M = zero;
        if (h & 31) {
          fresh = true;
        } else if (h == w0 + 32) {  // survivor h - 1 is this window's last lane
          fresh = false;
          W = Df{__shfl_sync(0xffffffffu, z2.hi, 31), __shfl_sync(0xffffffffu, z2.lo, 31)};
          ref = __shfl_sync(0xffffffffu, di, 31);
        } else {
          fresh = false;
          W = df_sqr(df_from_f64(kz[h - 1], 0));
          ref = kd[h - 1];
        }
        break;
      }
    }
  }
};

// Deflation, part 1 (one block): tolerance and scalings, case (1), the survivors' sorted
// positions in order.
__global__ void __launch_bounds__(kDeflateThreads) k_deflate_pre(Eig e, int* status) {
  __shared__ double sred[32];
  __shared__ unsigned long long sdm[32], szm[32];
  __shared__ int swc[32];
  __shared__ double s_tol, s_zn;
  const int N = e.N;
  const double rho = e.rhop[0];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  double zn2 = 0.0;
  unsigned long long dm = 0ull, zm = 0ull;  // max |d|, max |z| by their bit patterns
  for (int s = tid; s < N; s += nt) {
    const double z = e.zs[s];
    zn2 = fma(z, z, zn2);
    dm = max(dm, abs_bits(e.ds[s]));
    zm = max(zm, abs_bits(z));
  }
  zn2 = warp_sum(zn2);
  dm = warp_max_u64(dm);
  zm = warp_max_u64(zm);
  if (lane == 0) { sred[wid] = zn2; sdm[wid] = dm; szm[wid] = zm; }
  __syncthreads();
  if (wid == 0) {
    const int nw = nt >> 5;
    zn2 = lane < nw ? sred[lane] : 0.0;
    dm = lane < nw ? sdm[lane] : 0ull;
    zm = lane < nw ? szm[lane] : 0ull;
    zn2 = warp_sum(zn2);
    dm = warp_max_u64(dm);
    zm = warp_max_u64(zm);
    if (lane == 0) {
      const double dmax = __longlong_as_double((long long)dm);
      const double zmax = __longlong_as_double((long long)zm);
      const double t = fabs(rho) * zn2;
      s_tol = 8.0 * kU * fmax(dmax, t);
      s_zn = sqrt(zn2);
      // exact power-of-two scalings that bring max|d| and max|z| near 1 for the merge test
      const double dsc = (dmax > 0.0 && isfinite(dmax)) ? ldexp(1.0, -ilogb(dmax)) : 1.0;
      const double zsc = (zmax > 0.0 && isfinite(zmax)) ? ldexp(1.0, -ilogb(zmax)) : 1.0;
      const double tolS = s_tol * dsc;
      e.tol[0] = s_tol;
      e.dflt[0] = tolS * tolS;
      e.dflt[1] = dsc;
      e.dflt[2] = zsc;
      e.dflt[3] = tolS > 0.0 ? 1.0 / tolS : 0.0;
      if (!isfinite(s_tol) || !isfinite(rho)) latch(status, SVDUP_ENONFINITE);
    }
  }
  __syncthreads();
  const double tol = s_tol;
  const double c1 = fabs(rho) * s_zn;
  int base = 0;
  for (int s0 = 0; s0 < N; s0 += nt) {
    const int s = s0 + tid;
    bool surv = false;
    if (s < N) {
      const int d1 = (rho == 0.0 || c1 * fabs(e.zs[s]) <= tol) ? 1 : 0;
      e.defl[s] = d1;
      surv = !d1;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, surv);
    if (lane == 0) swc[wid] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < (nt >> 5); w++) {
      const int c = swc[w];
      off += w < wid ? c : 0;
      tot += c;
    }
    if (surv) e.spos[base + off + __popc(bal & ((1u << lane) - 1u))] = s;
    base += tot;
    __syncthreads();
  }
  if (tid == 0) e.dint[0] = base;
}

// Deflation, part 2 (a thread per survivor): scaled d and z, run flags, candidate bits.
__global__ void k_deflate_bits(Eig e) {
  const int nk = e.dint[0];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nwords = (nk + 31) >> 5;
  if ((i >> 5) > nwords) return;  // warp-uniform
  const double tol2 = e.dflt[0], dsc = e.dflt[1], zsc = e.dflt[2];
  bool ok = false;
  if (i < nk) {
    const int s = e.spos[i];
    const double di = e.ds[s] * dsc, zi = e.zs[s] * zsc;
    e.sd[i] = di;
    e.sz[i] = zi;
    e.sbrk[i] = 1;
    if (i > 0) {
      const int sp = e.spos[i - 1];
      const double dj = e.ds[sp] * dsc, zj = e.zs[sp] * zsc;
      const double W = zj * zj;
      ok = merges(di, zi, W, W * dj, tol2);
    }
  }
  const unsigned bal = __ballot_sync(0xffffffffu, ok);
  if ((threadIdx.x & 31) == 0) e.dmask[i >> 5] = bal;
}

// Deflation, part 3 (a warp per range of R survivors): the chains whose first pair lies
// in the range, walked in order from a run of one at the first chain's first survivor,
// up to the pole before the next range's first chain.  A run that merged that pole is
// listed (slot = the range) with its carrier.
__global__ void __launch_bounds__(32) k_deflate_walk(Eig e, int R) {
  const int nk = e.dint[0];
  const int lane = threadIdx.x;
  const int slot = blockIdx.x;
  const int r0 = slot * R;
  int ov = -1;
  Df oW = {0.0f, 0.0f}, oM = {0.0f, 0.0f};
  double oref = 0.0;
  if (r0 < nk) {
    const DeflWalk dw = {e.sd, e.sz, e.dmask, e.sbrk, nk, e.dflt[3]};
    const int r1 = min(nk, r0 + R);
    const int h0 = dw.first_head(r0, lane);
    if (h0 < r1) {
      const int H = dw.first_head(r1, lane);
      Df W = {0.0f, 0.0f};
      double ref = 0.0;
      bool fresh = (h0 & 31) != 0;
      if (!fresh) {  // a run of one at h0 - 1, in the previous window
        W = df_sqr(df_from_f64(e.sz[h0 - 1], 0));
        ref = e.sd[h0 - 1];
      }
      ov = dw.walk<false>(h0, fresh, W, Df{0.0f, 0.0f}, ref, H - 1, lane, oW, oM, oref);
    }
  }
  if (lane == 0) {
    e.ovh[slot] = ov;
    e.ovW[slot] = make_float2(oW.hi, oW.lo);
    e.ovM[slot] = make_float2(oM.hi, oM.lo);
    e.ovR[slot] = oref;
  }
}

// Deflation, part 4 (one block): the listed runs resumed in order (one warp); then the
// rotation index of every merge, the kept index of every run end, each survivor's run
// start, the final flags and the kept and deflated position lists.
__global__ void __launch_bounds__(kDeflateThreads) k_deflate_fix(Eig e, int nslots) {
  __shared__ int sov[kMaxOverrunList];
  __shared__ int sc_m[32], sc_e[32], sc_r[32];
  const int N = e.N;
  const int nk = e.dint[0];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  unsigned char* brk = e.sbrk;
  for (int s = tid; s < nslots; s += nt) sov[s] = e.ovh[s];
  __syncthreads();
  if (wid == 0) {
    const DeflWalk dw = {e.sd, e.sz, e.dmask, brk, nk, e.dflt[3]};
    int done = -1;
    for (int s = 0; s < nslots; s++) {
      const int H = sov[s];
      if (H < 0 || H <= done) continue;  // none, or redone by an earlier resume
      Df oW, oM;
      double oref;
      const float2 w = e.ovW[s], mm = e.ovM[s];
      done = dw.walk<true>(H, false, Df{w.x, w.y}, Df{mm.x, mm.y}, e.ovR[s], nk - 1, lane, oW, oM,
                           oref);
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  int base_m = 0, base_e = 0, carry_r = 0;
  for (int i0 = 0; i0 < nk; i0 += nt) {
    const int i = i0 + tid;
    const bool in = i < nk;
    const bool b = in ? brk[i] != 0 : true;
    const bool m = in && !b;
    const bool en = in && (i + 1 >= nk || brk[i + 1] != 0);
    int rs = (in && b) ? i : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, rs, o);
      if (lane >= o) rs = max(rs, t);
    }
    const unsigned bm = __ballot_sync(0xffffffffu, m), be = __ballot_sync(0xffffffffu, en);
    if (lane == 31) { sc_m[wid] = __popc(bm); sc_e[wid] = __popc(be); sc_r[wid] = rs; }
    __syncthreads();
    int om = base_m, oe = base_e, orr = carry_r, tm = 0, te = 0, tr = carry_r;
    for (int w = 0; w < (nt >> 5); w++) {
      const int cm_ = sc_m[w], ce = sc_e[w], cr = sc_r[w];
      if (w < wid) { om += cm_; oe += ce; orr = max(orr, cr); }
      tm += cm_;
      te += ce;
      tr = max(tr, cr);
    }
    if (in) {
      const int ps = e.spos[i];
      e.srs[i] = max(orr, rs);
      if (m) e.srix[i] = om + __popc(bm & lt);
      if (en) {
        const int kx = oe + __popc(be & lt);
        e.skix[i] = kx;
        e.idx[kx] = ps;
      }
      e.defl[ps] = en ? 0 : 2;  // 2: deflated by a rotation (the rotation kernel writes its column)
    }
    base_m += tm;
    base_e += te;
    carry_r = tr;
    __syncthreads();
  }
  int base_d = 0;
  for (int s0 = 0; s0 < N; s0 += nt) {
    const int s = s0 + tid;
    const bool dd = s < N && e.defl[s] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, dd);
    if (lane == 0) sc_m[wid] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < (nt >> 5); w++) {
      const int c = sc_m[w];
      off += w < wid ? c : 0;
      tot += c;
    }
    if (dd) e.didx[base_d + off + __popc(bal & lt)] = s;
    base_d += tot;
    __syncthreads();
  }
  if (tid == 0) {
    e.kp[0] = base_e;
    e.nrot[0] = base_m;
  }
}

// Deflation, part 5 (a thread per survivor): the carrier before each survivor from a
// segmented scan of (z^2, z^2 d) over the block plus the sum over the part of its run
// before the block; rotation records (position pair, cos, sin), rotated values, merged
// run ends, the kept set and its rho > 0 orientation for the solver (d -> -d, reversed,
// when rho < 0).
__global__ void __launch_bounds__(kDeflRecThreads) k_deflate_rec(Eig e) {
  __shared__ double sW[kDeflRecThreads], sM[kDeflRecThreads];
  __shared__ int sF[kDeflRecThreads];
  __shared__ double rW[kDeflRecThreads / 32], rM[kDeflRecThreads / 32];
  const int nk = e.dint[0];
  const int i0 = blockIdx.x * blockDim.x;
  if (i0 >= nk) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nt = blockDim.x;
  const int i = i0 + tid;
  const bool in = i < nk;
  const double rho = e.rhop[0], dsc = e.dflt[1], zsc = e.dflt[2];
  const double idsc = 1.0 / dsc, izsc = 1.0 / zsc;  // exact: powers of two
  // the run entering the block: survivors rs .. i0 - 1
  const int rs = e.srs[i0];
  double cW = 0.0, cM = 0.0;
  if (rs < i0) {
    for (int t = rs + tid; t < i0; t += nt) {
      const double z = e.sz[t], z2 = z * z;
      cW += z2;
      cM = fma(z2, e.sd[t], cM);
    }
    cW = warp_sum(cW);
    cM = warp_sum(cM);
    if (lane == 0) { rW[wid] = cW; rM[wid] = cM; }
    __syncthreads();
    cW = 0.0;
    cM = 0.0;
    for (int w = 0; w < (nt >> 5); w++) { cW += rW[w]; cM += rM[w]; }
  }
  const double zi = in ? e.sz[i] : 0.0, di = in ? e.sd[i] : 0.0;
  const bool b = in ? e.sbrk[i] != 0 : true;
  const double z2 = zi * zi;
  // inclusive segmented scan over the block (flag: a run starts at or after the element)
  double w = z2, m = z2 * di;
  int f = b ? 1 : 0;
  sW[tid] = w;
  sM[tid] = m;
  sF[tid] = f;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    double w2 = 0.0, m2 = 0.0;
    int f2 = 0;
    if (tid >= off) { w2 = sW[tid - off]; m2 = sM[tid - off]; f2 = sF[tid - off]; }
    __syncthreads();
    if (tid >= off && !f) { w += w2; m += m2; f = f2; }
    sW[tid] = w;
    sM[tid] = m;
    sF[tid] = f;
    __syncthreads();
  }
  if (!f) { w += cW; m += cM; }  // the run began before the block
  // the carrier through i - 1
  double Wp = cW, Mp = cM;
  if (tid > 0) {
    Wp = sW[tid - 1];
    Mp = sM[tid - 1];
    if (!sF[tid - 1]) { Wp += cW; Mp += cM; }
  }
  if (!in) return;
  if (!b) {  // rotation merging survivor i - 1 (the carrier) into i
    const double zprev = e.sbrk[i - 1] ? e.sz[i - 1] : Wp * rsqrt64(Wp);  // signed at a run start
    const double Wn = Wp + z2;
    const double irn = rsqrt64(Wn);
    const double cs = zi * irn, sn = zprev * irn;
    const double dprev = Mp * rcp64(Wp);
    const int pj = e.spos[i - 1], pi = e.spos[i];
    e.ds[pj] = (cs * cs * dprev + sn * sn * di) * idsc;
    e.zs[pj] = 0.0;
    const int r = e.srix[i];
    e.rj[r] = pj;
    e.ri[r] = pi;
    e.rc[r] = cs;
    e.rs[r] = sn;
  }
  if (i + 1 >= nk || e.sbrk[i + 1]) {  // a run end: kept
    const int ps = e.spos[i];
    double dv, zv;
    if (!b) {
      dv = (m * rcp64(w)) * idsc;
      zv = (w * rsqrt64(w)) * izsc;
    } else {
      dv = di * idsc;
      zv = zi * izsc;
    }
    e.ds[ps] = dv;
    e.zs[ps] = zv;
    const int kx = e.skix[i];
    e.dk[kx] = dv;
    e.zk[kx] = zv;
    const int kk = e.kp[0];
    const int t = rho > 0.0 ? kx : kk - 1 - kx;
    e.dc[t] = rho > 0.0 ? dv : -dv;
    e.z2c[t] = zv * zv;
  }
}

// survivors per walking warp: at least kDeflRange, and few enough ranges for the slots
static int defl_range(int N) {
  int R = kDeflRange;
  while ((N + R - 1) / R > kMaxOverrunList) R *= 2;
  return R;
}

void launch_deflate(cudaStream_t st, Eig e, int* status) {
  const int N = e.N;
  k_deflate_pre<<<1, kDeflateThreads, 0, st>>>(e, status);
  SVDUP_COUNT_LAUNCH();
  k_deflate_bits<<<(N + 32 + 255) / 256, 256, 0, st>>>(e);
  SVDUP_COUNT_LAUNCH();
  const int R = defl_range(N);
  const int nslots = std::max(1, (N + R - 1) / R);
  k_deflate_walk<<<nslots, 32, 0, st>>>(e, R);
  SVDUP_COUNT_LAUNCH();
  k_deflate_fix<<<1, kDeflateThreads, 0, st>>>(e, nslots);
  SVDUP_COUNT_LAUNCH();
  k_deflate_rec<<<std::max(1, (N + kDeflRecThreads - 1) / kDeflRecThreads), kDeflRecThreads, 0, st>>>(e);
  SVDUP_COUNT_LAUNCH();
}

// ---------------------------------------------------------------------------
// Secular equation (Sec. 3.1, Eq. GolubEigenvalUpdate):
//   w(mu) = 1 + R sum_i z_i^2 / (d_i - mu),  R > 0, d strictly ascending.
// Root j lies in (d_j, d_{j+1}) (j < k-1) or in (d_{k-1}, d_{k-1} + R ||z||^2].
// One warp per root (two per warp in the far-field form, below); the lanes split the
// poles and reduce.  The root is held as
// mu = d_o + tau with o the nearer pole (decided by the sign of w at the bracket
// midpoint), so every difference d_i - mu = (d_i - d_o) - tau keeps full relative
// accuracy when the root sits next to a pole.
// Iteration: the rational model of Bunch, Nielsen and Sorensen (1978): the poles left
// of the root are modelled by P_L + Q_L / (d_left - mu), those right of it by
// P_R + Q_R / (d_right - mu), each matching value and slope at the current iterate;
// the model's root in the bracket is one quadratic.  The bracket is kept from the
// signs of w and a model step that leaves it is replaced by bisection.  The quadratic's
// square root and divisions go through rsqrt64 and rcp64 (a few FP64 operations each
// instead of correctly rounded sequences): a step needs no last-bit accuracy, and the
// convergence tests and the bracket decide the root.  Finiteness is tested on the bit
// fields.
// ---------------------------------------------------------------------------
struct SecSums {
  double psiL, dpsiL, psiR, dpsiR, asum;
};

__device__ __forceinline__ SecSums secular_sums(const double* __restrict__ dc,
                                                const double* __restrict__ z2c, int k, int o,
                                                double tau, int jsplit, int lane) {
  SecSums r = {0.0, 0.0, 0.0, 0.0, 0.0};
  const double dO = dc[o];
  for (int i = lane; i < k; i += 32) {
    double del = (dc[i] - dO) - tau;
    double rc = rcp64(del);
    double t = z2c[i] * rc;
    double dt = t * rc;
    if (i <= jsplit) { r.psiL += t; r.dpsiL += dt; }
    else { r.psiR += t; r.dpsiR += dt; }
  }
  r.psiL = warp_sum(r.psiL);
  r.dpsiL = warp_sum(r.dpsiL);
  r.psiR = warp_sum(r.psiR);
  r.dpsiR = warp_sum(r.dpsiR);
  r.asum = r.psiR - r.psiL;  // poles left of the root give negative terms, right positive
  return r;
}

struct DirectSums {
  const double* dc;
  const double* z2c;
  int k;
  static constexpr double wtol = kU;
  __device__ SecSums operator()(int o, double tau, int jsplit, int lane) const {
    return secular_sums(dc, z2c, k, o, tau, jsplit, lane);
  }
};

// ---------------------------------------------------------------------------
// Far-field evaluation of the secular sums (this contests the paper's remark in
// Sec. 3.1 that the FMM cannot serve the secular equation because the roots are
// unknown: the SOURCES, the poles with weights z_i^2, are fixed, so their far field
// is a fixed function of mu that can be sampled once).
// The roots j in [64 b, min(64 b + 64, k - 1)) all lie in box b = [d_{64b}, d_{j1}],
// j1 = min(64 b + 64, k - 1), of half width r and centre c.  Poles within 3 r of c,
// and those of leaves b-1..b+1, are the near field and are summed directly with the
// offsets, as in the direct sums.  The rest lie outside [c - 3r, c + 3r]; their four
// sums (psi and psi' of the poles left of the box, the same right of it) are analytic
// on the box and are interpolated on kSqP Chebyshev nodes of the first kind
// (App. D STEP 3) with the barycentric formula.  The interpolation error is below
// 10 * 5^-kSqP of the far terms' magnitude (a pole 3 r from the centre lies outside
// the Bernstein ellipse of parameter 5), under the FP64 rounding of the sums.
// Coordinates are measured from the pole d_{64b}, so every difference keeps relative
// accuracy however far the box sits from zero.  The last root (beyond every pole) is
// always summed directly.
// ---------------------------------------------------------------------------
constexpr int kSqLeaf = 64;
constexpr int kSqP = 26;
constexpr int kSqMinK = 2048;  // smaller problems use the direct FP64 sums only

// Far-field form in FP32 pairs.  For k >= kSqMinK the FP64 evaluation of w itself carries
// a rounding bound of about k u (1 + R sum |t|) >= 2^-42 (1 + R sum |t|) (the attainable
// accuracy the secular tests use); the pair arithmetic (about 2^-44 per term, see
// svdup_df.cuh) stays inside it, so the far-field form sums in pairs and stops at
// |w| <= kSecTolPairs (1 + R sum |t|).  Each root's origin pole, whose offset can be
// arbitrarily small, is summed in FP64.  Poles and offsets are scaled by 2^-E, z^2 by 2^-Z
// (powers of two from k_sq_prep), which keeps every other term inside the FP32 range.
constexpr double kSecTolPairs = 0x1p-42;

// x 2^s for a pair, in FP64, applied in two halves (each inside the FP64 range).
__device__ __forceinline__ double pair_scaled(Df a, int s) { return df_to_f64_scaled(a, s); }

// z^2 / delta and z^2 / delta^2 in pairs for delta = dd - tau (dd = d_i - d_o exact in
// FP64; ntau = -tau 2^-E; z2 = z^2 2^-Z): results scaled by 2^(E - Z) and 2^(2E - Z).
__device__ __forceinline__ void pair_term(double dd, Df ntau, Df z2, int E, Df& t, Df& dt) {
  const Df r = df_rcp(df_add(df_from_f64(dd, E), ntau));
  t = df_mul(z2, r);
  dt = df_mul(t, r);
}

__device__ __forceinline__ int lower_bound_d(const double* a, int n, double v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Roots whose bracket is wider than the rest of their box -- the isolated largest
// poles, such as the large eigenvalues earlier updates have added, among the poles of
// a solve -- would stretch their box over the spectrum (and every pole into its near
// field).  From each end, while the end box of kSqLeaf roots has more than kSqNearPeel
// poles within two of its radii, its outermost root is taken out and solved alone by one
// warp with direct sums (at most kSqMaxWide per end; a chain of updates adds one such
// pole per update), as is the last root (beyond all poles).  The boxes of kSqLeaf roots
// cover roots first .. last; k_sq_boxes stores the layout in sqf.
constexpr int kSqMaxWide = 64;
constexpr int kSqNearPeel = 6 * kSqLeaf;

__device__ void sq_layout(const double* __restrict__ dc, int k, int* first, int* last) {
  int f = 0, l = k - 2;
  if (k >= kSqMinK) {
    // the box of roots a .. a + kSqLeaf - 1 spans [d_a, d_{a+kSqLeaf}]; it is too wide
    // when the poles within two radii of it are more than kSqNearPeel
    auto wide = [&](int a) {
      const double lo = dc[a], hi = dc[a + kSqLeaf], r = 0.5 * (hi - lo);
      return lower_bound_d(dc, k, hi + 2.0 * r) - lower_bound_d(dc, k, lo - 2.0 * r) > kSqNearPeel;
    };
    while (f < kSqMaxWide && f + 2 * kSqLeaf <= l && wide(f)) f++;
    while (k - 2 - l < kSqMaxWide && l - 2 * kSqLeaf >= f && wide(l + 1 - kSqLeaf)) l--;
  }
  *first = f;
  *last = l;
}

__device__ __forceinline__ int sq_boxes(int first, int last) {
  return (last - first + 1 + kSqLeaf - 1) / kSqLeaf;
}

// Boxes: sqb[2b] = d_{j0} (the coordinate origin, j0 = first + b kSqLeaf), sqb[2b+1] = r;
// sqn[2b], sqn[2b+1] = the near pole range [n0, n1): the box's roots lie in
// [d_{j0}, d_{j1}], every pole outside [n0, n1) is at least 2r beyond that interval, and
// the near range reaches at least one box width past each end.
__global__ void k_sq_boxes(const double* __restrict__ dc, const int* __restrict__ kp, double* sqb,
                           int* sqn, int* sqf) {
  const int k = kp[0];
  if (k < kSqMinK) return;
  int first, last;
  sq_layout(dc, k, &first, &last);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sqf[0] = first;
    sqf[1] = last;
    sqf[4] = 0;  // the solver's root counter
  }
  const int nb = sq_boxes(first, last);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    const int j0 = first + b * kSqLeaf, j1 = min(j0 + kSqLeaf, last + 1);
    const double lo = dc[j0], hi = dc[j1];
    const double r = 0.5 * (hi - lo);
    const int t_lo = lower_bound_d(dc, k, lo - 2.0 * r);     // first pole >= c - 3r
    const int t_hi = lower_bound_d(dc, k, hi + 2.0 * r);     // first pole >= c + 3r
    sqb[2 * b] = lo;
    sqb[2 * b + 1] = r;
    sqn[2 * b] = max(0, min(j0 - kSqLeaf, t_lo));
    sqn[2 * b + 1] = min(k, max(j1 + kSqLeaf, t_hi));
  }
}

// Far sums at the Chebyshev nodes of each box: sqv[(4 b + q) kSqP + beta] for q = psi_L,
// psi_L', psi_R, psi_R'.  One warp per (box, node).
// Scales of the pair form (one block): sqf[2] = E with |d|, |tau| < 2^E for every
// non-extreme root, sqf[3] = Z with z^2 <= 2^Z; z2f = z^2 2^-Z as pairs.
__global__ void __launch_bounds__(1024) k_sq_prep(const double* __restrict__ dc,
                                                  const double* __restrict__ z2c,
                                                  const int* __restrict__ kp, int* sqf,
                                                  float2* z2f) {
  __shared__ int sz;
  const int k = kp[0];
  if (k < kSqMinK) return;
  if (threadIdx.x == 0) sz = -1100;
  __syncthreads();
  int mz = -1100;
  for (int t = threadIdx.x; t < k; t += blockDim.x) mz = max(mz, exp2_of(z2c[t]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mz = max(mz, __shfl_xor_sync(0xffffffffu, mz, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&sz, mz);
  __syncthreads();
  const int Z = sz <= -1000 ? 0 : sz;
  // the roots' offsets stay within twice the pole range: one more bit
  const int E = max(exp2_of(dc[0]), exp2_of(dc[k - 1])) + 2;
  if (threadIdx.x == 0) {
    sqf[2] = E;
    sqf[3] = Z;
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    const Df v = df_from_f64(z2c[t], Z);
    z2f[t] = make_float2(v.hi, v.lo);
  }
}

// Far sums at the Chebyshev nodes of each box: sqv[(4 b + q) kSqP + beta] for q = psi_L,
// psi_L', psi_R', psi_R', in pairs (every pole is at least 2r from the node).  One warp
// per (box, node).
__global__ void k_sq_nodes(const double* __restrict__ dc, const float2* __restrict__ z2f,
                           const int* __restrict__ kp, const double* __restrict__ sqb,
                           const int* __restrict__ sqn, const int* __restrict__ sqf, double* sqv) {
  const int k = kp[0];
  if (k < kSqMinK) return;
  const int nb = sq_boxes(sqf[0], sqf[1]);
  const int E = sqf[2], Z = sqf[3];
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nb * kSqP; w += warps) {
    const int b = w / kSqP, beta = w - b * kSqP;
    const double base = sqb[2 * b], r = sqb[2 * b + 1];
    const int n0 = sqn[2 * b], n1 = sqn[2 * b + 1];
    const double yo = r * (1.0 + cospi((2.0 * beta + 1.0) / (2.0 * kSqP)));
    const Df nyo = df_neg(df_from_f64(yo, E));
    Df pL = {0.f, 0.f}, dL = {0.f, 0.f}, pR = {0.f, 0.f}, dR = {0.f, 0.f};
    for (int t = lane; t < n0; t += 32) {
      Df tt, dt;
      const float2 z = z2f[t];
      pair_term(dc[t] - base, nyo, Df{z.x, z.y}, E, tt, dt);
      pL = df_add(pL, tt);
      dL = df_add(dL, dt);
    }
    for (int t = n1 + lane; t < k; t += 32) {
      Df tt, dt;
      const float2 z = z2f[t];
      pair_term(dc[t] - base, nyo, Df{z.x, z.y}, E, tt, dt);
      pR = df_add(pR, tt);
      dR = df_add(dR, dt);
    }
    pL = df_warp_sum(pL);
    dL = df_warp_sum(dL);
    pR = df_warp_sum(pR);
    dR = df_warp_sum(dR);
    if (lane == 0) {
      double* v = sqv + (size_t)4 * b * kSqP;
      v[beta] = pair_scaled(pL, Z - E);
      v[kSqP + beta] = pair_scaled(dL, Z - 2 * E);
      v[2 * kSqP + beta] = pair_scaled(pR, Z - E);
      v[3 * kSqP + beta] = pair_scaled(dR, Z - 2 * E);
    }
  }
}

// ---------------------------------------------------------------------------
// Two roots per warp (far-field form).  A root's iteration is scalar FP64 arithmetic
// (the rational model, its quadratic, the bracket), the same for all lanes of the warp
// that iterates it; on GB300 an FP64 warp instruction costs the same whatever its active
// lanes, and this scalar work, not the sums, filled the FP64 pipe.  So each group of
// kSecG = 16 lanes iterates its own root: the scalar work is shared by two roots, and the
// sums of each root (its near poles and the far field's 26 nodes) are split over its
// lanes and reduced within the group (xor shuffles below kSecG stay inside it).  The
// steps are those of secular_root; the groups iterate in lockstep, a group that has
// converged keeps its result and idles until the other has.  (Four roots of 8 lanes
// halve the FP64 instructions again, but leave too few warps per SM to hide the
// dependent FP64 latency, and a warp waits for the slowest of four roots.)
// ---------------------------------------------------------------------------
constexpr int kSecG = 16;                           // lanes per root
constexpr int kSecRoots = 32 / kSecG;                // roots per warp
constexpr int kSecNQ = (kSqP + kSecG - 1) / kSecG;  // far-field nodes per lane

__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = kSecG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ Df group_df_sum(Df a) {
#pragma unroll
  for (int o = kSecG / 2; o > 0; o >>= 1) a = df_add(a, df_shfl_xor(a, o));
  return a;
}
__device__ __forceinline__ int group_max(int v) {
#pragma unroll
  for (int o = kSecG / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ bool group_any(bool p, int g) {
  return ((__ballot_sync(0xffffffffu, p) >> (kSecG * g)) & ((1ull << kSecG) - 1ull)) != 0u;
}
__device__ __forceinline__ bool warp_all(bool p) { return __all_sync(0xffffffffu, p); }

// One box's far-field data for the root of this lane's group.
struct FarBox {
  int n0, n1;
  double base, r;
  const double* vals;
};

struct FarSumsG {
  const double* dc;
  const double* z2c;
  const float2* z2f;
  const double* sx;
  const double* sw;
  int E, Z;
  // The far-field form's split sums for the group's root mu = d_o + tau in box fb (the
  // poles of the box's near range directly, the rest by barycentric interpolation of the
  // box's node values); every lane of the group returns them.  sub: this lane's index
  // in its group, g: the group.
  __device__ SecSums operator()(const FarBox& fb, int o, double tau, int jsplit, int sub,
                                int g) const {
    SecSums s = {0.0, 0.0, 0.0, 0.0, 0.0};
    const double dO = dc[o];
    const double* vals = fb.vals;
    const double yh = (((dO - fb.base) + tau) - fb.r) * rcp64(fb.r);
    bool big = false;
    for (int q = sub; q < kSqP; q += kSecG)
      big |= max(max(exp2_of(vals[q]), exp2_of(vals[kSqP + q])),
                 max(exp2_of(vals[2 * kSqP + q]), exp2_of(vals[3 * kSqP + q]))) > 120;
    const bool f64far = group_any(big, g);
    // barycentric weights of the nodes this lane holds (sub, sub + 8, ...)
    Df c[kSecNQ];
    int hq = -1;
#pragma unroll
    for (int qi = 0; qi < kSecNQ; qi++) {
      const int q = sub + kSecG * qi;
      c[qi] = Df{0.0f, 0.0f};
      if (q < kSqP) {
        const Df dfy = df_add(df_from_f64(yh, 0), df_neg(df_from_f64(sx[q], 0)));
        if (dfy.hi == 0.0f) hq = q;
        else c[qi] = df_mul(df_from_f64(sw[q], 0), df_rcp(dfy));
      }
    }
    const int hm = group_max(hq);
    if (hm >= 0) {  // mu sits exactly on a node
#pragma unroll
      for (int qi = 0; qi < kSecNQ; qi++)
        c[qi] = (sub + kSecG * qi == hm) ? Df{1.0f, 0.0f} : Df{0.0f, 0.0f};
    } else {
      Df cs = {0.0f, 0.0f};
#pragma unroll
      for (int qi = 0; qi < kSecNQ; qi++) cs = df_add(cs, c[qi]);
      const Df ic = df_rcp(group_df_sum(cs));
#pragma unroll
      for (int qi = 0; qi < kSecNQ; qi++) c[qi] = df_mul(c[qi], ic);
    }
    Df fL = {0.f, 0.f}, fdL = {0.f, 0.f}, fR = {0.f, 0.f}, fdR = {0.f, 0.f};
#pragma unroll
    for (int qi = 0; qi < kSecNQ; qi++) {
      const int q = sub + kSecG * qi;
      if (q < kSqP) {
        fL = df_add(fL, df_mul(c[qi], df_from_f64(vals[q], 0)));
        fdL = df_add(fdL, df_mul(c[qi], df_from_f64(vals[kSqP + q], 0)));
        fR = df_add(fR, df_mul(c[qi], df_from_f64(vals[2 * kSqP + q], 0)));
        fdR = df_add(fdR, df_mul(c[qi], df_from_f64(vals[3 * kSqP + q], 0)));
      }
    }
    // near poles in pairs, the origin pole (offset -tau) in FP64
    // (two accumulator sets per lane keep two terms in flight)
    const Df ntau = df_neg(df_from_f64(tau, E));
    Df pL = {0.f, 0.f}, dL = {0.f, 0.f}, pR = {0.f, 0.f}, dR = {0.f, 0.f};
    Df qL = {0.f, 0.f}, eL = {0.f, 0.f}, qR = {0.f, 0.f}, eR = {0.f, 0.f};
    for (int i = fb.n0 + sub; i < fb.n1; i += 2 * kSecG) {
      if (i != o) {
        Df t, dt;
        const float2 z = z2f[i];
        pair_term(dc[i] - dO, ntau, Df{z.x, z.y}, E, t, dt);
        if (i <= jsplit) { pL = df_add(pL, t); dL = df_add(dL, dt); }
        else { pR = df_add(pR, t); dR = df_add(dR, dt); }
      }
      const int i2 = i + kSecG;
      if (i2 < fb.n1 && i2 != o) {
        Df t, dt;
        const float2 z = z2f[i2];
        pair_term(dc[i2] - dO, ntau, Df{z.x, z.y}, E, t, dt);
        if (i2 <= jsplit) { qL = df_add(qL, t); eL = df_add(eL, dt); }
        else { qR = df_add(qR, t); eR = df_add(eR, dt); }
      }
    }
    double nL = pair_scaled(group_df_sum(df_add(pL, qL)), Z - E);
    double ndL = pair_scaled(group_df_sum(df_add(dL, eL)), Z - 2 * E);
    double nR = pair_scaled(group_df_sum(df_add(pR, qR)), Z - E);
    double ndR = pair_scaled(group_df_sum(df_add(dR, eR)), Z - 2 * E);
    if (group_any(!(finite_bits(nL) && finite_bits(ndL) && finite_bits(nR) && finite_bits(ndR)), g)) {
      // a term left the FP32 range: this root's near sums in FP64
      nL = ndL = nR = ndR = 0.0;
      for (int i = fb.n0 + sub; i < fb.n1; i += kSecG) {
        if (i == o) continue;
        const double rc = rcp64((dc[i] - dO) - tau);
        const double t = z2c[i] * rc, dt = t * rc;
        if (i <= jsplit) { nL += t; ndL += dt; }
        else { nR += t; ndR += dt; }
      }
      nL = group_sum(nL);
      ndL = group_sum(ndL);
      nR = group_sum(nR);
      ndR = group_sum(ndR);
    }
    if (f64far) {
      double cc[kSecNQ];
      int h2 = -1;
#pragma unroll
      for (int qi = 0; qi < kSecNQ; qi++) {
        const int q = sub + kSecG * qi;
        cc[qi] = 0.0;
        if (q < kSqP) {
          const double d = yh - sx[q];
          if (d == 0.0) h2 = q;
          else cc[qi] = sw[q] / d;
        }
      }
      const int hm2 = group_max(h2);
      double csum = 0.0;
#pragma unroll
      for (int qi = 0; qi < kSecNQ; qi++) {
        if (hm2 >= 0) cc[qi] = (sub + kSecG * qi == hm2) ? 1.0 : 0.0;
        csum += cc[qi];
      }
      const double icc = hm2 >= 0 ? 1.0 : 1.0 / group_sum(csum);
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
      for (int qi = 0; qi < kSecNQ; qi++) {
        const int q = sub + kSecG * qi;
        if (q < kSqP) {
          const double w = cc[qi] * icc;
          a0 += w * vals[q];
          a1 += w * vals[kSqP + q];
          a2 += w * vals[2 * kSqP + q];
          a3 += w * vals[3 * kSqP + q];
        }
      }
      s.psiL = group_sum(a0) + nL;
      s.dpsiL = group_sum(a1) + ndL;
      s.psiR = group_sum(a2) + nR;
      s.dpsiR = group_sum(a3) + ndR;
    } else {
      s.psiL = df_to_f64_scaled(group_df_sum(fL), 0) + nL;
      s.dpsiL = df_to_f64_scaled(group_df_sum(fdL), 0) + ndL;
      s.psiR = df_to_f64_scaled(group_df_sum(fR), 0) + nR;
      s.dpsiR = df_to_f64_scaled(group_df_sum(fdR), 0) + ndR;
    }
    {
      const double ri = -rcp64(tau);
      const double t = z2c[o] * ri, dt = t * ri;
      if (o <= jsplit) { s.psiL += t; s.dpsiL += dt; }
      else { s.psiR += t; s.dpsiR += dt; }
    }
    s.asum = s.psiR - s.psiL;
    return s;
  }
};

// secular_root's steps for a root j < k - 1 per group (active: the group has a root);
// returns 0 on convergence.  Every lane of the warp must call it.
__device__ int secular_root_group(const FarSumsG& sums, const FarBox& fb,
                                  const double* __restrict__ dc, double R, int j, bool active,
                                  int maxit, int sub, int g, int* o_out, double* tau_out) {
  const double wtol = kSecTolPairs;
  const double gap = dc[j + 1] - dc[j];
  int o = j;
  double tau = 0.5 * gap, lo, hi, aL, aR;
  SecSums sm = sums(fb, o, tau, j, sub, g);
  double w = 1.0 + R * (sm.psiL + sm.psiR);
  if (w >= 0.0) {  // root in (d_j, midpoint]
    o = j; lo = 0.0; hi = tau; aL = 0.0; aR = gap;
  } else {          // root in (midpoint, d_{j+1}): measure from d_{j+1}
    o = j + 1; tau = tau - gap; lo = tau; hi = 0.0; aL = -gap; aR = 0.0;
  }
  bool done = !active;
  int out_o = o;
  double out_t = tau;
  for (int it = 0; it < maxit; it++) {
    if (!done && (w == 0.0 || fabs(w) <= wtol * (1.0 + R * sm.asum))) {
      done = true; out_o = o; out_t = tau;
    }
    if (warp_all(done)) break;
    const double dL = aL - tau, dR = aR - tau;
    const double QL = sm.dpsiL * dL * dL, PL = sm.psiL - sm.dpsiL * dL;
    const double QR = sm.dpsiR * dR * dR, PR = sm.psiR - sm.dpsiR * dR;
    const double c = 1.0 + R * (PL + PR);
    const double A = c, B = c * (dL + dR) + R * (QL + QR), C = w * dL * dR;
    const double disc = fmax(B * B - 4.0 * A * C, 0.0);
    const double sq = disc > 0.0 ? disc * rsqrt64(disc) : 0.0;
    const double eta = (B > 0.0) ? (2.0 * C) * rcp64(B + sq) : (B - sq) * rcp64(2.0 * A);
    double tn = tau + eta;
    if (!finite_bits(tn) || !(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    if (!done && (tn == tau || fabs(tn - tau) <= 2.0 * kU * fabs(tau))) {
      done = true; out_o = o; out_t = tn;
    }
    if (warp_all(done)) break;
    const SecSums sn = sums(fb, o, done ? tau : tn, j, sub, g);
    if (!done) {
      tau = tn;
      sm = sn;
      w = 1.0 + R * (sm.psiL + sm.psiR);
      if (w < 0.0) lo = tau; else hi = tau;
      if (!(hi - lo > 2.0 * kU * fmax(fabs(lo), fabs(hi)))) { done = true; out_o = o; out_t = tau; }
    }
  }
  *o_out = done ? out_o : o;
  *tau_out = done ? out_t : tau;
  return done ? 0 : 1;
}

// The sums of one root by a whole block, for a root iterated by warp 0 alone (the
// block's other warps only help evaluate): warp 0 posts (o, tau, jsplit) and meets the
// helpers at named barrier 1; every warp adds its share of the poles into part[4][32];
// at barrier 2 warp 0 collects them.  The helpers leave when warp 0 posts cmd = 0.
struct LedSums {
  const double* dc;
  const double* z2c;
  int k;
  double* part;  // shared, 4 x 32
  double* s_tau;
  int* s_o;
  int* s_js;
  int* s_cmd;
  const float2* z2f;  // the pair form (scales E, Z), as FarSumsG
  int E, Z;
  static constexpr double wtol = kSecTolPairs;
  __device__ static void bar(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"((int)blockDim.x) : "memory");
  }
  __device__ void partial(int o, double tau, int jsplit) const {
    Df v[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    const double dO = dc[o];
    const Df ntau = df_neg(df_from_f64(tau, E));
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      if (i == o) continue;  // the origin pole: FP64, by warp 0
      Df t, dt;
      const float2 z = z2f[i];
      pair_term(dc[i] - dO, ntau, Df{z.x, z.y}, E, t, dt);
      if (i <= jsplit) { v[0] = df_add(v[0], t); v[1] = df_add(v[1], dt); }
      else { v[2] = df_add(v[2], t); v[3] = df_add(v[3], dt); }
    }
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const Df r = df_warp_sum(v[q]);
      if ((threadIdx.x & 31) == 0) part[q * 32 + w] = pair_scaled(r, (q & 1) ? Z - 2 * E : Z - E);
    }
  }
  // warp 0 only
  __device__ SecSums operator()(int o, double tau, int jsplit, int lane) const {
    if (lane == 0) { *s_o = o; *s_tau = tau; *s_js = jsplit; *s_cmd = 1; }
    bar(1);
    partial(o, tau, jsplit);
    bar(2);
    const int nw = blockDim.x >> 5;
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = warp_sum(lane < nw ? part[q * 32 + lane] : 0.0);
    if (!(finite_bits(v[0]) && finite_bits(v[1]) && finite_bits(v[2]) && finite_bits(v[3]))) {
      // a term left the FP32 range: FP64, warp 0
      const double dO = dc[o];
      for (int q = 0; q < 4; q++) v[q] = 0.0;
      for (int i = lane; i < k; i += 32) {
        if (i == o) continue;
        const double rc = rcp64((dc[i] - dO) - tau);
        const double t = z2c[i] * rc, dt = t * rc;
        if (i <= jsplit) { v[0] += t; v[1] += dt; }
        else { v[2] += t; v[3] += dt; }
      }
      for (int q = 0; q < 4; q++) v[q] = warp_sum(v[q]);
    }
    const double ri = -rcp64(tau);  // the origin pole
    const double t = z2c[o] * ri, dt = t * ri;
    if (o <= jsplit) { v[0] += t; v[1] += dt; }
    else { v[2] += t; v[3] += dt; }
    SecSums s = {v[0], v[1], v[2], v[3], v[2] - v[0]};
    return s;
  }
  // warps 1 ..
  __device__ void help() const {
    while (true) {
      bar(1);
      if (*s_cmd == 0) return;
      partial(*s_o, *s_tau, *s_js);
      bar(2);
    }
  }
};

// One root in the rho > 0 orientation; returns 0 on convergence.  `sums` evaluates the
// split sums of w at mu = d_o + tau (DirectSums, or LedSums for the far-field form's
// special roots).
template <class Sums>
__device__ int secular_root(const Sums& sums, const double* __restrict__ dc,
                            const double* __restrict__ z2c, int k, double R, double zn2, int j,
                            int lane, int maxit, int* o_out, double* tau_out) {
  int o;
  double tau, lo, hi, aL, aR;
  SecSums sm;
  double w;
  const bool last = (j == k - 1);
  if (!last) {
    double gap = dc[j + 1] - dc[j];
    o = j;
    tau = 0.5 * gap;
    sm = sums(o, tau, j, lane);
    w = 1.0 + R * (sm.psiL + sm.psiR);
    if (w >= 0.0) {  // root in (d_j, midpoint]
      o = j; lo = 0.0; hi = tau; aL = 0.0; aR = gap;
    } else {          // root in (midpoint, d_{j+1}): measure from d_{j+1}
      o = j + 1; tau = tau - gap; lo = tau; hi = 0.0; aL = -gap; aR = 0.0;
    }
  } else {
    o = j;
    hi = R * zn2 * (1.0 + 16.0 * kU) + 1e-300;
    lo = 0.0;
    tau = 0.5 * hi;
    aL = (k >= 2) ? (dc[k - 2] - dc[k - 1]) : 0.0;
    aR = 0.0;
    sm = sums(o, tau, j, lane);
    w = 1.0 + R * (sm.psiL + sm.psiR);
    if (w < 0.0) lo = tau; else hi = tau;
  }
  for (int it = 0; it < maxit; it++) {
    if (w == 0.0 || fabs(w) <= Sums::wtol * (1.0 + R * sm.asum)) {
      *o_out = o;
      *tau_out = tau;
      return 0;
    }
    double eta;
    bool ok = true;
    if (!last) {
      double dL = aL - tau, dR = aR - tau;
      double QL = sm.dpsiL * dL * dL, PL = sm.psiL - sm.dpsiL * dL;
      double QR = sm.dpsiR * dR * dR, PR = sm.psiR - sm.dpsiR * dR;
      double c = 1.0 + R * (PL + PR);
      double A = c, B = c * (dL + dR) + R * (QL + QR), C = w * dL * dR;
      const double disc = fmax(B * B - 4.0 * A * C, 0.0);
      const double sq = disc > 0.0 ? disc * rsqrt64(disc) : 0.0;
      eta = (B > 0.0) ? (2.0 * C) * rcp64(B + sq) : (B - sq) * rcp64(2.0 * A);
    } else {
      // all poles lie left of the root: the nearest one (k-1) exactly, the rest modelled
      // at the next pole (k-2) by value and slope
      double d2 = -tau;
      double t2 = z2c[k - 1] / d2;
      double pr = sm.psiL - t2, dpr = sm.dpsiL - t2 / d2;
      double d1 = (k >= 2) ? (aL - tau) : (d2 - 1.0);
      double Q1 = (k >= 2) ? dpr * d1 * d1 : 0.0;
      double P1 = (k >= 2) ? pr - dpr * d1 : 0.0;
      double Q2 = z2c[k - 1];
      double c = 1.0 + R * P1;
      if (c > 0.0) {
        double A = c, B = c * (d1 + d2) + R * (Q1 + Q2), C = w * d1 * d2;
        const double disc = fmax(B * B - 4.0 * A * C, 0.0);
        const double sq = disc > 0.0 ? disc * rsqrt64(disc) : 0.0;
        eta = (B >= 0.0) ? (B + sq) * rcp64(2.0 * A) : (2.0 * C) * rcp64(B - sq);
      } else {
        ok = false;
        eta = 0.0;
      }
    }
    double tn = tau + eta;
    if (!ok || !finite_bits(tn) || !(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    if (tn == tau || fabs(tn - tau) <= 2.0 * kU * fabs(tau)) {
      *o_out = o; *tau_out = tn; return 0;
    }
    tau = tn;
    sm = sums(o, tau, last ? k - 1 : j, lane);
    w = 1.0 + R * (sm.psiL + sm.psiR);
    if (w < 0.0) lo = tau; else hi = tau;
    if (!(hi - lo > 2.0 * kU * fmax(fabs(lo), fabs(hi)))) { *o_out = o; *tau_out = tau; return 0; }
  }
  *o_out = o;
  *tau_out = tau;
  return 1;
}

// Writes roots in both orientations: (orgc, tauc) for rho > 0 form, (org, tau, dorg)
// for the problem as given (rho < 0: root j' of the reflected problem is root k-1-j').
__device__ __forceinline__ void store_root(int j, int o, double t, int k, double rho,
                                           const double* __restrict__ dk, int* orgc,
                                           double* tauc, int* org, double* tau, double* dorg) {
  orgc[j] = o;
  tauc[j] = t;
  if (rho > 0.0) {
    org[j] = o;
    tau[j] = t;
    dorg[j] = dk[o];
  } else {
    const int jj = k - 1 - j, oo = k - 1 - o;
    org[jj] = oo;
    tau[jj] = -t;
    dorg[jj] = dk[oo];
  }
}

constexpr int kSecularThreads = 512;
constexpr int kSecStageMax = 12288;  // poles staged in shared memory up to this size (192 KB)

template <bool FARF>
__global__ void __launch_bounds__(FARF ? kSecularThreads : 256) k_secular(
    const double* __restrict__ dc, const double* __restrict__ z2c, const int* __restrict__ kp,
    const double* __restrict__ rhop, const double* __restrict__ dk, int* orgc, double* tauc,
    int* org, double* tau, double* dorg, int* status, int maxit, const double* __restrict__ sqb,
    const int* __restrict__ sqn, const int* __restrict__ sqf, const double* __restrict__ sqv,
    const float2* __restrict__ z2f, int stage_n) {
  __shared__ double s_zn2;
  __shared__ double s_x[kSqP], s_w[kSqP];
  const int k = kp[0];
  const double rho = rhop[0];
  const double R = fabs(rho);
  const bool far = FARF && sqv != nullptr && k >= kSqMinK;
  // The far-field form reads the poles and their pair weights once per term of every
  // iteration, from a few warps per SM: from shared memory (staged here when they fit,
  // stage_n >= k) instead of L2 that latency is no longer exposed.
  extern __shared__ double s_stage[];
  if (far && k <= stage_n) {
    float2* sz = (float2*)(s_stage + stage_n);
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      s_stage[i] = dc[i];
      sz[i] = z2f[i];
    }
    dc = s_stage;
    z2f = sz;
  }
  {  // ||z||^2 by the whole block (a warp alone would run k / 32 dependent FP64 adds)
    __shared__ double s_part[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) a += z2c[i];
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
      a = threadIdx.x < (int)(blockDim.x >> 5) ? s_part[threadIdx.x] : 0.0;
      a = warp_sum(a);
      if (threadIdx.x == 0) s_zn2 = a;
    }
  }
  if (threadIdx.x < kSqP) {  // Chebyshev nodes and barycentric weights (first kind)
    const double th = (2.0 * threadIdx.x + 1.0) / (2.0 * kSqP);
    s_x[threadIdx.x] = cospi(th);
    s_w[threadIdx.x] = (threadIdx.x & 1 ? -1.0 : 1.0) * sinpi(th);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int first = far ? sqf[0] : 0, last = far ? sqf[1] : k - 2;
  const int wl = threadIdx.x >> 5;
  if (far) {
    // The special roots -- the last root, whose bracket reaches far past the poles, and
    // the wide roots below `first` and above `last` -- one block each: warp 0 iterates,
    // the whole block evaluates the direct sums over every pole (LedSums).  Then every
    // warp takes kSecRoots consecutive boxed roots at a time, a group of kSecG lanes
    // each, from a counter (sqf[4], zeroed by k_sq_boxes): the blocks that solved a
    // special root join in when it is done, so the boxed roots never wait for them.
    const int nwl = first, nwr = k - 2 - last;
    const int nspec = 1 + nwl + nwr;
    for (int s = blockIdx.x; s < nspec; s += gridDim.x) {
      const int j = (s == 0) ? k - 1 : (s <= nwl ? s - 1 : last + (s - nwl));
      __shared__ double part[4 * 32];
      __shared__ double s_tau;
      __shared__ int s_o, s_js, s_cmd;
      // the last root's offset reaches R ||z||^2 past the largest pole: its own scale
      const int E = max(sqf[2], exp2_of(R * s_zn2) + 2);
      const LedSums ls = {dc, z2c, k, part, &s_tau, &s_o, &s_js, &s_cmd, z2f, E, sqf[3]};
      if (threadIdx.x < 32) {
        int o;
        double t;
        const int bad = secular_root(ls, dc, z2c, k, R, s_zn2, j, lane, maxit, &o, &t);
        if (lane == 0) s_cmd = 0;
        LedSums::bar(1);  // releases the helpers
        if (lane == 0) {
          if (bad) latch(status, SVDUP_ENOCONV);
          if (!isfinite(t)) latch(status, SVDUP_ENONFINITE);
          store_root(j, o, t, k, rho, dk, orgc, tauc, org, tau, dorg);
        }
      } else {
        ls.help();
      }
      __syncthreads();
    }
    int* next = const_cast<int*>(sqf) + 4;
    const FarSumsG fsg = {dc, z2c, z2f, s_x, s_w, sqf[2], sqf[3]};
    const int g = lane / kSecG, sub = lane % kSecG;
    while (true) {
      int q = 0;
      if (lane == 0) q = atomicAdd(next, 1);
      q = __shfl_sync(0xffffffffu, q, 0);
      if (first + kSecRoots * q > last) break;
      const int jr = first + kSecRoots * q + g;
      const bool active = jr <= last;
      const int j = active ? jr : first;  // an idle group evaluates a valid root
      const int b = (j - first) / kSqLeaf;
      const FarBox fb = {sqn[2 * b], sqn[2 * b + 1], sqb[2 * b], sqb[2 * b + 1],
                         sqv + (size_t)4 * b * kSqP};
      int o;
      double t;
      const int bad = secular_root_group(fsg, fb, dc, R, j, active, maxit, sub, g, &o, &t);
      if (active && sub == 0) {
        if (bad) latch(status, SVDUP_ENOCONV);
        if (!isfinite(t)) latch(status, SVDUP_ENONFINITE);
        store_root(j, o, t, k, rho, dk, orgc, tauc, org, tau, dorg);
      }
    }
    return;
  }
  // roots interleaved over the blocks (root j to block j mod G): neighbouring roots, whose
  // work is alike, spread over the SMs
  const int G = gridDim.x;
  const DirectSums direct = {dc, z2c, k};
  for (int j = wl * G + blockIdx.x; j < k; j += G * (blockDim.x >> 5)) {
    int o;
    double t;
    const int bad = secular_root(direct, dc, z2c, k, R, s_zn2, j, lane, maxit, &o, &t);
    if (lane == 0) {
      if (bad) latch(status, SVDUP_ENOCONV);
      if (!isfinite(t)) latch(status, SVDUP_ENONFINITE);
      store_root(j, o, t, k, rho, dk, orgc, tauc, org, tau, dorg);
    }
  }
}

// Streaming multiprocessors of the current device (queried once per device; threads
// that race on the first query store the same value).
int device_sm_count() {
  static std::atomic<int> cached[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  int c = cached[dev].load(std::memory_order_relaxed);
  if (c == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    c = n > 0 ? n : 152;
    cached[dev].store(c, std::memory_order_relaxed);
  }
  return c;
}

static int secular_blocks(int N) {
  int warps = N;                   // one warp per root
  int blocks = (warps * 32 + 255) / 256;
  return blocks < 1 ? 1 : blocks;
}

void launch_secular(cudaStream_t st, Eig e, int* status, int maxit) {
  const double* sqv = nullptr;
  if (e.sqv && e.N >= kSqMinK) {  // far-field set-up (the kernels skip small k themselves)
    const int nb = (e.N + kSqLeaf - 1) / kSqLeaf;
    k_sq_prep<<<1, 1024, 0, st>>>(e.dc, e.z2c, e.kp, e.sqf, e.z2f);
    SVDUP_COUNT_LAUNCH();
    k_sq_boxes<<<(nb + 127) / 128, 128, 0, st>>>(e.dc, e.kp, e.sqb, e.sqn, e.sqf);
    SVDUP_COUNT_LAUNCH();
    const int nw = nb * kSqP;
    k_sq_nodes<<<(nw * 32 + 255) / 256, 256, 0, st>>>(e.dc, e.z2f, e.kp, e.sqb, e.sqn, e.sqf,
                                                      e.sqv);
    SVDUP_COUNT_LAUNCH();
    sqv = e.sqv;
  }
  // With the far field, one block per SM: the first blocks take the special roots (one
  // each), then every warp kSecRoots boxed roots at a time from a counter.  Without it
  // (k < kSqMinK), a warp per root in blocks of 8 warps: a small solve then takes a few
  // SMs' worth of registers instead of whole SMs, which lets many small problems (a
  // batch's lanes) solve side by side.
  const int sms = device_sm_count();
  const int threads = sqv ? kSecularThreads : 256;
  const int blocks = sqv ? sms : std::min((e.N + threads / 32 - 1) / (threads / 32), 4 * sms);
  // the poles and pair weights staged in shared memory (16 B per pole) when they fit
  const int stage_n = (sqv && e.N <= kSecStageMax) ? e.N : 0;
  const size_t smem = (size_t)stage_n * (sizeof(double) + sizeof(float2));
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_secular<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  auto kern = sqv ? k_secular<true> : k_secular<false>;
  kern<<<blocks, threads, smem, st>>>(
      e.dc, e.z2c, e.kp, e.rhop, e.dk, e.orgc, e.tauc, e.org, e.tau, e.dorg, status, maxit, e.sqb,
      e.sqn, e.sqf, sqv, e.z2f, stage_n);
  SVDUP_COUNT_LAUNCH();
}

// The stand-alone secular entry point: d strictly ascending, z nonzero; the problem
// is brought to the rho > 0 orientation first.  A NaN or infinity in d or z latches
// SVDUP_ENONFINITE.
__global__ void k_secular_prep(int k, const double* __restrict__ d, const double* __restrict__ z,
                               const double* rhop, double* dc, double* z2c, double* dk, int* kp,
                               int* status) {
  const double rho = rhop[0];
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) kp[0] = k;
  if (t >= k) return;
  dk[t] = d[t];
  if (rho > 0.0) {
    dc[t] = d[t];
    z2c[t] = z[t] * z[t];
  } else {
    dc[t] = -d[k - 1 - t];
    z2c[t] = z[k - 1 - t] * z[k - 1 - t];
  }
  if (!isfinite(d[t]) || !isfinite(z[t])) latch(status, SVDUP_ENONFINITE);
}

void launch_secular_direct(cudaStream_t st, Eig e, int k, const double* d, const double* z,
                           int* status, int maxit) {
  k_secular_prep<<<(k + 255) / 256, 256, 0, st>>>(k, d, z, e.rhop, e.dc, e.z2c, e.dk, e.kp,
                                                  status);
  SVDUP_COUNT_LAUNCH();
  launch_secular(st, e, status, maxit);
}

// ---------------------------------------------------------------------------
// All N eigenvalues in ascending order: the roots (already ascending) merged with the
// deflated poles (kept values after rotation).  Ties: deflated before roots, then by
// index.  rank_root / rank_defl record where each one went.  The ranks are counted over
// shared-memory chunks of the deflated values by many blocks: one thread per eigenvalue
// (roots first, then deflated), each comparing its value with every deflated value
// (broadcast reads) and, for a deflated value, binary searching the ascending roots.
// ---------------------------------------------------------------------------
constexpr int kMergeChunk = 2048;

// IEEE doubles ordered as signed 64-bit integers (ties and signs preserved), so the
// comparisons run on the integer pipes rather than the FP64 unit.
__device__ __forceinline__ long long ordered_key(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

constexpr int kMergeLanes = 8;  // threads per eigenvalue, each counting a strided slice

__global__ void __launch_bounds__(256) k_merge_count(Eig e) {
  __shared__ long long sv[kMergeChunk];
  const int N = e.N, k = e.kp[0], nd = N - k;
  const int q = threadIdx.x % kMergeLanes;
  const int x = (blockIdx.x * blockDim.x + threadIdx.x) / kMergeLanes;
  const bool root = x < k;
  double val = 0.0;
  if (x < N) val = root ? e.dorg[x] + e.tau[x] : e.ds[e.didx[x - k]];
  const long long key = ordered_key(val);
  const int me = x - k;
  int cnt = 0;
  for (int c0 = 0; c0 < nd; c0 += kMergeChunk) {
    const int cn = min(kMergeChunk, nd - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < cn; t += blockDim.x) sv[t] = ordered_key(e.ds[e.didx[c0 + t]]);
    __syncthreads();
    if (x < N) {
      if (root) {
        for (int t = q; t < cn; t += kMergeLanes) cnt += (sv[t] <= key);
      } else {
        const int lim = me - c0;  // equal values rank by position in didx
        for (int t = q; t < cn; t += kMergeLanes) {
          const long long w = sv[t];
          cnt += (w < key) || (w == key && t < lim);
        }
      }
    }
  }
#pragma unroll
  for (int o = kMergeLanes / 2; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (x >= N || q != 0) return;
  if (root) {
    const int r = x + cnt;
    e.lam[r] = val;
    e.rank_root[x] = r;
  } else {
    int lo = 0, hi = k;  // roots strictly below the value, in the same integer order
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (ordered_key(e.dorg[mid] + e.tau[mid]) < key) lo = mid + 1; else hi = mid;
    }
    const int r = cnt + lo;
    e.lam[r] = val;
    e.rank_defl[e.didx[me]] = r;
  }
}

void launch_merge(cudaStream_t st, Eig e) {
  const long long threads = (long long)e.N * kMergeLanes;
  k_merge_count<<<(int)((threads + 255) / 256), 256, 0, st>>>(e);
  SVDUP_COUNT_LAUNCH();
}

// ---------------------------------------------------------------------------
// z recomputed from the computed roots (Loewner): the characteristic polynomial gives
//   prod_j (mu_j - d_i) = R zhat_i^2 prod_{j != i} (d_j - d_i)        (rho > 0 form),
// so the Cauchy-like vectors of Sec. 3.2 built from zhat are the exact eigenvectors of
// a problem whose exact eigenvalues are the computed roots, and stay orthogonal.
// Each pole j != i is paired with an adjacent root so every factor lies in (0, 1):
//   j < i: (mu_j - d_i)/(d_j - d_i),  j > i: (mu_{j-1} - d_i)/(d_j - d_i),
// and the remaining root mu_{k-1} contributes (mu_{k-1} - d_i)/R.  The numerator and
// denominator products are kept apart, each as a mantissa and a power of two (renormalised
// after every factor by the bit fields), so no factor takes a reciprocal: five FP64
// operations per factor.  One warp per index i; differences mu_j - d_i come from the
// offsets.
// ---------------------------------------------------------------------------
__global__ void k_loewner(Eig e) {
  const int k = e.kp[0];
  if (e.vf && k >= e.vfmin) return;  // the far-field form (svdup_vfmm.cu)
  const double rho = e.rhop[0];
  const double R = fabs(rho);
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const double* dc = e.dc;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < k; i += warps) {
    const double di = dc[i];
    double pn = 1.0, pd = 1.0;
    int en = 0, ed = 0;
    for (int j = lane; j < k; j += 32) {
      if (j == i) continue;
      const int jr = (j < i) ? j : j - 1;
      pn *= (dc[e.orgc[jr]] - di) + e.tauc[jr];
      pd *= dc[j] - di;
      renorm64(pn, en);
      renorm64(pd, ed);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      pn *= __shfl_xor_sync(0xffffffffu, pn, o);
      pd *= __shfl_xor_sync(0xffffffffu, pd, o);
      en += __shfl_xor_sync(0xffffffffu, en, o);
      ed += __shfl_xor_sync(0xffffffffu, ed, o);
      renorm64(pn, en);
      renorm64(pd, ed);
    }
    if (lane == 0) {
      const int sx = en - ed, h = sx / 2;
      double pr = (pn / pd) * ldexp(1.0, h) * ldexp(1.0, sx - h);
      pr *= ((dc[e.orgc[k - 1]] - di) + e.tauc[k - 1]) / R;
      double mag = sqrt(fmax(pr, 0.0));
      int io = (rho > 0.0) ? i : (k - 1 - i);
      double z = e.zk[io];
      e.zhat[io] = (z < 0.0) ? -mag : mag;
    }
  }
}

void launch_loewner(cudaStream_t st, Eig e) {
  launch_vf_loewner(st, e, e.vfmin);  // the far-field form when k >= vfmin
  k_loewner<<<secular_blocks(e.N), 256, 0, st>>>(e);
  SVDUP_COUNT_LAUNCH();
}

// ---------------------------------------------------------------------------
// Column norms of the Cauchy-like matrix (Eq. CTildeFinalForm1, RankOneUpdate STEP 7):
//   ||c_j||^2 = sum_t zhat_t^2 / delta_tj^2,  delta_tj = (dk_t - dk_org(j)) - tau_j,
// fused with the transposed product out[rank(j)] = (1/||c_j||) sum_t zhat_t y_t / delta_tj
// when a vector y (sorted, rotated basis) is given.  One warp per root j.
// ---------------------------------------------------------------------------
__global__ void k_norms(Eig e, const double* __restrict__ ysorted, double* out_final, int keep_inv) {
  const int k = e.kp[0];
  if (e.vf && k >= e.vfmin) return;  // the far-field form (svdup_vfmm.cu)
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < k; j += warps) {
    const double dO = e.dorg[j], tj = e.tau[j];
    double s2 = 0.0, sy = 0.0;
    for (int t = lane; t < k; t += 32) {
      double del = (e.dk[t] - dO) - tj;
      double c = e.zhat[t] * rcp64(del);
      s2 = fma(c, c, s2);
      if (ysorted) sy = fma(c, ysorted[e.idx[t]], sy);
    }
    s2 = warp_sum(s2);
    if (ysorted) sy = warp_sum(sy);
    if (lane == 0) {
      double inv = 1.0 / sqrt(s2);
      if (!keep_inv) e.inv[j] = inv;
      if (ysorted) out_final[e.rank_root[j]] = sy * inv;
    }
  }
}

__global__ void k_defl_copy(Eig e, const double* __restrict__ ysorted, double* out_final) {
  const int nd = e.N - e.kp[0];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nd; t += gridDim.x * blockDim.x) {
    int s = e.didx[t];
    out_final[e.rank_defl[s]] = ysorted[s];
  }
}

void launch_norms(cudaStream_t st, Eig e, const double* ysorted, double* out_final, bool pairs,
                  bool keep_inv) {
  // the far-field form when k >= vfmin (FP64) or vfmin_pairs (FP32 pairs)
  launch_vf_norms(st, e, pairs ? e.vfmin_pairs : e.vfmin, ysorted, out_final, keep_inv);
  if (pairs) {
    launch_norms_df(st, e, ysorted, out_final, secular_blocks(e.N), keep_inv);
  } else {
    k_norms<<<secular_blocks(e.N), 256, 0, st>>>(e, ysorted, out_final, keep_inv ? 1 : 0);
    SVDUP_COUNT_LAUNCH();
  }
  if (ysorted) {
    k_defl_copy<<<(e.N + 255) / 256, 256, 0, st>>>(e, ysorted, out_final);
    SVDUP_COUNT_LAUNCH();
  }
}

// ---------------------------------------------------------------------------
// Products of the full eigenvector matrix Q = P^T G^T [Ctilde (+) I] with vectors,
// used for the sign probe.  Q^T x: gather to sorted order, apply the rotations in
// order, then the transposed Cauchy product (k_norms with y).  Q x: Cauchy product,
// deflated entries copied, rotations transposed in reverse order, scatter.
// ---------------------------------------------------------------------------
// The vector lives in shared memory while one thread applies the rotations in order
// (global scratch `ysorted` itself when N is too large for shared memory).
static size_t vec_smem(int N) {
  size_t b = (size_t)N * sizeof(double);
  return b <= 160 * 1024 ? b : 0;
}

// The deflation rotations applied to one vector v (shared or global memory), by the
// whole block.  Rotation i acts on positions (a_i, b_i) with (cos, sin) = (c_i, s_i) and
// either opens a chain or continues the previous one (a_i = b_{i-1}); no position is
// read after it is written, so with x the original values each direction is an affine
// recurrence over the rotation list, evaluated as a block-wide scan of affine maps over
// per-thread chunks of the list:
//  forward (G, in order):      u_i = chained_i ? v_{i-1} : x_{a_i},  v_i = s_i u_i + c_i x_{b_i},
//                              out_{a_i} = c_i u_i - s_i x_{b_i},  out_{b_i} = v_i at a chain end;
//  transposed (G^T, reversed): w_i = chained_{i+1} ? c_{i+1} x_{b_i} + s_{i+1} w_{i+1} : x_{b_i},
//                              out_{b_i} = c_i w_i - s_i x_{a_i},
//                              out_{a_i} = c_i x_{a_i} + s_i w_i unless chained_i.
// The one value two chunks share (the boundary position of a chain crossing chunks) is
// read before the scan and kept in a register.
__device__ __forceinline__ bool rot_chained(const Eig& e, int i) {
  return i > 0 && e.rj[i] == e.ri[i - 1];
}

// Inclusive scan of affine maps v -> A v + B over the block's threads, composing in
// increasing thread order (dir > 0) or decreasing (dir < 0).  Returns the B of the
// composition of the chunks before the caller's (the carry entering its chunk).
__device__ double affine_carry(double A, double B, int dir, double* sA, double* sB) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int me = dir > 0 ? tid : nt - 1 - tid;  // position in composition order
  sA[me] = A;
  sB[me] = B;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    double Al = 1.0, Bl = 0.0;
    if (me >= off) { Al = sA[me - off]; Bl = sB[me - off]; }
    __syncthreads();
    if (me >= off) {
      const double Ar = sA[me], Br = sB[me];
      sA[me] = Ar * Al;
      sB[me] = fma(Ar, Bl, Br);
    }
    __syncthreads();
  }
  const double carry = me > 0 ? sB[me - 1] : 0.0;
  __syncthreads();
  return carry;
}

__device__ void rotate_vector(const Eig& e, double* v, bool transpose) {
  __shared__ double sA[1024], sB[1024];
  const int nr = e.nrot[0];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int per = (nr + nt - 1) / nt;
  const int i0 = min(nr, tid * per), i1 = min(nr, i0 + per);
  if (!transpose) {
    double A = 1.0, B = 0.0, xlast = 0.0;
    for (int i = i0; i < i1; i++) {
      const double c = e.rc[i], sn = e.rs[i];
      const double xb = v[e.ri[i]];
      if (rot_chained(e, i)) { A = sn * A; B = fma(sn, B, c * xb); }
      else { A = 0.0; B = fma(sn, v[e.rj[i]], c * xb); }
      xlast = xb;
    }
    double vc = affine_carry(A, B, 1, sA, sB);
    for (int i = i0; i < i1; i++) {
      const int a = e.rj[i], b = e.ri[i];
      const double c = e.rc[i], sn = e.rs[i];
      const double xb = (i == i1 - 1) ? xlast : v[b];
      const double u = rot_chained(e, i) ? vc : v[a];
      v[a] = c * u - sn * xb;
      vc = fma(sn, u, c * xb);
      if (i + 1 >= nr || e.rj[i + 1] != b) v[b] = vc;
    }
  } else {
    double A = 1.0, B = 0.0, xfirst = 0.0;
    if (i0 < i1) xfirst = v[e.rj[i0]];
    for (int i = i1 - 1; i >= i0; i--) {  // w_i as a map of w_{i1}
      const double xb = v[e.ri[i]];
      if (i + 1 < nr && rot_chained(e, i + 1)) {
        const double c1 = e.rc[i + 1], s1 = e.rs[i + 1];
        A = s1 * A;
        B = fma(s1, B, c1 * xb);
      } else {
        A = 0.0;
        B = xb;
      }
    }
    double w = affine_carry(A, B, -1, sA, sB);  // w_{i1}
    for (int i = i1 - 1; i >= i0; i--) {
      const int a = e.rj[i], b = e.ri[i];
      const double c = e.rc[i], sn = e.rs[i];
      const double xb = v[b];
      if (i + 1 < nr && rot_chained(e, i + 1)) w = fma(e.rs[i + 1], w, e.rc[i + 1] * xb);
      else w = xb;
      const double xa = (i == i0) ? xfirst : v[a];
      v[b] = c * w - sn * xa;
      if (!rot_chained(e, i)) v[a] = fma(c, xa, sn * w);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(1024) k_gather_rotate(Eig e, const double* __restrict__ xphys,
                                                        double* ysorted, int in_smem) {
  extern __shared__ double vsm[];
  double* v = in_smem ? vsm : ysorted;
  for (int s = threadIdx.x; s < e.N; s += blockDim.x) v[s] = xphys[e.perm[s]];
  __syncthreads();
  rotate_vector(e, v, false);
  if (in_smem)
    for (int s = threadIdx.x; s < e.N; s += blockDim.x) ysorted[s] = v[s];
}

void launch_apply_qt(cudaStream_t st, Eig e, const double* xphys, double* work, double* out_final,
                     bool pairs, bool keep_inv) {
  size_t sm = vec_smem(e.N);
  cudaFuncSetAttribute(k_gather_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_gather_rotate<<<1, 1024, sm, st>>>(e, xphys, work, sm > 0 ? 1 : 0);
  SVDUP_COUNT_LAUNCH();
  // the norms are recomputed (identical values in FP64); only the product is wanted here
  launch_norms(st, e, work, out_final, pairs, keep_inv);
}

__global__ void k_apply_q_core(Eig e, const double* __restrict__ xfinal, double* vsorted) {
  const int k = e.kp[0];
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const bool far = e.vf && k >= e.vfmin;  // the far-field form writes the kept entries
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < (far ? 0 : k); t += warps) {
    const double dt = e.dk[t];
    double acc = 0.0;
    for (int j = lane; j < k; j += 32) {
      double del = (dt - e.dorg[j]) - e.tau[j];
      acc = fma(e.inv[j] * rcp64(del), xfinal[e.rank_root[j]], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) vsorted[e.idx[t]] = e.zhat[t] * acc;
  }
  const int nd = e.N - k;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nd; u += gridDim.x * blockDim.x) {
    int s = e.didx[u];
    vsorted[s] = xfinal[e.rank_defl[s]];
  }
}

__global__ void __launch_bounds__(1024) k_unrotate_scatter(Eig e, double* vsorted, double* yphys,
                                                           int in_smem) {
  extern __shared__ double vsm[];
  double* v = in_smem ? vsm : vsorted;
  if (in_smem)
    for (int s = threadIdx.x; s < e.N; s += blockDim.x) v[s] = vsorted[s];
  __syncthreads();
  rotate_vector(e, v, true);
  for (int s = threadIdx.x; s < e.N; s += blockDim.x) yphys[e.perm[s]] = v[s];
}

void launch_apply_q(cudaStream_t st, Eig e, const double* xfinal, double* work, double* yphys,
                    bool pairs) {
  // the far-field form when k >= vfmin (FP64) or vfmin_pairs (FP32 pairs); the direct
  // kernels then copy the deflated entries only
  launch_vf_applyq(st, e, pairs ? e.vfmin_pairs : e.vfmin, xfinal, work);
  if (pairs) {
    launch_apply_q_core_df(st, e, xfinal, work, secular_blocks(e.N));
  } else {
    k_apply_q_core<<<secular_blocks(e.N), 256, 0, st>>>(e, xfinal, work);
    SVDUP_COUNT_LAUNCH();
  }
  size_t sm = vec_smem(e.N);
  cudaFuncSetAttribute(k_unrotate_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_unrotate_scatter<<<1, 1024, sm, st>>>(e, work, yphys, sm > 0 ? 1 : 0);
  SVDUP_COUNT_LAUNCH();
}

// ---------------------------------------------------------------------------
// Sign pairing of left and right vectors.  The left and right vectors come from
// independent eigen-updates (Alg. 6.1 STEPs 4-7), so each has an arbitrary sign.
// Uhat^T Ahat Vhat is diagonal with entries s_j sigmahat_j; with M = U^T Ahat V =
// S + p q^T (U, V orthogonal), h = Vhat^T Ahat^T Uhat w = Q4^T Q3^T M^T Q1 Q2 w for
// w = ones gives h_j = s_j sigmahat_j.  Here: y = M^T g for g = Q1 Q2 w.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_sign_combine(int m, int n, const double* __restrict__ S,
                                                       const double* __restrict__ p,
                                                       const double* __restrict__ q,
                                                       const double* __restrict__ g, double* y) {
  __shared__ double red[32];
  __shared__ double s_pg;
  double a = 0.0;
  for (int c = threadIdx.x; c < m; c += blockDim.x) a = fma(p[c], g[c], a);
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    a = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    a = warp_sum(a);
    if (threadIdx.x == 0) s_pg = a;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    y[c] = (c < m ? S[c] * g[c] : 0.0) + q[c] * s_pg;
}

void launch_sign_combine(cudaStream_t st, int m, int n, const double* S, const double* p,
                         const double* q, const double* g, double* y) {
  k_sign_combine<<<1, 1024, 0, st>>>(m, n, S, p, q, g, y);
  SVDUP_COUNT_LAUNCH();
}

// h in the right solve's final (ascending) order; right index r pairs with left index
// r - (n - m).  sign[r] = -1 where h_r < 0, else +1 (null-space columns keep +1).
__global__ void k_sign_finish(int m, int n, const double* __restrict__ h, double* sign) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  sign[r] = (r >= n - m && h[r] < 0.0) ? -1.0 : 1.0;
}

void launch_sign_finish(cudaStream_t st, int m, int n, const double* h, double* sign) {
  k_sign_finish<<<(n + 255) / 256, 256, 0, st>>>(m, n, h, sign);
  SVDUP_COUNT_LAUNCH();
}

// The signs applied to V after its second product (written unsigned, so that the
// product need not wait for the sign pairing): physical column c holds final index
// n - 1 - c.  Blocks of 1024 rows of one column of the paired part, four rows per thread
// with their loads issued together; blocks of unflipped columns exit at once.
__global__ void k_sign_apply(int m, int n, double* V, long long ldv, const double* __restrict__ sign) {
  const int c = blockIdx.x;
  if (c >= m || !(sign[n - 1 - c] < 0.0)) return;
  double* col = V + (long long)c * ldv;
  const int r0 = blockIdx.y * 1024 + threadIdx.x;
  double v[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int r = r0 + q * 256;
    v[q] = r < n ? col[r] : 0.0;
  }
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int r = r0 + q * 256;
    if (r < n) col[r] = -v[q];
  }
}

void launch_sign_apply(cudaStream_t st, int m, int n, double* V, long long ldv, const double* sign) {
  k_sign_apply<<<dim3(m, (n + 1023) / 1024), 256, 0, st>>>(m, n, V, ldv, sign);
  SVDUP_COUNT_LAUNCH();
}

__global__ void k_fill_ones(int n, double* w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = 1.0;
}

void launch_fill_ones(cudaStream_t st, int n, double* w) {
  k_fill_ones<<<(n + 255) / 256, 256, 0, st>>>(n, w);
  SVDUP_COUNT_LAUNCH();
}

// STEP 8: Shat = sqrt(D_n), D_n ascending -> Shat descending; negative rounding
// residue clamped to zero.
__global__ void k_sqrt_desc(int m, const double* __restrict__ lam, double* S, int* status) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  double v = lam[m - 1 - c];
  if (!isfinite(v)) latch(status, SVDUP_ENONFINITE);
  S[c] = sqrt(fmax(v, 0.0));
}

void launch_sqrt_desc(cudaStream_t st, int m, const double* lam, double* S, int* status) {
  k_sqrt_desc<<<(m + 255) / 256, 256, 0, st>>>(m, lam, S, status);
  SVDUP_COUNT_LAUNCH();
}


// ---------------------------------------------------------------------------
// Synthetic inputs for the autotuner (not part of the method): X (rows x N, entries
// uniform in [-1, 1) / sqrt(N)), poles d uniform in [0, 1), z uniform in [-1, 1), from
// the SplitMix64 generator (Steele, Lea and Flood 2014) applied to a counter.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double splitmix_unit(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);  // [0, 1) with 53 bits
}

__global__ void k_fill_random(int rows, int N, double* X, double* d, double* z,
                              unsigned long long seed) {
  const long long total = (long long)rows * N;
  const double sc = 1.0 / sqrt((double)N);
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    X[x] = (2.0 * splitmix_unit(seed * 0x100000001B3ULL + (unsigned long long)x) - 1.0) * sc;
    if (x < N) {
      d[x] = splitmix_unit((seed ^ 0xD1B54A32D192ED03ULL) + (unsigned long long)x);
      z[x] = 2.0 * splitmix_unit((seed ^ 0x8CB92BA72F3D8DD7ULL) + (unsigned long long)x) - 1.0;
    }
  }
}

void launch_fill_random(cudaStream_t st, int rows, int N, double* X, double* d, double* z,
                        unsigned long long seed) {
  k_fill_random<<<1024, 256, 0, st>>>(rows, N, X, d, z, seed);
  SVDUP_COUNT_LAUNCH();
}

}  // namespace svdup

// ---------------------------------------------------------------------------
// Diagnostic entry point: the library's own reciprocal and reciprocal square root on
// device arrays, so that tests can hold them against CUDA's division and square root.
// ---------------------------------------------------------------------------
namespace {
__global__ void k_check_rcp(int n, const double* __restrict__ x, double* r, double* rs) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (r) r[i] = svdup::rcp64(x[i]);
    if (rs) rs[i] = svdup::rsqrt64(x[i]);
  }
}
}  // namespace

extern "C" int svdup_check_rcp(void* stream, int n, const double* x, double* rcp, double* rsqrt) {
  if (n < 0 || (n > 0 && !x)) return SVDUP_EINVAL;
  if (n == 0) return SVDUP_OK;
  k_check_rcp<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, x, rcp, rsqrt);
  SVDUP_COUNT_LAUNCH();
  return cudaGetLastError() == cudaSuccess ? SVDUP_OK : SVDUP_ECUDA;
}
