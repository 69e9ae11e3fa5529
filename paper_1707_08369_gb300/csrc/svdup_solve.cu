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

#include "svdup_df.cuh"
#include "svdup_internal.cuh"

namespace svdup {

extern long long g_launch_count;

// ---------------------------------------------------------------------------
// Alg. 6.1 STEP 1.  The paper forms btilde = U S V^T b and atilde = V S^T U^T a and
// then, inside RankOneUpdate STEP 1, abar = U^T a1.  With U, V orthogonal (App. A)
// U^T btilde = S (V^T b) and V^T atilde = S^T (U^T a), so every z vector follows from
// p = U^T a and q = V^T b: one pass over U and one over V.
// One block per column: blocks [0, m) do columns of U, [m, m+n) columns of V, the
// last block computes alpha = a^T a and beta = b^T b.
// ---------------------------------------------------------------------------
__global__ void k_gemv_pq(int m, int n, const double* __restrict__ U, long long ldu,
                          const double* __restrict__ V, long long ldv, const double* __restrict__ a,
                          const double* __restrict__ b, double* p, double* q, double* ab) {
  __shared__ double red[2][32];
  int c = blockIdx.x;
  double s0 = 0.0, s1 = 0.0;
  if (c < m) {
    const double* col = U + (long long)c * ldu;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s0 = fma(col[r], a[r], s0);
  } else if (c < m + n) {
    const double* col = V + (long long)(c - m) * ldv;
    for (int r = threadIdx.x; r < n; r += blockDim.x) s0 = fma(col[r], b[r], s0);
  } else {
    for (int r = threadIdx.x; r < m; r += blockDim.x) s0 = fma(a[r], a[r], s0);
    for (int r = threadIdx.x; r < n; r += blockDim.x) s1 = fma(b[r], b[r], s1);
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { red[0][w] = s0; red[1][w] = s1; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    s0 = l < nw ? red[0][l] : 0.0;
    s1 = l < nw ? red[1][l] : 0.0;
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (l == 0) {
      if (c < m) p[c] = s0;
      else if (c < m + n) q[c - m] = s0;
      else { ab[0] = s0; ab[1] = s1; }
    }
  }
}

void launch_gemv_pq(cudaStream_t st, int m, int n, const double* U, long long ldu, const double* V,
                    long long ldv, const double* a, const double* b, double* p, double* q,
                    double* ab) {
  k_gemv_pq<<<m + n + 1, 256, 0, st>>>(m, n, U, ldu, V, ldv, a, b, p, q, ab);
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
// One block.  Reductions, case (1) and the compaction of its survivors run in
// parallel.  Case (3) on consecutive survivors (i-1, i): a rotation merges pole i-1
// into pole i, and the next pair (i, i+1) sees the merged values.  Along a run of
// merges starting at i0 the carrier after i holds
//     z~_i^2 = sum_{t=i0..i} z_t^2   and   d~_i = sum z_t^2 d_t / z~_i^2
// (each Givens step is a z^2-weighted mean), so the sequential test reduces to
//     |d_i - d~_{i-1}| |z_i| z~_{i-1} <= tol (z~_{i-1}^2 + z_i^2).
// Only pairs that pass with the original values (a bitmask found in parallel) can start
// a run, so the maximal chains of such pairs are walked in parallel by the block's
// warps, on shared-memory copies with just these two running sums, 32 pairs per step;
// the rare run that reaches into the next chain is resumed in order afterwards, so the
// boundaries are those of the sequential walk.  The rotation records (position pair,
// cos, sin) and the merged values are then formed in parallel from segmented prefix
// sums of z^2 and z^2 d over the runs.  This is the Bunch-Nielsen-Sorensen deflation
// in exact arithmetic; only the rounding of the merged values differs from applying
// the rotations one at a time.
// ---------------------------------------------------------------------------
constexpr int kDeflateThreads = 1024;
constexpr int kMaxOverrun = kMaxOverrunList;  // chains entered by the previous chain's run

// Block-wide exclusive prefix sum of one int per thread (Hillis-Steele over scnt);
// returns the exclusive prefix and writes the total to *total.
__device__ int block_excl_scan(int v, int* scnt, int* total) {
  const int tid = threadIdx.x, nt = blockDim.x;
  scnt[tid] = v;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    int u = tid >= off ? scnt[tid - off] : 0;
    __syncthreads();
    scnt[tid] += u;
    __syncthreads();
  }
  int incl = scnt[tid];
  *total = scnt[nt - 1];
  __syncthreads();
  return incl - v;
}

// Segmented inclusive scan over the threads' chunks of (flag, W, M): a chunk with
// flag set starts a new run at or after its start.  Returns the (W, M) of the run
// through the element just before the calling thread's chunk.
__device__ void run_carry(int lflag, double lW, double lM, int* sflag, double* sW, double* sM,
                          double* cW, double* cM) {
  const int tid = threadIdx.x, nt = blockDim.x;
  sflag[tid] = lflag;
  sW[tid] = lW;
  sM[tid] = lM;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    int f2 = 0;
    double W2 = 0.0, M2 = 0.0;
    if (tid >= off) { f2 = sflag[tid - off]; W2 = sW[tid - off]; M2 = sM[tid - off]; }
    __syncthreads();
    if (tid >= off && !sflag[tid]) { sW[tid] += W2; sM[tid] += M2; sflag[tid] = f2; }
    __syncthreads();
  }
  *cW = tid > 0 ? sW[tid - 1] : 0.0;
  *cM = tid > 0 ? sM[tid - 1] : 0.0;
  __syncthreads();
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

// The case-(3) walk on the survivors (scaled d and z, the candidate bitmask and the run
// flags brk, all in global scratch); every member is warp-collective.
struct DeflWalk {
  const unsigned* cmask;  // bit i: pair (i-1, i) passes with the original values
  const double* kd;
  const double* kz;
  unsigned char* brk;     // 1: survivor i starts a run
  int nk;
  double tol2;
  __device__ bool bit(int i) const { return i < nk && ((cmask[i >> 5] >> (i & 31)) & 1u); }
  // first position >= from whose bit equals want (nk if none)
  __device__ int next_bit(int from, bool want, int lane) const {
    if (from >= nk) return nk;
    const int nw = (nk + 31) >> 5;
    for (int w0 = from >> 5; w0 < nw; w0 += 32) {
      const int w = w0 + lane;
      unsigned m = 0u;
      if (w < nw) {
        m = want ? cmask[w] : ~cmask[w];
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
  // Walks the chain with first pair h up to pole lim (the pole before the next chain's
  // first pair, or nk - 1); returns 1 if the last run merged pole lim and a chain
  // follows, with the carrier in (W, M).
  __device__ int walk(int h, int lim, bool have, double& W, double& M, int lane) const {
    int pos = h;
    int ppos = -1;  // the window whose values are already loaded (next_z, next_d)
    double next_z = 0.0, next_d = 0.0;
    while (true) {
      if (!have) {
        const double zj = kz[pos - 1];
        W = zj * zj;
        M = W * kd[pos - 1];
      }
      const int i = pos + lane;
      const int nin = min(32, lim - pos + 1);
      double zi = 0.0, di = 0.0;
      if (ppos == pos) {
        zi = next_z;
        di = next_d;
      } else if (lane < nin) {
        zi = kz[i];
        di = kd[i];
      }
      // the next window, if the whole of this one merges, loads while this one is tested
      ppos = pos + 32;
      next_z = 0.0;
      next_d = 0.0;
      if (ppos + lane <= lim) {
        next_z = kz[ppos + lane];
        next_d = kd[ppos + lane];
      }
      const double z2 = zi * zi, dz = z2 * di;
      double iz2 = z2, idz = dz;  // inclusive prefix over the lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double a2 = __shfl_up_sync(0xffffffffu, iz2, o);
        const double ad = __shfl_up_sync(0xffffffffu, idz, o);
        if (lane >= o) { iz2 += a2; idz += ad; }
      }
      const bool ok = lane < nin && merges(di, zi, W + (iz2 - z2), M + (idz - dz), tol2);
      const unsigned fail = __ballot_sync(0xffffffffu, !ok);
      const int nm = fail ? __ffs(fail) - 1 : 32;  // lanes that merge
      if (lane < nm) brk[i] = 0;
      if (nm == nin) {  // every pole of the window merged
        W += __shfl_sync(0xffffffffu, iz2, nm - 1);
        M += __shfl_sync(0xffffffffu, idz, nm - 1);
        have = true;
        pos += nm;
        if (pos > lim) return lim + 1 < nk ? 1 : 0;
      } else {  // pole pos + nm failed: a new run only if its pair with the next passes
        have = false;
        pos += nm + 1;
        if (pos > lim || !bit(pos)) return 0;
      }
    }
  }
};

// Deflation, part 1 (one block): tolerance and scalings, case (1), the survivors'
// scaled d and z and sorted positions, the case-(3) candidate bitmask.
__global__ void __launch_bounds__(kDeflateThreads) k_deflate_pre(Eig e, int* status) {
  __shared__ double sred[3][32];
  __shared__ int scnt[kDeflateThreads];
  __shared__ double s_tol, s_zn, s_dsc, s_zsc;
  const int N = e.N;
  const double rho = e.rhop[0];
  int tid = threadIdx.x, nt = blockDim.x;
  double zn2 = 0.0, dmax = 0.0, zmax = 0.0;
  for (int s = tid; s < N; s += nt) {
    double z = e.zs[s], d = e.ds[s];
    zn2 = fma(z, z, zn2);
    dmax = fmax(dmax, fabs(d));
    zmax = fmax(zmax, fabs(z));
  }
  zn2 = warp_sum(zn2);
  dmax = warp_max(dmax);
  zmax = warp_max(zmax);
  if ((tid & 31) == 0) { sred[0][tid >> 5] = zn2; sred[1][tid >> 5] = dmax; sred[2][tid >> 5] = zmax; }
  __syncthreads();
  if (tid < 32) {
    int nw = nt >> 5;
    zn2 = tid < nw ? sred[0][tid] : 0.0;
    dmax = tid < nw ? sred[1][tid] : 0.0;
    zmax = tid < nw ? sred[2][tid] : 0.0;
    zn2 = warp_sum(zn2);
    dmax = warp_max(dmax);
    zmax = warp_max(zmax);
    if (tid == 0) {
      double t = fabs(rho) * zn2;
      s_tol = 8.0 * kU * fmax(dmax, t);
      s_zn = sqrt(zn2);
      // exact power-of-two scalings that bring max|d| and max|z| near 1 for the merge test
      s_dsc = (dmax > 0.0 && isfinite(dmax)) ? ldexp(1.0, -ilogb(dmax)) : 1.0;
      s_zsc = (zmax > 0.0 && isfinite(zmax)) ? ldexp(1.0, -ilogb(zmax)) : 1.0;
      e.tol[0] = s_tol;
      if (!isfinite(s_tol) || !isfinite(rho)) latch(status, SVDUP_ENONFINITE);
    }
  }
  __syncthreads();
  const double tol = s_tol, zn = s_zn, dsc = s_dsc, zsc = s_zsc;
  const double tolS = tol * dsc, tol2 = tolS * tolS;
  const int nwords = (N + 31) >> 5;
  unsigned* cmask = e.dmask;
  double* kd = e.dk;  // survivors' d * dsc (scratch: the compaction rewrites dk, zk, idx)
  double* kz = e.zk;  // survivors' z * zsc
  int* kpos = e.idx;  // survivors' sorted positions
  unsigned char* brk = (unsigned char*)e.didx;
  for (int w = tid; w < nwords; w += nt) cmask[w] = 0u;
  // case (1) on my contiguous chunk [b0, b1), then the survivors' positions in order
  const int chunk = (N + nt - 1) / nt;
  const int b0 = min(N, tid * chunk), b1 = min(N, b0 + chunk);
  int cnt = 0;
  for (int s = b0; s < b1; s++) {
    int d1 = (rho == 0.0 || fabs(rho) * zn * fabs(e.zs[s]) <= tol) ? 1 : 0;
    e.defl[s] = d1;
    cnt += !d1;
  }
  int nk;
  int pos = block_excl_scan(cnt, scnt, &nk);
  for (int s = b0; s < b1; s++) {
    if (e.defl[s]) continue;
    kpos[pos] = s;
    kd[pos] = e.ds[s] * dsc;
    kz[pos] = e.zs[s] * zsc;
    pos++;
  }
  __syncthreads();
  // case (3) pre-test with the original values: the candidate pairs
  for (int i = tid; i < nk; i += nt) {
    if (i > 0) {
      const double zj = kz[i - 1];
      const double W = zj * zj;
      if (merges(kd[i], kz[i], W, W * kd[i - 1], tol2)) atomicOr(&cmask[i >> 5], 1u << (i & 31));
    }
    brk[i] = 1;
  }
  if (tid == 0) {
    e.dint[0] = nk;
    e.dint[1] = 0;  // listed overruns
    e.dflt[0] = tol2;
    e.dflt[1] = dsc;
    e.dflt[2] = zsc;
  }
}

// Deflation, part 2 (many blocks): run boundaries, as the sequential walk finds them.
// Runs start only at pairs that pass with the original values (set bits of the
// bitmask); a chain is a maximal sequence of such pairs.  A run may continue past its
// chain's end through poles whose pairs fail alone but pass with the run's carrier, up
// to the pole before the next chain's first pair.  Global warp w walks the chains whose
// first pair lies in bitmask words w, w + W, ... from a fresh carrier, exactly as the
// sequential walk enters them, unless the previous chain's last run reached the next
// chain's first pole ("overran"); such chains are listed with the carrier for part 3.
// A warp steps 32 pairs at a time: from position pos with carrier (W, M), lane l tests
// pair (pos + l - 1, pos + l) against the carrier that exists if every earlier lane
// merged (W, M plus the lanes' exclusive prefix sums of z^2 and z^2 d): exactly the
// sequential carrier up to the first lane that fails.  Earlier lanes merge; a failing
// pole starts a new run with the next pair if that pair passes alone.
__global__ void __launch_bounds__(256) k_deflate_walk(Eig e) {
  const int nk = e.dint[0];
  const DeflWalk dw = {e.dmask, e.dk, e.zk, (unsigned char*)e.didx, nk, e.dflt[0]};
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int nw = (nk + 31) >> 5;
  for (int w = gw; w < nw; w += nwarps) {
    const unsigned m = dw.cmask[w];
    const unsigned prev = (w > 0) ? (dw.cmask[w - 1] >> 31) : 0u;
    unsigned heads = m & ~((m << 1) | prev);  // first pair of each chain
    while (heads) {
      const int h = (w << 5) + __ffs(heads) - 1;
      heads &= heads - 1;
      const int nh = dw.next_bit(dw.next_bit(h, false, lane), true, lane);  // next chain
      double W = 0.0, M = 0.0;
      if (dw.walk(h, nh - 1, false, W, M, lane) && lane == 0) {
        const int q = atomicAdd(&e.dint[1], 1);
        if (q < kMaxOverrun) { e.ovh[q] = nh; e.ovW[q] = W; e.ovM[q] = M; }
      }
    }
  }
}

// Deflation, part 3 (one block): the listed overruns resumed in order (one warp,
// cascading while runs keep overrunning; beyond kMaxOverrun listed, the whole walk again,
// sequentially), then the rotation records, the merged values and the compaction.
__global__ void __launch_bounds__(kDeflateThreads) k_deflate_post(Eig e, int in_smem) {
  extern __shared__ double dsm[];
  __shared__ int scnt[kDeflateThreads];
  __shared__ double sW[kDeflateThreads], sM[kDeflateThreads];
  const int N = e.N;
  const double rho = e.rhop[0];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nk = e.dint[0];
  const double dsc = e.dflt[1], zsc = e.dflt[2];
  const double idsc = 1.0 / dsc, izsc = 1.0 / zsc;  // exact: powers of two
  const double* kd = e.dk;
  const double* kz = e.zk;
  const int* kpos = e.idx;
  unsigned char* brk = (unsigned char*)e.didx;
  if (in_smem) {  // the sequential resumes and the records read these many times
    double* skd = dsm;
    double* skz = dsm + N;
    unsigned char* sbrk = (unsigned char*)(dsm + 2 * (size_t)N);
    for (int i = tid; i < nk; i += nt) {
      skd[i] = kd[i];
      skz[i] = kz[i];
      sbrk[i] = brk[i];
    }
    __syncthreads();
    kd = skd;
    kz = skz;
    brk = sbrk;
  }
  const int nov = e.dint[1];
  if (tid < 32 && nov > 0) {
    const int lane = tid;
    const DeflWalk dw = {e.dmask, kd, kz, brk, nk, e.dflt[0]};
    if (nov > kMaxOverrun) {
      for (int i = lane; i < nk; i += 32) brk[i] = 1;
      __syncwarp();
      int h = dw.next_bit(1, true, lane);
      bool have = false;
      double W = 0.0, M = 0.0;
      while (h < nk) {
        const int nh = dw.next_bit(dw.next_bit(h, false, lane), true, lane);
        have = dw.walk(h, nh - 1, have, W, M, lane) != 0;
        h = nh;
      }
    } else {
      if (lane == 0)  // ascending chain order (a short list)
        for (int x = 1; x < nov; x++)
          for (int y = x; y > 0 && e.ovh[y - 1] > e.ovh[y]; y--) {
            const int th = e.ovh[y]; e.ovh[y] = e.ovh[y - 1]; e.ovh[y - 1] = th;
            const double tw = e.ovW[y]; e.ovW[y] = e.ovW[y - 1]; e.ovW[y - 1] = tw;
            const double tm = e.ovM[y]; e.ovM[y] = e.ovM[y - 1]; e.ovM[y - 1] = tm;
          }
      __syncwarp();
      int done = 0;  // chains before this position hold their final boundaries
      for (int x = 0; x < nov; x++) {
        int h = e.ovh[x];
        if (h <= done) continue;  // listed by a chain that a resumed walk redid
        double W = e.ovW[x], M = e.ovM[x];
        while (true) {  // resume the sequential walk at chain h
          const int nh = dw.next_bit(dw.next_bit(h, false, lane), true, lane);
          for (int i = h + lane; i < nh; i += 32) brk[i] = 1;
          __syncwarp();
          const int more = dw.walk(h, nh - 1, true, W, M, lane);
          done = nh;
          if (!more) break;
          h = nh;
        }
      }
    }
  }
  __syncthreads();
  const int cpt = (nk + nt - 1) / nt;
  const int c0 = min(nk, tid * cpt), c1 = min(nk, c0 + cpt);
  const int chunk = (N + nt - 1) / nt;
  const int b0 = min(N, tid * chunk), b1 = min(N, b0 + chunk);
  int cnt, pos;
  // rotation records and merged values from the runs (segmented sums again)
  {
    double lW = 0.0, lM = 0.0;
    int lflag = 0, lrot = 0;
    for (int i = c0; i < c1; i++) {
      const double z2 = kz[i] * kz[i];
      if (brk[i]) { lflag = 1; lW = z2; lM = z2 * kd[i]; }
      else { lW += z2; lM = fma(z2, kd[i], lM); lrot++; }
    }
    int nrot;
    const int rbase = block_excl_scan(lrot, scnt, &nrot);
    double W, M;
    run_carry(lflag, lW, lM, scnt, sW, sM, &W, &M);
    int ridx = rbase;
    for (int i = c0; i < c1; i++) {
      const bool p = !brk[i];
      const double zi = kz[i], di = kd[i], z2 = zi * zi;
      if (!p) {
        W = z2;
        M = z2 * di;
      } else {
        // rotation merging survivor i-1 (the carrier) into i
        const double zprev = brk[i - 1] ? kz[i - 1] : W * rsqrt64(W);  // signed at a run start
        const double Wn = W + z2;
        const double irn = rsqrt64(Wn);
        const double cs = zi * irn, sn = zprev * irn;
        const double dprev = M * rcp64(W);
        const int pj = kpos[i - 1], pi = kpos[i];
        e.ds[pj] = (cs * cs * dprev + sn * sn * di) * idsc;
        e.zs[pj] = 0.0;
        e.defl[pj] = 2;  // deflated by a rotation: the rotation kernel writes its column
        e.rj[ridx] = pj; e.ri[ridx] = pi; e.rc[ridx] = cs; e.rs[ridx] = sn;
        ridx++;
        W = Wn;
        M = fma(z2, di, M);
      }
      if (!(i + 1 < nk && !brk[i + 1])) {  // not merged away by the next pair
        const int ps = kpos[i];
        if (p) { e.ds[ps] = (M * rcp64(W)) * idsc; e.zs[ps] = (W * rsqrt64(W)) * izsc; }
        else { e.ds[ps] = di * idsc; e.zs[ps] = zi * izsc; }
      }
    }
    if (tid == 0) e.nrot[0] = nrot;
  }
  __syncthreads();
  // compaction of the kept set
  cnt = 0;
  for (int s = b0; s < b1; s++) cnt += !e.defl[s];
  int kk;
  pos = block_excl_scan(cnt, scnt, &kk);  // kept entries before my chunk
  int dpos = b0 - pos;                     // deflated entries before my chunk
  for (int s = b0; s < b1; s++) {
    if (!e.defl[s]) {
      e.idx[pos] = s;
      e.dk[pos] = e.ds[s];
      e.zk[pos] = e.zs[s];
      pos++;
    } else {
      e.didx[dpos++] = s;
    }
  }
  if (tid == 0) e.kp[0] = kk;
  __syncthreads();
  // the rho > 0 orientation for the solver: reflect d -> -d (reversed) when rho < 0
  for (int t = tid; t < kk; t += nt) {
    if (rho > 0.0) {
      e.dc[t] = e.dk[t];
      double z = e.zk[t];
      e.z2c[t] = z * z;
    } else {
      e.dc[t] = -e.dk[kk - 1 - t];
      double z = e.zk[kk - 1 - t];
      e.z2c[t] = z * z;
    }
  }
}

void launch_deflate(cudaStream_t st, Eig e, int* status) {
  k_deflate_pre<<<1, kDeflateThreads, 0, st>>>(e, status);
  SVDUP_COUNT_LAUNCH();
  const int nwords = (e.N + 31) / 32;
  k_deflate_walk<<<std::max(1, (nwords + 7) / 8), 256, 0, st>>>(e);  // a warp per bitmask word
  SVDUP_COUNT_LAUNCH();
  // the survivors' d, z and run flags in shared memory when they fit (static: 20 KB)
  const size_t smem = (size_t)e.N * (2 * sizeof(double) + 1) + 16;
  const int in_smem = smem <= 200 * 1024 ? 1 : 0;
  cudaFuncSetAttribute(k_deflate_post, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       in_smem ? (int)smem : 0);
  k_deflate_post<<<1, kDeflateThreads, in_smem ? smem : 0, st>>>(e, in_smem);
  SVDUP_COUNT_LAUNCH();
}

// ---------------------------------------------------------------------------
// Secular equation (Sec. 3.1, Eq. GolubEigenvalUpdate):
//   w(mu) = 1 + R sum_i z_i^2 / (d_i - mu),  R > 0, d strictly ascending.
// Root j lies in (d_j, d_{j+1}) (j < k-1) or in (d_{k-1}, d_{k-1} + R ||z||^2].
// One warp per root; the lanes split the k poles and reduce.  The root is held as
// mu = d_o + tau with o the nearer pole (decided by the sign of w at the bracket
// midpoint), so every difference d_i - mu = (d_i - d_o) - tau keeps full relative
// accuracy when the root sits next to a pole.
// Iteration: the rational model of Bunch, Nielsen and Sorensen (1978): the poles left
// of the root are modelled by P_L + Q_L / (d_left - mu), those right of it by
// P_R + Q_R / (d_right - mu), each matching value and slope at the current iterate;
// the model's root in the bracket is one quadratic.  The bracket is kept from the
// signs of w and a model step that leaves it is replaced by bisection.
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
__device__ __forceinline__ double pair_scaled(Df a, int s) {
  const int h = s / 2;
  return df_to_f64(a, 0) * pow2d(max(-1022, min(1023, h))) * pow2d(max(-1022, min(1023, s - h)));
}

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
// field).  From each end, while one bracket gap is more than half the span of the next
// kSqLeaf roots, every root up to that gap is solved alone by one block with direct
// sums (at most kSqMaxWide per end), as is the last root (beyond all poles).  The boxes
// of kSqLeaf roots cover roots first .. last; k_sq_boxes stores the layout in sqf.
constexpr int kSqMaxWide = 16;

__device__ void sq_layout(const double* __restrict__ dc, int k, int* first, int* last) {
  int f = 0, l = k - 2;
  if (k >= kSqMinK) {
    while (f < kSqMaxWide) {
      const double span = dc[f + kSqLeaf] - dc[f];
      int g = f;
      double gmax = -1.0;
      for (int j = f; j < f + kSqLeaf; j++) {
        const double gap = dc[j + 1] - dc[j];
        if (gap > gmax) { gmax = gap; g = j; }
      }
      if (!(gmax > 0.5 * span) || g + 1 > kSqMaxWide) break;
      f = g + 1;
    }
    while (k - 2 - l < kSqMaxWide) {
      const double span = dc[l + 1] - dc[l + 1 - kSqLeaf];
      int g = l;
      double gmax = -1.0;
      for (int j = l; j > l - kSqLeaf; j--) {
        const double gap = dc[j + 1] - dc[j];
        if (gap > gmax) { gmax = gap; g = j; }
      }
      if (!(gmax > 0.5 * span) || k - 1 - g > kSqMaxWide) break;
      l = g - 1;
    }
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

struct FarSums {
  const double* dc;
  const double* z2c;
  int n0, n1;
  double base, r;
  const double* vals;  // 4 x kSqP node values of this box
  const double* sx;    // Chebyshev nodes (shared memory)
  const double* sw;    // barycentric weights (shared memory)
  const float2* z2f;   // z^2 2^-Z as pairs
  int E, Z;
  static constexpr double wtol = kSecTolPairs;
  __device__ SecSums operator()(int o, double tau, int jsplit, int lane) const {
    SecSums s = {0.0, 0.0, 0.0, 0.0, 0.0};
    const double dO = dc[o];
    // Barycentric weights of the far field at the box coordinate of mu, in pairs (within
    // the pair form's error budget): c_l = w_l / (y - x_l), normalised by their sum.
    const double yh = (((dO - base) + tau) - r) * rcp64(r);
    // node values beyond the pair range (exponent tests only): the FP64 form below
    const bool big = lane < kSqP && max(max(exp2_of(vals[lane]), exp2_of(vals[kSqP + lane])),
                                        max(exp2_of(vals[2 * kSqP + lane]),
                                            exp2_of(vals[3 * kSqP + lane]))) > 120;
    const bool f64far = __any_sync(0xffffffffu, big);
    Df c = {0.f, 0.f};
    int hit = 0;
    if (lane < kSqP) {
      const Df dfy = df_add(df_from_f64(yh, 0), df_neg(df_from_f64(sx[lane], 0)));
      if (dfy.hi == 0.0f) hit = 1;
      else c = df_mul(df_from_f64(sw[lane], 0), df_rcp(dfy));
    }
    const unsigned hm = __ballot_sync(0xffffffffu, hit);
    if (hm) {  // mu sits exactly on a node
      c = (lane == __ffs(hm) - 1) ? Df{1.0f, 0.0f} : Df{0.0f, 0.0f};
    } else {
      c = df_mul(c, df_rcp(df_warp_sum(c)));
    }
    Df fL = {0.f, 0.f}, fdL = {0.f, 0.f}, fR = {0.f, 0.f}, fdR = {0.f, 0.f};
    if (lane < kSqP) {  // far-left terms are negative, far-right positive
      fL = df_mul(c, df_from_f64(vals[lane], 0));
      fdL = df_mul(c, df_from_f64(vals[kSqP + lane], 0));
      fR = df_mul(c, df_from_f64(vals[2 * kSqP + lane], 0));
      fdR = df_mul(c, df_from_f64(vals[3 * kSqP + lane], 0));
    }
    // near poles in pairs, the origin pole (offset -tau) in FP64
    const Df ntau = df_neg(df_from_f64(tau, E));
    Df pL = {0.f, 0.f}, dL = {0.f, 0.f}, pR = {0.f, 0.f}, dR = {0.f, 0.f};
    for (int i = n0 + lane; i < n1; i += 32) {
      if (i == o) continue;
      Df t, dt;
      const float2 z = z2f[i];
      pair_term(dc[i] - dO, ntau, Df{z.x, z.y}, E, t, dt);
      if (i <= jsplit) { pL = df_add(pL, t); dL = df_add(dL, dt); }
      else { pR = df_add(pR, t); dR = df_add(dR, dt); }
    }
    double nL = pair_scaled(df_warp_sum(pL), Z - E), ndL = pair_scaled(df_warp_sum(dL), Z - 2 * E);
    double nR = pair_scaled(df_warp_sum(pR), Z - E), ndR = pair_scaled(df_warp_sum(dR), Z - 2 * E);
    if (!isfinite(nL + ndL + nR + ndR)) {  // a term left the FP32 range: this one in FP64
      nL = ndL = nR = ndR = 0.0;
      for (int i = n0 + lane; i < n1; i += 32) {
        if (i == o) continue;
        const double rc = rcp64((dc[i] - dO) - tau);
        const double t = z2c[i] * rc, dt = t * rc;
        if (i <= jsplit) { nL += t; ndL += dt; }
        else { nR += t; ndR += dt; }
      }
      nL = warp_sum(nL);
      ndL = warp_sum(ndL);
      nR = warp_sum(nR);
      ndR = warp_sum(ndR);
    }
    if (f64far) {
      double cc = 0.0;
      int h2 = 0;
      if (lane < kSqP) {
        const double d = yh - sx[lane];
        if (d == 0.0) h2 = 1;
        else cc = sw[lane] / d;
      }
      const unsigned hm2 = __ballot_sync(0xffffffffu, h2);
      if (hm2) cc = (lane == __ffs(hm2) - 1) ? 1.0 : 0.0;
      else cc = cc / warp_sum(cc);
      const bool on = lane < kSqP;
      s.psiL = warp_sum(on ? cc * vals[lane] : 0.0) + nL;
      s.dpsiL = warp_sum(on ? cc * vals[kSqP + lane] : 0.0) + ndL;
      s.psiR = warp_sum(on ? cc * vals[2 * kSqP + lane] : 0.0) + nR;
      s.dpsiR = warp_sum(on ? cc * vals[3 * kSqP + lane] : 0.0) + ndR;
    } else {
      s.psiL = df_to_f64(df_warp_sum(fL), 0) + nL;
      s.dpsiL = df_to_f64(df_warp_sum(fdL), 0) + ndL;
      s.psiR = df_to_f64(df_warp_sum(fR), 0) + nR;
      s.dpsiR = df_to_f64(df_warp_sum(fdR), 0) + ndR;
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
  const float2* z2f;  // the pair form (scales E, Z), as FarSums
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
    if (!isfinite(v[0] + v[1] + v[2] + v[3])) {  // a term left the FP32 range: FP64, warp 0
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
// split sums of w at mu = d_o + tau (DirectSums or FarSums).
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
      double disc = fmax(B * B - 4.0 * A * C, 0.0);
      double sq = sqrt(disc);
      eta = (B > 0.0) ? (2.0 * C) / (B + sq) : (B - sq) / (2.0 * A);
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
        double disc = fmax(B * B - 4.0 * A * C, 0.0);
        double sq = sqrt(disc);
        eta = (B >= 0.0) ? (B + sq) / (2.0 * A) : (2.0 * C) / (B - sq);
      } else {
        ok = false;
        eta = 0.0;
      }
    }
    double tn = tau + eta;
    if (!ok || !isfinite(tn) || !(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
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

constexpr int kSecularThreads = 1024;
constexpr int kSecularSpecial = 1 + 2 * kSqMaxWide;  // the last root and the wide roots

__global__ void __launch_bounds__(kSecularThreads) k_secular(
    const double* __restrict__ dc, const double* __restrict__ z2c, const int* __restrict__ kp,
    const double* __restrict__ rhop, const double* __restrict__ dk, int* orgc, double* tauc,
    int* org, double* tau, double* dorg, int* status, int maxit, const double* __restrict__ sqb,
    const int* __restrict__ sqn, const int* __restrict__ sqf, const double* __restrict__ sqv,
    const float2* __restrict__ z2f) {
  __shared__ double s_zn2;
  __shared__ double s_x[kSqP], s_w[kSqP];
  const int k = kp[0];
  const double rho = rhop[0];
  const double R = fabs(rho);
  const bool far = sqv != nullptr && k >= kSqMinK;
  if (threadIdx.x < 32) {
    double a = 0.0;
    for (int i = threadIdx.x; i < k; i += 32) a += z2c[i];
    a = warp_sum(a);
    if (threadIdx.x == 0) s_zn2 = a;
  }
  if (threadIdx.x < kSqP) {  // Chebyshev nodes and barycentric weights (first kind)
    const double th = (2.0 * threadIdx.x + 1.0) / (2.0 * kSqP);
    s_x[threadIdx.x] = cospi(th);
    s_w[threadIdx.x] = (threadIdx.x & 1 ? -1.0 : 1.0) * sinpi(th);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int first = far ? sqf[0] : 0, last = far ? sqf[1] : k - 2;
  if (far && blockIdx.x < kSecularSpecial) {
    // The first blocks (scheduled first, each alone on its SM: one block of
    // kSecularThreads per SM) solve the last root, whose bracket reaches far past the
    // poles, and the wide roots, with direct sums over the whole block.
    const int s = blockIdx.x;
    int j = -1;
    if (s == 0) j = k - 1;
    else if (s <= kSqMaxWide) j = (s - 1 < first) ? s - 1 : -1;
    else j = (last + s - kSqMaxWide <= k - 2) ? last + s - kSqMaxWide : -1;
    if (j < 0) return;
    // warp 0 iterates, the whole block evaluates the sums
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
    return;
  }
  const int off = far ? kSecularSpecial : 0;
  // roots interleaved over the blocks (root j to block j mod G): neighbouring roots, whose
  // work is alike, spread over the SMs
  const int G = gridDim.x - off, bm = blockIdx.x - off, wl = threadIdx.x >> 5;
  const DirectSums direct = {dc, z2c, k};
  for (int j = wl * G + bm; j < k; j += G * (blockDim.x >> 5)) {
    int o;
    double t;
    int bad;
    if (far && (j < first || j > last)) continue;  // done by blocks 0-2
    if (far) {
      const int b = (j - first) / kSqLeaf;
      const FarSums fs = {dc,      z2c,      sqn[2 * b], sqn[2 * b + 1], sqb[2 * b],
                          sqb[2 * b + 1], sqv + (size_t)4 * b * kSqP, s_x, s_w, z2f,
                          sqf[2],  sqf[3]};
      bad = secular_root(fs, dc, z2c, k, R, s_zn2, j, lane, maxit, &o, &t);
    } else {
      bad = secular_root(direct, dc, z2c, k, R, s_zn2, j, lane, maxit, &o, &t);
    }
    if (lane == 0) {
      if (bad) latch(status, SVDUP_ENOCONV);
      if (!isfinite(t)) latch(status, SVDUP_ENONFINITE);
      store_root(j, o, t, k, rho, dk, orgc, tauc, org, tau, dorg);
    }
  }
}

// Streaming multiprocessors of the current device (queried once per device).
int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 152;
  }
  return cached[dev];
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
  // a warp per root, at most one block per SM (the roots are interleaved over them)
  const int blocks =
      std::min((e.N + kSecularThreads / 32 - 1) / (kSecularThreads / 32), device_sm_count());
  k_secular<<<blocks + (sqv ? kSecularSpecial : 0), kSecularThreads, 0, st>>>(
      e.dc, e.z2c, e.kp, e.rhop, e.dk, e.orgc, e.tauc, e.org, e.tau, e.dorg, status, maxit, e.sqb,
      e.sqn, e.sqf, sqv, e.z2f);
  SVDUP_COUNT_LAUNCH();
}

// The stand-alone secular entry point: d strictly ascending, z nonzero; the problem
// is brought to the rho > 0 orientation first.
__global__ void k_secular_prep(int k, const double* __restrict__ d, const double* __restrict__ z,
                               const double* rhop, double* dc, double* z2c, double* dk, int* kp) {
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
}

void launch_secular_direct(cudaStream_t st, Eig e, int k, const double* d, const double* z,
                           int* status, int maxit) {
  k_secular_prep<<<(k + 255) / 256, 256, 0, st>>>(k, d, z, e.rhop, e.dc, e.z2c, e.dk, e.kp);
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
// Exponent bookkeeping for long FP64 products: x = m 2^e with m in [1, 2) after
// renorm (bit fields only; a zero stays zero).
__device__ __forceinline__ void renorm64(double& m, int& e) {
  const long long b = __double_as_longlong(m);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return;
  m = __longlong_as_double((b & ~(0x7ffll << 52)) | (1023ll << 52));
  e += ex - 1023;
}

__global__ void k_loewner(Eig e) {
  const int k = e.kp[0];
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
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < k; t += warps) {
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
