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

#include "svdup_internal.cuh"

namespace svdup {

extern long long g_launch_count;
#define SVDUP_COUNT_LAUNCH() (++g_launch_count)

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
// One block.  Reductions and case (1) run in parallel; the case-(3) scan is a
// sequential pass by one thread (each rotation changes the next comparison);
// compaction of the kept set is a block-wide prefix sum.  An optional vector y
// (a second direction in the same sorted basis) is rotated alongside z.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_deflate(Eig e, double* yvec, int* status) {
  __shared__ double sred[2][32];
  __shared__ int scnt[1024];
  __shared__ int s_ncand;
  __shared__ double s_tol, s_zn;
  const int N = e.N;
  const double rho = e.rhop[0];
  int tid = threadIdx.x, nt = blockDim.x;
  double zn2 = 0.0, dmax = 0.0;
  for (int s = tid; s < N; s += nt) {
    double z = e.zs[s], d = e.ds[s];
    zn2 = fma(z, z, zn2);
    dmax = fmax(dmax, fabs(d));
  }
  zn2 = warp_sum(zn2);
  dmax = warp_max(dmax);
  if ((tid & 31) == 0) { sred[0][tid >> 5] = zn2; sred[1][tid >> 5] = dmax; }
  __syncthreads();
  if (tid < 32) {
    int nw = nt >> 5;
    zn2 = tid < nw ? sred[0][tid] : 0.0;
    dmax = tid < nw ? sred[1][tid] : 0.0;
    zn2 = warp_sum(zn2);
    dmax = warp_max(dmax);
    if (tid == 0) {
      double t = fabs(rho) * zn2;
      s_tol = 8.0 * kU * fmax(dmax, t);
      s_zn = sqrt(zn2);
      e.tol[0] = s_tol;
      if (!isfinite(s_tol) || !isfinite(rho)) latch(status, SVDUP_ENONFINITE);
    }
  }
  __syncthreads();
  const double tol = s_tol, zn = s_zn;
  // thread t owns the contiguous chunk [b0, b1)
  const int chunk = (N + nt - 1) / nt;
  const int b0 = min(N, tid * chunk), b1 = min(N, b0 + chunk);
  // case (1), and the last kept position of my chunk
  int last = -1;
  for (int s = b0; s < b1; s++) {
    int d1 = (rho == 0.0 || fabs(rho) * zn * fabs(e.zs[s]) <= tol) ? 1 : 0;
    e.defl[s] = d1;
    if (!d1) last = s;
  }
  // prefix max of "last kept" over chunks -> previous kept position before my chunk
  scnt[tid] = last;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    int v = tid >= off ? scnt[tid - off] : -1;
    __syncthreads();
    scnt[tid] = max(scnt[tid], v);
    __syncthreads();
  }
  int prev = tid > 0 ? scnt[tid - 1] : -1;
  __syncthreads();
  // Case (3) in parallel with the original values: pair (j, s) with j the previous kept
  // position.  e.idx holds j for every kept s and e.didx the candidate list (both are
  // scratch until the compaction below).  The sequential order only matters where a
  // rotation changed (d_j, z_j) of the left partner: one thread walks the candidates
  // and, after each rotation, the chain's next kept position.
  int ncand = 0;
  for (int s = b0; s < b1; s++) {
    if (e.defl[s]) continue;
    e.idx[s] = prev;
    if (prev >= 0) {
      double zj = e.zs[prev], zs = e.zs[s];
      double r = hypot(zj, zs);
      if (fabs((e.ds[s] - e.ds[prev]) * (zs / r) * (zj / r)) <= tol) ncand++;
    }
    prev = s;
  }
  scnt[tid] = ncand;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    int v = tid >= off ? scnt[tid - off] : 0;
    __syncthreads();
    scnt[tid] += v;
    __syncthreads();
  }
  if (tid == nt - 1) s_ncand = scnt[nt - 1];
  int cpos = scnt[tid] - ncand;
  for (int s = b0; s < b1; s++) {
    if (e.defl[s]) continue;
    int j = e.idx[s];
    if (j >= 0) {
      double zj = e.zs[j], zs = e.zs[s];
      double r = hypot(zj, zs);
      if (fabs((e.ds[s] - e.ds[j]) * (zs / r) * (zj / r)) <= tol) e.didx[cpos++] = s;
    }
  }
  __syncthreads();
  if (tid == 0) {
    const int nc = s_ncand;
    int nr = 0, c = 0;
    int s = nc > 0 ? e.didx[c++] : -1;
    while (s >= 0) {
      int j = e.idx[s];
      double zj = e.zs[j], zs = e.zs[s];
      double r = hypot(zj, zs);
      double cs = zs / r, sn = zj / r;
      double dj = e.ds[j], dsv = e.ds[s];
      int chain = -1;
      if (fabs((dsv - dj) * cs * sn) <= tol) {
        e.ds[j] = cs * cs * dj + sn * sn * dsv;
        e.ds[s] = sn * sn * dj + cs * cs * dsv;
        e.zs[j] = 0.0;
        e.zs[s] = r;
        e.defl[j] = 1;
        if (yvec) {
          double yj = yvec[j], ys = yvec[s];
          yvec[j] = cs * yj - sn * ys;
          yvec[s] = sn * yj + cs * ys;
        }
        e.rj[nr] = j; e.ri[nr] = s; e.rc[nr] = cs; e.rs[nr] = sn;
        nr++;
        int nx = s + 1;  // the next kept position now pairs with the rotated s
        while (nx < N && e.defl[nx]) nx++;
        if (nx < N) chain = nx;
      }
      while (c < nc && e.didx[c] <= s) c++;
      if (chain >= 0) s = chain;
      else s = (c < nc) ? e.didx[c++] : -1;
    }
    e.nrot[0] = nr;
  }
  __syncthreads();
  // compaction of the kept set
  int cnt = 0;
  for (int s = b0; s < b1; s++) cnt += !e.defl[s];
  scnt[tid] = cnt;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {  // inclusive Hillis-Steele scan
    int v = tid >= off ? scnt[tid - off] : 0;
    __syncthreads();
    scnt[tid] += v;
    __syncthreads();
  }
  int kk = scnt[nt - 1];
  int pos = scnt[tid] - cnt;       // kept entries before my chunk
  int dpos = b0 - pos;             // deflated entries before my chunk
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

void launch_deflate(cudaStream_t st, Eig e, double* yvec, int* status) {
  k_deflate<<<1, 1024, 0, st>>>(e, yvec, status);
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
    r.asum += fabs(t);
  }
  r.psiL = warp_sum(r.psiL);
  r.dpsiL = warp_sum(r.dpsiL);
  r.psiR = warp_sum(r.psiR);
  r.dpsiR = warp_sum(r.dpsiR);
  r.asum = warp_sum(r.asum);
  return r;
}

// One root in the rho > 0 orientation; returns 0 on convergence.
__device__ int secular_root(const double* __restrict__ dc, const double* __restrict__ z2c, int k,
                            double R, double zn2, int j, int lane, int maxit, int* o_out,
                            double* tau_out) {
  int o;
  double tau, lo, hi, aL, aR;
  SecSums sm;
  double w;
  const bool last = (j == k - 1);
  if (!last) {
    double gap = dc[j + 1] - dc[j];
    o = j;
    tau = 0.5 * gap;
    sm = secular_sums(dc, z2c, k, o, tau, j, lane);
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
    sm = secular_sums(dc, z2c, k, o, tau, j, lane);
    w = 1.0 + R * (sm.psiL + sm.psiR);
    if (w < 0.0) lo = tau; else hi = tau;
  }
  for (int it = 0; it < maxit; it++) {
    if (w == 0.0 || fabs(w) <= kU * (1.0 + R * sm.asum)) { *o_out = o; *tau_out = tau; return 0; }
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
    sm = secular_sums(dc, z2c, k, o, tau, last ? k - 1 : j, lane);
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
__global__ void k_secular(const double* __restrict__ dc, const double* __restrict__ z2c,
                          const int* __restrict__ kp, const double* __restrict__ rhop,
                          const double* __restrict__ dk, int* orgc, double* tauc, int* org,
                          double* tau, double* dorg, int* status, int maxit) {
  __shared__ double s_zn2;
  const int k = kp[0];
  const double rho = rhop[0];
  const double R = fabs(rho);
  if (threadIdx.x < 32) {
    double a = 0.0;
    for (int i = threadIdx.x; i < k; i += 32) a += z2c[i];
    a = warp_sum(a);
    if (threadIdx.x == 0) s_zn2 = a;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < k; j += warps) {
    int o;
    double t;
    int bad = secular_root(dc, z2c, k, R, s_zn2, j, lane, maxit, &o, &t);
    if (lane == 0) {
      if (bad) latch(status, SVDUP_ENOCONV);
      if (!isfinite(t)) latch(status, SVDUP_ENONFINITE);
      orgc[j] = o;
      tauc[j] = t;
      if (rho > 0.0) {
        org[j] = o;
        tau[j] = t;
        dorg[j] = dk[o];
      } else {
        int jj = k - 1 - j, oo = k - 1 - o;
        org[jj] = oo;
        tau[jj] = -t;
        dorg[jj] = dk[oo];
      }
    }
  }
}

static int secular_blocks(int N) {
  int warps = N;                   // one warp per root
  int blocks = (warps * 32 + 255) / 256;
  return blocks < 1 ? 1 : blocks;
}

void launch_secular(cudaStream_t st, Eig e, int* status, int maxit) {
  k_secular<<<secular_blocks(e.N), 256, 0, st>>>(e.dc, e.z2c, e.kp, e.rhop, e.dk, e.orgc, e.tauc,
                                                e.org, e.tau, e.dorg, status, maxit);
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
// index.  rank_root / rank_defl record where each one went.
// ---------------------------------------------------------------------------
__global__ void k_merge(Eig e) {
  const int N = e.N, k = e.kp[0], nd = N - k;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
    if (x < k) {
      int j = x;
      double mu = e.dorg[j] + e.tau[j];
      int c = 0;
      for (int t = 0; t < nd; t++) c += (e.ds[e.didx[t]] <= mu);
      int r = j + c;
      e.lam[r] = mu;
      e.rank_root[j] = r;
    } else {
      int t = x - k;
      int s = e.didx[t];
      double v = e.ds[s];
      int c = 0;
      for (int u = 0; u < nd; u++) {
        double w = e.ds[e.didx[u]];
        c += (w < v) || (w == v && u < t);
      }
      // roots strictly below v (binary search: roots ascending)
      int lo = 0, hi = k;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        double mu = e.dorg[mid] + e.tau[mid];
        if (mu < v) lo = mid + 1; else hi = mid;
      }
      int r = c + lo;
      e.lam[r] = v;
      e.rank_defl[s] = r;
    }
  }
}

void launch_merge(cudaStream_t st, Eig e) {
  k_merge<<<(e.N + 255) / 256, 256, 0, st>>>(e);
  SVDUP_COUNT_LAUNCH();
}

// ---------------------------------------------------------------------------
// z recomputed from the computed roots (Loewner): the characteristic polynomial gives
//   prod_j (mu_j - d_i) = R zhat_i^2 prod_{j != i} (d_j - d_i)        (rho > 0 form),
// so the Cauchy-like vectors of Sec. 3.2 built from zhat are the exact eigenvectors of
// a problem whose exact eigenvalues are the computed roots, and stay orthogonal.
// Each pole j != i is paired with an adjacent root so every factor lies in (0, 1):
//   j < i: (mu_j - d_i)/(d_j - d_i),  j > i: (mu_{j-1} - d_i)/(d_j - d_i),
// and the remaining root mu_{k-1} contributes (mu_{k-1} - d_i)/R.
// One warp per index i; differences mu_j - d_i come from the offsets.
// ---------------------------------------------------------------------------
__global__ void k_loewner(Eig e) {
  const int k = e.kp[0];
  const double rho = e.rhop[0];
  const double R = fabs(rho);
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const double* dc = e.dc;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < k; i += warps) {
    const double di = dc[i];
    double pr = 1.0;
    for (int j = lane; j < k; j += 32) {
      if (j == i) continue;
      int jr = (j < i) ? j : j - 1;
      double num = (dc[e.orgc[jr]] - di) + e.tauc[jr];
      double den = dc[j] - di;
      pr *= num * rcp64(den);
    }
    pr = warp_prod(pr);
    if (lane == 0) {
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
__global__ void k_norms(Eig e, const double* __restrict__ ysorted, double* out_final) {
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
      e.inv[j] = inv;
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

void launch_norms(cudaStream_t st, Eig e, const double* ysorted, double* out_final) {
  k_norms<<<secular_blocks(e.N), 256, 0, st>>>(e, ysorted, out_final);
  SVDUP_COUNT_LAUNCH();
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
__global__ void __launch_bounds__(1024) k_gather_rotate(Eig e, const double* __restrict__ xphys,
                                                        double* ysorted) {
  for (int s = threadIdx.x; s < e.N; s += blockDim.x) ysorted[s] = xphys[e.perm[s]];
  __syncthreads();
  if (threadIdx.x == 0) {
    int nr = e.nrot[0];
    for (int r = 0; r < nr; r++) {
      int a = e.rj[r], b = e.ri[r];
      double c = e.rc[r], sn = e.rs[r];
      double ya = ysorted[a], yb = ysorted[b];
      ysorted[a] = c * ya - sn * yb;
      ysorted[b] = sn * ya + c * yb;
    }
  }
}

void launch_apply_qt(cudaStream_t st, Eig e, const double* xphys, double* work, double* out_final) {
  k_gather_rotate<<<1, 1024, 0, st>>>(e, xphys, work);
  SVDUP_COUNT_LAUNCH();
  // k_norms recomputes inv (identical values); only the product is wanted here.
  launch_norms(st, e, work, out_final);
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

__global__ void __launch_bounds__(1024) k_unrotate_scatter(Eig e, double* vsorted, double* yphys) {
  if (threadIdx.x == 0) {
    int nr = e.nrot[0];
    for (int r = nr - 1; r >= 0; r--) {
      int a = e.rj[r], b = e.ri[r];
      double c = e.rc[r], sn = e.rs[r];
      double va = vsorted[a], vb = vsorted[b];
      vsorted[a] = c * va + sn * vb;
      vsorted[b] = -sn * va + c * vb;
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < e.N; s += blockDim.x) yphys[e.perm[s]] = vsorted[s];
}

void launch_apply_q(cudaStream_t st, Eig e, const double* xfinal, double* work, double* yphys) {
  k_apply_q_core<<<secular_blocks(e.N), 256, 0, st>>>(e, xfinal, work);
  SVDUP_COUNT_LAUNCH();
  k_unrotate_scatter<<<1, 1024, 0, st>>>(e, work, yphys);
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

}  // namespace svdup
