// svdup_vfmm.cu -- the far field of the solve's own Cauchy-like sums: Loewner's zhat
// (Sec. 3.2), the column norms ||c_j|| with the transposed product Q^T y (RankOneUpdate
// STEP 7, Eq. CTildeFinalForm1) and the product Q x, by App. D's interpolation FMM
// applied to a single vector.  Summed directly, each is O(k^2) work on the FP64 pipe; here only
// the near leaves are summed directly and the rest goes through Chebyshev expansions
// (App. D STEPs 5-9) over a hierarchy of boxes.
//
// Geometry, in the solver's rho > 0 orientation (poles d_0 < ... < d_{k-1}; root mu_j
// in (d_j, d_{j+1}) for j < k - 1, mu_{k-1} > d_{k-1}): leaves of kVfLeaf consecutive
// indices, the last taking the remainder (so every leaf holds kVfLeaf .. 2 kVfLeaf - 1);
// box i of level h holds leaves [i 2^h, (i + 1) 2^h).  Boxes i, j of one level are well
// separated when |i - j| >= 2 and the gap between their intervals is at least the larger
// radius (the FP64 product's rule, svdup_tree.cu); a pair is listed at the coarsest
// level where it is well separated, so every leaf pair is either near (summed directly)
// or under exactly one listed pair.
//
// Loewner (rho > 0 form):
//   log zhat_i^2 = sum_{j<i} log((mu_j - d_i)/(d_j - d_i))
//                + sum_{j>i} log((mu_{j-1} - d_i)/(d_j - d_i)) + log((mu_{k-1} - d_i)/|rho|).
// Each log is an integral of the Cauchy kernel over the interval between a pole and the
// root it is paired with:
//   j < i:  log((mu_j - x)/(d_j - x))      =  int_{d_j}^{mu_j} ds / (s - x),
//   j > i:  log((mu_{j-1} - x)/(d_j - x))  = -int_{mu_{j-1}}^{d_j} ds / (s - x),
// so a source box acts on targets to its right through its "L" charge (unit density on
// [d_j, mu_j], j in the box) and on targets to its left through its "R" charge (on
// [mu_{j-1}, d_j]), each a Cauchy potential.  The near leaves' factors are multiplied
// directly as in the direct kernel; the far sum is exponentiated.  It is at least
// -log(3) per listed box (a box's factors telescope), so exp() stays far from underflow.
// Norms: ||c_j||^2 = sum_t zhat_t^2 / (d_t - mu_j)^2 (kernel 1/(s - x)^2, point charges
// zhat_t^2 at the poles, targets the roots); Q^T y: sum_t zhat_t y_t / (d_t - mu_j)
// (kernel 1/(s - x)).  The last root, beyond every pole, is summed directly, each leaf
// adding its own poles' terms.  Q x (the sign pairing's product): zhat_t sum_j w_j /
// (d_t - mu_j), w_j = x_j / ||c_j|| (point charges at the roots, targets the poles; the
// last root's term added directly to every target).
//
// Expansions: kVfP = 28 first-kind Chebyshev nodes per box.  A source box's charges are
// interpolated onto its nodes (STEP 5: the weight of node b is the Lagrange basis u_b
// integrated against the charge), through the Chebyshev series
//   u_b(t) = (1 + 2 sum_{m>=1} T_m(t_b) T_m(t)) / P,
// so only the charge moments D_m = int T_m (an interval) or q T_m(t) (a point) are summed
// per charge.  An interval's integrals come from the differences dT_m = T_m(t_a + D) -
// T_m(t_a), run by their own recurrence so that they keep the relative accuracy of the
// interval's length D:
//   int_{t_a}^{t_a + D} T_m = (dT_{m+1}/(m+1) - dT_{m-1}/(m-1)) / 2,
//   dT_{m+1} = 2 ((t_a + D) dT_m + D T_m(t_a)) - dT_{m-1}.
// A parent's moments take its children's node weights as point charges (STEP 6).  The
// translation (STEP 8, T operators) evaluates the kernel between the two boxes' nodes
// with every coordinate a difference from a box centre, so a box far narrower than the
// ulp of its position keeps its accuracy.  The local values of every level are
// interpolated onto the leaf nodes (STEP 8's S operators, taken from each level straight
// to the leaves), then onto the targets (STEP 9), by the barycentric formula, whose
// rounding does not grow towards the box ends as a Chebyshev-series evaluation's does.
// Truncation: an admissible pair puts the other box's singularities at least two radii
// from the interpolating box's centre, inside the Bernstein ellipse of parameter 2 +
// sqrt 3; the error decays as (2 + sqrt 3)^-P, 1e-16 at P = 28.
#include <cuda_runtime.h>

#include "svdup_internal.cuh"

namespace svdup {

namespace {

constexpr int P = kVfP;
constexpr int kLeafMax = 2 * kVfLeaf;  // a leaf holds fewer indices than this
constexpr int kMaxLevels = 32;

enum { PROB_LOEWNER = 0, PROB_NORMS = 1, PROB_APPLYQ = 2 };

// The device view of Eig::vf / Eig::vfc for the current k.
struct Vf {
  int k, nb, H, Lmax, tot;
  double* geo;   // per box: source centre, radius, target centre, radius
  double* W;     // per box: 2 sets x P node weights of the charges
  double* psi;   // per part and box: 2 sets x P partial local values at its target nodes
  double* loc;   // per leaf: 2 sets x P local values, every level summed
  double* last;  // per leaf: its poles' terms of the last root's two sums
  double* tab;   // P Chebyshev nodes, then P barycentric weights
  int* cnt;      // per box: arrival counter (entry 0: the last root's sums)
  int* near;     // per leaf: the count, then up to kVfNearMax near leaves
};

__device__ __forceinline__ int nb_at(int nb, int h) { return (nb + (1 << h) - 1) >> h; }

__device__ __forceinline__ Vf vf_view(const Eig& e, int k) {
  Vf v;
  v.k = k;
  v.nb = max(1, k / kVfLeaf);
  v.Lmax = vf_lmax(e.N);
  const int Hmax = tree_levels(v.Lmax);
  v.tot = tree_off(v.Lmax, Hmax);
  int h = 1;
  while (h < Hmax && nb_at(v.nb, h - 1) > 2) h++;
  v.H = h;
  v.tab = e.vf;
  v.geo = v.tab + 2 * P;
  v.W = v.geo + 4 * (size_t)v.tot;
  v.psi = v.W + 2 * (size_t)P * v.tot;
  v.loc = v.psi + 2 * (size_t)P * v.tot * kVfParts;
  v.last = v.loc + 2 * (size_t)P * (v.Lmax + 1);
  v.cnt = e.vfc;
  v.near = e.vfc + v.tot;
  return v;
}

__device__ __forceinline__ int box_id(const Vf& v, int h, int i) { return tree_off(v.Lmax, h) + i; }
__device__ __forceinline__ int leaf_lo(int b) { return b * kVfLeaf; }
__device__ __forceinline__ int leaf_hi(const Vf& v, int b) {
  return b == v.nb - 1 ? v.k : (b + 1) * kVfLeaf;
}

// Source box i and target box j of level h are well separated.
__device__ __forceinline__ bool vf_adm(const Vf& v, int h, int i, int j) {
  if (h >= v.H) return false;
  const int n = nb_at(v.nb, h);
  if (i < 0 || j < 0 || i >= n || j >= n) return false;
  if (i - j < 2 && j - i < 2) return false;
  const double* gs = v.geo + 4 * (size_t)box_id(v, h, i);
  const double* gt = v.geo + 4 * (size_t)box_id(v, h, j);
  const double rs = gs[1], rt = gt[3];
  return fabs(gs[0] - gt[2]) - rs - rt >= fmax(rs, rt);
}

// Some ancestor pair above level h is well separated.
__device__ __forceinline__ bool vf_covered_above(const Vf& v, int h, int i, int j) {
  for (int q = h + 1; q < v.H; q++) {
    i >>= 1;
    j >>= 1;
    if (vf_adm(v, q, i, j)) return true;
  }
  return false;
}

// The pair is in target box j's interaction list at level h: well separated, and no
// ancestor pair is.  (In exact arithmetic the children of a well-separated pair are well
// separated, so this is "its parents are not"; asking it of every ancestor keeps each
// leaf pair under at most one listed pair whatever the rounding of the tests.)
__device__ __forceinline__ bool vf_listed(const Vf& v, int h, int i, int j) {
  return vf_adm(v, h, i, j) && !vf_covered_above(v, h, i, j);
}

// Source leaf i is in target leaf l's near field: no pair of their ancestors is listed.
__device__ __forceinline__ bool vf_near(const Vf& v, int i, int l) {
  return !vf_adm(v, 0, i, l) && !vf_covered_above(v, 0, i, l);
}

// row[m] = r * int_{ta}^{ta + dl} T_m(t) dt, m < P (an interval charge of unit density in
// a box of radius r; dl is the interval's length over r).
__device__ __forceinline__ void interval_row(double ta, double dl, double r, double* row) {
  const double tb = ta + dl;
  row[0] = r * dl;
  row[1] = (r * dl) * (ta + 0.5 * dl);
  double Tp = 1.0, Tc = ta;   // T_{m-1}(ta), T_m(ta)
  double dp = 0.0, dq = dl;   // dT_{m-1}, dT_m
#pragma unroll
  for (int m = 1; m < P; m++) {
    const double dn = 2.0 * fma(tb, dq, dl * Tc) - dp;  // dT_{m+1}
    if (m >= 2) row[m] = (0.5 * r) * (dn * (1.0 / (m + 1)) - dp * (1.0 / (m - 1)));
    const double Tn = 2.0 * ta * Tc - Tp;
    Tp = Tc;
    Tc = Tn;
    dp = dq;
    dq = dn;
  }
}

// row[m] = T_m(t), m < P (a point charge; its weight is applied in the sum).
__device__ __forceinline__ void point_row(double t, double* row) {
  row[0] = 1.0;
  double Tp = 1.0, Tc = t;
#pragma unroll
  for (int m = 1; m < P; m++) {
    row[m] = Tc;
    const double Tn = 2.0 * t * Tc - Tp;
    Tp = Tc;
    Tc = Tn;
  }
}

// Node weights W_b = (D_0 + 2 sum_{m>=1} T_m(t_b) D_m) / P of box x from its moments
// sD (two sets); threads tid < 2P, (set, node) = (tid / P, tid % P).
__device__ __forceinline__ void weights_from_moments(const Vf& v, int x, const double (*sD)[P + 1],
                                                     const double* st) {
  const int tid = threadIdx.x;
  if (tid >= 2 * P) return;
  const int s = tid / P, b = tid - s * P;
  const double tb = st[b];
  double Tp = 1.0, Tc = tb, acc = 0.0;
  for (int m = 1; m < P; m++) {
    acc = fma(Tc, sD[s][m], acc);
    const double Tn = 2.0 * tb * Tc - Tp;
    Tp = Tc;
    Tc = Tn;
  }
  v.W[((size_t)2 * x + s) * P + b] = (sD[s][0] + 2.0 * acc) * (1.0 / P);
}

// Leaves: geometry and charge weights (STEP 5); then the upward pass (STEP 6): the
// second child of a parent to finish (an arrival counter) computes the parent, and so on
// up the levels, so no block waits for another.  Each charge's P moments go to a row of
// shared memory and thread (set, m) sums column m over the rows in order.
template <int PROB>
__global__ void __launch_bounds__(128) k_vf_leaf(Eig e, int kmin, const double* __restrict__ ysorted) {
  const int k = e.kp[0];
  if (k < kmin) return;
  const Vf v = vf_view(e, k);
  int i = blockIdx.x;
  if (i >= v.nb) return;
  __shared__ double st[P];
  __shared__ double sg[4];
  __shared__ double rows[kLeafMax][P + 1];
  __shared__ double wq[2][kLeafMax];
  __shared__ double sD[2][P + 1];
  __shared__ int s_go;
  const int tid = threadIdx.x;
  const int sm = tid / P, mm = tid - sm * P;  // (set, moment) of threads tid < 2P
  const double* __restrict__ dc = e.dc;
  const int* __restrict__ orgc = e.orgc;
  const double* __restrict__ tauc = e.tauc;
  const double rho = e.rhop[0];
  if (tid < P) {
    st[tid] = cheb_node(tid, P);
    if (i == 0) {  // the node and weight table for the other kernels
      const double th = (2.0 * tid + 1.0) / (2.0 * P);
      v.tab[tid] = st[tid];
      v.tab[P + tid] = (tid & 1 ? -1.0 : 1.0) * sinpi(th);
    }
  }
  const int j0 = leaf_lo(i), j1 = leaf_hi(v, i);
  if (tid == 0) {
    double slo, shi, tlo, thi;
    if (PROB == PROB_LOEWNER) {  // sources: the intervals [mu_{j0-1}, mu_{j1-1}]; targets: poles
      slo = j0 > 0 ? dc[orgc[j0 - 1]] + tauc[j0 - 1] : dc[0];
      shi = j1 < k ? dc[orgc[j1 - 1]] + tauc[j1 - 1] : dc[k - 1];
      tlo = dc[j0];
      thi = dc[j1 - 1];
    } else if (PROB == PROB_NORMS) {  // sources: poles; targets: the roots but the last
      const int jt = min(j1, k - 1) - 1;
      slo = dc[j0];
      shi = dc[j1 - 1];
      tlo = dc[orgc[j0]] + tauc[j0];
      thi = dc[orgc[jt]] + tauc[jt];
    } else {  // sources: the roots but the last; targets: poles
      const int jt = min(j1, k - 1) - 1;
      slo = dc[orgc[j0]] + tauc[j0];
      shi = dc[orgc[jt]] + tauc[jt];
      tlo = dc[j0];
      thi = dc[j1 - 1];
    }
    sg[0] = 0.5 * (slo + shi);
    sg[1] = 0.5 * (shi - slo);
    sg[2] = 0.5 * (tlo + thi);
    sg[3] = 0.5 * (thi - tlo);
    double* g = v.geo + 4 * (size_t)box_id(v, 0, i);
    for (int q = 0; q < 4; q++) g[q] = sg[q];
  }
  __syncthreads();
  const int nc = j1 - j0;  // < kLeafMax
  const double c = sg[0], r = sg[1], ir = 1.0 / r;
  double acc = 0.0;
  if (PROB == PROB_LOEWNER) {
    // pass 0: the L charges [d_j, mu_j] (set 0); pass 1: the R charges [mu_{j-1}, d_j]
    // (set 1).  The L charge of the last pole and the R charge of the first act on no
    // target and are left out.
    for (int pass = 0; pass < 2; pass++) {
      for (int q = tid; q < nc; q += blockDim.x) {
        const int j = j0 + q;
        double* row = rows[q];
        if (pass == 0 ? j == k - 1 : j == 0) {
          for (int m = 0; m < P; m++) row[m] = 0.0;
        } else if (pass == 0) {
          const int o = orgc[j];
          const double len = (o == j ? 0.0 : dc[o] - dc[j]) + tauc[j];  // mu_j - d_j
          interval_row((dc[j] - c) * ir, len * ir, r, row);
        } else {
          const int o = orgc[j - 1];
          const double len = (o == j ? 0.0 : dc[j] - dc[o]) - tauc[j - 1];  // d_j - mu_{j-1}
          interval_row(((dc[o] - c) + tauc[j - 1]) * ir, len * ir, r, row);
        }
      }
      __syncthreads();
      if (tid < 2 * P && sm == pass)
        for (int q = 0; q < nc; q++) acc += rows[q][mm];
      __syncthreads();
    }
  } else if (PROB == PROB_NORMS) {
    const double sgn = rho > 0.0 ? 1.0 : -1.0;
    for (int q = tid; q < nc; q += blockDim.x) {
      const int j = j0 + q;
      const int io = rho > 0.0 ? j : k - 1 - j;
      const double zh = e.zhat[io];
      wq[0][q] = zh * zh;
      wq[1][q] = ysorted ? sgn * zh * ysorted[e.idx[io]] : 0.0;
      point_row((dc[j] - c) * ir, rows[q]);
    }
    __syncthreads();
    if (tid < 2 * P)
      for (int q = 0; q < nc; q++) acc = fma(wq[sm][q], rows[q][mm], acc);
  } else {
    // Q x: charges w_j = x_j / ||c_j|| at the roots (ysorted holds x in the final order),
    // with the sign that makes the far field sgn * sum_j w_j / (d_t - mu_j) in the
    // rho > 0 orientation; the last root acts directly on every target
    const double sgn = rho > 0.0 ? 1.0 : -1.0;
    for (int q = tid; q < nc; q += blockDim.x) {
      const int j = j0 + q;
      wq[1][q] = 0.0;
      if (j == k - 1) {
        wq[0][q] = 0.0;
        point_row(0.0, rows[q]);
      } else {
        const int io = rho > 0.0 ? j : k - 1 - j;
        wq[0][q] = -sgn * e.inv[io] * ysorted[e.rank_root[io]];
        point_row(((dc[orgc[j]] - c) + tauc[j]) * ir, rows[q]);
      }
    }
    __syncthreads();
    if (tid < 2 * P)
      for (int q = 0; q < nc; q++) acc = fma(wq[sm][q], rows[q][mm], acc);
  }
  if (tid < 2 * P) sD[sm][mm] = acc;
  __syncthreads();
  weights_from_moments(v, box_id(v, 0, i), sD, st);
  __threadfence();
  __syncthreads();
  for (int h = 0; h + 1 < v.H; h++, i >>= 1) {
    const int par = i >> 1;
    const int nch = min(2, nb_at(v.nb, h) - 2 * par);
    const int xp = box_id(v, h + 1, par);
    if (nch == 2) {
      if (tid == 0) {
        const int t = atomicAdd(v.cnt + xp, 1);
        s_go = t;
        if (t == 1) v.cnt[xp] = 0;  // both children in: ready for the next use
      }
      __syncthreads();
      if (s_go == 0) return;  // the sibling computes the parent
      __threadfence();
    }
    const int xc = box_id(v, h, 2 * par);
    if (tid == 0) {
      double slo = 0.0, shi = 0.0, tlo = 0.0, thi = 0.0;
      for (int q = 0; q < nch; q++) {
        const double* g = v.geo + 4 * (size_t)(xc + q);
        const double cs = __ldcg(g), rs = __ldcg(g + 1), ct = __ldcg(g + 2), rt = __ldcg(g + 3);
        slo = q ? fmin(slo, cs - rs) : cs - rs;
        shi = q ? fmax(shi, cs + rs) : cs + rs;
        tlo = q ? fmin(tlo, ct - rt) : ct - rt;
        thi = q ? fmax(thi, ct + rt) : ct + rt;
      }
      sg[0] = 0.5 * (slo + shi);
      sg[1] = 0.5 * (shi - slo);
      sg[2] = 0.5 * (tlo + thi);
      sg[3] = 0.5 * (thi - tlo);
      double* g = v.geo + 4 * (size_t)xp;
      for (int q = 0; q < 4; q++) g[q] = sg[q];
    }
    __syncthreads();
    // the children's node weights as point charges in the parent
    const int ncp = nch * P;
    if (tid < ncp) {
      const int q = tid / P, b = tid - q * P;
      const double* g = v.geo + 4 * (size_t)(xc + q);
      const double cs = __ldcg(g), rs = __ldcg(g + 1);
      wq[0][tid] = __ldcg(v.W + ((size_t)2 * (xc + q)) * P + b);
      wq[1][tid] = __ldcg(v.W + ((size_t)2 * (xc + q) + 1) * P + b);
      point_row(((cs - sg[0]) + rs * st[b]) / sg[1], rows[tid]);
    }
    __syncthreads();
    if (tid < 2 * P) {
      double a = 0.0;
      for (int q = 0; q < ncp; q++) a = fma(wq[sm][q], rows[q][mm], a);
      sD[sm][mm] = a;
    }
    __syncthreads();
    weights_from_moments(v, xp, sD, st);
    __threadfence();
    __syncthreads();
  }
}

// Translations (STEP 8): one warp per (target box of any level, part); the part takes
// every kVfParts-th entry of the box's interaction list, and lane a < P holds the partial
// local value at node a.  Loewner: the L charge of boxes to the left, minus the R charge
// of boxes to the right, kernel 1/(s - x).  Norms: set 0 with 1/(s - x)^2, set 1 (Q^T y,
// when nsets = 2) with 1/(s - x).
template <int PROB>
__global__ void __launch_bounds__(32) k_vf_m2l(Eig e, int kmin, int nsets) {
  const int k = e.kp[0];
  if (k < kmin) return;
  const Vf v = vf_view(e, k);
  const int x = blockIdx.x / kVfParts, part = blockIdx.x - x * kVfParts;
  const int lane = threadIdx.x;
  if (x >= v.tot) return;
  int h = 0;
  while (h + 1 < v.H && x >= tree_off(v.Lmax, h + 1)) h++;
  const int j = x - tree_off(v.Lmax, h);
  const int n = nb_at(v.nb, h);
  if (j >= n) return;  // (boxes above the levels in use land here too)
  __shared__ double st[P];
  if (lane < P) st[lane] = v.tab[lane];
  __syncwarp();
  const double ct = v.geo[4 * (size_t)x + 2], rt = v.geo[4 * (size_t)x + 3];
  const double ta = st[lane < P ? lane : 0];
  double a0 = 0.0, a1 = 0.0;
  int seen = 0;
  for (int i0 = 0; i0 < n; i0 += 32) {
    unsigned bal = __ballot_sync(0xffffffffu, vf_listed(v, h, i0 + lane, j));
    while (bal) {
      const int is = i0 + __ffs(bal) - 1;
      bal &= bal - 1;
      if (seen++ % kVfParts != part) continue;
      const int xs = box_id(v, h, is);
      const double cs = v.geo[4 * (size_t)xs], rs = v.geo[4 * (size_t)xs + 1];
      const double base = (cs - ct) - rt * ta;  // s - x = base + rs t_b
      const int set = PROB == PROB_LOEWNER ? (is < j ? 0 : 1) : 0;
      const double w0 = lane < P ? v.W[((size_t)2 * xs + set) * P + lane] : 0.0;
      const double w1 = (PROB == PROB_NORMS && lane < P) ? v.W[((size_t)2 * xs + 1) * P + lane] : 0.0;
      double s0 = 0.0, s1 = 0.0;
      for (int b = 0; b < P; b++) {
        const double q0 = __shfl_sync(0xffffffffu, w0, b);
        const double rr = rcp64(fma(rs, st[b], base));
        if (PROB != PROB_NORMS) {
          s0 = fma(q0, rr, s0);
        } else {
          s0 = fma(q0, rr * rr, s0);
          if (nsets > 1) s1 = fma(__shfl_sync(0xffffffffu, w1, b), rr, s1);
        }
      }
      if (PROB == PROB_LOEWNER) a0 += set == 0 ? s0 : -s0;
      else if (PROB == PROB_APPLYQ) a0 += s0;
      else { a0 += s0; a1 += s1; }
    }
  }
  if (lane < P) {
    double* out = v.psi + ((size_t)part * v.tot + x) * 2 * P;
    out[lane] = a0;
    out[P + lane] = a1;
  }
}

// Barycentric interpolation at t of the values f_c held by lanes c < P (every lane
// passes its own t; lane c's value arrives by shuffle).  Nodes and weights in shared
// memory; a node hit exactly returns its value.
__device__ __forceinline__ double bary_lane(double f, double t, const double* st, const double* sw) {
  double num = 0.0, den = 0.0, hitv = 0.0;
  bool hit = false;
  for (int c = 0; c < P; c++) {
    const double fc = __shfl_sync(0xffffffffu, f, c);
    const double df = t - st[c];
    if (df == 0.0) {
      hit = true;
      hitv = fc;
    }
    const double q = df == 0.0 ? 0.0 : sw[c] * rcp64(df);
    num = fma(q, fc, num);
    den += q;
  }
  return hit ? hitv : num * rcp64(den);
}

// The downward pass (STEP 8, S operators): every level's local values (its parts summed
// in order) interpolated onto the leaf's nodes and summed in level order; and the leaf's
// near list.  One block per leaf, warp h for level h.
__global__ void k_vf_down(Eig e, int kmin, int nsets) {
  const int k = e.kp[0];
  if (k < kmin) return;
  const Vf v = vf_view(e, k);
  const int l = blockIdx.x;
  if (l >= v.nb) return;
  __shared__ double st[P], sw[P];
  __shared__ double part[kMaxLevels][2][P];
  if (threadIdx.x < P) {
    st[threadIdx.x] = v.tab[threadIdx.x];
    sw[threadIdx.x] = v.tab[P + threadIdx.x];
  }
  __syncthreads();
  const int h = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (h < v.H) {
    const int xl = box_id(v, 0, l), x = box_id(v, h, l >> h);
    for (int s = 0; s < nsets; s++) {
      double f = 0.0;
      if (lane < P)
        for (int q = 0; q < kVfParts; q++) f += v.psi[(((size_t)q * v.tot + x) * 2 + s) * P + lane];
      double val = f;
      if (h > 0) {
        const double ctl = v.geo[4 * (size_t)xl + 2], rtl = v.geo[4 * (size_t)xl + 3];
        const double cth = v.geo[4 * (size_t)x + 2], rth = v.geo[4 * (size_t)x + 3];
        const double t = fma(rtl, st[lane < P ? lane : 0], ctl - cth) / rth;
        val = bary_lane(f, t, st, sw);
      }
      if (lane < P) part[h][s][lane] = val;
    }
  }
  if (h == 0) {  // the near leaves, in order
    int* nl = v.near + (size_t)l * (kVfNearMax + 1);
    int n = 0;
    for (int i0 = 0; i0 < v.nb; i0 += 32) {
      const int i = i0 + lane;
      const bool f = i < v.nb && vf_near(v, i, l);
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      const int pos = n + __popc(bal & ((1u << lane) - 1u));
      if (f && pos < kVfNearMax) nl[1 + pos] = i;
      n += __popc(bal);
    }
    if (lane == 0) nl[0] = n;
  }
  __syncthreads();
  if (threadIdx.x < nsets * P) {
    const int s = threadIdx.x / P, a = threadIdx.x - s * P;
    double acc = 0.0;
    for (int q = 0; q < v.H; q++) acc += part[q][s][a];
    v.loc[((size_t)2 * l + s) * P + a] = acc;
  }
}

// Barycentric interpolation at one t of values in shared memory, by a whole warp (lanes
// c < P take node c).
__device__ __forceinline__ double bary_warp(const double* f, double t, const double* st,
                                            const double* sw, int lane) {
  double num = 0.0, den = 0.0;
  int hit = 0;
  if (lane < P) {
    const double df = t - st[lane];
    if (df == 0.0) hit = 1;
    const double q = df == 0.0 ? 0.0 : sw[lane] * rcp64(df);
    num = q * f[lane];
    den = q;
  }
  const unsigned hb = __ballot_sync(0xffffffffu, hit);
  num = warp_sum(num);
  den = warp_sum(den);
  return hb ? f[__ffs(hb) - 1] : num * rcp64(den);
}

// Loewner's near factors of target i (pole x = d_i) over poles [a, b), i excluded, into
// the running product pn 2^en / (pd 2^ed).
__device__ __forceinline__ void loewner_near(const double* __restrict__ dc,
                                             const int* __restrict__ orgc,
                                             const double* __restrict__ tauc, int a, int b,
                                             int i, double x, int lane, double& pn, int& en,
                                             double& pd, int& ed) {
  for (int j = a + lane; j < b; j += 32) {
    if (j == i) continue;
    const int jr = j < i ? j : j - 1;
    pn *= (dc[orgc[jr]] - x) + tauc[jr];
    pd *= dc[j] - x;
    renorm64(pn, en);
    renorm64(pd, ed);
  }
}

// Norm sums of root (dO + tau) over poles [a, b): zhat_t^2 / delta^2 and zhat_t y_t / delta.
__device__ __forceinline__ void norms_near(const Eig& e, const double* __restrict__ ysorted,
                                           int a, int b, int k, double rho, double dO, double tj,
                                           int lane, double& s2, double& sy) {
  const double sgn = rho > 0.0 ? 1.0 : -1.0;
  for (int t = a + lane; t < b; t += 32) {
    const int io = rho > 0.0 ? t : k - 1 - t;
    const double c = e.zhat[io] * rcp64((e.dc[t] - dO) - tj);
    s2 = fma(c, c, s2);
    if (ysorted) sy = fma(c, sgn * ysorted[e.idx[io]], sy);
  }
}

// Q x's near terms of target pole x = d_t over roots [a, b): sum_j w_j / (d_t - mu_j)
// (rho > 0 orientation, offsets from the roots' poles), w_j = x_j / ||c_j||.
__device__ __forceinline__ double applyq_near(const Eig& e, const double* __restrict__ xfinal,
                                              int a, int b, int k, double rho, double x,
                                              int lane) {
  double acc = 0.0;
  for (int j = a + lane; j < b; j += 32) {
    const int io = rho > 0.0 ? j : k - 1 - j;
    const double w = e.inv[io] * xfinal[e.rank_root[io]];
    acc = fma(w, rcp64((x - e.dc[e.orgc[j]]) - e.tauc[j]), acc);
  }
  return acc;
}

// Targets (STEP 9 and the near field, STEP 10): one warp per target, kLeafMax blocks per
// leaf (those past the leaf's targets return).  Loewner writes zhat; the norms write inv
// (unless keep_inv) and out_final[rank] = (Q^T y)_j when ysorted is given.  Each leaf's
// first target's warp also sums its poles' terms of the last root, and the last of them to
// finish adds the parts up in leaf order and writes that root.
template <int PROB>
__global__ void __launch_bounds__(32) k_vf_eval(Eig e, int kmin, const double* __restrict__ ysorted,
                                                double* __restrict__ out_final, int keep_inv) {
  const int k = e.kp[0];
  if (k < kmin) return;
  const Vf v = vf_view(e, k);
  const int l = blockIdx.x / kLeafMax, tq = blockIdx.x - l * kLeafMax;
  if (l >= v.nb) return;
  const int j0 = leaf_lo(l), j1 = leaf_hi(v, l);
  const int tend = PROB == PROB_NORMS ? min(j1, k - 1) : j1;
  const int j = j0 + tq;
  if (j >= tend) return;
  __shared__ double st[P], sw[P], loc0[P], loc1[P];
  __shared__ int snear[kVfNearMax];
  __shared__ int s_go;
  const int lane = threadIdx.x;
  const double* __restrict__ dc = e.dc;
  const int* __restrict__ orgc = e.orgc;
  const double* __restrict__ tauc = e.tauc;
  const double rho = e.rhop[0];
  const int* nl = v.near + (size_t)l * (kVfNearMax + 1);
  const int nn = nl[0];
  if (lane < P) {
    st[lane] = v.tab[lane];
    sw[lane] = v.tab[P + lane];
    loc0[lane] = v.loc[((size_t)2 * l) * P + lane];
    loc1[lane] = v.loc[((size_t)2 * l + 1) * P + lane];
  }
  for (int q = lane; q < min(nn, kVfNearMax); q += 32) snear[q] = nl[1 + q];
  __syncwarp();
  const int x = box_id(v, 0, l);
  const double ct = v.geo[4 * (size_t)x + 2], rt = v.geo[4 * (size_t)x + 3];
  const double R = fabs(rho);
  const int io = rho > 0.0 ? j : k - 1 - j;
  const bool all = nn > kVfNearMax;  // every pole near: the direct sums alone
  if (PROB == PROB_APPLYQ) {
    const double xi = dc[j];
    const double sgn = rho > 0.0 ? 1.0 : -1.0;
    const double far = all ? 0.0 : bary_warp(loc0, (xi - ct) / rt, st, sw, lane);
    double acc = 0.0;
    if (all) {
      acc = applyq_near(e, ysorted, 0, k - 1, k, rho, xi, lane);
    } else {
      for (int q = 0; q < nn; q++) {
        const int L = snear[q];
        acc += applyq_near(e, ysorted, leaf_lo(L), min(leaf_hi(v, L), k - 1), k, rho, xi, lane);
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      const int il = rho > 0.0 ? k - 1 : 0;  // the last root, directly
      acc += e.inv[il] * ysorted[e.rank_root[il]] *
             rcp64((xi - dc[orgc[k - 1]]) - tauc[k - 1]);
      out_final[e.idx[io]] = e.zhat[io] * (far + sgn * acc);
    }
  } else if (PROB == PROB_LOEWNER) {
    const double xi = dc[j];
    const double far = all ? 0.0 : bary_warp(loc0, (xi - ct) / rt, st, sw, lane);
    double pn = 1.0, pd = 1.0;
    int en = 0, ed = 0;
    const bool direct = all || !(far > -600.0);  // (the second is not met in practice)
    if (direct) {
      loewner_near(dc, orgc, tauc, 0, k, j, xi, lane, pn, en, pd, ed);
    } else {
      for (int q = 0; q < nn; q++) {
        const int L = snear[q];
        loewner_near(dc, orgc, tauc, leaf_lo(L), leaf_hi(v, L), j, xi, lane, pn, en, pd, ed);
      }
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
      const int sx = en - ed, hx = sx / 2;
      double pr = (pn / pd) * ldexp(1.0, hx) * ldexp(1.0, sx - hx);
      if (!direct) pr *= exp(far);
      pr *= ((dc[orgc[k - 1]] - xi) + tauc[k - 1]) / R;
      const double mag = sqrt(fmax(pr, 0.0));
      e.zhat[io] = (e.zk[io] < 0.0) ? -mag : mag;
    }
  } else {
    const double dO = dc[orgc[j]], tj = tauc[j];
    double f0 = 0.0, f1 = 0.0;
    if (!all) {
      const double t = ((dO - ct) + tj) / rt;
      f0 = bary_warp(loc0, t, st, sw, lane);
      if (ysorted) f1 = bary_warp(loc1, t, st, sw, lane);
    }
    double s2 = 0.0, sy = 0.0;
    if (all) {
      norms_near(e, ysorted, 0, k, k, rho, dO, tj, lane, s2, sy);
    } else {
      for (int q = 0; q < nn; q++) {
        const int L = snear[q];
        norms_near(e, ysorted, leaf_lo(L), leaf_hi(v, L), k, rho, dO, tj, lane, s2, sy);
      }
    }
    s2 = warp_sum(s2);
    sy = warp_sum(sy);
    if (lane == 0) {
      const double inv = 1.0 / sqrt(f0 + s2);
      if (!keep_inv) e.inv[io] = inv;
      if (ysorted) out_final[e.rank_root[io]] = (f1 + sy) * inv;
    }
    if (tq == 0) {
      // the last root: this leaf's poles' terms, then (last leaf to finish) the sum
      const int jl = k - 1;
      const double dL = dc[orgc[jl]], tL = tauc[jl];
      double p2 = 0.0, py = 0.0;
      norms_near(e, ysorted, j0, j1, k, rho, dL, tL, lane, p2, py);
      p2 = warp_sum(p2);
      py = warp_sum(py);
      if (lane == 0) {
        v.last[2 * (size_t)l] = p2;
        v.last[2 * (size_t)l + 1] = py;
        __threadfence();
        const int t = atomicAdd(v.cnt, 1);
        s_go = t == v.nb - 1;
        if (s_go) v.cnt[0] = 0;
      }
      __syncwarp();
      if (s_go) {
        __threadfence();
        double a2 = 0.0, ay = 0.0;
        for (int q = lane; q < v.nb; q += 32) {
          a2 += __ldcg(v.last + 2 * (size_t)q);
          ay += __ldcg(v.last + 2 * (size_t)q + 1);
        }
        a2 = warp_sum(a2);
        ay = warp_sum(ay);
        if (lane == 0) {
          const int iol = rho > 0.0 ? jl : 0;
          const double inv = 1.0 / sqrt(a2);
          if (!keep_inv) e.inv[iol] = inv;
          if (ysorted) out_final[e.rank_root[iol]] = ay * inv;
        }
      }
    }
  }
}

template <int PROB>
void vf_run(cudaStream_t st, Eig e, int kmin, const double* ysorted, double* out_final,
            bool keep_inv) {
  if (!e.vf || e.N < kmin) return;
  const int Lmax = vf_lmax(e.N), Hmax = tree_levels(Lmax), tot = vf_tot(e.N);
  const int nsets = PROB == PROB_NORMS ? (ysorted ? 2 : 1) : 1;
  cudaMemsetAsync(e.vfc, 0, sizeof(int) * (size_t)tot, st);
  k_vf_leaf<PROB><<<Lmax + 1, 128, 0, st>>>(e, kmin, ysorted);
  SVDUP_COUNT_LAUNCH();
  k_vf_m2l<PROB><<<tot * kVfParts, 32, 0, st>>>(e, kmin, nsets);
  SVDUP_COUNT_LAUNCH();
  k_vf_down<<<Lmax + 1, 32 * (Hmax < kMaxLevels ? Hmax : kMaxLevels), 0, st>>>(e, kmin, nsets);
  SVDUP_COUNT_LAUNCH();
  k_vf_eval<PROB><<<(Lmax + 1) * kLeafMax, 32, 0, st>>>(e, kmin, ysorted, out_final,
                                                        keep_inv ? 1 : 0);
  SVDUP_COUNT_LAUNCH();
}

}  // namespace

void launch_vf_loewner(cudaStream_t st, Eig e, int kmin) {
  vf_run<PROB_LOEWNER>(st, e, kmin, nullptr, nullptr, false);
}

void launch_vf_norms(cudaStream_t st, Eig e, int kmin, const double* ysorted, double* out_final,
                     bool keep_inv) {
  vf_run<PROB_NORMS>(st, e, kmin, ysorted, out_final, keep_inv);
}

void launch_vf_applyq(cudaStream_t st, Eig e, int kmin, const double* xfinal, double* vsorted) {
  vf_run<PROB_APPLYQ>(st, e, kmin, xfinal, vsorted, true);
}

}  // namespace svdup
