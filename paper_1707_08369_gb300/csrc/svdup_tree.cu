// svdup_tree.cu -- the hierarchy of App. D for the FP64 Cauchy product: the far field of
// a leaf pair is taken at the coarsest level where the pair's ancestors are well
// separated, so the translations per box are a handful at every level instead of one
// per admissible leaf pair.
//
// Levels h = 0 (the leaves of svdup_product.cu) .. H - 1; box i of level h holds leaves
// [i 2^h, (i + 1) 2^h) (source boxes over the pole leaves, target boxes over the root
// leaves), its interval the union of its leaves' boxes.  Boxes i, j of one level are well
// separated (admissible) when |i - j| >= 2 and the gap between their intervals is at
// least the larger radius (the leaf rule of svdup_product.cu at every level); children of
// an admissible pair are admissible, so every leaf pair is either near (not admissible at
// level 0) or lies under exactly one pair (i, j) that is admissible while its parents are
// not.  That pair is in the interaction list of target box j at its level.
//
// With Phi_h[i] the far-field expansion of source box i (its charges interpolated onto
// the box's p Chebyshev nodes, App. D STEP 5 at the leaves) and Psi_h[j] the local
// expansion of target box j (values at its nodes):
//   upward (STEP 6)     Phi_{h+1}[i] = sum_{children c} Phi_h[c] M_c,
//                       M_c(a', a) = u_a((x_{c,a'} - c_i) / r_i)   (child nodes in i)
//   translation (STEP 8, the T operators)
//                       Psi_h[j] = sum_{i in list_h(j)} Phi_h[i] T_ij,
//                       T_ij(a, b) = 1 / (xbar_{i,a} - ybar_{j,b})
//   downward (STEP 8, the S operators)
//                       Psi_h[j] += Psi_{h+1}[parent] L_j,
//                       L_j(b', b) = u_b'((y_{j,b} - c_parent) / r_parent)
// and the leaves' local expansions feed the output stage (STEP 9) beside the near field
// (STEP 10).  Each step is a GEMM over all rows of X at once; the T entries are formed in
// the GEMM from the two boxes' geometry, the shift matrices once per box.
#include <cuda_runtime.h>

#include "svdup_internal.cuh"

namespace svdup {

namespace {

// Levels in use: while the target boxes of the level below number more than two (a
// level of at most two boxes has no admissible pair).
__device__ __forceinline__ int tree_levels_dev(int Lt, int Hmax) {
  int h = 1;
  while (h < Hmax && ((Lt + (1 << (h - 1)) - 1) >> (h - 1)) > 2) h++;
  return h;
}

// Box geometry of every level.  Level 0 copies the leaf boxes; a box above is the union
// of its leaves' intervals (an empty target leaf -- no root -- contributes nothing).
__global__ void k_tree_geom(FmmPlan f) {
  const int Ls = f.L[0], Lt = f.L[1];
  const int H = tree_levels_dev(Lt, f.Hmax);
  if (blockIdx.x == 0 && threadIdx.x == 0) f.H[0] = H;
  const int tot = tree_off(f.Lmax, f.Hmax);
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < tot; x += gridDim.x * blockDim.x) {
    int h = 0;
    while (h + 1 < f.Hmax && x >= tree_off(f.Lmax, h + 1)) h++;
    const int i = x - tree_off(f.Lmax, h);
    // source box: leaves [i 2^h, min((i + 1) 2^h, Ls))
    const int a0 = i << h, a1 = min((i + 1) << h, Ls);
    double lo = 0.0, hi = -1.0;
    for (int a = a0; a < a1; a++) {
      const double l = f.sbox_c[a] - f.sbox_r[a], u = f.sbox_c[a] + f.sbox_r[a];
      if (hi < lo) { lo = l; hi = u; } else { lo = fmin(lo, l); hi = fmax(hi, u); }
    }
    if (hi < lo) { f.hsc[x] = 0.0; f.hsr[x] = 1.0; }
    else if (h == 0) { f.hsc[x] = f.sbox_c[i]; f.hsr[x] = f.sbox_r[i]; }
    else { f.hsc[x] = 0.5 * (lo + hi); f.hsr[x] = box_radius(lo, hi); }
    // target box: leaves [j 2^h, min((j + 1) 2^h, Lt))
    const int b0 = i << h, b1 = min((i + 1) << h, Lt);
    lo = 0.0; hi = -1.0;
    for (int b = b0; b < b1; b++) {
      if (f.tj1[b] <= f.tj0[b]) continue;
      const double l = f.tbox_c[b] - f.tbox_r[b], u = f.tbox_c[b] + f.tbox_r[b];
      if (hi < lo) { lo = l; hi = u; } else { lo = fmin(lo, l); hi = fmax(hi, u); }
    }
    f.hte[x] = hi < lo ? 1 : 0;
    if (hi < lo) { f.htc[x] = 0.0; f.htr[x] = 1.0; }
    else if (h == 0) { f.htc[x] = f.tbox_c[i]; f.htr[x] = f.tbox_r[i]; }
    else { f.htc[x] = 0.5 * (lo + hi); f.htr[x] = box_radius(lo, hi); }
  }
}

// Source box i and target box j of level h are well separated.
// (The leaf holding the root beyond all poles, j = Lt - 1 at level 0, is not forced near
// its neighbours, as in the flat near lists.)
__device__ __forceinline__ bool tree_adm(const FmmPlan& f, int h, int i, int j, int Ls, int Lt) {
  if (i - j < 2 && j - i < 2 && !(h == 0 && j == Lt - 1)) return false;
  if ((i << h) >= Ls || (j << h) >= Lt) return false;
  const int o = tree_off(f.Lmax, h);
  if (f.hte[o + j]) return false;
  const double ca = f.hsc[o + i], ra = f.hsr[o + i], cb = f.htc[o + j], rb = f.htr[o + j];
  return fabs(ca - cb) - ra - rb >= fmax(ra, rb);
}

// Interaction lists: one thread per target box of every level in use.
__global__ void k_tree_lists(FmmPlan f) {
  const int Ls = f.L[0], Lt = f.L[1], H = f.H[0];
  const int tot = tree_off(f.Lmax, f.Hmax);
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < tot; x += gridDim.x * blockDim.x) {
    int h = 0;
    while (h + 1 < f.Hmax && x >= tree_off(f.Lmax, h + 1)) h++;
    const int j = x - tree_off(f.Lmax, h);
    int n = 0;
    if (h < H && (j << h) < Lt) {
      int* lst = f.hl + (long long)x * (f.Lmax + 1);
      const int nbs = (Ls + (1 << h) - 1) >> h;
      for (int i = 0; i < nbs; i++) {
        if (!tree_adm(f, h, i, j, Ls, Lt)) continue;
        if (h + 1 < H && tree_adm(f, h + 1, i >> 1, j >> 1, Ls, Lt)) continue;  // parents' pair
        lst[n++] = i;
      }
    }
    f.hnl[x] = n;
  }
}

// Shift operators of every box below the top level in use: M2M (source box as a child)
// and L2L (target box as a child), p x p each, column-major as GEMM B operands (K x N).
__global__ void k_tree_shifts(FmmPlan f) {
  __shared__ double st[32], sw[32];
  cheb_tables(f.p, st, sw);
  const int p = f.p, H = f.H[0];
  const int tot = tree_off(f.Lmax, f.Hmax);
  for (long long y = blockIdx.x * (long long)blockDim.x + threadIdx.x; y < (long long)tot * p;
       y += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(y / p), q = (int)(y - (long long)x * p);
    int h = 0;
    while (h + 1 < f.Hmax && x >= tree_off(f.Lmax, h + 1)) h++;
    if (h + 1 >= H) continue;
    const int c = x - tree_off(f.Lmax, h);
    const int par = tree_off(f.Lmax, h + 1) + (c >> 1);
    double u[32];
    // M2M: child node q, mapped into the parent: row q of the operator (all parent nodes)
    const double xs = f.hsc[x] + f.hsr[x] * cheb_node(q, p);
    lagrange_all(p, box_coord(xs - f.hsc[par], f.hsr[par]), st, sw, u);
    double* M = f.M2M + (long long)x * p * p;
    for (int a = 0; a < p; a++) M[q + (long long)a * p] = u[a];
    // L2L: this box's node q in the parent: column q of the operator (all parent nodes)
    const double yt = f.htc[x] + f.htr[x] * cheb_node(q, p);
    lagrange_all(p, box_coord(yt - f.htc[par], f.htr[par]), st, sw, u);
    double* Lm = f.L2L + (long long)x * p * p;
    for (int b = 0; b < p; b++) Lm[b + (long long)q * p] = u[b];
  }
}

// ---------------------------------------------------------------------------
// The translations as FP64 GEMMs over all rows: one CTA per 64-row tile and output box,
// the p output columns (p <= 32) in one tile.  K runs over the input boxes' p
// coefficients back to back (no padding between boxes); the input boxes, and for the
// translations their geometry, sit in shared memory.  The translation entries
// 1 / (xbar - ybar) are formed in the GEMM (rcp64: four FP64 operations).
// ---------------------------------------------------------------------------
constexpr int TM = 64, TK = 16;  // output tile TM x 8 MJ (MJ = 3 for p <= 24, else 4)
constexpr int kMaxSeg = 512;  // input boxes of one output box (lists longer are cut in parts)
enum { TR_UP = 0, TR_M2L = 1, TR_DOWN = 2 };

template <int KIND, int MJ>
__global__ void __launch_bounds__(128) k_tree_gemm(FmmPlan f, int rows, int hin) {
  constexpr int TN = 8 * MJ;
  __shared__ double As[TK][TM];
  __shared__ double Bs[TK][TN + 1];
  __shared__ double tn[32];
  __shared__ int sbox[kMaxSeg];
  __shared__ double sc[kMaxSeg], sr[kMaxSeg];
  const int H = f.H[0], Ls = f.L[0], Lt = f.L[1], p = f.p;
  // The translations of every level run in one launch: blockIdx.y indexes the target
  // boxes of all levels.  The shifts run a level per launch (hin: the lower level).
  int h = hin, ob = blockIdx.y;
  if (KIND == TR_M2L) {
    h = 0;
    while (h + 1 < f.Hmax && ob >= tree_off(f.Lmax, h + 1)) h++;
    ob -= tree_off(f.Lmax, h);
  }
  const int ho = KIND == TR_UP ? h + 1 : h;  // output level
  if (ho >= H || (KIND == TR_DOWN && h + 1 >= H)) return;
  if (KIND == TR_UP ? (ob << ho) >= Ls : (ob << ho) >= Lt) return;
  const int oo = tree_off(f.Lmax, ho) + ob;
  int nseg;
  if (KIND == TR_UP) nseg = min(2, ((Ls + (1 << h) - 1) >> h) - 2 * ob);
  else if (KIND == TR_M2L) nseg = f.hnl[oo];
  else nseg = 1;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  for (int i = tid; i < p; i += 128) tn[i] = cheb_node(i, p);
  const double rj = KIND == TR_M2L ? f.htr[oo] : 0.0;
  const double* Abase = KIND == TR_DOWN ? f.Psi : f.Phi;
  const int r0 = blockIdx.x * TM;
  double acc[4][MJ];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < MJ; j++) acc[i][j] = 0.0;
  for (int s0 = 0; s0 < nseg; s0 += kMaxSeg) {  // input boxes in chunks of kMaxSeg
  const int ns = min(kMaxSeg, nseg - s0);
  __syncthreads();  // the previous chunk's boxes consumed
  for (int sg = tid; sg < ns; sg += 128) {
    int ib;
    if (KIND == TR_UP) ib = tree_off(f.Lmax, h) + 2 * ob + sg;
    else if (KIND == TR_M2L) ib = tree_off(f.Lmax, h) + f.hl[(long long)oo * (f.Lmax + 1) + s0 + sg];
    else ib = tree_off(f.Lmax, h + 1) + (ob >> 1);
    sbox[sg] = ib;
    if (KIND == TR_M2L) { sc[sg] = f.hsc[ib] - f.htc[oo]; sr[sg] = f.hsr[ib]; }
  }
  __syncthreads();
  const int K = ns * p;
  for (int kb = 0; kb < K; kb += TK) {
    for (int x = tid; x < TK * TM; x += 128) {
      const int kk = x / TM, r = x - kk * TM;
      const int g = kb + kk;
      double v = 0.0;
      if (g < K && r0 + r < rows) {
        const int sg = g / p, q = g - sg * p;
        v = Abase[((long long)sbox[sg] * p + q) * f.ldphi + r0 + r];
      }
      As[kk][r] = v;
    }
    for (int x = tid; x < TK * TN; x += 128) {
      const int kk = x / TN, c = x - kk * TN;
      const int g = kb + kk;
      double v = 0.0;
      if (g < K && c < p) {
        const int sg = g / p, q = g - sg * p;
        if (KIND == TR_M2L) v = rcp64((sc[sg] + sr[sg] * tn[q]) - rj * tn[c]);
        else if (KIND == TR_UP) v = f.M2M[(long long)sbox[sg] * p * p + q + (long long)c * p];
        else v = f.L2L[(long long)oo * p * p + q + (long long)c * p];
      }
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; kk++) {
      double a[4], bb[MJ];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < MJ; j++) bb[j] = Bs[kk][tx * MJ + j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < MJ; j++) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  }
  double* Out = (KIND == TR_UP ? f.Phi : f.Psi) + (long long)oo * p * f.ldphi;
#pragma unroll
  for (int j = 0; j < MJ; j++) {
    const int cc = tx * MJ + j;
    if (cc >= p) continue;
    double* col = Out + (long long)cc * f.ldphi;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int r = r0 + ty * 4 + i;
      if (r >= rows) continue;
      if (KIND == TR_DOWN) col[r] += acc[i][j];
      else col[r] = acc[i][j];
    }
  }
}

// Useful flops of the translations: 2 rows p^2 per (output box, input box) pair.
__global__ void k_tree_flops(FmmPlan f, int rows, double* acc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int H = f.H[0], Ls = f.L[0], Lt = f.L[1];
  const double u = 2.0 * rows * (double)f.p * f.p;
  double t = 0.0;
  for (int h = 0; h < H; h++) {
    const int o = tree_off(f.Lmax, h);
    const int nbs = (Ls + (1 << h) - 1) >> h, nbt = (Lt + (1 << h) - 1) >> h;
    for (int j = 0; j < nbt; j++) t += u * f.hnl[o + j];
    if (h + 1 < H) t += u * (nbs + nbt);  // every box below the top: one shift up, one down
  }
  acc[1] += t;
}

}  // namespace

void launch_tree_setup(cudaStream_t st, Eig e, FmmPlan f) {
  (void)e;
  const int tot = tree_off(f.Lmax, f.Hmax);
  k_tree_geom<<<(tot + 127) / 128, 128, 0, st>>>(f);
  SVDUP_COUNT_LAUNCH();
  k_tree_lists<<<(tot + 127) / 128, 128, 0, st>>>(f);
  SVDUP_COUNT_LAUNCH();
  const long long sp = (long long)tot * f.p;
  k_tree_shifts<<<(int)((sp + 127) / 128), 128, 0, st>>>(f);
  SVDUP_COUNT_LAUNCH();
}

template <int MJ>
void tree_translate(cudaStream_t st, FmmPlan f, int rows) {
  const int rt = (rows + TM - 1) / TM;
  for (int h = 0; h + 1 < f.Hmax; h++) {  // upward: level h into level h + 1
    k_tree_gemm<TR_UP, MJ><<<dim3(rt, tree_nb(f.Lmax, h + 1)), 128, 0, st>>>(f, rows, h);
    SVDUP_COUNT_LAUNCH();
  }
  // the translations of every level at once (they are independent)
  k_tree_gemm<TR_M2L, MJ><<<dim3(rt, tree_off(f.Lmax, f.Hmax)), 128, 0, st>>>(f, rows, 0);
  SVDUP_COUNT_LAUNCH();
  for (int h = f.Hmax - 2; h >= 0; h--) {  // downward: level h + 1 into level h
    k_tree_gemm<TR_DOWN, MJ><<<dim3(rt, tree_nb(f.Lmax, h)), 128, 0, st>>>(f, rows, h);
    SVDUP_COUNT_LAUNCH();
  }
}

void launch_tree_translate(cudaStream_t st, Eig e, FmmPlan f, int rows) {
  (void)e;
  if (f.p <= 24) tree_translate<3>(st, f, rows);
  else tree_translate<4>(st, f, rows);
}

void launch_tree_flops(cudaStream_t st, FmmPlan f, int rows, double* acc) {
  k_tree_flops<<<1, 32, 0, st>>>(f, rows, acc);
  SVDUP_COUNT_LAUNCH();
}

}  // namespace svdup
