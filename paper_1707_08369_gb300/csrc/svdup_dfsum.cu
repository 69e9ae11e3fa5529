// svdup_dfsum.cu -- the Cauchy-like sums of the eigenvector step in double-float
// arithmetic, for the mixed-precision mode (its vectors are FP32-accurate):
//   column norms   ||c_j||^2 = sum_t zhat_t^2 / delta_tj^2        (Eq. CTildeFinalForm1,
//                                                                 RankOneUpdate STEP 7)
//   Q^T y          out_j = (1/||c_j||) sum_t zhat_t y_t / delta_tj
//   Q x            v_t = zhat_t sum_j (x_j / ||c_j||) / delta_tj
// with delta_tj = (d_t - d_org(j)) - tau_j.  Each term keeps one FP64 operation, the
// pole difference d_t - d_org(j) (exact when the poles are close, by Sterbenz's lemma);
// the subtraction of tau_j, the reciprocal and the sums run on FP32 pairs (svdup_df.cuh).
//
// Accuracy and range.  The root's origin is its nearer bracketing pole, so |tau_j| is
// at most half the bracket, and for every pole t outside the bracket the subtraction of
// tau_j cancels at most a factor 3: each term carries about 2^-45 relative error.  The
// poles org(j)-1 .. org(j)+1 (those that may bracket root j) are summed in FP64, so the
// pair terms never meet the near-singular offsets.  d and tau are scaled by 2^-E (E the
// exponent of the largest of |d|, |tau|), the weights by their own largest exponents;
// after deflation the remaining offsets are far above 2^-100 of the largest pole, so
// every term lies inside the FP32 range.  A sum that still ends non-finite or zero is
// recomputed in FP64 by the same warp.
#include <cuda_runtime.h>

#include "svdup_df.cuh"
#include "svdup_internal.cuh"

namespace svdup {

namespace {

__device__ __forceinline__ Df ld(const float2* p, int i) {
  const float2 v = p[i];
  return Df{v.x, v.y};
}

__device__ __forceinline__ float2 st(Df a) { return make_float2(a.hi, a.lo); }

// 2^s applied in two halves, each inside the FP64 exponent range.
__device__ __forceinline__ double scale2(double x, int s) {
  const int h = s / 2;
  return x * pow2d(max(-1022, min(1023, h))) * pow2d(max(-1022, min(1023, s - h)));
}

__device__ __forceinline__ double pair_to_f64(Df a, int s) { return scale2(df_to_f64(a, 0), s); }

__device__ __forceinline__ int bmax_exp(int v, int* slot) {
  v = max(v, __shfl_xor_sync(0xffffffffu, v, 16));
  v = max(v, __shfl_xor_sync(0xffffffffu, v, 8));
  v = max(v, __shfl_xor_sync(0xffffffffu, v, 4));
  v = max(v, __shfl_xor_sync(0xffffffffu, v, 2));
  v = max(v, __shfl_xor_sync(0xffffffffu, v, 1));
  if ((threadIdx.x & 31) == 0) atomicMax(slot, v);
  return v;
}

}  // namespace

// Scales and pair copies for one solve (one block):
//   fsc[0] = E (largest exponent of |d|, |tau|), fsc[1] = Z (of |zhat|), fsc[2] = Y (of |y|),
//   fsc[3] = W (of |x_j / ||c_j|||);
//   tf[j] = tau_j 2^-E, zf[t] = zhat_t 2^-Z, yf[t] = y_idx(t) 2^-Y, wf[j] = (x_rank(j) inv_j) 2^-W.
// ysorted and xfinal may be null (those copies are skipped).
__global__ void __launch_bounds__(1024) k_df_prep(Eig e, const double* __restrict__ ysorted,
                                                  const double* __restrict__ xfinal) {
  __shared__ int sx[4];
  const int k = e.kp[0];
  if (e.vf && k >= e.vfmin_pairs) return;  // the far-field form replaces the pair sums
  if (threadIdx.x < 4) sx[threadIdx.x] = -1100;
  __syncthreads();
  int mE = -1100, mZ = -1100, mY = -1100, mW = -1100;
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    mE = max(mE, max(exp2_of(e.dk[t]), exp2_of(e.tau[t])));
    mZ = max(mZ, exp2_of(e.zhat[t]));
    if (ysorted) mY = max(mY, exp2_of(ysorted[e.idx[t]]));
    if (xfinal) mW = max(mW, exp2_of(e.inv[t] * xfinal[e.rank_root[t]]));
  }
  bmax_exp(mE, &sx[0]);
  bmax_exp(mZ, &sx[1]);
  bmax_exp(mY, &sx[2]);
  bmax_exp(mW, &sx[3]);
  __syncthreads();
  int sc[4];
#pragma unroll
  for (int i = 0; i < 4; i++) sc[i] = sx[i] <= -1000 ? 0 : sx[i];
  if (threadIdx.x < 4) e.fsc[threadIdx.x] = sc[threadIdx.x];
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    e.tf[t] = st(df_from_f64(e.tau[t], sc[0]));
    e.zf[t] = st(df_from_f64(e.zhat[t], sc[1]));
    if (ysorted) e.yf[t] = st(df_from_f64(ysorted[e.idx[t]], sc[2]));
    if (xfinal) e.wf[t] = st(df_from_f64(e.inv[t] * xfinal[e.rank_root[t]], sc[3]));
  }
}

// Column norms (and Q^T y when ysorted is set): one warp per root j.
__global__ void __launch_bounds__(256) k_norms_df(Eig e, const double* __restrict__ ysorted,
                                                  double* out_final, int keep_inv) {
  const int k = e.kp[0];
  if (e.vf && k >= e.vfmin_pairs) return;  // the far-field form (svdup_vfmm.cu)
  const int E = e.fsc[0], Z = e.fsc[1], Y = e.fsc[2];
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const double* __restrict__ dk = e.dk;
  const float2* __restrict__ zf = e.zf;
  const float2* __restrict__ yf = e.yf;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < k; j += warps) {
    const int O = e.org[j];
    const double dO = e.dorg[j], tj = e.tau[j];
    const Df ntau = df_neg(ld(e.tf, j));
    Df s2 = {0.f, 0.f}, sy = {0.f, 0.f};
    for (int t = lane; t < k; t += 32) {
      if ((unsigned)(t - O + 1) <= 2u) continue;  // bracket poles: FP64 below
      const Df del = df_add(df_from_f64(dk[t] - dO, E), ntau);
      const Df c = df_mul(ld(zf, t), df_rcp(del));
      s2 = df_add(s2, df_sqr(c));
      if (ysorted) sy = df_add(sy, df_mul(c, ld(yf, t)));
    }
    s2 = df_warp_sum(s2);
    if (ysorted) sy = df_warp_sum(sy);
    double S2 = 0.0, SY = 0.0;
    if (lane == 0) {
      S2 = pair_to_f64(s2, 2 * (Z - E));
      if (ysorted) SY = pair_to_f64(sy, Z - E + Y);
      for (int t = max(0, O - 1); t <= min(k - 1, O + 1); t++) {
        const double c = e.zhat[t] / ((dk[t] - dO) - tj);
        S2 = fma(c, c, S2);
        if (ysorted) SY = fma(c, ysorted[e.idx[t]], SY);
      }
    }
    S2 = __shfl_sync(0xffffffffu, S2, 0);
    SY = __shfl_sync(0xffffffffu, SY, 0);
    if (!(S2 > 0.0 && S2 <= 1.7e308 && fabs(SY) <= 1.7e308)) {  // out of the pair range: FP64
      S2 = 0.0;
      SY = 0.0;
      for (int t = lane; t < k; t += 32) {
        const double c = e.zhat[t] / ((dk[t] - dO) - tj);
        S2 = fma(c, c, S2);
        if (ysorted) SY = fma(c, ysorted[e.idx[t]], SY);
      }
      S2 = warp_sum(S2);
      SY = warp_sum(SY);
    }
    if (lane == 0) {
      const double inv = 1.0 / sqrt(S2);
      if (!keep_inv) e.inv[j] = inv;
      if (ysorted) out_final[e.rank_root[j]] = SY * inv;
    }
  }
}

// v_t = zhat_t sum_j (x_j inv_j) / delta_tj, one warp per pole t (and the deflated
// entries copied through), as k_apply_q_core.
__global__ void __launch_bounds__(256) k_apply_q_df(Eig e, const double* __restrict__ xfinal,
                                                    double* vsorted) {
  const int k = e.kp[0];
  const int E = e.fsc[0], W = e.fsc[3];
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const double* __restrict__ dorg = e.dorg;
  const int* __restrict__ org = e.org;
  const float2* __restrict__ tf = e.tf;
  const float2* __restrict__ wf = e.wf;
  const bool far = e.vf && k >= e.vfmin_pairs;  // the far-field form writes the kept entries
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < (far ? 0 : k); t += warps) {
    const double dt = e.dk[t];
    Df acc = {0.f, 0.f};
    for (int j = lane; j < k; j += 32) {
      if ((unsigned)(t - org[j] + 1) <= 2u) continue;  // roots that pole t may bracket
      const Df del = df_add(df_from_f64(dt - dorg[j], E), df_neg(ld(tf, j)));
      acc = df_add(acc, df_mul(ld(wf, j), df_rcp(del)));
    }
    acc = df_warp_sum(acc);
    double A = 0.0;
    if (lane == 0) {
      A = pair_to_f64(acc, W - E);
      for (int j = max(0, t - 2); j <= min(k - 1, t + 2); j++) {  // org(j) is j-1, j or j+1
        if ((unsigned)(t - org[j] + 1) > 2u) continue;
        A += (e.inv[j] * xfinal[e.rank_root[j]]) / ((dt - dorg[j]) - e.tau[j]);
      }
    }
    A = __shfl_sync(0xffffffffu, A, 0);
    if (!(fabs(A) <= 1.7e308)) {
      A = 0.0;
      for (int j = lane; j < k; j += 32)
        A += (e.inv[j] * xfinal[e.rank_root[j]]) / ((dt - dorg[j]) - e.tau[j]);
      A = warp_sum(A);
    }
    if (lane == 0) vsorted[e.idx[t]] = e.zhat[t] * A;
  }
  const int nd = e.N - k;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nd; u += gridDim.x * blockDim.x) {
    const int s = e.didx[u];
    vsorted[s] = xfinal[e.rank_defl[s]];
  }
}

// Loewner's zhat (Gu-Eisenstat; RankOneUpdate STEP 7's z recomputed from the roots) in
// the rho > 0 orientation, as k_loewner:
//   zhat_i^2 = prod_{j != i} [(d_org(j') - d_i) + tau_j'] / (d_j - d_i)
//              * [(d_org(k-1) - d_i) + tau_{k-1}] / |rho|,   j' = j (j < i), j - 1 (j > i),
// one warp per pole i.  Each factor pairs root j' with pole j, so the running product
// stays near 1; it is kept as a pair times 2^pe, renormalised after every factor.  The
// two factors of the bracketing poles i-1 and i+1 (with roots i-1 and i) and the last
// root's are FP64.
__global__ void __launch_bounds__(256) k_loewner_df(Eig e) {
  const int k = e.kp[0];
  if (e.vf && k >= e.vfmin_pairs) return;  // the far-field form (svdup_vfmm.cu)
  const double rho = e.rhop[0];
  const double R = fabs(rho);
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const double* __restrict__ dc = e.dc;
  const int* __restrict__ orgc = e.orgc;
  const double* __restrict__ tauc = e.tauc;
  if (k < 1) return;
  const int E = max(max(exp2_of(dc[0]), exp2_of(dc[k - 1])), exp2_of(tauc[k - 1])) + 1;
  auto renorm = [](Df& p, int& pe) {
    const int ex = ((__float_as_int(p.hi) >> 23) & 0xff) - 127;
    const float sc = pow2f(-ex);
    p.hi *= sc;
    p.lo *= sc;
    pe += ex;
  };
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < k; i += warps) {
    const double di = dc[i];
    Df pr = {1.0f, 0.0f};
    int pe = 0;
    for (int j = lane; j < k; j += 32) {
      if ((unsigned)(j - i + 1) <= 2u) continue;
      const int jr = (j < i) ? j : j - 1;
      const Df num = df_add(df_from_f64(dc[orgc[jr]] - di, E), df_from_f64(tauc[jr], E));
      const Df den = df_from_f64(dc[j] - di, E);
      pr = df_mul(pr, df_mul(num, df_rcp(den)));
      renorm(pr, pe);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const Df q = df_shfl_xor(pr, o);
      const int qe = __shfl_xor_sync(0xffffffffu, pe, o);
      pr = df_mul(pr, q);
      pe += qe;
      renorm(pr, pe);
    }
    if (lane == 0) {
      double P = pair_to_f64(pr, pe);
      if (i >= 1) P *= ((dc[orgc[i - 1]] - di) + tauc[i - 1]) / (dc[i - 1] - di);
      if (i + 1 < k) P *= ((dc[orgc[i]] - di) + tauc[i]) / (dc[i + 1] - di);
      P *= ((dc[orgc[k - 1]] - di) + tauc[k - 1]) / R;
      const double mag = sqrt(fmax(P, 0.0));
      const int io = (rho > 0.0) ? i : (k - 1 - i);
      const double z = e.zk[io];
      e.zhat[io] = (z < 0.0) ? -mag : mag;
    }
  }
}

void launch_loewner_df(cudaStream_t st, Eig e) {
  launch_vf_loewner(st, e, e.vfmin_pairs);  // the far-field form when k >= vfmin_pairs
  k_loewner_df<<<(e.N + 7) / 8, 256, 0, st>>>(e);  // one warp per pole
  SVDUP_COUNT_LAUNCH();
}

void launch_norms_df(cudaStream_t st, Eig e, const double* ysorted, double* out_final,
                     int blocks, bool keep_inv) {
  k_df_prep<<<1, 1024, 0, st>>>(e, ysorted, nullptr);
  SVDUP_COUNT_LAUNCH();
  k_norms_df<<<blocks, 256, 0, st>>>(e, ysorted, out_final, keep_inv ? 1 : 0);
  SVDUP_COUNT_LAUNCH();
}

void launch_apply_q_core_df(cudaStream_t st, Eig e, const double* xfinal, double* vsorted,
                            int blocks) {
  k_df_prep<<<1, 1024, 0, st>>>(e, nullptr, xfinal);
  SVDUP_COUNT_LAUNCH();
  k_apply_q_df<<<blocks, 256, 0, st>>>(e, xfinal, vsorted);
  SVDUP_COUNT_LAUNCH();
}

}  // namespace svdup
