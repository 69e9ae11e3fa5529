// svdup_internal.cuh -- device-side structures and helpers shared by the CUDA
// sources of libsvdup.so (not part of the public interface).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/svdup.h"

namespace svdup {

// ---------------------------------------------------------------------------
// Device status word: the first error wins (atomicCAS from 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void latch(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Launch accounting: every kernel launch calls note_launch (via SVDUP_COUNT_LAUNCH),
// which counts it (one atomic counter for the process) and, when the environment sets
// SVDUP_DEBUG, waits for the device and reports the launch site of the first failing
// kernel on stderr.  Launches recorded into a batch graph are counted when the graph
// is launched.
void note_launch(const char* file, int line);
#define SVDUP_COUNT_LAUNCH() ::svdup::note_launch(__FILE__, __LINE__)

constexpr double kU = 1.1102230246251565e-16;  // 2^-53, unit roundoff of IEEE double

// 1/x for IEEE double by Newton-Raphson on the reciprocal.  The seed comes from the
// significand alone, by the bit fields: m in [1, 2) (the top 23 fraction bits as an FP32
// number), its FP32 reciprocal (rcp.approx, about one ulp), then x's exponent negated and
// its sign put back, so no FP64 operation and no range limit is spent on the seed.  Two
// FP64 Newton steps r <- r + r (1 - x r) take it from 2^-22 to 2^-44 to below 2^-53.
// Zeros, subnormals, the largest binades (whose reciprocals are subnormal), infinities and
// NaNs take CUDA's division.  On this GPU every FP64 warp instruction costs the same
// whatever its active lanes; the seed keeps four of them per reciprocal.
__device__ __forceinline__ double rcp64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned ex = (unsigned)(b >> 52) & 0x7ffu;
  if (ex == 0u || ex >= 0x7fdu) return 1.0 / x;
  const float m = __int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffffu));
  float rm;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rm) : "f"(m));  // in (0.5, 1]
  const unsigned um = __float_as_uint(rm);
  const unsigned long long de = (unsigned long long)((um >> 23) & 0xffu) + 1919ull - ex;
  double r = __longlong_as_double((long long)((b & 0x8000000000000000ull) | (de << 52) |
                                              ((unsigned long long)(um & 0x7fffffu) << 29)));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// 1/sqrt(x) for a positive normal double, the same way: x = m 2^(e - eo) with m in [1, 4)
// (e - eo even), an FP32 rsqrt.approx of m, the exponent halved by the bit fields, then
// two FP64 Newton steps y <- y + y (1 - x y^2) / 2 (2^-22 -> 2^-44 -> rounding).  Other
// inputs take CUDA's square root and division.
__device__ __forceinline__ double rsqrt64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0 || ex == 0x7ff || (b >> 63)) return 1.0 / sqrt(x);
  const int e = ex - 1023, eo = e & 1;
  const float m = __int_as_float(((127 + eo) << 23) | (int)((b >> 29) & 0x7fffffu));
  float rm;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rm) : "f"(m));  // in (0.5, 1]
  const unsigned um = __float_as_uint(rm);
  const long long de = (long long)((um >> 23) & 0xffu) + 896 - (e - eo) / 2;
  double y = __longlong_as_double((long long)(((unsigned long long)de << 52) |
                                              ((unsigned long long)(um & 0x7fffffu) << 29)));
  double h = fma(-(x * y), y, 1.0);
  y = fma(0.5 * y, h, y);
  h = fma(-(x * y), y, 1.0);
  return fma(0.5 * y, h, y);
}

// Exponent bookkeeping for long FP64 products: x = m 2^e with m in [1, 2) after
// renorm (bit fields only; a zero stays zero).
__device__ __forceinline__ void renorm64(double& m, int& e) {
  const long long b = __double_as_longlong(m);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return;
  m = __longlong_as_double((b & ~(0x7ffll << 52)) | (1023ll << 52));
  e += ex - 1023;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_prod(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// One symmetric rank-one eigen-problem diag(d) + rho z z^T (RankOneUpdate, Sec. 6.2)
// in device memory.  N is known on the host; k (the non-deflated count) lives on the
// device so that nothing waits on the host between stages.
// ---------------------------------------------------------------------------
constexpr int kMaxOverrunList = 256;  // deflation: walking ranges (svdup_solve.cu)

struct Eig {
  int N;
  double* rhop;  // rho (1 value, device: it depends on device-computed norms)
  // sorted (ascending) poles and their z, after deflation rotations
  double* ds;
  double* zs;
  int* perm;  // sorted position -> physical column of the basis X
  int* defl;  // sorted position -> 1 if deflated
  // deflation rotations, in application order: positions (rj, ri), cos rc, sin rs
  int* nrot;
  int* rj;
  int* ri;
  double* rc;
  double* rs;
  // non-deflated set
  int* kp;     // k
  int* idx;    // k sorted positions
  int* didx;   // N - k deflated sorted positions
  double* dk;  // k poles
  double* zk;  // k z values
  // the same in the rho > 0 orientation used by the solver: dc ascending, z2c = z^2
  double* dc;
  double* z2c;
  // roots: mu_j = dk[org[j]] + tau[j]; dorg[j] = dk[org[j]]
  int* org;
  double* tau;
  double* dorg;
  int* orgc;     // roots in the rho > 0 orientation (solver and Loewner step)
  double* tauc;
  double* zhat;
  double* inv;  // 1 / ||c_j||
  // all N eigenvalues ascending, and where each came from
  double* lam;
  int* rank_root;  // root j -> final index
  int* rank_defl;  // sorted position s (deflated) -> final index, else -1
  double* tol;     // deflation tolerance (1 value)
  // deflation scratch: the survivors of case (1) (scaled d and z, sorted positions, run
  // flags, rotation index, kept index, run start), the candidate bitmask (N / 32 + 1
  // words), the survivor count (dint), scaled tolerance, scalings and 1 / tol (dflt), and
  // per walking range the run it carried into the next range (head, carrier)
  double* sd;
  double* sz;
  int* spos;
  unsigned char* sbrk;
  int* srix;
  int* skix;
  int* srs;
  unsigned* dmask;
  int* dint;
  double* dflt;
  int* ovh;
  float2* ovW;  // the carried run: sum z^2 and sum z^2 (d - ref) / tol as FP32 pairs,
  float2* ovM;
  double* ovR;  // and its first pole ref
  // far-field secular evaluation (null: direct sums only): per box of 64 roots its
  // origin and half width, its near pole range, and the far sums at its nodes
  double* sqb;
  int* sqn;
  int* sqf;  // the boxed roots first .. last, the pair-form scales E, Z; [4]: the solver's root counter
  float2* z2f;  // z^2 2^-Z as pairs (the far-field form)
  double* sqv;
  // double-float copies for the pair-arithmetic sums (svdup_dfsum.cu): scales fsc[4]
  // (exponents), tau, zhat, y and root weights as (hi, lo) FP32 pairs
  int* fsc;
  float2* tf;
  float2* zf;
  float2* yf;
  float2* wf;
  // the far field of the solve's own sums (svdup_vfmm.cu): per-box geometry, moments,
  // local values and leaf locals (vf), and the upward pass's arrival counters (vfc)
  double* vf;
  int* vfc;
  // the far-field form replaces the FP64 direct sums for k >= vfmin and the FP32-pair
  // direct sums for k >= vfmin_pairs (vf is allocated for N >= kVfMinK)
  int vfmin;
  int vfmin_pairs;
};

// Column mapping of a product's output: physical column of final index q is
//   out_rev ? (out_n - 1 - q) : q.  Yf, when set, replaces Y by an FP32 matrix (the
// mixed form's intermediate W; only its kernels write it).
struct OutMap {
  double* Y;
  long long ldy;
  int out_n;
  int out_rev;
  float* Yf;
};

// FMM (flat Chebyshev far field + direct near field) plan for one product.
// Source leaf a holds the sorted poles [a s - P, a s + s - P) (leaf K position g is pole
// g - P; the offset P starts a leaf at an isolated group of largest poles, see
// k_fmm_boxes).  Target leaf b < Lt - 1 holds the roots [b s - Pt, b s + s - Pt) that lie
// between poles; the last target leaf holds the extreme root (the largest for rho > 0,
// the smallest for rho < 0, which can lie far outside the poles) alone.
struct FmmPlan {
  int p;     // expansion order
  int s;     // leaf size
  int Lmax;  // upper bound on the number of source leaves (ceil(N / s) + 1); targets Lmax + 1
  int* L;    // device: source leaves Ls, target leaves Lt, leaf offsets P (poles), Pt (roots)
  double* sbox_c;
  double* sbox_r;
  double* tbox_c;
  double* tbox_r;
  int* tj0;  // per target leaf: first root
  int* tj1;  // per target leaf: one past the last root
  int* nnear;  // per target leaf: number of near source leaves
  int* near;   // per target leaf b: near source leaves, ascending, at near[b * Lmax + i]
  double* S;      // P2M operators, [leaf][alpha][t] (s x p col-major): zhat_t u_alpha(x_t)
  double* T;      // M2L operator, (Lmax p) x ((Lmax+1) p) col-major, zero where not admissible
  double* Lop;    // L2P operators, [leaf][jl][beta] (p x s col-major): u_beta(y_j) inv_j
  double* Phi;    // rows x (Lmax p) far-field expansions (FP64 tree: every level's boxes)
  double* Psi;    // rows x ((Lmax+1) p) local expansions (FP64 tree: every level's boxes)
  long long ldphi;
  void* rot;      // scratch of the deflation rotations (rotate_scratch_bytes(N, rows))
  // The hierarchy of App. D (FP64 mode, tree != 0): level h = 0 are the leaves, box i of
  // level h covers leaves [i 2^h, (i + 1) 2^h), tree_nb(Lmax, h) boxes at most; level h's
  // boxes start at tree_off(Lmax, h) in every per-box array and in Phi / Psi (columns
  // p tree_off + p i), so level 0 keeps the flat layout.
  int tree;
  int Hmax;       // levels allocated
  int* H;         // device: levels in use
  double *hsc, *hsr, *htc, *htr;  // source / target box centres and radii, every level
  int* hte;       // target box holds no root (1)
  int* hnl;       // per target box: interaction-list length
  int* hl;        // interaction lists: hl[(tree_off(h) + j) * (Lmax + 1) + i]
  double* M2M;    // per source box below the top: p x p, child coefficients -> parent's
  double* L2L;    // per target box below the top: p x p, parent's local -> this box's
};

// ---------------------------------------------------------------------------
// Chebyshev far-field helpers shared by the FMM set-up kernels (svdup_product.cu,
// svdup_tree.cu).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cheb_node(int alpha, int p) {
  return cospi((2.0 * alpha + 1.0) / (2.0 * p));  // alpha = 0..p-1  (App. D Eq. Define_ti)
}

// Half-width of a box [lo, hi]; a (near-)single-point box gets a small positive width
// relative to its position so that points map to finite coordinates near 0.
__device__ __forceinline__ double box_radius(double lo, double hi) {
  double r = 0.5 * (hi - lo);
  double floor_r = 1e-6 * fmax(fabs(lo), fabs(hi));
  return fmax(fmax(r, floor_r), 1e-300);
}

// Box coordinate in [-1, 1] (clamped: rounding can put a point a few ulps outside).
__device__ __forceinline__ double box_coord(double off, double r) {
  return fmin(1.0, fmax(-1.0, off / r));
}

// All p Lagrange basis values at x (App. D Eq. Define_uj) in the barycentric form on
// the first-kind Chebyshev nodes: u_alpha(x) = [w_alpha / (x - t_alpha)] / sum_beta
// [w_beta / (x - t_beta)], w_beta = (-1)^beta sin((2 beta + 1) pi / (2p)); a node hit
// exactly gives the unit vector.  Nodes and weights come from shared memory.
__device__ inline void lagrange_all(int p, double x, const double* st, const double* sw, double* out) {
  int hit = -1;
  double den = 0.0;
  for (int b = 0; b < p; b++) {
    const double df = x - st[b];
    if (df == 0.0) hit = b;
    const double c = df == 0.0 ? 0.0 : sw[b] / df;
    out[b] = c;
    den += c;
  }
  if (hit >= 0) {
    for (int b = 0; b < p; b++) out[b] = b == hit ? 1.0 : 0.0;
  } else {
    const double inv = 1.0 / den;
    for (int b = 0; b < p; b++) out[b] *= inv;
  }
}

__device__ inline void cheb_tables(int p, double* st, double* sw) {
  for (int b = threadIdx.x; b < p; b += blockDim.x) {
    const double th = (2.0 * b + 1.0) / (2.0 * p);
    st[b] = cospi(th);
    sw[b] = (b & 1 ? -1.0 : 1.0) * sinpi(th);
  }
  __syncthreads();
}

// Boxes of level h (over Lmax + 1 leaves) and the offset of level h in the per-box arrays.
__host__ __device__ inline int tree_nb(int Lmax, int h) { return ((Lmax + 1) + (1 << h) - 1) >> h; }
__host__ __device__ inline int tree_off(int Lmax, int h) {
  int o = 0;
  for (int i = 0; i < h; i++) o += tree_nb(Lmax, i);
  return o;
}
__host__ __device__ inline int tree_levels(int Lmax) {
  int h = 1;
  while (tree_nb(Lmax, h - 1) > 2) h++;
  return h;
}

// The far field of Loewner's zhat and of the column norms (svdup_vfmm.cu): leaves of
// kVfLeaf consecutive indices (the last takes the remainder), kVfP Chebyshev nodes per
// box, used when k >= kVfMinK.  Layout of Eig::vf for a problem of size N, with
// Lmax + 1 = max(1, N / kVfLeaf) leaves at most: geometry (4 per box: source centre and
// radius, target centre and radius), moments and local values (2 sets of kVfP per box,
// the local values in kVfParts partial sums), leaf locals (2 sets of kVfP per leaf), each
// leaf's part of the last root's sums (2), the Chebyshev nodes and barycentric weights;
// Eig::vfc holds the arrival counters (one per box) and each leaf's near list.
constexpr int kVfP = 28;
constexpr int kVfLeaf = 64;
constexpr int kVfMinK = 2048;
constexpr int kVfDefault = 4096;        // against the FP64 direct sums (measured crossover)
constexpr int kVfDefaultPairs = 12288;  // against the FP32-pair direct sums
constexpr int kVfParts = 4;     // translations of a box split over this many warps
constexpr int kVfNearMax = 64;  // near leaves listed per leaf (more: every pole is near)
__host__ __device__ inline int vf_lmax(int N) { return (N / kVfLeaf > 1 ? N / kVfLeaf : 1) - 1; }
__host__ __device__ inline int vf_tot(int N) {
  const int L = vf_lmax(N);
  return tree_off(L, tree_levels(L));
}
__host__ __device__ inline size_t vf_doubles(int N) {
  return 2 * (size_t)kVfP + (size_t)vf_tot(N) * (4 + 2 * kVfP * (1 + kVfParts)) +
         (size_t)(vf_lmax(N) + 1) * 2 * (kVfP + 1);
}
__host__ __device__ inline size_t vf_ints(int N) {
  return (size_t)vf_tot(N) + (size_t)(vf_lmax(N) + 1) * (kVfNearMax + 1);
}

// Mixed-precision (split BF16) form of the product on the tensor cores.  Every operand
// of the three contractions is stored pre-tiled in HBM as three BF16 planes
// (x = hi + mid + lo, Sec. 5 / App. D operators split the same way), each plane in the
// canonical K-major layout of the tcgen05 shared-memory descriptor, so one bulk copy
// moves a whole tile.  A operands are 128-row tiles; K tiles are 64 wide (16 for the
// local expansions Psi).  P = 16 Chebyshev nodes.
struct MixPlan {
  int rows, rt;  // rows of X and the number of 128-row tiles
  int s;         // leaf size (64 or 128)
  int Lmax;      // source leaves upper bound (ceil(N / s)); target leaves Lmax + 1
  int kx;        // X K-tiles per row tile: Lmax * s / 64
  int kphi;      // Phi K-tiles per row tile: ceil(Lmax * P / 64)
  int ntT;       // M2L N-tiles: ceil((Lmax + 1) * P / 128)
  unsigned char* Xp;    // [rt][kx] A tiles (128 x 64)
  unsigned char* Phip;  // [rt][kphi] A tiles (128 x 64)
  unsigned char* Psip;  // [rt][Lmax + 1] A tiles (128 x 16)
  unsigned char* Sp;    // [Lmax][s / 64] B tiles (16 x 64)
  unsigned char* Tp;    // [ntT][kphi] B tiles (128 x 64)
  unsigned char* Lp;    // [Lmax + 1] B tiles (s x 16)
  unsigned char* Cp;    // near-field pool: [(noff[b] + i) * (s / 64) + h] B tiles (s x 64)
  int* nnear;           // per target leaf: near source leaves (dense: every leaf)
  int* near;            // near[b * Lmax + i]
  int* noff;            // exclusive prefix sum of nnear
  int* order;           // target leaves by descending nnear (the output stage's job order)
  const int* fL;        // the plan's leaf counts and offsets (FmmPlan::L)
  // FP16 2-term split (SVDUP_MIXED_FP16X2): every tile holds two FP16 planes (hi, lo) of
  // its values times 2^sc, sc one power of two per tile, in the same geometry as the
  // three BF16 planes (the third plane unused); the scales, one byte per tile, parallel
  // the tile arrays.
  int fp16;
  signed char *scX, *scPhi, *scPsi, *scS, *scT, *scL, *scC;
  // The orthogonalising refinement's two GEMMs (RefPlan) reuse this kernel's pipeline:
  // for them rows, rt, kx and Xp describe X's plain split tiles and the fields below the
  // rest.
  int cols, ct;         // columns of X and their 128-column tiles
  double* Xr;           // X itself (FP64, column-major), updated in place
  long long ldxr;
  unsigned char* Xt;    // X^T split tiles [ct][ceil(rows / 64)] (128 columns x 64 rows)
  unsigned char* Et;    // E = X^T X - I split tiles [ct][ceil(cols / 64)]
  int kr;               // ceil(rows / 64)
  const int* gate;      // refinement runs only where *gate != 0
  // Pipeline waits give up after wait_ns of global time (0: one second).  stall != 0
  // is the failure test's switch: the drains then never hand a tensor-memory region
  // back, so the MMA issuer's wait runs out and the kernel reports SVDUP_ETIMEOUT.
  unsigned long long wait_ns;
  int stall;
};

// Scratch of the refinement of an up-to rows x cols matrix (svdup_mixed.cu).
struct RefWs {
  MixPlan mp;      // tile buffers and sizes (see above)
  double* probe;   // 4 x cols probe vectors, then 4 x rows and 4 x cols products
  double* res;     // the probe residual (1)
  int* gate;       // 1 when the residual exceeded the tolerance
};
size_t refine_ws_bytes(int rows, int cols);
RefWs refine_ws_carve(void* base, int rows, int cols);
// One Newton-Schulz step X <- X (3 I - X^T X) / 2 = X - X E / 2, E = X^T X - I, on the
// tensor cores (E in the 3-term BF16 split, X E in one BF16 product), queued only where
// a probe residual ||X^T X w - w|| / ||w|| over four fixed +-1 vectors w exceeds tol
// (tol <= 0: always).
void launch_refine(cudaStream_t st, double* X, long long ldx, int rows, int cols, RefWs ws,
                   double tol, int* status);

constexpr int kMixP = 16;
constexpr size_t kMixTileA = 3 * 128 * 64 * 2;  // A tile bytes (3 planes)

// Streaming multiprocessors of the current device (cached per device; svdup_solve.cu).
int device_sm_count();

// Host-side launchers (defined in svdup_solve.cu / svdup_product.cu / svdup_mixed.cu).  Each queues
// its kernels on `st` and adds to the launch counter.
void launch_gemv_pq(cudaStream_t st, int m, int n, const double* U, long long ldu, const double* V,
                    long long ldv, const double* a, const double* b, double* p, double* q,
                    double* ab, float2* abf, int* abe);
void launch_fill_left(cudaStream_t st, Eig e, int m, const double* S, const double* p,
                      const double* q, const double* ab, double* z2p, double* rho2, int* status);
void launch_fill_right(cudaStream_t st, Eig e, int m, int n, const double* S, const double* p,
                       const double* q, const double* ab, double* z4p, double* rho4, int* status);
void launch_fill_second(cudaStream_t st, Eig e, const double* lam_prev, const double* zsec);
void launch_fill_generic(cudaStream_t st, Eig e, const double* d, const double* z,
                         const double* rho, int* status);
void launch_deflate(cudaStream_t st, Eig e, int* status);
void launch_secular(cudaStream_t st, Eig e, int* status, int maxit);
void launch_secular_direct(cudaStream_t st, Eig e, int k, const double* d, const double* z,
                           int* status, int maxit);
void launch_merge(cudaStream_t st, Eig e);
void launch_loewner(cudaStream_t st, Eig e);
void launch_loewner_df(cudaStream_t st, Eig e);
// Far-field forms (svdup_vfmm.cu), for k >= kmin (every kernel returns at once below):
// Loewner's zhat, and the column norms with Q^T y (ysorted may be null).
void launch_vf_loewner(cudaStream_t st, Eig e, int kmin);
void launch_vf_norms(cudaStream_t st, Eig e, int kmin, const double* ysorted, double* out_final,
                     bool keep_inv);
// Q x for the sign pairing: vsorted[idx[t]] = zhat_t sum_j x_rank(j) inv_j / (d_t - mu_j).
void launch_vf_applyq(cudaStream_t st, Eig e, int kmin, const double* xfinal, double* vsorted);
// pairs = true: the sums in double-float arithmetic (svdup_dfsum.cu), for outputs that
// need FP32 accuracy only (the mixed mode's vectors and signs)
// keep_inv: the stored 1/||c_j|| stay as they are (the norms are recomputed for the
// product only), for calls that may run beside a product reading them
void launch_norms(cudaStream_t st, Eig e, const double* ysorted, double* out_final,
                  bool pairs = false, bool keep_inv = false);
void launch_apply_qt(cudaStream_t st, Eig e, const double* xphys, double* work, double* out_final,
                     bool pairs = false, bool keep_inv = false);
void launch_apply_q(cudaStream_t st, Eig e, const double* xfinal, double* work, double* yphys,
                    bool pairs = false);
void launch_norms_df(cudaStream_t st, Eig e, const double* ysorted, double* out_final, int blocks,
                     bool keep_inv = false);
void launch_apply_q_core_df(cudaStream_t st, Eig e, const double* xfinal, double* vsorted,
                            int blocks);
void launch_sign_combine(cudaStream_t st, int m, int n, const double* S, const double* p,
                         const double* q, const double* g, double* y);
void launch_sign_finish(cudaStream_t st, int m, int n, const double* h, double* sign);
void launch_sign_apply(cudaStream_t st, int m, int n, double* V, long long ldv, const double* sign);
void launch_fill_ones(cudaStream_t st, int n, double* w);
void launch_sqrt_desc(cudaStream_t st, int m, const double* lam, double* S, int* status);
// synthetic inputs for the autotuner
void launch_fill_random(cudaStream_t st, int rows, int N, double* X, double* d, double* z,
                        unsigned long long seed);

// scratch: rotate_scratch_bytes(N, rows) bytes, 16-byte aligned; mixed: FP32-accurate
// arithmetic (see svdup_product.cu)
size_t rotate_scratch_bytes(int N, int rows);
// Deflated columns (rotation outputs) go straight to their output column in om.
void launch_rotate_prepare(cudaStream_t st, Eig e, const void* X, long long ldx, int rows,
                           void* scratch, bool mixed, bool xf32);
void launch_rotate_apply(cudaStream_t st, Eig e, void* X, long long ldx, int rows,
                         void* scratch, bool mixed, OutMap om, bool xf32);
void launch_rotate_columns(cudaStream_t st, Eig e, double* X, long long ldx, int rows,
                           void* scratch, bool mixed, OutMap om);
void launch_gather_columns(cudaStream_t st, Eig e, const double* X, long long ldx, int rows,
                           double* Xs, long long ldxs, OutMap om);
void launch_fmm_boxes(cudaStream_t st, Eig e, FmmPlan f, int dense);
void launch_fmm_ops(cudaStream_t st, Eig e, FmmPlan f, int dense);
void launch_fmm_setup(cudaStream_t st, Eig e, FmmPlan f, int dense);
// Flop accumulators of a handle's timers: useful flops of P2M, M2L, OUT (0..2), executed
// tensor-core flops (3..5), algorithmic flops (6..8).
constexpr int kFlopSlots = 9;
// adds the useful flops of one product's P2M, M2L and output stages to acc[0..2] and
// their algorithmic flops to acc[6..8]
void launch_flop_count(cudaStream_t st, Eig e, FmmPlan f, int rows, int dense, double* acc);
// stage 0 = P2M, 1 = M2L, 2 = L2P + near field (dense: the whole product)
void launch_product_f64_stage(cudaStream_t st, int stage, Eig e, FmmPlan f, int rows,
                              const double* Xs, long long ldxs, OutMap om, int dense);
// FP64 hierarchy (svdup_tree.cu): boxes, interaction lists and shift operators of every
// level (after launch_fmm_ops), and the translations: upward shifts of the far-field
// expansions, the per-level translations into local expansions, downward shifts.
void launch_tree_setup(cudaStream_t st, Eig e, FmmPlan f);
void launch_tree_translate(cudaStream_t st, Eig e, FmmPlan f, int rows);
// useful flops of the hierarchy's translations, added to acc[1]
void launch_tree_flops(cudaStream_t st, FmmPlan f, int rows, double* acc);

// mixed-precision product (svdup_mixed.cu)
void launch_mix_gather(cudaStream_t st, Eig e, const void* X, bool xf32, long long ldx, int rows,
                       MixPlan mp, OutMap om);
void launch_mix_setup(cudaStream_t st, Eig e, FmmPlan f, MixPlan mp, int dense);
// stage 0 = P2M, 1 = M2L, 2 = L2P + near field (dense: the whole product)
void launch_mix_stage(cudaStream_t st, int stage, Eig e, FmmPlan f, MixPlan mp, OutMap om,
                      int dense, int* status);
// adds the executed tensor-core flops (2 per multiply-add of every split product) of the
// three stages to acc[0..2]
void launch_mix_flop_count(cudaStream_t st, Eig e, FmmPlan f, MixPlan mp, int dense,
                           double* acc);

}  // namespace svdup
