// svdup_api.cu -- host side of libsvdup.so: handles, workspace, and the order in which
// the stages of Alg. 6.1 are queued on the handle's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>

#include "svdup_internal.cuh"

namespace svdup {

// Kernels launched by this process (all handles and threads; the serving engine's
// scheduler thread launches beside the caller's).  Launches made while this thread
// records a batch graph are counted when the graph is launched, not here.
std::atomic<long long> g_launch_count{0};
static thread_local bool t_recording = false;

static int debug_mode() {
  static const int v = [] {
    const char* e = getenv("SVDUP_DEBUG");
    return (e && e[0] && e[0] != '0') ? 1 : 0;
  }();
  return v;
}

static std::atomic<int> g_debug_err{cudaSuccess};  // first failure seen in debug mode

void note_launch(const char* file, int line) {
  if (t_recording) return;  // a captured launch: no device synchronisation either
  g_launch_count.fetch_add(1, std::memory_order_relaxed);
  if (!debug_mode()) return;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    fprintf(stderr, "svdup: kernel launched at %s:%d failed: %s\n", file, line,
            cudaGetErrorString(e));
    int none = cudaSuccess;
    g_debug_err.compare_exchange_strong(none, (int)e);
  }
}

}  // namespace svdup

using namespace svdup;

struct TimerRec {
  int stage;
  cudaEvent_t a, b;
};

struct svdup_ctx {
  int device;
  cudaStream_t stream;
  int* status;  // device word
  char* ws;
  size_t ws_size;
  int maxit;
  double refine_tol;  // SVDUP_REFINE: probe residual above which the step runs
  int test_stall;     // svdup_check_timeout: the tensor-core drains hold their regions
  unsigned long long test_wait_ns;  // and the pipeline waits give up after this long
  double* ref_res;    // device: the last probe residuals of U and V (SVDUP_REFINE)
  char* hb;           // svdup_update_host's device copies of U, S, V, a, b (kept)
  size_t hb_size;
  // stage timers
  int timing;
  TimerRec* recs;
  int nrec, caprec;
  TimerRec* pool;  // recycled event pairs
  int npool, cappool;
  double ms[SVDUP_NSTAGE];
  long long cnt[SVDUP_NSTAGE];
  int open_stage;
  cudaEvent_t open_ev;
  double* flops_dev;  // kFlopSlots accumulators, device: useful flops of P2M, M2L, OUT,
                      // the executed tensor-core flops of the same stages (mixed modes),
                      // then their algorithmic flops (App. D's operation count)
  // product-path choices (set by svdup_autotune; defaults below): index 0 FP64, 1 mixed
  int dense_max[2];   // N <= dense_max: dense Cauchy product (no far field)
  int leaf128_min[2]; // N >= leaf128_min: leaves of 128 poles, else 64
  int vf_min, vf_min_pairs;  // Loewner and the norms: the far-field form from these k
  int dense_w128_min[2];  // dense products with N >= this: 128-column output tiles, else 64
  // the right-hand problem of an update runs on `side`, beside the left-hand one; the
  // products of each side run on prod[0] (U) and prod[1] (V)
  cudaStream_t side;   // the right-hand solves (high priority)
  cudaStream_t left;   // the left-hand solves (high priority)
  cudaStream_t prod[2];  // the products with U and with V (low priority)
  cudaEvent_t ev_fork, ev_mid, ev_join, ev_copy;
  // e1 ready, e2 ready, e3 ready, e4 ready, U done, V done, left done, e1 deflated,
  // e1 merged, e3 deflated, e3 merged, e2 deflated, e2 leaves, e4 deflated, e4 leaves
  cudaEvent_t ev[15];
};

namespace {

// Bump allocator over the workspace; `base == nullptr` only measures.
struct Arena {
  char* base;
  size_t off;
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    T* p = base ? (T*)(base + off) : nullptr;
    off += bytes;
    return p;
  }
};

Eig make_eig(Arena& ar, int N) {
  Eig e;
  memset(&e, 0, sizeof(e));
  e.N = N;
  size_t n = (size_t)(N > 0 ? N : 1);
  e.rhop = ar.take<double>(1);
  e.ds = ar.take<double>(n);
  e.zs = ar.take<double>(n);
  e.perm = ar.take<int>(n);
  e.defl = ar.take<int>(n);
  e.nrot = ar.take<int>(1);
  e.rj = ar.take<int>(n);
  e.ri = ar.take<int>(n);
  e.rc = ar.take<double>(n);
  e.rs = ar.take<double>(n);
  e.kp = ar.take<int>(1);
  e.idx = ar.take<int>(n);
  e.didx = ar.take<int>(n);
  e.dk = ar.take<double>(n);
  e.zk = ar.take<double>(n);
  e.dc = ar.take<double>(n);
  e.z2c = ar.take<double>(n);
  e.org = ar.take<int>(n);
  e.tau = ar.take<double>(n);
  e.dorg = ar.take<double>(n);
  e.orgc = ar.take<int>(n);
  e.tauc = ar.take<double>(n);
  e.zhat = ar.take<double>(n);
  e.inv = ar.take<double>(n);
  e.lam = ar.take<double>(n);
  e.rank_root = ar.take<int>(n);
  e.rank_defl = ar.take<int>(n);
  e.tol = ar.take<double>(1);
  e.sd = ar.take<double>(n);
  e.sz = ar.take<double>(n);
  e.spos = ar.take<int>(n);
  e.sbrk = ar.take<unsigned char>(n);
  e.srix = ar.take<int>(n);
  e.skix = ar.take<int>(n);
  e.srs = ar.take<int>(n);
  e.dmask = ar.take<unsigned>((n + 31) / 32 + 1);
  e.dint = ar.take<int>(4);
  e.dflt = ar.take<double>(4);
  e.ovh = ar.take<int>(kMaxOverrunList);
  e.ovW = ar.take<float2>(kMaxOverrunList);
  e.ovM = ar.take<float2>(kMaxOverrunList);
  e.ovR = ar.take<double>(kMaxOverrunList);
  const size_t nbox = (n + 63) / 64;
  e.sqb = ar.take<double>(2 * nbox);
  e.sqn = ar.take<int>(2 * nbox);
  e.sqf = ar.take<int>(8);
  e.z2f = ar.take<float2>(n);
  e.sqv = ar.take<double>(4 * 26 * nbox);
  e.fsc = ar.take<int>(4);
  e.tf = ar.take<float2>(n);
  e.zf = ar.take<float2>(n);
  e.yf = ar.take<float2>(n);
  e.wf = ar.take<float2>(n);
  e.vfmin = kVfDefault;
  e.vfmin_pairs = kVfDefaultPairs;
  if (N >= kVfMinK) {
    e.vf = ar.take<double>(vf_doubles(N));
    e.vfc = ar.take<int>(vf_ints(N));
  }
  return e;
}

// Expansion order from the accuracy.  App. D STEP 1 takes p = log5(1/eps), the
// convergence rate of two-sided Chebyshev interpolation of 1/(x - y) between leaves two
// radii apart (the paper's interaction lists).  The flat partition here admits leaf
// pairs one radius apart, where the error is 4 (2 + sqrt 3)^-p of the pair's largest
// kernel entry (the Bernstein-ellipse rate for a singularity two radii from the leaf
// centre), so p is chosen from that rate.  Leaf size: about 2p points per leaf in the
// paper (STEP 2); here leaves are wider so the near field stays a few leaves across on
// graded spectra (relative leaf widths shrink with more leaves) while the far field is
// a handful of large contractions.
int expansion_order(double eps) {
  int p = (int)ceil(log(4.0 / eps) / log(2.0 + sqrt(3.0)));
  if (p < 4) p = 4;
  if (p > 32) p = 32;
  return p;
}

// Defaults of the product-path choices (svdup_autotune measures and replaces them).
constexpr int kDefaultDenseMax = 512;
constexpr int kDefaultLeaf128Min = 2049;
constexpr int kDefaultLeaf128MinTree = 1 << 30;

int mode_index(int mode) { return (mode & SVDUP_MODE_MASK) == SVDUP_FP64 ? 0 : 1; }

bool use_dense(const svdup_ctx* h, int N, int mode) {
  if (mode & SVDUP_DENSE) return true;
  return N <= h->dense_max[mode_index(mode)];
}

// Leaf size, which is also the output tile width of the mixed dense product (the dense
// product lists every leaf as near): the far field's choice, or the dense one.
int leaf_size(const svdup_ctx* h, int N, int mode) {
  const int i = mode_index(mode);
  if (use_dense(h, N, mode)) return N >= h->dense_w128_min[i] ? 128 : 64;
  return N >= h->leaf128_min[i] ? 128 : 64;
}

// mixed: P = 16 nodes (the split products' K granularity; 5^-16 is far below the FP32
// accumulation error) and no FP64 expansions (the split tiles of the MixPlan hold them).
FmmPlan make_plan(Arena& ar, int N, int rows, double eps, int leaf, bool mixed) {
  FmmPlan f;
  memset(&f, 0, sizeof(f));
  f.p = mixed ? kMixP : expansion_order(eps);
  const size_t rrows = (size_t)(rows > 0 ? rows : 1);
  if (mixed) rows = 1;
  f.s = leaf;
  f.Lmax = (N + f.s - 1) / f.s + 1;  // one more for the leaf offset (k_fmm_boxes)
  size_t L = (size_t)f.Lmax;
  f.L = ar.take<int>(4);
  f.sbox_c = ar.take<double>(L);
  f.sbox_r = ar.take<double>(L);
  f.tbox_c = ar.take<double>(L + 1);
  f.tbox_r = ar.take<double>(L + 1);
  f.tj0 = ar.take<int>(L + 1);
  f.tj1 = ar.take<int>(L + 1);
  f.nnear = ar.take<int>(L + 1);
  f.near = ar.take<int>((L + 1) * L);
  f.S = ar.take<double>(L * f.s * f.p);
  f.Lop = ar.take<double>((L + 1) * f.s * f.p);
  f.ldphi = rows > 0 ? rows : 1;
  // FP64: the hierarchy of App. D (svdup_tree.cu); mixed: the flat translation matrix
  f.tree = mixed ? 0 : 1;
  size_t nbox = L;  // expansion column blocks
  if (f.tree) {
    f.Hmax = tree_levels(f.Lmax);
    const size_t tot = (size_t)tree_off(f.Lmax, f.Hmax);
    f.H = ar.take<int>(1);
    f.hsc = ar.take<double>(tot);
    f.hsr = ar.take<double>(tot);
    f.htc = ar.take<double>(tot);
    f.htr = ar.take<double>(tot);
    f.hte = ar.take<int>(tot);
    f.hnl = ar.take<int>(tot);
    f.hl = ar.take<int>(tot * (L + 1));
    f.M2M = ar.take<double>(tot * f.p * f.p);
    f.L2L = ar.take<double>(tot * f.p * f.p);
    nbox = tot;
  } else {
    f.T = ar.take<double>(L * f.p * (L + 1) * f.p);
  }
  if (rows > 0) {  // operand scratch (a shared plan takes its partner's)
    f.Phi = ar.take<double>((size_t)f.ldphi * nbox * f.p);
    f.Psi = ar.take<double>((size_t)f.ldphi * (nbox + 1) * f.p);
    f.rot = ar.take<unsigned char>(rotate_scratch_bytes(N, (int)rrows));
  }
  return f;
}

// Split-tile buffers of the mixed product for up to `rows` rows and N columns (plan f).
// A second plan for the same rows: its own leaves and operators (set up while the first
// product still runs), the operand scratch (Phi, Psi, rotation scratch) shared.
FmmPlan make_plan_shared(Arena& ar, int N, double eps, int leaf, bool mixed, const FmmPlan& sh) {
  FmmPlan f = make_plan(ar, N, 0, eps, leaf, mixed);
  f.ldphi = sh.ldphi;
  f.Phi = sh.Phi;
  f.Psi = sh.Psi;
  f.rot = sh.rot;
  return f;
}

MixPlan make_mix(Arena& ar, int rows, const FmmPlan& f) {
  MixPlan mp;
  memset(&mp, 0, sizeof(mp));
  mp.rows = rows;
  mp.rt = (rows + 127) / 128;
  mp.s = f.s;
  mp.fL = f.L;
  mp.Lmax = f.Lmax;
  mp.kx = f.Lmax * f.s / 64;
  mp.kphi = (f.Lmax * kMixP + 63) / 64;
  mp.ntT = ((f.Lmax + 1) * kMixP + 127) / 128;
  const size_t hs = (size_t)f.s / 64, L = (size_t)f.Lmax;
  mp.Xp = ar.take<unsigned char>((size_t)mp.rt * mp.kx * kMixTileA);
  mp.Phip = ar.take<unsigned char>((size_t)mp.rt * mp.kphi * kMixTileA);
  mp.Psip = ar.take<unsigned char>((size_t)mp.rt * (L + 1) * (3 * 128 * kMixP * 2));
  mp.Sp = ar.take<unsigned char>(L * hs * (3 * kMixP * 64 * 2));
  mp.Tp = ar.take<unsigned char>((size_t)mp.ntT * mp.kphi * kMixTileA);
  mp.Lp = ar.take<unsigned char>((L + 1) * (3 * (size_t)f.s * kMixP * 2));
  mp.Cp = ar.take<unsigned char>((L + 1) * L * hs * (3 * (size_t)f.s * 64 * 2));
  mp.nnear = ar.take<int>(L + 1);
  mp.near = ar.take<int>((L + 1) * L);
  mp.noff = ar.take<int>(L + 2);
  mp.order = ar.take<int>(L + 1);
  mp.scX = ar.take<signed char>((size_t)mp.rt * mp.kx);
  mp.scPhi = ar.take<signed char>((size_t)mp.rt * mp.kphi);
  mp.scPsi = ar.take<signed char>((size_t)mp.rt * (L + 1));
  mp.scS = ar.take<signed char>(L * hs);
  mp.scT = ar.take<signed char>((size_t)mp.ntT * mp.kphi);
  mp.scL = ar.take<signed char>(L + 1);
  mp.scC = ar.take<signed char>((L + 1) * L * hs);
  return mp;
}

// The second product's mixed plan: own operator tiles and lists, shared split operands.
MixPlan make_mix_shared(Arena& ar, const FmmPlan& f, const MixPlan& sh) {
  MixPlan mp = sh;
  mp.fL = f.L;
  const size_t hs = (size_t)f.s / 64, L = (size_t)f.Lmax;
  mp.Sp = ar.take<unsigned char>(L * hs * (3 * kMixP * 64 * 2));
  mp.Tp = ar.take<unsigned char>((size_t)mp.ntT * mp.kphi * kMixTileA);
  mp.Lp = ar.take<unsigned char>((L + 1) * (3 * (size_t)f.s * kMixP * 2));
  mp.Cp = ar.take<unsigned char>((L + 1) * L * hs * (3 * (size_t)f.s * 64 * 2));
  mp.nnear = ar.take<int>(L + 1);
  mp.near = ar.take<int>((L + 1) * L);
  mp.noff = ar.take<int>(L + 2);
  mp.order = ar.take<int>(L + 1);
  mp.scS = ar.take<signed char>(L * hs);
  mp.scT = ar.take<signed char>((size_t)mp.ntT * mp.kphi);
  mp.scL = ar.take<signed char>(L + 1);
  mp.scC = ar.take<signed char>((L + 1) * L * hs);
  return mp;
}

bool is_mixed(int mode) {
  const int prec = mode & SVDUP_MODE_MASK;
  return prec == SVDUP_MIXED_BF16X3 || prec == SVDUP_MIXED_FP16X2;
}

bool is_fp16(int mode) { return (mode & SVDUP_MODE_MASK) == SVDUP_MIXED_FP16X2; }

bool mode_ok(int mode) {
  int prec = mode & SVDUP_MODE_MASK;
  if (prec != SVDUP_FP64 && prec != SVDUP_MIXED_BF16X3 && prec != SVDUP_MIXED_FP16X2) return false;
  return (mode & ~(SVDUP_MODE_MASK | SVDUP_DENSE | SVDUP_REFINE)) == 0;
}

int ensure_ws(svdup_ctx* h, size_t bytes) {
  if (bytes <= h->ws_size) return SVDUP_OK;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SVDUP_ECUDA;
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_size = 0;
  void* p = nullptr;
  size_t want = bytes + bytes / 8;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    return SVDUP_ENOMEM;
  }
  h->ws = (char*)p;
  h->ws_size = want;
  return SVDUP_OK;
}

int check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {  // a failure that note_launch consumed in debug mode
    const int d = g_debug_err.exchange(cudaSuccess);
    if (d != cudaSuccess) e = (cudaError_t)d;
  }
  return e == cudaSuccess ? SVDUP_OK : SVDUP_ECUDA;
}

int set_device(svdup_ctx* h) {
  return cudaSetDevice(h->device) == cudaSuccess ? SVDUP_OK : SVDUP_ECUDA;
}

// The per-update workspace.
// Update workspace.  The left-hand (U) and right-hand (V) problems own their scratch
// (ysort, the product's plan, W and Xs) so that they can run side by side.
struct UpdateWs {
  float2* abf;  // a, b as scaled FP32 pairs (STEP 1)
  int* abe;     // their scales
  double *p, *q, *ab, *z2p, *z4p, *ysortL, *ysortR, *zsec2, *zsec4, *ones, *g1, *g, *yv, *h1,
      *h, *sign, *work;
  Eig E1, E2, E3, E4;
  double *XsL, *XsR, *WL, *WR;
  float *WLf, *WRf;  // the mixed form's intermediates (FP32-accurate by construction)
  FmmPlan FL, FR, FL2, FR2;  // the second products' plans (mixed: own operators)
  MixPlan ML, MR, ML2, MR2;
  char* refbase;  // the refinement's scratch (SVDUP_REFINE), for n x n and smaller
};

UpdateWs layout_update(Arena& ar, int m, int n, double eps, int leaf, bool mixed,
                       bool fp16 = false, bool refine = false) {
  UpdateWs u;
  u.refbase = refine ? ar.take<char>(refine_ws_bytes(n, n)) : nullptr;
  u.p = ar.take<double>(m);
  u.q = ar.take<double>(n);
  u.ab = ar.take<double>(2);
  u.abf = ar.take<float2>((size_t)m + n);
  u.abe = ar.take<int>(2);
  u.z2p = ar.take<double>(m);
  u.z4p = ar.take<double>(n);
  u.ysortL = ar.take<double>(m);
  u.ysortR = ar.take<double>(n);
  u.zsec2 = ar.take<double>(m);
  u.zsec4 = ar.take<double>(n);
  u.ones = ar.take<double>(m);
  u.g1 = ar.take<double>(m);
  u.g = ar.take<double>(m);
  u.yv = ar.take<double>(n);
  u.h1 = ar.take<double>(n);
  u.h = ar.take<double>(n);
  u.sign = ar.take<double>(n);
  u.work = ar.take<double>(n);
  u.E1 = make_eig(ar, m);
  u.E2 = make_eig(ar, m);
  u.E3 = make_eig(ar, n);
  u.E4 = make_eig(ar, n);
  u.XsL = mixed ? nullptr : ar.take<double>((size_t)m * m);
  u.XsR = mixed ? nullptr : ar.take<double>((size_t)n * n);
  u.WL = mixed ? nullptr : ar.take<double>((size_t)m * m);
  u.WR = mixed ? nullptr : ar.take<double>((size_t)n * n);
  u.WLf = mixed ? ar.take<float>((size_t)m * m) : nullptr;
  u.WRf = mixed ? ar.take<float>((size_t)n * n) : nullptr;
  u.FL = make_plan(ar, m, m, eps, leaf, mixed);
  u.FR = make_plan(ar, n, n, eps, leaf, mixed);
  memset(&u.ML, 0, sizeof(u.ML));
  memset(&u.MR, 0, sizeof(u.MR));
  u.FL2 = u.FL;
  u.FR2 = u.FR;
  u.ML2 = u.ML;
  u.MR2 = u.MR;
  if (mixed) {
    u.ML = make_mix(ar, m, u.FL);
    u.MR = make_mix(ar, n, u.FR);
    u.FL2 = make_plan_shared(ar, m, eps, leaf, mixed, u.FL);
    u.FR2 = make_plan_shared(ar, n, eps, leaf, mixed, u.FR);
    u.ML2 = make_mix_shared(ar, u.FL2, u.ML);
    u.MR2 = make_mix_shared(ar, u.FR2, u.MR);
    u.ML.fp16 = u.MR.fp16 = u.ML2.fp16 = u.MR2.fp16 = fp16 ? 1 : 0;
  }
  return u;
}

// Stage timers: an event pair per timed interval, resolved at svdup_timing_read.
cudaEvent_t take_event(svdup_ctx* h) {
  cudaEvent_t e = nullptr;
  if (h->npool > 0) {
    TimerRec& r = h->pool[--h->npool];
    e = r.a;
    if (r.b) {  // split pairs back into single events
      if (h->npool + 1 > h->cappool) {
        h->cappool = h->cappool ? 2 * h->cappool : 64;
        h->pool = (TimerRec*)realloc(h->pool, h->cappool * sizeof(TimerRec));
      }
      h->pool[h->npool++] = TimerRec{-1, r.b, nullptr};
    }
    return e;
  }
  cudaEventCreate(&e);
  return e;
}

// With timing == SVDUP_TIMING_STAGES every stage is timed and the update runs on one
// stream; with SVDUP_TIMING_KERNELS only the three product-stage kernels are, each on
// the stream it is launched on, and the update keeps its multi-stream schedule.  The
// host queues a stage's begin, launch and end back to back, so one open slot suffices.
bool stage_timed(const svdup_ctx* h, int stage) {
  if (h->timing == SVDUP_TIMING_STAGES) return true;
  return h->timing == SVDUP_TIMING_KERNELS &&
         (stage == SVDUP_STAGE_P2M || stage == SVDUP_STAGE_M2L || stage == SVDUP_STAGE_OUT);
}

void stage_begin(svdup_ctx* h, int stage, cudaStream_t st) {
  if (!stage_timed(h, stage)) return;
  h->open_stage = stage;
  h->open_ev = take_event(h);
  cudaEventRecord(h->open_ev, st);
}

void stage_end(svdup_ctx* h, cudaStream_t st) {
  if (!h->timing || h->open_stage < 0) return;
  cudaEvent_t b = take_event(h);
  cudaEventRecord(b, st);
  if (h->nrec + 1 > h->caprec) {
    h->caprec = h->caprec ? 2 * h->caprec : 256;
    h->recs = (TimerRec*)realloc(h->recs, h->caprec * sizeof(TimerRec));
  }
  h->recs[h->nrec++] = TimerRec{h->open_stage, h->open_ev, b};
  h->open_stage = -1;
}

// One solve: deflation, roots, final ordering, zhat; the column norms follow separately
// (fused with a transposed product when the next solve needs its z).
// pairs: Loewner's zhat in double-float arithmetic (svdup_dfsum.cu), for solves whose
// zhat feeds vectors only (never the z of another solve) in the mixed mode
// Optional events mark the deflation (enough for the first half of the rotations) and
// the merge (the final order, enough for the rest of a product's column work).
void queue_solve(svdup_ctx* h, cudaStream_t st, Eig e, bool pairs = false,
                 cudaEvent_t ev_defl = nullptr, cudaEvent_t ev_merge = nullptr) {
  launch_deflate(st, e, h->status);
  if (ev_defl) cudaEventRecord(ev_defl, st);
  launch_secular(st, e, h->status, h->maxit);
  launch_merge(st, e);
  if (ev_merge) cudaEventRecord(ev_merge, st);
  if (pairs) launch_loewner_df(st, e);
  else launch_loewner(st, e);
}

// Y[:, out(q)] = (X Q)[:, q] for the solve e (X rows x N, modified in place by the
// deflation rotations).  Xs is a rows x N scratch.  The stage timers record on the
// handle's stream: with timing on, every product runs there (st == h->stream).
void queue_product(svdup_ctx* h, cudaStream_t st, Eig e, FmmPlan f, int rows, double* X, long long ldx,
                   double* Xs, OutMap om, int mode) {
  int dense = use_dense(h, e.N, mode) ? 1 : 0;
  stage_begin(h, SVDUP_STAGE_GATHER, st);
  launch_rotate_columns(st, e, X, ldx, rows, f.rot, false, om);
  launch_gather_columns(st, e, X, ldx, rows, Xs, rows, om);
  stage_end(h, st);
  stage_begin(h, SVDUP_STAGE_SETUP, st);
  launch_fmm_setup(st, e, f, dense);
  if (!dense && f.tree) launch_tree_setup(st, e, f);
  stage_end(h, st);
  if (!dense) {
    stage_begin(h, SVDUP_STAGE_P2M, st);
    launch_product_f64_stage(st, 0, e, f, rows, Xs, rows, om, dense);
    stage_end(h, st);
    stage_begin(h, SVDUP_STAGE_M2L, st);
    if (f.tree) launch_tree_translate(st, e, f, rows);
    else launch_product_f64_stage(st, 1, e, f, rows, Xs, rows, om, dense);
    stage_end(h, st);
  }
  stage_begin(h, SVDUP_STAGE_OUT, st);
  launch_product_f64_stage(st, 2, e, f, rows, Xs, rows, om, dense);
  stage_end(h, st);
  if (h->timing) {
    launch_flop_count(st, e, f, rows, dense, h->flops_dev);
    if (!dense && f.tree) launch_tree_flops(st, f, rows, h->flops_dev);
  }
}

// The same product in split BF16 on the tensor cores (svdup_mixed.cu), in four phases
// that an update spreads over its streams as their inputs become ready:
//   prepare  the first half of the rotation scan           (deflation)
//   xside    [leaves], the rotations' replay, the split X   (roots and final order)
//   ops      [leaves], near lists, operator tiles           (zhat and column norms)
//   mma      the three tensor-core stages
// The gather places X's columns by the leaf offset that the leaves step finds, so the
// leaves come with whichever of xside and ops runs first.
MixPlan mix_rows(MixPlan mp, int rows) {
  mp.rows = rows;
  mp.rt = (rows + 127) / 128;
  return mp;
}

// X is FP64, or the FP32 intermediate when xf32.
void mix_prepare(svdup_ctx* h, cudaStream_t st, Eig e, FmmPlan f, int rows, const void* X,
                 bool xf32, long long ldx) {
  stage_begin(h, SVDUP_STAGE_GATHER, st);
  launch_rotate_prepare(st, e, X, ldx, rows, f.rot, true, xf32);
  stage_end(h, st);
}

void mix_xside(svdup_ctx* h, cudaStream_t st, Eig e, FmmPlan f, MixPlan mp, int rows, void* X,
               bool xf32, long long ldx, OutMap om, bool leaves) {
  mp = mix_rows(mp, rows);
  if (leaves) {
    stage_begin(h, SVDUP_STAGE_SETUP, st);
    launch_fmm_boxes(st, e, f, 0);
    stage_end(h, st);
  }
  stage_begin(h, SVDUP_STAGE_GATHER, st);
  launch_rotate_apply(st, e, X, ldx, rows, f.rot, true, om, xf32);
  launch_mix_gather(st, e, X, xf32, ldx, rows, mp, om);
  stage_end(h, st);
}

void mix_ops(svdup_ctx* h, cudaStream_t st, Eig e, FmmPlan f, MixPlan mp, int rows, int mode,
             bool leaves) {
  const int dense = use_dense(h, e.N, mode) ? 1 : 0;
  mp = mix_rows(mp, rows);
  stage_begin(h, SVDUP_STAGE_SETUP, st);
  if (leaves) launch_fmm_boxes(st, e, f, 0);
  launch_fmm_ops(st, e, f, 0);
  launch_mix_setup(st, e, f, mp, dense);
  stage_end(h, st);
}

void mix_mma(svdup_ctx* h, cudaStream_t st, Eig e, FmmPlan f, MixPlan mp, int rows, OutMap om,
             int mode) {
  const int dense = use_dense(h, e.N, mode) ? 1 : 0;
  mp = mix_rows(mp, rows);
  mp.stall = h->test_stall;
  mp.wait_ns = h->test_wait_ns;
  if (!dense) {
    stage_begin(h, SVDUP_STAGE_P2M, st);
    launch_mix_stage(st, 0, e, f, mp, om, dense, h->status);
    stage_end(h, st);
    stage_begin(h, SVDUP_STAGE_M2L, st);
    launch_mix_stage(st, 1, e, f, mp, om, dense, h->status);
    stage_end(h, st);
  }
  stage_begin(h, SVDUP_STAGE_OUT, st);
  launch_mix_stage(st, 2, e, f, mp, om, dense, h->status);
  stage_end(h, st);
  if (h->timing) {
    launch_flop_count(st, e, f, rows, dense, h->flops_dev);
    launch_mix_flop_count(st, e, f, mix_rows(mp, rows), dense, h->flops_dev + 3);
  }
}

// All four phases on one stream.
void queue_product_mixed(svdup_ctx* h, cudaStream_t st, Eig e, FmmPlan f, MixPlan mp, int rows,
                         void* X, bool xf32, long long ldx, OutMap om, int mode) {
  mix_prepare(h, st, e, f, rows, X, xf32, ldx);
  mix_xside(h, st, e, f, mp, rows, X, xf32, ldx, om, true);
  mix_ops(h, st, e, f, mp, rows, mode, false);
  mix_mma(h, st, e, f, mp, rows, om, mode);
}

// ---------------------------------------------------------------------------
// Batches: lane contexts share the parent's status word and counters but own a
// stream and a workspace.
// ---------------------------------------------------------------------------
// The side stream and the three events of the two-stream update.
int make_side(svdup_ctx* h) {
  // The solve chains are latency-bound and on the critical path; the products fill the
  // GPU around them.  Higher priority lets the solves' blocks go first.
  int lo = 0, hi = 0;
  bool ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi) == cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&h->left, cudaStreamNonBlocking, hi) == cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&h->prod[0], cudaStreamNonBlocking, lo) == cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&h->prod[1], cudaStreamNonBlocking, lo) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&h->ev_mid, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&h->ev_copy, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < 15; i++)
    ok = ok && cudaEventCreateWithFlags(&h->ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    h->side = nullptr;  // the update then runs on one stream
    return SVDUP_ECUDA;
  }
  return SVDUP_OK;
}

void free_side(svdup_ctx* h) {
  if (!h->side) return;
  cudaStreamSynchronize(h->side);
  cudaStreamSynchronize(h->left);
  cudaStreamSynchronize(h->prod[0]);
  cudaStreamSynchronize(h->prod[1]);
  cudaEventDestroy(h->ev_fork);
  cudaEventDestroy(h->ev_mid);
  cudaEventDestroy(h->ev_join);
  cudaEventDestroy(h->ev_copy);
  for (int i = 0; i < 15; i++) cudaEventDestroy(h->ev[i]);
  cudaStreamDestroy(h->prod[0]);
  cudaStreamDestroy(h->prod[1]);
  cudaStreamDestroy(h->left);
  cudaStreamDestroy(h->side);
  h->side = nullptr;
}

svdup_ctx* lane_create(const svdup_ctx* parent) {
  svdup_ctx* l = (svdup_ctx*)calloc(1, sizeof(svdup_ctx));
  if (!l) return nullptr;
  l->device = parent->device;
  if (cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    free(l);
    return nullptr;
  }
  if (make_side(l) != SVDUP_OK) {
    cudaStreamDestroy(l->stream);
    free(l);
    return nullptr;
  }
  l->status = parent->status;
  l->flops_dev = parent->flops_dev;
  l->ref_res = parent->ref_res;
  l->refine_tol = parent->refine_tol;
  l->maxit = parent->maxit;
  l->vf_min = parent->vf_min;
  l->vf_min_pairs = parent->vf_min_pairs;
  l->open_stage = -1;
  for (int i = 0; i < 2; i++) {
    l->dense_max[i] = parent->dense_max[i];
    l->leaf128_min[i] = parent->leaf128_min[i];
    l->dense_w128_min[i] = parent->dense_w128_min[i];
  }
  return l;
}

void lane_destroy(svdup_ctx* l) {
  if (!l) return;
  cudaStreamSynchronize(l->stream);
  free_side(l);
  if (l->ws) cudaFree(l->ws);
  if (l->hb) cudaFree(l->hb);
  cudaStreamDestroy(l->stream);
  free(l->recs);
  free(l->pool);
  free(l);
}

size_t update_ws_bytes(const svdup_ctx* h, int m, int n, double eps, int mode) {
  Arena meas = {nullptr, 0};
  layout_update(meas, m, n, eps, leaf_size(h, n, mode), is_mixed(mode));
  return meas.off;
}

bool problem_ok(const svdup_problem& p) {
  return p.U && p.S && p.V && p.a && p.b && p.m >= 1 && p.n >= p.m && p.ldu >= p.m &&
         p.ldv >= p.n;
}

}  // namespace

struct svdup_batch {
  svdup_ctx* parent;
  int count, lanes;
  svdup_problem* probs;
  int* lane_of;  // problem -> lane, problems queued in index order within a lane
  svdup_ctx** lane;
  cudaStream_t origin;
  cudaEvent_t fork;
  cudaEvent_t* join;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  double eps;
  int mode;
  long long kernels;  // launches recorded into the graph
};

namespace {

void batch_free(svdup_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->lane)
    for (int l = 0; l < b->lanes; l++) lane_destroy(b->lane[l]);
  if (b->join)
    for (int l = 0; l < b->lanes; l++)
      if (b->join[l]) cudaEventDestroy(b->join[l]);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  free(b->lane);
  free(b->join);
  free(b->probs);
  free(b->lane_of);
  free(b);
}

// Largest first to the least-loaded lane; cost ~ n^2 (m + n) (solves and products).
void assign_lanes(svdup_batch* b) {
  int* order = (int*)malloc(sizeof(int) * b->count);
  double* cost = (double*)malloc(sizeof(double) * b->count);
  double* load = (double*)calloc(b->lanes, sizeof(double));
  for (int i = 0; i < b->count; i++) {
    order[i] = i;
    const double m = b->probs[i].m, n = b->probs[i].n;
    cost[i] = n * n * (m + n);
  }
  // insertion sort by cost, descending (counts are modest)
  for (int i = 1; i < b->count; i++) {
    int v = order[i], j = i - 1;
    while (j >= 0 && cost[order[j]] < cost[v]) { order[j + 1] = order[j]; j--; }
    order[j + 1] = v;
  }
  for (int q = 0; q < b->count; q++) {
    int best = 0;
    for (int l = 1; l < b->lanes; l++)
      if (load[l] < load[best]) best = l;
    b->lane_of[order[q]] = best;
    load[best] += cost[order[q]];
  }
  free(order);
  free(cost);
  free(load);
}

// Queue every problem on its lane, between a fork on `origin` and a join back to it.
int batch_queue(svdup_batch* b) {
  if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) return SVDUP_ECUDA;
  for (int l = 0; l < b->lanes; l++)
    if (cudaStreamWaitEvent(b->lane[l]->stream, b->fork, 0) != cudaSuccess) return SVDUP_ECUDA;
  for (int i = 0; i < b->count; i++) {
    const svdup_problem& p = b->probs[i];
    int rc = svdup_update(b->lane[b->lane_of[i]], p.m, p.n, p.U, p.ldu, p.S, p.V, p.ldv, p.a, p.b,
                          b->eps, b->mode);
    if (rc) return rc;
  }
  for (int l = 0; l < b->lanes; l++) {
    if (cudaEventRecord(b->join[l], b->lane[l]->stream) != cudaSuccess) return SVDUP_ECUDA;
    if (cudaStreamWaitEvent(b->origin, b->join[l], 0) != cudaSuccess) return SVDUP_ECUDA;
  }
  return SVDUP_OK;
}

int batch_plan(svdup_t h, int count, const svdup_problem* probs, double eps, int mode, int lanes,
               svdup_batch** out) {
  *out = nullptr;
  if (!h || count < 1 || !probs || !(eps > 0.0 && eps < 1.0) || !mode_ok(mode)) return SVDUP_EINVAL;
  if (lanes == 0) lanes = 16;
  if (lanes < 1 || lanes > 64) return SVDUP_EINVAL;
  if (lanes > count) lanes = count;
  for (int i = 0; i < count; i++)
    if (!problem_ok(probs[i])) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  svdup_batch* b = (svdup_batch*)calloc(1, sizeof(svdup_batch));
  if (!b) return SVDUP_ENOMEM;
  b->parent = h;
  b->count = count;
  b->lanes = lanes;
  b->eps = eps;
  b->mode = mode;
  b->probs = (svdup_problem*)malloc(sizeof(svdup_problem) * count);
  b->lane_of = (int*)malloc(sizeof(int) * count);
  b->lane = (svdup_ctx**)calloc(lanes, sizeof(svdup_ctx*));
  b->join = (cudaEvent_t*)calloc(lanes, sizeof(cudaEvent_t));
  if (!b->probs || !b->lane_of || !b->lane || !b->join) { batch_free(b); return SVDUP_ENOMEM; }
  memcpy(b->probs, probs, sizeof(svdup_problem) * count);
  assign_lanes(b);
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    return SVDUP_ECUDA;
  }
  for (int l = 0; l < lanes; l++) {
    b->lane[l] = lane_create(h);
    if (!b->lane[l] || cudaEventCreateWithFlags(&b->join[l], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      batch_free(b);
      return SVDUP_ECUDA;
    }
  }
  // workspaces sized for each lane's largest problem now (nothing allocates later)
  for (int l = 0; l < lanes; l++) {
    size_t need = 0;
    for (int i = 0; i < count; i++)
      if (b->lane_of[i] == l) {
        size_t w = update_ws_bytes(h, probs[i].m, probs[i].n, eps, mode);
        if (w > need) need = w;
      }
    int rc = ensure_ws(b->lane[l], need);
    if (rc) { batch_free(b); return rc; }
  }
  *out = b;
  return SVDUP_OK;
}

}  // namespace

extern "C" {

int svdup_create(svdup_t* out, int device, void* stream, unsigned flags) {
  (void)flags;
  if (!out) return SVDUP_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return SVDUP_ECUDA;
  svdup_ctx* h = (svdup_ctx*)calloc(1, sizeof(svdup_ctx));
  if (!h) return SVDUP_ENOMEM;
  h->device = device;
  h->stream = (cudaStream_t)stream;
  h->maxit = 64;
  h->refine_tol = 1e-6;
  h->vf_min = kVfDefault;
  h->vf_min_pairs = kVfDefaultPairs;
  h->open_stage = -1;
  for (int i = 0; i < 2; i++) {
    h->dense_max[i] = kDefaultDenseMax;
    h->leaf128_min[i] = kDefaultLeaf128Min;
    h->dense_w128_min[i] = kDefaultLeaf128Min;
  }
  h->leaf128_min[0] = kDefaultLeaf128MinTree;  // FP64: the hierarchy keeps leaves small
  const char* mi = getenv("SVDUP_SECULAR_MAXIT");
  if (mi) h->maxit = atoi(mi);
  if (cudaMalloc(&h->status, sizeof(int)) != cudaSuccess) {
    free(h);
    return SVDUP_ENOMEM;
  }
  if (cudaMalloc(&h->flops_dev, kFlopSlots * sizeof(double)) != cudaSuccess ||
      cudaMemsetAsync(h->flops_dev, 0, kFlopSlots * sizeof(double), h->stream) != cudaSuccess) {
    cudaFree(h->status);
    free(h);
    return SVDUP_ENOMEM;
  }
  if (cudaMalloc(&h->ref_res, 2 * sizeof(double)) != cudaSuccess ||
      cudaMemsetAsync(h->ref_res, 0, 2 * sizeof(double), h->stream) != cudaSuccess) {
    cudaFree(h->flops_dev);
    cudaFree(h->status);
    free(h);
    return SVDUP_ENOMEM;
  }
  if (cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) != cudaSuccess ||
      make_side(h) != SVDUP_OK) {
    cudaFree(h->status);
    cudaFree(h->flops_dev);
    cudaFree(h->ref_res);
    free(h);
    return SVDUP_ECUDA;
  }
  *out = h;
  return SVDUP_OK;
}

int svdup_destroy(svdup_t h) {
  if (!h) return SVDUP_EINVAL;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  free_side(h);
  if (h->ws) cudaFree(h->ws);
  if (h->hb) cudaFree(h->hb);
  cudaFree(h->status);
  cudaFree(h->flops_dev);
  cudaFree(h->ref_res);
  for (int i = 0; i < h->nrec; i++) { cudaEventDestroy(h->recs[i].a); cudaEventDestroy(h->recs[i].b); }
  for (int i = 0; i < h->npool; i++) {
    cudaEventDestroy(h->pool[i].a);
    if (h->pool[i].b) cudaEventDestroy(h->pool[i].b);
  }
  free(h->recs);
  free(h->pool);
  free(h);
  return SVDUP_OK;
}

int svdup_timing(svdup_t h, int enable) {
  if (!h || enable < 0 || enable > SVDUP_TIMING_KERNELS) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SVDUP_ECUDA;
  // recycle outstanding records
  for (int i = 0; i < h->nrec; i++) {
    if (h->npool + 1 > h->cappool) {
      h->cappool = h->cappool ? 2 * h->cappool : 64;
      h->pool = (TimerRec*)realloc(h->pool, h->cappool * sizeof(TimerRec));
    }
    h->pool[h->npool++] = h->recs[i];
  }
  h->nrec = 0;
  for (int s = 0; s < SVDUP_NSTAGE; s++) { h->ms[s] = 0.0; h->cnt[s] = 0; }
  h->timing = enable;
  h->open_stage = -1;
  if (cudaMemsetAsync(h->flops_dev, 0, kFlopSlots * sizeof(double), h->stream) != cudaSuccess)
    return SVDUP_ECUDA;
  return SVDUP_OK;
}

int svdup_timing_read(svdup_t h, double* ms, long long* count, double* flops, double* mma_flops,
                      int nstage) {
  if (!h || nstage < 0 || nstage > SVDUP_NSTAGE) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  double fl[kFlopSlots] = {};
  if (cudaMemcpyAsync(fl, h->flops_dev, kFlopSlots * sizeof(double), cudaMemcpyDeviceToHost, h->stream) !=
      cudaSuccess)
    return SVDUP_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SVDUP_ECUDA;
  for (int i = 0; i < h->nrec; i++) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, h->recs[i].a, h->recs[i].b) != cudaSuccess) return SVDUP_ECUDA;
    h->ms[h->recs[i].stage] += t;
    h->cnt[h->recs[i].stage] += 1;
    if (h->npool + 1 > h->cappool) {
      h->cappool = h->cappool ? 2 * h->cappool : 64;
      h->pool = (TimerRec*)realloc(h->pool, h->cappool * sizeof(TimerRec));
    }
    h->pool[h->npool++] = h->recs[i];
  }
  h->nrec = 0;
  for (int s = 0; s < nstage; s++) {
    if (ms) ms[s] = h->ms[s];
    if (count) count[s] = h->cnt[s];
    int slot = s == SVDUP_STAGE_P2M ? 0 : s == SVDUP_STAGE_M2L ? 1 : s == SVDUP_STAGE_OUT ? 2 : -1;
    if (flops) flops[s] = slot >= 0 ? fl[slot] : 0.0;
    if (mma_flops) mma_flops[s] = slot >= 0 ? fl[3 + slot] : 0.0;
  }
  return SVDUP_OK;
}

int svdup_timing_read_alg(svdup_t h, double* alg_flops, int nstage) {
  if (!h || nstage < 0 || nstage > SVDUP_NSTAGE) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  double fl[kFlopSlots] = {};
  if (cudaMemcpyAsync(fl, h->flops_dev, kFlopSlots * sizeof(double), cudaMemcpyDeviceToHost,
                      h->stream) != cudaSuccess)
    return SVDUP_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SVDUP_ECUDA;
  for (int s = 0; s < nstage; s++) {
    int slot = s == SVDUP_STAGE_P2M ? 0 : s == SVDUP_STAGE_M2L ? 1 : s == SVDUP_STAGE_OUT ? 2 : -1;
    if (alg_flops) alg_flops[s] = slot >= 0 ? fl[6 + slot] : 0.0;
  }
  return SVDUP_OK;
}

int svdup_sync(svdup_t h) {
  if (!h) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  int st = 0;
  if (cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream) !=
      cudaSuccess)
    return SVDUP_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SVDUP_ECUDA;
  if (st != 0) {
    if (cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) != cudaSuccess) return SVDUP_ECUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SVDUP_ECUDA;
  }
  return st;
}

const char* svdup_error_string(int code) {
  switch (code) {
    case SVDUP_OK: return "ok";
    case SVDUP_EINVAL: return "invalid argument";
    case SVDUP_ENOMEM: return "out of device memory for the workspace";
    case SVDUP_ENOCONV: return "secular root did not converge within the iteration cap";
    case SVDUP_ENONFINITE: return "non-finite value in the inputs or an intermediate";
    case SVDUP_ECUDA: return "CUDA runtime error";
    case SVDUP_EORDER: return "singular values are not in descending order";
    case SVDUP_ETIMEOUT: return "a device-side wait gave up after its time limit";
    default: return "unknown error";
  }
}

long long svdup_launch_count(svdup_t h) {
  (void)h;
  return g_launch_count.load(std::memory_order_relaxed);
}

int svdup_update(svdup_t h, int m, int n, double* U, int ldu, double* S, double* V, int ldv,
                 const double* a, const double* b, double eps, int mode) {
  if (!h || !U || !S || !V || !a || !b) return SVDUP_EINVAL;
  if (m < 1 || n < m || ldu < m || ldv < n) return SVDUP_EINVAL;
  if (!(eps > 0.0 && eps < 1.0)) return SVDUP_EINVAL;
  if (!mode_ok(mode)) return SVDUP_EINVAL;
  const bool mixed = is_mixed(mode);
  if (set_device(h)) return SVDUP_ECUDA;
  Arena meas = {nullptr, 0};
  const int leaf = leaf_size(h, n, mode);
  const bool refine = (mode & SVDUP_REFINE) != 0;
  layout_update(meas, m, n, eps, leaf, mixed, false, refine);
  int rc = ensure_ws(h, meas.off);
  if (rc) return rc;
  Arena ar = {h->ws, 0};
  UpdateWs u = layout_update(ar, m, n, eps, leaf, mixed, is_fp16(mode), refine);
  u.E1.vfmin = u.E2.vfmin = u.E3.vfmin = u.E4.vfmin = h->vf_min;
  u.E1.vfmin_pairs = u.E2.vfmin_pairs = u.E3.vfmin_pairs = u.E4.vfmin_pairs = h->vf_min_pairs;
  cudaStream_t st = h->stream;

  // STEP 1 (rewritten): p = U^T a, q = V^T b, alpha, beta
  stage_begin(h, SVDUP_STAGE_GEMV, h->stream);
  launch_gemv_pq(st, m, n, U, ldu, V, ldv, a, b, u.p, u.q, u.ab, u.abf, u.abe);
  stage_end(h, h->stream);
  // Streams: the left-hand solves (E1, E2) on `left`, the right-hand ones (E3, E4) on
  // `side`, the products with U on prod[0] and with V on prod[1]; the handle's stream
  // forks them after STEP 1 and joins them before the signs are applied and STEP 8.
  // A side's first product needs only its first solve, so it runs beside the second
  // solve, and the second product follows the second solve.  V's second product writes
  // its columns unsigned; the sign pairing (which hands the left vectors' sums to the
  // right) runs meanwhile, and its signs are applied to V after the join.  With stage
  // timing on, everything runs on one stream.
  const bool multi = h->timing != SVDUP_TIMING_STAGES && h->side;
  cudaStream_t sR = multi ? h->side : st;
  cudaStream_t sL = multi ? h->left : st;
  cudaStream_t pU = multi ? h->prod[0] : st;
  cudaStream_t pV = multi ? h->prod[1] : st;
  auto hand = [&](cudaEvent_t ev, cudaStream_t from, cudaStream_t to) -> bool {
    return !multi || (cudaEventRecord(ev, from) == cudaSuccess &&
                      cudaStreamWaitEvent(to, ev, 0) == cudaSuccess);
  };
  if (!hand(h->ev_fork, st, sR) || (multi && cudaStreamWaitEvent(sL, h->ev_fork, 0) != cudaSuccess))
    return SVDUP_ECUDA;
  OutMap om1 = {u.WL, (long long)m, m, 0, u.WLf};
  OutMap om2 = {U, (long long)ldu, m, 1};
  OutMap om3 = {u.WR, (long long)n, n, 0, u.WRf};
  OutMap om4 = {V, (long long)ldv, n, 1};
  if (mixed && multi) {
    // Each product's column work starts as soon as its solve has deflated (the scan's
    // first half) and merged (the replay, the split X), beside the rest of the solve;
    // the second products' leaves and operators are set up on the solve streams while
    // the first products still run.
    auto wait = [&](cudaStream_t s_, cudaEvent_t ev) {
      return cudaStreamWaitEvent(s_, ev, 0) == cudaSuccess;
    };
    // STEPs 3, 6: first right solve; STEP 7: second right solve
    launch_fill_right(sR, u.E3, m, n, S, u.p, u.q, u.ab, u.z4p, u.E4.rhop, h->status);
    queue_solve(h, sR, u.E3, false, h->ev[9], h->ev[10]);
    launch_apply_qt(sR, u.E3, u.z4p, u.ysortR, u.zsec4, mixed);
    if (cudaEventRecord(h->ev[2], sR) != cudaSuccess) return SVDUP_ECUDA;  // E3 ready
    launch_fill_second(sR, u.E4, u.E3.lam, u.zsec4);
    queue_solve(h, sR, u.E4, mixed, h->ev[13]);
    launch_fmm_boxes(sR, u.E4, u.FR2, 0);  // V2's leaves (the roots suffice)
    if (cudaEventRecord(h->ev[14], sR) != cudaSuccess) return SVDUP_ECUDA;
    launch_norms(sR, u.E4, nullptr, nullptr, mixed);
    mix_ops(h, sR, u.E4, u.FR2, u.MR2, n, mode, false);
    if (cudaEventRecord(h->ev[3], sR) != cudaSuccess) return SVDUP_ECUDA;  // E4, V2's operators
    // STEPs 2, 4: first left solve; its transposed product gives the second left z
    launch_fill_left(sL, u.E1, m, S, u.p, u.q, u.ab, u.z2p, u.E2.rhop, h->status);
    queue_solve(h, sL, u.E1, false, h->ev[7], h->ev[8]);
    launch_apply_qt(sL, u.E1, u.z2p, u.ysortL, u.zsec2, mixed);
    if (cudaEventRecord(h->ev[0], sL) != cudaSuccess) return SVDUP_ECUDA;  // E1 ready
    // STEP 5: second left solve
    launch_fill_second(sL, u.E2, u.E1.lam, u.zsec2);
    queue_solve(h, sL, u.E2, mixed, h->ev[11]);
    launch_fmm_boxes(sL, u.E2, u.FL2, 0);  // U2's leaves (the roots suffice)
    if (cudaEventRecord(h->ev[12], sL) != cudaSuccess) return SVDUP_ECUDA;
    launch_norms(sL, u.E2, nullptr, nullptr, mixed);
    mix_ops(h, sL, u.E2, u.FL2, u.ML2, m, mode, false);
    if (cudaEventRecord(h->ev[1], sL) != cudaSuccess) return SVDUP_ECUDA;  // E2, U2's operators
    // products: U -> W -> U (descending), V -> W -> V (descending; the signs follow)
    if (!wait(pU, h->ev[7])) return SVDUP_ECUDA;
    mix_prepare(h, pU, u.E1, u.FL, m, U, false, ldu);
    if (!wait(pU, h->ev[8])) return SVDUP_ECUDA;
    mix_xside(h, pU, u.E1, u.FL, u.ML, m, U, false, ldu, om1, true);
    if (!wait(pU, h->ev[0])) return SVDUP_ECUDA;
    mix_ops(h, pU, u.E1, u.FL, u.ML, m, mode, false);
    mix_mma(h, pU, u.E1, u.FL, u.ML, m, om1, mode);
    if (!wait(pV, h->ev[9])) return SVDUP_ECUDA;
    mix_prepare(h, pV, u.E3, u.FR, n, V, false, ldv);
    if (!wait(pV, h->ev[10])) return SVDUP_ECUDA;
    mix_xside(h, pV, u.E3, u.FR, u.MR, n, V, false, ldv, om3, true);
    if (!wait(pV, h->ev[2])) return SVDUP_ECUDA;
    mix_ops(h, pV, u.E3, u.FR, u.MR, n, mode, false);
    mix_mma(h, pV, u.E3, u.FR, u.MR, n, om3, mode);
    // the second products: X is the first product's output (stream order)
    if (!wait(pV, h->ev[13])) return SVDUP_ECUDA;
    mix_prepare(h, pV, u.E4, u.FR2, n, u.WRf, true, n);
    if (!wait(pV, h->ev[14])) return SVDUP_ECUDA;
    mix_xside(h, pV, u.E4, u.FR2, u.MR2, n, u.WRf, true, n, om4, false);
    if (!wait(pV, h->ev[3])) return SVDUP_ECUDA;
    mix_mma(h, pV, u.E4, u.FR2, u.MR2, n, om4, mode);
    if (!wait(pU, h->ev[11])) return SVDUP_ECUDA;
    mix_prepare(h, pU, u.E2, u.FL2, m, u.WLf, true, m);
    if (!wait(pU, h->ev[12])) return SVDUP_ECUDA;
    mix_xside(h, pU, u.E2, u.FL2, u.ML2, m, u.WLf, true, m, om2, false);
    if (!wait(pU, h->ev[1])) return SVDUP_ECUDA;
    mix_mma(h, pU, u.E2, u.FL2, u.ML2, m, om2, mode);
  } else {
    stage_begin(h, SVDUP_STAGE_SOLVE, h->stream);
    // STEPs 3, 6: first right solve; STEP 7: second right solve
    launch_fill_right(sR, u.E3, m, n, S, u.p, u.q, u.ab, u.z4p, u.E4.rhop, h->status);
    queue_solve(h, sR, u.E3);
    launch_apply_qt(sR, u.E3, u.z4p, u.ysortR, u.zsec4, mixed);
    if (!hand(h->ev[2], sR, pV)) return SVDUP_ECUDA;  // E3 ready: V's first product
    launch_fill_second(sR, u.E4, u.E3.lam, u.zsec4);
    queue_solve(h, sR, u.E4, mixed);
    launch_norms(sR, u.E4, nullptr, nullptr, mixed);
    if (multi && cudaEventRecord(h->ev[3], sR) != cudaSuccess) return SVDUP_ECUDA;  // E4 ready
    // STEPs 2, 4: first left solve; its transposed product gives the second left z
    launch_fill_left(sL, u.E1, m, S, u.p, u.q, u.ab, u.z2p, u.E2.rhop, h->status);
    queue_solve(h, sL, u.E1);
    launch_apply_qt(sL, u.E1, u.z2p, u.ysortL, u.zsec2, mixed);
    if (!hand(h->ev[0], sL, pU)) return SVDUP_ECUDA;  // E1 ready: U's first product
    // STEP 5: second left solve
    launch_fill_second(sL, u.E2, u.E1.lam, u.zsec2);
    queue_solve(h, sL, u.E2, mixed);
    launch_norms(sL, u.E2, nullptr, nullptr, mixed);
    stage_end(h, h->stream);
    // products: U -> W -> U (descending), V -> W -> V (descending; the signs follow)
    if (mixed) {
      queue_product_mixed(h, pU, u.E1, u.FL, u.ML, m, U, false, ldu, om1, mode);
      queue_product_mixed(h, pV, u.E3, u.FR, u.MR, n, V, false, ldv, om3, mode);
    } else {
      queue_product(h, pU, u.E1, u.FL, m, U, ldu, u.XsL, om1, mode);
      queue_product(h, pV, u.E3, u.FR, n, V, ldv, u.XsR, om3, mode);
    }
    // V's second product, after its first (stream order) and E4 (the event above)
    if (multi && cudaStreamWaitEvent(pV, h->ev[3], 0) != cudaSuccess) return SVDUP_ECUDA;
    if (mixed) queue_product_mixed(h, pV, u.E4, u.FR, u.MR, n, u.WRf, true, n, om4, mode);
    else queue_product(h, pV, u.E4, u.FR, n, u.WR, n, u.XsR, om4, mode);
    if (!hand(h->ev[1], sL, pU)) return SVDUP_ECUDA;  // E2 ready: U's second product
    if (mixed) queue_product_mixed(h, pU, u.E2, u.FL, u.ML, m, u.WLf, true, m, om2, mode);
    else queue_product(h, pU, u.E2, u.FL, m, u.WL, m, u.XsL, om2, mode);
  }
  // sign pairing of right vectors with left vectors (before S is overwritten); in the
  // mixed mode its sums run on FP32 pairs (only the signs are used)
  stage_begin(h, SVDUP_STAGE_SIGN, h->stream);
  launch_fill_ones(sL, m, u.ones);
  launch_apply_q(sL, u.E2, u.ones, u.work, u.g1, mixed);
  launch_apply_q(sL, u.E1, u.g1, u.work, u.g, mixed);
  launch_sign_combine(sL, m, n, S, u.p, u.q, u.g, u.yv);
  if (!hand(h->ev_mid, sL, sR)) return SVDUP_ECUDA;
  // (the stored norms of E3 and E4 stay: V's products read them, possibly meanwhile)
  launch_apply_qt(sR, u.E3, u.yv, u.ysortR, u.h1, mixed, true);
  launch_apply_qt(sR, u.E4, u.h1, u.ysortR, u.h, mixed, true);
  launch_sign_finish(sR, m, n, u.h, u.sign);
  stage_end(h, h->stream);
  // join before the signs are applied to V and before STEP 8 (it overwrites S, which
  // the right-hand fill and the signs read)
  if (!hand(h->ev[4], pU, st) || !hand(h->ev[5], pV, st) || !hand(h->ev_join, sR, st) ||
      !hand(h->ev[6], sL, st))
    return SVDUP_ECUDA;
  launch_sign_apply(st, m, n, V, ldv, u.sign);
  // STEP 8
  launch_sqrt_desc(st, m, u.E2.lam, S, h->status);
  if (refine) {  // the gated orthogonalising step, on Uhat, then on Vhat
    RefWs wu = refine_ws_carve(u.refbase, m, m);
    launch_refine(st, U, ldu, m, m, wu, h->refine_tol, h->status);
    cudaMemcpyAsync(h->ref_res, wu.res, sizeof(double), cudaMemcpyDeviceToDevice, st);
    RefWs wv = refine_ws_carve(u.refbase, n, n);
    launch_refine(st, V, ldv, n, n, wv, h->refine_tol, h->status);
    cudaMemcpyAsync(h->ref_res + 1, wv.res, sizeof(double), cudaMemcpyDeviceToDevice, st);
  }
  return check_launch();
}

int svdup_refine(svdup_t h, int rows, int cols, double* X, int ldx, double tol, double* residual) {
  if (!h || !X || cols < 1 || rows < cols || ldx < rows || !(tol == tol)) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  int rc = ensure_ws(h, refine_ws_bytes(rows, cols));
  if (rc) return rc;
  RefWs w = refine_ws_carve(h->ws, rows, cols);
  launch_refine(h->stream, X, ldx, rows, cols, w, tol, h->status);
  if (residual &&
      cudaMemcpyAsync(residual, w.res, sizeof(double), cudaMemcpyDeviceToDevice, h->stream) !=
          cudaSuccess)
    return SVDUP_ECUDA;
  return check_launch();
}

int svdup_check_timeout(svdup_t h, int rows, int N, const double* X, int ldx, const double* d,
                        const double* z, double rho, double* Y, int ldy, double* lam) {
  if (!h) return SVDUP_EINVAL;
  h->test_stall = 1;
  h->test_wait_ns = 1000000ull;  // 1 ms
  const int rc = svdup_cauchy_product(h, rows, N, X, ldx, d, z, rho, Y, ldy, lam, 1e-12,
                                      SVDUP_MIXED_BF16X3);
  h->test_stall = 0;
  h->test_wait_ns = 0;
  return rc;
}

int svdup_set_refine_tol(svdup_t h, double tol) {
  if (!h || !(tol == tol)) return SVDUP_EINVAL;
  h->refine_tol = tol;
  return SVDUP_OK;
}

int svdup_refine_residuals(svdup_t h, double* out2) {
  if (!h || !out2) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  if (cudaMemcpyAsync(out2, h->ref_res, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return SVDUP_ECUDA;
  return SVDUP_OK;
}

int svdup_update_host(svdup_t h, int m, int n, double* U, int ldu, double* S, double* V, int ldv,
                      const double* a, const double* b, double eps, int mode) {
  if (!h || !U || !S || !V || !a || !b) return SVDUP_EINVAL;
  if (m < 1 || n < m || ldu < m || ldv < n) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bu = (size_t)m * m * sizeof(double), bv = (size_t)n * n * sizeof(double);
  const size_t need = al(bu) + al(bv) + 2 * al(m * sizeof(double)) + al(n * sizeof(double));
  if (h->hb_size < need) {  // the device copies stay with the handle between calls
    cudaStreamSynchronize(h->stream);
    if (h->hb) cudaFree(h->hb);
    h->hb = nullptr;
    h->hb_size = 0;
    if (cudaMalloc(&h->hb, need) != cudaSuccess) {
      cudaGetLastError();
      h->hb = nullptr;
      return SVDUP_ENOMEM;
    }
    h->hb_size = need;
  }
  char* q = h->hb;
  double* dU = (double*)q; q += al(bu);
  double* dV = (double*)q; q += al(bv);
  double* dS = (double*)q; q += al(m * sizeof(double));
  double* da = (double*)q; q += al(m * sizeof(double));
  double* db = (double*)q;
  cudaStream_t st = h->stream;
  int rc = SVDUP_OK;
  if (cudaMemcpy2DAsync(dU, m * sizeof(double), U, (size_t)ldu * sizeof(double),
                        m * sizeof(double), m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dS, S, m * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpy2DAsync(dV, n * sizeof(double), V, (size_t)ldv * sizeof(double),
                        n * sizeof(double), n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(da, a, m * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(db, b, n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    rc = SVDUP_ECUDA;
  }
  if (!rc) rc = svdup_update(h, m, n, dU, m, dS, dV, n, da, db, eps, mode);
  if (!rc) {
    // U is final once its last product has run (ev[4] on its product stream, recorded
    // at the update's join; nothing after the join writes U unless the refinement
    // runs): its copy back then overlaps the right side's end and V's copy.  (Splitting
    // each matrix's copies over two streams per direction measured no faster: the
    // copies run at the host link's rate either way.)
    const bool early = h->side && h->timing != SVDUP_TIMING_STAGES && !(mode & SVDUP_REFINE);
    cudaStream_t su = early ? h->left : st;
    if (early && cudaStreamWaitEvent(su, h->ev[4], 0) != cudaSuccess) rc = SVDUP_ECUDA;
    if (!rc && (cudaMemcpy2DAsync(U, (size_t)ldu * sizeof(double), dU, m * sizeof(double),
                                  m * sizeof(double), m, cudaMemcpyDeviceToHost, su) != cudaSuccess ||
                cudaMemcpyAsync(S, dS, m * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpy2DAsync(V, (size_t)ldv * sizeof(double), dV, n * sizeof(double),
                                  n * sizeof(double), n, cudaMemcpyDeviceToHost, st) != cudaSuccess))
      rc = SVDUP_ECUDA;
    if (!rc && early &&
        (cudaEventRecord(h->ev_copy, su) != cudaSuccess || cudaStreamWaitEvent(st, h->ev_copy, 0) != cudaSuccess))
      rc = SVDUP_ECUDA;
  }
  if (!rc) rc = svdup_sync(h);
  cudaStreamSynchronize(st);
  return rc;
}

int svdup_rank_one_eig(svdup_t h, int N, const double* d, const double* z, double rho, int* k,
                       int* idx, double* dk, int* org, double* tau, double* zhat, double* inv_norm,
                       double* lam) {
  if (!h || N < 1 || !d || !z || !k || !idx || !dk || !org || !tau || !zhat || !inv_norm || !lam)
    return SVDUP_EINVAL;
  if (!(rho != 0.0) || !isfinite(rho)) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  Arena meas = {nullptr, 0};
  make_eig(meas, N);
  meas.take<double>(1);
  int rc = ensure_ws(h, meas.off);
  if (rc) return rc;
  Arena ar = {h->ws, 0};
  Eig e = make_eig(ar, N);
  e.vfmin = h->vf_min;
  e.vfmin_pairs = h->vf_min_pairs;
  double* rhod = ar.take<double>(1);
  cudaStream_t st = h->stream;
  if (cudaMemcpyAsync(rhod, &rho, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SVDUP_ECUDA;
  launch_fill_generic(st, e, d, z, rhod, h->status);
  queue_solve(h, st, e);
  launch_norms(st, e, nullptr, nullptr);
  cudaMemcpyAsync(k, e.kp, sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(idx, e.idx, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(dk, e.dk, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(org, e.org, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(tau, e.tau, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(zhat, e.zhat, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(inv_norm, e.inv, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(lam, e.lam, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  return check_launch();
}

int svdup_rank_one_apply(svdup_t h, int N, const double* d, const double* z, double rho,
                         const double* x, double* y, double* lam) {
  if (!h || N < 1 || !d || !z || !x || !y || !lam) return SVDUP_EINVAL;
  if (!(rho != 0.0) || !isfinite(rho)) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  Arena meas = {nullptr, 0};
  make_eig(meas, N);
  meas.take<double>(1);
  meas.take<double>(N);
  int rc = ensure_ws(h, meas.off);
  if (rc) return rc;
  Arena ar = {h->ws, 0};
  Eig e = make_eig(ar, N);
  e.vfmin = h->vf_min;
  e.vfmin_pairs = h->vf_min_pairs;
  double* rhod = ar.take<double>(1);
  double* work = ar.take<double>(N);
  cudaStream_t st = h->stream;
  if (cudaMemcpyAsync(rhod, &rho, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SVDUP_ECUDA;
  launch_fill_generic(st, e, d, z, rhod, h->status);
  queue_solve(h, st, e);
  launch_norms(st, e, nullptr, nullptr);
  launch_apply_q(st, e, x, work, y, false);
  cudaMemcpyAsync(lam, e.lam, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  return check_launch();
}

int svdup_secular(svdup_t h, int k, const double* d, const double* z, double rho, int* org,
                  double* tau) {
  if (!h || k < 1 || !d || !z || !org || !tau) return SVDUP_EINVAL;
  if (!(rho != 0.0) || !isfinite(rho)) return SVDUP_EINVAL;
  if (set_device(h)) return SVDUP_ECUDA;
  Arena meas = {nullptr, 0};
  make_eig(meas, k);
  int rc = ensure_ws(h, meas.off);
  if (rc) return rc;
  Arena ar = {h->ws, 0};
  Eig e = make_eig(ar, k);
  cudaStream_t st = h->stream;
  if (cudaMemcpyAsync(e.rhop, &rho, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SVDUP_ECUDA;
  launch_secular_direct(st, e, k, d, z, h->status, h->maxit);
  cudaMemcpyAsync(org, e.org, k * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(tau, e.tau, k * sizeof(double), cudaMemcpyDeviceToDevice, st);
  return check_launch();
}

int svdup_cauchy_product(svdup_t h, int rows, int N, const double* X, int ldx, const double* d,
                         const double* z, double rho, double* Y, int ldy, double* lam, double eps,
                         int mode) {
  if (!h || rows < 1 || N < 1 || !X || !d || !z || !Y || !lam) return SVDUP_EINVAL;
  if (ldx < rows || ldy < rows || !(eps > 0.0 && eps < 1.0)) return SVDUP_EINVAL;
  if (!(rho != 0.0) || !isfinite(rho)) return SVDUP_EINVAL;
  if (!mode_ok(mode)) return SVDUP_EINVAL;
  const bool mixed = is_mixed(mode);
  if (set_device(h)) return SVDUP_ECUDA;
  auto lay = [&](Arena& ar, Eig* e, double** Xw, double** Xs, FmmPlan* f, MixPlan* mp,
                 double** rhod) {
    *e = make_eig(ar, N);
    e->vfmin = h->vf_min;
    e->vfmin_pairs = h->vf_min_pairs;
    *rhod = ar.take<double>(1);
    *Xw = ar.take<double>((size_t)rows * N);
    *Xs = mixed ? nullptr : ar.take<double>((size_t)rows * N);
    *f = make_plan(ar, N, rows, eps, leaf_size(h, N, mode), mixed);
    if (mixed) {
      *mp = make_mix(ar, rows, *f);
      mp->fp16 = is_fp16(mode) ? 1 : 0;
    }
  };
  Eig e;
  double *Xw, *Xs, *rhod;
  FmmPlan f;
  MixPlan mp;
  memset(&mp, 0, sizeof(mp));
  Arena meas = {nullptr, 0};
  lay(meas, &e, &Xw, &Xs, &f, &mp, &rhod);
  int rc = ensure_ws(h, meas.off);
  if (rc) return rc;
  Arena ar = {h->ws, 0};
  lay(ar, &e, &Xw, &Xs, &f, &mp, &rhod);
  cudaStream_t st = h->stream;
  if (cudaMemcpyAsync(rhod, &rho, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SVDUP_ECUDA;
  if (cudaMemcpy2DAsync(Xw, (size_t)rows * sizeof(double), X, (size_t)ldx * sizeof(double),
                        (size_t)rows * sizeof(double), N, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return SVDUP_ECUDA;
  launch_fill_generic(st, e, d, z, rhod, h->status);
  queue_solve(h, st, e, mixed);
  launch_norms(st, e, nullptr, nullptr, mixed);
  OutMap om = {Y, (long long)ldy, N, 0};
  if (mixed) queue_product_mixed(h, st, e, f, mp, rows, Xw, false, rows, om, mode);
  else queue_product(h, st, e, f, rows, Xw, rows, Xs, om, mode);
  cudaMemcpyAsync(lam, e.lam, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  return check_launch();
}

int svdup_batch_create(svdup_t h, int count, const svdup_problem* probs, double eps, int mode,
                       int lanes, svdup_batch_t* out) {
  if (!out) return SVDUP_EINVAL;
  svdup_batch* b = nullptr;
  int rc = batch_plan(h, count, probs, eps, mode, lanes, &b);
  if (rc) return rc;
  // Record the batch into a graph: capture on the batch's own origin stream (the
  // handle's stream may be the legacy default stream, which cannot be captured).
  if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    return SVDUP_ECUDA;
  }
  t_recording = true;  // recorded, not launched: counted per graph launch
  rc = batch_queue(b);
  t_recording = false;
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(b->origin, &g);
  b->graph = g;
  if (rc == SVDUP_OK && ce != cudaSuccess) rc = SVDUP_ECUDA;
  if (rc == SVDUP_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) rc = SVDUP_ECUDA;
  b->kernels = 0;
  if (rc == SVDUP_OK) {
    size_t nn = 0;
    if (cudaGraphGetNodes(b->graph, nullptr, &nn) == cudaSuccess) {
      cudaGraphNode_t* nodes = (cudaGraphNode_t*)malloc(sizeof(cudaGraphNode_t) * (nn ? nn : 1));
      if (nodes && cudaGraphGetNodes(b->graph, nodes, &nn) == cudaSuccess)
        for (size_t i = 0; i < nn; i++) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
            b->kernels++;
        }
      free(nodes);
    }
  }
  if (rc) {
    cudaGetLastError();
    batch_free(b);
    return rc;
  }
  *out = b;
  return SVDUP_OK;
}

int svdup_batch_launch(svdup_batch_t b) {
  if (!b || !b->exec) return SVDUP_EINVAL;
  if (set_device(b->parent)) return SVDUP_ECUDA;
  if (cudaGraphLaunch(b->exec, b->parent->stream) != cudaSuccess) {
    cudaGetLastError();
    return SVDUP_ECUDA;
  }
  g_launch_count.fetch_add(b->kernels, std::memory_order_relaxed);
  return SVDUP_OK;
}

long long svdup_batch_kernels(svdup_batch_t b) { return b ? b->kernels : -1; }

int svdup_batch_destroy(svdup_batch_t b) {
  if (!b) return SVDUP_EINVAL;
  cudaSetDevice(b->parent->device);
  cudaStreamSynchronize(b->parent->stream);
  batch_free(b);
  return SVDUP_OK;
}

int svdup_update_batched(svdup_t h, int count, const svdup_problem* probs, double eps, int mode,
                         int lanes) {
  svdup_batch* b = nullptr;
  int rc = batch_plan(h, count, probs, eps, mode, lanes, &b);
  if (rc) return rc;
  // the handle's stream -> origin -> lanes -> origin -> the handle's stream
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(e0, h->stream) != cudaSuccess ||
      cudaStreamWaitEvent(b->origin, e0, 0) != cudaSuccess) {
    rc = SVDUP_ECUDA;
  }
  if (!rc) rc = batch_queue(b);
  if (!rc && (cudaEventRecord(e1, b->origin) != cudaSuccess ||
              cudaStreamWaitEvent(h->stream, e1, 0) != cudaSuccess))
    rc = SVDUP_ECUDA;
  int st = svdup_sync(h);
  if (!rc) rc = st;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  batch_free(b);
  cudaGetLastError();
  return rc;
}

int svdup_tuning_get(svdup_t h, int mode, int* dense_max, int* leaf128_min) {
  if (!h || !mode_ok(mode & SVDUP_MODE_MASK)) return SVDUP_EINVAL;
  const int i = mode_index(mode);
  if (dense_max) *dense_max = h->dense_max[i];
  if (leaf128_min) *leaf128_min = h->leaf128_min[i];
  return SVDUP_OK;
}

int svdup_tuning_set(svdup_t h, int mode, int dense_max, int leaf128_min) {
  if (!h || !mode_ok(mode & SVDUP_MODE_MASK) || dense_max < 0 || leaf128_min < 1) return SVDUP_EINVAL;
  const int i = mode_index(mode);
  h->dense_max[i] = dense_max;
  h->leaf128_min[i] = leaf128_min;
  return SVDUP_OK;
}

int svdup_autotune(svdup_t h, int mode, int nmax) {
  if (!h || !mode_ok(mode & SVDUP_MODE_MASK) || nmax < 256) return SVDUP_EINVAL;
  mode &= SVDUP_MODE_MASK;
  if (set_device(h)) return SVDUP_ECUDA;
  const int i = mode_index(mode);
  const int keep_dense = h->dense_max[i], keep_leaf = h->leaf128_min[i];
  const int keep_w = h->dense_w128_min[i];
  int nlim = 256;
  while (nlim * 2 <= nmax) nlim *= 2;
  const size_t maxN = (size_t)nlim;
  double *X = nullptr, *Y = nullptr, *d = nullptr, *z = nullptr, *lam = nullptr;
  int rc = SVDUP_OK;
  if (cudaMalloc(&X, maxN * maxN * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&Y, maxN * maxN * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d, maxN * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&z, maxN * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&lam, maxN * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rc = SVDUP_ENOMEM;
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (!rc && (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess))
    rc = SVDUP_ECUDA;
  int dense_max = 0, leaf128_min = 1 << 30, dense_w128_min = 1 << 30;
  bool dense_lost = false;
  // the mixed dense product has a second tile shape (128-column output tiles)
  const int ncand = is_mixed(mode) ? 4 : 3;
  for (int N = 256; !rc && N <= nlim; N *= 2) {
    launch_fill_random(h->stream, N, N, X, d, z, 0x5eedULL + (unsigned long long)N);
    // candidates: 0 dense (64-column tiles), 1 far field with 64-pole leaves, 2 with
    // 128-pole leaves, 3 dense with 128-column tiles (mixed modes)
    float best = 1e30f;
    int best_c = 0;
    float tc[4] = {0, 0, 0, 0};
    for (int c = 0; c < ncand && !rc; c++) {
      const bool dense = (c == 0 || c == 3);
      h->dense_max[i] = dense ? N : 0;
      h->leaf128_min[i] = (c == 2) ? 1 : (1 << 30);
      h->dense_w128_min[i] = (c == 3) ? 1 : (1 << 30);
      const int m = mode | (dense ? SVDUP_DENSE : 0);
      float best_t = 1e30f;
      for (int rep = 0; rep < 3 && !rc; rep++) {  // first run warms the workspace
        cudaEventRecord(t0, h->stream);
        rc = svdup_cauchy_product(h, N, N, X, N, d, z, 1.0, Y, N, lam, 1e-12, m);
        cudaEventRecord(t1, h->stream);
        if (!rc) rc = svdup_sync(h);
        float ms = 0.f;
        if (!rc && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess && rep > 0 && ms < best_t)
          best_t = ms;
      }
      tc[c] = best_t;
      if (best_t < best) { best = best_t; best_c = c; }
    }
    if (rc) break;
    if ((best_c == 0 || best_c == 3) && !dense_lost) dense_max = N;
    else dense_lost = true;
    if (tc[2] < tc[1] && N < leaf128_min) leaf128_min = N;
    if (ncand == 4 && tc[3] < tc[0] && N < dense_w128_min) dense_w128_min = N;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(X); cudaFree(Y); cudaFree(d); cudaFree(z); cudaFree(lam);
  if (rc) {
    h->dense_max[i] = keep_dense;
    h->leaf128_min[i] = keep_leaf;
    h->dense_w128_min[i] = keep_w;
    return rc;
  }
  h->dense_max[i] = dense_max;
  h->leaf128_min[i] = leaf128_min;
  h->dense_w128_min[i] = dense_w128_min;
  return SVDUP_OK;
}

int svdup_tuning_get_tile(svdup_t h, int mode, int* dense_tile128_min) {
  if (!h || !mode_ok(mode & SVDUP_MODE_MASK) || !dense_tile128_min) return SVDUP_EINVAL;
  *dense_tile128_min = h->dense_w128_min[mode_index(mode)];
  return SVDUP_OK;
}

int svdup_tuning_set_tile(svdup_t h, int mode, int dense_tile128_min) {
  if (!h || !mode_ok(mode & SVDUP_MODE_MASK) || dense_tile128_min < 1) return SVDUP_EINVAL;
  h->dense_w128_min[mode_index(mode)] = dense_tile128_min;
  return SVDUP_OK;
}

int svdup_set_far_sums(svdup_t h, int kmin, int kmin_pairs) {
  if (!h || kmin < 1 || kmin_pairs < 1) return SVDUP_EINVAL;
  h->vf_min = kmin < kVfMinK ? kVfMinK : kmin;
  h->vf_min_pairs = kmin_pairs < kVfMinK ? kVfMinK : kmin_pairs;
  return SVDUP_OK;
}

int svdup_update_workspace(svdup_t h, int m, int n, double eps, int mode, size_t* bytes) {
  if (!h || !bytes || m < 1 || n < m || !(eps > 0.0 && eps < 1.0) || !mode_ok(mode))
    return SVDUP_EINVAL;
  *bytes = update_ws_bytes(h, m, n, eps, mode);
  return SVDUP_OK;
}

}  // extern "C"
