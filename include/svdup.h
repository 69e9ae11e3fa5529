/*
 * svdup.h -- C ABI of the GB300 rank-one SVD update library (libsvdup.so).
 *
 * Operation (Gandhi & Rajgor, "Updating Singular Value Decomposition for Rank One
 * Matrix Perturbation", Sec. 6, Alg. 6.1): given the SVD A = U diag(S) V^T of an
 * m x n matrix (m <= n, Sec. 3) and vectors a (m), b (n), compute the SVD
 * Ahat = A + a b^T = Uhat diag(Shat) Vhat^T.  The update is carried out as the
 * paper's four symmetric rank-one eigen-updates (App. A, Alg. 6.1 STEPs 2-7):
 * secular-equation roots (Sec. 3.1), Cauchy-like eigenvector matrices with
 * normalised columns (Sec. 3.2, Eq. CTildeFinalForm1), and the products U*Ctilde,
 * V*Ctilde evaluated by a Chebyshev far-field/near-field (FMM) decomposition of
 * the Cauchy matrix (Sec. 5, App. D).
 *
 * Conventions for every entry point:
 *  - Matrices are column-major IEEE double; ld* is the leading dimension.
 *  - Device pointers must be on the handle's device; they stay owned by the
 *    caller.  The library owns only its workspace (allocated lazily and kept by
 *    the handle until svdup_destroy).
 *  - Work is queued on the handle's CUDA stream and returns without waiting.
 *    Argument errors are returned immediately and nothing is queued.  Errors
 *    found on the device (no convergence, non-finite data) are latched in a
 *    status word and returned by the next svdup_sync.
 *  - No C++ exception crosses this interface.  All functions are thread-compatible:
 *    one handle must not be used from two host threads at once.
 */
#ifndef SVDUP_H
#define SVDUP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define SVDUP_OK 0
#define SVDUP_EINVAL 1     /* bad argument (NULL, m > n, ld < rows, eps not in (0,1), ...) */
#define SVDUP_ENOMEM 2     /* workspace allocation failed */
#define SVDUP_ENOCONV 3    /* a secular root hit the iteration cap (Sec. 3.1) */
#define SVDUP_ENONFINITE 4 /* NaN or Inf in the inputs or an intermediate */
#define SVDUP_ECUDA 5      /* a CUDA runtime call failed */
#define SVDUP_EORDER 6     /* S is not in descending order */
#define SVDUP_ETIMEOUT 7   /* a device-side wait gave up after its time limit (about 1 s) */

/* ---- update modes (svdup_update's mode argument) -------------------------- */
#define SVDUP_FP64 0          /* every step in FP64 */
#define SVDUP_MIXED_BF16X3 1  /* products in 3-term BF16 split, FP32 accumulation */
#define SVDUP_MIXED_FP16X2 2  /* products in 2-term FP16 split, one power-of-two scale per
                                 tile, FP32 accumulation (about 2^-22 per operand) */
#define SVDUP_MODE_MASK 0xff
#define SVDUP_DENSE 0x100     /* flag: force the dense Cauchy product (no far field) */
#define SVDUP_REFINE 0x200    /* flag: after the update, one gated orthogonalising step on
                                 Uhat and on Vhat (svdup_refine, at the handle's tolerance) */

typedef struct svdup_ctx* svdup_t;

/* Create a handle bound to CUDA device `device` and stream `stream`
 * (a cudaStream_t; NULL selects the legacy default stream).  `flags` is
 * reserved (pass 0).  Returns SVDUP_OK and stores the handle in *h. */
int svdup_create(svdup_t* h, int device, void* stream, unsigned flags);

/* Release the handle's workspace (waits for its stream first). */
int svdup_destroy(svdup_t h);

/* Wait for the handle's stream; return and clear the first device error latched
 * since the previous svdup_sync (SVDUP_OK if none). */
int svdup_sync(svdup_t h);

/* Text of a return code (static storage). */
const char* svdup_error_string(int code);

/* Number of kernels this library has launched in this process, over all handles,
 * servers and threads (a launch counter, for accounting; take differences).  A batch
 * graph's kernels count once per svdup_batch_launch.  h is not used. */
long long svdup_launch_count(svdup_t h);

/* ---- stage timers ------------------------------------------------------ */
/* Stages timed by CUDA events on the handle's stream while timing is enabled: */
#define SVDUP_STAGE_GEMV 0    /* p = U^T a, q = V^T b */
#define SVDUP_STAGE_SOLVE 1   /* deflation, secular roots, zhat, norms (4 solves) */
#define SVDUP_STAGE_SIGN 2    /* sign pairing probe (Cauchy matrix-vector products) */
#define SVDUP_STAGE_GATHER 3  /* rotations and column gather before each product */
#define SVDUP_STAGE_SETUP 4   /* far-field operators (boxes, near ranges, S, T, L) */
#define SVDUP_STAGE_P2M 5     /* far-field expansions Phi = X S */
#define SVDUP_STAGE_M2L 6     /* translations Psi = Phi T */
#define SVDUP_STAGE_OUT 7     /* L2P + near field (or the dense product) */
#define SVDUP_NSTAGE 8

/* Timer modes (svdup_timing's enable argument):
 *  SVDUP_TIMING_STAGES   every stage above is timed; the update then runs all its work
 *                        on the handle's stream, in dependency order, so that the stage
 *                        intervals do not overlap.
 *  SVDUP_TIMING_KERNELS  only the three product-stage kernels (P2M, M2L, OUT) are timed,
 *                        each by an event pair on the stream it is launched on; the
 *                        update keeps its multi-stream schedule, so the times are those
 *                        of the kernels as they run beside the solves. */
#define SVDUP_TIMING_STAGES 1
#define SVDUP_TIMING_KERNELS 2

/* Set the timer mode (0 disables); setting it clears the totals.  Timing adds two
 * event records per timed interval and one small counting kernel per product, and
 * does not change results.  Any other value returns SVDUP_EINVAL. */
int svdup_timing(svdup_t h, int enable);

/* Wait for the stream and return, per stage, the summed device time in ms, the
 * number of timed intervals, the useful floating-point operations of the product
 * stages (2 per multiply-add of the stage's contraction; 0 for the other stages) and
 * the tensor-core flops the mixed modes executed (2 per multiply-add of every split
 * partial product, padding included; 0 in FP64 mode) since timing was enabled.
 * Arrays hold nstage entries (nstage <= SVDUP_NSTAGE); any of them may be NULL. */
int svdup_timing_read(svdup_t h, double* ms, long long* count, double* flops, double* mma_flops,
                      int nstage);

/* The algorithmic flops of the product stages since timing was enabled: App. D's
 * operation count of the FMM, 14 N p multiply-adds per right-hand side for N points
 * at expansion order p (leaves of 2p points), split as STEPs 5-6 (2 N p) to P2M,
 * STEPs 7-8 (5 N p) to M2L and STEPs 9-10 (7 N p) to OUT, with 2 flops per
 * multiply-add and N the non-deflated size of each product; 2 rows N^2 for the dense
 * product (in OUT).  Stages other than the three product stages read 0.  This is the
 * method's own work, not what the kernels execute (svdup_timing_read). */
int svdup_timing_read_alg(svdup_t h, double* alg_flops, int nstage);

/*
 * The full rank-one SVD update, Alg. 6.1 STEPs 1-8, in place (device pointers):
 *   U  m x m (ldu >= m), in: U, out: Uhat, columns ordered as Shat.
 *   S  m,               in: singular values in descending order (ties allowed),
 *                       out: Shat, descending.  (STEP 8: Shat = sqrt(D_n), a
 *                       negative rounding residue clamped to 0.)
 *   V  n x n (ldv >= n), in: V, out: Vhat; Vhat[:, :m] pairs with Uhat and Shat,
 *                       Vhat[:, m:] is an orthonormal basis of the null space.
 *   a  m, b n           the rank-one term a b^T (read only).
 *   eps                 target accuracy of the Cauchy products, 0 < eps < 1.  In FP64
 *                       mode the expansion order p is chosen so that the far field's
 *                       error for the closest admissible leaf pair (a gap of one leaf
 *                       radius), 4 (2 + sqrt 3)^-p of that pair's largest kernel entry,
 *                       is at most eps: p = ceil(log(4/eps) / log(2 + sqrt 3)), 23 at
 *                       eps = 1e-12, clamped to [4, 32].  (App. D STEP 1's
 *                       p = log5(1/eps) is the rate of the paper's interaction lists,
 *                       whose leaves are two radii apart.)  The mixed modes use p = 16.
 *   mode                SVDUP_FP64, SVDUP_MIXED_BF16X3 or SVDUP_MIXED_FP16X2, optionally
 *                       | SVDUP_DENSE;
 *                       any other value returns SVDUP_EINVAL.
 * The signs of Vhat's columns are chosen so that u_j^T Ahat v_j >= 0.
 * Requires 1 <= m <= n.  U, V are assumed orthogonal (as the paper does, App. A).
 * Sizes: element offsets are 64-bit and the workspace grows with m and n
 * (svdup_update_workspace reports it); parity with the FP64 oracle has been shown up
 * to m = n = 8192 and 2048 x 4096.
 */
int svdup_update(svdup_t h, int m, int n, double* U, int ldu, double* S, double* V, int ldv,
                 const double* a, const double* b, double eps, int mode);

/*
 * Orthogonalising refinement (no counterpart in the paper: a correction of the
 * orthogonality that split-precision products lose).  One Newton-Schulz step toward the
 * nearest matrix with orthonormal columns,
 *   X <- X (3 I - X^T X) / 2 = X - X E / 2,   E = X^T X - I,
 * in place on X (device, rows x cols column-major, ldx >= rows, rows >= cols >= 1), on
 * the tensor cores: E in the 3-term BF16 split with FP32 accumulation per 64-term tile
 * and double-float sums across tiles (about 2^-24 per term), X E in one BF16 product
 * (about 2^-8 of |E|).  The step is gated on the device: a probe residual
 * r = max_q ||X^T X w_q - w_q|| / ||w_q|| over four fixed +-1 vectors (FP64, two passes
 * over X) is measured first, and the step runs only if r > tol (tol <= 0: always).
 * After the step, r falls to about max(r^2, the split's own floor of a few 1e-8..1e-7).
 * residual: optional device double that receives r (measured before the step).
 * Queued on the handle's stream; scratch from the handle's workspace (about
 * 3 x 6 x rows x cols bytes of split tiles).
 */
int svdup_refine(svdup_t h, int rows, int cols, double* X, int ldx, double tol, double* residual);

/* The gate tolerance of SVDUP_REFINE updates (default 1e-6; <= 0 refines always). */
int svdup_set_refine_tol(svdup_t h, double tol);

/* Wait for the stream; out2[0], out2[1] = the probe residuals of Uhat and Vhat that the
 * last SVDUP_REFINE update measured before its steps. */
int svdup_refine_residuals(svdup_t h, double* out2);

/*
 * The same update with HOST buffers (end-to-end form): the inputs are copied to
 * the device on the handle's stream, the update runs, the results are copied back,
 * and the call waits for completion.  Returns the first error of the whole call.
 * Host buffers should be pinned for full copy bandwidth (any host memory works).
 * The device copies (8 (m^2 + n^2 + 2m + n) bytes) stay allocated on the handle
 * between calls, grown when a larger problem comes, and are freed by svdup_destroy;
 * U's copy back starts as soon as U is final, beside the rest of the update.
 */
int svdup_update_host(svdup_t h, int m, int n, double* U, int ldu, double* S, double* V, int ldv,
                      const double* a, const double* b, double eps, int mode);

/*
 * One symmetric rank-one eigen-update in compact form (RankOneUpdate STEPs 2-5,
 * Sec. 6.2; deflation Sec. 3.1; Cauchy-like vectors Sec. 3.2), device pointers:
 *   in:  N, d (N poles, any order), z (N), rho != 0.
 *   out: k (1 int)               number of non-deflated poles,
 *        idx (N ints)            their positions in the ascending order of d (first k),
 *        dk (N)                  their poles after deflation rotations (first k),
 *        org (N ints), tau (N)   root j = dk[org[j]] + tau[j], ascending (first k),
 *        zhat (N)                z recomputed from the roots (first k),
 *        inv_norm (N)            1/||c_j|| of the Cauchy columns (first k),
 *        lam (N)                 all N eigenvalues, ascending.
 * Deflation: |rho| ||z|| |z_i| <= tol removes pole i; two poles whose rotated
 * coupling |(d_j - d_i) c s| <= tol merge by a Givens rotation; tol = 8 u max(max|d|,
 * |rho| ||z||^2), u = 2^-53.
 */
int svdup_rank_one_eig(svdup_t h, int N, const double* d, const double* z, double rho, int* k,
                       int* idx, double* dk, int* org, double* tau, double* zhat, double* inv_norm,
                       double* lam);

/*
 * y = Q x for the eigenvectors Q of diag(d) + rho z z^T (RankOneUpdate STEP 7's product
 * with one vector, as the sign pairing applies it), device pointers:
 *   in:  N, d (N poles, any order), z (N), rho != 0, x (N; entry q multiplies the
 *        eigenvector of the q-th smallest eigenvalue);
 *   out: y (N, in the order of d), lam (N eigenvalues, ascending).
 * The same solve and deflation as svdup_rank_one_eig, the sums in FP64 (far-field form
 * from the handle's svdup_set_far_sums threshold).
 */
int svdup_rank_one_apply(svdup_t h, int N, const double* d, const double* z, double rho,
                         const double* x, double* y, double* lam);

/*
 * Secular roots alone (Sec. 3.1, Eq. GolubEigenvalUpdate), device pointers:
 * d (k, strictly ascending), z (k, nonzero), rho != 0 -> org (k ints), tau (k) with
 * root j = d[org[j]] + tau[j], ascending; org[j] is the pole nearer to root j.
 */
int svdup_secular(svdup_t h, int k, const double* d, const double* z, double rho, int* org,
                  double* tau);

/*
 * Secular roots with no device allocation (the paper has no counterpart: this is an
 * interface variant of svdup_secular).  For callers that cannot allocate device
 * memory -- a host application whose memory pool already holds the device memory it
 * may use, a plug-in that must not call the CUDA allocator, a latency-critical loop in
 * which cudaMalloc/cudaFree would synchronise the device -- and so cannot create a
 * handle.  Same operation and output as svdup_secular: device pointers d (k, strictly
 * ascending), z (k, nonzero), rho != 0 -> org (k ints), tau (k), root j =
 * d[org[j]] + tau[j], ascending.
 *   stream  a cudaStream_t of the calling thread's current device (NULL: the legacy
 *           default stream); the work is queued there and the call returns without
 *           waiting.
 *   info    device int owned by the caller: set to 0, then to the first device error
 *           (SVDUP_ENOCONV, SVDUP_ENONFINITE) once the stream reaches that point.
 * Scratch lives in one fixed array in the library's device memory, about
 * 48 * SVDUP_SECULAR_STATIC_MAX_K bytes, held by every GPU that loads the library until
 * the process exits; k > SVDUP_SECULAR_STATIC_MAX_K returns SVDUP_EINVAL.  Nothing is
 * allocated or freed.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it.  Every call on a device uses the same array:
 * calls whose work overlaps on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.
 */
#define SVDUP_SECULAR_STATIC_MAX_K 16384
int svdup_secular_static(void* stream, int k, const double* d, const double* z, double rho,
                         int* org, double* tau, int* info);

/*
 * Cauchy product Y = X * Ctilde for the eigen-system of diag(d) + rho z z^T
 * (RankOneUpdate STEPs 3-7, Sec. 6.2; Eq. UCTildeProduct), device pointers:
 *   X rows x N (ldx), columns in the order of d; Y rows x N (ldy), column q is the
 *   eigenvector of the q-th smallest eigenvalue (lam, N, ascending, also returned).
 *   eps and mode as in svdup_update.
 */
int svdup_cauchy_product(svdup_t h, int rows, int N, const double* X, int ldx, const double* d,
                         const double* z, double rho, double* Y, int ldy, double* lam, double eps,
                         int mode);

/*
 * Diagnostic (no counterpart in the paper): the library's own FP64 reciprocal and
 * reciprocal square root, which its FP64 kernels use in place of division and sqrt
 * (Newton-Raphson from an FP32 seed of the significand, exponent set by bit fields;
 * zeros, subnormals, the largest binades, infinities and NaNs fall back to CUDA's
 * division and sqrt).  Device arrays of n doubles: rcp[i] = 1/x[i], rsqrt[i] =
 * 1/sqrt(x[i]) (either output may be NULL); queued on `stream` (a cudaStream_t, NULL:
 * the legacy default stream).
 */
int svdup_check_rcp(void* stream, int n, const double* x, double* rcp, double* rsqrt);

/*
 * Failure test of the tensor-core pipeline (no counterpart in the paper).  Queues the
 * mixed (SVDUP_MIXED_BF16X3) Cauchy product of svdup_cauchy_product, same arguments,
 * with two test settings for that call only: the drains never hand a tensor-memory
 * region back to the MMA issuer, and every pipeline wait gives up after 1 ms instead of
 * one second.  The MMA issuer's wait therefore runs out; each CTA waits for the MMAs and
 * bulk copies it issued, frees its tensor memory and exits, and SVDUP_ETIMEOUT is
 * latched: the next svdup_sync returns it, Y holds no result, and the handle and the
 * CUDA context stay usable.  Returns the argument and launch status like
 * svdup_cauchy_product.
 */
int svdup_check_timeout(svdup_t h, int rows, int N, const double* X, int ldx, const double* d,
                        const double* z, double rho, double* Y, int ldy, double* lam);

/* ---- batches of independent updates ------------------------------------- */
/* One problem of a batch: the arguments of svdup_update (device pointers). */
typedef struct svdup_problem {
  int m, n;
  double* U;
  int ldu;
  double* S;
  double* V;
  int ldv;
  const double* a;
  const double* b;
} svdup_problem;

typedef struct svdup_batch* svdup_batch_t;

/*
 * Plan a batch of independent updates (no counterpart in the paper: a way to run
 * many Alg. 6.1 updates at once).  The problems are spread over `lanes` streams
 * forked from the handle's stream (largest first, each to the least-loaded lane);
 * every lane gets its own workspace, sized here for its largest problem, and shares
 * the handle's status word.  The whole batch is recorded once into a CUDA graph, so a
 * launch is a single graph launch on the handle's stream.  The graph is bound to the
 * given pointers and sizes: launching it again updates the same buffers in place
 * (chained updates).  lanes: 1..64 (0 picks 16).  The problem array is copied.
 */
int svdup_batch_create(svdup_t h, int count, const svdup_problem* probs, double eps, int mode,
                       int lanes, svdup_batch_t* out);
/* Queue the planned batch on the handle's stream (asynchronous; svdup_sync on the
 * handle waits and returns the first device error of any problem). */
int svdup_batch_launch(svdup_batch_t b);
/* Number of kernel launches one svdup_batch_launch replays (graph nodes). */
long long svdup_batch_kernels(svdup_batch_t b);
int svdup_batch_destroy(svdup_batch_t b);
/* The same batch without a graph: plans, queues, waits, releases.  Returns the first
 * error of the whole call. */
int svdup_update_batched(svdup_t h, int count, const svdup_problem* probs, double eps, int mode,
                         int lanes);

/*
 * Autotuning of the product path for `mode` (no counterpart in the paper).  For
 * N = 256, 512, ... up to nmax it times the Cauchy product (rows = N, synthetic poles
 * and vectors generated on the device) with the dense tile product, the far field with
 * leaves of 64 poles, with leaves of 128, and (mixed modes) the dense product with
 * 128-column instead of 64-column output tiles on the tensor cores, and keeps on the
 * handle the largest N at which a dense product was fastest (dense_max), the smallest N
 * at which leaves of 128 beat 64 (leaf128_min) and the smallest N at which the dense
 * product's 128-column tiles beat 64 (dense_tile128_min).  svdup_tuning_get /
 * svdup_tuning_set and svdup_tuning_get_tile / svdup_tuning_set_tile read and restore
 * these numbers (to cache them between processes).
 */
int svdup_autotune(svdup_t h, int mode, int nmax);
int svdup_tuning_get(svdup_t h, int mode, int* dense_max, int* leaf128_min);
int svdup_tuning_set(svdup_t h, int mode, int dense_max, int leaf128_min);
int svdup_tuning_get_tile(svdup_t h, int mode, int* dense_tile128_min);
int svdup_tuning_set_tile(svdup_t h, int mode, int dense_tile128_min);

/*
 * Far-field form of the solve's own sums (Sec. 3.2's Loewner zhat and the column norms
 * ||c_j|| with Q^T y, RankOneUpdate STEP 7; summed through App. D's interpolation FMM
 * instead of directly, O(k p) instead of O(k^2) work), for the eigen-problems of this
 * handle whose non-deflated size k is at least
 *   kmin        where the direct sums run in FP64 (SVDUP_FP64, and the first solves of
 *               the mixed modes, whose zhat forms the second solves' z): default 4096;
 *   kmin_pairs  where they run in FP32 pairs (the second solves and the norms of the
 *               mixed modes): default 12288.
 * The defaults are the measured crossovers on GB300 (FP64 costs as much as about 60
 * FP32 operations there, so the pair sums stay ahead up to larger k).  Values below 2048
 * are raised to 2048; INT_MAX keeps the direct sums.  The far-field form agrees with the
 * FP64 direct sums to about 1e-15 relative.
 */
int svdup_set_far_sums(svdup_t h, int kmin, int kmin_pairs);

/* Bytes of workspace svdup_update needs on this handle for an m x n problem in `mode`
 * (the handle keeps the largest such workspace it has needed). */
int svdup_update_workspace(svdup_t h, int m, int n, double eps, int mode, size_t* bytes);

/* ---- serving: resident SVDs and a continuous stream of updates ------------- */
/*
 * A serving engine on one device (no counterpart in the paper, whose motivation in
 * Sec. 1 is streaming data).  Callers register SVDs that stay resident in their own
 * device buffers and then submit rank-one updates of them at any time.  One scheduler
 * thread admits requests continuously: the oldest pending request whose matrix has no
 * update in flight goes to a free lane (a stream with its own workspace) as soon as one
 * is free and the free-HBM ledger (the workspace bytes held by the lanes, capped by
 * hbm_budget) has room for it.  It opens a group: later pending requests of the same
 * size class (n in the same power-of-two range) whose matrices are idle join it, up to
 * the group size (svdup_server_set_group, default 4), and the lane queues the group's
 * updates back to back on its stream.  Updates of different matrices run concurrently
 * on the device; updates of one matrix apply in submission order.  Latency is measured
 * on the host from submission to the moment the result is posted, when the request's
 * whole group has completed.
 *   lanes       1..64 concurrent updates (0 picks 8)
 *   hbm_budget  bytes of workspace the engine may hold at once (0: 3/4 of free memory)
 */
typedef struct svdup_server* svdup_server_t;
int svdup_server_create(int device, int lanes, size_t hbm_budget, double eps, int mode,
                        svdup_server_t* out);
/* Register a resident SVD (device pointers, as in svdup_update; the caller keeps them
 * alive and leaves them alone while the engine runs).  *id receives its handle. */
int svdup_server_register(svdup_server_t s, int m, int n, double* U, int ldu, double* S,
                          double* V, int ldv, int* id);
/* Submit an update of matrix id with HOST vectors a (m) and b (n), copied before the
 * call returns.  *ticket identifies the request.  Never blocks on the device. */
int svdup_server_submit(svdup_server_t s, int id, const double* a, const double* b,
                        long long* ticket);
/* Wait for a request; returns its status (SVDUP_OK or the device error of its update)
 * and its latency in ms (may be NULL).  timeout_ms < 0 waits without limit; a request
 * still running at the limit returns SVDUP_ETIMEOUT. */
int svdup_server_wait(svdup_server_t s, long long ticket, double timeout_ms, double* latency_ms);
/* Wait for every submitted request. */
int svdup_server_drain(svdup_server_t s);
/* Totals since create: completed updates, latency percentiles (ms), the largest number
 * of updates in flight at once, and the largest workspace bytes held at once. */
int svdup_server_stats(svdup_server_t s, long long* completed, double* p50_ms, double* p99_ms,
                       int* max_in_flight, size_t* max_ws_bytes);
/* Requests a lane takes per cycle, 1..16 (1: one update per lane cycle). */
int svdup_server_set_group(svdup_server_t s, int group_max);
/* Lane cycles launched, the requests in them, and the largest group so far. */
int svdup_server_group_stats(svdup_server_t s, long long* groups, long long* grouped,
                             int* max_group);
/* Stop the scheduler (after draining) and release everything the engine allocated. */
int svdup_server_destroy(svdup_server_t s);

#ifdef __cplusplus
}
#endif
#endif /* SVDUP_H */
