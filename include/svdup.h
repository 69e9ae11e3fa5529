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
#define SVDUP_MIXED_FP16X2 2  /* products in 2-term scaled FP16 split, FP32 accumulation */
#define SVDUP_MODE_MASK 0xff
#define SVDUP_DENSE 0x100     /* flag: force the dense Cauchy product (no far field) */
#define SVDUP_REFINE 0x200    /* flag (mixed modes): one orthogonalising refinement step */

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

/* Number of distinct kernels this library launched on the handle's stream since
 * create (a launch counter, for accounting). */
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

/* Enable (1) or disable (0) the stage timers; enabling clears the totals.  Timing
 * adds two event records per stage and does not change results. */
int svdup_timing(svdup_t h, int enable);

/* Wait for the stream and return, per stage, the summed device time in ms, the
 * number of timed intervals, the useful floating-point operations of the product
 * stages (2 per multiply-add of the stage's contraction; 0 for the other stages) and
 * the tensor-core flops the mixed modes executed (2 per multiply-add of every split
 * partial product, padding included; 0 in FP64 mode) since timing was enabled.
 * Arrays hold nstage entries (nstage <= SVDUP_NSTAGE); any of them may be NULL. */
int svdup_timing_read(svdup_t h, double* ms, long long* count, double* flops, double* mma_flops,
                      int nstage);

/*
 * The full rank-one SVD update, Alg. 6.1 STEPs 1-8, in place (device pointers):
 *   U  m x m (ldu >= m), in: U, out: Uhat, columns ordered as Shat.
 *   S  m,               in: singular values in descending order (ties allowed),
 *                       out: Shat, descending.  (STEP 8: Shat = sqrt(D_n), a
 *                       negative rounding residue clamped to 0.)
 *   V  n x n (ldv >= n), in: V, out: Vhat; Vhat[:, :m] pairs with Uhat and Shat,
 *                       Vhat[:, m:] is an orthonormal basis of the null space.
 *   a  m, b n           the rank-one term a b^T (read only).
 *   eps                 accuracy of the Cauchy products, 0 < eps < 1; the
 *                       expansion order is p = ceil(log5(1/eps)) (App. D STEP 1).
 *   mode                SVDUP_FP64 / SVDUP_MIXED_* plus optional flags.
 * The signs of Vhat's columns are chosen so that u_j^T Ahat v_j >= 0.
 * Requires 1 <= m <= n.  U, V are assumed orthogonal (as the paper does, App. A).
 */
int svdup_update(svdup_t h, int m, int n, double* U, int ldu, double* S, double* V, int ldv,
                 const double* a, const double* b, double eps, int mode);

/*
 * The same update with HOST buffers (end-to-end form): the inputs are copied to
 * the device on the handle's stream, the update runs, the results are copied back,
 * and the call waits for completion.  Returns the first error of the whole call.
 * Host buffers should be pinned for full copy bandwidth (any host memory works).
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

#ifdef __cplusplus
}
#endif
#endif /* SVDUP_H */
