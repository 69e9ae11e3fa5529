/*
 * svdup_oracle.c -- plain, slow FP64 CPU oracle for the rank-one SVD update of
 * Gandhi & Rajgor, "Updating Singular Value Decomposition for Rank One Matrix
 * Perturbation" (arXiv 1707.08369).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py load this library.  It shares no code, header,
 * table or constant generator with the CUDA library, and it never calls it.
 *
 * What each part follows:
 *   oracle_schur2          Alg. 6.1 STEP 2/3 and App. A: Q diag(r1,r2) Q^T of [[g,1],[1,0]].
 *   oracle_gemv_t          RankOneUpdate STEP 1 (Sec. 6.2): abar = U^T a1.
 *   oracle_secular_roots   Sec. 3.1: zeros of w(mu) = 1 + rho sum z_i^2/(d_i - mu),
 *                          by plain bisection in each interlacing bracket.
 *   deflation              Sec. 3.1, deflation cases (1) (a zero/negligible z_i) and
 *                          (3) (repeated eigenvalues), in the Bunch-Nielsen-Sorensen
 *                          manner: a Givens rotation moves the z weight of one of two
 *                          (numerically) equal poles onto the other.
 *   eigenvectors           Sec. 3.2, normalised Cauchy-like form: column j is
 *                          (z_i / (d_i - mu_j))_i / ||.||.  z is recomputed from the
 *                          computed roots by the characteristic-polynomial identity
 *                          (Loewner) so that the columns are the exact eigenvectors of
 *                          the problem whose exact eigenvalues are the computed roots.
 *   oracle_rank_one_apply  Q X for a thin X: the products of Alg. 6.1 STEPs 5 and 7 on
 *                          a few sampled vectors (full-size checks column by column).
 *   oracle_rank_one_update RankOneUpdate STEPs 1-7 with the dense product X*Q in place
 *                          of the FMM of STEP 6 (the dense product is the quantity the
 *                          FMM approximates).
 *   oracle_svd_update      Alg. 6.1 STEPs 1-8, then columns in descending order and the
 *                          sign of each right vector chosen so that u_j^T Ahat v_j >= 0.
 *   oracle_jacobi_svd      independent check: one-sided Jacobi (Hestenes) SVD.
 *
 * Every floating-point quantity is IEEE double.  Matrices are column-major.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENOCONV 3

/* unit roundoff of IEEE double */
#define ORC_U (ldexp(1.0, -53))

/* ------------------------------------------------------------------------- */
/* Alg. 6.1 STEP 2/3 (App. A): [[g,1],[1,0]] = Q diag(r1, r2) Q^T.             */
/* out = {r1, r2, Q00, Q10, Q01, Q11}; r1 >= r2, column k of Q is (r_k,1)/norm. */
/* r1*r2 = -1 (the determinant), so the smaller-magnitude root is taken as     */
/* -1/(larger) to avoid cancellation.                                          */
/* ------------------------------------------------------------------------- */
void oracle_schur2(double g, double* out)
{
    double s = sqrt(g * g + 4.0);
    double r1, r2;
    if (g >= 0.0) { r1 = 0.5 * (g + s); r2 = -1.0 / r1; }
    else          { r2 = 0.5 * (g - s); r1 = -1.0 / r2; }
    double n1 = sqrt(r1 * r1 + 1.0), n2 = sqrt(r2 * r2 + 1.0);
    out[0] = r1;      out[1] = r2;
    out[2] = r1 / n1; out[3] = 1.0 / n1;   /* first column  */
    out[4] = r2 / n2; out[5] = 1.0 / n2;   /* second column */
}

/* y = A^T x for A rows x cols (column-major, leading dimension lda). */
void oracle_gemv_t(int rows, int cols, const double* A, int lda, const double* x, double* y)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < cols; j++) {
        const double* col = A + (size_t)j * lda;
        double s = 0.0;
        for (int r = 0; r < rows; r++) s += col[r] * x[r];
        y[j] = s;
    }
}

/* y = A x for A rows x cols. */
static void gemv_n(int rows, int cols, const double* A, int lda, const double* x, double* y)
{
    for (int r = 0; r < rows; r++) y[r] = 0.0;
    for (int j = 0; j < cols; j++) {
        const double* col = A + (size_t)j * lda;
        double xj = x[j];
        for (int r = 0; r < rows; r++) y[r] += col[r] * xj;
    }
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.1: the secular function at mu = d[org] + tau.                        */
/* Each difference d_i - mu is formed as (d_i - d[org]) - tau so that a root  */
/* that sits very close to its pole keeps full relative accuracy.             */
/* ------------------------------------------------------------------------- */
static double secular_w(int k, const double* d, const double* z, double rho, int org, double tau)
{
    double s = 0.0;
    double dorg = d[org];
    for (int i = 0; i < k; i++) {
        double del = (d[i] - dorg) - tau;
        s += z[i] * z[i] / del;
    }
    return 1.0 + rho * s;
}

/* Bisection for root j of a problem with rho > 0, d strictly ascending, z_i != 0.
 * Root j lies in (d_j, d_{j+1}) for j < k-1 and in (d_{k-1}, d_{k-1} + rho||z||^2]
 * for j = k-1; w increases from -inf to +inf across each bracket.  The origin is
 * the pole nearer to the root (decided by the sign of w at the bracket midpoint),
 * and the unknown is the offset tau from it.  Bisection stops when no double lies
 * strictly between the bracket ends. */
static int bisect_root_pos(int k, const double* d, const double* z, double rho, double znorm2,
                           int j, int* org_out, double* tau_out)
{
    int o;
    double lo, hi;
    if (j < k - 1) {
        double half = 0.5 * (d[j + 1] - d[j]);
        double wm = secular_w(k, d, z, rho, j, half);
        if (wm >= 0.0) { o = j;     lo = 0.0;             hi = d[j + 1] - d[j]; }
        else           { o = j + 1; lo = d[j] - d[j + 1]; hi = 0.0; }
    } else {
        o = k - 1; lo = 0.0; hi = rho * znorm2;
        int guard = 0;
        while (secular_w(k, d, z, rho, o, hi) < 0.0 && guard++ < 64) hi *= 2.0;
    }
    int it;
    for (it = 0; it < 4000; it++) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        double w = secular_w(k, d, z, rho, o, mid);
        if (w > 0.0) hi = mid; else lo = mid;
    }
    /* never return the pole itself */
    double tau;
    if (lo == 0.0) tau = hi;
    else if (hi == 0.0) tau = lo;
    else tau = 0.5 * (lo + hi);
    *org_out = o;
    *tau_out = tau;
    return it < 4000 ? ORC_OK : ORC_ENOCONV;
}

/* Sec. 3.1: all k roots of 1 + rho sum z_i^2/(d_i - mu), d strictly ascending,
 * z_i != 0, rho != 0.  Root j is returned as the pair (org[j], tau[j]) with
 * mu_j = d[org[j]] + tau[j]; roots are in ascending order.  A negative rho is
 * handled by reflection: eig(D + rho z z^T) = -eig(-D + |rho| z z^T). */
int oracle_secular_roots(int k, const double* d, const double* z, double rho, int* org, double* tau)
{
    if (k <= 0 || rho == 0.0) return ORC_EINVAL;
    double* dd = (double*)malloc(sizeof(double) * k);
    double* zz = (double*)malloc(sizeof(double) * k);
    if (!dd || !zz) { free(dd); free(zz); return ORC_ENOMEM; }
    double r = rho;
    if (rho > 0.0) {
        for (int i = 0; i < k; i++) { dd[i] = d[i]; zz[i] = z[i]; }
    } else {
        for (int i = 0; i < k; i++) { dd[i] = -d[k - 1 - i]; zz[i] = z[k - 1 - i]; }
        r = -rho;
    }
    double znorm2 = 0.0;
    for (int i = 0; i < k; i++) znorm2 += zz[i] * zz[i];
    int status = ORC_OK;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < k; j++) {
        int o; double t;
        int st = bisect_root_pos(k, dd, zz, r, znorm2, j, &o, &t);
        if (st != ORC_OK) {
            #pragma omp atomic write
            status = st;
        }
        if (rho > 0.0) { org[j] = o; tau[j] = t; }
        else { org[k - 1 - j] = k - 1 - o; tau[k - 1 - j] = -t; }
    }
    free(dd); free(zz);
    return status;
}

/* mu_j - d_i from offsets: (d[org_j] - d_i) + tau_j. */
static double root_minus_pole(const double* d, const int* org, const double* tau, int j, int i)
{
    return (d[org[j]] - d[i]) + tau[j];
}

/* Loewner recomputation of z from the computed roots (Sec. 3.2 reading; the
 * characteristic polynomial identity prod_j (mu_j - d_i) = rho zhat_i^2 prod_{j!=i} (d_j - d_i)).
 * Each pole j != i is paired with an adjacent root so every factor is a ratio in (0,1);
 * the formula is written for rho > 0 and the reflected problem is used for rho < 0. */
static void loewner_zhat(int k, const double* d, const double* z, double rho,
                         const int* org, const double* tau, double* zhat)
{
    /* reflected copies for rho < 0 */
    double* dd = (double*)malloc(sizeof(double) * k);
    int* oo = (int*)malloc(sizeof(int) * k);
    double* tt = (double*)malloc(sizeof(double) * k);
    double r = rho;
    if (rho > 0.0) {
        for (int i = 0; i < k; i++) { dd[i] = d[i]; oo[i] = org[i]; tt[i] = tau[i]; }
    } else {
        for (int i = 0; i < k; i++) {
            dd[i] = -d[k - 1 - i];
            oo[i] = k - 1 - org[k - 1 - i];
            tt[i] = -tau[k - 1 - i];
        }
        r = -rho;
    }
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < k; i++) {
        double prod = root_minus_pole(dd, oo, tt, k - 1, i) / r;
        for (int j = 0; j < i; j++)
            prod *= root_minus_pole(dd, oo, tt, j, i) / (dd[j] - dd[i]);
        for (int j = i + 1; j < k; j++)
            prod *= root_minus_pole(dd, oo, tt, j - 1, i) / (dd[j] - dd[i]);
        double mag = sqrt(prod > 0.0 ? prod : 0.0);
        int iz = (rho > 0.0) ? i : (k - 1 - i);
        zhat[iz] = (z[iz] < 0.0) ? -mag : mag;
    }
    free(dd); free(oo); free(tt);
}

/* ------------------------------------------------------------------------- */
/* The eigen-system of D + rho z z^T in compact form.                          */
/* ------------------------------------------------------------------------- */
typedef struct {
    int N, k, nrot;
    int* perm;        /* sorted position s -> original index                 */
    double* ds;       /* poles in sorted positions (after rotations)         */
    int* rj; int* ri; double* rc; double* rs;   /* rotations (sorted positions) */
    int* idx;         /* k non-deflated sorted positions                     */
    double* dk;       /* their poles                                          */
    double* zhat;     /* recomputed z (k)                                     */
    int* org; double* tau;  /* roots (k)                                     */
    double* inv_norm; /* 1/||c_j|| (k)                                        */
    double* lam;      /* all N eigenvalues, ascending                         */
    int* src;         /* final column c: root j (>=0) or -(s+1) deflated pos s */
} eigsys;

static void eigsys_free(eigsys* e)
{
    free(e->perm); free(e->ds); free(e->rj); free(e->ri); free(e->rc); free(e->rs);
    free(e->idx); free(e->dk); free(e->zhat); free(e->org); free(e->tau);
    free(e->inv_norm); free(e->lam); free(e->src);
    memset(e, 0, sizeof(*e));
}

typedef struct { double v; int kind; int id; } lamkey;  /* kind 0 deflated, 1 root */

static int cmp_lamkey(const void* a, const void* b)
{
    const lamkey* x = (const lamkey*)a;
    const lamkey* y = (const lamkey*)b;
    if (x->v < y->v) return -1;
    if (x->v > y->v) return 1;
    if (x->kind != y->kind) return x->kind - y->kind;
    return x->id - y->id;
}

typedef struct { double v; int id; } sortkey;
static int cmp_sortkey(const void* a, const void* b)
{
    const sortkey* x = (const sortkey*)a;
    const sortkey* y = (const sortkey*)b;
    if (x->v < y->v) return -1;
    if (x->v > y->v) return 1;
    return x->id - y->id;
}

/* The deflation tolerance: 8 u max(max|d_i|, |rho| ||z||^2). */
static double deflation_tol(int N, const double* d, double rho, double znorm2)
{
    double dmax = 0.0;
    for (int i = 0; i < N; i++) if (fabs(d[i]) > dmax) dmax = fabs(d[i]);
    double t = fabs(rho) * znorm2;
    return 8.0 * ORC_U * (dmax > t ? dmax : t);
}

static int eigsys_build(int N, const double* d, const double* z, double rho, eigsys* e)
{
    memset(e, 0, sizeof(*e));
    e->N = N;
    e->perm = (int*)malloc(sizeof(int) * N);
    e->ds = (double*)malloc(sizeof(double) * N);
    double* zs = (double*)malloc(sizeof(double) * N);
    char* defl = (char*)calloc(N, 1);
    e->rj = (int*)malloc(sizeof(int) * N); e->ri = (int*)malloc(sizeof(int) * N);
    e->rc = (double*)malloc(sizeof(double) * N); e->rs = (double*)malloc(sizeof(double) * N);
    e->idx = (int*)malloc(sizeof(int) * N);
    e->lam = (double*)malloc(sizeof(double) * N);
    e->src = (int*)malloc(sizeof(int) * N);
    sortkey* sk = (sortkey*)malloc(sizeof(sortkey) * N);
    if (!e->perm || !e->ds || !zs || !defl || !e->rj || !e->ri || !e->rc || !e->rs ||
        !e->idx || !e->lam || !e->src || !sk) {
        free(zs); free(defl); free(sk); eigsys_free(e); return ORC_ENOMEM;
    }
    /* sort the poles ascending, keeping the permutation */
    for (int i = 0; i < N; i++) { sk[i].v = d[i]; sk[i].id = i; }
    qsort(sk, N, sizeof(sortkey), cmp_sortkey);
    for (int s = 0; s < N; s++) { e->perm[s] = sk[s].id; e->ds[s] = d[sk[s].id]; zs[s] = z[sk[s].id]; }
    free(sk);

    double znorm2 = 0.0;
    for (int s = 0; s < N; s++) znorm2 += zs[s] * zs[s];
    double znorm = sqrt(znorm2);
    double tol = deflation_tol(N, e->ds, rho, znorm2);

    /* deflation case (1): negligible coupling |rho| ||z|| |z_i| <= tol */
    for (int s = 0; s < N; s++)
        if (rho == 0.0 || fabs(rho) * znorm * fabs(zs[s]) <= tol) defl[s] = 1;

    /* deflation case (3): (numerically) equal neighbouring poles */
    int j = -1;
    e->nrot = 0;
    for (int s = 0; s < N; s++) {
        if (defl[s]) continue;
        if (j < 0) { j = s; continue; }
        double r = hypot(zs[j], zs[s]);
        double c = zs[s] / r, sn = zs[j] / r;
        if (fabs((e->ds[s] - e->ds[j]) * c * sn) <= tol) {
            double dj = e->ds[j], dsv = e->ds[s];
            e->ds[j] = c * c * dj + sn * sn * dsv;
            e->ds[s] = sn * sn * dj + c * c * dsv;
            zs[j] = 0.0; zs[s] = r; defl[j] = 1;
            e->rj[e->nrot] = j; e->ri[e->nrot] = s; e->rc[e->nrot] = c; e->rs[e->nrot] = sn;
            e->nrot++;
        }
        j = s;
    }

    int k = 0;
    for (int s = 0; s < N; s++) if (!defl[s]) e->idx[k++] = s;
    e->k = k;
    e->dk = (double*)malloc(sizeof(double) * (k > 0 ? k : 1));
    double* zk = (double*)malloc(sizeof(double) * (k > 0 ? k : 1));
    e->zhat = (double*)malloc(sizeof(double) * (k > 0 ? k : 1));
    e->org = (int*)malloc(sizeof(int) * (k > 0 ? k : 1));
    e->tau = (double*)malloc(sizeof(double) * (k > 0 ? k : 1));
    e->inv_norm = (double*)malloc(sizeof(double) * (k > 0 ? k : 1));
    if (!e->dk || !zk || !e->zhat || !e->org || !e->tau || !e->inv_norm) {
        free(zk); free(zs); free(defl); eigsys_free(e); return ORC_ENOMEM;
    }
    for (int t = 0; t < k; t++) { e->dk[t] = e->ds[e->idx[t]]; zk[t] = zs[e->idx[t]]; }

    int status = ORC_OK;
    if (k > 0) {
        status = oracle_secular_roots(k, e->dk, zk, rho, e->org, e->tau);
        loewner_zhat(k, e->dk, zk, rho, e->org, e->tau, e->zhat);
        /* column norms ||c_j||^2 = sum_i zhat_i^2 / (d_i - mu_j)^2 */
        #pragma omp parallel for schedule(static)
        for (int jj = 0; jj < k; jj++) {
            double s2 = 0.0;
            for (int i = 0; i < k; i++) {
                double del = (e->dk[i] - e->dk[e->org[jj]]) - e->tau[jj];
                double c = e->zhat[i] / del;
                s2 += c * c;
            }
            e->inv_norm[jj] = 1.0 / sqrt(s2);
        }
    }

    /* all eigenvalues, ascending (ties: deflated first, then by index) */
    lamkey* lk = (lamkey*)malloc(sizeof(lamkey) * N);
    int c = 0;
    for (int s = 0; s < N; s++) if (defl[s]) { lk[c].v = e->ds[s]; lk[c].kind = 0; lk[c].id = s; c++; }
    for (int t = 0; t < k; t++) { lk[c].v = e->dk[e->org[t]] + e->tau[t]; lk[c].kind = 1; lk[c].id = t; c++; }
    qsort(lk, N, sizeof(lamkey), cmp_lamkey);
    for (int q = 0; q < N; q++) {
        e->lam[q] = lk[q].v;
        e->src[q] = lk[q].kind ? lk[q].id : -(lk[q].id + 1);
    }
    free(lk); free(zk); free(zs); free(defl);
    return status;
}

/* Column col of the N x N eigenvector matrix, in the ORIGINAL ordering of d. */
static void eigsys_column(const eigsys* e, int col, double* q /* N */, double* work /* N */)
{
    int N = e->N;
    for (int s = 0; s < N; s++) work[s] = 0.0;
    int src = e->src[col];
    if (src >= 0) {
        int j = src;
        double dorg = e->dk[e->org[j]];
        for (int t = 0; t < e->k; t++) {
            double del = (e->dk[t] - dorg) - e->tau[j];
            work[e->idx[t]] = e->zhat[t] / del * e->inv_norm[j];
        }
    } else {
        work[-(src + 1)] = 1.0;
    }
    /* Q = G_1^T ... G_r^T Q': apply the transposed rotations, last one first */
    for (int r = e->nrot - 1; r >= 0; r--) {
        int a = e->rj[r], b = e->ri[r];
        double c = e->rc[r], s = e->rs[r];
        double va = work[a], vb = work[b];
        work[a] = c * va + s * vb;
        work[b] = -s * va + c * vb;
    }
    for (int s = 0; s < N; s++) q[e->perm[s]] = work[s];
}

/* Full eigen-decomposition of diag(d) + rho z z^T: lam ascending (N), and if Q is
 * not NULL the N x N eigenvector matrix (column-major, ldq = N). */
int oracle_rank_one_eig(int N, const double* d, const double* z, double rho, double* lam, double* Q)
{
    if (N <= 0) return ORC_EINVAL;
    eigsys e;
    int st = eigsys_build(N, d, z, rho, &e);
    if (st == ORC_ENOMEM) return st;
    for (int q = 0; q < N; q++) lam[q] = e.lam[q];
    if (Q) {
        #pragma omp parallel
        {
            double* work = (double*)malloc(sizeof(double) * N);
            #pragma omp for schedule(static)
            for (int c = 0; c < N; c++) eigsys_column(&e, c, Q + (size_t)c * N, work);
            free(work);
        }
    }
    eigsys_free(&e);
    return st;
}

/* Compact output of one solve, for element-wise comparison with the GPU:
 * k, the non-deflated sorted positions idx (into ascending d), their poles dk,
 * the roots (org, tau), zhat and inv_norm.  Arrays must hold N entries. */
int oracle_rank_one_compact(int N, const double* d, const double* z, double rho, int* k_out,
                            int* idx, double* dk, int* org, double* tau, double* zhat, double* inv_norm,
                            double* lam)
{
    if (N <= 0) return ORC_EINVAL;
    eigsys e;
    int st = eigsys_build(N, d, z, rho, &e);
    if (st == ORC_ENOMEM) return st;
    *k_out = e.k;
    for (int t = 0; t < e.k; t++) {
        idx[t] = e.idx[t]; dk[t] = e.dk[t]; org[t] = e.org[t]; tau[t] = e.tau[t];
        zhat[t] = e.zhat[t]; inv_norm[t] = e.inv_norm[t];
    }
    for (int q = 0; q < N; q++) lam[q] = e.lam[q];
    eigsys_free(&e);
    return st;
}

/* RankOneUpdate (Sec. 6.2) with the direction already expressed in the basis:
 * given X (rows x N), poles d (N), z = X^T a1 (N) and rho, computes the eigen-
 * decomposition D + rho z z^T = Q diag(lam) Q^T and Y[:, c] = (X Q)[:, cols[c]]
 * for c < ncols (all N columns when cols is NULL; then ncols is ignored).
 * lam (N) ascending is always returned. */
int oracle_rank_one_update_z(int rows, int N, const double* X, int ldx, const double* d,
                             const double* z, double rho, double* lam,
                             double* Y, int ldy, int ncols, const int* cols)
{
    if (rows < 0 || N <= 0 || ldx < rows || ldy < rows) return ORC_EINVAL;
    eigsys e;
    int st = eigsys_build(N, d, z, rho, &e);
    if (st == ORC_ENOMEM) return st;
    for (int q = 0; q < N; q++) lam[q] = e.lam[q];
    int nc = cols ? ncols : N;
    if (Y && rows > 0) {
        #pragma omp parallel
        {
            double* work = (double*)malloc(sizeof(double) * N);
            double* qv = (double*)malloc(sizeof(double) * N);
            #pragma omp for schedule(dynamic, 4)
            for (int c = 0; c < nc; c++) {
                int col = cols ? cols[c] : c;
                eigsys_column(&e, col, qv, work);
                gemv_n(rows, N, X, ldx, qv, Y + (size_t)c * ldy);
            }
            free(work); free(qv);
        }
    }
    eigsys_free(&e);
    return st;
}

/* Y = Q X: the eigenvector matrix Q of diag(d) + rho z z^T (Sec. 3.2; column c belongs
 * to the c-th smallest eigenvalue, rows follow the order of d) applied to a thin X
 * (N x s, column-major, leading dimension N), one column of Q at a time.  This is the
 * product of Alg. 6.1 STEPs 5 and 7 evaluated for a few sampled vectors, so that sizes
 * whose full product is out of reach can still be checked column by column.  lam (N)
 * receives the eigenvalues, ascending. */
int oracle_rank_one_apply(int N, const double* d, const double* z, double rho, int s,
                          const double* X, double* Y, double* lam)
{
    if (N <= 0 || s < 0) return ORC_EINVAL;
    eigsys e;
    int st = eigsys_build(N, d, z, rho, &e);
    if (st == ORC_ENOMEM) return st;
    for (int q = 0; q < N; q++) lam[q] = e.lam[q];
    int fail = 0;
    #pragma omp parallel
    {
        double* work = (double*)malloc(sizeof(double) * N);
        double* qv = (double*)malloc(sizeof(double) * N);
        if (!work || !qv) {
            #pragma omp atomic write
            fail = 1;
        }
        #pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < s; t++) {
            if (!work || !qv) continue;
            const double* x = X + (size_t)t * N;
            double* y = Y + (size_t)t * N;
            for (int r = 0; r < N; r++) y[r] = 0.0;
            for (int c = 0; c < N; c++) {
                if (x[c] == 0.0) continue;
                eigsys_column(&e, c, qv, work);
                for (int r = 0; r < N; r++) y[r] += qv[r] * x[c];
            }
        }
        free(work); free(qv);
    }
    eigsys_free(&e);
    return fail ? ORC_ENOMEM : st;
}

/* RankOneUpdate (Sec. 6.2), STEPs 1-7, literally: abar = X^T a1 (STEP 1), then the
 * eigen-decomposition (STEPs 2-5) and the dense product (STEPs 6-7).
 * X is rows x N; Y receives X*Q (rows x N); d_out receives the N eigenvalues. */
int oracle_rank_one_update(int rows, int N, const double* X, int ldx, const double* d,
                           const double* a1, double rho, double* d_out, double* Y, int ldy)
{
    double* abar = (double*)malloc(sizeof(double) * N);
    if (!abar) return ORC_ENOMEM;
    oracle_gemv_t(rows, N, X, ldx, a1, abar);
    int st = oracle_rank_one_update_z(rows, N, X, ldx, d, abar, rho, d_out, Y, ldy, N, NULL);
    free(abar);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Alg. 6.1: A = U S V^T (m <= n), Ahat = A + a b^T -> Un, Sn, Vn.              */
/* U m x m (ldu), S m singular values (any order), V n x n (ldv); outputs are  */
/* separate arrays (Un m x m with ld m, Sn m descending, Vn n x n with ld n).  */
/* ------------------------------------------------------------------------- */
int oracle_svd_update(int m, int n, const double* U, int ldu, const double* S,
                      const double* V, int ldv, const double* a, const double* b,
                      double* Un, double* Sn, double* Vn)
{
    if (m <= 0 || n < m || ldu < m || ldv < n) return ORC_EINVAL;
    int st = ORC_OK, s2;
    size_t mm = (size_t)m * m, nn = (size_t)n * n;
    double* Vtb = (double*)malloc(sizeof(double) * n);
    double* Uta = (double*)malloc(sizeof(double) * m);
    double* bt = (double*)malloc(sizeof(double) * m);   /* btilde = U S V^T b */
    double* at = (double*)malloc(sizeof(double) * n);   /* atilde = V S^T U^T a */
    double* tmp = (double*)malloc(sizeof(double) * n);
    double* a1 = (double*)malloc(sizeof(double) * m);
    double* b1 = (double*)malloc(sizeof(double) * m);
    double* a2 = (double*)malloc(sizeof(double) * n);
    double* b2 = (double*)malloc(sizeof(double) * n);
    double* Du = (double*)malloc(sizeof(double) * m);
    double* Dv = (double*)malloc(sizeof(double) * n);
    double* Dt = (double*)malloc(sizeof(double) * n);
    double* Dn = (double*)malloc(sizeof(double) * n);
    double* Ut = (double*)malloc(sizeof(double) * mm);
    double* Vt = (double*)malloc(sizeof(double) * nn);
    double* Vo = (double*)malloc(sizeof(double) * nn);
    double* Uo = (double*)malloc(sizeof(double) * mm);
    if (!Vtb || !Uta || !bt || !at || !tmp || !a1 || !b1 || !a2 || !b2 || !Du || !Dv || !Dt ||
        !Dn || !Ut || !Vt || !Vo || !Uo) { st = ORC_ENOMEM; goto done; }

    /* STEP 1 */
    oracle_gemv_t(n, n, V, ldv, b, Vtb);                   /* V^T b            */
    for (int i = 0; i < m; i++) tmp[i] = S[i] * Vtb[i];    /* S V^T b          */
    gemv_n(m, m, U, ldu, tmp, bt);                         /* btilde = U S V^T b */
    oracle_gemv_t(m, m, U, ldu, a, Uta);                   /* U^T a            */
    for (int i = 0; i < n; i++) tmp[i] = (i < m) ? S[i] * Uta[i] : 0.0;
    gemv_n(n, n, V, ldv, tmp, at);                         /* atilde = V S^T U^T a */
    double beta = 0.0, alpha = 0.0;
    for (int i = 0; i < n; i++) beta += b[i] * b[i];
    for (int i = 0; i < m; i++) alpha += a[i] * a[i];
    for (int i = 0; i < m; i++) Du[i] = S[i] * S[i];
    for (int i = 0; i < n; i++) Dv[i] = (i < m) ? S[i] * S[i] : 0.0;

    /* STEP 2: [a btilde] Qu = [a1 b1] */
    double qu[6], qv[6];
    oracle_schur2(beta, qu);
    for (int i = 0; i < m; i++) { a1[i] = qu[2] * a[i] + qu[3] * bt[i]; b1[i] = qu[4] * a[i] + qu[5] * bt[i]; }
    /* STEP 3: [b atilde] Qv = [a2 b2] */
    oracle_schur2(alpha, qv);
    for (int i = 0; i < n; i++) { a2[i] = qv[2] * b[i] + qv[3] * at[i]; b2[i] = qv[4] * b[i] + qv[5] * at[i]; }

    /* STEP 4, 5: left singular vectors */
    s2 = oracle_rank_one_update(m, m, U, ldu, Du, a1, qu[0], Dt, Ut, m); if (s2) st = s2;
    s2 = oracle_rank_one_update(m, m, Ut, m, Dt, b1, qu[1], Dn, Uo, m); if (s2) st = s2;
    /* STEP 8: singular values (ascending here), clamped at zero */
    for (int i = 0; i < m; i++) Dn[i] = sqrt(Dn[i] > 0.0 ? Dn[i] : 0.0);
    /* descending order */
    for (int c = 0; c < m; c++) {
        Sn[c] = Dn[m - 1 - c];
        memcpy(Un + (size_t)c * m, Uo + (size_t)(m - 1 - c) * m, sizeof(double) * m);
    }

    /* STEP 6, 7: right singular vectors */
    s2 = oracle_rank_one_update(n, n, V, ldv, Dv, a2, qv[0], Dt, Vt, n); if (s2) st = s2;
    s2 = oracle_rank_one_update(n, n, Vt, n, Dt, b2, qv[1], Dn, Vo, n); if (s2) st = s2;
    for (int c = 0; c < n; c++)
        memcpy(Vn + (size_t)c * n, Vo + (size_t)(n - 1 - c) * n, sizeof(double) * n);

    /* pair signs: u_j^T Ahat v_j >= 0, Ahat v = U (S (V^T v)) + a (b^T v) */
    #pragma omp parallel
    {
        double* w1 = (double*)malloc(sizeof(double) * n);
        double* w2 = (double*)malloc(sizeof(double) * m);
        double* w3 = (double*)malloc(sizeof(double) * m);
        #pragma omp for schedule(dynamic, 2)
        for (int j = 0; j < m; j++) {
            double* vj = Vn + (size_t)j * n;
            oracle_gemv_t(n, m, V, ldv, vj, w1);       /* (V^T v)[0:m] (serial inside) */
            double btv = 0.0;
            for (int i = 0; i < n; i++) btv += b[i] * vj[i];
            for (int i = 0; i < m; i++) w2[i] = S[i] * w1[i];
            gemv_n(m, m, U, ldu, w2, w3);
            double t = 0.0;
            const double* uj = Un + (size_t)j * m;
            for (int i = 0; i < m; i++) t += uj[i] * (w3[i] + a[i] * btv);
            if (t < 0.0) for (int i = 0; i < n; i++) vj[i] = -vj[i];
        }
        free(w1); free(w2); free(w3);
    }

done:
    free(Vtb); free(Uta); free(bt); free(at); free(tmp); free(a1); free(b1); free(a2); free(b2);
    free(Du); free(Dv); free(Dt); free(Dn); free(Ut); free(Vt); free(Vo); free(Uo);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Independent check: one-sided Jacobi SVD (Hestenes) of A (m x n, m <= n).    */
/* Columns of W = A^T are rotated pairwise until mutually orthogonal; then     */
/* A = J diag(s) Y^T with s_p = ||w_p||, Y = W diag(1/s), J the accumulated    */
/* rotations.  Outputs: U (m x m), S (m, descending), Vt (n x m thin V).       */
/* ------------------------------------------------------------------------- */
int oracle_jacobi_svd(int m, int n, const double* A, int lda, double* U, double* S, double* V)
{
    if (m <= 0 || n < m || lda < m) return ORC_EINVAL;
    double* W = (double*)malloc(sizeof(double) * (size_t)n * m);
    double* J = (double*)malloc(sizeof(double) * (size_t)m * m);
    if (!W || !J) { free(W); free(J); return ORC_ENOMEM; }
    for (int p = 0; p < m; p++)
        for (int i = 0; i < n; i++) W[(size_t)p * n + i] = A[p + (size_t)i * lda];
    for (size_t i = 0; i < (size_t)m * m; i++) J[i] = 0.0;
    for (int p = 0; p < m; p++) J[(size_t)p * m + p] = 1.0;
    double tol = (double)m * ORC_U;
    int converged = 0;
    for (int sweep = 0; sweep < 100 && !converged; sweep++) {
        converged = 1;
        for (int p = 0; p < m - 1; p++) {
            for (int q = p + 1; q < m; q++) {
                double* wp = W + (size_t)p * n;
                double* wq = W + (size_t)q * n;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < n; i++) { al += wp[i] * wp[i]; be += wq[i] * wq[i]; ga += wp[i] * wq[i]; }
                if (ga == 0.0 || fabs(ga) <= tol * sqrt(al * be)) continue;
                converged = 0;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < n; i++) {
                    double x = wp[i], y = wq[i];
                    wp[i] = c * x - s * y; wq[i] = s * x + c * y;
                }
                double* jp = J + (size_t)p * m;
                double* jq = J + (size_t)q * m;
                for (int i = 0; i < m; i++) {
                    double x = jp[i], y = jq[i];
                    jp[i] = c * x - s * y; jq[i] = s * x + c * y;
                }
            }
        }
    }
    /* norms, then descending order */
    sortkey* sk = (sortkey*)malloc(sizeof(sortkey) * m);
    for (int p = 0; p < m; p++) {
        double s2 = 0.0;
        for (int i = 0; i < n; i++) s2 += W[(size_t)p * n + i] * W[(size_t)p * n + i];
        sk[p].v = -sqrt(s2); sk[p].id = p;
    }
    qsort(sk, m, sizeof(sortkey), cmp_sortkey);
    for (int c = 0; c < m; c++) {
        int p = sk[c].id;
        double sv = -sk[c].v;
        S[c] = sv;
        for (int i = 0; i < m; i++) U[(size_t)c * m + i] = J[(size_t)p * m + i];
        for (int i = 0; i < n; i++) V[(size_t)c * n + i] = sv > 0.0 ? W[(size_t)p * n + i] / sv : 0.0;
    }
    free(sk); free(W); free(J);
    return converged ? ORC_OK : ORC_ENOCONV;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
