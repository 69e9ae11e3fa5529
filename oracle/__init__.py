"""Plain FP64 CPU oracle for the rank-one SVD update (Gandhi & Rajgor, arXiv 1707.08369).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` leg of ``bench.py``; never by the library.  It
shares no code with the CUDA path.  The arithmetic lives in ``svdup_oracle.c``
(plain C, OpenMP over independent roots and output columns); this module only
builds/loads it and marshals numpy arrays.

Functions and the passages they follow:
  schur2            Alg. 6.1 STEP 2/3 (and App. A): [[g,1],[1,0]] = Q diag(r1,r2) Q^T
  gemv_t            RankOneUpdate STEP 1 (Sec. 6.2): X^T a
  secular_roots     Sec. 3.1, zeros of the secular function, by bisection
  rank_one_eig      RankOneUpdate STEPs 2-5 (Sec. 6.2) with deflation (Sec. 3.1)
  rank_one_compact  the same, returned as (k, idx, poles, org, tau, zhat, 1/||c_j||)
  rank_one_update   RankOneUpdate STEPs 1-7 with a dense product (Sec. 6.2)
  rank_one_apply    Q X for a thin X (the products of Alg. 6.1 STEPs 5 and 7 on a few vectors)
  svd_update        Alg. 6.1 STEPs 1-8, descending order, paired signs
  svd_update_sampled  Alg. 6.1 with every singular value but only sampled columns of the
                    vectors, for sizes whose dense products are out of reach
  jacobi_svd        independent one-sided Jacobi SVD (Hestenes)
  newton_schulz_step  one orthogonalising step X (3 I - X^T X) / 2 of the precision form's
                    refinement (not in the paper; its definition written out in FP64)
  probe_residual    max over four fixed +-1 probes w of ||X^T X w - w|| / ||w|| (the
                    refinement's gate)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "svdup_oracle.c")
# A prebuilt variant of the library may be named in SVDUP_ORACLE_LIB: the
# planted-mistake tests compile altered copies of svdup_oracle.c and run the pins
# against each of them in a child process.
_VARIANT = os.environ.get("SVDUP_ORACLE_LIB")
_LIB_PATH = _VARIANT or os.path.join(_HERE, "liboracle.so")
_lib = None

OK, EINVAL, ENOMEM, ENOCONV = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile svdup_oracle.c into oracle/liboracle.so with gcc (-fopenmp)."""
    if _VARIANT:
        return _LIB_PATH
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_schur2.argtypes = [D, P]
        lib.oracle_gemv_t.argtypes = [I, I, P, I, P, P]
        lib.oracle_secular_roots.argtypes = [I, P, P, D, P, P]
        lib.oracle_rank_one_eig.argtypes = [I, P, P, D, P, P]
        lib.oracle_rank_one_compact.argtypes = [I, P, P, D, P, P, P, P, P, P, P, P]
        lib.oracle_rank_one_update_z.argtypes = [I, I, P, I, P, P, D, P, P, I, I, P]
        lib.oracle_rank_one_update.argtypes = [I, I, P, I, P, P, D, P, P, I]
        lib.oracle_rank_one_apply.argtypes = [I, P, P, D, I, P, P, P]
        lib.oracle_svd_update.argtypes = [I, I, P, I, P, P, I, P, P, P, P, P]
        lib.oracle_jacobi_svd.argtypes = [I, I, P, I, P, P, P]
        lib.oracle_num_threads.restype = I
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _vec(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())


def _mat(a):
    """Column-major float64 copy of a 2-D array."""
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def schur2(g: float):
    """Returns (r1, r2, Q) with [[g,1],[1,0]] = Q diag(r1, r2) Q^T."""
    out = np.zeros(6)
    _load().oracle_schur2(float(g), _p(out))
    Q = np.array([[out[2], out[4]], [out[3], out[5]]])
    return out[0], out[1], Q


def gemv_t(A, x):
    A = _mat(A)
    x = _vec(x)
    y = np.zeros(A.shape[1])
    _load().oracle_gemv_t(A.shape[0], A.shape[1], _p(A), A.shape[0], _p(x), _p(y))
    return y


def secular_roots(d, z, rho):
    """Roots of 1 + rho sum z_i^2/(d_i - mu) for strictly ascending d and nonzero z.
    Returns (org, tau): mu_j = d[org[j]] + tau[j], ascending."""
    d = _vec(d); z = _vec(z)
    k = d.size
    org = np.zeros(k, dtype=np.int32)
    tau = np.zeros(k)
    st = _load().oracle_secular_roots(k, _p(d), _p(z), float(rho), _p(org), _p(tau))
    if st not in (OK, ENOCONV):
        raise RuntimeError("oracle_secular_roots failed: %d" % st)
    return org, tau


def rank_one_eig(d, z, rho, vectors=True):
    """diag(d) + rho z z^T = Q diag(lam) Q^T, lam ascending."""
    d = _vec(d); z = _vec(z)
    N = d.size
    lam = np.zeros(N)
    Q = np.zeros((N, N), order="F") if vectors else None
    st = _load().oracle_rank_one_eig(N, _p(d), _p(z), float(rho), _p(lam),
                                      _p(Q) if vectors else None)
    if st not in (OK, ENOCONV):
        raise RuntimeError("oracle_rank_one_eig failed: %d" % st)
    return (lam, Q) if vectors else lam


def rank_one_compact(d, z, rho):
    """Compact eigen-system: dict(k, idx, dk, org, tau, zhat, inv_norm, lam)."""
    d = _vec(d); z = _vec(z)
    N = d.size
    k = ctypes.c_int(0)
    idx = np.zeros(N, dtype=np.int32); org = np.zeros(N, dtype=np.int32)
    dk = np.zeros(N); tau = np.zeros(N); zhat = np.zeros(N); inv = np.zeros(N); lam = np.zeros(N)
    st = _load().oracle_rank_one_compact(N, _p(d), _p(z), float(rho), ctypes.byref(k), _p(idx), _p(dk),
                                          _p(org), _p(tau), _p(zhat), _p(inv), _p(lam))
    if st not in (OK, ENOCONV):
        raise RuntimeError("oracle_rank_one_compact failed: %d" % st)
    k = k.value
    return dict(k=k, idx=idx[:k], dk=dk[:k], org=org[:k], tau=tau[:k], zhat=zhat[:k],
                inv_norm=inv[:k], lam=lam)


def rank_one_update_z(X, d, z, rho, cols=None):
    """Y = (X Q)[:, cols] for diag(d) + rho z z^T = Q diag(lam) Q^T.  Returns (lam, Y)."""
    X = _mat(X)
    d = _vec(d); z = _vec(z)
    rows, N = X.shape
    lam = np.zeros(N)
    if cols is None:
        Y = np.zeros((rows, N), order="F")
        st = _load().oracle_rank_one_update_z(rows, N, _p(X), max(rows, 1), _p(d), _p(z), float(rho),
                                               _p(lam), _p(Y), max(rows, 1), N, None)
    else:
        cols = np.ascontiguousarray(np.asarray(cols, dtype=np.int32))
        Y = np.zeros((rows, cols.size), order="F")
        st = _load().oracle_rank_one_update_z(rows, N, _p(X), max(rows, 1), _p(d), _p(z), float(rho),
                                               _p(lam), _p(Y), max(rows, 1), cols.size, _p(cols))
    if st not in (OK, ENOCONV):
        raise RuntimeError("oracle_rank_one_update_z failed: %d" % st)
    return lam, Y


def rank_one_update(X, d, a1, rho):
    """RankOneUpdate(X, a1, D, rho) of Sec. 6.2 (dense product).  Returns (lam, X Q)."""
    X = _mat(X)
    d = _vec(d); a1 = _vec(a1)
    rows, N = X.shape
    lam = np.zeros(N)
    Y = np.zeros((rows, N), order="F")
    st = _load().oracle_rank_one_update(rows, N, _p(X), rows, _p(d), _p(a1), float(rho), _p(lam), _p(Y), rows)
    if st not in (OK, ENOCONV):
        raise RuntimeError("oracle_rank_one_update failed: %d" % st)
    return lam, Y


def rank_one_apply(d, z, rho, X):
    """Q X for the eigenvectors Q of diag(d) + rho z z^T (column c: the c-th smallest
    eigenvalue) and a thin X (N x s).  Returns (lam ascending, Y = Q X)."""
    d = _vec(d); z = _vec(z)
    N = d.size
    X = _mat(np.asarray(X, dtype=np.float64).reshape(N, -1))
    s = X.shape[1]
    lam = np.zeros(N)
    Y = np.zeros((N, s), order="F")
    st = _load().oracle_rank_one_apply(N, _p(d), _p(z), float(rho), s, _p(X), _p(Y), _p(lam))
    if st not in (OK, ENOCONV):
        raise RuntimeError("oracle_rank_one_apply failed: %d" % st)
    return lam, Y


def svd_update(U, S, V, a, b):
    """Alg. 6.1: SVD of U diag(S) V^T + a b^T.  Returns (Un, Sn, Vn), Sn descending."""
    U = _mat(U); V = _mat(V)
    S = _vec(S); a = _vec(a); b = _vec(b)
    m, n = U.shape[0], V.shape[0]
    Un = np.zeros((m, m), order="F"); Sn = np.zeros(m); Vn = np.zeros((n, n), order="F")
    st = _load().oracle_svd_update(m, n, _p(U), m, _p(S), _p(V), n, _p(a), _p(b), _p(Un), _p(Sn), _p(Vn))
    if st not in (OK, ENOCONV):
        raise RuntimeError("oracle_svd_update failed: %d" % st)
    return Un, Sn, Vn


def svd_update_sampled(U, S, V, a, b, cols):
    """Alg. 6.1 at sizes whose dense products are out of reach: every singular value
    of Ahat = U diag(S) V^T + a b^T (descending), and only the columns `cols` (indices
    into the descending order, each < m) of Uhat and Vhat.  Returns (Sn, Un_cols, Vn_cols).

    The arithmetic is that of svd_update with STEP 1 read through the input SVD (the
    Sec. 6.2 direction U^T a1 expressed by p = U^T a and q = V^T b, since U^T btilde =
    S q[:m] and V^T atilde = [S p; 0]); the second solve of each side takes z = Q^T z'
    from the first.  Column j of Uhat is U Q1 Q2 e_(m-1-j) and of Vhat V Q3 Q4 e_(n-1-j)
    (the solves are ascending), and v_j is negated where u_j^T Ahat v_j < 0, as in
    svd_update."""
    U = np.asarray(U, dtype=np.float64); V = np.asarray(V, dtype=np.float64)
    S = _vec(S); a = _vec(a); b = _vec(b)
    m, n = U.shape[0], V.shape[0]
    cols = np.asarray(cols, dtype=np.int64).ravel()
    if cols.size and (cols.min() < 0 or cols.max() >= m):
        raise ValueError("sampled columns must lie in [0, m)")
    # STEP 1
    p = gemv_t(U, a)
    q = gemv_t(V, b)
    alpha, beta = float(a @ a), float(b @ b)
    # STEPs 2 and 3: [a btilde] Qu = [a1 b1], [b atilde] Qv = [a2 b2], in the basis
    r1, r2, Qu = schur2(beta)
    r3, r4, Qv = schur2(alpha)
    sq = S * q[:m]
    sp = np.concatenate([S * p, np.zeros(n - m)])
    z1 = Qu[0, 0] * p + Qu[1, 0] * sq
    z2p = Qu[0, 1] * p + Qu[1, 1] * sq
    z3 = Qv[0, 0] * q + Qv[1, 0] * sp
    z4p = Qv[0, 1] * q + Qv[1, 1] * sp
    Du = S * S
    Dv = np.concatenate([S * S, np.zeros(n - m)])

    def side(X, D, za, zb_prime, ra, rb, N):
        lam1, zrow = rank_one_update_z(zb_prime[None, :], D, za, ra)   # z of the second solve
        E = np.zeros((N, cols.size))
        E[N - 1 - cols, np.arange(cols.size)] = 1.0
        lam2, Q2E = rank_one_apply(lam1, zrow[0], rb, E)
        _, W = rank_one_apply(D, za, ra, Q2E)
        return lam2, X @ W

    lam_u, Un = side(U, Du, z1, z2p, r1, r2, m)                  # STEPs 4, 5
    _, Vn = side(V, Dv, z3, z4p, r3, r4, n)                      # STEPs 6, 7
    Sn = np.sqrt(np.maximum(lam_u, 0.0))[::-1].copy()            # STEP 8
    # pair the signs: u_j^T Ahat v_j >= 0, Ahat v = U (S (V^T v)[:m]) + a (b^T v)
    for c in range(cols.size):
        v = Vn[:, c]
        t = Un[:, c] @ (U @ (S * (V.T @ v)[:m]) + a * (b @ v))
        if t < 0.0:
            Vn[:, c] = -v
    return Sn, Un, Vn


def jacobi_svd(A):
    """One-sided Jacobi SVD of A (m x n, m <= n): A = U diag(S) Vt^T with Vt n x m."""
    A = _mat(A)
    m, n = A.shape
    U = np.zeros((m, m), order="F"); S = np.zeros(m); Vt = np.zeros((n, m), order="F")
    st = _load().oracle_jacobi_svd(m, n, _p(A), m, _p(U), _p(S), _p(Vt))
    if st not in (OK, ENOCONV):
        raise RuntimeError("oracle_jacobi_svd failed: %d" % st)
    return U, S, Vt


def newton_schulz_step(X):
    """X (3 I - X^T X) / 2 in FP64: one Newton-Schulz step toward the polar factor of X.
    Its plain definition; numpy's matmul is the only primitive."""
    X = np.asarray(X, dtype=np.float64)
    G = X.T @ X
    return X @ (1.5 * np.eye(X.shape[1]) - 0.5 * G)


def probe_signs(cols):
    """The four +-1 probe vectors of the refinement gate (cols x 4): entry (c, q) is the
    parity of the SplitMix64 finaliser of 0x9E3779B97F4A7C15 * (4 c + q + 1) (mod 2^64),
    -1 when odd."""
    M = (1 << 64) - 1
    out = np.empty((cols, 4))
    for c in range(cols):
        for q in range(4):
            x = (0x9E3779B97F4A7C15 * (4 * c + q + 1)) & M
            x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & M
            x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & M
            x ^= x >> 31
            out[c, q] = -1.0 if (x & 1) else 1.0
    return out


def probe_residual(X):
    """max_q ||X^T X w_q - w_q|| / ||w_q|| over the four probe vectors (FP64)."""
    X = np.asarray(X, dtype=np.float64)
    W = probe_signs(X.shape[1])
    R = X.T @ (X @ W) - W
    return float(np.max(np.linalg.norm(R, axis=0) / np.sqrt(X.shape[1])))
