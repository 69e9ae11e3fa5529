"""Pins for the CPU oracle: each checks it against something other than itself
(closed forms, identities of the secular equation, LAPACK through numpy for
special cases, hand-worked values in tests/golden/), so that a dropped term, a
wrong sign or index, or a transposed operand in the oracle fails a test.
CPU only."""
import math
import os

import numpy as np
import pytest

from paper_1707_08369_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U53 = 2.0 ** -53


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


def _kv(line):
    out = {}
    for tok in line.split()[1:]:
        k, v = tok.split("=")
        out[k] = np.array([float(x) for x in v.split(",")])
    return out


# ---------------------------------------------------------------- Schur 2x2
@pytest.mark.parametrize("g", [0.0, 1.0, 3.5, 64.0, 1e8, -2.0, -1e6])
def test_schur2_closed_form(orc, g):
    """Alg. 6.1 STEP 2/3: [[g,1],[1,0]] = Q diag(r1,r2) Q^T; r1 r2 = -1 (det),
    r1 + r2 = g (trace), Q orthogonal."""
    r1, r2, Q = orc.schur2(g)
    M = np.array([[g, 1.0], [1.0, 0.0]])
    assert r1 >= r2
    assert abs(r1 * r2 + 1.0) <= 8 * U53
    assert abs((r1 + r2) - g) <= 8 * U53 * max(1.0, abs(g))
    assert np.abs(Q.T @ Q - np.eye(2)).max() <= 8 * U53
    assert np.abs(Q @ np.diag([r1, r2]) @ Q.T - M).max() <= 8 * U53 * max(1.0, abs(g))


# ---------------------------------------------------------------- GEMV
def test_gemv_exact_integers(orc):
    """RankOneUpdate STEP 1 (abar = U^T a1): small integers sum exactly."""
    g = np.random.default_rng(3)
    A = g.integers(-9, 10, size=(37, 23)).astype(np.float64)
    x = g.integers(-9, 10, size=37).astype(np.float64)
    y = orc.gemv_t(A, x)
    ref = [sum(int(A[r, c]) * int(x[r]) for r in range(37)) for c in range(23)]
    assert np.array_equal(y, np.array(ref, dtype=np.float64))


# ---------------------------------------------------------------- secular roots
def _mu(d, org, tau):
    return d[org] + tau


def test_secular_worked_example(orc):
    """Sec. 3.1 on the hand-worked 2x2 example in golden/worked_2x2.txt."""
    kv = _kv([r for r in _golden("worked_2x2.txt") if r.startswith("secular")][0])
    org, tau = orc.secular_roots(kv["d"], kv["z"], float(kv["rho"][0]))
    mu = _mu(kv["d"], org, tau)
    assert np.allclose(mu, kv["roots"], rtol=0, atol=4 * U53 * 5)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("sgn", [1.0, -1.0])
def test_secular_n2_closed_form(orc, seed, sgn):
    """n = 2: the roots of the quadratic det(D + rho z z^T - mu I) = 0."""
    g = np.random.default_rng(seed)
    d = np.sort(g.uniform(-2, 2, 2))
    z = g.standard_normal(2)
    rho = sgn * g.uniform(0.1, 3)
    org, tau = orc.secular_roots(d, z, rho)
    mu = _mu(d, org, tau)
    s = d[0] + d[1] + rho * (z @ z)
    disc = math.sqrt((d[0] - d[1] + rho * (z[0] ** 2 - z[1] ** 2)) ** 2 + 4 * rho ** 2 * z[0] ** 2 * z[1] ** 2)
    ref = np.sort([0.5 * (s - disc), 0.5 * (s + disc)])
    assert np.allclose(mu, ref, rtol=0, atol=16 * U53 * (abs(s) + disc))


def _secular_case(seed, k, rho_sign=1.0, spread="uniform"):
    g = np.random.default_rng(seed)
    if spread == "uniform":
        d = np.sort(g.uniform(0, 1, k))
    else:  # graded, like squared singular values spanning 8 decades
        d = np.sort(10.0 ** (-8 * g.uniform(0, 1, k)))
    z = g.standard_normal(k)
    rho = rho_sign * g.uniform(0.2, 5)
    return d, z, rho


@pytest.mark.parametrize("seed,k,sgn,spread", [(0, 5, 1, "uniform"), (1, 17, -1, "uniform"),
                                               (2, 64, 1, "graded"), (3, 40, -1, "graded"),
                                               (4, 200, 1, "uniform")])
def test_secular_identities(orc, seed, k, sgn, spread):
    """Sec. 3.1: (i) strict interlacing of poles and roots, (ii) the trace
    identity sum mu = sum d + rho ||z||^2, (iii) the characteristic ratio
    w(x) = prod_j (mu_j - x) / prod_i (d_i - x) at points away from the spectrum,
    (iv) the secular residual at each root is at rounding level."""
    d, z, rho = _secular_case(seed, k, sgn, spread)
    org, tau = orc.secular_roots(d, z, rho)
    mu = _mu(d, org, tau)
    assert np.all(np.diff(mu) > 0)
    if rho > 0:
        assert np.all(mu[:-1] > d[:-1]) and np.all(mu[:-1] < d[1:])
        assert d[-1] < mu[-1] <= d[-1] + rho * (z @ z) * (1 + 1e-14)
    else:
        assert np.all(mu[1:] < d[1:]) and np.all(mu[1:] > d[:-1])
        assert d[0] + rho * (z @ z) * (1 + 1e-14) <= mu[0] < d[0]
    tr = d.sum() + rho * (z @ z)
    assert abs(mu.sum() - tr) <= 64 * U53 * (np.abs(d).sum() + abs(rho) * (z @ z))
    g = np.random.default_rng(seed + 100)
    for x in g.uniform(d.max() + 1, d.max() + 5, 4).tolist() + g.uniform(d.min() - 5, d.min() - 1, 4).tolist():
        w = 1.0 + rho * np.sum(z * z / (d - x))
        ratio = np.prod((mu - x) / (d - x))
        assert abs(w - ratio) <= 1e-10 * max(1.0, abs(w))
    # residual with the offsets: |w(mu_j)| small relative to the size of its terms
    for j in range(k):
        delta = (d - d[org[j]]) - tau[j]
        terms = rho * z * z / delta
        assert abs(1.0 + terms.sum()) <= 1e-9 * (1.0 + np.abs(terms).sum())


@pytest.mark.parametrize("seed,k", [(10, 8), (11, 33), (12, 64)])
def test_secular_vs_lapack(orc, seed, k):
    """Brute force: the eigenvalues of the explicit matrix diag(d) + rho z z^T
    (LAPACK through numpy) equal the secular roots."""
    d, z, rho = _secular_case(seed, k, 1.0 if seed % 2 == 0 else -1.0)
    org, tau = orc.secular_roots(d, z, rho)
    mu = _mu(d, org, tau)
    M = np.diag(d) + rho * np.outer(z, z)
    ref = np.linalg.eigvalsh(M)
    assert np.abs(mu - ref).max() <= 32 * k * U53 * np.abs(ref).max()


# ---------------------------------------------------------------- eigen-system with vectors
@pytest.mark.parametrize("seed,k,sgn", [(20, 6, 1), (21, 50, -1), (22, 120, 1)])
def test_rank_one_eig_vectors(orc, seed, k, sgn):
    """Sec. 3.2: columns z_i/(d_i - mu_j), normalised, are the eigenvectors:
    residual, orthogonality, and agreement with LAPACK eigenvectors up to sign."""
    d, z, rho = _secular_case(seed, k, sgn, "graded" if seed == 22 else "uniform")
    perm = np.random.default_rng(seed).permutation(k)       # unsorted input order
    d, z = d[perm], z[perm]
    lam, Q = orc.rank_one_eig(d, z, rho)
    M = np.diag(d) + rho * np.outer(z, z)
    nrm = np.abs(M).max() * k
    assert np.abs(M @ Q - Q * lam).max() <= 64 * U53 * nrm
    assert np.abs(Q.T @ Q - np.eye(k)).max() <= 64 * k * U53
    w, E = np.linalg.eigh(M)
    assert np.abs(lam - w).max() <= 64 * k * U53 * np.abs(w).max()
    if seed != 22:  # well-separated spectrum: vectors are unique up to sign
        s = np.sign(np.sum(E * Q, axis=0))
        assert np.abs(E * s - Q).max() <= 1e-9


def test_deflation_zero_component(orc):
    """Sec. 3.1 deflation case (1): z_i = 0 leaves d_i an eigenvalue with the unit
    vector e_i as its eigenvector; case (3): equal poles keep one copy."""
    d = np.array([0.3, 0.1, 0.7, 0.5, 0.9])
    z = np.array([0.4, 0.0, 1.1, -0.6, 0.2])
    lam, Q = orc.rank_one_eig(d, z, 1.5)
    i = int(np.argmin(np.abs(lam - 0.1)))
    assert lam[i] == 0.1
    assert abs(abs(Q[1, i]) - 1.0) <= 1e-15 and np.abs(np.delete(Q[:, i], 1)).max() == 0.0
    M = np.diag(d) + 1.5 * np.outer(z, z)
    assert np.abs(M @ Q - Q * lam).max() <= 1e-14
    # exactly repeated poles
    d2 = np.array([0.2, 0.5, 0.5, 0.5, 0.8])
    z2 = np.array([0.3, 0.4, -0.2, 0.7, 0.5])
    lam2, Q2 = orc.rank_one_eig(d2, z2, -0.7)
    M2 = np.diag(d2) - 0.7 * np.outer(z2, z2)
    assert np.sum(np.abs(lam2 - 0.5) <= 2 * U53) == 2
    assert np.abs(M2 @ Q2 - Q2 * lam2).max() <= 1e-14
    assert np.abs(Q2.T @ Q2 - np.eye(5)).max() <= 1e-14
    assert np.abs(lam2 - np.linalg.eigvalsh(M2)).max() <= 1e-14


def test_deflation_near_equal_poles(orc):
    """Near-equal poles (gap 1e-13, the graded workload's pairs) deflate by a
    Givens rotation and the result is still an exact eigen-decomposition."""
    g = np.random.default_rng(7)
    d = np.sort(g.uniform(0, 1, 30))
    d[11] = d[10] + 1e-15
    d[21] = d[20] + 1e-13
    z = g.standard_normal(30)
    lam, Q = orc.rank_one_eig(d, z, 0.8)
    M = np.diag(d) + 0.8 * np.outer(z, z)
    assert np.abs(M @ Q - Q * lam).max() <= 1e-13
    assert np.abs(Q.T @ Q - np.eye(30)).max() <= 1e-13
    assert np.abs(lam - np.linalg.eigvalsh(M)).max() <= 1e-13


def test_deflation_unequal_weights(orc):
    """Sec. 3.1 case (3) with unequal weights: when z_i << z_j the rotation
    angle is small, so poles 1e-10 apart still deflate (|gap c s| <= tol).  The
    rotated poles then differ visibly from the originals, and a mix-up of the two
    rotated values moves an eigenvalue by about the gap."""
    g = np.random.default_rng(8)
    d = np.sort(g.uniform(0, 1, 30))
    d[11] = d[10] + 1e-10
    z = g.standard_normal(30)
    z[10] = 1e-7
    for rho in (0.8, -0.6):
        c = orc.rank_one_compact(d, z, rho)
        assert c["k"] == 29                      # the pair deflated to one pole
        lam, Q = orc.rank_one_eig(d, z, rho)
        M = np.diag(d) + rho * np.outer(z, z)
        w = np.linalg.eigvalsh(M)
        assert np.abs(lam - w).max() <= 1e-13
        assert np.abs(M @ Q - Q * lam).max() <= 1e-13
        assert np.abs(Q.T @ Q - np.eye(30)).max() <= 1e-13


@pytest.mark.parametrize("seed,k,sgn,spread", [(30, 50, 1, "uniform"), (31, 64, -1, "uniform"),
                                               (32, 40, 1, "graded")])
def test_rank_one_compact_fields(orc, seed, k, sgn, spread):
    """The compact eigen-system that the element-wise GPU comparisons use:
    (i) no deflation for generic data, idx the identity and dk the sorted poles;
    (ii) mu_j = dk[org_j] + tau_j are the eigenvalues (LAPACK), the origin is
    the nearer end of root j's interlacing bracket (Sec. 3.1) and tau points into it;
    (iii) the Loewner vector equals z to rounding, since the roots are exact to
    rounding (Sec. 3.2: rho zhat_i^2 prod_{j!=i}(d_j - d_i) = prod_j (mu_j - d_i));
    (iv) zhat_i/(d_i - mu_j) * inv_norm_j are unit columns and LAPACK's vectors."""
    g = np.random.default_rng(seed)
    d = np.sort(g.uniform(0, 1, k)) if spread == "uniform" else np.sort(10.0 ** (-4 * g.uniform(0, 1, k)))
    z = g.standard_normal(k)
    rho = sgn * g.uniform(0.5, 2.0)
    perm = g.permutation(k)
    c = orc.rank_one_compact(d[perm], z[perm], rho)
    assert c["k"] == k
    assert np.array_equal(c["idx"], np.arange(k)) and np.array_equal(c["dk"], d)
    zs = z                                          # z in sorted order
    mu = c["dk"][c["org"]] + c["tau"]
    M = np.diag(d) + rho * np.outer(zs, zs)
    w, E = np.linalg.eigh(M)
    assert np.abs(mu - w).max() <= 32 * k * U53 * np.abs(w).max()
    assert np.array_equal(c["lam"], np.sort(mu))
    j = np.arange(k)
    if sgn > 0:
        lo_pole, hi_pole = j, j + 1                 # root j in (d_j, d_{j+1})
    else:
        lo_pole, hi_pole = j - 1, j                 # root j in (d_{j-1}, d_j)
    org = c["org"]
    assert np.all((org == lo_pole) | (org == hi_pole))
    assert np.all(c["tau"][org == lo_pole] > 0) and np.all(c["tau"][org == hi_pole] < 0)
    inner = (lo_pole >= 0) & (hi_pole < k)
    gap = d[np.minimum(hi_pole, k - 1)] - d[np.maximum(lo_pole, 0)]
    assert np.all(np.abs(c["tau"][inner]) <= 0.5 * gap[inner] * (1 + 4 * U53))
    assert np.all(np.abs(c["zhat"] - zs) <= 4 * k * U53 * np.abs(zs))
    C = c["zhat"][:, None] / ((d[:, None] - d[org][None, :]) - c["tau"][None, :]) * c["inv_norm"][None, :]
    assert np.abs((C * C).sum(axis=0) - 1.0).max() <= 4 * k * U53
    if spread == "uniform":                         # separated roots: unique up to sign
        s = np.sign(np.sum(E * C, axis=0))
        assert np.abs(E * s - C).max() <= 1e-9
    assert np.abs(M @ C - C * mu).max() <= 64 * U53 * np.abs(M).max() * k


# ---------------------------------------------------------------- the full update (Alg. 6.1)
def _check_svd(orc, U, S, V, a, b, rtol=1e-12, graded=False):
    """Alg. 6.1 works with Ahat Ahat^T and Ahat^T Ahat (App. A), so the computed
    squared singular values carry an absolute error of order u ||Ahat||^2; on
    graded spectra the small sigmahat (below sqrt(u) ||Ahat||) are only that
    accurate, and left/right vectors inside such clusters pair only to that level.
    Those cases check the squared values and the eigen-residuals of the two
    Gram matrices instead of the reconstruction at 1e-11."""
    m, n = U.shape[0], V.shape[0]
    A = U @ np.diag(S) @ V[:, :m].T
    Ah = A + np.outer(a, b)
    Un, Sn, Vn = orc.svd_update(U, S, V, a, b)
    nrm = np.linalg.norm(Ah, 2)
    ref = np.linalg.svd(Ah, compute_uv=False)
    assert np.all(np.diff(Sn) <= 0)
    assert np.abs(Sn ** 2 - ref ** 2).max() <= 64 * m * U53 * nrm ** 2
    if not graded:
        assert np.abs(Sn - ref).max() <= rtol * nrm
    assert np.abs(Un.T @ Un - np.eye(m)).max() <= 1e-12
    assert np.abs(Vn.T @ Vn - np.eye(n)).max() <= 1e-12
    assert np.linalg.norm(Ah @ (Ah.T @ Un) - Un * Sn ** 2) <= 64 * m * U53 * nrm ** 2
    assert np.linalg.norm(Ah.T @ (Ah @ Vn[:, :m]) - Vn[:, :m] * Sn ** 2) <= 64 * n * U53 * nrm ** 2
    recon_tol = 1e-6 if graded else 1e-11
    assert np.linalg.norm(Ah @ Vn[:, :m] - Un * Sn) <= recon_tol * nrm
    if n > m:
        assert np.linalg.norm(Ah @ Vn[:, m:]) <= recon_tol * nrm
    # signs are paired: u_j^T Ahat v_j = sigma_j >= 0
    assert np.all(np.einsum("ij,ij->j", Un, Ah @ Vn[:, :m]) >= -1e-12 * nrm)
    # Frobenius identity ||Ahat||_F^2 = ||A||_F^2 + 2 (U^T a)^T S (V^T b)[:m] + |a|^2 |b|^2
    p = U.T @ a
    q = V.T @ b
    fro = np.sum(S ** 2) + 2 * p @ (S * q[:m]) + (a @ a) * (b @ b)
    assert abs(np.sum(Sn ** 2) - fro) <= 1e-12 * fro
    # Weyl interlacing for a rank-one change: sigma_{i+1}(A) <= sigmahat_i <= sigma_{i-1}(A)
    Sd = np.sort(S)[::-1]
    tol = (1e-7 if graded else 1e-12) * nrm
    for i in range(m):
        if i + 1 < m:
            assert Sn[i] >= Sd[i + 1] - tol
        if i - 1 >= 0:
            assert Sn[i] <= Sd[i - 1] + tol
    return Un, Sn, Vn, Ah


def test_svd_worked_example(orc):
    """Alg. 6.1 on the hand-worked example in golden/worked_2x2.txt."""
    kv = _kv([r for r in _golden("worked_2x2.txt") if r.startswith("svd")][0])
    U = np.eye(2); V = np.eye(2)
    Un, Sn, Vn = orc.svd_update(U, kv["sigma"], V, kv["a"], kv["b"])
    assert np.allclose(Sn, kv["sigmahat"], rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_svd_2x2_closed_form(orc, seed):
    """m = n = 2: sigma1^2 + sigma2^2 = ||Ahat||_F^2 and sigma1 sigma2 = |det Ahat|."""
    g = np.random.default_rng(seed)
    A = g.standard_normal((2, 2))
    a = g.standard_normal(2); b = g.standard_normal(2)
    U, S, Vt = np.linalg.svd(A)
    Un, Sn, Vn = orc.svd_update(U, S, Vt.T, a, b)
    Ah = A + np.outer(a, b)
    F = np.sum(Ah ** 2); det = abs(np.linalg.det(Ah))
    s1 = math.sqrt(0.5 * (F + math.sqrt(max(F * F - 4 * det * det, 0.0))))
    s2 = det / s1
    assert np.allclose(Sn, [s1, s2], rtol=0, atol=1e-13 * s1)


def test_svd_small_gaussian(orc):
    """The 64x64 Gaussian workload, with the input SVD from the oracle's own
    Jacobi SVD; values against LAPACK, plus every invariant."""
    A, a, b = wl.small_gaussian()
    U, S, Vt = orc.jacobi_svd(A)
    _check_svd(orc, U, S, Vt, a, b)


@pytest.mark.parametrize("m,n,seed", [(5, 9, 1), (16, 40, 2), (33, 33, 3)])
def test_svd_rectangular(orc, m, n, seed):
    A, a, b = wl.small_gaussian(m, n, seed)
    U, S, Vh = np.linalg.svd(A)
    _check_svd(orc, U, S, Vh.T, a, b)


def test_svd_graded_with_pairs(orc):
    """The graded spectrum with near-equal pairs (deflation), at a small size."""
    g = wl.rng(99)
    m, n = 96, 160
    S = wl.graded_sigma(m, g)
    U = wl.haar(m, g); V = wl.haar(n, g)
    a = g.standard_normal(m); b = g.standard_normal(n)
    _check_svd(orc, U, S, V, a, b, graded=True)


def test_svd_invariant_pair(orc):
    """Deflation through the data: with a orthogonal to u_i and b orthogonal to
    v_i, (sigma_i, u_i, v_i) stays a singular triple of Ahat."""
    g = wl.rng(5)
    m, n = 12, 12
    U = wl.haar(m, g); V = wl.haar(n, g)
    S = np.sort(g.uniform(0.5, 2.0, m))[::-1]
    a = g.standard_normal(m); b = g.standard_normal(n)
    i = 4
    a -= U[:, i] * (U[:, i] @ a)
    b -= V[:, i] * (V[:, i] @ b)
    Un, Sn, Vn, Ah = _check_svd(orc, U, S, V, a, b)
    j = int(np.argmin(np.abs(Sn - S[i])))
    assert abs(Sn[j] - S[i]) <= 1e-14 * S[0]
    assert abs(abs(Un[:, j] @ U[:, i]) - 1) <= 1e-13
    assert abs(abs(Vn[:, j] @ V[:, i]) - 1) <= 1e-13


def test_svd_duplicated_sigma(orc):
    """Exactly repeated singular values (deflation case (3))."""
    g = wl.rng(8)
    m, n = 10, 14
    U = wl.haar(m, g); V = wl.haar(n, g)
    S = np.array([3.0, 2.0, 2.0, 2.0, 1.5, 1.0, 1.0, 0.5, 0.25, 0.1])
    a = g.standard_normal(m); b = g.standard_normal(n)
    _check_svd(orc, U, S, V, a, b)


@pytest.mark.parametrize("m,n,seed", [(48, 48, 60), (50, 90, 61)])
def test_svd_update_sampled_columns(orc, m, n, seed):
    """The sampled form of Alg. 6.1 (every singular value, a few columns of the
    vectors, for sizes whose dense products are out of reach): its values are LAPACK's
    for the explicit Ahat, each sampled pair is a unit singular pair with the paired
    sign (Ahat v_j = sigma_j u_j, Ahat^T u_j = sigma_j v_j), and it agrees with the dense
    form column by column."""
    g = wl.rng(seed)
    U = wl.haar(m, g)
    V = wl.haar(n, g)
    S = np.sort(g.uniform(0.1, 3.0, m))[::-1]
    a = g.standard_normal(m)
    b = g.standard_normal(n)
    cols = np.array([0, 1, m // 2, m - 2, m - 1])
    Sn, Un, Vn = orc.svd_update_sampled(U, S, V, a, b, cols)
    Ah = U @ np.diag(S) @ V[:, :m].T + np.outer(a, b)
    ref = np.linalg.svd(Ah, compute_uv=False)
    assert np.abs(Sn - ref).max() <= 1e-14 * ref[0]
    for c, j in enumerate(cols):
        u, v = Un[:, c], Vn[:, c]
        assert abs(u @ u - 1.0) <= 64 * U53 and abs(v @ v - 1.0) <= 64 * U53
        assert np.linalg.norm(Ah @ v - Sn[j] * u) <= 1e-14 * ref[0]
        assert np.linalg.norm(Ah.T @ u - Sn[j] * v) <= 1e-14 * ref[0]
    Uo, So, Vo = orc.svd_update(U, S, V, a, b)
    assert np.abs(Un - Uo[:, cols]).max() <= 1e-13
    assert np.abs(Vn - Vo[:, cols]).max() <= 1e-13


def test_rank_one_apply_is_the_eigenvector_product(orc):
    """Q X column by column (the sampled products): on unit vectors it returns LAPACK's
    eigenvectors up to sign, and it is linear in X."""
    g = np.random.default_rng(62)
    N = 40
    d = np.sort(g.uniform(0.0, 1.0, N))
    z = g.standard_normal(N)
    rho = 0.9
    E = np.eye(N)[:, [0, 7, 39]]
    lam, QE = orc.rank_one_apply(d, z, rho, E)
    w, W = np.linalg.eigh(np.diag(d) + rho * np.outer(z, z))
    assert np.abs(lam - w).max() <= 64 * N * U53 * np.abs(w).max()
    ref = W[:, [0, 7, 39]]
    sgn = np.sign(np.sum(ref * QE, axis=0))
    assert np.abs(ref * sgn - QE).max() <= 1e-12
    X = g.standard_normal((N, 3))
    _, Y = orc.rank_one_apply(d, z, rho, X)
    _, Y2 = orc.rank_one_apply(d, z, rho, 2.0 * X[:, :1] - X[:, 1:2])
    assert np.abs(Y2[:, 0] - (2.0 * Y[:, 0] - Y[:, 1])).max() <= 1e-13


def test_jacobi_svd_vs_lapack(orc):
    g = np.random.default_rng(4)
    for m, n in [(1, 1), (3, 7), (20, 20), (31, 45)]:
        A = g.standard_normal((m, n))
        U, S, Vt = orc.jacobi_svd(A)
        ref = np.linalg.svd(A, compute_uv=False)
        assert np.abs(S - ref).max() <= 1e-13 * max(ref.max(), 1)
        assert np.abs(U @ np.diag(S) @ Vt.T - A).max() <= 1e-13 * max(ref.max(), 1)
        assert np.abs(U.T @ U - np.eye(m)).max() <= 1e-13
        assert np.abs(Vt.T @ Vt - np.eye(m)).max() <= 1e-13


def test_paper_table2_error_metric(orc):
    """Sec. 7, Eq. (error), Table 2 shapes (n = 10..50, entries uniform in [1, 9]):
    the exact update is far below the paper's printed errors (which came from
    unseeded runs and are context, not a target)."""
    for row in _golden("table2_errors.txt"):
        n, err_paper = int(row.split()[0]), float(row.split()[1])
        A, a, b = wl.uniform_square(n, 1.0, 9.0, wl.BASE_SEED + n)
        U, S, Vh = np.linalg.svd(A)
        Un, Sn, Vn = orc.svd_update(U, S, Vh.T, a, b)
        Ah = A + np.outer(a, b)
        err = np.abs(Ah - Un @ np.diag(Sn) @ Vn[:, :n].T).max() / np.linalg.svd(Ah, compute_uv=False).max()
        assert err < 1e-13
        assert err < 1e-6 * err_paper


def test_chebyshev_nodes_golden():
    """App. D Step 3 nodes, hand-worked for p = 4 (golden/worked_2x2.txt)."""
    kv = _kv([r for r in _golden("worked_2x2.txt") if r.startswith("cheb")][0])
    p = int(kv["p"][0])
    t = np.cos((2 * np.arange(1, p + 1) - 1) * np.pi / (2 * p))
    assert np.allclose(t, kv["nodes"], rtol=0, atol=1e-16)


# ------------------------------------------------------------------ refinement step
def test_newton_schulz_step_on_scaled_orthogonal(orc):
    """X = c Q: X^T X = c^2 I, so the step gives exactly c (3 - c^2) / 2 Q."""
    g = np.random.default_rng(31)
    Q = np.linalg.qr(g.standard_normal((60, 40)))[0]
    for c in (0.9, 1.0, 1.1):
        X1 = orc.newton_schulz_step(c * Q)
        assert np.abs(X1 - c * (3 - c * c) / 2 * Q).max() <= 1e-14


def test_newton_schulz_step_converges_quadratically(orc):
    """X = Q (I + eps S), S symmetric: the singular values 1 + eps s_i map to
    f(1 + x) = 1 - 3 x^2 / 2 - x^3 / 2, so the eigenvalues of X1^T X1 - I are
    -3 (eps s_i)^2 to leading order."""
    g = np.random.default_rng(32)
    Q = np.linalg.qr(g.standard_normal((50, 50)))[0]
    S = g.standard_normal((50, 50)); S = (S + S.T) / 2
    s = np.linalg.eigvalsh(S)
    for eps in (1e-3, 1e-4):
        X = Q @ (np.eye(50) + eps * S)
        X1 = orc.newton_schulz_step(X)
        ev = np.linalg.eigvalsh(X1.T @ X1 - np.eye(50))
        want = -3.0 * (eps * s) ** 2
        assert np.abs(np.sort(ev) - np.sort(want)).max() <= 2.0 * (eps * np.abs(s).max()) ** 3 + 1e-14


def test_probe_residual_definition(orc):
    """For c Q the residual is |c^2 - 1| exactly (X^T X w - w = (c^2 - 1) w); the probes
    are +-1 and differ from each other."""
    g = np.random.default_rng(33)
    Q = np.linalg.qr(g.standard_normal((70, 30)))[0]
    assert orc.probe_residual(Q) <= 1e-14
    for c in (0.999, 1.002):
        assert abs(orc.probe_residual(c * Q) - abs(c * c - 1)) <= 1e-13
    W = orc.probe_signs(257)
    assert set(np.unique(W)) == {-1.0, 1.0}
    assert all(np.abs(W[:, i] - W[:, j]).max() > 0 for i in range(4) for j in range(i))
    assert abs(W.mean()) < 0.15
