"""Property tests of the oracle on random inputs over many scales (hypothesis): the
secular roots interlace the poles and sum to the trace (Sec. 3.1), they are LAPACK's
eigenvalues of diag(d) + rho z z^T, and the full eigen-system with deflation (poles
repeated or nearly so, zero weights) is an orthogonal eigen-decomposition.  CPU only;
skipped where hypothesis is not installed."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings, HealthCheck = hyp.given, hyp.settings, hyp.HealthCheck

U53 = 2.0 ** -53
SETTINGS = settings(max_examples=300, deadline=None, derandomize=True,
                    suppress_health_check=[HealthCheck.too_slow])


@st.composite
def secular_problem(draw, max_k=40):
    """Strictly ascending poles at scale 10^e, nonzero weights, rho = +-10^f."""
    k = draw(st.integers(1, max_k))
    seed = draw(st.integers(0, 2 ** 32 - 1))
    e = draw(st.integers(-8, 8))
    f = draw(st.integers(-3, 3))
    sgn = draw(st.sampled_from([1.0, -1.0]))
    g = np.random.default_rng(seed)
    d = np.unique(g.uniform(-1.0, 1.0, k)) * 10.0 ** e
    z = g.standard_normal(d.size) * 10.0 ** (e / 2)
    z[np.abs(z) < 1e-3 * 10.0 ** (e / 2)] = 10.0 ** (e / 2)  # keep every weight clear of 0
    return d, z, sgn * 10.0 ** f


@st.composite
def deflating_problem(draw, max_n=30):
    """Poles with exact repeats, near repeats (relative gap 1e-14) and zero weights."""
    n = draw(st.integers(2, max_n))
    seed = draw(st.integers(0, 2 ** 32 - 1))
    g = np.random.default_rng(seed)
    d = g.uniform(0.0, 1.0, n)
    reps = g.integers(0, n, size=n // 3)
    d[reps] = d[(reps + 1) % n]                        # exact repeats
    near = g.integers(0, n, size=n // 4)
    d[near] = d[(near + 2) % n] * (1 + 1e-14)          # near repeats
    z = g.standard_normal(n)
    z[g.integers(0, n, size=n // 5)] = 0.0             # zero weights
    if not np.any(z):
        z[0] = 1.0
    rho = float(g.choice([-1.0, 1.0]) * 10.0 ** g.uniform(-2, 2))
    return d, z, rho


@SETTINGS
@given(secular_problem())
def test_roots_interlace_and_sum_to_the_trace(orc, prob):
    d, z, rho = prob
    org, tau = orc.secular_roots(d, z, rho)
    mu = d[org] + tau
    k = d.size
    z2 = float(z @ z)
    assert np.all(np.diff(mu) > 0)
    if rho > 0:
        assert np.all(mu[:-1] > d[:-1]) and np.all(mu[:-1] < d[1:])
        assert mu[-1] > d[-1] and mu[-1] <= d[-1] + rho * z2 * (1 + 4 * U53)
    else:
        assert np.all(mu[1:] < d[1:]) and np.all(mu[1:] > d[:-1])
        assert mu[0] < d[0] and mu[0] >= d[0] + rho * z2 * (1 + 4 * U53)
    # trace of diag(d) + rho z z^T
    scale = np.abs(d).sum() + abs(rho) * z2
    assert abs(mu.sum() - (d.sum() + rho * z2)) <= 8 * k * U53 * scale


@SETTINGS
@given(secular_problem())
def test_roots_are_lapack_eigenvalues(orc, prob):
    d, z, rho = prob
    org, tau = orc.secular_roots(d, z, rho)
    mu = d[org] + tau
    w = np.linalg.eigvalsh(np.diag(d) + rho * np.outer(z, z))
    assert np.abs(mu - w).max() <= 32 * d.size * U53 * np.abs(w).max()


@SETTINGS
@given(deflating_problem())
def test_deflated_eigensystem_is_orthogonal_and_exact(orc, prob):
    d, z, rho = prob
    lam, Q = orc.rank_one_eig(d, z, rho)
    n = d.size
    M = np.diag(d) + rho * np.outer(z, z)
    nrm = np.abs(M).max() * n
    assert np.all(np.diff(lam) >= 0)
    assert np.abs(M @ Q - Q * lam).max() <= 64 * U53 * nrm
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 64 * n * U53
    w = np.linalg.eigvalsh(M)
    assert np.abs(lam - w).max() <= 64 * n * U53 * max(np.abs(w).max(), 1e-300)
