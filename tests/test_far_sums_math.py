"""The mathematics of the far-field form of the solve's own sums (Löwner's zhat, the
column norms, Q^T y and Q x; reading R19), on the CPU.  CPU only (numpy); nothing here
runs or imports the CUDA path.

- Löwner's paired factors as Cauchy integrals: for x right of a pole d and its paired
  root mu, log((mu - x)/(d - x)) = int_d^mu ds / (s - x); for x left of them,
  log((mu - x)/(d - x)) = -int_mu^d ds / (s - x).  Both closed forms are checked against
  numerical quadrature of the kernel.
- The interval moments int_{ta}^{ta+D} T_m(t) dt from the difference recurrence
  dT_{m+1} = 2((ta + D) dT_m + D T_m(ta)) - dT_{m-1}, against Gauss-Legendre
  quadrature on the interval (exact for these degrees), for intervals from 1e-12 to 1 of
  the box: the recurrence keeps relative accuracy in D (an antiderivative's difference
  loses it for short intervals).
- Node weights from moments, W_b = (D_0 + 2 sum_{m>=1} T_m(t_b) D_m) / P, against the
  Lagrange basis integrated directly.
- The two-sided interpolation error of the Cauchy kernel and of its square at p = 28 for
  the closest admissible pair (a gap of the larger radius): below 4 (2 + sqrt 3)^-p
  relative, about 1e-16.
"""
import numpy as np
import pytest

P = 28


def cheb(p):
    return np.cos((2 * np.arange(p) + 1) * np.pi / (2 * p))


def interval_moments(ta, dl, p=P):
    """int_{ta}^{ta+dl} T_m, m < p, by the difference recurrence."""
    tb = ta + dl
    I = np.zeros(p)
    I[0] = dl
    I[1] = dl * (ta + 0.5 * dl)
    Tp, Tc = 1.0, ta
    dp, dq = 0.0, dl
    for m in range(1, p):
        dn = 2.0 * (tb * dq + dl * Tc) - dp
        if m >= 2:
            I[m] = 0.5 * (dn / (m + 1) - dp / (m - 1))
        Tp, Tc = Tc, 2.0 * ta * Tc - Tp
        dp, dq = dq, dn
    return I


def moments_exact(ta, dl, p=P):
    """The same integrals by Gauss-Legendre quadrature on the interval itself (exact for
    the degrees involved, and free of the cancellation of an antiderivative's
    difference: every term is dl times a bounded average)."""
    s, w = np.polynomial.legendre.leggauss(20)  # exact up to degree 39
    t = ta + 0.5 * dl * (s + 1)
    T = np.cos(np.arange(p)[:, None] * np.arccos(np.clip(t, -1, 1))[None, :])
    return 0.5 * dl * (T @ w)


def weights_from_moments(D, p=P):
    tb = cheb(p)
    W = np.empty(p)
    for b in range(p):
        T = np.cos(np.arange(p) * np.arccos(tb[b]))
        W[b] = (D[0] + 2.0 * np.dot(T[1:], D[1:])) / p
    return W


def lagrange(p, t):
    nodes = cheb(p)
    w = (-1.0) ** np.arange(p) * np.sin((2 * np.arange(p) + 1) * np.pi / (2 * p))
    q = w / (np.asarray(t)[:, None] - nodes[None, :])
    return q / q.sum(axis=1, keepdims=True)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_loewner_factor_is_a_cauchy_integral(seed):
    g = np.random.default_rng(seed)
    for _ in range(20):
        d = g.uniform(-1, 1)
        mu = d + g.uniform(1e-3, 0.5)
        # x right of the pair: log((mu - x)/(d - x)) = int_d^mu ds/(s - x)
        x = mu + g.uniform(0.1, 3.0)
        s, w = np.polynomial.legendre.leggauss(40)
        ss = 0.5 * (mu - d) * (s + 1) + d
        quad = 0.5 * (mu - d) * np.sum(w / (ss - x))
        assert abs(np.log((mu - x) / (d - x)) - quad) <= 1e-14
        # x left of the pair (root below its pole): -int_mu^d ds/(s - x)
        mu2 = d - g.uniform(1e-3, 0.5)
        x = mu2 - g.uniform(0.1, 3.0)
        ss = 0.5 * (d - mu2) * (s + 1) + mu2
        quad = 0.5 * (d - mu2) * np.sum(w / (ss - x))
        assert abs(np.log((mu2 - x) / (d - x)) - (-quad)) <= 1e-14


@pytest.mark.parametrize("dl", [1e-12, 1e-8, 1e-4, 1e-2, 0.3, 1.0])
def test_interval_moments_keep_relative_accuracy(dl):
    g = np.random.default_rng(int(1e3 * dl) + 7)
    for _ in range(10):
        ta = g.uniform(-1, 1 - dl)
        got = interval_moments(ta, dl)
        ref = moments_exact(ta, dl)
        # each moment is dl times an average of T_m over the interval (|T_m| <= 1): the
        # error is a small multiple of u dl (m u dl at the box's ends)
        assert np.all(np.abs(got - ref) <= 64 * P * 2.0 ** -53 * dl), np.abs(got - ref).max() / dl


def test_node_weights_are_the_integrated_lagrange_basis():
    ta, dl = -0.3, 0.45
    W = weights_from_moments(interval_moments(ta, dl))
    s, w = np.polynomial.legendre.leggauss(30)
    tt = 0.5 * dl * (s + 1) + ta
    direct = 0.5 * dl * (w[:, None] * lagrange(P, tt)).sum(axis=0)
    assert np.abs(W - direct).max() <= 1e-15


@pytest.mark.parametrize("power", [1, 2])
def test_closest_admissible_pair_at_p28(power):
    """Source box [-1, 1] (radius 1), target box of radius rt whose gap to it is
    max(1, rt); sources and targets random; the kernel 1/(s - x)^power interpolated at
    28 nodes in both boxes against direct evaluation."""
    g = np.random.default_rng(power)
    bound = 4 * (2 + np.sqrt(3)) ** -P
    for rt in (0.5, 1.0, 2.0):
        gap = max(1.0, rt)
        ct = 1.0 + gap + rt
        s = g.uniform(-1, 1, 200)
        x = ct + rt * g.uniform(-1, 1, 200)
        K = 1.0 / (s[None, :] - x[:, None]) ** power
        ns, nt = cheb(P), ct + rt * cheb(P)
        Kn = 1.0 / (ns[None, :] - nt[:, None]) ** power
        approx = lagrange(P, (x - ct) / rt) @ Kn @ lagrange(P, s).T
        assert np.abs(approx - K).max() <= bound * np.abs(K).max() + 64 * 2.0 ** -53 * np.abs(K).max()
