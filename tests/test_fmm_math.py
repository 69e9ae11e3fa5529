"""The far field of the Cauchy products (App. D) on the CPU: the kernel 1/(x - y)
between a source leaf and a target leaf, interpolated at p Chebyshev nodes of the
first kind in both variables.  This is the operator chain P2M (source values to the
source nodes), M2L (kernel between the nodes) and L2P (target nodes to the targets)
that the library evaluates as three contractions.  Its error is measured against
direct summation of the kernel as p grows.

- The paper's interaction geometry (leaves of radius r whose centres are at least 4r
  apart, i.e. a gap of 2r) converges faster than 5^-p: the error is below 5^-p from
  p = 10 on, and below 2.5 * 5^-p before.  That is the rate behind App. D STEP 1's
  p = ceil(log5(1/eps)).
- The flat partition's closest admissible pair (a gap of one radius) has error
  4 (2 + sqrt 3)^-p.  That is the Bernstein-ellipse rate for a singularity 2r from the
  centre of a leaf of radius r.  There p = ceil(log5(1/eps)) leaves a worst-case error
  of about 200 eps at eps = 1e-12 (p = 18); p = ceil(log(4/eps) / log(2 + sqrt 3)) = 23
  meets it.
CPU only (numpy)."""
import numpy as np
import pytest


def cheb(p):
    """Chebyshev nodes of the first kind on [-1, 1] (App. D STEP 3)."""
    return np.cos((2 * np.arange(1, p + 1) - 1) * np.pi / (2 * p))


def lagrange(p, t):
    """Values L_i(t) of the Lagrange basis on the p nodes, for points t in [-1, 1]
    (barycentric form with the first-kind weights (-1)^i sin((2i + 1) pi / 2p))."""
    nodes = cheb(p)
    w = (-1.0) ** np.arange(p) * np.sin((2 * np.arange(p) + 1) * np.pi / (2 * p))
    d = t[:, None] - nodes[None, :]
    hit = d == 0.0
    d[hit] = 1.0
    q = w / d
    L = q / q.sum(axis=1, keepdims=True)
    for r, c in zip(*np.nonzero(hit)):
        L[r] = 0.0
        L[r, c] = 1.0
    return L


def far_field_error(p, ra, rb, gap, npts=300):
    """max |K - K_p| / max |K| over a source leaf [-ra, ra] and a target leaf of radius
    rb whose near edge is `gap` past the source leaf's, K(x, y) = 1 / (x - y)."""
    cb = ra + gap + rb
    xs = np.linspace(-ra, ra, npts)
    ys = np.linspace(cb - rb, cb + rb, npts)
    K = 1.0 / (xs[:, None] - ys[None, :])
    T = 1.0 / ((ra * cheb(p))[:, None] - (cb + rb * cheb(p))[None, :])       # M2L
    Kp = lagrange(p, xs / ra) @ T @ lagrange(p, (ys - cb) / rb).T             # P2M, L2P
    return np.abs(Kp - K).max() / np.abs(K).max()


def test_interpolation_is_exact_at_the_nodes():
    p = 9
    assert np.abs(lagrange(p, cheb(p)) - np.eye(p)).max() == 0.0
    # polynomials of degree < p are reproduced exactly (to rounding)
    t = np.linspace(-1, 1, 101)
    poly = lambda s: 3 * s ** 7 - s ** 4 + 0.5 * s - 2
    assert np.abs(lagrange(p, t) @ poly(cheb(p)) - poly(t)).max() <= 1e-13


@pytest.mark.parametrize("p,c", [(4, 2.5), (6, 2.5), (10, 1.0), (14, 1.0), (18, 1.0)])
def test_paper_geometry_meets_five_to_the_minus_p(p, c):
    """Centres 4r apart (gap 2r), equal radii: error <= c 5^-p."""
    assert far_field_error(p, 1.0, 1.0, 2.0) <= c * 5.0 ** -p


def test_closest_flat_pair_converges_as_two_plus_sqrt3():
    """Gap of one radius: the error is 4 (2 + sqrt 3)^-p, so at p = 18 it is some 200
    times 1e-12, above the eps that p = ceil(log5(1/eps)) was chosen for."""
    rho = 2.0 + np.sqrt(3.0)
    for p in (8, 12, 18):
        assert abs(far_field_error(p, 1.0, 1.0, 1.0) * rho ** p - 4.0) <= 0.04
    assert 1e-10 <= far_field_error(18, 1.0, 1.0, 1.0) <= 1e-9
    # the order that meets eps = 1e-12 at this gap, and the one below it does not
    p_needed = int(np.ceil(np.log(4.0 / 1e-12) / np.log(rho)))
    assert p_needed == 23
    assert far_field_error(p_needed, 1.0, 1.0, 1.0) <= 1e-12 < far_field_error(p_needed - 1, 1.0, 1.0, 1.0)


def test_unequal_leaves_follow_the_larger_radius():
    """Admissibility asks for a gap of max(r_a, r_b): with r_b = r_a / 2 and that gap
    the rate is the same 2 + sqrt 3 (the singularity is 2 r_a from the source centre)."""
    e12, e18 = far_field_error(12, 1.0, 0.5, 1.0), far_field_error(18, 1.0, 0.5, 1.0)
    assert abs((e12 / e18) ** (1.0 / 6.0) - (2.0 + np.sqrt(3.0))) <= 0.05
