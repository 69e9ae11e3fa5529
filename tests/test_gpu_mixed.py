"""Parity of the split-precision tensor-core products (SVDUP_MIXED_BF16X3 and
SVDUP_MIXED_FP16X2) with the CPU oracle, through the C ABI.

The mixed form keeps FP64 in the secular solve, the root offsets and the recomputed z
(so eigenvalues are exactly those of the FP64 path) and forms the products from
three-term BF16 splits (24 significant bits per operand) with FP32 accumulation over
one K tile in tensor memory and double-float accumulation across tiles: about 2^-24
relative per operand, a few units of 2^-24 per tile.  An output column of X Ctilde is
a sum of k terms x_t c_tj with sum_t |x_t c_tj| <= ||x|| ||c_j|| = ||x||.  The tests
state the bound they use: 2e-6 elementwise for one product of orthonormal rows, and
for a full update at most 1e-6 added to the reconstruction error of the FP64 oracle
(whose own error is set by the Gram formulation, about u ||Ahat||^2 in the squared
singular values).

The FP16 form splits every operand into two FP16 numbers at one power-of-two scale per
tile (22 significant bits down to 2^-3 of the tile's largest magnitude, absolute error
below 2^-39 of it beyond) and forms three partial products per K tile: about 2^-22
relative per operand, four times the BF16 form's, and its stated bounds are four times
as wide (8e-6 elementwise for one product; 4e-6 added to the oracle's reconstruction).
"""
import numpy as np
import pytest

from paper_1707_08369_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_TOL = 2e-6
# (elementwise bound for one product, bound added to the reconstruction error, vectors)
TOLS = {"MIXED_BF16X3": (2e-6, 1e-6, 1e-4), "MIXED_FP16X2": (8e-6, 4e-6, 4e-4)}
MODES = sorted(TOLS)


@pytest.fixture(scope="module")
def sv():
    import paper_1707_08369_gb300 as sv
    from paper_1707_08369_gb300 import build
    build.build()
    sv.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return sv


@pytest.fixture(scope="module")
def hnd(sv):
    return sv.Handle(0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def devF(x):
    return torch.from_numpy(np.asfortranarray(x).T.copy()).cuda().t()


@pytest.mark.parametrize("rows,N,dense,seed,spread", [
    (7, 33, True, 0, "u"),        # one ragged row tile, one ragged leaf
    (130, 200, True, 1, "u"),     # two row tiles, several leaves
    (96, 700, False, 2, "u"),     # far field on, uniform poles
    (257, 1500, False, 3, "g"),   # far field on, graded poles, ragged tiles
    (64, 1500, True, 4, "g"),     # forced dense on the same problem size
    (300, 2600, False, 5, "g"),   # leaf size 128
])
@pytest.mark.parametrize("mode_name", MODES)
def test_mixed_cauchy_product_vs_oracle(sv, hnd, orc, rows, N, dense, seed, spread, mode_name):
    g = np.random.default_rng(seed)
    d = g.uniform(0, 1, N) if spread == "u" else 10 ** (-6 * g.uniform(0, 1, N))
    z = g.standard_normal(N)
    rho = g.uniform(0.5, 2.0) * (1 if seed % 2 == 0 else -1)
    X = wl.haar(max(rows, N), g)[:rows, :N]
    lam_o, Y_o = orc.rank_one_update_z(X, d, z, rho)
    mode = getattr(sv, mode_name) | (sv.DENSE if dense else 0)
    lam_g, Y_g = hnd.cauchy_product(devF(X), dev(d), dev(z), rho, eps=1e-12, mode=mode)
    Y_g = Y_g.cpu().numpy()
    assert np.abs(lam_g.cpu().numpy() - lam_o).max() <= 1e-13 * np.abs(lam_o).max()
    err = np.abs(Y_g - Y_o).max()
    assert err <= TOLS[mode_name][0], err


def _invariants(U, S, V, a, b, Un, Sn, Vn):
    m, n = U.shape[0], V.shape[0]
    Ah = U @ np.diag(S) @ V[:, :m].T + np.outer(a, b)
    nrm = np.linalg.norm(Ah, 2)
    recon = np.linalg.norm(Ah @ Vn[:, :m] - Un * Sn) / nrm
    orthU = np.abs(Un.T @ Un - np.eye(m)).max()
    orthV = np.abs(Vn.T @ Vn - np.eye(n)).max()
    return recon, orthU, orthV


@pytest.mark.parametrize("mode_name", MODES)
@pytest.mark.parametrize("m,n,seed", [(48, 80, 3), (100, 100, 4), (513, 600, 5)])
def test_mixed_update_shapes(sv, hnd, orc, m, n, seed, mode_name):
    g = wl.rng(seed + 50)
    A = g.standard_normal((m, n))
    a = g.standard_normal(m); b = g.standard_normal(n)
    U, S, Vh = np.linalg.svd(A)
    Uo, So, Vo = orc.svd_update(U, S, Vh.T, a, b)
    tU, tS, tV = devF(U), dev(S), devF(Vh.T)
    hnd.update(tU, tS, tV, dev(a), dev(b), eps=1e-12, mode=getattr(sv, mode_name))
    Un, Sn, Vn = tU.cpu().numpy(), tS.cpu().numpy(), tV.cpu().numpy()
    _, rtol, vtol = TOLS[mode_name]
    # the roots are FP64 in both forms: singular values to the FP64 tolerance
    assert np.abs(Sn - So).max() <= 1e-12 * So[0]
    recon, orthU, orthV = _invariants(U, S, Vh.T, a, b, Un, Sn, Vn)
    recon_o, _, _ = _invariants(U, S, Vh.T, a, b, Uo, So, Vo)
    assert recon <= recon_o + rtol and orthU <= 10 * rtol and orthV <= 10 * rtol, (
        recon, recon_o, orthU, orthV)
    assert np.abs(Un - Uo).max() <= vtol
    assert np.abs(Vn[:, :m] - Vo[:, :m]).max() <= vtol


@pytest.mark.parametrize("mode_name", MODES)
def test_mixed_update_fmm_loguniform(sv, hnd, orc, mode_name):
    """Square n = 1536, log-uniform spectrum: far field on, split products."""
    U, S, V, a, b = wl.loguniform_sq(1536, seed=wl.BASE_SEED + 77)
    Uo, So, Vo = orc.svd_update(U, S, V, a, b)
    tU, tS, tV = devF(U), dev(S), devF(V)
    hnd.update(tU, tS, tV, dev(a), dev(b), eps=1e-12, mode=getattr(sv, mode_name))
    _, rtol, _ = TOLS[mode_name]
    Un, Sn, Vn = tU.cpu().numpy(), tS.cpu().numpy(), tV.cpu().numpy()
    assert np.abs(Sn - So).max() <= 1e-12 * So[0]
    recon, orthU, orthV = _invariants(U, S, V, a, b, Un, Sn, Vn)
    # The Gram formulation (App. A) fixes eigenvalues to about u ||Ahat||^2, which
    # bounds the reconstruction of any implementation, the FP64 oracle's included: the
    # split products may add at most 1e-6 to the oracle's own reconstruction error.
    recon_o, _, _ = _invariants(U, S, V, a, b, Uo, So, Vo)
    assert recon <= recon_o + rtol, (recon, recon_o)
    assert orthU <= 10 * rtol and orthV <= 10 * rtol, (orthU, orthV)


def test_mixed_matches_fp64_eigenvalues(sv, hnd):
    """The mixed forms keep the secular roots in FP64; the z of each side's second solve
    comes from double-float sums (about 2^-45 per term) instead of FP64 ones, so their
    singular values agree with the FP64 form's to far below the 1e-12 S_1 bar (1e-14 S_1
    here), and the two mixed forms with each other bitwise (the products do not feed
    the roots)."""
    U, S, V, a, b = wl.loguniform_sq(700, seed=wl.BASE_SEED + 5)
    outs = []
    for mode in (sv.FP64, sv.MIXED_BF16X3, sv.MIXED_FP16X2):
        tU, tS, tV = devF(U), dev(S), devF(V)
        hnd.update(tU, tS, tV, dev(a), dev(b), eps=1e-12, mode=mode)
        outs.append(tS.cpu().numpy())
    assert np.abs(outs[1] - outs[0]).max() <= 1e-14 * outs[0][0]
    assert np.array_equal(outs[1], outs[2])


def test_mixed_rejects_unsupported_modes(sv, hnd):
    U = devF(np.eye(4)); S = dev(np.ones(4)); V = devF(np.eye(4)); a = dev(np.ones(4))
    for mode in (3, sv.MIXED_BF16X3 | 0x4000, sv.MIXED_FP16X2 | 0x4000):
        with pytest.raises(sv.SvdupError) as ei:
            hnd.update(U, S, V, a, dev(np.ones(4)), mode=mode)
        assert ei.value.code == sv.EINVAL


@pytest.mark.parametrize("mode_name", MODES)
def test_dense_product_tile_widths_agree(sv, orc, mode_name):
    """The dense mixed product has two output-tile widths (64 and 128 columns) that the
    autotuner chooses between; both give the oracle's product within the mode's bound."""
    g = np.random.default_rng(61)
    N, rows = 300, 200
    d = g.uniform(0, 1, N); z = g.standard_normal(N); rho = 1.1
    X = wl.haar(N, g)[:rows, :N]
    lam_o, Y_o = orc.rank_one_update_z(X, d, z, rho)
    h = sv.Handle(0)
    try:
        mode = getattr(sv, mode_name)
        for w128 in (1 << 30, 1):
            h.set_tile_tuning(mode, w128)
            _, Y_g = h.cauchy_product(devF(X), dev(d), dev(z), rho, eps=1e-12, mode=mode | sv.DENSE)
            assert np.abs(Y_g.cpu().numpy() - Y_o).max() <= TOLS[mode_name][0]
    finally:
        h.close()
