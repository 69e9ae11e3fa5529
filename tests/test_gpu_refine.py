"""The orthogonalising refinement (one Newton-Schulz step X (3 I - X^T X) / 2 on the
tensor cores) against the oracle's FP64 step, through the C ABI.

Stated error of the GPU step: E = X^T X - I comes from 3-term BF16 split products (about
2^-24 relative per term, FP32 within a 64-term tile, double-float across tiles) and the
correction X E / 2 from one BF16 product (2^-8 of |E|).  The leading products of E
accumulate in FP32 over a 64-term tile, which leaves a random error of a few 1e-8 in each
entry of E (about 1e-7 at the largest).  For a matrix whose columns are orthonormal to
within 1e-5 the step's output agrees with the FP64 step to 1e-7 elementwise, and its
orthogonality (max |X^T X - I|) is at most 3e-7.  The gate: with the probe residual
below the tolerance X is left untouched (bitwise)."""
import numpy as np
import pytest

from paper_1707_08369_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def devF(x):
    return torch.from_numpy(np.asfortranarray(x).T.copy()).cuda().t()


def _perturbed(rows, cols, delta, seed):
    g = np.random.default_rng(seed)
    Q = wl.haar(rows, g)[:, :cols]
    return Q + delta * g.standard_normal((rows, cols)) / np.sqrt(rows)


@pytest.mark.parametrize("rows,cols,seed", [(700, 700, 1), (900, 500, 2), (200, 129, 3)])
def test_refine_matches_fp64_step(sv, hnd, orc, rows, cols, seed):
    X = _perturbed(rows, cols, 1e-5, seed)
    want = orc.newton_schulz_step(X)
    r_o = orc.probe_residual(X)
    tX = devF(X)
    r_g = float(hnd.refine(tX, tol=0.0).item())
    got = tX.cpu().numpy()
    assert abs(r_g - r_o) <= 1e-12 + 1e-9 * r_o, (r_g, r_o)
    assert np.abs(got - want).max() <= 1e-7
    orth0 = np.abs(X.T @ X - np.eye(cols)).max()
    orth1 = np.abs(got.T @ got - np.eye(cols)).max()
    assert orth1 <= 3e-7 and orth1 < orth0 / 5, (orth0, orth1)


def test_refine_gate_leaves_x_alone(sv, hnd, orc):
    X = _perturbed(300, 300, 1e-5, 4)
    tX = devF(X)
    r = float(hnd.refine(tX, tol=1e-2).item())
    assert abs(r - orc.probe_residual(X)) <= 1e-12
    assert np.array_equal(tX.cpu().numpy(), X)


@pytest.mark.parametrize("mode_name", ["MIXED_BF16X3", "MIXED_FP16X2"])
def test_update_with_refinement(sv, orc, mode_name):
    """An update with SVDUP_REFINE at tolerance 0: both outputs are refined; singular
    values unchanged, orthogonality better than without, the reconstruction within the
    mode's bound of the oracle's."""
    U, S, V, a, b = wl.loguniform_sq(1000, seed=wl.BASE_SEED + 91)
    Uo, So, Vo = orc.svd_update(U, S, V, a, b)
    Ah = U @ np.diag(S) @ V.T + np.outer(a, b)
    nrm = np.linalg.norm(Ah, 2)
    h = sv.Handle(0)
    try:
        h.set_refine_tol(0.0)
        res = {}
        for flags in (0, sv.REFINE):
            tU, tS, tV = devF(U), torch.from_numpy(S.copy()).cuda(), devF(V)
            h.update(tU, tS, tV, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(),
                     eps=1e-12, mode=getattr(sv, mode_name) | flags)
            Un, Sn, Vn = tU.cpu().numpy(), tS.cpu().numpy(), tV.cpu().numpy()
            res[flags] = (np.abs(Un.T @ Un - np.eye(1000)).max(),
                          np.abs(Vn.T @ Vn - np.eye(1000)).max(),
                          np.linalg.norm(Ah @ Vn - Un * Sn) / nrm, Sn)
        ru, rv = h.refine_residuals()
        assert ru > 0.0 and rv > 0.0
    finally:
        h.close()
    (oU0, oV0, rec0, S0), (oU1, oV1, rec1, S1) = res[0], res[sv.REFINE]
    assert np.array_equal(S0, S1)
    assert np.abs(S1 - So).max() <= 1e-12 * So[0]
    assert oU1 <= 3e-7 and oV1 <= 3e-7 and oU1 < oU0 and oV1 < oV0, (oU0, oU1, oV0, oV1)
    rec_o = np.linalg.norm(Ah @ Vo - Uo * So) / nrm
    assert rec1 <= rec_o + 4e-6, (rec1, rec_o)
