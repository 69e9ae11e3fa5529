"""The far-field form of the solve's own sums (csrc/svdup_vfmm.cu): Loewner's zhat
(Sec. 3.2) and the column norms 1/||c_j|| with Q^T y (RankOneUpdate STEP 7), summed
through App. D's interpolation FMM (here from a non-deflated size k of 2048 on; the
library's defaults start it where it overtakes the direct sums).

Four kinds of check, through the C ABI:
- against the oracle (its own bisection roots, direct products and sums), at the
  compact eigen-system tests' bars: the deflated set exactly, zhat within 1e-11
  max|zhat|, 1/||c_j|| within 1e-10 relative.  The norms of roots inside a cluster far
  from the origin (1e-6 wide at 5) are as sensitive to the roots' last bits as the
  roots' offsets are small (the oracle and the device agree there to 1e-4, with the
  direct sums and with the far field alike), so those spectra compare the norms with the
  direct sums only;
- against the direct sums on the same device (a second handle with
  svdup_set_far_sums(h, INT_MAX, INT_MAX): the same deflation and the same roots), elementwise
  within the direct sums' own rounding bound, 4 k u relative for zhat (a product of k
  ratios, two roundings each) and 2 k u for 1/||c_j|| (k positive terms), and in RMS
  within 2e-14 (the far field's interpolation error is about 1e-16; the direct sums'
  rounding is a random walk of about sqrt(k) u, 1e-14 at k = 8192);
- y = Q x, the sign pairing's product, whose far field takes the roots as sources
  (svdup_rank_one_apply): against the oracle's Q x within 1e-9 of max|y| (the columns of
  Q carry the roots' differences) and against the direct sums within 1e-12;
- whole updates (n = 4096, where Q^T y forms the second solves' z) with and without the
  far-field form: FP64, singular values within 1e-13 S_1 and columns whose squared value
  is 1e-3 (relatively) from its neighbours within 1e-9; split BF16 (whose direct sums run
  in FP32 pairs, 2^-44 relative), 1e-12 S_1 and 1e-5.
Spectra: uniform, log-uniform squared with rho = ||b||^2 (the benchmark's first solve:
heavy deflation, k about 5000 of 8192), multi-scale clusters (poles from 1e-12 to 3,
clusters 1e-5 wide at 0.3 and 1e-6 wide at 5, rho < 0) and graded 10^(-8 U) with
rho < 0.  A fifth spectrum puts the last quarter of the poles within 1e-9 of 5, where
they are 200 ulps apart and merge by the deflation rotations: there the kept poles are
weighted means whose last bits depend on the summation order, which moves the norms of
the cluster's roots by far more than 1e-10 between any two implementations, so it is
compared with the direct sums only (same poles, same roots), where the far field's boxes
are narrower than the ulp of their position.
"""
import numpy as np
import pytest

from paper_1707_08369_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U53 = 2.0 ** -53
OFF = 2 ** 31 - 1


@pytest.fixture(scope="module")
def sv():
    import paper_1707_08369_gb300 as sv
    from paper_1707_08369_gb300 import build
    build.build()
    sv.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return sv


@pytest.fixture(scope="module")
def handles(sv):
    far = sv.Handle(0)
    far.set_far_sums(2048, 2048)
    direct = sv.Handle(0)
    direct.set_far_sums(OFF, OFF)
    return far, direct


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def spectrum(case, N, g):
    if case == "uniform":
        return g.uniform(0, 1, N), 1.7
    if case == "loguni":
        d = np.sort(wl.loguniform_sigma(N, g)) ** 2
        b = g.standard_normal(N)
        return d, float(b @ b)
    if case in ("multi", "tight"):
        q = N // 4
        w = 1e-6 if case == "multi" else 1e-9
        d = np.concatenate([10 ** g.uniform(-12, 0, q), g.uniform(0.3, 0.30001, q),
                            g.uniform(2, 3, q), g.uniform(5, 5 + w, N - 3 * q)])
        return d, -0.8
    if case == "graded":
        return 10 ** (-8 * g.uniform(0, 1, N)), -2.0
    raise ValueError(case)


# (case, N, seed, norms compared with the oracle)
CASES = [("uniform", 4096, 0, True), ("loguni", 8192, 1, True), ("multi", 5000, 2, False),
         ("graded", 3000, 3, True), ("tight", 5000, 4, False)]


@pytest.mark.parametrize("case,N,seed,norms_vs_oracle", CASES)
def test_far_sums_vs_oracle_and_direct(sv, handles, orc, case, N, seed, norms_vs_oracle):
    g = wl.rng(wl.BASE_SEED + 300 + seed)
    d, rho = spectrum(case, N, g)
    z = g.standard_normal(N)
    far, direct = handles
    out = far.rank_one_eig(dev(d), dev(z), rho)
    k = int(out["k"].item())
    assert k >= 2048, k  # the far-field form is in use
    zh = out["zhat"].cpu().numpy()[:k]
    inv = out["inv_norm"].cpu().numpy()[:k]
    ref = orc.rank_one_compact(d, z, rho)
    assert k == ref["k"]
    assert np.array_equal(out["idx"].cpu().numpy()[:k], ref["idx"])
    assert np.abs(zh - ref["zhat"]).max() <= 1e-11 * np.abs(ref["zhat"]).max()
    if norms_vs_oracle:
        assert np.all(np.abs(inv - ref["inv_norm"]) <= 1e-10 * np.abs(ref["inv_norm"]))
    # the same problem with the direct sums
    o2 = direct.rank_one_eig(dev(d), dev(z), rho)
    assert int(o2["k"].item()) == k
    assert torch.equal(out["tau"][:k], o2["tau"][:k]) and torch.equal(out["org"][:k], o2["org"][:k])
    zd = o2["zhat"].cpu().numpy()[:k]
    idd = o2["inv_norm"].cpu().numpy()[:k]
    rz = np.abs(zh - zd) / np.abs(zd)
    ri = np.abs(inv - idd) / np.abs(idd)
    assert rz.max() <= 4 * k * U53, rz.max()
    assert ri.max() <= 2 * k * U53, ri.max()
    assert np.sqrt(np.mean(rz ** 2)) <= 2e-14 and np.sqrt(np.mean(ri ** 2)) <= 2e-14


@pytest.mark.parametrize("case,N,seed", [("uniform", 4096, 10), ("loguni", 8192, 11),
                                         ("graded", 3000, 13), ("tight", 5000, 14)])
def test_apply_q_vs_oracle_and_direct(sv, handles, orc, case, N, seed):
    """y = Q x (the sign pairing's product) with Q x's far-field form: against the oracle's
    Q x (its own roots; 1e-9 of max|y|) and against the direct sums on the same roots
    (1e-12 of max|y|)."""
    g = wl.rng(wl.BASE_SEED + 320 + seed)
    d, rho = spectrum(case, N, g)
    z = g.standard_normal(N)
    x = g.standard_normal(N)
    far, direct = handles
    y1, lam1 = far.rank_one_apply(dev(d), dev(z), rho, dev(x))
    y2, _ = direct.rank_one_apply(dev(d), dev(z), rho, dev(x))
    y1, y2 = y1.cpu().numpy(), y2.cpu().numpy()
    scale = np.abs(y2).max()
    assert np.abs(y1 - y2).max() <= 1e-12 * scale, np.abs(y1 - y2).max() / scale
    if case != "tight":
        lam_o, yo = orc.rank_one_apply(d, z, rho, x)
        # the largest root (rho ||z||^2 past the poles) within the evaluation bound k u
        assert np.abs(lam1.cpu().numpy() - lam_o).max() <= 4 * N * U53 * np.abs(lam_o).max()
        assert np.abs(y1 - yo[:, 0]).max() <= 1e-9 * scale


@pytest.mark.parametrize("mode,sbar,vbar", [("FP64", 1e-13, 1e-9), ("MIXED_BF16X3", 1e-12, 1e-5)])
def test_update_with_and_without_far_sums(sv, handles, mode, sbar, vbar):
    far, direct = handles
    n = 4096
    U, S, V, a, b = wl.loguniform_sq(n, seed=wl.BASE_SEED + 310, device=torch.device("cuda", 0))
    res = []
    for h in (far, direct):
        def colmajor(X):
            return torch.from_numpy(np.asfortranarray(X).T.copy()).cuda().t()
        tU, tV = colmajor(U), colmajor(V)
        tS = torch.from_numpy(np.ascontiguousarray(S)).cuda()
        h.update(tU, tS, tV, dev(a), dev(b), eps=1e-12, mode=getattr(sv, mode), check=True)
        res.append((tS.cpu().numpy(), tU.cpu().numpy(), tV.cpu().numpy()))
    (S1, U1, V1), (S2, U2, V2) = res
    assert np.abs(S1 - S2).max() <= sbar * S2[0]
    # The second solves' poles move by the rounding of their z (about 1e-14 relative), so
    # a column moves by about that over its relative gap; columns whose squared value is
    # at least 1e-3 (relatively) from both neighbours are compared.
    sq = S2 ** 2
    gaps = np.minimum(np.abs(np.diff(sq, prepend=np.inf)), np.abs(np.diff(sq, append=-np.inf)))
    sep = np.flatnonzero(gaps > 1e-3 * sq)
    assert sep.size > n // 4
    assert np.abs(U1[:, sep] - U2[:, sep]).max() <= vbar
    assert np.abs(V1[:, sep] - V2[:, sep]).max() <= vbar
