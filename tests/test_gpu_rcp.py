"""The library's own FP64 reciprocal and reciprocal square root (rcp64, rsqrt64: an FP32
seed of the significand, the exponent by bit fields, two FP64 Newton steps), which its
FP64 kernels use in place of division and sqrt, held against CUDA's division (IEEE,
correctly rounded, bit-equal to the host's) and square root over every exponent band,
both signs, and the fallback edges.  Stated bounds: rcp64 within 1 ulp of the correctly
rounded 1/x, rsqrt64 within 2 ulp of 1/sqrt(x) taken in extended precision, and the
fallback inputs (zero, subnormal, the largest binades, inf, NaN) bit-equal to CUDA's."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1707_08369_gb300 as sv
    from paper_1707_08369_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return sv.load()


def _run(lib, x):
    tx = torch.from_numpy(x).cuda()
    r = torch.empty_like(tx)
    rs = torch.empty_like(tx)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.svdup_check_rcp(st, x.size, p(tx), p(r), p(rs)) == 0
    torch.cuda.synchronize()
    return tx, r.cpu().numpy(), rs.cpu().numpy()


def _inputs():
    g = np.random.default_rng(5)
    e = np.arange(-1022, 1024)
    m = 1.0 + g.uniform(0, 1, (e.size, 6))
    m[:, 0] = 1.0                                  # powers of two
    m[:, 1] = np.nextafter(2.0, 0.0)               # just below the next power
    m[:, 2] = np.nextafter(1.0, 2.0)               # just above
    x = np.ldexp(m, e[:, None]).ravel()
    return x[np.isfinite(x) & (x > 0)]


def test_rcp64_every_binade(lib):
    x = _inputs()
    x = np.concatenate([x, -x])
    _, r, _ = _run(lib, x)
    want = 1.0 / x                                  # IEEE division: correctly rounded
    ulp = np.abs(r - want) / np.spacing(np.abs(want))
    ok = np.isfinite(want) & (np.abs(want) >= np.finfo(np.float64).tiny)
    assert ulp[ok].max() <= 1.0, ulp[ok].max()
    # the subnormal results (the largest binades) come from CUDA's division: exact
    assert np.array_equal(r[~ok], want[~ok])


def test_rsqrt64_every_binade(lib):
    x = _inputs()
    tx, _, rs = _run(lib, x)
    ref = (1 / np.sqrt(x.astype(np.longdouble))).astype(np.float64)
    ulp = np.abs(rs - ref) / np.spacing(ref)
    assert ulp.max() <= 2.0, ulp.max()
    cuda = torch.rsqrt(tx).cpu().numpy()  # CUDA's own rsqrt, for comparison
    assert (np.abs(cuda - ref) / np.spacing(ref)).max() <= 2.0


def test_fallback_edges_match_cuda(lib):
    tiny = np.finfo(np.float64).tiny
    x = np.array([0.0, -0.0, 5e-324, tiny / 3, -tiny / 7, np.inf, -np.inf, np.nan,
                  np.finfo(np.float64).max, 2.0 ** 1022 * 1.5, 2.0 ** 1021 * 1.9, tiny])
    tx, r, rs = _run(lib, x)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        want = 1.0 / x
    assert np.array_equal(r, want, equal_nan=True)
    cuda_rs = (1.0 / torch.sqrt(tx)).cpu().numpy()
    fb = ~(x > 0) | ~np.isfinite(x) | (x < tiny)   # inputs that take the fallback
    assert np.array_equal(rs[fb], cuda_rs[fb], equal_nan=True)
