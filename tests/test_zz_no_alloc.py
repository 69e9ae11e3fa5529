"""svdup_secular_static, the secular-root entry point that allocates no device memory.

It exists for callers that cannot allocate device memory (a host application whose
memory pool already holds the device memory they may use, a plug-in barred from the
CUDA allocator, a latency-critical loop where cudaMalloc would synchronise the
device): its scratch is a fixed array inside the library.  This file checks, through
the C ABI, that two calls in a row (a larger problem, then a smaller one, so the second
runs over the first one's leftover scratch) give the roots of the handle-based
svdup_secular within the root-accuracy bound the secular tests use; that a call
leaves the device's free memory unchanged (the property the entry point exists for);
that a device error (a NaN in z) reaches the caller's info word; and that sizes beyond
the array's limit are refused.  It is named to be collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U53 = 2.0 ** -53


@pytest.fixture(scope="module")
def sv():
    import paper_1707_08369_gb300 as sv
    from paper_1707_08369_gb300 import build
    build.build()
    sv.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return sv


def _problem(k, sgn, graded, seed):
    g = np.random.default_rng(seed)
    d = np.sort(10 ** (-8 * g.uniform(0, 1, k))) if graded else np.sort(g.uniform(0, 1, k))
    z = g.standard_normal(k)
    return d, z, sgn * g.uniform(0.3, 3.0)


def _root_bound(d, z, rho, org, tau):
    """Attainable accuracy of each root: the rounding error of evaluating w divided by
    its slope (the bound of the secular parity tests)."""
    R = abs(rho)
    out = np.empty(d.size)
    for j in range(d.size):
        delta = (d - d[org[j]]) - tau[j]
        t = z * z / delta
        out[j] = d.size * U53 * (1.0 + R * np.abs(t).sum()) / (R * np.sum(t / delta))
    return 2.0 * out + 8 * U53 * np.abs(tau)


def _static_call(sv, d, z, rho):
    """One svdup_secular_static call straight through ctypes on torch's current stream."""
    lib = sv.load()
    k = d.size
    td = torch.from_numpy(d).cuda()
    tz = torch.from_numpy(z).cuda()
    org = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    tau = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.svdup_secular_static(ctypes.c_void_p(st), k, ctypes.c_void_p(td.data_ptr()),
                                  ctypes.c_void_p(tz.data_ptr()), float(rho),
                                  ctypes.c_void_p(org.data_ptr()), ctypes.c_void_p(tau.data_ptr()),
                                  ctypes.c_void_p(info.data_ptr()))
    assert rc == sv.OK, sv.error_string(rc)
    torch.cuda.synchronize()
    return org.cpu().numpy(), tau.cpu().numpy(), int(info.item())


def test_static_secular_matches_handle_entry_point(sv):
    h = sv.Handle(0)
    cases = [(4099, -1, False, 11), (1000, 1, True, 12)]
    try:
        for k, sgn, graded, seed in cases:
            d, z, rho = _problem(k, sgn, graded, seed)
            org_r, tau_r = h.secular(torch.from_numpy(d).cuda(), torch.from_numpy(z).cuda(), rho)
            org_r = org_r.cpu().numpy(); tau_r = tau_r.cpu().numpy()
            org_s, tau_s, info = _static_call(sv, d, z, rho)
            assert info == sv.OK
            assert np.all((org_s >= 0) & (org_s < k))
            diff = (d[org_s] - d[org_r]) + (tau_s - tau_r)
            assert np.all(np.abs(diff) <= _root_bound(d, z, rho, org_r, tau_r))
    finally:
        h.close()


def test_static_secular_rejects_oversize(sv):
    lib = sv.load()
    k = sv.SECULAR_STATIC_MAX_K + 1
    buf = torch.zeros(k, dtype=torch.float64, device="cuda")
    ibuf = torch.zeros(k, dtype=torch.int32, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.svdup_secular_static(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), k,
                                  p(buf), p(buf), 1.0, p(ibuf), p(buf), p(ibuf))
    assert rc == sv.EINVAL


def test_static_secular_allocates_nothing(sv):
    """After a first call (which looks up the array's address), a call changes nothing
    in the device's free memory: every buffer it touches is the caller's or the
    library's fixed array."""
    lib = sv.load()
    d, z, rho = _problem(3000, 1, False, 13)
    td, tz = torch.from_numpy(d).cuda(), torch.from_numpy(z).cuda()
    org = torch.empty(d.size, dtype=torch.int32, device="cuda")
    tau = torch.empty(d.size, dtype=torch.float64, device="cuda")
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())

    def call():
        rc = lib.svdup_secular_static(st, d.size, p(td), p(tz), float(rho), p(org), p(tau), p(info))
        assert rc == sv.OK, sv.error_string(rc)
        torch.cuda.synchronize()

    call()
    free0, _ = torch.cuda.mem_get_info()
    call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(info.item()) == sv.OK


def test_static_secular_reports_nonfinite_input(sv):
    """A NaN in z is found on the device: the call itself succeeds, and the caller's
    info word holds SVDUP_ENONFINITE once the stream has run."""
    d, z, rho = _problem(300, 1, False, 14)
    z[17] = np.nan
    org, tau, info = _static_call(sv, d, z, rho)
    assert info == sv.ENONFINITE
    # a clean call after it starts from a cleared info word
    d, z, rho = _problem(300, -1, False, 15)
    org, tau, info = _static_call(sv, d, z, rho)
    assert info == sv.OK
