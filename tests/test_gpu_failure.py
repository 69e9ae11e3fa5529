"""Failure handling on the GPU without a fault: the tensor-core pipeline's bounded
waits.  svdup_check_timeout runs a mixed Cauchy product whose drains never hand a
tensor-memory region back (a release that nothing performs) with a 1 ms wait limit; the
MMA issuer's wait runs out, every CTA waits for its own MMAs and bulk copies, frees its
tensor memory and exits, and SVDUP_ETIMEOUT reaches the host at the next sync.  The
same handle then computes a correct product: the context stays usable."""
import ctypes

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


def devF(x):
    return torch.from_numpy(np.asfortranarray(x).T.copy()).cuda().t()


# far field on (leaves of 128: seven K tiles per output item); dense (five leaves of 64):
# both with more K tiles per CTA than the three K-tile accumulators, so the MMA issuer waits for
# a region that the stalled drains never release
@pytest.mark.parametrize("rows,N", [(300, 2600), (130, 300)])
def test_pipeline_timeout_is_reported_and_recoverable(sv, orc, rows, N):
    g = np.random.default_rng(41)
    d = g.uniform(0, 1, N)
    z = g.standard_normal(N)
    rho = 1.3
    X = wl.haar(max(rows, N), g)[:rows, :N]
    h = sv.Handle(0)
    try:
        tX, td, tz = devF(X), torch.from_numpy(d).cuda(), torch.from_numpy(z).cuda()
        Y = torch.zeros((N, rows), dtype=torch.float64, device="cuda").t()
        lam = torch.zeros(N, dtype=torch.float64, device="cuda")
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        rc = sv.load().svdup_check_timeout(h._h, rows, N, p(tX), rows, p(td), p(tz), rho, p(Y),
                                           rows, p(lam))
        assert rc == sv.OK
        assert h.sync() == sv.ETIMEOUT
        assert h.sync() == sv.OK  # the status word was cleared by the sync
        lam_o, Y_o = orc.rank_one_update_z(X, d, z, rho)
        lam_g, Y_g = h.cauchy_product(devF(X), td, tz, rho, eps=1e-12, mode=sv.MIXED_BF16X3)
        assert np.abs(Y_g.cpu().numpy() - Y_o).max() <= 2e-6
    finally:
        h.close()
