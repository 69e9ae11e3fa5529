"""The serving engine (svdup_server_*): resident SVDs, a continuous stream of rank-one
updates, admission by free lanes and a free-HBM ledger.

Each request runs the same kernels on the same inputs as a lone svdup_update, and the
updates of one matrix apply in submission order, so every matrix must end bit-identical
to applying its updates alone, one after another: the tests compare with
torch.equal while requests for different matrices overlap on the device."""
import numpy as np
import pytest

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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


SHAPES = [(40, 60), (100, 100), (300, 300), (200, 350), (620, 700)]


def _mats(seed):
    g = np.random.default_rng(seed)
    out = []
    for m, n in SHAPES:
        U, S, Vh = np.linalg.svd(g.standard_normal((m, n)))
        out.append((U, S, np.asfortranarray(Vh.T)))
    return out


def _requests(count, seed):
    g = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        i = int(g.integers(len(SHAPES)))
        m, n = SHAPES[i]
        reqs.append((i, g.standard_normal(m), g.standard_normal(n)))
    return reqs


def _lone(sv, mats, reqs, mode):
    h = sv.Handle(0)
    res = [(devF(U), dev(S), devF(V)) for U, S, V in mats]
    for i, a, b in reqs:
        U, S, V = res[i]
        h.update(U, S, V, dev(a), dev(b), eps=1e-12, mode=mode)
    h.close()
    return res


@pytest.mark.parametrize("mode_name,lanes,budget,group", [
    ("FP64", 4, 0, 1), ("MIXED_BF16X3", 3, 0, 1), ("FP64", 4, "one", 1),
    ("FP64", 2, 0, 4), ("MIXED_BF16X3", 2, 0, 8), ("MIXED_FP16X2", 3, "one", 4)])
def test_server_matches_lone_updates(sv, mode_name, lanes, budget, group):
    """group > 1: a lane takes up to `group` requests of one size class per cycle; the
    results must still equal lone updates in submission order."""
    mode = getattr(sv, mode_name)
    mats = _mats(11)
    reqs = _requests(36, 12)
    ref = _lone(sv, mats, reqs, mode)
    if budget == "one":  # room for the largest update's workspace only
        h = sv.Handle(0)
        budget = max(h.update_workspace(m, n, 1e-12, mode) for m, n in SHAPES)
        h.close()
    srv = sv.Server(0, lanes=lanes, hbm_budget=budget, eps=1e-12, mode=mode)
    srv.set_group(group)
    live = [(devF(U), dev(S), devF(V)) for U, S, V in mats]
    ids = [srv.register(U, S, V) for U, S, V in live]
    tickets = [srv.submit(ids[i], a, b) for i, a, b in reqs]
    for t in tickets:
        st, lat = srv.wait(t)
        assert st == sv.OK and lat > 0.0
    stats = srv.stats()
    gs = srv.group_stats()
    srv.close()
    assert gs["grouped"] == len(reqs) and gs["max_group"] <= group
    if group > 1:
        assert gs["max_group"] >= 2  # requests of one size class shared a lane cycle
    assert stats["completed"] == len(reqs)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0.0
    if budget:
        assert stats["max_ws_bytes"] <= budget
    else:
        assert stats["max_in_flight"] >= 2  # different matrices overlapped on the device
    for (U1, S1, V1), (U2, S2, V2) in zip(ref, live):
        assert torch.equal(S1, S2) and torch.equal(U1, U2) and torch.equal(V1, V2)


def test_server_rejects_bad_requests(sv):
    srv = sv.Server(0, lanes=2)
    U, S, V = _mats(3)[0]
    mid = srv.register(devF(U), dev(S), devF(V))
    with pytest.raises(sv.SvdupError):
        srv.submit(mid + 5, np.ones(40), np.ones(60))
    st, _ = srv.wait(srv.submit(mid, np.ones(40), np.ones(60)))
    assert st == sv.OK
    srv.close()
