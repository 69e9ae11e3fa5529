"""Batches of independent updates (svdup_batch_create / svdup_batch_launch /
svdup_update_batched) and the product-path autotuner, through the C ABI.

Every member of a batch runs the same kernels on the same inputs as when it runs
alone, only on another stream with its own workspace, so its results must be
bit-identical to a lone svdup_update: the tests compare with np.array_equal.  Sizes
are drawn log-uniform like the batched workload (n from 8 to 700 here, so the oracle
and the lone runs stay quick)."""
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _problems(count, seed, rect=False):
    g = np.random.default_rng(seed)
    ns = np.round(8 * (700 / 8) ** g.uniform(0, 1, count)).astype(int)
    out = []
    for n in ns:
        m = int(n if not rect else max(1, int(n * g.uniform(0.5, 1.0))))
        A = g.standard_normal((m, int(n)))
        U, S, Vh = np.linalg.svd(A)
        out.append((U, S, np.asfortranarray(Vh.T), g.standard_normal(m), g.standard_normal(int(n))))
    return out


def _to_dev(probs):
    return [(devF(U), dev(S), devF(V), dev(a), dev(b)) for U, S, V, a, b in probs]


@pytest.mark.parametrize("mode_name,rect", [("FP64", False), ("MIXED_BF16X3", True)])
def test_batch_graph_matches_lone_updates(sv, mode_name, rect):
    mode = getattr(sv, mode_name)
    probs = _problems(24, 5 if rect else 4, rect)
    h = sv.Handle(0)
    lone = _to_dev(probs)
    for U, S, V, a, b in lone:
        h.update(U, S, V, a, b, eps=1e-12, mode=mode)
    mix = _to_dev(probs)
    bt = h.batch_plan(mix, eps=1e-12, mode=mode, lanes=6)
    assert bt.kernels() > 0
    bt.launch()
    for (U1, S1, V1, _, _), (U2, S2, V2, _, _) in zip(lone, mix):
        assert torch.equal(S1, S2) and torch.equal(U1, U2) and torch.equal(V1, V2)
    # a second launch applies the same rank-one terms again: chained updates
    for U, S, V, a, b in lone:
        h.update(U, S, V, a, b, eps=1e-12, mode=mode)
    bt.launch()
    for (U1, S1, V1, _, _), (U2, S2, V2, _, _) in zip(lone, mix):
        assert torch.equal(S1, S2) and torch.equal(U1, U2) and torch.equal(V1, V2)
    bt.close()
    h.close()


def test_batch_results_against_oracle(sv, orc):
    probs = _problems(10, 7)
    h = sv.Handle(0)
    items = _to_dev(probs)
    h.update_batched(items, eps=1e-12, mode=sv.FP64, lanes=4)
    for (U, S, V, a, b), (tU, tS, tV, _, _) in zip(probs, items):
        Uo, So, Vo = orc.svd_update(U, S, V, a, b)
        assert np.abs(tS.cpu().numpy() - So).max() <= 1e-12 * So[0]
    h.close()


def test_batch_rejects_bad_problem(sv):
    h = sv.Handle(0)
    items = _to_dev(_problems(3, 8))
    U, S, V, a, b = items[1]
    items[1] = (U, S, V, a, dev(np.ones(S.numel() + 1)))  # b longer than V: n changes, V wrong
    with pytest.raises((sv.SvdupError, ValueError)):
        h.batch_plan(items)
    h.close()


def test_autotune_and_tuning_roundtrip(sv):
    h = sv.Handle(0)
    dmax, l128 = h.autotune(sv.MIXED_BF16X3, nmax=1024)
    assert 0 <= dmax <= 1024 and l128 >= 1
    h.set_tuning(sv.FP64, 300, 5000)
    assert h.tuning(sv.FP64) == (300, 5000)
    assert h.tuning(sv.MIXED_BF16X3) == (dmax, l128)
    h.close()
