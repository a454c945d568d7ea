"""Batched left inverse over uneven independent instances (one CUDA graph per apply).

Instances follow the batched recipe (square periodic grids of side 32..192, 4-24 levels,
K in [16, 64] so that n_w > K occurs, 1-32 right-hand sides, mixed precision).  Every
instance's output must match the FP64 oracle applied to that instance alone (mixed
tolerance 1e-5, whichever kernel variant the autotuner picked), a replay of the captured
graph must reproduce the same bits, new buffers must trigger a new capture with the same
results, and instances with no right-hand sides are skipped.
"""

import numpy as np
import pytest

from oracle import basis, compare, swift
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def zl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_13327_b300 import zl as mod
    return mod


def instances(count):
    ws = synth.batched_instances()
    # the first instances plus every instance with n_w > K among the first 60
    pick = list(range(count)) + [i for i, w in enumerate(ws[:60]) if w.nw > w.K and i >= count]
    return [ws[i] for i in pick]


@pytest.fixture(scope="module")
def batch(zl):
    ws = instances(10)
    Zs = [synth.ensemble(w).astype(np.float32) for w in ws]
    lams = [basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc) for w in ws]
    b = zl.zl_setup_batch([{"Z": torch.from_numpy(Z).cuda(), "spectrum": lam, "nx": w.Nx, "ny": w.Ny, "prec": "mixed",
                            "tau": w.tau, "max_rhs": w.R} for w, Z, lam in zip(ws, Zs, lams)])
    oracles = [swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau) for w, Z, lam in zip(ws, Zs, lams)]
    xs = [synth.rhs(w, dtype=np.float32) for w in ws]
    return b, ws, oracles, xs


def test_batch_matches_oracle_per_instance(zl, batch):
    b, ws, oracles, xs = batch
    assert any(w.nw > w.K for w in ws)
    assert all(0 <= v <= 5 for v in b.variants)
    outs = b.apply_left_inverse([torch.from_numpy(x).cuda() for x in xs])
    torch.cuda.synchronize()
    for i, (w, o, x) in enumerate(zip(ws, outs, xs)):
        assert b.plans[i].device_error() == 0
        ref = swift.apply_left_inverse(oracles[i], x.astype(np.float64))
        compare.check(o.cpu().numpy(), ref, TOL_MIXED, 2, f"instance {i} {w} variant {b.variants[i]}")


def test_graph_replay_and_recapture(zl, batch):
    b, ws, oracles, xs = batch
    xg = [torch.from_numpy(x).cuda() for x in xs]
    outs = [torch.empty((x.shape[0], p.K, p.L), device="cuda") for x, p in zip(xg, b.plans)]
    first = [o.clone() for o in b.apply_left_inverse(xg, outs)]
    for o in outs:
        o.fill_(float("nan"))
    b.apply_left_inverse(xg, outs)                                # replay of the captured graph
    assert all(torch.equal(a, c) for a, c in zip(first, outs))
    xg2 = [x.clone() for x in xg]                                 # new buffers: a new capture
    outs2 = b.apply_left_inverse(xg2)
    assert all(torch.equal(a, c) for a, c in zip(first, outs2))


def test_instances_without_rhs_are_skipped(zl, batch):
    b, ws, oracles, xs = batch
    xg = [torch.from_numpy(x).cuda() for x in xs]
    xg[1] = xg[1][:0]
    xg[3] = xg[3][:0]
    outs = b.apply_left_inverse(xg)
    torch.cuda.synchronize()
    assert outs[1].shape[0] == 0 and outs[3].shape[0] == 0
    ref = swift.apply_left_inverse(oracles[2], xs[2].astype(np.float64))
    compare.check(outs[2].cpu().numpy(), ref, TOL_MIXED, 2, "instance 2")


def test_each_plan_alone_equals_the_batch(zl, batch):
    """The batch's plans are ordinary plans: applied alone they give the batch's result."""
    b, ws, oracles, xs = batch
    xg = [torch.from_numpy(x).cuda() for x in xs]
    outs = b.apply_left_inverse(xg)
    for i in (0, 4):
        alone = zl.zl_apply_left_inverse(b.plans[i], xg[i])
        assert torch.equal(alone, outs[i])
