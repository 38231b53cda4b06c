"""Batches of heterogeneous simulations in one persistent launch per phase
(CUDA-graph replay): every simulation's outputs equal its standalone run."""
import numpy as np
import pytest

from paper_2108_12369_gb300 import workloads as W
from tests.parity import compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12369_gb300 import build, pct as P
    build.build()
    return P


def _instances():
    ws = W.batch_instances(count=7, max_paths=24000)
    ws.append(W.neo1_2d_straight(n_angles=20, paths_per_angle=333))
    ws.append(W.head_3d_spline(n_angles=5, paths_per_angle=401, n=(40, 36, 30), h=(5.0, 5.5, 5.0)))
    return ws


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_equals_standalone_runs(pct, autotune):
    ws = _instances()
    assert {w["phantom"]["dim"] for w in ws} == {2, 3}
    batch = pct.Batch(ws, autotune=autotune)
    t = batch.params()
    assert t["order"] in (0, 1) and t["fill_prefetch"] in (0, 1)
    assert all(r in (64, 128, 256) for r in t["rows_per_item"]) and all(g in (1, 2) for g in t["grid_mult"])
    for rep in range(2):  # graph replay (the first fill tunes the fill's shape when asked)
        batch.count()
        outs = batch.fill()
        if autotune and rep == 0:
            t1 = batch.params()
            assert t1["rows_per_item"][:2] == t["rows_per_item"][:2] and t1["order"] == t["order"]
        torch.cuda.synchronize()
        for w, o in zip(ws, outs):
            ref = pct.simulate(pct.Phantom(w["phantom"]), pct.GeometryArgs(w), pct.PREC_MIXED)
            torch.cuda.synchronize()
            for k in ("row_ptr", "col", "val", "b", "x_true"):
                assert torch.equal(o[k], ref[k]), (w["name"], k)


def test_batch_member_matches_oracle(pct, orc):
    w = W.head_3d_spline(n_angles=4, paths_per_angle=250, n=(48, 48, 40), h=(4.0, 4.0, 4.0))
    batch = pct.Batch([W.neo1_2d_straight(n_angles=4, paths_per_angle=100), w])
    batch.count()
    out = batch.fill()[1]
    torch.cuda.synchronize()
    ref = orc.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"], threads=8)
    compare(out, ref)


@pytest.mark.parametrize("share", [0.0, 0.5, 1.0])
def test_batch_with_both_forms(pct, share):
    """PCT_BATCH_LEAN with workspace beyond the all-lean size: the largest
    instances keep the full form (their fills run as full-form launches, the
    rest as lean ones); every output equals its standalone run bit for bit."""
    ws = _instances()
    lean_min = pct.batch_workspace_size(ws, lean=True)
    full = pct.batch_workspace_size(ws)
    assert full > lean_min
    batch = pct.Batch(ws, autotune=True, lean=True, workspace_bytes=lean_min + int(share * (full - lean_min)))
    for rep in range(2):
        batch.count()
        outs = batch.fill()
        torch.cuda.synchronize()
        for w, o in zip(ws, outs):
            ref = pct.simulate(pct.Phantom(w["phantom"]), pct.GeometryArgs(w), pct.PREC_MIXED)
            torch.cuda.synchronize()
            for k in ("row_ptr", "col", "val", "b", "x_true"):
                assert torch.equal(o[k], ref[k]), (w["name"], k, share)
