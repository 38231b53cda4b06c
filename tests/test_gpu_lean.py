"""The lean mixed form (PCT_PREC_MIXED_LEAN): the count keeps no segment
records, the fill sets each row's segments up again with the count's own
code.  Its output must equal the mixed form's bit for bit -- row pointers,
indices, values and WEPL -- on regular rows, on rows the cooperative form
hands to the per-lane walker (near-degenerate segments of axis-aligned and
lattice-diagonal rays, rows beyond the cooperative limits), through the host-memory fill, and
inside a lean batch; and it needs a fraction of the workspace."""
import math

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


def _axis_aligned():
    w = W.neo1_2d_straight(n_angles=4, paths_per_angle=700)
    w["angles"] = np.array([0.0, math.pi / 2, math.pi / 4, 3 * math.pi / 4])
    w["model"] = W.model(W.STRAIGHT, (-130.0, 130.0))
    return w


CASES = {
    "neo2": lambda: W.neo2_2d_spline(n_angles=18, paths_per_angle=301, n=512, h=0.4),
    "head3d": lambda: W.head_3d_spline(n_angles=7, paths_per_angle=333, n=(100, 100, 80), h=(2.0, 2.0, 2.0)),
    "axis_aligned": _axis_aligned,
    "beyond_coop": lambda: W.neo2_2d_spline(n_angles=4, paths_per_angle=60, n=512, h=0.4, spline_segments=70),
    "highland_3d": lambda: dict(W.head_3d_spline(n_angles=3, paths_per_angle=500, n=(64, 64, 50), h=(3.2, 3.2, 3.2)),
                                model=W.model(W.SPLINE, (-102.4, 102.4), (-80.0, 80.0), sigma_in=0.01,
                                              mcs=W.MCS_HIGHLAND, noise_rel=0.01)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_lean_equals_mixed(pct, case):
    w = CASES[case]()
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    a = pct.simulate(ph, geo, pct.PREC_MIXED)
    b = pct.simulate(ph, geo, pct.PREC_MIXED_LEAN)
    torch.cuda.synchronize()
    for k in ("row_ptr", "col", "val", "b", "x_true"):
        assert torch.equal(a[k], b[k]), k
    assert b["workspace"].numel() < a["workspace"].numel()
    if w["model"]["model"] == W.SPLINE:  # 34+ segment records per row dropped
        assert b["workspace"].numel() < 0.3 * a["workspace"].numel()


def test_lean_matches_oracle(pct, orc):
    w = CASES["head3d"]()
    g = pct.simulate(pct.Phantom(w["phantom"]), pct.GeometryArgs(w), pct.PREC_MIXED_LEAN)
    torch.cuda.synchronize()
    ref = orc.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"], threads=8)
    compare(g, ref)


def test_lean_host_fill_and_projectors(pct):
    w = CASES["neo2"]()
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    ref = pct.simulate(ph, geo, pct.PREC_MIXED)
    ws = torch.empty(pct.simulate_workspace_size(ph, geo, pct.PREC_MIXED_LEAN), dtype=torch.uint8, device="cuda")
    x = torch.empty(ph.nvox, dtype=torch.float32, device="cuda")
    rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, device="cuda")
    pct.phantom_rasterize(ph, x)
    pct.simulate_count(ph, geo, pct.PREC_MIXED_LEAN, ws, rp)
    nnz = int(rp[-1])
    h_rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, pin_memory=True)
    h_col = torch.empty(nnz, dtype=torch.int32, pin_memory=True)
    h_val = torch.empty(nnz, dtype=torch.float32, pin_memory=True)
    h_b = torch.empty(geo.n_rows, dtype=torch.float32, pin_memory=True)
    staging = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    pct.simulate_fill_host(ph, geo, pct.PREC_MIXED_LEAN, ws, rp, x, staging, h_rp, h_col, h_val, h_b)
    assert torch.equal(h_col, ref["col"].cpu()) and torch.equal(h_val, ref["val"].cpu())
    assert torch.equal(h_b, ref["b"].cpu())
    # matrix-free forward in the lean form equals the mixed form's
    n = geo.n_rows
    pw = torch.empty(pct.projector_workspace_size(ph, geo, n, pct.PREC_MIXED_LEAN), dtype=torch.uint8, device="cuda")
    y1 = torch.empty(n, dtype=torch.float32, device="cuda")
    y2 = torch.empty(n, dtype=torch.float32, device="cuda")
    pct.forward(ph, geo, None, 0, n, x, y1, pw, precision=pct.PREC_MIXED_LEAN)
    pw2 = torch.empty(pct.projector_workspace_size(ph, geo, n, pct.PREC_MIXED), dtype=torch.uint8, device="cuda")
    pct.forward(ph, geo, None, 0, n, x, y2, pw2, precision=pct.PREC_MIXED)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


def test_lean_batch_equals_standalone(pct):
    ws = W.batch_instances(count=6, max_paths=20000)
    ws.append(W.head_3d_spline(n_angles=3, paths_per_angle=401, n=(40, 36, 30), h=(5.0, 5.5, 5.0)))
    batch = pct.Batch(ws, lean=True, autotune=True)
    assert pct.batch_workspace_size(ws, lean=True) < 0.3 * pct.batch_workspace_size(ws)
    for _ in range(2):
        batch.count()
        outs = batch.fill()
        torch.cuda.synchronize()
        for w, o in zip(ws, outs):
            ref = pct.simulate(pct.Phantom(w["phantom"]), pct.GeometryArgs(w), pct.PREC_MIXED)
            torch.cuda.synchronize()
            for k in ("row_ptr", "col", "val", "b", "x_true"):
                assert torch.equal(o[k], ref[k]), (w["name"], k)
