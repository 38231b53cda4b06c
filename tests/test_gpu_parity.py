"""GPU parity: libpct (through the C ABI) against the CPU oracle on the same
seeded inputs.  Indices and row pointers bit-exact; values and WEPL within
1e-6 relative per row (the all-FP64 form is checked to be bit-identical)."""
import math

import numpy as np
import pytest

from paper_2108_12369_gb300 import workloads as W
from tests.parity import compare, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12369_gb300 import build, pct as P
    build.build()
    return P


PRECS = ["f64", "mixed"]


def _prec(pct, name):
    return {"f64": pct.PREC_F64, "mixed": pct.PREC_MIXED}[name]


def run_gpu(pct, w, prec):
    ph = pct.Phantom(w["phantom"])
    geo = pct.GeometryArgs(w)
    try:
        out = pct.simulate(ph, geo, _prec(pct, prec))
    except pct.PctError as e:
        if e.status == pct.EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    torch.cuda.synchronize()
    return out


def run_oracle(orc, w, rows=None, threads=8):
    return orc.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"],
                        rows=rows, threads=threads)


@pytest.mark.parametrize("desc", [
    W.phantom(2, (200, 200), (1.0, 1.0), skin=False),
    W.phantom(2, (512, 512), (0.4, 0.4), skin=True),
    W.phantom(2, (200, 160), (1.0, 1.0), skin=True, raster=W.CENTER),
    W.phantom(3, (60, 60, 48), (3.3, 3.3, 3.4), skin=False),
    W.phantom(3, (40, 40, 32), (5.0, 5.0, 5.0), skin=True, kind=W.EXTRUDED, raster=W.CENTER),
    W.phantom(2, (200, 160), (1.0, 1.0), skin=True, raster=W.AREA, area_samples=8),
    W.phantom(2, (96, 96), (2.0, 2.0), skin=False, raster=W.AREA, area_samples=5),
    W.phantom(3, (50, 50, 40), (4.0, 4.0, 4.0), skin=True, raster=W.AREA, area_samples=3),
    W.phantom(3, (40, 40, 32), (5.0, 5.0, 5.0), skin=False, kind=W.EXTRUDED, raster=W.AREA, area_samples=4),
])
def test_raster_bit_exact(pct, orc, desc):
    ph = pct.Phantom(desc)
    x = torch.empty(ph.nvox, dtype=torch.float32, device="cuda")
    pct.phantom_rasterize(ph, x)
    torch.cuda.synchronize()
    want = orc.Phantom(desc).raster().astype(np.float32)
    assert np.array_equal(to_np(x), want)


@pytest.mark.parametrize("prec", PRECS)
def test_neo1_straight_full(pct, orc, prec):
    """NEO 1, 200x200 px, 180 angles x 500 straight paths: every row."""
    w = W.neo1_2d_straight()
    g = run_gpu(pct, w, prec)
    ref = run_oracle(orc, w)
    st = compare(g, ref, exact_values=(prec == "f64"))
    assert g["nnz"] == ref["row_ptr"][-1] > 10_000_000
    print(prec, st)


@pytest.mark.parametrize("prec", PRECS)
def test_neo2_spline_reduced(pct, orc, prec):
    """NEO 2 on 512x512 px of 0.4 mm, spline paths with MCS and 1% noise,
    36 angles x 300 protons (several thread blocks, ragged tail)."""
    w = W.neo2_2d_spline(n_angles=36, paths_per_angle=301)
    g = run_gpu(pct, w, prec)
    ref = run_oracle(orc, w)
    st = compare(g, ref, exact_values=(prec == "f64"))
    print(prec, st)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("model", [W.STRAIGHT_MCS, W.SPLINE])
def test_head_3d_reduced(pct, orc, prec, model):
    w = W.head_3d_spline(n_angles=9, paths_per_angle=333, n=(100, 100, 80), h=(2.0, 2.0, 2.0))
    w["model"] = dict(w["model"], model=model, rho=0.3)
    g = run_gpu(pct, w, prec)
    ref = run_oracle(orc, w)
    st = compare(g, ref, exact_values=(prec == "f64"))
    print(prec, model, st)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["neo2_spline", "head_3d_straight_mcs"])
def test_highland_widths(pct, orc, prec, case):
    """Exit widths from the Highland / PDG formula per proton (Sec. II-B),
    200 MeV in water; the FP64 form bit for bit, the mixed form within 1e-6."""
    if case == "neo2_spline":
        w = W.neo2_2d_spline(n_angles=24, paths_per_angle=301, n=256, h=0.8)
        w["model"] = dict(w["model"], mcs=W.MCS_HIGHLAND, beam_mev=200.0, x0_mm=W.X0_WATER_MM)
    else:
        w = W.head_3d_spline(n_angles=7, paths_per_angle=333, n=(100, 100, 80), h=(2.0, 2.0, 2.0))
        w["model"] = dict(w["model"], model=W.STRAIGHT_MCS, mcs=W.MCS_HIGHLAND, beam_mev=150.0)
    g = run_gpu(pct, w, prec)
    ref = run_oracle(orc, w)
    st = compare(g, ref, exact_values=(prec == "f64"))
    print(prec, case, st)


@pytest.mark.parametrize("prec", PRECS)
def test_area_raster_simulation(pct, orc, prec):
    """A weighted-area phantom (Sec. II-A): x_true and the WEPL built on it."""
    w = W.neo2_2d_spline(n_angles=12, paths_per_angle=200, n=200, h=1.0)
    w["phantom"] = W.phantom(2, (200, 160), (1.0, 1.0), skin=True, raster=W.AREA, area_samples=6)
    g = run_gpu(pct, w, prec)
    ref = run_oracle(orc, w)
    assert np.array_equal(to_np(g["x_true"]), ref["x_true"])
    compare(g, ref, exact_values=(prec == "f64"))


@pytest.mark.parametrize("prec", PRECS)
def test_extruded_and_constant_chord(pct, orc, prec):
    w = W.head_3d_spline(n_angles=5, paths_per_angle=200, n=(64, 64, 40), h=(3.0, 3.0, 4.0))
    w["phantom"] = dict(w["phantom"], kind=W.EXTRUDED)
    w["model"] = dict(w["model"], chord=W.CHORD_CONSTANT)
    g = run_gpu(pct, w, prec)
    ref = run_oracle(orc, w)
    assert np.all(to_np(g["val"]) == np.float32(3.0))
    compare(g, ref, exact_values=(prec == "f64"))


@pytest.mark.parametrize("prec", PRECS)
def test_axis_aligned_angles_and_grid_edges(pct, orc, prec):
    """Angles 0, 90, 180, 270 degrees put straight paths along grid lines (an
    axis with no or nearly no extent: inert, or a segment the walker takes);
    45 and 135 degrees send them near lattice corners (near-ties the FP64
    definition decides); offsets span beyond the grid."""
    w = W.neo1_2d_straight(n_angles=4, paths_per_angle=2000)
    w["angles"] = np.array([0.0, math.pi / 2, math.pi, 1.5 * math.pi])
    w["model"] = W.model(W.STRAIGHT, (-130.0, 130.0))
    g = run_gpu(pct, w, prec)
    ref = run_oracle(orc, w)
    compare(g, ref, exact_values=(prec == "f64"))
    # diagonal angles through corners: 45 degrees with offsets on the lattice
    w["angles"] = np.array([math.pi / 4, 3 * math.pi / 4])
    w["paths_per_angle"] = 500
    g = run_gpu(pct, w, prec)
    ref = run_oracle(orc, w)
    compare(g, ref, exact_values=(prec == "f64"))


@pytest.mark.parametrize("prec", PRECS)
def test_empty_and_missing_rows(pct, orc, prec):
    w = W.neo1_2d_straight(n_angles=0, paths_per_angle=100)
    g = run_gpu(pct, w, prec)
    assert g["nnz"] == 0 and to_np(g["row_ptr"]).tolist() == [0]
    w = W.neo1_2d_straight(n_angles=3, paths_per_angle=0)
    g = run_gpu(pct, w, prec)
    assert g["nnz"] == 0 and to_np(g["row_ptr"]).tolist() == [0]
    w = W.neo1_2d_straight(n_angles=5, paths_per_angle=77)
    w["model"] = W.model(W.STRAIGHT, (150.0, 170.0))  # beyond the grid's half-diagonal
    g = run_gpu(pct, w, prec)
    assert g["nnz"] == 0 and np.all(to_np(g["b"]) == 0)
    w = W.neo1_2d_straight(n_angles=1, paths_per_angle=1)
    g = run_gpu(pct, w, prec)
    compare(g, run_oracle(orc, w), exact_values=(prec == "f64"))


@pytest.mark.parametrize("prec", PRECS)
def test_c_allocator_path_matches_two_phase(pct, prec):
    w = W.neo2_2d_spline(n_angles=6, paths_per_angle=100, n=128, h=1.6)
    a = run_gpu(pct, w, prec)
    ph = pct.Phantom(w["phantom"])
    b = pct.simulate_c_alloc(ph, pct.GeometryArgs(w), _prec(pct, prec))
    for k in ("row_ptr", "col", "val", "b", "x_true"):
        assert torch.equal(a[k], b[k]), k


def test_mixed_and_f64_forms_agree_on_indices(pct):
    w = W.neo2_2d_spline(n_angles=20, paths_per_angle=500, n=256, h=0.8)
    a = run_gpu(pct, w, "f64")
    b = run_gpu(pct, w, "mixed")
    assert torch.equal(a["row_ptr"], b["row_ptr"]) and torch.equal(a["col"], b["col"])


def test_deterministic(pct):
    w = W.neo2_2d_spline(n_angles=10, paths_per_angle=200, n=128, h=1.6)
    for prec in PRECS:
        a = run_gpu(pct, w, prec)
        b = run_gpu(pct, w, prec)
        for k in ("row_ptr", "col", "val", "b"):
            assert torch.equal(a[k], b[k])


def test_rows_beyond_cooperative_limits(pct, orc):
    """Rows the warp-cooperative kernels hand to the per-lane walker: splines
    of 70 pieces (72 segments, more than one warp's 64-segment table) and
    straight rows with more than 4096 plane crossings (0.1 mm pixels on a
    2200 x 2200 grid, near-diagonal through the centre)."""
    w = W.neo2_2d_spline(n_angles=6, paths_per_angle=100, n=128, h=1.6)
    w["model"] = dict(w["model"], spline_segments=70)
    compare(run_gpu(pct, w, "mixed"), run_oracle(orc, w))
    w = W.neo1_2d_straight(n_angles=2, paths_per_angle=50)
    w["phantom"] = W.phantom(2, (2200, 2200), (0.1, 0.1), skin=False)
    w["angles"] = np.array([math.pi / 4 + 0.01, 3 * math.pi / 4 - 0.013])
    w["model"] = W.model(W.STRAIGHT, (-10.0, 10.0))
    g = run_gpu(pct, w, "mixed")
    ref = run_oracle(orc, w)
    assert np.diff(ref["row_ptr"]).min() > 4096
    compare(g, ref)


@pytest.mark.parametrize("K", [34, 35, 48])
def test_both_shared_memory_layouts(pct, orc, K):
    """Splines of 34 pieces (36 segments: the smaller per-warp layout, full)
    and of 35 and 48 pieces (37 and 50 segments: the 64-segment layout), 2D
    and 3D, against the oracle."""
    w = W.neo2_2d_spline(n_angles=6, paths_per_angle=150, n=128, h=1.6)
    w["model"] = dict(w["model"], spline_segments=K)
    compare(run_gpu(pct, w, "mixed"), run_oracle(orc, w))
    w = W.head_3d_spline(n_angles=3, paths_per_angle=200, n=(40, 40, 32), h=(2.0, 2.0, 2.0))
    w["model"] = dict(w["model"], spline_segments=K)
    compare(run_gpu(pct, w, "mixed"), run_oracle(orc, w))
