"""Parity at the full workload sizes, in the launch configuration bench.py
times (two-phase count / fill, mixed precision): the NEO-2 spline workload
(512 x 512 px of 0.4 mm, 360 angles x 10,000 protons, 3.6M rows) and the 3D
head workload (200 x 200 x 160 voxels, 90 angles x 200k protons, 18M rows).
The oracle recomputes a sample of rows one by one: an even stride through
all rows, the first and last rows, and rows around thread-block and angle
boundaries.  Sampled rows must match exactly in length and voxel indices,
and within 1e-6 of the row sum in values and of max(b, row sum x max RSP)
in WEPL."""
import numpy as np
import pytest

from paper_2108_12369_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12369_gb300 import build, pct as P
    build.build()
    return P


def sample_rows(n_rows: int, paths_per_angle: int, stride: int) -> np.ndarray:
    s = set(range(0, n_rows, stride))
    s.update(range(min(5, n_rows)))
    s.update(range(max(0, n_rows - 5), n_rows))
    for edge in (127, 128, 4095, 4096, paths_per_angle - 1, paths_per_angle, 7 * paths_per_angle + 3):
        if edge < n_rows:
            s.add(edge)
    return np.array(sorted(s), dtype=np.int64)


def check_sampled(pct, orc, w, stride):
    ph = pct.Phantom(w["phantom"])
    geo = pct.GeometryArgs(w)
    g = pct.simulate(ph, geo, pct.PREC_MIXED)
    torch.cuda.synchronize()
    rp = g["row_ptr"]
    assert bool((rp[1:] >= rp[:-1]).all()) and int(rp[-1]) == g["nnz"]
    rows = sample_rows(geo.n_rows, w["paths_per_angle"], stride)
    ref = orc.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"], rows=rows,
                       threads=16)
    assert np.array_equal(g["x_true"].cpu().numpy(), ref["x_true"])
    r = torch.from_numpy(rows).cuda()
    start, end = rp[r], rp[r + 1]
    lens = (end - start).cpu().numpy()
    assert np.array_equal(lens, np.diff(ref["row_ptr"]))
    # gather the sampled rows' entries on the device
    pos = torch.repeat_interleave(start, end - start)
    off = torch.arange(pos.numel(), device="cuda") - torch.repeat_interleave(
        torch.cumsum(end - start, 0) - (end - start), end - start)
    idx = pos + off
    col = g["col"][idx].cpu().numpy()
    val = g["val"][idx].cpu().numpy().astype(np.float64)
    b = g["b"][r].cpu().numpy().astype(np.float64)
    assert np.array_equal(col, ref["col"])
    rowid = np.repeat(np.arange(len(rows)), lens)
    rowsum = np.bincount(rowid, weights=ref["val"], minlength=len(rows))
    err = np.abs(val - ref["val"]) / np.maximum(rowsum[rowid], 1e-30)
    assert err.size == 0 or err.max() <= 1e-6, err.max()
    scale = np.maximum(np.abs(ref["b"]), rowsum * float(ref["x_true"].max()))
    errb = np.abs(b - ref["b"]) / np.maximum(scale, 1e-30)
    assert errb.max() <= 1e-6, errb.max()
    return len(rows), int(lens.sum()), float(err.max() if err.size else 0.0), float(errb.max())


def test_neo2_full_size_sampled_rows(pct, orc):
    print(check_sampled(pct, orc, W.neo2_2d_spline(), stride=1201))


def test_head_3d_full_size_sampled_rows(pct, orc):
    print(check_sampled(pct, orc, W.head_3d_spline(), stride=6007))
