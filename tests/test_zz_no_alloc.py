"""The allocation-free entry point pct_scan_counts_static, for callers that
cannot allocate device memory: its row pointers must equal those of the
workspace-based scan inside pct_simulate_count, call after call.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test."""
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


def _workspace_row_ptr(pct, w):
    ph = pct.Phantom(w["phantom"])
    geo = pct.GeometryArgs(w)
    ws = torch.empty(pct.simulate_workspace_size(ph, geo, pct.PREC_MIXED), dtype=torch.uint8, device="cuda")
    rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, device="cuda")
    pct.simulate_count(ph, geo, pct.PREC_MIXED, ws, rp)
    return rp


def test_static_scan_matches_workspace_scan_two_calls_in_a_row(pct):
    cases = [W.neo2_2d_spline(n_angles=12, paths_per_angle=777, n=256, h=0.8),
             W.neo1_2d_straight(n_angles=30, paths_per_angle=1001)]
    for w in cases:
        ref = _workspace_row_ptr(pct, w)
        counts = ref[1:] - ref[:-1]
        out = torch.full_like(ref, -99)
        out[1:] = counts
        pct.scan_counts_static(out, len(counts))
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_static_scan_tiles_and_ragged_tail_twice(pct):
    rng = np.random.default_rng(5)
    for n in (3 * 4096 + 17, 1):
        counts = rng.integers(0, 2000, n).astype(np.int64)
        want = np.concatenate([[0], np.cumsum(counts)])
        for _ in range(2):  # the shared scratch keeps the last call's contents
            rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
            rp[1:] = torch.from_numpy(counts).cuda()
            pct.scan_counts_static(rp, n)
            torch.cuda.synchronize()
            assert np.array_equal(rp.cpu().numpy(), want)


def test_static_scan_rejects_rows_beyond_its_scratch(pct):
    rp = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(pct.PctError) as e:
        pct.scan_counts_static(rp, pct.STATIC_SCAN_MAX_ROWS + 1)
    assert e.value.status == pct.EINVAL
    assert "static scratch limit" in pct.last_error()
