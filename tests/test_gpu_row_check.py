"""The fill's row check (Sec. II-C: row i of A holds exactly proton i's
entries): a fill given row pointers that are not its count's reports the rows
that disagree (pct_simulate_check; pct_simulate_fill_host returns EINVAL),
keeps every store inside the range row_ptr gives each row, and reports nothing
for a consistent fill.  The inconsistent row pointers are made on the host
(one row one entry shorter or longer), for every arithmetic form."""
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


def setup(pct, prec):
    w = W.head_3d_spline(n_angles=3, paths_per_angle=700, n=(48, 48, 40))
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    ws = torch.empty(pct.simulate_workspace_size(ph, geo, prec), dtype=torch.uint8, device="cuda")
    x = torch.empty(ph.nvox, dtype=torch.float32, device="cuda")
    rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, device="cuda")
    pct.phantom_rasterize(ph, x)
    pct.simulate_count(ph, geo, prec, ws, rp)
    return ph, geo, ws, x, rp


def fill(pct, ph, geo, prec, ws, x, rp, nnz_alloc):
    col = torch.full((nnz_alloc + 64,), -7, dtype=torch.int32, device="cuda")
    val = torch.full((nnz_alloc + 64,), -7.0, dtype=torch.float32, device="cuda")
    b = torch.empty(geo.n_rows, dtype=torch.float32, device="cuda")
    pct.simulate_fill(ph, geo, prec, ws, rp, x, col, val, b)
    return col, val


PRECS = ["mixed", "lean", "f64"]


@pytest.mark.parametrize("prec_name", PRECS)
def test_consistent_fill_reports_nothing(pct, prec_name):
    prec = {"mixed": pct.PREC_MIXED, "lean": pct.PREC_MIXED_LEAN, "f64": pct.PREC_F64}[prec_name]
    ph, geo, ws, x, rp = setup(pct, prec)
    nnz = int(rp[-1])
    fill(pct, ph, geo, prec, ws, x, rp, nnz)
    assert pct.simulate_check(ws) == 0


@pytest.mark.parametrize("prec_name", PRECS)
@pytest.mark.parametrize("delta", [-1, 1])
def test_a_row_of_other_length_is_reported(pct, prec_name, delta):
    prec = {"mixed": pct.PREC_MIXED, "lean": pct.PREC_MIXED_LEAN, "f64": pct.PREC_F64}[prec_name]
    ph, geo, ws, x, rp = setup(pct, prec)
    nnz = int(rp[-1])
    ref_col, ref_val = fill(pct, ph, geo, prec, ws, x, rp, nnz)
    lens = (rp[1:] - rp[:-1]).cpu()
    r = int(torch.nonzero(lens > 3)[len(torch.nonzero(lens > 3)) // 2])  # a row with entries, mid-way
    bad = rp.clone()
    bad[r + 1:] += delta  # row r one entry shorter (-1) or longer (+1)
    col, val = fill(pct, ph, geo, prec, ws, x, bad, nnz + 1)
    assert pct.simulate_check(ws) == 1
    s, e = int(rp[r]), int(rp[r + 1])
    # rows before r as before; rows after r the same entries, moved by delta
    assert torch.equal(col[:s], ref_col[:s]) and torch.equal(val[:s], ref_val[:s])
    assert torch.equal(col[e + delta:nnz + delta], ref_col[e:nnz])
    assert torch.equal(val[e + delta:nnz + delta], ref_val[e:nnz])
    # row r: its first entries in place; no store outside the rows' ranges
    assert torch.equal(col[s:e - 1], ref_col[s:e - 1])
    assert bool((col[nnz + delta:] == -7).all())
    if delta > 0:
        assert int(col[e]) == -7  # the slot the shorter count leaves unwritten
    # the host fill returns the mismatch as an error
    h_rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, pin_memory=True)
    h_col = torch.empty(nnz + 1, dtype=torch.int32, pin_memory=True)
    h_val = torch.empty(nnz + 1, dtype=torch.float32, pin_memory=True)
    h_b = torch.empty(geo.n_rows, dtype=torch.float32, pin_memory=True)
    staging = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    pct.simulate_count(ph, geo, prec, ws, rp)  # zeroes the check
    with pytest.raises(pct.PctError) as err:
        pct.simulate_fill_host(ph, geo, prec, ws, bad, x, staging, h_rp, h_col, h_val, h_b)
    assert err.value.status == pct.EINVAL and "different number of entries" in str(err.value)
