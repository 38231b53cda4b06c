"""Projectors y = A x and g = A^T r (Sec. II, A x = b): explicit CSR and
matrix-free (paths recomputed) against the oracle's CSR in FP64, plus the
adjoint (dot-product) identity."""
import numpy as np
import pytest

from paper_2108_12369_gb300 import workloads as W
from tests.parity import to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")


@pytest.fixture(scope="module")
def pct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12369_gb300 import build, pct as P
    build.build()
    return P


@pytest.fixture(scope="module")
def case(pct, orc):
    w = W.neo2_2d_spline(n_angles=24, paths_per_angle=400, n=256, h=0.8)
    ref = orc.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"], threads=8)
    n_rows = len(ref["b"])
    A = sp.csr_matrix((ref["val"], ref["col"], ref["row_ptr"]), shape=(n_rows, len(ref["x_true"])))
    ph = pct.Phantom(w["phantom"])
    geo = pct.GeometryArgs(w)
    g = pct.simulate(ph, geo, pct.PREC_F64)
    rng = np.random.default_rng(0)
    x = rng.uniform(0.5, 1.5, A.shape[1]).astype(np.float32)
    r = rng.normal(size=A.shape[0]).astype(np.float32)
    return dict(w=w, A=A, ph=ph, geo=geo, g=g, x=x, r=r)


def test_csr_forward(pct, case):
    A, g = case["A"], case["g"]
    x = torch.from_numpy(case["x"]).cuda()
    y = torch.empty(A.shape[0], device="cuda")
    pct.forward(None, None, g, 0, A.shape[0], x, y)
    want = A @ case["x"].astype(np.float64)
    scale = abs(A) @ np.abs(case["x"].astype(np.float64))
    assert np.all(np.abs(to_np(y) - want) <= 2e-6 * np.maximum(scale, 1e-30) + 1e-30)


def test_csr_forward_row_range(pct, case):
    A, g = case["A"], case["g"]
    x = torch.from_numpy(case["x"]).cuda()
    y = torch.empty(1000, device="cuda")
    pct.forward(None, None, g, 2500, 1000, x, y)
    want = A[2500:3500] @ case["x"].astype(np.float64)
    assert np.allclose(to_np(y), want, rtol=2e-6, atol=1e-4)


def test_csr_adjoint(pct, case):
    A, g = case["A"], case["g"]
    r = torch.from_numpy(case["r"]).cuda()
    out = torch.zeros(A.shape[1], device="cuda")
    pct.adjoint(None, None, g, 0, A.shape[0], r, out)
    want = A.T @ case["r"].astype(np.float64)
    scale = abs(A).T @ np.abs(case["r"].astype(np.float64))
    assert np.all(np.abs(to_np(out) - want) <= 1e-5 * np.maximum(scale, 1e-30) + 1e-30)


def test_matrix_free_forward_and_adjoint(pct, case):
    A, g, ph, geo = case["A"], case["g"], case["ph"], case["geo"]
    ws = torch.empty(pct.simulate_workspace_size(ph, geo, pct.PREC_F64), dtype=torch.uint8, device="cuda")
    x = torch.from_numpy(case["x"]).cuda()
    y_mf = torch.empty(A.shape[0], device="cuda")
    # two chunks, as a caller streaming rows would
    half = A.shape[0] // 2
    pct.forward(ph, geo, None, 0, half, x, y_mf[:half], ws)
    pct.forward(ph, geo, None, half, A.shape[0] - half, x, y_mf[half:], ws)
    want = A @ case["x"].astype(np.float64)
    scale = abs(A) @ np.abs(case["x"].astype(np.float64))
    assert np.all(np.abs(to_np(y_mf) - want) <= 1e-6 * np.maximum(scale, 1e-30) + 1e-30)
    r = torch.from_numpy(case["r"]).cuda()
    gm = torch.zeros(A.shape[1], device="cuda")
    pct.adjoint(ph, geo, None, 0, half, r[:half], gm, ws)
    pct.adjoint(ph, geo, None, half, A.shape[0] - half, r[half:], gm, ws)
    want = A.T @ case["r"].astype(np.float64)
    scale = abs(A).T @ np.abs(case["r"].astype(np.float64))
    assert np.all(np.abs(to_np(gm) - want) <= 1e-5 * np.maximum(scale, 1e-30) + 1e-30)


def test_dot_product_identity(pct, case):
    A, g = case["A"], case["g"]
    x = torch.from_numpy(case["x"]).cuda()
    r = torch.from_numpy(case["r"]).cuda()
    y = torch.empty(A.shape[0], device="cuda")
    gt = torch.zeros(A.shape[1], device="cuda")
    pct.forward(None, None, g, 0, A.shape[0], x, y)
    pct.adjoint(None, None, g, 0, A.shape[0], r, gt)
    lhs = float(torch.dot(y.double(), r.double()))
    rhs = float(torch.dot(x.double(), gt.double()))
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs))
