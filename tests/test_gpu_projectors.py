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


@pytest.mark.parametrize("prec_name", ["mixed", "f64"])
def test_matrix_free_forward_and_adjoint(pct, case, prec_name):
    prec = {"mixed": pct.PREC_MIXED, "f64": pct.PREC_F64}[prec_name]
    A, g, ph, geo = case["A"], case["g"], case["ph"], case["geo"]
    half = A.shape[0] // 2
    ws = torch.empty(pct.projector_workspace_size(ph, geo, A.shape[0] - half, prec), dtype=torch.uint8,
                     device="cuda")
    x = torch.from_numpy(case["x"]).cuda()
    y_mf = torch.empty(A.shape[0], device="cuda")
    # two chunks, as a caller streaming rows would
    pct.forward(ph, geo, None, 0, half, x, y_mf[:half], ws, precision=prec)
    pct.forward(ph, geo, None, half, A.shape[0] - half, x, y_mf[half:], ws, precision=prec)
    want = A @ case["x"].astype(np.float64)
    scale = abs(A) @ np.abs(case["x"].astype(np.float64))
    assert np.all(np.abs(to_np(y_mf) - want) <= 1e-6 * np.maximum(scale, 1e-30) + 1e-30)
    r = torch.from_numpy(case["r"]).cuda()
    gm = torch.zeros(A.shape[1], device="cuda")
    pct.adjoint(ph, geo, None, 0, half, r[:half], gm, ws, precision=prec)
    pct.adjoint(ph, geo, None, half, A.shape[0] - half, r[half:], gm, ws, precision=prec)
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


def test_autograd_gradient_is_the_adjoint_residual(pct, case):
    from paper_2108_12369_gb300.autograd import Projector, project
    A, w = case["A"], case["w"]
    ref = case["g"]
    b = ref["b"]
    for proj in (Projector(w, chunk_rows=3000), Projector(w, csr=ref)):
        x = torch.from_numpy(case["x"]).cuda().requires_grad_(True)
        y = project(x, proj)
        loss = 0.5 * ((y - b) ** 2).sum()
        loss.backward()
        res = A @ case["x"].astype(np.float64) - to_np(b).astype(np.float64)
        want = A.T @ res
        scale = abs(A).T @ np.abs(res)
        assert np.all(np.abs(to_np(x.grad) - want) <= 1e-4 * np.maximum(scale, 1e-30) + 1e-6)


def test_gradient_matches_finite_differences_32cube(pct, orc):
    """Gradient of 1/2 |A x - b|^2 on a 32^3 head instance against central
    differences (exact for a quadratic up to rounding) and the explicit
    CSR transpose."""
    from paper_2108_12369_gb300.autograd import Projector, project
    w = W.head_3d_spline(n_angles=12, paths_per_angle=300, n=(32, 32, 32), h=(6.25, 6.25, 5.0))
    proj = Projector(w, chunk_rows=1000)
    ref = orc.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"], threads=8)
    A = sp.csr_matrix((ref["val"], ref["col"], ref["row_ptr"]), shape=(len(ref["b"]), 32 ** 3))
    rng = np.random.default_rng(2)
    x0 = rng.uniform(0.8, 1.2, 32 ** 3)
    b = torch.from_numpy(ref["b"].astype(np.float32)).cuda()
    x = torch.from_numpy(x0.astype(np.float32)).cuda().requires_grad_(True)
    loss = 0.5 * ((project(x, proj) - b) ** 2).sum()
    loss.backward()
    g = to_np(x.grad).astype(np.float64)
    g_csr = A.T @ (A @ x0.astype(np.float32).astype(np.float64) - ref["b"])
    assert np.allclose(g, g_csr, rtol=1e-4, atol=1e-3 * np.abs(g_csr).max())
    cols = np.flatnonzero(np.abs(g_csr) > 0.05 * np.abs(g_csr).max())[:8]
    assert len(cols) >= 4
    eps = 0.05
    for j in cols:
        def L(delta):
            xx = x0.astype(np.float32).copy()
            xx[j] += delta
            y = to_np(proj.forward(torch.from_numpy(xx).cuda())).astype(np.float64)
            return 0.5 * np.sum((y - ref["b"]) ** 2)
        fd = (L(eps) - L(-eps)) / (2 * eps)
        assert abs(fd - g[j]) <= 2e-3 * max(abs(g[j]), 1.0), (j, fd, g[j])
