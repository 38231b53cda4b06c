"""String-averaging projections (Sec. II-D) on the GPU against the oracle's
FP64 SAP, on simulated systems; the paper's setting (M = 100 strings,
lambda = 0.1, 20 iterations) as a reconstruction check.

Tolerance: each projection is non-expansive (lambda in (0, 2)), so rounding
differences do not grow; they add up.  One FP32 projection perturbs the
touched components by about 8 u (|y_j| + |c a_ij|) with u = 2^-24 (sums of
a few hundred terms, the quotient, the update), so after `iterations` sweeps
of strings of m rows the difference stays below
iterations * m * 8 u * max|x| in the worst case; the test uses that bound."""
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


def _system(pct, w):
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    sim = pct.simulate(ph, geo, pct.PREC_MIXED)
    torch.cuda.synchronize()
    return sim, ph.nvox


@pytest.mark.parametrize("M,lam,iters", [(1, 1.0, 1), (7, 0.5, 3), (100, 0.1, 2), (5000, 1.5, 1)])
def test_sap_matches_oracle(pct, orc, M, lam, iters):
    w = W.neo2_2d_spline(n_angles=12, paths_per_angle=300, n=96, h=2.0)
    sim, n = _system(pct, w)
    rp, col, val, b = (sim[k].cpu().numpy() for k in ("row_ptr", "col", "val", "b"))
    rng = np.random.default_rng(M)
    x0 = rng.uniform(0.0, 1.5, n).astype(np.float32)
    want = orc.sap(rp, col, val.astype(np.float64), b.astype(np.float64), n, M, lam, iters, x0.astype(np.float64))
    x = torch.from_numpy(x0).cuda()
    pct.sap(sim, sim["b"], n, M, lam, iters, x)
    torch.cuda.synchronize()
    got = x.cpu().numpy().astype(np.float64)
    m = -(-(len(rp) - 1) // M)  # rows per string (at most)
    bound = iters * m * 8 * 2.0**-24 * max(1.0, np.abs(want).max())
    err = np.abs(got - want).max()
    assert err <= bound, (err, bound)


def test_sap_zero_iterations_and_empty_strings(pct):
    w = W.neo1_2d_straight(n_angles=4, paths_per_angle=10)
    sim, n = _system(pct, w)
    x = torch.rand(n, device="cuda")
    x0 = x.clone()
    pct.sap(sim, sim["b"], n, 3, 0.5, 0, x)
    torch.cuda.synchronize()
    assert torch.equal(x, x0)
    # more strings than rows: the empty strings keep x and weigh in the average
    pct.sap(sim, sim["b"], n, 200, 1.0, 1, x, weights=np.full(200, 1 / 200))
    torch.cuda.synchronize()
    assert torch.isfinite(x).all()


def test_sap_rejects_bad_weights_and_small_workspace(pct):
    w = W.neo1_2d_straight(n_angles=2, paths_per_angle=5)
    sim, n = _system(pct, w)
    x = torch.zeros(n, device="cuda")
    with pytest.raises(pct.PctError) as e:
        pct.sap(sim, sim["b"], n, 4, 0.1, 1, x, weights=[0.5, 0.5, 0.5, 0.5])
    assert e.value.status == pct.EINVAL
    ws = torch.empty(pct.sap_workspace_size(n, 4) - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(pct.PctError) as e:
        pct.sap(sim, sim["b"], n, 4, 0.1, 1, x, workspace=ws)
    assert e.value.status == pct.ENOMEM


def test_sap_reconstructs_neo1_with_the_papers_settings(pct):
    """NEO 1, straight paths, constant 1 mm chords as in the paper's examples
    (b from exact chords), 4.5 histories per pixel, M = 100, lambda = 0.1,
    20 iterations from 0: the image error falls at every checkpoint, the
    residual falls, and brain (RSP 1.04) reconstructs brighter than a
    ventricle (0.9)."""
    w = W.neo1_2d_straight(n_angles=180, paths_per_angle=1000)
    w["model"] = dict(w["model"], chord=W.CHORD_CONSTANT)
    sim, n = _system(pct, w)
    x_true = sim["x_true"]
    x = torch.zeros(n, device="cuda")
    A = torch.sparse_csr_tensor(sim["row_ptr"], sim["col"].long(), sim["val"], size=(len(sim["b"]), n))
    res = [torch.linalg.norm(sim["b"]).item()]
    err = [torch.linalg.norm(x_true).item()]
    ws = torch.empty(pct.sap_workspace_size(n, 100), dtype=torch.uint8, device="cuda")
    for _ in range(4):
        pct.sap(sim, sim["b"], n, 100, 0.1, 5, x, workspace=ws)
        torch.cuda.synchronize()
        res.append(torch.linalg.norm(A @ x - sim["b"]).item())
        err.append(torch.linalg.norm(x - x_true).item())
    print("SAP NEO-1 residual", res, "image error", err)
    assert all(e1 < e0 for e0, e1 in zip(err[:-1], err[1:])), err
    assert res[-1] < 0.2 * res[0] and err[-1] < 0.4 * err[0]  # measured on GB300: 0.10 and 0.29
    img = x.view(200, 200).cpu().numpy()
    brain = img[100 - 2:100 + 2, 100 + 40 - 2:100 + 40 + 2].mean()
    vent = img[100 - 1:100 + 1, 100 + 10 - 2:100 + 10 + 2].mean()
    assert brain > vent, (brain, vent)
