"""Pins of the FP64 CPU oracle to things other than itself: an independent
Philox implementation (numpy), libm, closed forms (chords of ellipses,
clipped segment lengths, plane-crossing counts), hand-worked rasters
(tests/golden/), brute-force supersampling on tiny grids, textbook Hermite
curves and arc lengths, and distribution statistics."""
import math
from pathlib import Path

import numpy as np
import pytest

from paper_2108_12369_gb300 import workloads as W

GOLDEN = Path(__file__).resolve().parent / "golden"


def _numpy_block(key, row, block, n=4):
    """Words of Philox block `block` of proton `row` from numpy's generator.

    numpy increments the 256-bit counter before each block, so it is started
    at (row + block * 2^64) - 1."""
    v = (row + (block << 64) - 1) % (1 << 256)
    ctr = np.array([(v >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    return np.random.Philox(key=np.array(key, dtype=np.uint64), counter=ctr).random_raw(n)


# --------------------------------------------------------------------------
# Random numbers (Sec. II-B, BNRNG; rand() replaced by Philox4x64-10)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("key,ctr", [
    ([0, 0], [0, 0, 0, 0]),
    ([2**64 - 1, 2**64 - 1], [2**64 - 1, 2**64 - 1, 2**64 - 1, 2**64 - 2]),
    ([210812369, 0], [12345, 7, 0, 0]),
    ([0x243F6A8885A308D3, 0x13198A2E03707344], [1, 2, 3, 4]),
])
def test_philox_matches_numpy(orc, key, ctr):
    # numpy's Philox (an independent implementation of Philox4x64-10)
    # increments its 256-bit counter before each block.
    g = np.random.Philox(key=key, counter=ctr)
    ref = g.random_raw(4)
    c = list(ctr)
    for i in range(4):  # 256-bit little-endian increment
        c[i] = (c[i] + 1) % 2**64
        if c[i] != 0:
            break
    out = orc.philox4x64_10(c, key)
    assert [int(v) for v in out] == [int(v) for v in ref]


def test_uniform_mapping_and_stream_layout(orc):
    seed, stream, row = 99, 5, 123456
    raw = _numpy_block([seed, stream], row, 0)
    for j in range(4):
        want = (float(int(raw[j]) >> 11) + 0.5) * 2.0**-53
        assert orc.uniform(seed, stream, row, j) == want
    raw = _numpy_block([seed, stream], row, 1)
    assert orc.uniform(seed, stream, row, 6) == (float(int(raw[2]) >> 11) + 0.5) * 2.0**-53


def test_uniform_statistics(orc):
    u = np.array([orc.uniform(7, 0, r, j) for r in range(2000) for j in range(8)])
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(u))
    hist = np.histogram(u, bins=16, range=(0, 1))[0]
    chi2 = ((hist - len(u) / 16) ** 2 / (len(u) / 16)).sum()
    assert chi2 < 50  # 15 dof, p ~ 1e-5


def test_log_against_libm(orc):
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(0, 1, 20000), 10.0 ** rng.uniform(-300, 0, 20000),
                         rng.uniform(0.99, 1.01, 5000), [1.0, 0.5, 0.25, 2.0**-1000, 1e-308]])
    worst = 0.0
    for x in xs:
        if x <= 0:
            continue
        ref = math.log(x)
        got = orc.log(x)
        if ref == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, abs(got - ref) / math.ulp(ref))
    assert worst <= 2.0, worst
    assert orc.log(1.0) == 0.0
    for e in (-1, -2, -20, -1000):
        assert abs(orc.log(2.0**e) - e * math.log(2.0)) <= 2 * math.ulp(e * math.log(2.0))


def test_polar_method_first_attempt_matches_independent_draws(orc):
    seed = 4242
    checked = 0
    for row in range(300):
        raw = _numpy_block([seed, 0], row, 1, 2)
        u1, u2 = [(float(int(w) >> 11) + 0.5) * 2.0**-53 for w in raw]
        v1, v2 = 2 * u1 - 1, 2 * u2 - 1
        s = v1 * v1 + v2 * v2
        z, j = orc.normal_pairs(seed, 0, row, 4, 1)
        if 0 < s < 1:
            f = math.sqrt(-2 * math.log(s) / s)
            assert j == 6
            assert abs(z[0] - v1 * f) <= 1e-14 * max(1.0, abs(v1 * f))
            assert abs(z[1] - v2 * f) <= 1e-14 * max(1.0, abs(v2 * f))
            checked += 1
        else:
            assert j >= 8  # rejected: at least one more attempt
    assert checked > 200


def test_normals_are_standard_and_independent(orc):
    scipy_stats = pytest.importorskip("scipy.stats")
    z = np.concatenate([orc.normal_pairs(11, 0, r, 4, 4)[0] for r in range(6000)])
    assert abs(z.mean()) < 4 / math.sqrt(len(z))
    assert abs(z.var() - 1) < 0.03
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-3
    pairs = z.reshape(-1, 2)
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 0.03


# --------------------------------------------------------------------------
# Phantom raster (Sec. II-A)
# --------------------------------------------------------------------------
def _disc_phantom(dim, n, h, regions, raster):
    return {"dim": dim, "kind": W.ELLIPSOID, "raster": raster, "n": tuple(n) + (1,) * (3 - len(n)),
            "h": tuple(h) + (1.0,) * (3 - len(h)), "regions": regions}


def test_corner_raster_golden_2d(orc):
    want = np.loadtxt(GOLDEN / "raster_circle_r1.5_4x4.txt")
    ph = orc.Phantom(_disc_phantom(2, (4, 4), (1.0, 1.0),
                                   [{"c": (0, 0, 0), "a": (1.5, 1.5, 1.5), "rsp": 1.0}], W.CORNER))
    got = ph.raster().reshape(4, 4)
    assert np.array_equal(got, want)


def test_center_raster_disc_2d(orc):
    ph = orc.Phantom(_disc_phantom(2, (4, 4), (1.0, 1.0),
                                   [{"c": (0, 0, 0), "a": (1.5, 1.5, 1.5), "rsp": 2.0}], W.CENTER))
    got = ph.raster().reshape(4, 4)
    want = np.zeros((4, 4))
    want[1:3, 1:3] = 2.0  # centres (+-0.5, +-0.5) only
    assert np.array_equal(got, want)


def test_corner_raster_golden_3d(orc):
    ph = orc.Phantom(_disc_phantom(3, (4, 4, 4), (1.0, 1.0, 1.0),
                                   [{"c": (0, 0, 0), "a": (1.5, 1.5, 1.5), "rsp": 1.0}], W.CORNER))
    x = ph.raster().reshape(4, 4, 4)  # [iz, iy, ix]
    for ix, iy, iz, v in np.loadtxt(GOLDEN / "raster_sphere_r1.5_4x4x4_center_voxel.txt"):
        assert x[int(iz), int(iy), int(ix)] == v


def test_painter_order_and_extrusion(orc):
    regs = [{"c": (0, 0, 0), "a": (50, 50, 50), "rsp": 1.0},
            {"c": (0, 0, 0), "a": (20, 20, 20), "rsp": 3.0}]
    ph = orc.Phantom(_disc_phantom(2, (10, 10), (10.0, 10.0), regs, W.CENTER))
    x = ph.raster().reshape(10, 10)
    assert x[5, 5] == 3.0 and x[5, 7] == 1.0 and x[0, 0] == 0.0
    d3 = _disc_phantom(3, (10, 10, 6), (10.0, 10.0, 10.0), regs, W.CENTER)
    d3["kind"] = W.EXTRUDED  # elliptical cylinder: every z slice equals the 2D raster
    x3 = orc.Phantom(d3).raster().reshape(6, 10, 10)
    for iz in range(6):
        assert np.array_equal(x3[iz], x)


@pytest.mark.parametrize("h", [1.0, 0.5, 0.25])
def test_raster_area_and_volume_converge(orc, h):
    a, b, c = 30.0, 20.0, 12.0
    n2 = int(80 / h)
    ph = orc.Phantom(_disc_phantom(2, (n2, n2), (h, h),
                                   [{"c": (0, 0, 0), "a": (a, b, 1), "rsp": 1.0}], W.CORNER))
    area = ph.raster().sum() * h * h
    perim = math.pi * (3 * (a + b) - math.sqrt((3 * a + b) * (a + 3 * b)))
    assert abs(area - math.pi * a * b) <= 0.5 * perim * h  # boundary-pixel bound
    if h >= 0.5:
        n3 = int(70 / h)
        ph3 = orc.Phantom(_disc_phantom(3, (n3, n3, n3), (h, h, h),
                                        [{"c": (0, 0, 0), "a": (a, b, c), "rsp": 1.0}], W.CORNER))
        vol = ph3.raster().sum() * h ** 3
        p = 1.6075
        surf = 4 * math.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3) ** (1 / p)
        assert abs(vol - 4 / 3 * math.pi * a * b * c) <= 0.5 * surf * h * math.sqrt(3)


# --------------------------------------------------------------------------
# Hull chords (Sec. II-B: entry / exit points of the phantom)
# --------------------------------------------------------------------------
def test_hull_chord_closed_form(orc):
    rng = np.random.default_rng(3)
    regs = [{"c": (5.0, -3.0, 2.0), "a": (90.0, 70.0, 80.0), "rsp": 1.0}]
    ph2 = orc.Phantom(_disc_phantom(2, (10, 10), (1.0, 1.0), regs, W.CENTER))
    ph3 = orc.Phantom(_disc_phantom(3, (10, 10, 10), (1.0, 1.0, 1.0), regs, W.CENTER))
    for _ in range(200):
        # horizontal line y = y0: chord 2 a sqrt(1 - ((y0 - cy)/b)^2)
        y0 = rng.uniform(-80, 75)
        hit, li, lo = ph2.hull_hit(0, (0.0, y0), (1.0, 0.0))
        q = 1 - ((y0 + 3.0) / 70.0) ** 2
        assert hit == (q > 0)
        if hit:
            assert abs((lo - li) - 2 * 90.0 * math.sqrt(q)) <= 1e-12 * 180
            assert abs((li + lo) / 2 - 5.0) <= 1e-12 * 100  # chord midpoint on the centre x
        # 3D line along z through (x0, y0): chord 2 c sqrt(1 - x^2/a^2 - y^2/b^2)
        x0 = rng.uniform(-60, 60)
        hit, li, lo = ph3.hull_hit(0, (x0, y0, 0.0), (0.0, 0.0, 1.0))
        q = 1 - ((x0 - 5.0) / 90.0) ** 2 - ((y0 + 3.0) / 70.0) ** 2
        assert hit == (q > 0)
        if hit:
            assert abs((lo - li) - 2 * 80.0 * math.sqrt(q)) <= 1e-12 * 160
        # oblique direction, not unit length: chord scales by 1/|g|
        th = rng.uniform(0, 2 * math.pi)
        g = np.array([math.cos(th), math.sin(th)]) * 1.7
        hit, li, lo = ph2.hull_hit(0, (5.0, -3.0), g)
        # through the centre: chord = 2 / sqrt((gx/a)^2 + (gy/b)^2) in units of lam
        want = 2 / math.sqrt((g[0] / 90) ** 2 + (g[1] / 70) ** 2)
        assert hit and abs((lo - li) - want) <= 1e-12 * want


# --------------------------------------------------------------------------
# Voxel traversal (Sec. II-C, DDA; a_ij = chord length in voxel j)
# --------------------------------------------------------------------------
def _grid_phantom(orc, dim, n, h):
    return orc.Phantom(_disc_phantom(dim, n, h, [{"c": (0, 0, 0), "a": (1, 1, 1), "rsp": 1.0}],
                                     W.CENTER))


def _clip_length(P, Q, lo, hi):
    """Liang-Barsky: length of segment PQ inside the box [lo, hi]."""
    P, Q = np.asarray(P, float), np.asarray(Q, float)
    d = Q - P
    t0, t1 = 0.0, 1.0
    for a in range(len(P)):
        if d[a] == 0:
            if not (lo[a] <= P[a] <= hi[a]):
                return 0.0
            continue
        ta, tb = (lo[a] - P[a]) / d[a], (hi[a] - P[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0) * float(np.linalg.norm(d)), t0, t1


def test_axis_aligned_rays_through_centres(orc):
    ph = _grid_phantom(orc, 2, (200, 200), (1.0, 1.0))
    for iy in (0, 57, 199):
        y = -100 + iy + 0.5
        cols, lens = ph.segment((-150.0, y), (150.0, y))
        assert np.array_equal(cols, np.arange(200) + 200 * iy)
        assert np.allclose(lens, 1.0, rtol=0, atol=1e-12)  # exact up to rounding
        cols, lens = ph.segment((150.0, y), (-150.0, y))
        assert np.array_equal(cols, np.arange(199, -1, -1) + 200 * iy)


def test_diagonal_through_corners_moves_diagonally(orc):
    ph = _grid_phantom(orc, 2, (200, 200), (1.0, 1.0))
    cols, lens = ph.segment((-120.0, -120.0), (120.0, 120.0))
    k = np.arange(200)
    assert np.array_equal(cols, k + 200 * k)
    assert np.allclose(lens, math.sqrt(2), rtol=1e-12, atol=0)
    assert np.all(lens > 0)


def test_row_sums_equal_clipped_length_and_counts(orc):
    rng = np.random.default_rng(5)
    for dim, n, h in ((2, (50, 40), (1.0, 0.7)), (3, (20, 16, 12), (1.0, 1.25, 0.8))):
        ph = _grid_phantom(orc, dim, n, h)
        lo = np.array([-0.5 * n[a] * h[a] for a in range(dim)])
        hi = -lo
        for _ in range(300):
            P = rng.uniform(1.3 * lo, 1.3 * hi)
            Q = rng.uniform(1.3 * lo, 1.3 * hi)
            cols, lens = ph.segment(P, Q)
            res = _clip_length(P, Q, lo, hi)
            L = res if isinstance(res, float) else res[0]
            assert abs(lens.sum() - L) <= 1e-12 * max(1.0, L)
            assert np.all(lens > 0)
            if L > 0:
                _, t0, t1 = res
                # generic segment: one interval plus one per interior plane crossed
                want = 1
                for a in range(dim):
                    xa, xb = sorted((P[a] + t0 * (Q[a] - P[a]), P[a] + t1 * (Q[a] - P[a])))
                    k = np.arange(n[a] + 1)
                    X = lo[a] + k * h[a]
                    want += int(np.sum((X > xa + 1e-9) & (X < xb - 1e-9)))
                assert len(cols) == want


def test_brute_force_supersampling_tiny_grids(orc):
    rng = np.random.default_rng(7)
    kept = 0
    for dim, n in ((2, (4, 4)), (3, (3, 3, 3))):
        h = (1.0,) * dim
        ph = _grid_phantom(orc, dim, n, h)
        lo = np.array([-0.5 * n[a] for a in range(dim)])
        for _ in range(150):
            P = rng.uniform(lo - 1, -lo + 1)
            Q = rng.uniform(lo - 1, -lo + 1)
            cols, lens = ph.segment(P, Q)
            N = 200000
            L = float(np.linalg.norm(Q - P))
            step = L / N
            if len(lens) and lens.min() < 20 * step:
                continue  # an interval too short for the sampler to resolve
            s = (np.arange(N) + 0.5) / N
            pts = P[None, :] + s[:, None] * (Q - P)[None, :]
            idx = np.floor(pts - lo[None, :]).astype(np.int64)
            ok = np.all((idx >= 0) & (idx < np.array(n)[None, :]), axis=1)
            lin = idx[:, 0] + n[0] * idx[:, 1] + (n[0] * n[1] * idx[:, 2] if dim == 3 else 0)
            lin = np.where(ok, lin, -1)
            change = np.flatnonzero(np.diff(lin)) + 1
            starts = np.concatenate([[0], change])
            runs = np.diff(np.concatenate([starts, [N]]))
            vox = lin[starts]
            keep = vox >= 0
            assert np.array_equal(vox[keep], cols)
            assert np.all(np.abs(runs[keep] * step - lens) <= 2 * step)
            kept += 1
    assert kept > 200


def test_reversed_segment_reverses_row(orc):
    rng = np.random.default_rng(9)
    ph = _grid_phantom(orc, 3, (16, 16, 16), (1.0, 1.0, 1.0))
    for _ in range(100):
        P, Q = rng.uniform(-10, 10, 3), rng.uniform(-10, 10, 3)
        c1, l1 = ph.segment(P, Q)
        c2, l2 = ph.segment(Q, P)
        assert np.array_equal(c1, c2[::-1])
        assert np.allclose(l1, l2[::-1], rtol=1e-9, atol=1e-12)


def test_segment_edge_cases(orc):
    ph = _grid_phantom(orc, 2, (10, 10), (1.0, 1.0))
    assert len(ph.segment((20.0, 20.0), (30.0, 25.0))[0]) == 0        # outside
    assert len(ph.segment((-5.0, 7.0), (5.0, 7.0))[0]) == 0           # on the line y = 7 > 5
    c, l = ph.segment((0.2, 0.3), (0.7, 0.9))                          # inside one pixel
    assert np.array_equal(c, [5 + 10 * 5]) and abs(l[0] - math.hypot(0.5, 0.6)) < 1e-15
    c, l = ph.segment((0.5, 0.5), (0.5, 0.5))                          # zero length
    assert len(c) == 0 or (len(c) == 1 and l[0] == 0.0)
    c, l = ph.segment((-5.0, -5.0), (-5.0, 5.0))                       # on the grid edge x = -5
    assert np.array_equal(c, 10 * np.arange(10)) and np.allclose(l, 1.0, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# Paths (Sec. II-B)
# --------------------------------------------------------------------------
def _spline_sim(orc, K=32, sigma=(1.0, 0.015, 0.015), rho=0.0, dim=2, model=W.SPLINE):
    if dim == 2:
        w = W.neo2_2d_spline(n_angles=12, paths_per_angle=50, spline_segments=K)
    else:
        w = W.head_3d_spline(n_angles=6, paths_per_angle=40, n=(40, 40, 32), h=(5.0, 5.0, 5.0),
                             spline_segments=K)
    m = dict(w["model"])
    m.update(model=model, sigma_lat=sigma[0], sigma_in=sigma[1], sigma_out=sigma[2], rho=rho,
             spline_segments=K)
    ph = orc.Phantom(w["phantom"])
    x = ph.raster().astype(np.float32)
    return orc.Simulation(ph, x, w["angles"], w["paths_per_angle"], m, w["seed"]), w


def _hermite(P0, P1, m0, m1, s):
    s = np.asarray(s)[:, None]
    H = np.array([[2, -3, 0, 1], [1, -2, 1, 0], [-2, 3, 0, 0], [1, -1, 0, 0]], float)
    S = np.concatenate([s ** 3, s ** 2, s, np.ones_like(s)], axis=1)
    B = S @ H.T  # columns h00 h10 h01 h11
    return B[:, 0:1] * P0 + B[:, 1:2] * m0 + B[:, 2:3] * P1 + B[:, 3:4] * m1


@pytest.mark.parametrize("dim", [2, 3])
def test_spline_vertices_are_the_hermite_curve(orc, dim):
    sim, w = _spline_sim(orc, K=16, dim=dim)
    ph = w["phantom"]
    R = 2 * math.sqrt(sum((ph["n"][a] * ph["h"][a]) ** 2 for a in range(dim)))
    hull = ph["regions"][0]
    checked = 0
    for row in range(0, sim.n_rows, 7):
        V = sim.path(row)
        if len(V) == 2:
            continue
        P0, P1 = V[1], V[-2]
        g0 = (V[1] - V[0]) / R
        g1 = (V[-1] - V[-2]) / R
        # P0 on the hull surface and on the incoming line
        q = sum(((P0[a] - hull["c"][a]) / hull["a"][a]) ** 2 for a in range(dim))
        assert abs(q - 1) < 1e-12
        l = float(np.dot(P1 - P0, g0))
        want = _hermite(P0, P1, l * g0, l * g1, np.arange(17) / 16)
        assert np.allclose(V[1:-1], want, rtol=0, atol=1e-9)
        checked += 1
    assert checked > 20


def test_polyline_length_converges_to_arc_length(orc):
    errs = []
    for K in (4, 8, 16, 32):
        sim, w = _spline_sim(orc, K=K, sigma=(3.0, 0.05, 0.05))
        e = []
        for row in range(0, sim.n_rows, 13):
            V = sim.path(row)
            if len(V) == 2:
                continue
            P0, P1 = V[1], V[-2]
            R = 2 * math.hypot(512 * 0.4, 512 * 0.4)
            g0, g1 = (V[1] - V[0]) / R, (V[-1] - V[-2]) / R
            l = float(np.dot(P1 - P0, g0))
            xg, wg = np.polynomial.legendre.leggauss(64)
            s = 0.5 * (xg + 1)
            d = 1e-6
            Hp = (_hermite(P0, P1, l * g0, l * g1, s + d) - _hermite(P0, P1, l * g0, l * g1, s - d)) / (2 * d)
            arc = 0.5 * np.sum(wg * np.linalg.norm(Hp, axis=1))
            poly = np.sum(np.linalg.norm(np.diff(V[1:-1], axis=0), axis=1))
            e.append(arc - poly)
        errs.append(np.mean(e))
    errs = np.array(errs)
    assert np.all(errs > 0)  # a chord polyline is never longer than the arc
    ratios = errs[:-1] / errs[1:]
    assert np.all((ratios > 3.0) & (ratios < 5.0)), ratios  # O(1/K^2)


def test_straight_lines_follow_the_beam_frame(orc):
    w = W.neo1_2d_straight(n_angles=8, paths_per_angle=20)
    ph = orc.Phantom(w["phantom"])
    sim = orc.Simulation(ph, ph.raster().astype(np.float32), w["angles"], 20, w["model"], w["seed"])
    for row in range(sim.n_rows):
        k = row // 20
        th = w["angles"][k]
        u = np.array([math.cos(th), math.sin(th)])
        t = np.array([-math.sin(th), math.cos(th)])
        u0 = (float(int(_numpy_block([w["seed"], 0], row, 0, 1)[0]) >> 11) + 0.5) * 2.0**-53
        toff = -100 + 200 * u0
        V = sim.path(row)[:, :2]
        assert len(V) == 2
        d = V[1] - V[0]
        assert abs(d[0] * u[1] - d[1] * u[0]) < 1e-9 * np.linalg.norm(d)  # along u
        assert np.dot(d, u) > 0
        assert abs(np.dot(V[0], t) - toff) < 1e-9 and abs(np.dot(V[1], t) - toff) < 1e-9


def test_mcs_exit_draws_are_bivariate_normal(orc):
    sig_lat, sig_out, rho = 1.0, 0.015, 0.6
    w = W.neo2_2d_spline(n_angles=4, paths_per_angle=3000)
    m = dict(w["model"])
    m.update(model=W.STRAIGHT_MCS, sigma_in=0.0, sigma_lat=sig_lat, sigma_out=sig_out, rho=rho)
    ph = orc.Phantom(w["phantom"])
    sim = orc.Simulation(ph, ph.raster().astype(np.float32), w["angles"], 3000, m, w["seed"])
    hull = w["phantom"]["regions"][0]
    R = 2 * math.hypot(204.8, 204.8)
    lats, angs = [], []
    for row in range(sim.n_rows):
        V = sim.path(row)[:, :2]
        if len(V) == 2:
            continue
        th = w["angles"][row // 3000]
        u = np.array([math.cos(th), math.sin(th)])
        t = np.array([-math.sin(th), math.cos(th)])
        toff = float(np.dot(V[1], t))  # entry point P0 lies on the incoming line
        # far intersection of that line with the hull ellipse (closed form)
        A = toff * t
        a2 = (u[0] / hull["a"][0]) ** 2 + (u[1] / hull["a"][1]) ** 2
        b1 = u[0] * A[0] / hull["a"][0] ** 2 + u[1] * A[1] / hull["a"][1] ** 2
        c0 = (A[0] / hull["a"][0]) ** 2 + (A[1] / hull["a"][1]) ** 2 - 1
        Q1 = A + (-b1 + math.sqrt(b1 * b1 - a2 * c0)) / a2 * u
        lats.append(float(np.dot(V[2] - Q1, t)))
        angs.append(float(np.dot((V[3] - V[2]) / R, t)))
    lats, angs = np.array(lats), np.array(angs)
    n = len(lats)
    assert n > 5000
    assert abs(lats.std() - sig_lat) < 4 * sig_lat / math.sqrt(2 * n)
    assert abs(angs.std() - sig_out) < 4 * sig_out / math.sqrt(2 * n)
    assert abs(np.corrcoef(lats, angs)[0, 1] - rho) < 4 * (1 - rho * rho) / math.sqrt(n)


def _independent_pairs(seed, stream, row, n_pairs):
    """The first n_pairs polar-method pairs of proton `row` (uniforms from 4 on),
    from numpy's Philox words and libm's log: independent of the oracle."""
    out, j, blocks = [], 4, {}

    def u(k):
        b = k >> 2
        if b not in blocks:
            blocks[b] = _numpy_block([seed, stream], row, b)
        return (float(int(blocks[b][k & 3]) >> 11) + 0.5) * 2.0**-53

    while len(out) < n_pairs:
        v1, v2 = 2 * u(j) - 1, 2 * u(j + 1) - 1
        j += 2
        s = v1 * v1 + v2 * v2
        if 0 < s < 1:
            f = math.sqrt(-2 * math.log(s) / s)
            out.append((v1 * f, v2 * f))
    return out


def _far_hull_point(P0, g, hull, dim):
    """Far intersection of the line P0 + mu g with the hull (closed form)."""
    a = np.array(hull["a"][:dim])
    c = np.array(hull["c"][:dim])
    e, f = g[:dim] / a, (P0[:dim] - c) / a
    A2, B1, C0 = e @ e, e @ f, f @ f - 1
    return P0 + (-B1 + math.sqrt(B1 * B1 - A2 * C0)) / A2 * g


def _mcs_3d_sim(orc, P, rho, sig=(1.0, 0.02, 0.015)):
    w = W.head_3d_spline(n_angles=6, paths_per_angle=P, n=(100, 100, 80), h=(2.0, 2.0, 2.0))
    m = dict(w["model"])
    m.update(model=W.STRAIGHT_MCS, sigma_lat=sig[0], sigma_in=sig[1], sigma_out=sig[2], rho=rho)
    ph = orc.Phantom(w["phantom"])
    sim = orc.Simulation(ph, ph.raster().astype(np.float32), w["angles"], P, m, w["seed"])
    R = 2 * math.sqrt(200.0 ** 2 + 200.0 ** 2 + 160.0 ** 2)
    return sim, w, R


def _mcs_3d_recover(V, th, R, hull):
    """Entry slopes (t, v) and exit pairs in the ut- and uv-planes of a 3D
    STRAIGHT_MCS path V = [P0 - R g0, P0, P1, P1 + R g1] (Sec. II-B)."""
    t = np.array([-math.sin(th), math.cos(th), 0.0])
    v = np.array([0.0, 0.0, 1.0])
    g0 = (V[1] - V[0]) / R
    g1 = (V[3] - V[2]) / R
    n_t = np.array([-g0[1], g0[0], 0.0])
    n_v = np.cross(g0, n_t)
    Q1 = _far_hull_point(V[1], g0, hull, 3)
    d, dg = V[2] - Q1, g1 - g0
    return {"in_t": float(g0 @ t), "in_v": float(g0 @ v),
            "lat_t": float(d @ n_t / (n_t @ n_t)), "lat_v": float(d @ n_v / (n_v @ n_v)),
            "ang_t": float(dg @ n_t / (n_t @ n_t)), "ang_v": float(dg @ n_v / (n_v @ n_v))}


def test_mcs_3d_draws_equal_independent_draws(orc):
    """Every draw of a 3D MCS proton, recovered from its path geometry, equals
    the same draw recomputed outside the oracle: exit (displacement, slope) in
    the ut-plane from pair 1, in the uv-plane (along n_v = g0 x n_t) from pair
    2, entry slopes along t and v from pair 3 (Sec. II-B, bivariate normal)."""
    sig_lat, sig_in, sig_out, rho = 1.0, 0.02, 0.015, 0.4
    sim, w, R = _mcs_3d_sim(orc, 40, rho, (sig_lat, sig_in, sig_out))
    hull = w["phantom"]["regions"][0]
    rc = math.sqrt(1 - rho * rho)
    checked = 0
    for row in range(sim.n_rows):
        V = sim.path(row)
        (a1, a2), (b1, b2), (c1, c2) = _independent_pairs(w["seed"], 0, row, 3)
        th = w["angles"][row // 40]
        if len(V) == 2:  # missed the hull: only the entry slopes shape the line
            g0 = (V[1] - V[0]) / (2 * R)
            assert abs(g0 @ np.array([-math.sin(th), math.cos(th), 0]) - sig_in * c1) < 1e-12
            assert abs(g0[2] - sig_in * c2) < 1e-12
            continue
        got = _mcs_3d_recover(V, th, R, hull)
        want = {"lat_t": sig_lat * a1, "ang_t": sig_out * (rho * a1 + rc * a2),
                "lat_v": sig_lat * b1, "ang_v": sig_out * (rho * b1 + rc * b2),
                "in_t": sig_in * c1, "in_v": sig_in * c2}
        for k in want:
            tol = 1e-9 if k.startswith("lat") else 1e-11
            assert abs(got[k] - want[k]) < tol, (row, k, got[k], want[k])
        checked += 1
    assert checked > 150


def test_mcs_3d_exit_pairs_and_entry_slopes_statistics(orc):
    """The 3D draws have the requested sigmas, the correlation rho within each
    plane, none across planes, and independent entry slopes (Sec. II-B: MCS in
    the ut- and uv-planes)."""
    sig_lat, sig_in, sig_out, rho = 1.5, 0.02, 0.01, -0.5
    P = 1600
    sim, w, R = _mcs_3d_sim(orc, P, rho, (sig_lat, sig_in, sig_out))
    hull = w["phantom"]["regions"][0]
    rec = []
    for row in range(sim.n_rows):
        V = sim.path(row)
        if len(V) == 4:
            rec.append(_mcs_3d_recover(V, w["angles"][row // P], R, hull))
    n = len(rec)
    assert n > 5000
    col = {k: np.array([r[k] for r in rec]) for k in rec[0]}
    for k, s in (("lat_t", sig_lat), ("lat_v", sig_lat), ("ang_t", sig_out), ("ang_v", sig_out),
                 ("in_t", sig_in), ("in_v", sig_in)):
        assert abs(col[k].mean()) < 4 * s / math.sqrt(n), k
        assert abs(col[k].std() - s) < 4 * s / math.sqrt(2 * n), k
    tol = 4 * (1 - rho * rho) / math.sqrt(n)
    assert abs(np.corrcoef(col["lat_t"], col["ang_t"])[0, 1] - rho) < tol
    assert abs(np.corrcoef(col["lat_v"], col["ang_v"])[0, 1] - rho) < tol
    for a, b in (("lat_t", "lat_v"), ("ang_t", "ang_v"), ("lat_t", "ang_v"), ("in_t", "in_v"),
                 ("in_t", "lat_t"), ("in_v", "lat_v")):
        assert abs(np.corrcoef(col[a], col[b])[0, 1]) < 4 / math.sqrt(n), (a, b)


def test_entry_slopes_2d_statistics(orc):
    """2D: the entry slope recovered from the incoming line against u has
    sigma_in (the MCS statistics tests above it set sigma_in = 0)."""
    sig_in = 0.03
    w = W.neo2_2d_spline(n_angles=4, paths_per_angle=2500)
    m = dict(w["model"])
    m.update(model=W.STRAIGHT_MCS, sigma_in=sig_in)
    ph = orc.Phantom(w["phantom"])
    sim = orc.Simulation(ph, ph.raster().astype(np.float32), w["angles"], 2500, m, w["seed"])
    R = 2 * math.hypot(204.8, 204.8)
    sl = []
    for row in range(sim.n_rows):
        V = sim.path(row)[:, :2]
        th = w["angles"][row // 2500]
        u = np.array([math.cos(th), math.sin(th)])
        t = np.array([-math.sin(th), math.cos(th)])
        g0 = (V[1] - V[0]) / (R if len(V) == 4 else 2 * R)
        assert abs(g0 @ u - 1) < 1e-12  # g0 = u + slope t, not normalised
        sl.append(float(g0 @ t))
    sl = np.array(sl)
    n = len(sl)
    assert abs(sl.mean()) < 4 * sig_in / math.sqrt(n)
    assert abs(sl.std() - sig_in) < 4 * sig_in / math.sqrt(2 * n)


# --------------------------------------------------------------------------
# WEPL (Sec. II-C: b_i = <a_i, x_true>, optional noise)
# --------------------------------------------------------------------------
def test_wepl_homogeneous_phantom_equals_rsp_times_length(orc):
    desc = _disc_phantom(2, (64, 48), (1.0, 1.0), [{"c": (0, 0, 0), "a": (1e4, 1e4, 1e4), "rsp": 1.04}],
                         W.CORNER)
    ph = orc.Phantom(desc)
    x = ph.raster().astype(np.float32)
    assert np.all(x == np.float32(1.04))
    m = W.model(W.STRAIGHT, (-40.0, 40.0))
    sim = orc.Simulation(ph, x, W.angles(30), 40, m, 17)
    for row in range(0, sim.n_rows, 3):
        cols, vals, bc, bn = sim.row(row)
        V = sim.path(row)[:, :2]
        L = _clip_length(V[0], V[1], np.array([-32.0, -24.0]), np.array([32.0, 24.0]))
        L = L if isinstance(L, float) else L[0]
        assert abs(bc - float(np.float32(1.04)) * L) <= 1e-12 * max(L, 1)
        assert bn == bc


@pytest.mark.parametrize("h", [1.0, 0.5, 0.25])
def test_wepl_layered_ellipses_converges(orc, h):
    regs = [{"c": (0, 0, 0), "a": (80, 60, 1), "rsp": 1.0},
            {"c": (0, 0, 0), "a": (50, 40, 1), "rsp": 2.0}]
    n = int(200 / h)
    ph = orc.Phantom(_disc_phantom(2, (n, n), (h, h), regs, W.CENTER))
    x = ph.raster().astype(np.float32)
    m = W.model(W.STRAIGHT, (-90.0, 90.0))
    ang = W.angles(16)
    sim = orc.Simulation(ph, x, ang, 25, m, 23)
    errs = []
    for row in range(sim.n_rows):
        V = sim.path(row)[:, :2]
        d = (V[1] - V[0]) / np.linalg.norm(V[1] - V[0])
        toff = V[0][0] * (-d[1]) + V[0][1] * d[0]

        def chord(a, b):
            # chord of the line {toff * t_hat + s * d} through the ellipse (a, b)
            A = np.array([-d[1], d[0]]) * toff
            a2 = (d[0] / a) ** 2 + (d[1] / b) ** 2
            b1 = d[0] * A[0] / a ** 2 + d[1] * A[1] / b ** 2
            c0 = (A[0] / a) ** 2 + (A[1] / b) ** 2 - 1
            disc = b1 * b1 - a2 * c0
            return 2 * math.sqrt(disc) / a2 if disc > 0 else 0.0

        want = 1.0 * chord(80, 60) + (2.0 - 1.0) * chord(50, 40)
        _, _, bc, _ = sim.row(row)
        errs.append(abs(bc - want))
        # each of the <= 4 boundary crossings misassigns at most ~2 pixels' chords
        assert abs(bc - want) <= 4 * 2 * 2.0 * h * math.sqrt(2)
    test_wepl_layered_ellipses_converges.errs = getattr(test_wepl_layered_ellipses_converges, "errs", {})
    test_wepl_layered_ellipses_converges.errs[h] = float(np.mean(errs))
    e = test_wepl_layered_ellipses_converges.errs
    if 1.0 in e and 0.25 in e:
        assert e[0.25] < 0.5 * e[1.0]  # first order in h


def test_noise_statistics(orc):
    w = W.neo2_2d_spline(n_angles=20, paths_per_angle=1500, n=128, h=1.6)
    res = orc.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"],
                       threads=4)
    bc, bn = res["b_clean"], res["b"]
    r = (bn[bc > 1] / bc[bc > 1]) - 1
    assert len(r) > 20000
    assert abs(r.mean()) < 4 * 0.01 / math.sqrt(len(r))
    assert abs(r.std() - 0.01) < 0.0005
    assert np.all(bn[bc == 0] == 0)


# --------------------------------------------------------------------------
# Weighted-area raster (Sec. II-A, the third raster option)
# --------------------------------------------------------------------------
def test_area_raster_one_sample_is_the_centre_raster(orc):
    for dim, n, h in ((2, (40, 30), (2.5, 3.0)), (3, (20, 18, 12), (5.0, 6.0, 7.0))):
        base = W.phantom(dim, n, h, skin=True)
        cen = orc.Phantom(dict(base, raster=W.CENTER)).raster()
        ar = orc.Phantom(dict(base, raster=W.AREA, area_samples=1)).raster()
        assert np.array_equal(cen, ar)


def test_area_raster_interior_pixels_are_exact(orc):
    desc = _disc_phantom(2, (64, 64), (1.0, 1.0), [{"c": (0, 0, 0), "a": (20, 12, 1), "rsp": 1.04}], W.AREA)
    x = orc.Phantom(dict(desc, area_samples=8)).raster().reshape(64, 64)
    # pixel [iy, ix] covers [ix - 32, ix - 31) x [iy - 32, iy - 31)
    assert x[32, 32] == 1.04 and x[32 + 5, 32 - 6] == 1.04  # wholly inside
    assert x[0, 0] == 0.0
    edge = x[32 + 3, 32 + 19]  # pixel [19, 20) x [3, 4): the boundary (x = 19.1 at y = 3.5) crosses it
    assert 0.0 < edge < 1.04


@pytest.mark.parametrize("dim", [2, 3])
def test_area_raster_converges_to_area_and_volume(orc, dim):
    a = (20.0, 12.0, 9.0)
    if dim == 2:
        desc = _disc_phantom(2, (48, 32), (1.0, 1.0), [{"c": (0.3, -0.2, 0), "a": a, "rsp": 1.0}], W.AREA)
        exact, cell = math.pi * a[0] * a[1], 1.0
    else:
        desc = _disc_phantom(3, (48, 32, 24), (1.0, 1.0, 1.0), [{"c": (0.3, -0.2, 0.1), "a": a, "rsp": 1.0}], W.AREA)
        exact, cell = 4.0 / 3.0 * math.pi * a[0] * a[1] * a[2], 1.0
    errs = []
    for S in (1, 2, 4, 8):
        x = orc.Phantom(dict(desc, area_samples=S)).raster()
        errs.append(abs(x.sum() * cell - exact) / exact)
    assert errs[-1] < 1e-4, errs  # S = 8: 5.9e-5 (2D), 1.7e-5 (3D)
    assert errs[-1] < errs[1], errs
