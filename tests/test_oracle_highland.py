"""Pins of the oracle's Highland / PDG multiple-scattering widths (Sec. II-B:
the exit displacement and angle come from the Highland formula with the PDG
constants, drawn as a bivariate normal).

- kinematics: beta c p from T by the gamma / beta route, independent of the
  oracle's (pc)^2 / E route;
- the formula's shape: theta0 beta c p / (13.6 sqrt(x / X0)) - 1 grows as
  0.038 ln x (a change of x by a factor k adds 0.038 ln k) and vanishes at
  x = X0 beta^2;
- the draws: exit pairs of 3D STRAIGHT_MCS protons, recovered from their
  paths and divided by the widths of their chords, have unit sigmas and the
  thin-slab correlation sqrt(3) / 2 in both planes."""
import math

import numpy as np
import pytest

from paper_2108_12369_gb300 import workloads as W
from tests.test_oracle_pins import _far_hull_point, _mcs_3d_recover

MP = 938.272088  # proton mass, MeV (PDG)


@pytest.mark.parametrize("T", [70.0, 150.0, 200.0, 230.0, 1000.0])
def test_kinematics_by_the_gamma_beta_route(orc, T):
    gamma = 1.0 + T / MP
    beta2 = 1.0 - 1.0 / (gamma * gamma)
    bcp = gamma * MP * beta2  # beta c p = gamma m beta^2 c^2
    _, got = orc.highland(T, 360.8, 100.0)
    assert abs(got - bcp) <= 1e-12 * bcp


def test_formula_shape(orc):
    T, X0 = 200.0, 360.8
    _, bcp = orc.highland(T, X0, 1.0)
    gamma = 1.0 + T / MP
    beta2 = 1.0 - 1.0 / (gamma * gamma)

    def corr(x):
        th, _ = orc.highland(T, X0, x)
        return th * bcp / (13.6 * math.sqrt(x / X0)) - 1.0

    for x, k in ((10.0, 2.0), (50.0, 4.0), (200.0, 0.5), (3.0, 10.0)):
        assert abs((corr(k * x) - corr(x)) - 0.038 * math.log(k)) < 1e-12
    assert abs(corr(X0 * beta2)) < 1e-12
    # 200 MeV after 20 cm of water: 28.3 mrad (constant-energy Highland)
    assert abs(orc.highland(T, X0, 200.0)[0] - 0.02833) < 5e-5


def test_highland_draws_normalised_3d(orc):
    P = 1600
    w = W.head_3d_spline(n_angles=6, paths_per_angle=P, n=(100, 100, 80), h=(2.0, 2.0, 2.0))
    m = W.model(W.STRAIGHT_MCS, w["model"]["t_range"], w["model"]["v_range"], sigma_in=0.01,
                mcs=W.MCS_HIGHLAND, beam_mev=200.0)
    ph = orc.Phantom(w["phantom"])
    sim = orc.Simulation(ph, ph.raster().astype(np.float32), w["angles"], P, m, w["seed"])
    R = 2 * math.sqrt(200.0 ** 2 + 200.0 ** 2 + 160.0 ** 2)
    hull = w["phantom"]["regions"][0]
    nl, na = {"t": [], "v": []}, {"t": [], "v": []}
    for row in range(sim.n_rows):
        V = sim.path(row)
        if len(V) != 4:
            continue
        rec = _mcs_3d_recover(V, w["angles"][row // P], R, hull)
        g0 = (V[1] - V[0]) / R
        x = float(np.linalg.norm(_far_hull_point(V[1], g0, hull, 3) - V[1]))  # chord through the hull
        th, _ = orc.highland(200.0, W.X0_WATER_MM, x)
        for p in ("t", "v"):
            nl[p].append(rec["lat_" + p] / (x * th / math.sqrt(3.0)))
            na[p].append(rec["ang_" + p] / th)
    n = len(nl["t"])
    assert n > 5000
    rho = math.sqrt(3.0) / 2
    for p in ("t", "v"):
        a, b = np.array(nl[p]), np.array(na[p])
        assert abs(a.std() - 1) < 4 / math.sqrt(2 * n) and abs(b.std() - 1) < 4 / math.sqrt(2 * n)
        assert abs(np.corrcoef(a, b)[0, 1] - rho) < 4 * (1 - rho * rho) / math.sqrt(n)
    assert abs(np.corrcoef(nl["t"], nl["v"])[0, 1]) < 4 / math.sqrt(n)
