"""The synthetic inputs that stand in for the paper's experiments: values the
paper fixes for the rip-channel beach of Sec. 5.4 (Eq. 48)."""
import math

import numpy as np

from paper_1909_04153_gb300 import workloads as W


def test_eq48_plane_beach_and_channel():
    # away from the channel (y = +-15 m, cos^10 = 0) Eq. 48 is the plane beach
    # z = 0.1 - (18 - x) / 30: 1:30 slope, shoreline at x = 15 m, 0.5 m of
    # water at the maker
    x = np.linspace(0.0, 20.0, 11)
    for y in (-15.0, 15.0):
        np.testing.assert_allclose(W.hamm_rip_bed(x, y), 0.1 - (18.0 - x) / 30.0, atol=1e-15)
    assert abs(W.hamm_rip_bed(15.0, 15.0)) < 1e-15
    # at x = 18 m the bed is at +0.1 m whatever y
    np.testing.assert_allclose(W.hamm_rip_bed(18.0, np.linspace(-15, 15, 7)), 0.1, atol=1e-15)
    # on the channel centre line the deepening is 3 exp(-(18 - x)/3) times the plane depth term
    for xv in (6.0, 12.0, 16.5):
        s = 18.0 - xv
        assert abs(W.hamm_rip_bed(xv, 0.0) - (0.1 - s / 30.0 * (1.0 + 3.0 * math.exp(-s / 3.0)))) < 1e-15
    # the channel is symmetric about its centre line
    y = np.linspace(0.0, 15.0, 9)
    np.testing.assert_allclose(W.hamm_rip_bed(10.0, y), W.hamm_rip_bed(10.0, -y), atol=1e-15)


def test_hamm_rip_case():
    c = W.hamm_rip(nx=100, ny=60)
    p = c["params"]
    assert p["dx"] == 0.2 and p["dy"] == 0.5 and p["friction"] == 0.0025 and p["dt_init"] == 0.003
    assert p["bc"] == (W.MAKER, W.WALL, W.WALL, W.WALL)
    assert c["bed"].shape == (61, 101)
    comps = c["comps"]
    assert comps.shape == (68, 4)
    np.testing.assert_allclose(np.diff(comps[:, 1]), 0.01, atol=1e-12)
    # 4 sqrt(m0) = Hs
    assert abs(4.0 * math.sqrt(0.5 * np.sum(comps[:, 0] ** 2)) - 0.13) < 1e-12


def test_conical_island_geometry():
    # Sec. 5.1: 30 m x 30 m basin, 601 x 601 cells, 0.32 m of water, an island of
    # 7.2 m base diameter and side slope 1/4 at the centre; its still-water
    # shoreline is then a circle of radius 3.6 - 4 (0.32) = 2.32 m (the radius the
    # paper scales run-up by); solitary wave of H/d = 0.18; sponges W and E,
    # walls S and N
    c = W.conical_island()
    p = c["params"]
    assert p["nx"] == 601 and p["ny"] == 601 and abs(p["dx"] * 601 - 30.0) < 1e-12
    assert p["bc"] == (W.SPONGE, W.SPONGE, W.WALL, W.WALL) and p["friction"] == 0.0
    bed = c["bed"]
    xk = np.arange(602) * p["dx"]
    X, Y = np.meshgrid(xk, xk)
    r = np.hypot(X - 15.0, Y - 15.0)
    assert np.all(bed[r >= 3.6] == -0.32)
    inside = (r < 3.6) & (r > 0.1)
    np.testing.assert_allclose(bed[inside], -0.32 + (3.6 - r[inside]) / 4.0, atol=1e-14)
    # the shoreline: bed crosses 0 at r = 2.32 m
    ring = np.abs(r - 2.32) < 0.5 * p["dx"]
    assert np.all(np.abs(bed[ring]) <= 0.25 * 0.5 * p["dx"] + 1e-12)
    # solitary wave: crest 0.18 x 0.32 m, travelling east (P = c eta > 0)
    assert abs(c["eta0"].max() - 0.18 * 0.32) < 1e-3 * 0.0576
    assert np.all(c["P0"] >= 0.0) and c["Q0"] is None
    np.testing.assert_allclose(c["P0"] / np.maximum(c["eta0"], 1e-300),
                               math.sqrt(9.81 * (0.32 + 0.0576)), rtol=1e-12,
                               atol=0.0, err_msg="flux = celerity x eta")
