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
