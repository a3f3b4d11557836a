"""Pins of the oracle's diagnostics (Sec. IV, Figs. 2, 3, 5, 7) on fields whose
answers are known in closed form."""
import math

import numpy as np

from oracle import diagnostics as dg


def test_two_level_field():
    """Half the nodes at rho1 = 0.8, half at 0.2: <rho1>_{rho1>0.5} = 0.8, count = N/2."""
    nz, ny, nx = 4, 6, 8
    m = np.zeros((11, nz, ny, nx))
    m[0] = 0.2
    m[0, :, :, : nx // 2] = 0.8
    m[1] = 1.0 - m[0]
    m[2] = 0.01
    d = dg.diagnostics(m, ncomp=2)
    n = nz * ny * nx
    assert d["n_in"] == n // 2
    assert abs(d["rho1_avg"] - 0.8) < 1e-15
    assert d["mass"][0] == math.fsum([0.8] * (n // 2) + [0.2] * (n // 2))
    assert abs(d["mass"][0] + d["mass"][1] - n) < 1e-12
    assert abs(d["momentum"][0] - 0.01 * n) < 1e-13
    assert d["min_rho"] == 1.0 and d["flags"] == 0


def test_threshold_is_strict_and_flags():
    m = np.zeros((10, 2, 2, 2))
    m[0] = 0.5
    m[0, 0, 0, 0] = 0.75
    d = dg.diagnostics(m, ncomp=1)
    assert d["n_in"] == 1 and d["rho1_avg"] == 0.75
    m[0, 1, 1, 1] = -0.1
    assert dg.diagnostics(m, ncomp=1)["flags"] == dg.FLAG_NONPOSITIVE
    m[3, 0, 1, 0] = np.nan
    assert dg.diagnostics(m, ncomp=1)["flags"] & dg.FLAG_NONFINITE


def test_probe_sites_and_local_error():
    """Fig. 3 sites: 1-based (32,64,64), (64,64,64), (128,128,128) in a 128 box."""
    assert dg.probe_sites((128, 128, 128)) == [(31, 63, 63), (63, 63, 63), (127, 127, 127)]
    assert dg.probe_sites((192, 192, 384)) == [(95, 95, 95), (191, 95, 95), (383, 191, 191)]
    a = np.ones((4, 4, 4))
    b = a.copy()
    a[3, 3, 3] = 2.0
    b[3, 3, 3] = 1.5
    assert dg.local_relative_error(a, b, [(3, 3, 3), (0, 0, 0)]) == [0.25, 0.0]
