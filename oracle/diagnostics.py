"""Field diagnostics of the validation section, FP64 (test infrastructure only).

* total mass per component and total momentum (conserved by BGK collision and
  periodic streaming, Eqs. (7) and (9));
* the droplet density <rho>_{rho > 0.5}: the mean of rho over the nodes where
  rho > 0.5 (strict), Sec. IV, Figs. 2, 5, 7.  For two components the
  averaged field is the droplet component rho^1 (the colour maps of Figs. 1,
  4, 6 range from 0 to 1);
* the minimum total density and a flag for non-finite values (stability
  monitor; not in the paper).
* the local relative error |rho_N - rho_P| / max(rho_N) between a run
  without and a run with populations at probe sites, Sec. IV, Fig. 3.

Sums use math.fsum, so they are correctly rounded and independent of order.
"""
from __future__ import annotations

import math

import numpy as np

FLAG_NONFINITE = 1
FLAG_NONPOSITIVE = 2


def diagnostics(m: np.ndarray, ncomp: int = 1) -> dict:
    """Diagnostics of canonical moments.

    ncomp=1: m has 10 fields (rho, j, P); the droplet average uses rho.
    ncomp=2: m has 11 fields (rho1, rho2, j, P); total rho = rho1 + rho2 and
    the droplet average uses rho1.
    """
    m = np.asarray(m, dtype=np.float64)
    if ncomp == 1:
        rho_c = [m[0]]
        j = m[1:4]
    elif ncomp == 2:
        rho_c = [m[0], m[1]]
        j = m[2:5]
    else:
        raise ValueError("ncomp must be 1 or 2")
    rho = rho_c[0] if ncomp == 1 else rho_c[0] + rho_c[1]
    mass = [math.fsum(r.ravel()) for r in rho_c] + [0.0] * (2 - ncomp)
    momentum = [math.fsum(j[a].ravel()) for a in range(3)]
    drop = rho_c[0]
    sel = drop > 0.5
    n_in = int(np.count_nonzero(sel))
    s_in = math.fsum(drop[sel].ravel())
    finite = bool(np.all(np.isfinite(m)))
    min_rho = float(np.min(rho)) if finite else float("nan")
    flags = 0
    if not finite:
        flags |= FLAG_NONFINITE
    if finite and min_rho <= 0.0:
        flags |= FLAG_NONPOSITIVE
    return {
        "mass": mass,
        "momentum": momentum,
        "rho1_sum": s_in,
        "n_in": n_in,
        "rho1_avg": (s_in / n_in) if n_in else 0.0,
        "min_rho": min_rho,
        "flags": flags,
    }


def probe_sites(shape_zyx, reference_box: int = 128):
    """The three probe sites of Fig. 3, scaled to the box.

    The caption prints (32,64,64), (64,64,64) and (128,128,128) in a box of
    128 nodes per side; read as 1-based indices they become 0-based
    (31,63,63), (63,63,63), (127,127,127), then scaled by L/128 per axis.
    Returned as (x, y, z) tuples.
    """
    nz, ny, nx = shape_zyx
    sites = []
    for p in ((32, 64, 64), (64, 64, 64), (128, 128, 128)):
        sx = (p[0] * nx) // reference_box - 1
        sy = (p[1] * ny) // reference_box - 1
        sz = (p[2] * nz) // reference_box - 1
        sites.append((max(sx, 0), max(sy, 0), max(sz, 0)))
    return sites


def local_relative_error(rho_n: np.ndarray, rho_p: np.ndarray, sites) -> list:
    """|rho_N - rho_P| / max(rho_N) at each (x, y, z) site (Sec. IV, Fig. 3)."""
    rmax = float(np.max(rho_n))
    return [abs(float(rho_n[z, y, x]) - float(rho_p[z, y, x])) / rmax for (x, y, z) in sites]
