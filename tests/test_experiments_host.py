"""Host-side analysis of the droplet experiments (no GPU): the periodic
droplet counter against the oracle's breadth-first count, the pressure jump
of a synthetic two-level field, and the probe sites of Fig. 3."""
import numpy as np
import pytest

from oracle import two_component as tc

pytest.importorskip("scipy")

from paper_2301_01622_gb300 import experiments as ex  # noqa: E402


@pytest.mark.parametrize("seed", range(6))
def test_periodic_count_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in rng.integers(4, 12, size=3))
    field = rng.uniform(0.0, 1.0, size=shape)
    for thr in (0.5, 0.7, 0.85):
        assert ex.count_droplets(field, thr) == tc.count_droplets(field, thr)


def test_periodic_count_wraps_every_axis():
    a = np.zeros((8, 9, 10))
    a[0, 3, 3] = a[7, 3, 3] = 1          # across z
    a[4, 0, 5] = a[4, 8, 5] = 1          # across y
    a[2, 2, 0] = a[2, 2, 9] = 1          # across x
    assert ex.count_droplets(a) == 3 == tc.count_droplets(a)


def test_pressure_jump_of_two_level_field():
    n, R = 32, 8.0
    rho1, rho2, _ = ex.inputs.droplets(n, n, n, [(16, 16, 16)], [R], [(0, 0, 0)])
    m = np.zeros((11, n, n, n))
    m[0], m[1] = rho1 * 1.03, rho2       # inside: total density 1.03, outside 1.0
    assert abs(ex.pressure_jump(m, (16, 16, 16), R) - 0.03 / 3.0) < 1e-6


def test_probe_sites():
    assert ex.probe_sites((128, 128, 128)) == [(31, 63, 63), (63, 63, 63), (127, 127, 127)]
    assert ex.probe_sites((64, 64, 64)) == [(15, 31, 31), (31, 31, 31), (63, 63, 63)]
