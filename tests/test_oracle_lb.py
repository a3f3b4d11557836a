"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: lattice
isotropy identities, a textbook form of the equilibrium, closed-form
one-step results, an exact Navier-Stokes decay rate (nu = cs^2 (tau - 1/2),
Sec. III B), Galilean advection, a linear amplification matrix derived
independently, conservation laws, and the population-storing form of the
same scheme.  A dropped term, wrong sign, wrong index or transposed operand
in the oracle's Eq. (4)/(8)/(9)/(1)-(3) fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import CS2, D3Q19, D3Q27, lb
from paper_2301_01622_gb300 import inputs

LATTICES = [D3Q19, D3Q27]
IDS = ["D3Q19", "D3Q27"]


def _delta(a, b):
    return 1.0 if a == b else 0.0


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_lattice_isotropy(lat):
    """Sum w = 1, odd moments vanish, 2nd = cs^2 delta, 4th = cs^4 (dd + dd + dd)."""
    c = lat.c.astype(float)
    w = lat.w
    assert abs(w.sum() - 1.0) < 1e-15
    for a in range(3):
        assert abs((w * c[:, a]).sum()) < 1e-15
    for a, b in itertools.product(range(3), repeat=2):
        assert abs((w * c[:, a] * c[:, b]).sum() - CS2 * _delta(a, b)) < 1e-15
    for a, b, g in itertools.product(range(3), repeat=3):
        assert abs((w * c[:, a] * c[:, b] * c[:, g]).sum()) < 1e-15
    for a, b, g, d in itertools.product(range(3), repeat=4):
        iso = CS2 * CS2 * (_delta(a, b) * _delta(g, d) + _delta(a, g) * _delta(b, d) + _delta(a, d) * _delta(b, g))
        assert abs((w * c[:, a] * c[:, b] * c[:, g] * c[:, d]).sum() - iso) < 1e-15
    # velocity set closed under inversion, distinct
    assert len({tuple(v) for v in lat.c}) == lat.Q
    assert {tuple(v) for v in lat.c} == {tuple(-v) for v in lat.c}


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_reconstruction_reproduces_moments(lat):
    """P R H = H: the reconstruction keeps exactly the ten moments (Sec. II, g = 0)."""
    m = inputs.random_moments(5, 4, 3, seed=7)
    back = lb.project(lb.reconstruct(m, lat), lat)
    np.testing.assert_allclose(back, m, rtol=0, atol=1e-14)


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_equilibrium_matches_textbook_expansion(lat):
    """h^eq of Eq. (5) equals the textbook second-order equilibrium
    w rho [1 + c.u/cs^2 + (c.u)^2/(2 cs^4) - u^2/(2 cs^2)], and its moments are
    (rho, rho u, cs^2 rho I + rho u u)."""
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.9, 1.1, size=(2, 2, 3))
    u = rng.uniform(-0.1, 0.1, size=(3, 2, 2, 3))
    m = lb.equilibrium_moments(rho, u)
    fl = lb.LocalFields(m)
    for i in range(lat.Q):
        c = lat.c[i].astype(float)
        cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
        usq = (u * u).sum(axis=0)
        textbook = lat.w[i] * rho * (1 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - usq / (2 * CS2))
        # P = P^eq: no non-equilibrium part, so Eq. (4) is h^eq alone
        np.testing.assert_allclose(lb.reconstruct_direction(fl, lat, i, None), textbook, rtol=0, atol=1e-15)
    f = np.stack([lb.reconstruct_direction(fl, lat, i, None) for i in range(lat.Q)])
    mom = lb.project(f, lat)
    # hand values: P_xx = rho (1/3 + u_x^2), P_xy = rho u_x u_y
    np.testing.assert_allclose(mom[4], rho * (1.0 / 3.0 + u[0] ** 2), atol=1e-15)
    np.testing.assert_allclose(mom[7], rho * u[0] * u[1], atol=1e-15)
    np.testing.assert_allclose(mom[1], rho * u[0], atol=1e-15)


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_coll2_literal_equals_moment_form(lat, tau):
    """Eq. (8) written literally equals the linear moment form
    h'_i = w_i [rho + 3 c.j + 4.5 c c : A' - 1.5 tr A'],
    A' = (1 - omega)(P - cs^2 rho I) + omega j j / rho  (the u u terms cancel)."""
    m = inputs.random_moments(4, 3, 2, seed=11)
    omega = 1.0 / tau
    rho = m[0]
    j = m[1:4]
    P = lb.tensor_from_fields(m[4:10])
    A = [[(1 - omega) * (P[a][b] - CS2 * rho * _delta(a, b)) + omega * j[a] * j[b] / rho for b in range(3)]
         for a in range(3)]
    trA = A[0][0] + A[1][1] + A[2][2]
    fl = lb.LocalFields(m)
    for i in range(lat.Q):
        c = lat.c[i]
        cj = c[0] * j[0] + c[1] * j[1] + c[2] * j[2]
        ccA = sum(c[a] * c[b] * A[a][b] for a in range(3) for b in range(3))
        ref = lat.w[i] * (rho + 3 * cj + 4.5 * ccA - 1.5 * trA)
        np.testing.assert_allclose(lb.reconstruct_direction(fl, lat, i, omega), ref, rtol=0, atol=5e-16)


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_collided_moments_closed_form(lat):
    """Moments of h' (Eq. (8)): rho and j unchanged, P' = P^eq + (1 - omega)(P - P^eq)."""
    m = inputs.random_moments(3, 3, 3, seed=5)
    tau = 0.7
    omega = 1.0 / tau
    got = lb.project(lb.reconstruct(m, lat, omega), lat)
    rho = m[0]
    u = m[1:4] / rho
    for k, (a, b) in enumerate(lb.PAIRS):
        peq = rho / 3.0 * _delta(a, b) + rho * u[a] * u[b]
        np.testing.assert_allclose(got[4 + k], peq + (1 - omega) * (m[4 + k] - peq), atol=2e-15)
    np.testing.assert_allclose(got[:4], m[:4], atol=2e-15)


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_uniform_state_relaxes_by_one_minus_omega(lat):
    """A uniform state with non-equilibrium P: streaming is the identity, so one
    step multiplies P - P^eq by exactly (1 - omega) and keeps rho, j."""
    n = 3
    rho0, u0 = 1.02, np.array([0.03, -0.02, 0.01])
    pneq = np.array([0.004, -0.002, 0.001, 0.0015, -0.0007, 0.0003])
    m = np.empty((10, n, n, n))
    m[0] = rho0
    m[1:4] = (rho0 * u0)[:, None, None, None]
    for k, (a, b) in enumerate(lb.PAIRS):
        m[4 + k] = rho0 / 3.0 * _delta(a, b) + rho0 * u0[a] * u0[b] + pneq[k]
    for tau in (0.55, 0.8, 1.0, 1.9):
        out = lb.step_moment_only(m, lat, tau)
        for k, (a, b) in enumerate(lb.PAIRS):
            expect = rho0 / 3.0 * _delta(a, b) + rho0 * u0[a] * u0[b] + (1 - 1 / tau) * pneq[k]
            np.testing.assert_allclose(out[4 + k], expect, rtol=0, atol=1e-15)
        np.testing.assert_allclose(out[:4], m[:4], rtol=0, atol=1e-15)


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_point_perturbation_one_step_by_hand(lat):
    """Rest fluid (P = cs^2 rho I, j = 0) with rho = 1 + delta at one node of a 4^3 box.

    By hand: every source emits h'_i = w_i rho, so after one step the node
    x0 + c_i holds rho = 1 + w_i delta, j = w_i delta c_i,
    P = cs^2 I + w_i delta c_i c_i, and every other node is unchanged."""
    delta = 0.1
    x0 = (1, 2, 1)
    rho, u = inputs.point_perturbation(4, 4, 4, at=x0, delta=delta)
    m = lb.equilibrium_moments(rho, u)
    out = lb.step_moment_only(m, lat, tau=0.77)
    seen = np.zeros((4, 4, 4), dtype=bool)
    for i in range(lat.Q):
        c = lat.c[i]
        x, y, z = ((x0[0] + c[0]) % 4, (x0[1] + c[1]) % 4, (x0[2] + c[2]) % 4)
        seen[z, y, x] = True
        w = lat.w[i]
        assert abs(out[0, z, y, x] - (1 + w * delta)) < 1e-15
        for a in range(3):
            assert abs(out[1 + a, z, y, x] - w * delta * c[a]) < 1e-16
        for k, (a, b) in enumerate(lb.PAIRS):
            assert abs(out[4 + k, z, y, x] - (_delta(a, b) / 3.0 + w * delta * c[a] * c[b])) < 1e-15
    rest = ~seen
    np.testing.assert_allclose(out[0][rest], 1.0, atol=1e-15)
    np.testing.assert_allclose(out[1:4][:, rest], 0.0, atol=1e-16)


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_moment_only_equals_regularized_population(lat):
    """The moment-only scheme and the population-storing regularized LB are the
    same map (the reconstruction keeps the ten moments): 1e-12 after 200 steps
    on the 32^3 Taylor-Green vortex, tau = 0.8."""
    n = 32 if lat.Q == 19 else 16
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05)
    m0 = lb.equilibrium_moments(rho, u)
    m = lb.run_moment_only(m0, lat, 0.8, 200)
    f = lb.run_population(lb.populations_from_moments(m0, lat), lat, 0.8, 200, "regularized")
    mp = lb.project(f, lat)
    for k in range(10):
        assert np.abs(m[k] - mp[k]).max() <= 1e-12 * max(np.abs(mp[k]).max(), 1e-3)


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_bgk_equals_moment_only_at_tau_one(lat):
    """At tau = 1 BGK sets f' = f^eq, which has no ghost part: BGK with stored
    populations, the regularized scheme and the moment-only scheme coincide."""
    m0 = inputs.random_moments(6, 5, 4, seed=9)
    f = lb.populations_from_moments(m0, lat)
    fb = lb.run_population(f, lat, 1.0, 5, "bgk")
    m = lb.run_moment_only(m0, lat, 1.0, 5)
    np.testing.assert_allclose(lb.project(fb, lat), m, rtol=0, atol=1e-14)


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_bgk_differs_from_moment_only_by_ghosts(lat):
    """Away from tau = 1 the population-storing BGK keeps ghost components that the
    reconstruction discards (Sec. II: RSC does not match the population scheme
    exactly), but on a smooth flow the difference stays small."""
    n = 16
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05)
    m0 = lb.equilibrium_moments(rho, u)
    f = lb.run_population(lb.populations_from_moments(m0, lat), lat, 0.6, 50, "bgk")
    mb = lb.project(f, lat)
    m = lb.run_moment_only(m0, lat, 0.6, 50)
    dj = np.abs(mb[1:4] - m[1:4]).max() / np.abs(m[1:4]).max()
    assert 1e-12 < dj < 5e-2


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_conservation(lat):
    """BGK collision and periodic streaming conserve total mass and momentum."""
    rho, u = inputs.taylor_green_3d(12, 10, 8, u0=0.05, noise=1e-3, seed=4)
    m = lb.equilibrium_moments(rho, u)
    # add a non-equilibrium part so the collision has work to do
    m[4:] += inputs.random_moments(12, 10, 8, seed=8)[4:] * 0.01
    before = [math.fsum(m[k].ravel()) for k in range(4)]
    m = lb.run_moment_only(m, lat, 0.63, 40)
    after = [math.fsum(m[k].ravel()) for k in range(4)]
    assert abs(after[0] - before[0]) <= 1e-13 * abs(before[0])
    for a in range(1, 4):
        assert abs(after[a] - before[a]) <= 1e-13 * m[0].size


def _mode_step_matrix(lat, tau, kvec):
    """Linear amplification of a Fourier mode exp(i k.x) around rest (rho=1, u=0).

    Derived independently of the oracle: with A = P - cs^2 rho I, the
    linearised collision is A' = (1 - omega) A, and pull streaming of
    h'_i = w_i [rho + 3 c.j + 4.5 cc:A' - 1.5 tr A'] multiplies the
    contribution of direction i by exp(-i k.c_i).  Works in the canonical
    basis (rho, j, P) via the linear map to (rho, j, A)."""
    omega = 1.0 / tau
    # canonical -> (rho, j, A): A_aa = P_aa - rho / 3
    T = np.eye(10)
    T[4, 0] = T[5, 0] = T[6, 0] = -CS2
    Tinv = np.linalg.inv(T)
    C = np.diag([1, 1, 1, 1] + [1 - omega] * 6)  # linear collision in (rho, j, A)
    S = np.zeros((10, 10), dtype=complex)
    for i in range(lat.Q):
        c = lat.c[i].astype(float)
        row = np.zeros(10)  # h'_i as a linear form of (rho, j, A')
        row[0] = 1.0
        row[1:4] = 3.0 * c
        for k, (a, b) in enumerate(lb.PAIRS):
            mult = 1.0 if a == b else 2.0
            row[4 + k] = 4.5 * c[a] * c[b] * mult - (1.5 if a == b else 0.0)
        col = np.zeros(10)  # canonical moments carried by one unit of h
        col[0] = 1.0
        col[1:4] = c
        for k, (a, b) in enumerate(lb.PAIRS):
            col[4 + k] = c[a] * c[b]
        S += lat.w[i] * np.exp(-1j * kvec.dot(c)) * np.outer(col, row)
    return S @ C @ T, Tinv


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
def test_linear_fourier_mode(lat):
    """A 1e-7 Fourier mode evolves by the closed-form amplification matrix."""
    n = 8
    rng = np.random.default_rng(21)
    kint = np.array([1, 2, 3])
    kvec = 2 * np.pi * kint / n
    G, _ = _mode_step_matrix(lat, 0.7, kvec)
    amp = 1e-7 * (rng.standard_normal(10) + 1j * rng.standard_normal(10))
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    phase = np.exp(1j * (kvec[0] * x + kvec[1] * y + kvec[2] * z))
    base = np.zeros(10)
    base[0] = 1.0
    base[4] = base[5] = base[6] = CS2
    m = base[:, None, None, None] + np.real(amp[:, None, None, None] * phase)
    out = lb.step_moment_only(m, lat, 0.7)
    mode = np.real((G @ amp)[:, None, None, None] * phase)
    expect = base[:, None, None, None] + mode
    # the mode is ~1e-7; nonlinear terms (j j / rho) are ~1e-14
    assert np.abs(out - expect).max() <= 1e-5 * np.abs(mode).max()


@pytest.mark.parametrize("lat", LATTICES, ids=IDS)
@pytest.mark.parametrize("tau", [0.8, 0.6])
def test_shear_wave_viscosity(lat, tau):
    """2D Taylor-Green cell decays as exp(-2 nu k^2 t), nu = cs^2 (tau - 1/2)
    (Sec. III B), within 1%: fit of ln|u| over t in [20, 200] on 32^2 x 2."""
    n = 32
    rho, u = inputs.shear_wave_2d(n, n, 2, u0=1e-3)
    m = lb.equilibrium_moments(rho, u)
    ts, amps = [], []
    for t in range(1, 201):
        m = lb.step_moment_only(m, lat, tau)
        if t >= 20:
            ts.append(t)
            amps.append(np.sqrt(np.mean((m[1] / m[0]) ** 2 + (m[2] / m[0]) ** 2)))
    k = 2 * np.pi / n
    nu_fit = -np.polyfit(ts, np.log(amps), 1)[0] / (2 * k * k)
    nu = CS2 * (tau - 0.5)
    assert abs(nu_fit - nu) / nu < 0.01


def test_advected_shear_wave_galilean():
    """A shear wave u_y = a sin(kx) riding on a uniform u_x = U is carried at
    speed U (the rho u u part of P^eq is the advective flux); 1% on the speed,
    2% on the viscosity (O(U^2) Galilean error of second-order equilibria)."""
    n, U, tau = 32, 0.05, 0.8
    x = np.arange(n)[None, None, :] * np.ones((2, 1, n))
    rho = np.ones((2, 1, n))
    u = np.zeros((3, 2, 1, n))
    u[0] = U
    u[1] = 1e-3 * np.sin(2 * np.pi * x / n)
    m = lb.equilibrium_moments(rho, u)
    k = 2 * np.pi / n
    ts, ph, am = [], [], []
    for t in range(1, 301):
        m = lb.step_moment_only(m, D3Q19, tau)
        if t >= 20 and t % 10 == 0:
            vy = (m[2] / m[0])[0, 0]
            coef = np.sum(vy * np.exp(-1j * k * np.arange(n)))
            ts.append(t)
            ph.append(np.angle(coef))
            am.append(abs(coef))
    speed = -np.polyfit(ts, np.unwrap(ph), 1)[0] / k
    nu_fit = -np.polyfit(ts, np.log(am), 1)[0] / (k * k)
    assert abs(speed - U) / U < 0.01
    assert abs(nu_fit - CS2 * (tau - 0.5)) / (CS2 * (tau - 0.5)) < 0.02


def test_node_form_matches_grid_form():
    """The per-node evaluator used for sampled checks agrees with the grid stepper."""
    m = inputs.random_moments(5, 6, 7, seed=13)
    for lat in LATTICES:
        grid = lb.step_moment_only(m, lat, 0.9)
        for (x, y, z) in [(0, 0, 0), (4, 5, 6), (2, 3, 1), (4, 0, 6)]:
            np.testing.assert_allclose(lb.node_moment_only(m, lat, 0.9, x, y, z), grid[:, z, y, x],
                                       rtol=0, atol=1e-15)
