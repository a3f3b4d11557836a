"""Single-component lattice Boltzmann, FP64, written from the paper's equations.

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.

State of the moment-only scheme ("LB without populations", Sec. II-III): per
node the ten hydrodynamic fields of Eqs. (1)-(3), in the canonical order

    m = (rho, j_x, j_y, j_z, P_xx, P_yy, P_zz, P_xy, P_xz, P_yz),  j = rho u,

stored field-major as an array of shape (10, nz, ny, nx), x fastest.  All
boundaries are periodic (the paper does not state its boundaries; the
workloads it runs are periodic boxes).

Three steppers are provided:

* ``step_moment_only``  -- the paper's method.  Per step and per direction
  i, the post-collision population of Eq. (8) is reconstructed, written
  literally as
      h'_i = w_i rho (1 + c_i.u / cs^2 + Q_i:uu) + (1 - omega) w_i Q_i:(P - P^eq),
      Q_iab = (c_ia c_ib - cs^2 delta_ab) / (2 cs^4),   P^eq = cs^2 rho I + rho u u,
  from the moments of every node, pull-streamed along c_i (Eq. (9):
  h_i(x, t+1) = h'_i[H(x - c_i, t)]) and summed into the new moments with
  Eqs. (1)-(3).  Populations exist only one direction at a time.
* ``step_regularized_population`` -- the same collision applied to stored
  populations f (f is projected with Eqs. (1)-(3), re-expanded with Eq. (8)
  and streamed).  This is the population-storing scheme the moment-only
  method reproduces (Sec. II: the reconstruction keeps exactly the ten
  moments).
* ``step_bgk_population`` -- plain BGK on stored populations, Eq. (7)
  applied to f itself (ghost components kept): the "standard LB with
  populations" the paper compares against in Sec. IV.

Everything is float64 numpy; no blocking or reordering beyond one direction
at a time.
"""
from __future__ import annotations

import numpy as np

from .lattice import CS2, Lattice

NFIELDS = 10
# index pairs (a, b) of the six independent entries of P, in canonical order
PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def _check_moments(m: np.ndarray) -> np.ndarray:
    m = np.asarray(m, dtype=np.float64)
    if m.ndim != 4 or m.shape[0] != NFIELDS:
        raise ValueError(f"moments must have shape (10, nz, ny, nx), got {m.shape}")
    return m


def tensor_from_fields(p6: np.ndarray) -> list:
    """Full symmetric 3x3 nested list of arrays from the six stored entries."""
    t = [[None] * 3 for _ in range(3)]
    for k, (a, b) in enumerate(PAIRS):
        t[a][b] = p6[k]
        t[b][a] = p6[k]
    return t


def unpack(m: np.ndarray):
    """(rho, u, P) from canonical moments; u = j / rho (Eqs. (1)-(3)), P as 3x3 list."""
    m = _check_moments(m)
    rho = m[0]
    u = m[1:4] / rho
    P = tensor_from_fields(m[4:10])
    return rho, u, P


def equilibrium_pressure(rho: np.ndarray, u: np.ndarray) -> list:
    """Second-order equilibrium momentum flux P^eq_ab = cs^2 rho delta_ab + rho u_a u_b.

    This is the second moment of h^eq in Eq. (5).
    """
    return [[CS2 * rho * (a == b) + rho * u[a] * u[b] for b in range(3)] for a in range(3)]


def equilibrium_moments(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Canonical moments of a fluid at local equilibrium (P = P^eq)."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    peq = equilibrium_pressure(rho, u)
    m = np.empty((NFIELDS,) + rho.shape, dtype=np.float64)
    m[0] = rho
    m[1:4] = rho * u
    for k, (a, b) in enumerate(PAIRS):
        m[4 + k] = peq[a][b]
    return m


def hermite_q(c_i: np.ndarray) -> np.ndarray:
    """Q_iab = (c_ia c_ib - cs^2 delta_ab) / (2 cs^4)   (Sec. II, after Eq. (4))."""
    c = c_i.astype(np.float64)
    return (np.outer(c, c) - CS2 * np.eye(3)) / (2.0 * CS2 * CS2)


def _contract(q: np.ndarray, t) -> np.ndarray:
    """Q_ab T_ab summed over all nine (a, b)."""
    acc = 0.0
    for a in range(3):
        for b in range(3):
            if q[a, b] != 0.0:
                acc = acc + q[a, b] * t[a][b]
    return acc


class LocalFields:
    """rho, u, P and P^eq of every node, computed once per step from the moments."""

    def __init__(self, m: np.ndarray):
        self.rho, self.u, self.P = unpack(m)
        self.peq = equilibrium_pressure(self.rho, self.u)
        self.uu = [[self.u[a] * self.u[b] for b in range(3)] for a in range(3)]
        self.pneq = [[self.P[a][b] - self.peq[a][b] for b in range(3)] for a in range(3)]


def reconstruct_direction(m, lat: Lattice, i: int, omega: float | None) -> np.ndarray:
    """Population h_i at every node, reconstructed from the moments.

    ``m`` is a canonical moment array or a ``LocalFields`` built from one.
    omega=None: Eq. (4), h_i = h_i^eq + h_i^neq (Eqs. (5), (6)),
    ghosts g_i = 0.
    omega given: the post-collision population of Eq. (8),
    h'_i = h_i^eq + (1 - omega) h_i^neq.
    """
    fl = m if isinstance(m, LocalFields) else LocalFields(m)
    rho, u = fl.rho, fl.u
    c = lat.c[i]
    w = lat.w[i]
    q = hermite_q(c)
    cu = (c[0] * u[0] + c[1] * u[1] + c[2] * u[2]) / CS2          # c_ia u_ia, u_ia = u_a / cs^2
    quu = _contract(q, fl.uu)
    h_eq = w * rho * (1.0 + cu + quu)                              # Eq. (5)
    h_neq = w * _contract(q, fl.pneq)                              # Eq. (6)
    if omega is None:
        return h_eq + h_neq                                        # Eq. (4)
    return h_eq + (1.0 - omega) * h_neq                            # Eq. (8)


def reconstruct(m: np.ndarray, lat: Lattice, omega: float | None = None) -> np.ndarray:
    """All Q reconstructed populations, shape (Q, nz, ny, nx) (Eq. (4) / (8))."""
    fl = LocalFields(m)
    return np.stack([reconstruct_direction(fl, lat, i, omega) for i in range(lat.Q)])


def project(f: np.ndarray, lat: Lattice) -> np.ndarray:
    """H = P f: the ten moments of a population set, Eqs. (1)-(3)."""
    f = np.asarray(f, dtype=np.float64)
    m = np.zeros((NFIELDS,) + f.shape[1:], dtype=np.float64)
    for i in range(lat.Q):
        c = lat.c[i]
        m[0] += f[i]
        for a in range(3):
            if c[a]:
                m[1 + a] += c[a] * f[i]
        for k, (a, b) in enumerate(PAIRS):
            if c[a] * c[b]:
                m[4 + k] += c[a] * c[b] * f[i]
    return m


def stream_pull(field: np.ndarray, c_i: np.ndarray) -> np.ndarray:
    """Periodic pull streaming of one population: out(x) = field(x - c_i).

    ``field`` has shape (nz, ny, nx); np.roll with shift s gives out[x] = in[x - s].
    """
    return np.roll(field, shift=(int(c_i[2]), int(c_i[1]), int(c_i[0])), axis=(0, 1, 2))


def step_moment_only(m: np.ndarray, lat: Lattice, tau: float) -> np.ndarray:
    """One time step of the moment-only scheme (reconstruct, collide, pull-stream, project).

    Per direction: h'_i from Eq. (8) at every source node, streamed with
    Eq. (9) (no sum over i: the sum belongs to Eqs. (1)-(3)), then added
    into the new moments with Eqs. (1)-(3).  Returns the new canonical moments.
    """
    m = _check_moments(m)
    omega = 1.0 / tau
    fl = LocalFields(m)
    new = np.zeros_like(m)
    for i in range(lat.Q):
        c = lat.c[i]
        h = stream_pull(reconstruct_direction(fl, lat, i, omega), c)
        new[0] += h
        for a in range(3):
            if c[a]:
                new[1 + a] += c[a] * h
        for k, (a, b) in enumerate(PAIRS):
            if c[a] * c[b]:
                new[4 + k] += c[a] * c[b] * h
    return new


def run_moment_only(m: np.ndarray, lat: Lattice, tau: float, nsteps: int) -> np.ndarray:
    for _ in range(nsteps):
        m = step_moment_only(m, lat, tau)
    return m


def populations_from_moments(m: np.ndarray, lat: Lattice) -> np.ndarray:
    """Initial populations f = R H for the population-storing schemes (Eq. (4))."""
    return reconstruct(_check_moments(m), lat, omega=None)


def step_regularized_population(f: np.ndarray, lat: Lattice, tau: float) -> np.ndarray:
    """Population-storing regularized step: f -> H = P f -> h' (Eq. (8)) -> stream."""
    fl = LocalFields(project(f, lat))
    omega = 1.0 / tau
    return np.stack([stream_pull(reconstruct_direction(fl, lat, i, omega), lat.c[i]) for i in range(lat.Q)])


def step_bgk_population(f: np.ndarray, lat: Lattice, tau: float) -> np.ndarray:
    """Standard BGK with stored populations: f' = (1 - omega) f + omega f^eq (Eq. (7) on f), stream."""
    fl = LocalFields(project(f, lat))
    rho, u = fl.rho, fl.u
    omega = 1.0 / tau
    out = np.empty_like(f)
    for i in range(lat.Q):
        c = lat.c[i]
        q = hermite_q(c)
        cu = (c[0] * u[0] + c[1] * u[1] + c[2] * u[2]) / CS2
        quu = _contract(q, fl.uu)
        feq = lat.w[i] * rho * (1.0 + cu + quu)                    # Eq. (5)
        out[i] = stream_pull((1.0 - omega) * f[i] + omega * feq, c)
    return out


def run_population(f: np.ndarray, lat: Lattice, tau: float, nsteps: int, scheme: str = "regularized") -> np.ndarray:
    step = step_regularized_population if scheme == "regularized" else step_bgk_population
    for _ in range(nsteps):
        f = step(f, lat, tau)
    return f


def node_moment_only(m: np.ndarray, lat: Lattice, tau: float, x: int, y: int, z: int) -> np.ndarray:
    """New moments of ONE node after one moment-only step (pure-Python per-node form).

    Used to check sampled outputs of full-size GPU runs: it reads only the Q
    source nodes x - c_i (periodic) and applies Eq. (8) / (9) / (1)-(3)
    to each, so it costs O(Q) regardless of the grid size.
    """
    m = _check_moments(m)
    nz, ny, nx = m.shape[1:]
    omega = 1.0 / tau
    out = np.zeros(NFIELDS, dtype=np.float64)
    for i in range(lat.Q):
        c = lat.c[i]
        src = m[:, (z - c[2]) % nz, (y - c[1]) % ny, (x - c[0]) % nx].reshape(NFIELDS, 1, 1, 1)
        h = float(reconstruct_direction(src, lat, i, omega).reshape(()))
        out[0] += h
        for a in range(3):
            out[1 + a] += c[a] * h
        for k, (a, b) in enumerate(PAIRS):
            out[4 + k] += c[a] * c[b] * h
    return out
