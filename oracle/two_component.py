"""Two-component colour-gradient LB with near-contact forcing, FP64 (test infrastructure only).

State: 11 canonical fields per node, (rho1, rho2, j_x, j_y, j_z, P_xx, P_yy,
P_zz, P_xy, P_xz, P_yz), shape (11, nz, ny, nx), periodic box.  The total
fluid (rho = rho1 + rho2, j, P) is one LB fluid with one relaxation time
(viscosity ratio one, Sec. IV); the colours are split by the
colour-gradient model (Sec. III A) and pushed apart near contact by the
LBNCI force (Sec. III B).

The paper delegates the colour-gradient operator forms to another work that
is not reproduced in it; the forms below are the readings stated in the
repository's design notes, one per step:

1. phase field phi = (rho1 - rho2) / (rho1 + rho2) (Sec. III B) and its
   isotropic lattice gradient G = (1/cs^2) sum_k w_k c_k phi(x + c_k);
   unit normal n = G / |G| where |G| >= g_min, else n = 0.
2. near-contact force F_rep = -A_h[h] n_out delta_I (Sec. III B) with
   n_out = -n (outward from the phi > 0 fluid), delta_I = |G|, and
   A_h[h] = A_h if the node is in near contact, else 0: a node of the
   interface band |G| >= g_nci is in near contact when phi exceeds
   phi(x) + PHI_RISE at one of the probe nodes x + round(k n_out),
   k = 1..h_c (another interface lies within h_c nodes along the outward
   normal).  So F = A_h G on those nodes.  The band threshold keeps the
   far-field tails of the tanh profile, where |G| is tiny, out of the
   detector; the rise margin keeps exact ties (symmetric configurations)
   from being decided by rounding.
3. collision of the reconstructed populations h (Eq. (4)) by BGK (Eq. (7))
   with a Guo forcing term, u_F = (j + F/2) / rho:
       h'_i = (1 - omega) h_i + omega h_i^eq(rho, u_F) + (1 - omega/2) S_i,
       S_i = w_i [(c_i - u_F)/cs^2 + (c_i.u_F) c_i / cs^4] . F
   (for F = 0 this is Eq. (8)), plus the colour-gradient perturbation
       Delta_i = (A_s / 2) |G| [w_i (c_i.n)^2 - w_i cs^2]
   applied to these populations (Sec. III A, last sentence) where the normal
   is defined (|G| >= g_min); elsewhere Delta_i = 0 (with n = 0 the bracket
   would not sum to zero and would create mass).
   With a smooth norm (eps > 0, a reading for gradients only):
   |G|_eps = sqrt(|G|^2 + eps^2), n = G / |G|_eps at every node and
       Delta_i = (A_s / 2) |G|_eps [w_i (c_i.n)^2 - w_i cs^2 |n|^2],
   which sums to zero and whose second moment is A_s cs^4 |G|_eps n n.
4. recolouring of the collided populations (Sec. III A):
       h1'_i = (rho1/rho) h'_i + beta (rho1 rho2 / rho) w_i (c_i.n) / |c_i|   (0 for c_i = 0),
       h2'_i = h'_i - h1'_i.
5. pull streaming of both colours (Eq. (9)) and projection (Eqs. (1)-(3)):
       rho1(x, t+1) = sum_i h1'_i(x - c_i), and rho, j, P from h' = h1' + h2'.

``step_moment_only`` keeps only the 11 fields (populations exist one
direction at a time).  ``step_regularized_population`` stores the two colour
population sets f1, f2 and applies steps 1-5 to h = R(P(f1 + f2)); it is the
same map in exact arithmetic.  ``step_bgk_population`` collides the stored
f = f1 + f2 itself (ghosts kept): the "with populations" scheme of Sec. IV.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lb
from .lattice import CS2, Lattice

NFIELDS = 11
PHI_RISE = 0.01  # phi must exceed phi(x) by this much at a probe to signal another interface


@dataclass(frozen=True)
class CGParams:
    beta: float = 0.7     # recolouring strength
    A_s: float = 0.01     # perturbation (surface tension) strength
    A_h: float = 0.0      # near-contact repulsion strength
    g_min: float = 1e-8   # |G| below which the normal is zero
    h_c: int = 3          # near-contact probe range (nodes)
    g_nci: float = 0.05   # |G| above which a node belongs to the interface band of the detector
    eps: float = 0.0      # > 0: smooth norm |G|_eps = sqrt(|G|^2 + eps^2), normal G/|G|_eps everywhere


def _check(m):
    m = np.asarray(m, dtype=np.float64)
    if m.ndim != 4 or m.shape[0] != NFIELDS:
        raise ValueError(f"two-component moments must have shape (11, nz, ny, nx), got {m.shape}")
    return m


def total_moments(m: np.ndarray) -> np.ndarray:
    """The one-fluid moments (rho, j, P) of the mixture, canonical 10-field layout."""
    m = _check(m)
    return np.concatenate([(m[0] + m[1])[None], m[2:]])


def phase_field(m: np.ndarray) -> np.ndarray:
    """phi = (rho1 - rho2) / (rho1 + rho2), Sec. III B."""
    m = _check(m)
    return (m[0] - m[1]) / (m[0] + m[1])


def gradient(phi: np.ndarray, lat: Lattice) -> np.ndarray:
    """G_a(x) = (1/cs^2) sum_k w_k c_ka phi(x + c_k), shape (3, nz, ny, nx)."""
    G = np.zeros((3,) + phi.shape)
    for k in range(lat.Q):
        c = lat.c[k]
        if not c.any():
            continue
        # value at x + c_k: roll by -c_k
        shifted = np.roll(phi, shift=(-int(c[2]), -int(c[1]), -int(c[0])), axis=(0, 1, 2))
        for a in range(3):
            if c[a]:
                G[a] += lat.w[k] * c[a] * shifted
    return G / CS2


def unit_normal(G: np.ndarray, g_min: float, eps: float = 0.0):
    """(|G|, n, defined): n = G/|G| where |G| >= g_min, n = 0 elsewhere; with
    eps > 0 the smooth norm |G|_eps = sqrt(|G|^2 + eps^2) and n = G/|G|_eps at
    every node (|n| < 1, the step stays differentiable where G -> 0)."""
    if eps > 0.0:
        gn = np.sqrt(G[0] ** 2 + G[1] ** 2 + G[2] ** 2 + eps * eps)
        return gn, G / gn, np.ones(gn.shape, dtype=bool)
    gn = np.sqrt(G[0] ** 2 + G[1] ** 2 + G[2] ** 2)
    iface = gn >= g_min
    n = np.zeros_like(G)
    for a in range(3):
        n[a][iface] = G[a][iface] / gn[iface]
    return gn, n, iface


def near_contact(phi: np.ndarray, n: np.ndarray, iface: np.ndarray, h_c: int) -> np.ndarray:
    """Boolean field of interface nodes with another interface within h_c nodes
    along the outward normal n_out = -n (phi rises above phi(x) at a probe)."""
    nz, ny, nx = phi.shape
    z, y, x = np.nonzero(iface)
    out = np.zeros(phi.shape, dtype=bool)
    if z.size == 0:
        return out
    nout = -n[:, z, y, x]
    hit = np.zeros(z.size, dtype=bool)
    here = phi[z, y, x]
    for k in range(1, h_c + 1):
        px = (x + np.rint(k * nout[0]).astype(np.int64)) % nx
        py = (y + np.rint(k * nout[1]).astype(np.int64)) % ny
        pz = (z + np.rint(k * nout[2]).astype(np.int64)) % nz
        hit |= phi[pz, py, px] > here + PHI_RISE
    out[z[hit], y[hit], x[hit]] = True
    return out


class CollisionFields:
    """Everything the collision of one step needs, computed once per step."""

    def __init__(self, m: np.ndarray, lat: Lattice, tau: float, prm: CGParams):
        m = _check(m)
        self.rho1, self.rho2 = m[0], m[1]
        self.tot = total_moments(m)
        self.fl = lb.LocalFields(self.tot)          # rho, u = j/rho, P, P^eq(u)
        self.rho = self.fl.rho
        self.phi = (self.rho1 - self.rho2) / self.rho
        self.G = gradient(self.phi, lat)
        self.gnorm, self.n, self.iface = unit_normal(self.G, prm.g_min, prm.eps)
        if prm.A_h != 0.0:
            self.near = near_contact(self.phi, self.n, self.gnorm >= prm.g_nci, prm.h_c)
        else:
            self.near = np.zeros(self.phi.shape, dtype=bool)
        self.F = np.where(self.near[None], prm.A_h * self.G, 0.0)
        self.uF = (self.tot[1:4] + 0.5 * self.F) / self.rho
        self.omega = 1.0 / tau
        self.prm = prm


def collided_direction(cf: CollisionFields, lat: Lattice, i: int):
    """(h'_i, h1'_i): total and colour-1 post-collision populations of direction i."""
    c = lat.c[i].astype(np.float64)
    w = lat.w[i]
    om = cf.omega
    rho = cf.rho
    h = lb.reconstruct_direction(cf.fl, lat, i, None)                     # Eq. (4)
    u = cf.uF
    cu = (c[0] * u[0] + c[1] * u[1] + c[2] * u[2]) / CS2
    usq = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
    heq = w * rho * (1.0 + cu + 0.5 * cu * cu - 0.5 * usq / CS2)         # Eq. (5) at u_F
    F = cf.F
    cF = c[0] * F[0] + c[1] * F[1] + c[2] * F[2]
    uFdot = u[0] * F[0] + u[1] * F[1] + u[2] * F[2]
    S = w * ((cF - uFdot) / CS2 + (c[0] * u[0] + c[1] * u[1] + c[2] * u[2]) * cF / (CS2 * CS2))
    cn = c[0] * cf.n[0] + c[1] * cf.n[1] + c[2] * cf.n[2]
    # the perturbation acts only where the interface normal is defined; with the
    # smooth norm (|n| < 1) its trace term carries |n|^2 so that it still sums to zero
    if cf.prm.eps > 0.0:
        nn = cf.n[0] ** 2 + cf.n[1] ** 2 + cf.n[2] ** 2
        pert = 0.5 * cf.prm.A_s * cf.gnorm * (w * cn * cn - w * CS2 * nn)
    else:
        pert = np.where(cf.iface, 0.5 * cf.prm.A_s * cf.gnorm * (w * cn * cn - w * CS2), 0.0)
    hp = (1.0 - om) * h + om * heq + (1.0 - 0.5 * om) * S + pert          # Eq. (7) + forcing + perturbation
    cnorm = np.sqrt((c * c).sum())
    recol = 0.0 if cnorm == 0 else cf.prm.beta * (cf.rho1 * cf.rho2 / rho) * w * cn / cnorm
    h1 = (cf.rho1 / rho) * hp + recol
    return hp, h1


def step_moment_only(m: np.ndarray, lat: Lattice, tau: float, prm: CGParams) -> np.ndarray:
    """One step of the two-component moment-only scheme (11 fields in, 11 out)."""
    cf = CollisionFields(m, lat, tau, prm)
    new_tot = np.zeros((10,) + cf.rho.shape)
    new_rho1 = np.zeros(cf.rho.shape)
    for i in range(lat.Q):
        c = lat.c[i]
        hp, h1 = collided_direction(cf, lat, i)
        hp = lb.stream_pull(hp, c)
        new_rho1 += lb.stream_pull(h1, c)
        new_tot[0] += hp
        for a in range(3):
            if c[a]:
                new_tot[1 + a] += c[a] * hp
        for k, (a, b) in enumerate(lb.PAIRS):
            if c[a] * c[b]:
                new_tot[4 + k] += c[a] * c[b] * hp
    out = np.empty_like(m)
    out[0] = new_rho1
    out[1] = new_tot[0] - new_rho1
    out[2:] = new_tot[1:]
    return out


def run_moment_only(m, lat, tau, prm, nsteps):
    for _ in range(nsteps):
        m = step_moment_only(m, lat, tau, prm)
    return m


def populations_from_moments(m: np.ndarray, lat: Lattice) -> np.ndarray:
    """Colour population sets (f1, f2), shape (2, Q, ...), from 11-field moments:
    f = R(total moments) (Eq. (4)), split by the colour fractions."""
    m = _check(m)
    f = lb.populations_from_moments(total_moments(m), lat)
    rho = m[0] + m[1]
    return np.stack([f * (m[0] / rho), f * (m[1] / rho)])


def project(f12: np.ndarray, lat: Lattice) -> np.ndarray:
    """11-field moments of colour population sets."""
    tot = lb.project(f12[0] + f12[1], lat)
    out = np.empty((NFIELDS,) + tot.shape[1:])
    out[0] = f12[0].sum(axis=0)
    out[1] = f12[1].sum(axis=0)
    out[2:] = tot[1:]
    return out


def _population_step(f12, lat, tau, prm, regularized: bool):
    m = project(f12, lat)
    cf = CollisionFields(m, lat, tau, prm)
    if not regularized:
        f = f12[0] + f12[1]
    out = np.empty_like(f12)
    for i in range(lat.Q):
        hp, h1 = collided_direction(cf, lat, i)
        if not regularized:
            # BGK on the stored population: replace the reconstructed h_i by f_i
            h = lb.reconstruct_direction(cf.fl, lat, i, None)
            hp = hp + (1.0 - cf.omega) * (f[i] - h)
            cn = sum(lat.c[i][a] * cf.n[a] for a in range(3))
            cnorm = np.sqrt((lat.c[i] ** 2).sum())
            recol = 0.0 if cnorm == 0 else prm.beta * (cf.rho1 * cf.rho2 / cf.rho) * lat.w[i] * cn / cnorm
            h1 = (cf.rho1 / cf.rho) * hp + recol
        out[0, i] = lb.stream_pull(h1, lat.c[i])
        out[1, i] = lb.stream_pull(hp - h1, lat.c[i])
    return out


def step_regularized_population(f12, lat, tau, prm):
    return _population_step(f12, lat, tau, prm, True)


def step_bgk_population(f12, lat, tau, prm):
    return _population_step(f12, lat, tau, prm, False)


def run_population(f12, lat, tau, prm, nsteps, scheme="regularized"):
    step = step_regularized_population if scheme == "regularized" else step_bgk_population
    for _ in range(nsteps):
        f12 = step(f12, lat, tau, prm)
    return f12


def count_droplets(rho1: np.ndarray, threshold: float = 0.5) -> int:
    """Connected components (6-neighbour, periodic) of rho1 > threshold."""
    mask = rho1 > threshold
    nz, ny, nx = mask.shape
    label = np.zeros(mask.shape, dtype=np.int64)
    count = 0
    for start in zip(*np.nonzero(mask)):
        if label[start]:
            continue
        count += 1
        stack = [start]
        label[start] = count
        while stack:
            z, y, x = stack.pop()
            for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                q = ((z + dz) % nz, (y + dy) % ny, (x + dx) % nx)
                if mask[q] and not label[q]:
                    label[q] = count
                    stack.append(q)
    return count
