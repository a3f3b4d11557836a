"""Droplet experiments of the paper's validation section, run on the library.

Everything here drives the C-ABI library (``llb``) and analyses the moments it
returns on the host; no lattice-Boltzmann arithmetic happens here.

* ``droplet_outcome`` -- an off-axis droplet collision (Sec. IV, Figs. 1, 2, 6, 7):
  the number of droplets (connected regions of rho1 > 0.5) and <rho1>_{rho1 > 0.5}
  over time, with and without the near-contact repulsion.
* ``laplace_sweep`` -- static droplets of several radii: the pressure jump
  dp = cs^2 (rho_in - rho_out) against 1/R (Laplace's law dp = 2 sigma / R in
  three dimensions) gives the surface tension of the colour-gradient model.
* ``viscosity_sweep`` -- a shear wave in a uniform mixture (no interface) of
  the two-component step: its decay rate gives the mixture viscosity, to be
  compared with nu = cs^2 (tau - 1/2) (Sec. III B).
* ``local_error_curves`` -- the local relative error |rho_N - rho_P| / rho_N,max
  between the scheme without populations (N) and the standard scheme with
  populations (P) at the probe sites of Fig. 3 (Sec. IV).

Run ``python -m paper_2301_01622_gb300.experiments outcome|laplace|viscosity|e3`` to
print the records as JSON.
"""
from __future__ import annotations

import json
import sys

import numpy as np

from . import inputs, llb

CS2 = 1.0 / 3.0


# ----------------------------------------------------------------------------- host analysis


def label_periodic(mask: np.ndarray):
    """Connected regions (6-neighbour) of a boolean (nz, ny, nx) field with
    periodic wrap in all three directions.  Returns (labels, count); labels
    are 0 outside the mask and 1..count inside."""
    from scipy import ndimage

    lab, n = ndimage.label(mask)
    if n == 0:
        return lab, 0
    parent = np.arange(n + 1)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    # regions touching opposite faces of the box are one region across the wrap
    for axis in range(3):
        lo = np.take(lab, 0, axis=axis)
        hi = np.take(lab, -1, axis=axis)
        both = (lo > 0) & (hi > 0)
        for a, b in set(zip(lo[both].tolist(), hi[both].tolist())):
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(a) for a in range(n + 1)])
    uniq = np.unique(roots[1:])
    remap = np.zeros(n + 1, dtype=np.int64)
    remap[1:] = np.searchsorted(uniq, roots[1:]) + 1
    return remap[lab], int(uniq.size)


def count_droplets(rho1: np.ndarray, threshold: float = 0.5) -> int:
    """Number of droplets: connected regions of rho1 > threshold (periodic)."""
    return label_periodic(np.asarray(rho1) > threshold)[1]


def pressure_jump(m: np.ndarray, centre, radius: float, margin: float = 4.0):
    """dp = cs^2 (<rho>_in - <rho>_out) of a droplet from two-component
    canonical moments m (11, nz, ny, nx): <rho>_in over nodes closer than
    radius - margin to the centre, <rho>_out over nodes farther than
    radius + margin (periodic minimum-image distance)."""
    rho = m[0] + m[1]
    nz, ny, nx = rho.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = [(c - o + n / 2) % n - n / 2 for c, o, n in ((x, centre[0], nx), (y, centre[1], ny), (z, centre[2], nz))]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    inside = r < radius - margin
    outside = r > radius + margin
    return CS2 * (float(rho[inside].mean()) - float(rho[outside].mean()))


def probe_sites(shape):
    """The three probe sites of Fig. 3 (1-based (32,64,64), (64,64,64),
    (128,128,128) in a box of 128), 0-based and scaled to the box."""
    nx, ny, nz = shape
    out = []
    for (a, b, c) in ((32, 64, 64), (64, 64, 64), (128, 128, 128)):
        out.append((int(round(a * nx / 128)) - 1, int(round(b * ny / 128)) - 1, int(round(c * nz / 128)) - 1))
    return out


# ----------------------------------------------------------------------------- runs


def _ctx(shape, lattice, tau, **params):
    nx, ny, nz = shape
    return llb.llb_create(nx, ny, nz, lattice, tau, llb.llb_params_default(**params))


def _moments(ctx, shape, nf=11):
    nx, ny, nz = shape
    return llb.llb_get_moments(ctx, np.empty((nf, nz, ny, nx), dtype=np.float32)).astype(np.float64)


def droplet_outcome(A_h, shape=(384, 192, 192), radius=30.0, speed=0.05, impact=15.0, steps=20000,
                    diag_every=500, count_every=5000, lattice=27, tau=1.0, A_s=0.01, beta=0.7,
                    storage=llb.LLB_F32):
    """Off-axis collision of two droplets approaching at +-speed along x:
    the droplet count every count_every steps and <rho1>_{rho1>0.5} every
    diag_every steps.  Returns a dict with the time series and the final count."""
    r1, r2, u = inputs.droplet_pair(*shape, radius, speed, impact)
    ctx = _ctx(shape, lattice, tau, ncomp=2, storage=storage, A_h=A_h, A_s=A_s, beta=beta)
    rec = {"A_h": A_h, "shape": list(shape), "radius": radius, "speed": speed, "impact": impact, "tau": tau,
           "A_s": A_s, "beta": beta, "lattice": lattice, "steps": steps, "t": [], "rho1_avg": [], "mass1": [],
           "counts": []}
    try:
        llb.llb_init_equilibrium(ctx, np.stack([r1, r2]), u)
        t = 0
        while True:
            d = llb.llb_diagnostics(ctx)
            rec["t"].append(t)
            rec["rho1_avg"].append(d["rho1_avg"])
            rec["mass1"].append(d["mass"][0])
            if t % count_every == 0 or t == steps:
                rec["counts"].append([t, count_droplets(_moments(ctx, shape)[0])])
            if t >= steps:
                break
            n = min(diag_every, steps - t)
            llb.llb_step(ctx, n)
            t += n
    finally:
        llb.llb_destroy(ctx)
    rec["final_count"] = rec["counts"][-1][1]
    return rec


def laplace_sweep(radii=(8.0, 10.0, 12.0, 16.0, 20.0), n=80, steps=6000, lattice=27, tau=1.0, A_s=0.01, beta=0.7,
                  storage=llb.LLB_F32):
    """Static droplets of each radius at the centre of an n^3 periodic box:
    the pressure jump after `steps` steps, and the least-squares fit
    dp = 2 sigma (1/R) + c."""
    rows = []
    for R in radii:
        shape = (n, n, n)
        centre = (n / 2, n / 2, n / 2)
        r1, r2, u = inputs.droplets(n, n, n, [centre], [R], [(0.0, 0.0, 0.0)])
        ctx = _ctx(shape, lattice, tau, ncomp=2, storage=storage, A_h=0.0, A_s=A_s, beta=beta)
        try:
            llb.llb_init_equilibrium(ctx, np.stack([r1, r2]), u)
            llb.llb_step(ctx, steps)
            m = _moments(ctx, shape)
        finally:
            llb.llb_destroy(ctx)
        rows.append({"R": R, "dp": pressure_jump(m, centre, R), "umax": float(np.abs(m[2:5] / (m[0] + m[1])).max())})
    inv_r = np.array([1.0 / r["R"] for r in rows])
    dp = np.array([r["dp"] for r in rows])
    A = np.stack([inv_r, np.ones_like(inv_r)], axis=1)
    (slope, icpt), *_ = np.linalg.lstsq(A, dp, rcond=None)
    fit = slope * inv_r + icpt
    return {"rows": rows, "sigma": slope / 2.0, "intercept": icpt,
            "max_rel_residual": float(np.abs(dp - fit).max() / np.abs(dp).max()), "n": n, "steps": steps,
            "lattice": lattice, "tau": tau, "A_s": A_s, "beta": beta}


def viscosity_sweep(taus=(0.6, 0.8, 1.0, 1.5), n=64, steps=600, u0=1e-3, lattice=19, storage=llb.LLB_F64):
    """Two-dimensional Taylor-Green cell (uniform along z) in a uniform
    mixture rho1 = rho2 = 1/2: u decays as exp(-2 nu k^2 t).  The fitted
    decay of the velocity amplitude over [steps/4, steps] gives nu."""
    rows = []
    k = 2 * np.pi / n
    rho, u = inputs.shear_wave_2d(n, n, 4, u0=u0)
    rho12 = np.stack([0.5 * rho, 0.5 * rho])
    for tau in taus:
        ctx = _ctx((n, n, 4), lattice, tau, ncomp=2, storage=storage, A_h=0.0)
        ts, amps = [], []
        try:
            llb.llb_init_equilibrium(ctx, rho12, u)
            t = 0
            for t_next in np.linspace(steps // 4, steps, 7).astype(int):
                llb.llb_step(ctx, int(t_next - t))
                t = int(t_next)
                m = llb.llb_get_moments(ctx, np.empty((11, 4, n, n)))
                ux = m[2] / (m[0] + m[1])
                ts.append(t)
                amps.append(float(np.abs(ux).max()))
        finally:
            llb.llb_destroy(ctx)
        slope = np.polyfit(np.array(ts, dtype=float), np.log(np.array(amps)), 1)[0]
        nu = -slope / (2 * k * k)
        rows.append({"tau": tau, "nu": nu, "nu_theory": CS2 * (tau - 0.5), "rel_err": nu / (CS2 * (tau - 0.5)) - 1})
    return {"rows": rows, "n": n, "steps": steps, "lattice": lattice}


def local_error_curves(ncomp=2, shape=(128, 128, 128), steps=3000, every=50, lattice=19, tau=1.0, A_h=0.05,
                       A_s=0.01, beta=0.7, radius=15.0, speed=0.05, impact=12.75, storage=llb.LLB_F32):
    """|rho_N - rho_P| / rho_N,max at the three probe sites, every `every`
    steps: N = the moment-only scheme, P = BGK with stored populations, on the
    same initial field.  Two components: rho is the droplet component rho1
    and the field is an off-axis droplet pair (radius 15, impact parameter
    0.85 of the radius, as in Sec. IV); one component: rho is the density of
    the Taylor-Green field with 1e-3 velocity noise.  rho_N,max is the
    maximum of rho over the box in the moment-only run at that time."""
    nx, ny, nz = shape
    sites = probe_sites(shape)
    nf = 11 if ncomp == 2 else 10
    if ncomp == 2:
        r1, r2, u = inputs.droplet_pair(nx, ny, nz, radius, speed, impact)
        rho0 = np.stack([r1, r2])
        kw = dict(ncomp=2, storage=storage, A_h=A_h, A_s=A_s, beta=beta)
    else:
        rho0, u = inputs.taylor_green_3d(nx, ny, nz, u0=0.05, noise=1e-3, seed=2301)
        kw = dict(storage=storage)
    ctxs = [_ctx(shape, lattice, tau, scheme=llb.LLB_SCHEME_MOMENT, **kw),
            _ctx(shape, lattice, tau, scheme=llb.LLB_SCHEME_POPULATION_BGK, **kw)]
    rec = {"ncomp": ncomp, "shape": list(shape), "lattice": lattice, "tau": tau, "sites": sites, "t": [],
           "err": [[] for _ in sites]}
    try:
        for c in ctxs:
            llb.llb_init_equilibrium(c, rho0, u)
        t = 0
        while True:
            mN = _moments(ctxs[0], shape, nf)[0]
            mP = _moments(ctxs[1], shape, nf)[0]
            rmax = float(mN.max())
            rec["t"].append(t)
            for k, (x, y, z) in enumerate(sites):
                rec["err"][k].append(abs(float(mN[z, y, x]) - float(mP[z, y, x])) / rmax)
            if t >= steps:
                break
            n = min(every, steps - t)
            for c in ctxs:
                llb.llb_step(c, n)
            t += n
    finally:
        for c in ctxs:
            llb.llb_destroy(c)
    rec["max_err"] = [max(e) for e in rec["err"]]
    return rec


def main(argv):
    what = argv[1] if len(argv) > 1 else "outcome"
    if what == "outcome":
        out = [droplet_outcome(a) for a in (0.0, 0.01, 0.05)]
    elif what == "laplace":
        out = [laplace_sweep(lattice=q) for q in (19, 27)]
        out += [laplace_sweep(lattice=19, A_s=0.02), laplace_sweep(lattice=19, tau=0.8), laplace_sweep(lattice=19, tau=1.2)]
    elif what == "viscosity":
        out = [viscosity_sweep(lattice=q) for q in (19, 27)]
    elif what == "e3":
        out = [local_error_curves(ncomp=2), local_error_curves(ncomp=1)]
    else:
        raise SystemExit("usage: python -m paper_2301_01622_gb300.experiments outcome|laplace|viscosity|e3")
    print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv)
