"""Helpers for the GPU parity tests: run libllb through its C ABI and compare
with the oracle on the same seeded inputs.

Two error measures are used:

* per field (the bound the tests assert): each shifted field -- the density
  deviation rho - 1, each component of j, each entry of A = P - cs^2 rho I
  (and rho1 for two components) -- compared on its own,
  max |gpu - oracle| / max |oracle| over that one field.  A component of j
  or A whose largest value is below 1e-3 of the largest component of its
  tensor (a component that vanishes by symmetry, such as j_z of a pair
  moving in the x-y plane) is measured against that 1e-3 floor instead of
  its own rounding-level maximum;
* per group (reported beside it): the same quotient over a whole group of
  canonical fields (rho; j; P), which dilutes the small fields of a group.
"""
import numpy as np

from paper_2301_01622_gb300 import llb

CS2 = 1.0 / 3.0

# group slices of the canonical one-component moments
GROUPS_1 = {"rho": slice(0, 1), "j": slice(1, 4), "P": slice(4, 10)}
GROUPS_2 = {"rho": slice(0, 2), "j": slice(2, 5), "P": slice(5, 11)}

NAMES_1 = ["drho", "jx", "jy", "jz", "Axx", "Ayy", "Azz", "Axy", "Axz", "Ayz"]
NAMES_2 = ["rho1"] + NAMES_1


def run_gpu(shape, lattice, tau, steps, *, m0=None, rho=None, u=None, storage=llb.LLB_F64,
            kernel=llb.LLB_KERNEL_AUTO, scheme=llb.LLB_SCHEME_MOMENT, ncomp=1, out_dtype=np.float64, **params):
    nx, ny, nz = shape
    p = llb.llb_params_default(storage=storage, kernel=kernel, scheme=scheme, ncomp=ncomp, **params)
    ctx = llb.llb_create(nx, ny, nz, lattice, tau, p)
    try:
        if m0 is not None:
            llb.llb_init_moments(ctx, np.ascontiguousarray(m0))
        else:
            llb.llb_init_equilibrium(ctx, np.ascontiguousarray(rho), np.ascontiguousarray(u))
        llb.llb_step(ctx, steps)
        nf = 10 if ncomp == 1 else 11
        out = llb.llb_get_moments(ctx, np.empty((nf, nz, ny, nx), dtype=out_dtype))
        used_kernel = llb.llb_state_device(ctx)[2]
    finally:
        llb.llb_destroy(ctx)
    return out.astype(np.float64), used_kernel


def shifted(m):
    """Shifted fields of canonical moments: (rho1,) rho - 1, j, A = P - cs^2 rho I."""
    m = np.asarray(m, dtype=np.float64)
    two = m.shape[0] == 11
    rho = m[0] + m[1] if two else m[0]
    j = m[2:5] if two else m[1:4]
    P = m[5:11] if two else m[4:10]
    A = P.copy()
    for a in range(3):
        A[a] = P[a] - CS2 * rho
    parts = ([m[0:1]] if two else []) + [(rho - 1.0)[None], j, A]
    return np.concatenate(parts)


TENSOR_FLOOR = 1e-3


def field_errors(got, ref):
    """Per shifted field: max |got - ref| / max |ref|; components of j and A
    are scaled by at least TENSOR_FLOOR times the largest component of their
    tensor (absolute error if everything is zero)."""
    g, r = shifted(got), shifted(ref)
    two = g.shape[0] == 11
    names = NAMES_2 if two else NAMES_1
    o = 1 if two else 0
    tensors = {"j": range(o + 1, o + 4), "A": range(o + 4, o + 10)}
    floor = {}
    for idx in tensors.values():
        top = max(float(np.abs(r[k]).max()) for k in idx)
        for k in idx:
            floor[k] = TENSOR_FLOOR * top
    errs = {}
    for k, name in enumerate(names):
        scale = max(float(np.abs(r[k]).max()), floor.get(k, 0.0))
        d = np.abs(g[k] - r[k]).max()
        errs[name] = float(d / scale) if scale > 0 else float(d)
    return errs


def group_errors(got, ref, groups=None):
    """max |got - ref| over a group's fields divided by max |ref| over the group."""
    if groups is None:
        groups = GROUPS_2 if np.asarray(ref).shape[0] == 11 else GROUPS_1
    errs = {}
    for name, sl in groups.items():
        scale = np.abs(ref[sl]).max()
        errs[name] = float(np.abs(got[sl] - ref[sl]).max() / scale) if scale > 0 else float(np.abs(got[sl]).max())
    return errs


def assert_fields(got, ref, tol, what="", tols=None):
    """Assert the per-field bound (tols: per-field overrides, each stated where used)."""
    errs = field_errors(got, ref)
    lim = {k: (tols or {}).get(k, tol) for k in errs}
    bad = {k: v for k, v in errs.items() if not v <= lim[k]}
    assert not bad, f"{what}: per-field relative errors above bound: {bad} (all: {errs}; groups: {group_errors(got, ref)})"
    return errs


def assert_groups(got, ref, tol, groups=None, what=""):
    errs = group_errors(got, ref, groups)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{what}: relative errors above {tol:g}: {errs}"
    return errs
