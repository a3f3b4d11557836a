"""Helpers for the GPU parity tests: run libllb through its C ABI and compare
with the oracle on the same seeded inputs."""
import numpy as np

from paper_2301_01622_gb300 import llb

# group slices of the canonical one-component moments
GROUPS_1 = {"rho": slice(0, 1), "j": slice(1, 4), "P": slice(4, 10)}


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


def group_errors(got, ref, groups=GROUPS_1):
    """max |got - ref| over a group's fields divided by max |ref| over the group."""
    errs = {}
    for name, sl in groups.items():
        scale = np.abs(ref[sl]).max()
        errs[name] = float(np.abs(got[sl] - ref[sl]).max() / scale) if scale > 0 else float(np.abs(got[sl]).max())
    return errs


def assert_groups(got, ref, tol, groups=GROUPS_1, what=""):
    errs = group_errors(got, ref, groups)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{what}: relative errors above {tol:g}: {errs}"
    return errs
