"""llb_diagnostics_noalloc: the diagnostics entry point for callers that
cannot allocate device memory (code under a framework that owns the device
allocator, real-time loops that may not allocate, fixed memory budgets).  It
must give the same sums as llb_diagnostics on the same field, call after
call, since every call reuses one fixed scratch array in device memory; both
of its input types (FP64 and FP32 canonical moments) are exercised.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2301_01622_gb300 import inputs, llb

pytestmark = pytest.mark.gpu


def _noalloc(dev, shape, stream=None):
    nx, ny, nz = shape
    return llb.llb_diagnostics_noalloc(dev, nx, ny, nz, stream)


def _close(a, b, n, tol=1e-12, scale=None):
    """a and b agree within tol times the size of each sum (scale: per-sum
    magnitudes; default n, the node count)."""
    scale = scale or {}
    assert a["n_in"] == b["n_in"]
    assert a["flags"] == b["flags"]
    assert abs(a["mass"][0] - b["mass"][0]) <= tol * scale.get("mass", n)
    for k in range(3):
        assert abs(a["momentum"][k] - b["momentum"][k]) <= tol * scale.get("momentum", n)
    assert abs(a["rho1_sum"] - b["rho1_sum"]) <= tol * scale.get("rho1_sum", n)
    assert abs(a["rho1_avg"] - b["rho1_avg"]) <= max(tol * max(1.0, abs(b["rho1_avg"])), 1e-12)
    assert abs(a["min_rho"] - b["min_rho"]) <= max(tol * abs(b["min_rho"]), 1e-15)


def _same(a, b):
    for k in ("mass", "momentum"):
        assert list(a[k]) == list(b[k])
    for k in ("rho1_sum", "n_in", "rho1_avg", "min_rho", "flags"):
        assert a[k] == b[k]


@pytest.mark.parametrize("in_dtype", ["f64", "f32"])
@pytest.mark.parametrize("storage", [llb.LLB_F64, llb.LLB_F32])
@pytest.mark.parametrize("shape", [(45, 33, 17), (256, 64, 32)], ids=["small", "multi-row"])
def test_noalloc_matches_llb_diagnostics_twice(storage, shape, in_dtype):
    """Two calls in a row (and a third after a different field) against
    llb_diagnostics on the context that holds the same moments.  With FP32
    input the canonical field carries the rounding of each value to FP32
    (relative 2^-24), so the sums may differ from the state's by that much
    times the sum of magnitudes; with FP64 input they agree to 1e-12 per node."""
    torch = pytest.importorskip("torch")
    nx, ny, nz = shape
    n = nx * ny * nz
    m0 = inputs.random_moments(nx, ny, nz, seed=23, rho_spread=0.6)
    p = llb.llb_params_default(storage=storage)
    ctx = llb.llb_create(nx, ny, nz, 19, 0.8, p)
    try:
        llb.llb_init_moments(ctx, m0)
        llb.llb_step(ctx, 3)
        ref = llb.llb_diagnostics(ctx)
        dev = torch.empty((10, nz, ny, nx), dtype=torch.float64, device="cuda")
        llb.llb_get_moments_device(ctx, dev)
        llb.llb_synchronize(ctx)
        host = dev.cpu().numpy()
        if in_dtype == "f32":
            dev = dev.float().contiguous()
            torch.cuda.synchronize()
        first = _noalloc(dev, shape)
        second = _noalloc(dev, shape)
        # a different field in between must not leak into the next result
        other = torch.ones_like(dev)
        third = _noalloc(other, shape)
        fourth = _noalloc(dev, shape)
    finally:
        llb.llb_destroy(ctx)
    if in_dtype == "f64":
        for r in (first, second, fourth):
            _close(r, ref, n)
    else:
        eps32 = 2.0 ** -24
        # no node may sit within FP32 rounding of the 0.5 threshold, or the counts could differ
        assert not np.any(np.abs(host[0] - 0.5) <= 2 * eps32)
        scale = {"mass": np.abs(host[0]).sum() + n * 1e-9, "momentum": np.abs(host[1:4]).sum(axis=(1, 2, 3)).max(),
                 "rho1_sum": np.abs(host[0]).sum()}
        for r in (first, second, fourth):
            _close(r, ref, n, tol=eps32, scale=scale)
    # the same input gives bit-identical results call after call
    _same(first, second)
    _same(first, fourth)
    assert third["n_in"] == n and third["mass"][0] == n


def test_noalloc_rejects_oversized_and_bad_arguments():
    torch = pytest.importorskip("torch")
    dev = torch.zeros(16, dtype=torch.float32, device="cuda")
    fn = llb.lib().llb_diagnostics_noalloc
    out = llb.llb_diag()
    # more nodes than the fixed scratch can reduce: rejected before any launch
    assert fn(dev.data_ptr(), llb.LLB_F32, 1024, 1024, 65, None, C.byref(out)) == llb.LLB_EINVAL
    assert fn(dev.data_ptr(), 7, 2, 2, 2, None, C.byref(out)) == llb.LLB_EINVAL
    assert fn(None, llb.LLB_F32, 2, 2, 2, None, C.byref(out)) == llb.LLB_EINVAL
    assert fn(dev.data_ptr(), llb.LLB_F32, 0, 2, 2, None, C.byref(out)) == llb.LLB_EINVAL
