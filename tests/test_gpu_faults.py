"""Failure handling without faulting the GPU: a device wait that cannot
complete (its barrier is armed for a byte that never arrives) runs out after
its bound, is reported as LLB_ETIMEOUT and leaves the CUDA context usable; an
allocation larger than the device fails cleanly with LLB_ENOMEM."""
import numpy as np
import pytest

from oracle import D3Q19, lb
from paper_2301_01622_gb300 import inputs, llb

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_context_stays_usable():
    n = 128
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05)
    p = llb.llb_params_default(kernel=llb.LLB_KERNEL_TMA, wait_budget_ms=20, debug_flags=1)
    ctx = llb.llb_create(n, n, n, 19, 0.8, p)
    try:
        llb.llb_init_equilibrium(ctx, rho, u)
        llb.llb_step(ctx, 3)
        with pytest.raises(llb.LLBError) as e:
            llb.llb_synchronize(ctx)
        assert e.value.status == llb.LLB_ETIMEOUT
        # the context is sticky-failed from now on
        with pytest.raises(llb.LLBError) as e2:
            llb.llb_step(ctx, 1)
        assert e2.value.status == llb.LLB_ESTATE
    finally:
        llb.llb_destroy(ctx)
    # the device and the CUDA context still work: a fresh run matches the oracle
    m = 24
    rho, u = inputs.taylor_green_3d(m, m, m, u0=0.05)
    ctx = llb.llb_create(m, m, m, 19, 0.8, llb.llb_params_default(storage=llb.LLB_F64))
    try:
        llb.llb_init_equilibrium(ctx, rho, u)
        llb.llb_step(ctx, 5)
        got = llb.llb_get_moments(ctx, np.empty((10, m, m, m)))
    finally:
        llb.llb_destroy(ctx)
    ref = lb.run_moment_only(lb.equilibrium_moments(rho, u), D3Q19, 0.8, 5)
    assert np.abs(got - ref).max() < 1e-12


def test_bad_wait_parameters_rejected():
    for kw in ({"wait_budget_ms": 0}, {"debug_flags": 4}):
        with pytest.raises(llb.LLBError):
            llb.llb_footprint_query(8, 8, 8, 19, llb.llb_params_default(**kw))


def test_allocation_failure_is_clean():
    # 1400^3 nodes x 27 FP64 populations: ~590 GB per copy, more than the device holds
    p = llb.llb_params_default(storage=llb.LLB_F64, scheme=llb.LLB_SCHEME_POPULATION)
    with pytest.raises(llb.LLBError) as e:
        llb.llb_create(1400, 1400, 1400, 27, 0.8, p)
    assert e.value.status == llb.LLB_ENOMEM
    ctx = llb.llb_create(8, 8, 8, 19, 0.8, llb.llb_params_default())
    llb.llb_destroy(ctx)
