"""GPU parity of the population-storing baselines against the oracle."""
import numpy as np
import pytest

from oracle import D3Q19, D3Q27, lb
from paper_2301_01622_gb300 import inputs, llb

from gpu_helpers import assert_groups, run_gpu

pytestmark = pytest.mark.gpu

LAT = {19: D3Q19, 27: D3Q27}


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("shape", [(32, 32, 32), (37, 11, 6), (1, 2, 3)], ids=lambda s: "x".join(map(str, s)))
def test_regularized_population_fp64(q, shape):
    """Population-storing regularized LB (the same map as the moment-only step)
    vs the oracle's population stepper, FP64, 1e-12."""
    nx, ny, nz = shape
    m0 = inputs.random_moments(nx, ny, nz, seed=31) if shape != (32, 32, 32) else \
        lb.equilibrium_moments(*inputs.taylor_green_3d(32, 32, 32, u0=0.05))
    steps = 50 if shape == (32, 32, 32) else 4
    f = lb.run_population(lb.populations_from_moments(m0, LAT[q]), LAT[q], 0.8, steps, "regularized")
    ref = lb.project(f, LAT[q])
    got, _ = run_gpu(shape, q, 0.8, steps, m0=m0, storage=llb.LLB_F64, scheme=llb.LLB_SCHEME_POPULATION)
    assert_groups(got, ref, 1e-12, what="regularized population")


@pytest.mark.parametrize("q", [19, 27])
def test_bgk_population_fp64(q):
    m0 = inputs.random_moments(13, 10, 7, seed=41)
    f = lb.run_population(lb.populations_from_moments(m0, LAT[q]), LAT[q], 0.65, 6, "bgk")
    ref = lb.project(f, LAT[q])
    got, _ = run_gpu((13, 10, 7), q, 0.65, 6, m0=m0, storage=llb.LLB_F64, scheme=llb.LLB_SCHEME_POPULATION_BGK)
    assert_groups(got, ref, 1e-12, what="bgk population")


@pytest.mark.parametrize("q", [19, 27])
def test_population_fp32_matches_moment_fp32(q):
    """Equal accuracy: the FP32 population baseline and the FP32 moment-only
    step both stay within 1e-5 of the FP64 oracle on the bench field."""
    n, tau = 32, 0.6
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=2301)
    ref = lb.run_moment_only(lb.equilibrium_moments(rho, u), LAT[q], tau, 200)
    pop, _ = run_gpu((n, n, n), q, tau, 200, rho=rho, u=u, storage=llb.LLB_F32, scheme=llb.LLB_SCHEME_POPULATION)
    mom, _ = run_gpu((n, n, n), q, tau, 200, rho=rho, u=u, storage=llb.LLB_F32)
    assert_groups(pop, ref, 1e-5, what="population fp32")
    assert_groups(mom, ref, 1e-5, what="moment fp32")


def test_population_diagnostics():
    m0 = inputs.random_moments(9, 8, 7, seed=2)
    p = llb.llb_params_default(storage=llb.LLB_F64, scheme=llb.LLB_SCHEME_POPULATION)
    ctx = llb.llb_create(9, 8, 7, 19, 0.8, p)
    try:
        llb.llb_init_moments(ctx, m0)
        d0 = llb.llb_diagnostics(ctx)
        llb.llb_step(ctx, 10)
        d1 = llb.llb_diagnostics(ctx)
    finally:
        llb.llb_destroy(ctx)
    assert abs(d0["mass"][0] - m0[0].sum()) < 1e-11
    assert abs(d1["mass"][0] - d0["mass"][0]) < 1e-11
    np.testing.assert_allclose(d1["momentum"], d0["momentum"], atol=1e-12)
