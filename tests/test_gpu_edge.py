"""Degenerate calls: zero steps leave the state alone (plain, graph, batch),
the adjoint over zero steps is the identity on the cotangent with dL/dtau = 0,
the host-to-host step refuses zero steps, negative counts are refused."""
import numpy as np
import pytest

from oracle import lb
from paper_2301_01622_gb300 import inputs, llb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ncomp", [1, 2])
def test_zero_steps_are_a_no_op(ncomp):
    n = 12
    if ncomp == 2:
        r1, r2, u = inputs.droplets(n, n, n, [(4.0, 6.0, 6.0), (8.5, 6.0, 6.0)], [2.5, 2.5],
                                    [(0.02, 0, 0), (-0.02, 0, 0)])
        tot = lb.equilibrium_moments(r1 + r2, u)
        m0 = np.ascontiguousarray(np.concatenate([r1[None], r2[None], tot[1:]]))
    else:
        m0 = inputs.random_moments(n, n, n, seed=2)
    p = llb.llb_params_default(storage=llb.LLB_F64, ncomp=ncomp)
    ctx = llb.llb_create(n, n, n, 19, 0.8, p)
    try:
        llb.llb_init_moments(ctx, m0)
        ref = llb.llb_get_moments(ctx, np.empty(m0.shape))
        llb.llb_step(ctx, 0)
        llb.llb_step_graph(ctx, 0)
        assert llb.llb_steps_done(ctx) == 0
        assert np.array_equal(llb.llb_get_moments(ctx, np.empty(m0.shape)), ref)
        for bad in (-1,):
            with pytest.raises(llb.LLBError) as e:
                llb.llb_step(ctx, bad)
            assert e.value.status == llb.LLB_EINVAL
        if ncomp == 1:
            with pytest.raises(llb.LLBError) as e:
                llb.llb_step_host(ctx, m0, np.empty_like(m0), 0)
            assert e.value.status == llb.LLB_EINVAL
    finally:
        llb.llb_destroy(ctx)


@pytest.mark.parametrize("storage", [llb.LLB_F64, llb.LLB_F32], ids=["f64", "f32"])
def test_adjoint_of_zero_steps_is_the_identity(storage):
    n = 10
    m0 = inputs.random_moments(n, n, n, seed=6)
    g = np.random.default_rng(8).uniform(-1, 1, m0.shape)
    ctx = llb.llb_create(n, n, n, 19, 0.8, llb.llb_params_default(storage=storage))
    try:
        llb.llb_init_moments(ctx, m0)
        gfin = torch.from_numpy(g).cuda()
        gini = torch.empty_like(gfin)
        dtau = llb.llb_adjoint(ctx, 0, gfin, gini)
        back = llb.llb_get_moments(ctx, np.empty(m0.shape))
    finally:
        llb.llb_destroy(ctx)
    tol = 1e-15 if storage == llb.LLB_F64 else 1e-6
    assert dtau == 0.0
    assert np.abs(gini.cpu().numpy() - g).max() <= tol * np.abs(g).max()
    assert np.abs(back - m0).max() <= (1e-15 if storage == llb.LLB_F64 else 1e-6)


def test_batch_zero_steps_are_a_no_op():
    dims = [(8, 8, 8), (12, 9, 6)]
    p = llb.llb_params_default(ncomp=2, storage=llb.LLB_F64)
    b = llb.llb_batch_create(dims, 19, 0.9, p)
    try:
        refs = []
        for k, d in enumerate(dims):
            r1, r2, u = inputs.droplets(*d, [(d[0] / 2, d[1] / 2, d[2] / 2)], [2.0], [(0.01, 0, 0)])
            llb.llb_init_equilibrium(llb.llb_batch_domain(b, k), np.stack([r1, r2]), u)
            refs.append(llb.llb_get_moments(llb.llb_batch_domain(b, k), np.empty((11,) + d[::-1])))
        llb.llb_batch_step(b, 0)
        llb.llb_batch_step_graph(b, 0)
        for k, d in enumerate(dims):
            ctx = llb.llb_batch_domain(b, k)
            assert llb.llb_steps_done(ctx) == 0
            assert np.array_equal(llb.llb_get_moments(ctx, np.empty((11,) + d[::-1])), refs[k])
    finally:
        llb.llb_batch_destroy(b)
