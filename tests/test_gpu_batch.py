"""Batched ensembles: boxes of different sizes advanced by one persistent
launch per step give exactly what each box gives alone, and the oracle's
two-component step."""
import numpy as np
import pytest

from oracle import D3Q19, D3Q27, lb
from oracle import two_component as tc
from paper_2301_01622_gb300 import inputs, llb

from gpu_helpers import assert_groups

pytestmark = pytest.mark.gpu

DIMS = [(24, 20, 16), (33, 17, 12), (16, 16, 16), (40, 24, 20), (70, 9, 5)]
LAT = {19: D3Q19, 27: D3Q27}
GROUPS_2 = {"rho": slice(0, 2), "j": slice(2, 5), "P": slice(5, 11)}


def _field(d, k):
    nx, ny, nz = d
    r = max(2.5, min(nx, ny, nz) / 6)
    c1 = (nx / 2 - r - 1.5, ny / 2 - 0.5, nz / 2)
    c2 = (nx / 2 + r + 1.5, ny / 2 + 0.5, nz / 2)
    return inputs.droplets(nx, ny, nz, [c1, c2], [r, r], [(0.03 + 0.01 * k, 0, 0), (-0.03, 0, 0)])


def _params(storage):
    return llb.llb_params_default(ncomp=2, storage=storage, A_h=0.01, A_s=0.02, beta=0.7,
                                  g_min=1e-8 if storage == llb.LLB_F64 else 1e-6)


def _run_alone(d, k, q, steps, storage):
    r1, r2, u = _field(d, k)
    ctx = llb.llb_create(*d, q, 0.9, _params(storage))
    try:
        llb.llb_init_equilibrium(ctx, np.stack([r1, r2]), u)
        llb.llb_step(ctx, steps)
        return llb.llb_get_moments(ctx, np.empty((11,) + d[::-1]))
    finally:
        llb.llb_destroy(ctx)


def _run_batch(q, steps, storage, graph=False, tune=False):
    b = llb.llb_batch_create(DIMS, q, 0.9, _params(storage))
    try:
        for k, d in enumerate(DIMS):
            r1, r2, u = _field(d, k)
            llb.llb_init_equilibrium(llb.llb_batch_domain(b, k), np.stack([r1, r2]), u)
        if tune:
            llb.llb_batch_autotune(b, 2)
        if graph:
            llb.llb_batch_step_graph(b, steps // 2)
            llb.llb_batch_step_graph(b, steps - steps // 2)
        else:
            llb.llb_batch_step(b, steps)
        assert llb.llb_batch_nodes(b) == sum(int(np.prod(d)) for d in DIMS)
        out = []
        for k, d in enumerate(DIMS):
            ctx = llb.llb_batch_domain(b, k)
            assert llb.llb_steps_done(ctx) == steps
            out.append(llb.llb_get_moments(ctx, np.empty((11,) + d[::-1])))
        return out
    finally:
        llb.llb_batch_destroy(b)


@pytest.mark.parametrize("q", [19, 27])
def test_batch_equals_boxes_alone(q):
    steps = 12
    got = _run_batch(q, steps, llb.LLB_F32)
    for k, d in enumerate(DIMS):
        assert np.array_equal(got[k], _run_alone(d, k, q, steps, llb.LLB_F32)), d


@pytest.mark.parametrize("q", [19, 27])
def test_batch_graph_and_autotune(q):
    """Graph replay is bit-identical to plain launches; the autotuned tile
    variant (another instantiation, possibly fused differently by the
    compiler) agrees to FP32 rounding."""
    steps = 9
    a = _run_batch(q, steps, llb.LLB_F32)
    b = _run_batch(q, steps, llb.LLB_F32, graph=True)
    c = _run_batch(q, steps, llb.LLB_F32, graph=True, tune=True)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y)
        assert_groups(z, x, 1e-6, GROUPS_2, what="autotuned variant")


def test_batch_box_matches_oracle():
    steps = 6
    got = _run_batch(27, steps, llb.LLB_F64)
    prm = tc.CGParams(beta=0.7, A_s=0.02, A_h=0.01, h_c=3, g_min=1e-8)
    for k in (0, 4):
        r1, r2, u = _field(DIMS[k], k)
        tot = lb.equilibrium_moments(r1 + r2, u)
        m0 = np.concatenate([r1[None], r2[None], tot[1:]])
        ref = tc.run_moment_only(m0, D3Q27, 0.9, prm, steps)
        assert_groups(got[k], ref, 1e-12, GROUPS_2, what=f"box {DIMS[k]}")


def test_borrowed_box_cannot_step_alone():
    b = llb.llb_batch_create(DIMS[:2], 19, 0.9, _params(llb.LLB_F32))
    try:
        ctx = llb.llb_batch_domain(b, 0)
        with pytest.raises(llb.LLBError):
            llb.llb_step(ctx, 1)
        llb.llb_destroy(ctx)   # ignored: the batch owns the box
        llb.llb_batch_step(b, 1)
        assert llb.llb_steps_done(llb.llb_batch_domain(b, 1)) == 1
    finally:
        llb.llb_batch_destroy(b)
