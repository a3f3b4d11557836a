"""Hand-written adjoint of the two-component moment-only step (colour
gradient with the smooth interface normal, no near-contact switch): the
gradient of a phase-field mismatch loss with respect to the initial moments
and tau, checked against FP64 central differences of the library's own
forward run (16^3 off-axis droplet pair), across checkpoint intervals, and in
FP32 against FP64."""
import numpy as np
import pytest

from oracle import lb
from paper_2301_01622_gb300 import inputs, llb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, STEPS, TAU = 16, 20, 0.9
PRM = dict(ncomp=2, beta=0.7, A_s=0.02, A_h=0.0, grad_eps=0.02)


def _m0(speed=0.05, seed=None):
    c1 = (N / 2 - 5.0, N / 2 - 1.0, N / 2)
    c2 = (N / 2 + 5.0, N / 2 + 1.0, N / 2)
    r1, r2, u = inputs.droplets(N, N, N, [c1, c2], [4.0, 4.0], [(speed, 0, 0), (-speed, 0, 0)])
    if seed is not None:   # seeded perturbation of the initial droplet velocities
        u = u + 0.01 * np.random.default_rng(seed).uniform(-1, 1, u.shape) * (r1 > 0.5)
    tot = lb.equilibrium_moments(r1 + r2, u)
    return np.ascontiguousarray(np.concatenate([r1[None], r2[None], tot[1:]]))


def _forward(m0, tau, storage=llb.LLB_F64, steps=STEPS):
    ctx = llb.llb_create(N, N, N, 27, tau, llb.llb_params_default(storage=storage, **PRM))
    try:
        llb.llb_init_moments(ctx, m0)
        llb.llb_step(ctx, steps)
        return llb.llb_get_moments(ctx, np.empty((11, N, N, N)))
    finally:
        llb.llb_destroy(ctx)


def _phi(m):
    return (m[0] - m[1]) / (m[0] + m[1])


def _loss_and_grad(mN, target):
    """L = sum (phi - phi_target)^2 and dL/dm_N (canonical fields)."""
    phi = _phi(mN)
    r = phi - target
    rho = mN[0] + mN[1]
    g = np.zeros_like(mN)
    g[0] = 2 * r * 2 * mN[1] / rho ** 2
    g[1] = -2 * r * 2 * mN[0] / rho ** 2
    return float((r * r).sum()), g


def _adjoint(m0, gN, tau, storage=llb.LLB_F64, every=5):
    ctx = llb.llb_create(N, N, N, 27, tau, llb.llb_params_default(storage=storage, **PRM))
    try:
        llb.llb_init_moments(ctx, m0)
        gfin = torch.from_numpy(gN).cuda()
        gini = torch.empty_like(gfin)
        dtau = llb.llb_adjoint(ctx, STEPS, gfin, gini, every=every)
        back = llb.llb_get_moments(ctx, np.empty((11, N, N, N)))
        return gini.cpu().numpy(), dtau, back
    finally:
        llb.llb_destroy(ctx)


@pytest.fixture(scope="module")
def case():
    target = _phi(_forward(_m0(seed=7), TAU))
    m0 = _m0()
    L, gN = _loss_and_grad(_forward(m0, TAU), target)
    g0, dtau, back = _adjoint(m0, gN, TAU)
    return m0, target, L, g0, dtau, back


def test_adjoint_restores_state_and_is_nontrivial(case):
    m0, _, L, g0, dtau, back = case
    np.testing.assert_allclose(back, m0, rtol=0, atol=1e-15)
    assert L > 0 and np.abs(g0).max() > 0 and dtau != 0


def test_gradient_vs_finite_differences(case):
    m0, target, _, g0, dtau, _ = case
    h = 1e-6
    scale = np.abs(g0[2:5]).max()
    # the largest j entries of the gradient plus a few rho1 entries near the interface
    flat = np.argsort(np.abs(g0[2:5]).ravel())[::-1][:5]
    picks = [(2 + i // (N ** 3),) + tuple(np.unravel_index(i % N ** 3, (N, N, N))) for i in flat]
    band = np.argwhere((m0[0] > 0.2) & (m0[0] < 0.8))
    for z, y, x in band[np.random.default_rng(1).choice(len(band), 3, replace=False)]:
        picks.append((0, z, y, x))
    for f, z, y, x in picks:
        mp, mm = m0.copy(), m0.copy()
        mp[f, z, y, x] += h
        mm[f, z, y, x] -= h
        fd = (_loss_and_grad(_forward(mp, TAU), target)[0] - _loss_and_grad(_forward(mm, TAU), target)[0]) / (2 * h)
        assert abs(fd - g0[f, z, y, x]) <= 1e-4 * max(abs(fd), 1e-2 * scale), (f, z, y, x, fd, g0[f, z, y, x])
    fd = (_loss_and_grad(_forward(m0, TAU + h), target)[0] - _loss_and_grad(_forward(m0, TAU - h), target)[0]) / (2 * h)
    assert abs(fd - dtau) <= 1e-4 * abs(fd), (fd, dtau)


def test_checkpoint_interval_does_not_change_gradient(case):
    m0, target, _, g0, dtau, _ = case
    _, gN = _loss_and_grad(_forward(m0, TAU), target)
    g1, dt1, _ = _adjoint(m0, gN, TAU, every=1)
    g7, dt7, _ = _adjoint(m0, gN, TAU, every=7)
    np.testing.assert_array_equal(g1, g0)
    np.testing.assert_array_equal(g7, g0)
    assert dt1 == dtau and dt7 == dtau


def test_fp32_adjoint_close_to_fp64(case):
    m0, target, _, g0, dtau, _ = case
    mN32 = _forward(m0, TAU, storage=llb.LLB_F32)
    _, gN = _loss_and_grad(mN32, target)
    g32, dt32, _ = _adjoint(m0, gN, TAU, storage=llb.LLB_F32)
    err = np.abs(g32[2:5] - g0[2:5]).max() / np.abs(g0[2:5]).max()
    assert err < 2e-3, err
    assert abs(dt32 - dtau) <= 2e-3 * abs(dtau)


def test_adjoint_requires_smooth_normal_and_no_switch():
    m0 = _m0()
    g = torch.zeros((11, N, N, N), dtype=torch.float64, device="cuda")
    for over in (dict(grad_eps=0.0), dict(A_h=0.01)):
        prm = dict(PRM, **over)
        ctx = llb.llb_create(N, N, N, 27, TAU, llb.llb_params_default(storage=llb.LLB_F64, **prm))
        try:
            llb.llb_init_moments(ctx, m0)
            with pytest.raises(llb.LLBError) as e:
                llb.llb_adjoint(ctx, 2, g, torch.empty_like(g))
            assert e.value.status == llb.LLB_EINVAL
        finally:
            llb.llb_destroy(ctx)


def test_autograd_wrapper_two_components(case):
    """torch.autograd through evolve(..., two_component=...) gives the same
    initial-moment gradient and dL/dtau as the direct adjoint call."""
    from paper_2301_01622_gb300.autograd import evolve
    m0, target, _, g0, dtau, _ = case
    m = torch.from_numpy(m0).cuda().requires_grad_(True)
    tau = torch.tensor(TAU, dtype=torch.float64, requires_grad=True)
    cg = dict(beta=PRM["beta"], A_s=PRM["A_s"], grad_eps=PRM["grad_eps"])
    mN = evolve(m, tau, STEPS, lattice=27, every=5, two_component=cg)
    phi = (mN[0] - mN[1]) / (mN[0] + mN[1])
    L = ((phi - torch.from_numpy(target).cuda()) ** 2).sum()
    L.backward()
    np.testing.assert_allclose(m.grad.cpu().numpy(), g0, rtol=1e-9, atol=1e-12 * np.abs(g0).max())
    assert abs(float(tau.grad) - dtau) <= 1e-9 * abs(dtau)


def test_gradient_vs_oracle_finite_differences():
    """Reference gradient from the FP64 oracle: central differences of the
    oracle's two-component moment-only runs (smooth normal, eps > 0, no
    near-contact force) for a linear functional of the final phase field,
    J = sum w phi(t_N), on a 12^3 off-axis pair, against llb_adjoint's
    gradient with respect to the initial j, rho1 and tau."""
    from oracle import D3Q27
    from oracle import two_component as tc

    n, steps, tau = 12, 6, 0.9
    c1 = (n / 2 - 3.5, n / 2 - 0.5, n / 2)
    c2 = (n / 2 + 3.5, n / 2 + 0.5, n / 2)
    r1, r2, u = inputs.droplets(n, n, n, [c1, c2], [2.5, 2.5], [(0.04, 0, 0), (-0.04, 0, 0)])
    tot = lb.equilibrium_moments(r1 + r2, u)
    m0 = np.ascontiguousarray(np.concatenate([r1[None], r2[None], tot[1:]]))
    w = np.random.default_rng(3).standard_normal((n, n, n))
    prm = tc.CGParams(beta=0.7, A_s=0.02, A_h=0.0, eps=0.02)

    def J(m, t):
        out = tc.run_moment_only(m, D3Q27, t, prm, steps)
        return float((w * (out[0] - out[1]) / (out[0] + out[1])).sum())

    # dJ/dm at the final state: phi = (rho1 - rho2)/(rho1 + rho2)
    fin = tc.run_moment_only(m0, D3Q27, tau, prm, steps)
    rho = fin[0] + fin[1]
    gN = np.zeros_like(fin)
    gN[0] = w * 2 * fin[1] / rho ** 2
    gN[1] = -w * 2 * fin[0] / rho ** 2
    ctx = llb.llb_create(n, n, n, 27, tau, llb.llb_params_default(storage=llb.LLB_F64, **PRM))
    try:
        llb.llb_init_moments(ctx, m0)
        gi = torch.empty((11, n, n, n), dtype=torch.float64, device="cuda")
        dtau = llb.llb_adjoint(ctx, steps, torch.from_numpy(gN).cuda(), gi, every=2)
    finally:
        llb.llb_destroy(ctx)
    gi = gi.cpu().numpy()
    eps = 1e-6
    # interface and bulk nodes; fields rho1, rho2, j_x, j_y, P_xy
    for (f, z, y, x) in [(0, 6, 5, 3), (0, 6, 6, 9), (1, 5, 6, 4), (2, 6, 5, 2), (3, 6, 6, 8), (2, 0, 0, 0), (8, 6, 6, 6)]:
        mp, mm = m0.copy(), m0.copy()
        mp[f, z, y, x] += eps
        mm[f, z, y, x] -= eps
        fd = (J(mp, tau) - J(mm, tau)) / (2 * eps)
        assert abs(fd - gi[f, z, y, x]) <= 1e-5 * max(abs(fd), 0.1), (f, z, y, x, fd, gi[f, z, y, x])
    fd = (J(m0, tau + eps) - J(m0, tau - eps)) / (2 * eps)
    assert abs(fd - dtau) <= 1e-5 * max(abs(fd), 0.1)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("shape", [(37, 11, 9), (70, 6, 5), (16, 16, 16)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("storage", [llb.LLB_F64, llb.LLB_F32], ids=["f64", "f32"])
def test_tiled_first_pass_equals_reference_form(q, shape, storage):
    """The tiled first pass (projections published once per node through a
    shared-memory ring) gives the gradient of the reference one-thread-per-node
    pass on ragged multi-tile boxes: 1e-12 (FP64), 1e-5 (FP32) of the largest
    entry; dL/dtau alike."""
    nx, ny, nz = shape
    r = min(nx, ny, nz) / 4 + 1.0
    r1, r2, u = inputs.droplets(nx, ny, nz, [(nx / 3, ny / 2 - 0.5, nz / 2), (2 * nx / 3, ny / 2 + 0.5, nz / 2)],
                                [r, r], [(0.04, 0, 0), (-0.04, 0, 0)])
    tot = lb.equilibrium_moments(r1 + r2, u)
    m0 = np.ascontiguousarray(np.concatenate([r1[None], r2[None], tot[1:]]))
    g = np.random.default_rng(5).uniform(-1, 1, m0.shape)
    out = []
    for flags in (0, 2):
        ctx = llb.llb_create(nx, ny, nz, q, TAU, llb.llb_params_default(storage=storage, debug_flags=flags, **PRM))
        try:
            llb.llb_init_moments(ctx, m0)
            gfin = torch.from_numpy(g).cuda()
            gini = torch.empty_like(gfin)
            dtau = llb.llb_adjoint(ctx, 6, gfin, gini, every=4)
            out.append((gini.cpu().numpy(), dtau))
        finally:
            llb.llb_destroy(ctx)
    (gt, dt), (gr, dr) = out
    tol = 1e-12 if storage == llb.LLB_F64 else 1e-5
    assert np.isfinite(gt).all()
    assert np.abs(gt - gr).max() <= tol * np.abs(gr).max()
    assert abs(dt - dr) <= tol * abs(dr)
