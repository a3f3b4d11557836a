"""Hand-written adjoint of the moment-only step: gradients with respect to
the initial moments, an initial velocity field and tau, checked against
central finite differences (FP64) of the library's own forward run and of the
FP64 oracle, and between checkpoint intervals."""
import numpy as np
import pytest

from oracle import D3Q19, D3Q27, lb
from paper_2301_01622_gb300 import inputs, llb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAT = {19: D3Q19, 27: D3Q27}


def _m0(n, seed, dtype=torch.float64):
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=seed)
    m = lb.equilibrium_moments(rho, u)
    m[4:] += 1e-3 * inputs.random_moments(n, n, n, seed=seed + 1)[4:]   # some non-equilibrium part
    return torch.from_numpy(m).to(device="cuda", dtype=dtype)


def _loss(mN, w):
    # a non-linear field-mismatch loss: 0.5 |u - w|^2 with u = j / rho, plus the
    # squared deviatoric flux (kept O(u^2) so that central differences are not
    # swamped by the rounding of a large constant part)
    u = mN[1:4] / mN[0]
    dev = torch.cat([mN[4:7] - mN[0] / 3.0, mN[7:]])
    return 0.5 * ((u - w) ** 2).sum() + 10.0 * (dev * dev).sum()


@pytest.mark.parametrize("q", [19, 27])
def test_gradient_vs_finite_differences(q):
    from paper_2301_01622_gb300.autograd import evolve
    n, steps, tau0 = 12, 25, 0.8
    m0 = _m0(n, 3 + q).requires_grad_(True)
    tau = torch.tensor(tau0, dtype=torch.float64, requires_grad=True)
    w = torch.zeros((3, n, n, n), dtype=torch.float64, device="cuda")
    L = _loss(evolve(m0, tau, steps, lattice=q, every=5), w)
    L.backward()
    g = m0.grad.detach().cpu().numpy()
    gt = float(tau.grad)
    rng = np.random.default_rng(q)
    eps = 1e-6
    with torch.no_grad():
        for _ in range(6):
            f, z, y, x = int(rng.integers(10)), int(rng.integers(n)), int(rng.integers(n)), int(rng.integers(n))
            mp, mm = m0.detach().clone(), m0.detach().clone()
            mp[f, z, y, x] += eps
            mm[f, z, y, x] -= eps
            fd = (float(_loss(evolve(mp, tau0, steps, lattice=q), w)) -
                  float(_loss(evolve(mm, tau0, steps, lattice=q), w))) / (2 * eps)
            assert abs(fd - g[f, z, y, x]) <= 1e-4 * max(abs(fd), 1e-6), (f, fd, g[f, z, y, x])
        fd = (float(_loss(evolve(m0.detach(), tau0 + eps, steps, lattice=q), w)) -
              float(_loss(evolve(m0.detach(), tau0 - eps, steps, lattice=q), w))) / (2 * eps)
        assert abs(fd - gt) <= 1e-4 * abs(fd)


def test_gradient_wrt_initial_velocity():
    """Through an equilibrium initialisation written in torch: dL/du0."""
    from paper_2301_01622_gb300.autograd import evolve
    n, steps, tau0 = 10, 20, 0.7
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=11)
    u0 = torch.from_numpy(u).cuda().requires_grad_(True)
    target = torch.from_numpy(inputs.taylor_green_3d(n, n, n, u0=0.04, seed=12)[1]).cuda()

    def run(uu):
        rho_t = torch.ones((n, n, n), dtype=torch.float64, device="cuda")
        j = rho_t * uu
        P = [rho_t / 3 * (a == b) + rho_t * uu[a] * uu[b] for (a, b) in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))]
        m0 = torch.stack([rho_t, j[0], j[1], j[2]] + P)
        mN = evolve(m0, tau0, steps)
        return 0.5 * ((mN[1:4] / mN[0] - target) ** 2).sum()

    run(u0).backward()
    g = u0.grad.cpu().numpy()
    eps = 1e-6
    with torch.no_grad():
        for (a, z, y, x) in [(0, 1, 2, 3), (1, 5, 5, 5), (2, 9, 0, 4)]:
            up, um = u0.detach().clone(), u0.detach().clone()
            up[a, z, y, x] += eps
            um[a, z, y, x] -= eps
            fd = (float(run(up)) - float(run(um))) / (2 * eps)
            assert abs(fd - g[a, z, y, x]) <= 1e-4 * max(abs(fd), 1e-6)


def test_checkpoint_interval_does_not_change_the_gradient():
    n, steps = 16, 30
    m0 = _m0(n, 5)
    g = torch.randn((10, n, n, n), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    out = []
    for every in (1, 4, 7, 30, 0):
        c = llb.llb_create(n, n, n, 19, 0.75, llb.llb_params_default(storage=llb.LLB_F64))
        try:
            llb.llb_init_moments_device(c, m0)
            gi = torch.empty_like(m0)
            dt = llb.llb_adjoint(c, steps, g, gi, every=every)
            after = torch.empty_like(m0)
            llb.llb_get_moments_device(c, after)
            llb.llb_synchronize(c)
            assert torch.equal(after, m0) or float((after - m0).abs().max()) < 1e-15  # state restored
        finally:
            llb.llb_destroy(c)
        out.append((gi, dt))
    for gi, dt in out[1:]:
        assert torch.equal(gi, out[0][0]) and dt == out[0][1]


def test_gradient_vs_oracle_finite_differences():
    """Reference gradient from the FP64 oracle (central differences of
    oracle runs) for a linear functional of the final moments."""
    n, steps, tau = 6, 8, 0.8
    m0 = inputs.random_moments(n, n, n, seed=17)
    rng = np.random.default_rng(2)
    wfin = rng.standard_normal((10, n, n, n))
    m0t = torch.from_numpy(m0).cuda()
    c = llb.llb_create(n, n, n, 27, tau, llb.llb_params_default(storage=llb.LLB_F64))
    try:
        llb.llb_init_moments_device(c, m0t)
        gi = torch.empty_like(m0t)
        dtau = llb.llb_adjoint(c, steps, torch.from_numpy(wfin).cuda(), gi, every=3)
    finally:
        llb.llb_destroy(c)
    gi = gi.cpu().numpy()

    def J(m, t):
        return float((wfin * lb.run_moment_only(m, D3Q27, t, steps)).sum())

    eps = 1e-6
    for (f, z, y, x) in [(0, 1, 2, 3), (2, 0, 0, 0), (5, 4, 1, 2), (8, 5, 5, 5), (9, 2, 3, 1)]:
        mp, mm = m0.copy(), m0.copy()
        mp[f, z, y, x] += eps
        mm[f, z, y, x] -= eps
        fd = (J(mp, tau) - J(mm, tau)) / (2 * eps)
        assert abs(fd - gi[f, z, y, x]) <= 1e-6 * max(abs(fd), 1.0)
    fd = (J(m0, tau + eps) - J(m0, tau - eps)) / (2 * eps)
    assert abs(fd - dtau) <= 1e-6 * max(abs(fd), 1.0)


def test_fp32_adjoint_runs_and_matches_fp64():
    """FP32 forward and adjoint (the bench configuration's precision) agree
    with the FP64 adjoint to FP32 accuracy on 32^3, 60 steps."""
    n, steps = 32, 60
    m64 = _m0(n, 9)
    g = torch.randn((10, n, n, n), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    res = {}
    for st, dt in ((llb.LLB_F64, torch.float64), (llb.LLB_F32, torch.float32)):
        c = llb.llb_create(n, n, n, 19, 0.7, llb.llb_params_default(storage=st))
        try:
            llb.llb_init_moments_device(c, m64.to(dt))
            gi = torch.empty((10, n, n, n), dtype=dt, device="cuda")
            dtau = llb.llb_adjoint(c, steps, g.to(dt), gi)
        finally:
            llb.llb_destroy(c)
        res[st] = (gi.double(), dtau)
    a, b = res[llb.LLB_F64], res[llb.LLB_F32]
    assert float((a[0] - b[0]).abs().max() / a[0].abs().max()) < 1e-4
    assert abs(a[1] - b[1]) < 1e-4 * abs(a[1])
