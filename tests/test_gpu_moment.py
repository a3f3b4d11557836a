"""GPU parity of the moment-only step (one component) against the FP64 oracle.

Tolerances: FP64 storage 1e-12 relative, FP32 storage 1e-5 relative after
200 steps, measured per moment group (rho; j; P) as
max |gpu - oracle| / max |oracle| over the group's fields.
"""
import functools

import numpy as np
import pytest

from oracle import D3Q19, D3Q27, lb
from oracle import diagnostics as odg
from paper_2301_01622_gb300 import inputs, llb

from gpu_helpers import assert_groups, run_gpu

pytestmark = pytest.mark.gpu

LAT = {19: D3Q19, 27: D3Q27}
KERNELS = [llb.LLB_KERNEL_TMA, llb.LLB_KERNEL_TILED, llb.LLB_KERNEL_DIRECT]
KIDS = ["tma", "tiled", "direct"]


def tma_fits(shape):
    """The FP64 TMA kernel (tile 32 x 8) needs a padded row of >= 40 elements and >= 10 rows."""
    nx, ny, _ = shape
    return ((nx + 16 + 7) // 8) * 8 >= 40 and ny + 2 >= 10


@functools.lru_cache(maxsize=None)
def oracle_tg(q, n, tau, steps, noise):
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=noise, seed=2301)
    return lb.run_moment_only(lb.equilibrium_moments(rho, u), LAT[q], tau, steps)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("kernel", KERNELS, ids=KIDS)
def test_taylor_green_fp64_200_steps(q, kernel):
    """32^3 Taylor-Green, u0 = 0.05, tau = 0.8, FP64, 200 steps: 1e-12."""
    n, tau = 32, 0.8
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05)
    got, used = run_gpu((n, n, n), q, tau, 200, rho=rho, u=u, storage=llb.LLB_F64, kernel=kernel)
    assert used == kernel
    assert_groups(got, oracle_tg(q, n, tau, 200, 0.0), 1e-12, what=f"D3Q{q} fp64")


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("kernel", KERNELS, ids=KIDS)
def test_taylor_green_fp32_200_steps(q, kernel):
    """Same run with FP32 storage and arithmetic: 1e-5 after 200 steps."""
    n, tau = 32, 0.8
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05)
    # the default FP32 TMA tile (64 x 4) is wider than this box; variant 2 is 32 x 8
    variant = 2 if kernel == llb.LLB_KERNEL_TMA else 0
    got, used = run_gpu((n, n, n), q, tau, 200, rho=rho, u=u, storage=llb.LLB_F32, kernel=kernel, variant=variant)
    assert used == kernel
    assert_groups(got, oracle_tg(q, n, tau, 200, 0.0), 1e-5, what=f"D3Q{q} fp32")


@pytest.mark.parametrize("q", [19, 27])
def test_noisy_taylor_green_fp32_tau06(q):
    """The bench workload's field (Taylor-Green + 1e-3 noise, tau = 0.6) on 32^3, FP32, 200 steps."""
    n, tau = 32, 0.6
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=2301)
    got, _ = run_gpu((n, n, n), q, tau, 200, rho=rho, u=u, storage=llb.LLB_F32)
    assert_groups(got, oracle_tg(q, n, tau, 200, 1e-3), 1e-5, what=f"D3Q{q} fp32 noisy")


SHAPES = [(67, 45, 37), (33, 9, 5), (31, 17, 3), (5, 70, 2), (1, 1, 1), (2, 3, 4), (4, 4, 4), (64, 16, 8), (97, 1, 3),
          (25, 8, 1), (129, 40, 2), (17, 8, 70), (300, 12, 9)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("kernel", KERNELS, ids=KIDS)
def test_ragged_shapes_random_moments_fp64(shape, q, kernel):
    """Random non-equilibrium moments, shapes spanning several tiles, ragged
    tails and degenerate 1- and 2-node axes: 1e-12 after 3 steps."""
    nx, ny, nz = shape
    if kernel == llb.LLB_KERNEL_TMA and not tma_fits(shape):
        with pytest.raises(llb.LLBError) as e:
            run_gpu(shape, q, 0.7, 1, m0=inputs.random_moments(nx, ny, nz, seed=1), kernel=kernel)
        assert e.value.status == llb.LLB_EINVAL
        return
    m0 = inputs.random_moments(nx, ny, nz, seed=nx * 10007 + ny * 101 + nz)
    ref = lb.run_moment_only(m0, LAT[q], 0.7, 3)
    got, used = run_gpu(shape, q, 0.7, 3, m0=m0, storage=llb.LLB_F64, kernel=kernel)
    assert used == kernel
    assert_groups(got, ref, 1e-12, what=f"{shape} D3Q{q}")


@functools.lru_cache(maxsize=None)
def _oracle_ragged(q):
    rho, u = inputs.taylor_green_3d(133, 37, 29, u0=0.05, noise=1e-3, seed=7)
    return lb.run_moment_only(lb.equilibrium_moments(rho, u), LAT[q], 0.7, 20)


KERNEL_VARIANTS = [(llb.LLB_KERNEL_TMA, v) for v in range(3)] + [(llb.LLB_KERNEL_TILED, v) for v in range(6)]


@pytest.mark.parametrize("kernel, variant", KERNEL_VARIANTS,
                         ids=[f"{'tma' if k == llb.LLB_KERNEL_TMA else 'tiled'}-v{v}" for k, v in KERNEL_VARIANTS])
@pytest.mark.parametrize("q", [19, 27])
def test_kernel_variants_match_oracle(variant, kernel, q):
    """Every tuning variant of the z-marching kernels (tile shape, ring depth,
    CTAs/SM, split-phase plane barrier, approximate 1/rho, L2 prefetch) computes the same
    step: ragged multi-tile box, FP32, 1e-5 after 20 steps."""
    shape = (133, 37, 29)
    rho, u = inputs.taylor_green_3d(*shape, u0=0.05, noise=1e-3, seed=7)
    try:
        got, used = run_gpu(shape, q, 0.7, 20, rho=rho, u=u, storage=llb.LLB_F32, kernel=kernel, variant=variant)
    except llb.LLBError as e:
        # a variant whose shared memory does not fit this lattice is refused at creation
        assert e.status == llb.LLB_EINVAL
        pytest.skip("variant does not fit on this lattice")
    assert used == kernel
    assert_groups(got, _oracle_ragged(q), 1e-5, what=f"variant {variant}")


def test_tma_kernel_has_three_variants():
    """Variants 3..5 exist for the plain-load kernel only: asking the TMA
    kernel for one is refused at creation, and variant 6 for either kernel."""
    with pytest.raises(llb.LLBError) as e:
        llb.llb_create(64, 64, 64, 19, 0.8, llb.llb_params_default(kernel=llb.LLB_KERNEL_TILED, variant=6))
    assert e.value.status == llb.LLB_EINVAL
    p = llb.llb_params_default(kernel=llb.LLB_KERNEL_TMA, variant=3)
    with pytest.raises(llb.LLBError) as e:
        llb.llb_create(64, 64, 64, 19, 0.8, p)
    assert e.value.status == llb.LLB_EINVAL


@pytest.mark.parametrize("q", [19, 27])
def test_zero_steps_round_trip(q):
    m0 = inputs.random_moments(7, 5, 3, seed=3)
    got, _ = run_gpu((7, 5, 3), q, 0.9, 0, m0=m0, storage=llb.LLB_F64)
    np.testing.assert_allclose(got, m0, rtol=0, atol=2e-16)


@pytest.mark.parametrize("q", [19, 27])
def test_tiled_is_deterministic_and_matches_direct(q):
    n = 40
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=5)
    a, _ = run_gpu((n, n, n), q, 0.6, 20, rho=rho, u=u, storage=llb.LLB_F32, kernel=llb.LLB_KERNEL_TMA, variant=2)
    b, _ = run_gpu((n, n, n), q, 0.6, 20, rho=rho, u=u, storage=llb.LLB_F32, kernel=llb.LLB_KERNEL_TMA, variant=2)
    c, _ = run_gpu((n, n, n), q, 0.6, 20, rho=rho, u=u, storage=llb.LLB_F32, kernel=llb.LLB_KERNEL_TILED)
    d, _ = run_gpu((n, n, n), q, 0.6, 20, rho=rho, u=u, storage=llb.LLB_F32, kernel=llb.LLB_KERNEL_DIRECT)
    assert np.array_equal(a, b)
    assert_groups(a, c, 1e-6, what="tma vs tiled")
    assert_groups(a, d, 1e-6, what="tma vs direct")


def _sample_nodes(nx, ny, nz, rng, count=60):
    pts = set()
    for x in (0, 1, 30, 31, 32, 33, nx - 1):
        for y in (0, 7, 8, ny - 1):
            for z in (0, nz // 2, nz - 1):
                pts.add((x % nx, y % ny, z % nz))
    for _ in range(count):
        pts.add((int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))))
    return sorted(pts)


@pytest.mark.parametrize("q", [19, 27])
def test_full_size_256_sampled_nodes(q):
    """The bench configuration (256^3, Taylor-Green + 1e-3 noise, tau = 0.6,
    FP32, the kernel bench.py times): one step, sampled nodes against the
    oracle's per-node evaluation of the same initial field."""
    n, tau = 256, 0.6
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=2301)
    m0 = lb.equilibrium_moments(rho, u)
    got, used = run_gpu((n, n, n), q, tau, 1, rho=rho, u=u, storage=llb.LLB_F32, kernel=llb.LLB_KERNEL_AUTO)
    assert used == llb.LLB_KERNEL_TILED
    rng = np.random.default_rng(q)
    pts = _sample_nodes(n, n, n, rng)
    ref = np.stack([lb.node_moment_only(m0, LAT[q], tau, x, y, z) for (x, y, z) in pts], axis=1)
    gs = np.stack([got[:, z, y, x] for (x, y, z) in pts], axis=1)
    assert_groups(gs[:, :, None, None], ref[:, :, None, None], 1e-6, what="256^3 sampled")


@pytest.mark.parametrize("q", [19, 27])
def test_full_size_conservation(q):
    """Mass and momentum over 50 steps of the 256^3 FP32 bench workload (FP64 reductions)."""
    n, tau = 256, 0.6
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=2301)
    p = llb.llb_params_default(storage=llb.LLB_F32)
    ctx = llb.llb_create(n, n, n, q, tau, p)
    try:
        llb.llb_init_equilibrium(ctx, rho, u)
        d0 = llb.llb_diagnostics(ctx)
        llb.llb_step(ctx, 50)
        d1 = llb.llb_diagnostics(ctx)
    finally:
        llb.llb_destroy(ctx)
    N = n ** 3
    # exact in exact arithmetic; FP32 storage rounds each node's density
    # deviation every step, which moves the total by ~1e-11 relative here
    assert abs(d1["mass"][0] - d0["mass"][0]) <= 1e-9 * N
    for a in range(3):
        assert abs(d1["momentum"][a] - d0["momentum"][a]) <= 1e-9 * N
    assert d1["flags"] == 0 and d1["min_rho"] > 0.9


@pytest.mark.parametrize("storage", [llb.LLB_F64, llb.LLB_F32])
def test_diagnostics_match_oracle(storage):
    """llb_diagnostics vs the oracle's FP64 diagnostics on the same field."""
    nx, ny, nz = 45, 33, 17
    m0 = inputs.random_moments(nx, ny, nz, seed=17, rho_spread=0.6)
    if storage == llb.LLB_F32:
        # the device stores d = rho - 1 in FP32; give the oracle the same values
        d32 = (m0[0] - 1.0).astype(np.float32).astype(np.float64)
        m0 = m0.copy()
        m0[0] = 1.0 + d32
        m0[1:4] = m0[1:4].astype(np.float32).astype(np.float64)
    p = llb.llb_params_default(storage=storage)
    ctx = llb.llb_create(nx, ny, nz, 19, 0.8, p)
    try:
        llb.llb_init_moments(ctx, m0)
        d = llb.llb_diagnostics(ctx)
    finally:
        llb.llb_destroy(ctx)
    ref = odg.diagnostics(m0, ncomp=1)
    assert d["n_in"] == ref["n_in"]
    assert abs(d["mass"][0] - ref["mass"][0]) <= 1e-12 * abs(ref["mass"][0])
    for a in range(3):
        assert abs(d["momentum"][a] - ref["momentum"][a]) <= 1e-12 * nx * ny * nz
    assert abs(d["rho1_avg"] - ref["rho1_avg"]) <= 1e-13
    assert abs(d["min_rho"] - ref["min_rho"]) <= 1e-15
    assert d["flags"] == 0


def test_init_rejects_unphysical_input():
    """rho <= 0 or NaN in the input is reported as LLB_EUNSTABLE (checked on the device)."""
    m0 = inputs.random_moments(8, 8, 8, seed=2)
    bad = m0.copy()
    bad[0, 3, 3, 3] = -0.5
    nan = m0.copy()
    nan[6, 1, 2, 3] = np.nan
    ctx = llb.llb_create(8, 8, 8, 19, 0.8, llb.llb_params_default())
    try:
        for b in (bad, nan):
            with pytest.raises(llb.LLBError) as e:
                llb.llb_init_moments(ctx, b)
            assert e.value.status == llb.LLB_EUNSTABLE
        llb.llb_init_moments(ctx, m0)  # the context is still usable
        llb.llb_step(ctx, 2)
        assert llb.llb_steps_done(ctx) == 2
    finally:
        llb.llb_destroy(ctx)


def test_diagnostics_flag_nonfinite_state():
    """A non-finite value in the state (loaded through the unchecked device
    path) is flagged by the diagnostics, and propagates through a step."""
    torch = pytest.importorskip("torch")
    m0 = inputs.random_moments(16, 16, 16, seed=4)
    m0[5, 2, 3, 4] = np.inf
    ctx = llb.llb_create(16, 16, 16, 19, 0.8, llb.llb_params_default(storage=llb.LLB_F64))
    try:
        dev = torch.from_numpy(m0).cuda()
        torch.cuda.synchronize()
        llb.llb_init_moments_device(ctx, dev)
        d0 = llb.llb_diagnostics(ctx)
        llb.llb_step(ctx, 1)
        d1 = llb.llb_diagnostics(ctx)
    finally:
        llb.llb_destroy(ctx)
    assert d0["flags"] & llb.LLB_FLAG_NONFINITE
    assert d1["flags"] & llb.LLB_FLAG_NONFINITE


@pytest.mark.parametrize("q", [19, 27])
def test_checkpoint_restart(q):
    """A checkpoint is the moment field: stopping, saving in FP64 and
    restarting reproduces a continuous FP64 run to round-off."""
    n, tau = 24, 0.7
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=8)
    full, _ = run_gpu((n, n, n), q, tau, 30, rho=rho, u=u, storage=llb.LLB_F64)
    half, _ = run_gpu((n, n, n), q, tau, 15, rho=rho, u=u, storage=llb.LLB_F64)
    rest, _ = run_gpu((n, n, n), q, tau, 15, m0=half, storage=llb.LLB_F64)
    assert_groups(rest, full, 1e-14, what="restart")


@pytest.mark.parametrize("ncomp", [1, 2])
@pytest.mark.parametrize("storage", [llb.LLB_F32, llb.LLB_F64], ids=["f32", "f64"])
def test_bit_identical_restart_from_the_raw_state(storage, ncomp):
    """A checkpoint of the raw state copy (caller-owned buffers, saved after
    15 steps and written into a fresh context's current copy) resumes the run
    bit for bit: 15 + 15 steps equal 30 continuous steps exactly."""
    torch = pytest.importorskip("torch")
    n, q, tau = 24, 27 if ncomp == 2 else 19, 0.8
    if ncomp == 2:
        r1, r2, u = inputs.droplets(n, n, n, [(8.0, 11.5, 12.0), (16.0, 12.5, 12.0)], [3.5, 3.5],
                                    [(0.03, 0, 0), (-0.03, 0, 0)])
        tot = lb.equilibrium_moments(r1 + r2, u)
        m0 = np.ascontiguousarray(np.concatenate([r1[None], r2[None], tot[1:]]))
        kw = dict(ncomp=2, beta=0.7, A_s=0.02, A_h=0.01)
    else:
        m0 = lb.equilibrium_moments(*inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=3))
        kw = {}
    dt = torch.float32 if storage == llb.LLB_F32 else torch.float64
    nbytes = llb.llb_state_bytes(n, n, n, q, llb.llb_params_default(storage=storage, **kw))

    def run(steps, restore=None):
        bufs = [torch.zeros(nbytes // (4 if storage == llb.LLB_F32 else 8), dtype=dt, device="cuda")
                for _ in range(2)]
        ctx = llb.llb_create(n, n, n, q, tau, llb.llb_params_default(storage=storage, buffers=bufs, **kw))
        try:
            llb.llb_init_moments(ctx, m0)
            cur = next(b for b in bufs if b.data_ptr() == llb.llb_state_device(ctx)[0])
            if restore is not None:
                torch.cuda.synchronize()
                cur.copy_(restore)
                torch.cuda.synchronize()
            llb.llb_step(ctx, steps)
            llb.llb_synchronize(ctx)
            saved = next(b for b in bufs if b.data_ptr() == llb.llb_state_device(ctx)[0]).clone()
            out = llb.llb_get_moments(ctx, np.empty(m0.shape))
        finally:
            llb.llb_destroy(ctx)
        return saved, out

    _, full = run(30)
    half, _ = run(15)
    _, rest = run(15, restore=half)
    assert np.array_equal(rest, full)


def test_device_buffers_and_stream_from_torch():
    """Caller-owned device buffers and a caller stream (torch), device-side init/get."""
    torch = pytest.importorskip("torch")
    n, q, tau = 20, 19, 0.8
    m0 = inputs.random_moments(n, n, n, seed=12)
    nbytes = llb.llb_state_bytes(n, n, n, q, llb.llb_params_default(storage=llb.LLB_F64))
    bufs = [torch.empty(nbytes // 8, dtype=torch.float64, device="cuda") for _ in range(2)]
    s = torch.cuda.Stream()
    p = llb.llb_params_default(storage=llb.LLB_F64, buffers=bufs, stream=s.cuda_stream)
    ctx = llb.llb_create(n, n, n, q, tau, p)
    try:
        dev_in = torch.from_numpy(m0).cuda()
        torch.cuda.synchronize()
        llb.llb_init_moments_device(ctx, dev_in)
        llb.llb_step(ctx, 4)
        dev_out = torch.empty_like(dev_in)
        llb.llb_get_moments_device(ctx, dev_out)
        llb.llb_synchronize(ctx)
        got = dev_out.cpu().numpy()
    finally:
        llb.llb_destroy(ctx)
    assert_groups(got, lb.run_moment_only(m0, D3Q19, tau, 4), 1e-12, what="device buffers")


@pytest.mark.parametrize("nsteps", [1, 4, 5])
def test_step_graph_matches_step(nsteps):
    """Steps replayed from a captured CUDA graph give bit-identical results,
    also across repeated replays and both flip-flop parities."""
    n = 48
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=3)
    out = []
    for use_graph in (False, True):
        ctx = llb.llb_create(n, n, n, 19, 0.7, llb.llb_params_default())
        try:
            llb.llb_init_equilibrium(ctx, rho, u)
            for _ in range(3):
                (llb.llb_step_graph if use_graph else llb.llb_step)(ctx, nsteps)
            assert llb.llb_steps_done(ctx) == 3 * nsteps
            out.append(llb.llb_get_moments(ctx, np.empty((10, n, n, n))))
        finally:
            llb.llb_destroy(ctx)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("q", [19, 27])
def test_autotune_keeps_state(q):
    """The autotuner times kernels without advancing the state, then the chosen
    kernel still matches the oracle."""
    n = 72
    rho, u = inputs.taylor_green_3d(n, n, n, u0=0.05, noise=1e-3, seed=9)
    ctx = llb.llb_create(n, n, n, q, 0.7, llb.llb_params_default())
    try:
        llb.llb_init_equilibrium(ctx, rho, u)
        before = llb.llb_get_moments(ctx, np.empty((10, n, n, n)))
        kernel, variant = llb.llb_autotune(ctx, 3)
        after = llb.llb_get_moments(ctx, np.empty((10, n, n, n)))
        assert np.array_equal(before, after) and llb.llb_steps_done(ctx) == 0
        assert kernel in (llb.LLB_KERNEL_TILED, llb.LLB_KERNEL_TMA, llb.LLB_KERNEL_DIRECT)
        llb.llb_step(ctx, 5)
        got = llb.llb_get_moments(ctx, np.empty((10, n, n, n)))
    finally:
        llb.llb_destroy(ctx)
    ref = lb.run_moment_only(lb.equilibrium_moments(rho, u), LAT[q], 0.7, 5)
    assert_groups(got, ref, 1e-5, what=f"autotuned kernel {kernel} variant {variant}")


@pytest.mark.parametrize("nsteps", [1, 3])
@pytest.mark.parametrize("storage", [llb.LLB_F32, llb.LLB_F64, llb.LLB_F16S, llb.LLB_BF16S],
                         ids=["f32", "f64", "f16", "bf16"])
@pytest.mark.parametrize("shape", [(64, 48, 40), (67, 45, 37), (33, 9, 5), (40, 24, 264)],
                         ids=lambda s: "x".join(map(str, s)))
def test_step_host_matches_sequential(shape, storage, nsteps):
    """llb_step_host (copies overlapped with per-slab steps) gives bit for bit
    what llb_init_moments + llb_step + llb_get_moments give."""
    nx, ny, nz = shape
    m0 = inputs.random_moments(nx, ny, nz, seed=nx + ny + nz)
    hdt = np.float64 if storage == llb.LLB_F64 else np.float32
    h_in = np.ascontiguousarray(m0.astype(hdt))
    out = []
    for piped in (False, True):
        ctx = llb.llb_create(nx, ny, nz, 19, 0.7, llb.llb_params_default(storage=storage))
        try:
            res = np.empty_like(h_in)
            if piped:
                llb.llb_step_host(ctx, h_in, res, nsteps)
            else:
                llb.llb_init_moments(ctx, h_in)
                llb.llb_step(ctx, nsteps)
                llb.llb_get_moments(ctx, res)
            assert llb.llb_steps_done(ctx) == nsteps
            # the context holds the stepped state afterwards
            again = llb.llb_get_moments(ctx, np.empty_like(h_in))
        finally:
            llb.llb_destroy(ctx)
        assert np.array_equal(again, res)
        out.append(res)
    assert np.array_equal(out[0], out[1])


def test_step_host_rejects_unphysical_input_and_other_kernels_fall_back():
    """rho <= 0 in the input is reported as LLB_EUNSTABLE; a context on the
    direct kernel takes the non-overlapped path and gives the same result."""
    n = 16
    m0 = inputs.random_moments(n, n, n, seed=5)
    bad = m0.copy()
    bad[0, 2, 3, 4] = -1.0
    ctx = llb.llb_create(n, n, n, 19, 0.8, llb.llb_params_default(storage=llb.LLB_F64))
    try:
        with pytest.raises(llb.LLBError) as e:
            llb.llb_step_host(ctx, bad, np.empty_like(bad), 1)
        assert e.value.status == llb.LLB_EUNSTABLE
        good = llb.llb_step_host(ctx, m0, np.empty_like(m0), 2)
    finally:
        llb.llb_destroy(ctx)
    ctx = llb.llb_create(n, n, n, 19, 0.8, llb.llb_params_default(storage=llb.LLB_F64, kernel=llb.LLB_KERNEL_DIRECT))
    try:
        direct = llb.llb_step_host(ctx, m0, np.empty_like(m0), 2)
    finally:
        llb.llb_destroy(ctx)
    assert_groups(direct, good, 1e-14, what="direct vs tiled host step")
