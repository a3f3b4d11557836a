"""A box of more than 2^31 nodes (1296^3 = 2.18e9, FP16 storage: 87 GB of
state plus an 87 GB FP32 canonical buffer): every index and byte offset of the
conversions and the step runs past 32 bits.  One step, checked at sampled nodes
(corners, the periodic faces, nodes whose linear index exceeds 2^31) against the
oracle's per-node step from the stored (16-bit rounded) inputs."""
import numpy as np
import pytest

from oracle import D3Q19, lb
from paper_2301_01622_gb300 import inputs, llb

from gpu_helpers import NAMES_1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SIDE, TAU = 1296, 0.8


def _neigh(m, x, y, z, n):
    """(10, 3, 3, 3) periodic neighbourhood of (x, y, z) as float64 on the host."""
    idx = [torch.tensor([(v - 1) % n, v, (v + 1) % n], device=m.device) for v in (x, y, z)]
    nb = m[:, idx[2][:, None, None], idx[1][None, :, None], idx[0][None, None, :]]
    return nb.double().cpu().numpy()


def test_more_than_2_31_nodes_one_step_fp16():
    n = N_SIDE
    assert n ** 3 > 2 ** 31
    p = llb.llb_params_default(storage=llb.LLB_F16S)
    need = 10 * n ** 3 * 4 + 2 * llb.llb_state_bytes(n, n, n, 19, p)
    free, _ = torch.cuda.mem_get_info()
    if free < need * 1.05:
        pytest.skip(f"needs {need / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free")
    rng = np.random.default_rng(17)
    sites = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, n // 2), (n - 1, 0, n - 1), (5, 7, 1290),
             (1295, 1000, 1285), (640, 641, 1279)]
    sites += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(12)]
    assert sum((z * n + y) * n + x > 2 ** 31 for x, y, z in sites) >= 4
    m = inputs.random_moments_device(n, n, n, seed=31)
    ctx = llb.llb_create(n, n, n, 19, TAU, p)
    try:
        llb.llb_init_moments_device(ctx, m)
        llb.llb_get_moments_device(ctx, m)       # the stored inputs, 16-bit rounded
        torch.cuda.synchronize()
        before = {s: _neigh(m, *s, n) for s in sites}
        scale = np.array([float(m[f].abs().max()) for f in range(10)])
        llb.llb_step(ctx, 1)
        llb.llb_get_moments_device(ctx, m)
        torch.cuda.synchronize()
        after = {s: m[:, s[2], s[1], s[0]].double().cpu().numpy() for s in sites}
    finally:
        llb.llb_destroy(ctx)
        del m
        torch.cuda.empty_cache()
    # per field, relative to the field's largest value: the 16-bit rounding of the
    # step's output (the inputs are the stored values themselves)
    for s in sites:
        ref = lb.node_moment_only(before[s], D3Q19, TAU, 1, 1, 1)
        err = np.abs(after[s] - ref) / scale
        assert err.max() <= 2e-3, (s, dict(zip(NAMES_1, err)))
