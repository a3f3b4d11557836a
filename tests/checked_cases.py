"""Cases of the bounds-checked build, run in a process of their own with
LLB_CHECKED=1 (libllb_checked.so loaded instead of libllb.so).

Every case runs a few steps of one kernel on a small, mostly ragged box (tiles
that stick out of the box in x and y, boxes smaller than one tile, a z extent
shorter than a work chunk), then asks the library for the first out-of-range
index its kernels recorded, and compares the moments with the FP64 oracle (the
adjoint cases: the tiled first pass with its reference form).
Prints one JSON object per case:
  {"case": name, "site": s, "index": i, "err": e, "tol": t, "skip": why|null}
Called by tests/test_gpu_checked.py; not a test module itself.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)

from oracle import D3Q19, D3Q27, lb  # noqa: E402
from oracle import two_component as tc  # noqa: E402
from paper_2301_01622_gb300 import inputs, llb  # noqa: E402

from gpu_helpers import group_errors  # noqa: E402

LAT = {19: D3Q19, 27: D3Q27}
TOL = {llb.LLB_F64: 1e-12, llb.LLB_F32: 1e-5, llb.LLB_F16S: 3e-2, llb.LLB_BF16S: 0.25}
SNAME = {llb.LLB_F64: "f64", llb.LLB_F32: "f32", llb.LLB_F16S: "f16", llb.LLB_BF16S: "bf16"}
KNAME = {llb.LLB_KERNEL_DIRECT: "direct", llb.LLB_KERNEL_TILED: "tiled", llb.LLB_KERNEL_TMA: "tma"}

# one component: below one tile, one-node extents, ragged multi-tile boxes
SHAPES_1 = [(1, 1, 1), (2, 3, 1), (4, 4, 4), (9, 6, 5), (70, 10, 9), (130, 9, 7)]
# two components (n >= 4 each way)
SHAPES_2 = [(4, 4, 4), (9, 6, 5), (37, 11, 7), (70, 10, 9)]
STEPS = 4
TAU_1, TAU_2 = 0.8, 0.9
CG = tc.CGParams(beta=0.7, A_s=0.02, A_h=0.01, h_c=3, g_min=1e-8)

_oracle = {}


def _emit(case, site=0, index=0, err=0.0, tol=0.0, skip=None):
    print(json.dumps({"case": case, "site": site, "index": index, "err": err, "tol": tol, "skip": skip}),
          flush=True)


def _status(case):
    en, site, idx = llb.llb_checked_status()
    if en != 1:
        raise RuntimeError("the library loaded is not the bounds-checked build")
    return site, idx


def _one_comp_ref(q, shape, scheme="moment"):
    key = ("1", q, shape, scheme)
    if key not in _oracle:
        m0 = inputs.random_moments(*shape, seed=7)
        if scheme == "moment":
            ref = lb.run_moment_only(m0, LAT[q], TAU_1, STEPS)
        else:
            f = lb.run_population(lb.populations_from_moments(m0, LAT[q]), LAT[q], TAU_1, STEPS, scheme)
            ref = lb.project(f, LAT[q])
        _oracle[key] = (m0, ref)
    return _oracle[key]


def _drops(shape):
    nx, ny, nz = shape
    r = max(1.5, min(nx, ny, nz) / 4)
    c1 = (nx / 2 - r - 1.0, ny / 2 - 0.5, nz / 2)
    c2 = (nx / 2 + r + 1.0, ny / 2 + 0.5, nz / 2)
    r1, r2, u = inputs.droplets(nx, ny, nz, [c1, c2], [r, r], [(0.03, 0, 0), (-0.03, 0, 0)])
    tot = lb.equilibrium_moments(r1 + r2, u)
    return np.concatenate([r1[None], r2[None], tot[1:]])


def _two_comp_ref(q, shape, scheme="moment"):
    key = ("2", q, shape, scheme)
    if key not in _oracle:
        m0 = _drops(shape)
        if scheme == "moment":
            ref = tc.run_moment_only(m0, LAT[q], TAU_2, CG, STEPS)
        else:
            f = tc.run_population(tc.populations_from_moments(m0, LAT[q]), LAT[q], TAU_2, CG, STEPS, scheme)
            ref = tc.project(f, LAT[q])
        _oracle[key] = (m0, ref)
    return _oracle[key]


def _run(shape, q, tau, m0, params, *, host_step=False):
    nx, ny, nz = shape
    ctx = llb.llb_create(nx, ny, nz, q, tau, params)
    try:
        out = np.empty(m0.shape, dtype=np.float64)
        if host_step:
            llb.llb_step_host(ctx, np.ascontiguousarray(m0), out, STEPS)
        else:
            llb.llb_init_moments(ctx, np.ascontiguousarray(m0))
            llb.llb_step(ctx, STEPS)
            llb.llb_get_moments(ctx, out)
    finally:
        llb.llb_destroy(ctx)
    return out


def _case(name, fn, tol):
    try:
        got, ref = fn()
    except llb.LLBError as e:
        if e.status == llb.LLB_EINVAL:
            site, idx = _status(name)
            _emit(name, site, idx, skip=f"not offered for this shape: {e}")
            return
        raise
    site, idx = _status(name)
    err = max(group_errors(got, ref).values())
    _emit(name, site, idx, float(err), tol)


def one_component():
    for q in (19, 27):
        for shape in SHAPES_1:
            sh = "x".join(map(str, shape))
            m0, ref = _one_comp_ref(q, shape)
            runs = [(llb.LLB_KERNEL_TILED, s, v) for s in (llb.LLB_F64, llb.LLB_F16S, llb.LLB_BF16S) for v in (0,)]
            runs += [(llb.LLB_KERNEL_TILED, llb.LLB_F32, v) for v in range(6)]
            runs += [(llb.LLB_KERNEL_DIRECT, s, 0) for s in (llb.LLB_F64, llb.LLB_F32)]
            runs += [(llb.LLB_KERNEL_TMA, llb.LLB_F32, v) for v in range(3)] + [(llb.LLB_KERNEL_TMA, llb.LLB_F64, 0)]
            for kernel, storage, v in runs:
                name = f"d3q{q}-{sh}-{KNAME[kernel]}-{SNAME[storage]}-v{v}"
                p = llb.llb_params_default(storage=storage, kernel=kernel, variant=v)
                _case(name, lambda p=p: (_run(shape, q, TAU_1, m0, p), ref), TOL[storage])
            # the host-to-host step launches the tiled kernel on z-slabs
            for storage in (llb.LLB_F32, llb.LLB_F64):
                p = llb.llb_params_default(storage=storage, kernel=llb.LLB_KERNEL_TILED)
                _case(f"d3q{q}-{sh}-step_host-{SNAME[storage]}",
                      lambda p=p: (_run(shape, q, TAU_1, m0, p, host_step=True), ref), TOL[storage])


def populations():
    for q in (19, 27):
        for shape in [(1, 2, 3), (9, 6, 5), (37, 11, 7)]:
            sh = "x".join(map(str, shape))
            for scheme, code in (("regularized", llb.LLB_SCHEME_POPULATION), ("bgk", llb.LLB_SCHEME_POPULATION_BGK)):
                m0, ref = _one_comp_ref(q, shape, scheme)
                for storage in (llb.LLB_F64, llb.LLB_F32):
                    p = llb.llb_params_default(storage=storage, scheme=code)
                    _case(f"d3q{q}-{sh}-pop-{scheme}-{SNAME[storage]}",
                          lambda p=p: (_run(shape, q, TAU_1, m0, p), ref), TOL[storage])
        for shape in [(4, 4, 4), (9, 6, 5), (37, 11, 7)]:
            sh = "x".join(map(str, shape))
            for scheme, code in (("regularized", llb.LLB_SCHEME_POPULATION), ("bgk", llb.LLB_SCHEME_POPULATION_BGK)):
                m0, ref = _two_comp_ref(q, shape, scheme)
                p = llb.llb_params_default(storage=llb.LLB_F64, scheme=code, ncomp=2, beta=CG.beta, A_s=CG.A_s,
                                           A_h=CG.A_h, g_min=CG.g_min, h_c=CG.h_c)
                _case(f"d3q{q}-{sh}-pop2-{scheme}-f64",
                      lambda p=p: (_run(shape, q, TAU_2, m0, p), ref), TOL[llb.LLB_F64])


def two_component():
    for q in (19, 27):
        for shape in SHAPES_2:
            sh = "x".join(map(str, shape))
            m0, ref = _two_comp_ref(q, shape)
            for storage, variants in ((llb.LLB_F64, (0,)), (llb.LLB_F32, range(6))):
                for v in variants:
                    p = llb.llb_params_default(storage=storage, variant=v, ncomp=2, beta=CG.beta, A_s=CG.A_s,
                                               A_h=CG.A_h, g_min=CG.g_min if storage == llb.LLB_F64 else 1e-6,
                                               h_c=CG.h_c)
                    # FP32: the colour split of a two-node-wide interface on a
                    # small box, few steps: 1e-4 of each group
                    tol = TOL[storage] if storage == llb.LLB_F64 else 1e-4
                    _case(f"d3q{q}-{sh}-cg-{SNAME[storage]}-v{v}",
                          lambda p=p: (_run(shape, q, TAU_2, m0, p), ref), tol)
                    if v == 0:  # the host-to-host step launches the kernel on z-slabs
                        _case(f"d3q{q}-{sh}-cg-step_host-{SNAME[storage]}",
                              lambda p=p: (_run(shape, q, TAU_2, m0, p, host_step=True), ref), tol)


def batches():
    dims = SHAPES_2
    for q in (19, 27):
        for storage in (llb.LLB_F64, llb.LLB_F32):
            for v in ((0,) if storage == llb.LLB_F64 else range(6)):
                p = llb.llb_params_default(storage=storage, variant=v, ncomp=2, beta=CG.beta, A_s=CG.A_s,
                                           A_h=CG.A_h, g_min=CG.g_min if storage == llb.LLB_F64 else 1e-6,
                                           h_c=CG.h_c)
                name = f"d3q{q}-batch-cg-{SNAME[storage]}-v{v}"

                def fn(p=p):
                    b = llb.llb_batch_create(dims, q, TAU_2, p)
                    try:
                        for k, d in enumerate(dims):
                            llb.llb_init_moments(llb.llb_batch_domain(b, k), _two_comp_ref(q, d)[0])
                        llb.llb_batch_step(b, STEPS)
                        got = [llb.llb_get_moments(llb.llb_batch_domain(b, k), np.empty((11,) + d[::-1]))
                               for k, d in enumerate(dims)]
                    finally:
                        llb.llb_batch_destroy(b)
                    return (np.concatenate([g.reshape(11, -1) for g in got], axis=1),
                            np.concatenate([_two_comp_ref(q, d)[1].reshape(11, -1) for d in dims], axis=1))

                _case(name, fn, TOL[storage] if storage == llb.LLB_F64 else 1e-4)


def adjoints():
    """Two-component adjoint (tiled first pass) against its reference form."""
    import torch
    for q in (19, 27):
        for shape in [(4, 4, 4), (9, 6, 5), (37, 11, 7)]:
            sh = "x".join(map(str, shape))
            m0 = _drops(shape)
            g = np.random.default_rng(3).uniform(-1, 1, m0.shape)
            for storage in (llb.LLB_F64, llb.LLB_F32):
                def fn(storage=storage):
                    res = []
                    for flags in (0, 2):
                        p = llb.llb_params_default(storage=storage, ncomp=2, beta=CG.beta, A_s=CG.A_s, A_h=0.0,
                                                   grad_eps=0.02, debug_flags=flags)
                        ctx = llb.llb_create(*shape, q, TAU_2, p)
                        try:
                            llb.llb_init_moments(ctx, m0)
                            gfin = torch.from_numpy(g).cuda()
                            gini = torch.empty_like(gfin)
                            llb.llb_adjoint(ctx, STEPS, gfin, gini, every=2)
                            res.append(gini.cpu().numpy())
                        finally:
                            llb.llb_destroy(ctx)
                    return res[0], res[1]
                _case(f"d3q{q}-{sh}-adjoint-{SNAME[storage]}", fn, TOL[storage])


GROUPS = {"one": one_component, "two": two_component, "pop": populations, "batch": batches, "adjoint": adjoints}

if __name__ == "__main__":
    for g in (sys.argv[1:] or list(GROUPS)):
        GROUPS[g]()
