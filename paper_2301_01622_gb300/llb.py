"""Thin ctypes binding of libllb (the C ABI declared in include/llb.h).

Argument marshalling only: each function has the C name, checks the status
code and raises ``LLBError`` on failure.  Every step of the lattice
Boltzmann update runs inside the library's CUDA kernels; there is no Python
or CPU fallback, and loading fails loudly when libllb.so has not been built.

Buffers may be numpy arrays (host), torch tensors (host or device) or raw
integer addresses.  Canonical moments are arrays of shape (nf, nz, ny, nx),
field-major, x fastest, with nf = 10 (one component) or 11 (two).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LLB_CHECKED=1 loads the bounds-checked build (libllb_checked.so) instead
LIB_PATH = os.path.join(HERE, "libllb_checked.so" if os.environ.get("LLB_CHECKED") == "1" else "libllb.so")

LLB_OK, LLB_EINVAL, LLB_ENOMEM, LLB_ECUDA, LLB_EUNSTABLE, LLB_ETIMEOUT, LLB_ESTATE = 0, -1, -2, -3, -4, -5, -6
LLB_F64, LLB_F32, LLB_F16S, LLB_BF16S = 0, 1, 2, 3
LLB_SCHEME_MOMENT, LLB_SCHEME_POPULATION, LLB_SCHEME_POPULATION_BGK = 0, 1, 2
LLB_KERNEL_AUTO, LLB_KERNEL_DIRECT, LLB_KERNEL_TILED, LLB_KERNEL_TMA = 0, 1, 2, 3
LLB_FLAG_NONFINITE, LLB_FLAG_NONPOSITIVE = 1, 2


class llb_params(C.Structure):
    _fields_ = [
        ("ncomp", C.c_int), ("storage", C.c_int), ("scheme", C.c_int), ("kernel", C.c_int), ("variant", C.c_int),
        ("beta", C.c_double), ("A_s", C.c_double), ("A_h", C.c_double), ("g_min", C.c_double),
        ("h_c", C.c_int), ("stream", C.c_void_p), ("buffers", C.c_void_p * 2), ("wait_budget_ms", C.c_int),
        ("debug_flags", C.c_int), ("grad_eps", C.c_double),
    ]


class llb_diag(C.Structure):
    _fields_ = [
        ("mass", C.c_double * 2), ("momentum", C.c_double * 3), ("rho1_sum", C.c_double),
        ("n_in", C.c_longlong), ("rho1_avg", C.c_double), ("min_rho", C.c_double),
        ("flags", C.c_int), ("reserved", C.c_int),
    ]

    def as_dict(self) -> dict:
        return {"mass": list(self.mass), "momentum": list(self.momentum), "rho1_sum": self.rho1_sum,
                "n_in": int(self.n_in), "rho1_avg": self.rho1_avg, "min_rho": self.min_rho, "flags": int(self.flags)}


class llb_footprint(C.Structure):
    _fields_ = [("arrays", C.c_int), ("fields", C.c_int), ("bytes_per_node", C.c_size_t),
                ("state_bytes", C.c_size_t), ("stream_bytes_per_node", C.c_size_t)]


class LLBError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status}) {detail}".strip())


_lib = None

_SIGS = {
    "llb_params_default": (None, [C.POINTER(llb_params)]),
    "llb_footprint_query": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(llb_params), C.POINTER(llb_footprint)]),
    "llb_state_bytes": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(llb_params), C.POINTER(C.c_size_t)]),
    "llb_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(llb_params)]),
    "llb_destroy": (None, [C.c_void_p]),
    "llb_init_moments": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "llb_init_moments_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "llb_init_equilibrium": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "llb_step": (C.c_int, [C.c_void_p, C.c_int]),
    "llb_step_graph": (C.c_int, [C.c_void_p, C.c_int]),
    "llb_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "llb_get_moments": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "llb_step_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "llb_get_moments_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "llb_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(llb_diag)]),
    "llb_synchronize": (C.c_int, [C.c_void_p]),
    "llb_diagnostics_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                          C.POINTER(llb_diag)]),
    "llb_steps_done": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "llb_state_device": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "llb_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int), C.c_int, C.c_double,
                                   C.POINTER(llb_params)]),
    "llb_batch_destroy": (None, [C.c_void_p]),
    "llb_batch_domain": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "llb_batch_nodes": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "llb_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "llb_batch_step_graph": (C.c_int, [C.c_void_p, C.c_int]),
    "llb_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "llb_adjoint": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                              C.POINTER(C.c_double)]),
    "llb_checked_status": (C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "llb_status_string": (C.c_char_p, [C.c_int]),
    "llb_last_error": (C.c_char_p, [C.c_void_p]),
}


def lib():
    """Load libllb.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{os.path.basename(LIB_PATH)} not found at {LIB_PATH}; build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def status_string(status: int) -> str:
    return lib().llb_status_string(int(status)).decode()


def _ptr(buf):
    """Address of a numpy array, torch tensor, or int."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return buf.ctypes.data
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr()
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _dtype_code(buf) -> int:
    if isinstance(buf, np.ndarray):
        dt = buf.dtype
        if dt == np.float64:
            return LLB_F64
        if dt == np.float32:
            return LLB_F32
    elif hasattr(buf, "dtype"):
        s = str(buf.dtype)
        if s.endswith("float64"):
            return LLB_F64
        if s.endswith("float32"):
            return LLB_F32
    raise TypeError("buffers must be float64 or float32")


def _check(rc: int, where: str, ctx=None):
    if rc != LLB_OK:
        detail = ""
        if ctx is not None:
            msg = lib().llb_last_error(ctx)
            detail = msg.decode() if msg else ""
        raise LLBError(rc, where, detail)


def llb_params_default(**overrides) -> llb_params:
    p = llb_params()
    lib().llb_params_default(C.byref(p))
    for k, v in overrides.items():
        if k == "buffers":
            p.buffers[0] = _ptr(v[0]) if v[0] is not None else None
            p.buffers[1] = _ptr(v[1]) if v[1] is not None else None
        elif k == "stream":
            p.stream = v
        else:
            setattr(p, k, v)
    return p


def llb_footprint_query(nx, ny, nz, lattice, params: llb_params | None = None) -> llb_footprint:
    out = llb_footprint()
    _check(lib().llb_footprint_query(nx, ny, nz, lattice, C.byref(params) if params else None, C.byref(out)),
           "llb_footprint_query")
    return out


def llb_state_bytes(nx, ny, nz, lattice, params: llb_params | None = None) -> int:
    out = C.c_size_t()
    _check(lib().llb_state_bytes(nx, ny, nz, lattice, C.byref(params) if params else None, C.byref(out)),
           "llb_state_bytes")
    return int(out.value)


def llb_create(nx, ny, nz, lattice, tau, params: llb_params | None = None):
    ctx = C.c_void_p()
    _check(lib().llb_create(C.byref(ctx), nx, ny, nz, lattice, float(tau), C.byref(params) if params else None),
           "llb_create")
    return ctx


def llb_destroy(ctx):
    if ctx:
        lib().llb_destroy(ctx)


def llb_init_moments(ctx, host_m):
    _check(lib().llb_init_moments(ctx, _ptr(host_m), _dtype_code(host_m)), "llb_init_moments", ctx)


def llb_init_moments_device(ctx, dev_m):
    _check(lib().llb_init_moments_device(ctx, _ptr(dev_m), _dtype_code(dev_m)), "llb_init_moments_device", ctx)


def llb_init_equilibrium(ctx, host_rho, host_u):
    dt = _dtype_code(host_rho)
    if _dtype_code(host_u) != dt:
        raise TypeError("rho and u must have the same dtype")
    _check(lib().llb_init_equilibrium(ctx, _ptr(host_rho), _ptr(host_u), dt), "llb_init_equilibrium", ctx)


def llb_step(ctx, nsteps: int = 1):
    _check(lib().llb_step(ctx, int(nsteps)), "llb_step", ctx)


def llb_step_graph(ctx, nsteps: int = 1):
    _check(lib().llb_step_graph(ctx, int(nsteps)), "llb_step_graph", ctx)


def llb_autotune(ctx, trials: int = 5):
    k, v = C.c_int(), C.c_int()
    _check(lib().llb_autotune(ctx, int(trials), C.byref(k), C.byref(v)), "llb_autotune", ctx)
    return k.value, v.value


def llb_adjoint(ctx, nsteps, gfinal_dev, ginit_dev, every: int = 0) -> float:
    """Gradient of a loss w.r.t. the initial canonical moments (written into
    ginit_dev) and tau (returned), given dL/d(final moments) in gfinal_dev."""
    dt = _dtype_code(gfinal_dev)
    if _dtype_code(ginit_dev) != dt:
        raise TypeError("gfinal and ginit must have the same dtype")
    dtau = C.c_double()
    _check(lib().llb_adjoint(ctx, int(nsteps), int(every), _ptr(gfinal_dev), _ptr(ginit_dev), dt, C.byref(dtau)),
           "llb_adjoint", ctx)
    return float(dtau.value)


def llb_get_moments(ctx, host_out):
    _check(lib().llb_get_moments(ctx, _ptr(host_out), _dtype_code(host_out)), "llb_get_moments", ctx)
    return host_out


def llb_step_host(ctx, host_in, host_out, nsteps=1):
    """Host moments in, nsteps steps, host moments out, with the copies
    overlapped with the device work (see include/llb.h)."""
    dt = _dtype_code(host_in)
    if _dtype_code(host_out) != dt:
        raise TypeError("host_in and host_out must have the same dtype")
    _check(lib().llb_step_host(ctx, _ptr(host_in), _ptr(host_out), dt, int(nsteps)), "llb_step_host", ctx)
    return host_out


def llb_get_moments_device(ctx, dev_out):
    _check(lib().llb_get_moments_device(ctx, _ptr(dev_out), _dtype_code(dev_out)), "llb_get_moments_device", ctx)
    return dev_out


def llb_diagnostics(ctx) -> dict:
    d = llb_diag()
    _check(lib().llb_diagnostics(ctx, C.byref(d)), "llb_diagnostics", ctx)
    return d.as_dict()


def llb_diagnostics_noalloc(dev_m, nx, ny, nz, stream=None) -> dict:
    """Diagnostics of canonical moments already on the device, without any
    device allocation (fixed scratch inside the library; see include/llb.h)."""
    d = llb_diag()
    _check(lib().llb_diagnostics_noalloc(_ptr(dev_m), _dtype_code(dev_m), nx, ny, nz, stream, C.byref(d)),
           "llb_diagnostics_noalloc")
    return d.as_dict()


def llb_synchronize(ctx):
    _check(lib().llb_synchronize(ctx), "llb_synchronize", ctx)


def llb_checked_status():
    """(enabled, site, index): the first out-of-range access recorded by the
    bounds-checked build since the last call (site 0: none).  Synchronises."""
    en, site, idx = C.c_int(0), C.c_int(0), C.c_longlong(0)
    _check(lib().llb_checked_status(C.byref(en), C.byref(site), C.byref(idx)), "llb_checked_status")
    return en.value, site.value, idx.value


def llb_steps_done(ctx) -> int:
    v = C.c_longlong()
    _check(lib().llb_steps_done(ctx, C.byref(v)), "llb_steps_done")
    return int(v.value)


def llb_state_device(ctx):
    p, dt, k = C.c_void_p(), C.c_int(), C.c_int()
    _check(lib().llb_state_device(ctx, C.byref(p), C.byref(dt), C.byref(k)), "llb_state_device")
    return p.value, dt.value, k.value


def llb_last_error(ctx) -> str:
    return lib().llb_last_error(ctx).decode()


def llb_batch_create(dims, lattice, tau, params: llb_params):
    """dims: sequence of (nx, ny, nz); returns the batch handle."""
    flat = (C.c_int * (3 * len(dims)))(*[int(v) for d in dims for v in d])
    b = C.c_void_p()
    _check(lib().llb_batch_create(C.byref(b), len(dims), flat, lattice, float(tau), C.byref(params)),
           "llb_batch_create")
    return b


def llb_batch_destroy(b):
    if b:
        lib().llb_batch_destroy(b)


def llb_batch_domain(b, d):
    ctx = C.c_void_p()
    _check(lib().llb_batch_domain(b, int(d), C.byref(ctx)), "llb_batch_domain")
    return ctx


def llb_batch_nodes(b) -> int:
    v = C.c_longlong()
    _check(lib().llb_batch_nodes(b, C.byref(v)), "llb_batch_nodes")
    return int(v.value)


def llb_batch_step(b, nsteps: int = 1):
    _check(lib().llb_batch_step(b, int(nsteps)), "llb_batch_step")


def llb_batch_step_graph(b, nsteps: int = 1):
    _check(lib().llb_batch_step_graph(b, int(nsteps)), "llb_batch_step_graph")


def llb_batch_autotune(b, trials: int = 3) -> int:
    v = C.c_int()
    _check(lib().llb_batch_autotune(b, int(trials), C.byref(v)), "llb_batch_autotune")
    return v.value
