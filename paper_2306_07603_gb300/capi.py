"""Thin ctypes binding of the C ABI in include/ifdlbm.h (argument marshalling only).

Every function below has the name and meaning of the C entry point it
wraps; all computation happens in libifdlbm.so (sm_103a CUDA). PyTorch is
used only to hand the library a CUDA stream and a device allocator (its
caching allocator). There is no CPU fallback: if the library is missing,
loading fails with an error naming the build step.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libifdlbm.so")

IFDLBM_OK = 0
IFDLBM_ERR_INVALID_ARG = -1
IFDLBM_ERR_CUDA = -2
IFDLBM_ERR_OOM = -3
IFDLBM_ERR_DIVERGED = -4
IFDLBM_ERR_TIMEOUT = -5
IFDLBM_FP64 = 0
IFDLBM_FP32DEV = 1
IFDLBM_KERNEL_AUTO = 0
IFDLBM_KERNEL_STAGED = 1
IFDLBM_KERNEL_FUSED = 2
IFDLBM_KPROF_COLLIDE = 0
IFDLBM_KPROF_HALF = 1
IFDLBM_KPROF_FULL = 2
IFDLBM_KPROF_REDUCE = 3
IFDLBM_KPROF_FUSED = 4
IFDLBM_KPROF_COUNT = 5
IFDLBM_STATIC_MAX_NODES = 2097152
IFDLBM_LAMBDA_LAGGED = 0
IFDLBM_LAMBDA_IMPLICIT = 1
IFDLBM_WALLP_ZEROTH = 0
IFDLBM_WALLP_FIRST = 1
IFDLBM_DT_GRID = 0
IFDLBM_DT_CONTRAVARIANT = 1
IFDLBM_SCHED_GRID = 0
IFDLBM_SCHED_STATIC = 1
IFDLBM_SCHED_DYNAMIC = 2


class ifdlbm_geometry(C.Structure):
    _fields_ = [("L", C.c_double), ("H", C.c_double), ("theta_deg", C.c_double)]


class ifdlbm_options(C.Structure):
    _fields_ = [("cfl", C.c_double), ("c", C.c_double), ("eta_b", C.c_double),
                ("gamma_min", C.c_double), ("dt", C.c_double), ("rho0", C.c_double),
                ("precision", C.c_int), ("kernel", C.c_int), ("graph_chunk", C.c_int),
                ("fused_threads", C.c_int), ("fused_rows", C.c_int), ("schedule", C.c_int),
                ("dt_mode", C.c_int), ("lambda_mode", C.c_int), ("power_fp32", C.c_int),
                ("wall_pressure", C.c_int)]


class ifdlbm_cavity(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("geom", ifdlbm_geometry),
                ("Re", C.c_double), ("n", C.c_double), ("U_lid", C.c_double)]


class ifdlbm_quad_cavity(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("corners", C.c_double * 8),
                ("H", C.c_double), ("Re", C.c_double), ("n", C.c_double),
                ("U_lid", C.c_double)]


class ifdlbm_info_t(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("precision", C.c_int), ("kernel", C.c_int),
                ("dt", C.c_double), ("K", C.c_double), ("gamma_min", C.c_double),
                ("eta_b", C.c_double), ("courant_max", C.c_double), ("steps", C.c_int64),
                ("device_bytes", C.c_int64), ("h2d_bytes", C.c_int64),
                ("fused_threads", C.c_int), ("fused_rows", C.c_int), ("schedule", C.c_int),
                ("ntasks", C.c_int)]


class ifdlbm_tuning(C.Structure):
    _fields_ = [("fused_threads", C.c_int), ("fused_rows", C.c_int), ("schedule", C.c_int),
                ("ntasks", C.c_int), ("ms_per_step", C.c_double), ("candidates", C.c_int),
                ("pad", C.c_int)]


class ifdlbm_eddy(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("xi", C.c_double), ("eta", C.c_double),
                ("psi", C.c_double), ("i", C.c_int), ("j", C.c_int), ("found", C.c_int),
                ("refined", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_H = C.c_void_p
_P = C.c_void_p
_SIGS = {
    "ifdlbm_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, C.c_void_p]),
    "ifdlbm_default_options": (C.c_int, [C.POINTER(ifdlbm_options)]),
    "ifdlbm_create": (C.c_int, [C.c_int, C.c_int, ifdlbm_geometry, C.c_double, C.c_double,
                                C.c_double, C.POINTER(ifdlbm_options), C.c_void_p,
                                C.POINTER(_H)]),
    "ifdlbm_create_batch": (C.c_int, [C.c_int, C.POINTER(ifdlbm_cavity),
                                      C.POINTER(ifdlbm_options), C.c_void_p, C.POINTER(_H)]),
    "ifdlbm_create_quad_batch": (C.c_int, [C.c_int, C.POINTER(ifdlbm_quad_cavity),
                                           C.POINTER(ifdlbm_options), C.c_void_p,
                                           C.POINTER(_H)]),
    "ifdlbm_step": (C.c_int, [_H, C.c_int]),
    "ifdlbm_macros": (C.c_int, [_H, _P, _P, _P, _P]),
    "ifdlbm_batch_macros": (C.c_int, [_H, C.c_int, _P, _P, _P, _P]),
    "ifdlbm_macros_dev": (C.c_int, [_H, C.c_int, _P, _P, _P, _P]),
    "ifdlbm_residual": (C.c_int, [_H, _P]),
    "ifdlbm_batch_residual_async": (C.c_int, [_H, _P, _P]),
    "ifdlbm_residual_dev": (C.c_int, [_H, _P]),
    "ifdlbm_probe_dev": (C.c_int, [_H, C.c_int, _P, _P]),
    "ifdlbm_batch_residual": (C.c_int, [_H, _P]),
    "ifdlbm_get_state": (C.c_int, [_H, C.c_int, _P, _P]),
    "ifdlbm_set_state": (C.c_int, [_H, C.c_int, _P, _P]),
    "ifdlbm_state_bytes": (C.c_int64, [_H]),
    "ifdlbm_save_state_dev": (C.c_int, [_H, _P]),
    "ifdlbm_load_state_dev": (C.c_int, [_H, _P]),
    "ifdlbm_info": (C.c_int, [_H, C.c_int, C.POINTER(ifdlbm_info_t)]),
    "ifdlbm_sync": (C.c_int, [_H]),
    "ifdlbm_destroy": (C.c_int, [_H]),
    "ifdlbm_last_error": (C.c_char_p, [_H]),
    "ifdlbm_launch_count": (C.c_int64, []),
    "ifdlbm_residual_fields_static": (C.c_int, [C.c_int, C.c_int, _P, _P, _P, _P, _P, _P, _P,
                                                C.c_void_p]),
    "ifdlbm_selftest_pow": (C.c_int, [_H, C.c_int, _P, C.c_double, _P, _P]),
    "ifdlbm_selftest_pow_f32": (C.c_int, [_H, C.c_int, _P, C.c_double, _P]),
    "ifdlbm_selftest_pow_tab": (C.c_int, [_H, C.c_int, C.c_int, _P, _P]),
    "ifdlbm_inject_tma_timeout": (C.c_int, [_H, C.c_int]),
    "ifdlbm_adjoint_seed_energy": (C.c_int, [_H, _P, _P, _P]),
    "ifdlbm_autotune": (C.c_int, [_H, C.c_int, C.c_void_p]),
    "ifdlbm_adjoint_step": (C.c_int, [_H, _P, _P, _P]),
    "ifdlbm_intermediate_bytes": (C.c_int64, [_H]),
    "ifdlbm_save_intermediates_dev": (C.c_int, [_H, _P]),
    "ifdlbm_adjoint_step_saved": (C.c_int, [_H, _P, _P, _P, _P, _P]),
    "ifdlbm_adjoint_seed_psi": (C.c_int, [_H, _P, C.c_void_p, _P, _P]),
    "ifdlbm_profile": (C.c_int, [_H, C.c_int]),
    "ifdlbm_find_eddies": (C.c_int, [C.c_int, C.c_int, ifdlbm_geometry, _P, C.c_void_p]),
    "ifdlbm_eddies": (C.c_int, [_H, C.c_int, C.c_void_p]),
    "ifdlbm_profile_read": (C.c_int, [_H, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libifdlbm.so and declare every entry point's signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -m paper_2306_07603_gb300.build); there is no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class IfdlbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ifdlbm error {code}: {msg}")
        self.code = code


def _check(rc, h=None):
    if rc != IFDLBM_OK:
        msg = load_library().ifdlbm_last_error(h)
        raise IfdlbmError(rc, (msg or b"").decode())
    return rc


def _ptr(a):
    """Pointer of a C-contiguous float64 numpy array or a CUDA tensor, or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data
    return a.data_ptr()  # torch tensor on the device


# ---------------------------------------------------------------------------
# Device allocator: torch's caching allocator on the handle's stream
# ---------------------------------------------------------------------------
_alloc_cbs = None


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _alloc_cbs
    import torch

    if _alloc_cbs is not None:
        return

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # out of memory: the library reports IFDLBM_ERR_OOM
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _alloc_cbs = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(load_library().ifdlbm_set_allocator(_alloc_cbs[0], _alloc_cbs[1], None))


# ---------------------------------------------------------------------------
# Entry points with the C names (marshalling only)
# ---------------------------------------------------------------------------
def ifdlbm_default_options() -> ifdlbm_options:
    opt = ifdlbm_options()
    _check(load_library().ifdlbm_default_options(C.byref(opt)))
    return opt


def ifdlbm_create(nx, ny, geometry, Re, n, U_lid, opt=None, stream=0):
    h = _H()
    g = ifdlbm_geometry(*geometry) if not isinstance(geometry, ifdlbm_geometry) else geometry
    _check(load_library().ifdlbm_create(int(nx), int(ny), g, float(Re), float(n), float(U_lid),
                                        C.byref(opt) if opt is not None else None,
                                        C.c_void_p(int(stream)), C.byref(h)))
    return h


def ifdlbm_create_batch(cavities, opt=None, stream=0):
    arr = (ifdlbm_cavity * len(cavities))(*cavities)
    h = _H()
    _check(load_library().ifdlbm_create_batch(len(cavities), arr,
                                              C.byref(opt) if opt is not None else None,
                                              C.c_void_p(int(stream)), C.byref(h)))
    return h


def ifdlbm_create_quad_batch(quads, opt=None, stream=0):
    arr = (ifdlbm_quad_cavity * len(quads))(*quads)
    h = _H()
    _check(load_library().ifdlbm_create_quad_batch(len(quads), arr,
                                                   C.byref(opt) if opt is not None else None,
                                                   C.c_void_p(int(stream)), C.byref(h)))
    return h


def ifdlbm_step(h, nsteps):
    return _check(load_library().ifdlbm_step(h, int(nsteps)), h)


def ifdlbm_macros(h, rho=None, u=None, v=None, psi=None):
    return _check(load_library().ifdlbm_macros(h, _ptr(rho), _ptr(u), _ptr(v), _ptr(psi)), h)


def ifdlbm_batch_macros(h, cavity, rho=None, u=None, v=None, psi=None):
    return _check(load_library().ifdlbm_batch_macros(h, int(cavity), _ptr(rho), _ptr(u), _ptr(v),
                                                     _ptr(psi)), h)


def ifdlbm_macros_dev(h, cavity, rho=None, u=None, v=None, psi=None):
    return _check(load_library().ifdlbm_macros_dev(h, int(cavity), _ptr(rho), _ptr(u), _ptr(v),
                                                   _ptr(psi)), h)


def ifdlbm_residual(h, out):
    return _check(load_library().ifdlbm_residual(h, _ptr(out)), h)


def ifdlbm_residual_dev(h, out):
    return _check(load_library().ifdlbm_residual_dev(h, _ptr(out)), h)


def ifdlbm_probe_dev(h, probes, out):
    """probes: CUDA int32 tensor [n][3] of (cavity, i, j); out: CUDA float64 tensor [n][3]."""
    return _check(load_library().ifdlbm_probe_dev(h, int(probes.shape[0]), _ptr(probes),
                                                  _ptr(out)), h)


def ifdlbm_batch_residual(h, out):
    return _check(load_library().ifdlbm_batch_residual(h, _ptr(out)), h)


def ifdlbm_batch_residual_async(h, out, status=None):
    """out: page-locked float64 tensor [ncav, 4] (or array); status: page-locked
    int32 tensor of one element, or None. Valid once the stream reaches the copy."""
    if status is not None and (status.dtype.itemsize != 4 or status.numel() < 1):
        raise ValueError("status must hold one 32-bit word")
    return _check(load_library().ifdlbm_batch_residual_async(h, _ptr(out), _ptr(status)), h)


def ifdlbm_get_state(h, cavity, fhat=None, lambda_prev=None):
    return _check(load_library().ifdlbm_get_state(h, int(cavity), _ptr(fhat), _ptr(lambda_prev)), h)


def ifdlbm_set_state(h, cavity, fhat, lambda_prev):
    return _check(load_library().ifdlbm_set_state(h, int(cavity), _ptr(fhat), _ptr(lambda_prev)), h)


def ifdlbm_state_bytes(h):
    return int(load_library().ifdlbm_state_bytes(h))


def ifdlbm_save_state_dev(h, dst):
    return _check(load_library().ifdlbm_save_state_dev(h, _ptr(dst)), h)


def ifdlbm_load_state_dev(h, src):
    return _check(load_library().ifdlbm_load_state_dev(h, _ptr(src)), h)


def ifdlbm_info(h, cavity=0) -> ifdlbm_info_t:
    info = ifdlbm_info_t()
    _check(load_library().ifdlbm_info(h, int(cavity), C.byref(info)), h)
    return info


def ifdlbm_sync(h):
    return _check(load_library().ifdlbm_sync(h), h)


def ifdlbm_destroy(h):
    return _check(load_library().ifdlbm_destroy(h))


def ifdlbm_last_error(h=None) -> str:
    return (load_library().ifdlbm_last_error(h) or b"").decode()


def ifdlbm_launch_count() -> int:
    return int(load_library().ifdlbm_launch_count())


def _device_f64(name, t, need):
    """Checks that `t` is a contiguous float64 CUDA tensor on the current
    device with at least `need` elements (the C entry point takes bare device
    pointers and cannot check any of this itself)."""
    if isinstance(t, np.ndarray) or not hasattr(t, "is_cuda"):
        raise TypeError(f"{name}: expected a CUDA tensor (the call takes device memory only)")
    import torch

    if not t.is_cuda:
        raise ValueError(f"{name}: tensor is on the host; device memory is required")
    if t.dtype != torch.float64:
        raise ValueError(f"{name}: expected float64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    if t.numel() < need:
        raise ValueError(f"{name}: {t.numel()} elements, {need} needed")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: tensor is on cuda:{t.device.index}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")


def ifdlbm_residual_fields_static(nx, ny, u1, v1, p1, u0, v0, p0, out, stream=0):
    """Eq. (2.19) residuals of caller-owned device fields; allocates nothing.

    u1, v1, p1, u0, v0, p0: float64 CUDA tensors of at least nx*ny elements,
    contiguous, on the current device; out: the same with at least 3."""
    nx, ny = int(nx), int(ny)
    need = nx * ny if nx > 0 and ny > 0 else 0
    for name, t in (("u1", u1), ("v1", v1), ("p1", p1), ("u0", u0), ("v0", v0), ("p0", p0)):
        _device_f64(name, t, need)
    _device_f64("out", out, 3)
    return _check(load_library().ifdlbm_residual_fields_static(
        int(nx), int(ny), _ptr(u1), _ptr(v1), _ptr(p1), _ptr(u0), _ptr(v0), _ptr(p0), _ptr(out),
        C.c_void_p(int(stream))))


def ifdlbm_autotune(h, trial_steps=10) -> "ifdlbm_tuning":
    best = ifdlbm_tuning()
    _check(load_library().ifdlbm_autotune(h, int(trial_steps), C.byref(best)), h)
    return best


def ifdlbm_adjoint_seed_energy(h, state, adj, dparams):
    return _check(load_library().ifdlbm_adjoint_seed_energy(h, _ptr(state), _ptr(adj),
                                                            _ptr(dparams)), h)


def ifdlbm_adjoint_seed_psi(h, state, nodes, adj, dparams):
    """nodes: sequence of (i, j) per cavity."""
    arr = (C.c_int * (2 * len(nodes)))(*[int(v) for ij in nodes for v in ij])
    return _check(load_library().ifdlbm_adjoint_seed_psi(h, _ptr(state), arr, _ptr(adj),
                                                         _ptr(dparams)), h)


def ifdlbm_adjoint_step(h, state_n, adj, dparams):
    return _check(load_library().ifdlbm_adjoint_step(h, _ptr(state_n), _ptr(adj), _ptr(dparams)), h)


def ifdlbm_intermediate_bytes(h):
    return int(load_library().ifdlbm_intermediate_bytes(h))


def ifdlbm_save_intermediates_dev(h, dst):
    return _check(load_library().ifdlbm_save_intermediates_dev(h, _ptr(dst)), h)


def ifdlbm_adjoint_step_saved(h, state_n, state_np1, inter, adj, dparams):
    return _check(load_library().ifdlbm_adjoint_step_saved(
        h, _ptr(state_n), _ptr(state_np1), _ptr(inter), _ptr(adj), _ptr(dparams)), h)


def ifdlbm_selftest_pow(h, x, m, fast, ref):
    return _check(load_library().ifdlbm_selftest_pow(h, int(x.numel()), _ptr(x), float(m),
                                                     _ptr(fast), _ptr(ref)), h)


def ifdlbm_selftest_pow_tab(h, cavity, x, out):
    """out[:n] = the FP32 form's C xf^m for cavity `cavity`, out[n:] = C * CUDA pow
    (x: float64 CUDA tensor of n arguments, out: float64 CUDA tensor of 2n)."""
    n = int(x.numel())
    _device_f64("x", x, n)
    _device_f64("out", out, 2 * n)
    return _check(load_library().ifdlbm_selftest_pow_tab(h, int(cavity), n, _ptr(x), _ptr(out)), h)


def ifdlbm_inject_tma_timeout(h, enable=True):
    return _check(load_library().ifdlbm_inject_tma_timeout(h, int(bool(enable))), h)


def ifdlbm_selftest_pow_f32(h, x, m, out):
    return _check(load_library().ifdlbm_selftest_pow_f32(h, int(x.numel()), _ptr(x), float(m),
                                                         _ptr(out)), h)


def ifdlbm_profile(h, enable):
    return _check(load_library().ifdlbm_profile(h, int(bool(enable))), h)


def ifdlbm_profile_read(h, kernel):
    """Returns (total milliseconds, launches) of kernel `kernel` since profiling began."""
    ms = C.c_double()
    n = C.c_int64()
    _check(load_library().ifdlbm_profile_read(h, int(kernel), C.byref(ms), C.byref(n)), h)
    return ms.value, n.value


def ifdlbm_find_eddies(nx, ny, geometry, psi):
    """Host-only: (primary, bottom-left, bottom-right) eddies of a [ny][nx] psi array."""
    out = (ifdlbm_eddy * 3)()
    g = ifdlbm_geometry(*geometry) if not isinstance(geometry, ifdlbm_geometry) else geometry
    _check(load_library().ifdlbm_find_eddies(int(nx), int(ny), g, _ptr(psi), out))
    return list(out)


def ifdlbm_eddies(h, cavity=0):
    """(primary, bottom-left, bottom-right) eddies of cavity `cavity` of a handle."""
    out = (ifdlbm_eddy * 3)()
    _check(load_library().ifdlbm_eddies(h, int(cavity), out), h)
    return list(out)
