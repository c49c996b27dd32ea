"""Convenience wrapper owning one library handle (one cavity or a batch).

It only marshals arguments to the C ABI (``capi``); every step of the
method runs in libifdlbm.so on the GPU. The handle gets its own CUDA stream
from PyTorch and allocates through PyTorch's caching allocator.
"""
from __future__ import annotations

import numpy as np

from . import capi

_PREC = {"fp64": capi.IFDLBM_FP64, "fp32dev": capi.IFDLBM_FP32DEV}
_KERN = {"auto": capi.IFDLBM_KERNEL_AUTO, "staged": capi.IFDLBM_KERNEL_STAGED,
         "fused": capi.IFDLBM_KERNEL_FUSED}
_SCHED = {"grid": capi.IFDLBM_SCHED_GRID, "static": capi.IFDLBM_SCHED_STATIC,
          "dynamic": capi.IFDLBM_SCHED_DYNAMIC}


def make_options(precision="fp64", kernel="auto", eta_b=None, cfl=None, c=None, dt=None,
                 gamma_min=None, graph_chunk=None, fused_threads=None, fused_rows=None,
                 schedule=None, dt_mode=None, lambda_mode=None, power_fp32=None,
                 wall_pressure=None):
    opt = capi.ifdlbm_default_options()
    opt.precision = _PREC[precision]
    opt.kernel = _KERN[kernel]
    for name, val in (("eta_b", eta_b), ("cfl", cfl), ("c", c), ("dt", dt),
                      ("gamma_min", gamma_min), ("graph_chunk", graph_chunk),
                      ("fused_threads", fused_threads), ("fused_rows", fused_rows)):
        if val is not None:
            setattr(opt, name, val)
    if schedule is not None:
        opt.schedule = _SCHED[schedule] if isinstance(schedule, str) else int(schedule)
    if dt_mode is not None:
        opt.dt_mode = {"grid": capi.IFDLBM_DT_GRID,
                       "contravariant": capi.IFDLBM_DT_CONTRAVARIANT}[dt_mode]
    if power_fp32 is not None:
        opt.power_fp32 = int(bool(power_fp32))
    if wall_pressure is not None:
        opt.wall_pressure = {"zeroth": capi.IFDLBM_WALLP_ZEROTH,
                             "first": capi.IFDLBM_WALLP_FIRST}[wall_pressure]
    if lambda_mode is not None:
        opt.lambda_mode = {"lagged": capi.IFDLBM_LAMBDA_LAGGED,
                           "implicit": capi.IFDLBM_LAMBDA_IMPLICIT}[lambda_mode]
    return opt


def cavity(nx, ny, Re, n, theta_deg=60.0, U_lid=0.1, L=1.0, H=1.0):
    """A cavity description (ifdlbm_cavity)."""
    return capi.ifdlbm_cavity(int(nx), int(ny), capi.ifdlbm_geometry(L, H, theta_deg),
                              float(Re), float(n), float(U_lid))


def quad_cavity(nx, ny, corners, Re, n, U_lid=0.1, H=1.0):
    """A cavity on a general quadrilateral (ifdlbm_quad_cavity); corners are
    ((x0, y0) bottom-left, (x1, y1) bottom-right, (x2, y2) top-left,
    (x3, y3) top-right), the lid being the top edge."""
    flat = [float(v) for xy in corners for v in xy]
    if len(flat) != 8:
        raise ValueError("corners: four (x, y) pairs")
    return capi.ifdlbm_quad_cavity(int(nx), int(ny), (capi.C.c_double * 8)(*flat), float(H),
                                   float(Re), float(n), float(U_lid))


class Solver:
    """Owns one handle over a batch of cavities: all ``cavity(...)`` records
    (trapezoids) or all ``quad_cavity(...)`` records (general quadrilaterals)."""

    def __init__(self, cavities, stream=None, **options):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the IFDLBM library has no CPU path")
        capi.load_library()
        capi.use_torch_allocator()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.cavities = list(cavities)
        self.opt = make_options(**options)
        quads = [isinstance(c, capi.ifdlbm_quad_cavity) for c in self.cavities]
        if any(quads) and not all(quads):
            raise ValueError("a batch holds either trapezoid or quadrilateral cavities")
        create = capi.ifdlbm_create_quad_batch if any(quads) else capi.ifdlbm_create_batch
        self.h = create(self.cavities, self.opt, self.stream.cuda_stream)

    @property
    def ncav(self):
        return len(self.cavities)

    def step(self, nsteps=1):
        capi.ifdlbm_step(self.h, nsteps)
        return self

    def residual(self):
        out = np.zeros((self.ncav, 4))
        capi.ifdlbm_batch_residual(self.h, out)
        return out

    def macros(self, cavity=0):
        c = self.cavities[cavity]
        f = {k: np.zeros((c.ny, c.nx)) for k in ("rho", "u", "v", "psi")}
        capi.ifdlbm_batch_macros(self.h, cavity, f["rho"], f["u"], f["v"], f["psi"])
        return f

    def eddies(self, cavity=0):
        """Primary, bottom-left and bottom-right eddy centres (ifdlbm_eddies)."""
        return capi.ifdlbm_eddies(self.h, cavity)

    def get_state(self, cavity=0):
        c = self.cavities[cavity]
        fhat = np.zeros((9, c.ny, c.nx))
        lam = np.zeros((c.ny, c.nx))
        capi.ifdlbm_get_state(self.h, cavity, fhat, lam)
        return fhat, lam

    def set_state(self, cavity, fhat, lam):
        capi.ifdlbm_set_state(self.h, cavity, np.ascontiguousarray(fhat, dtype=np.float64),
                              np.ascontiguousarray(lam, dtype=np.float64))

    def info(self, cavity=0):
        return capi.ifdlbm_info(self.h, cavity)

    def autotune(self, trial_steps=10):
        """Pick the fused kernel's CTA width, rows per task and schedule (state unchanged)."""
        return capi.ifdlbm_autotune(self.h, trial_steps)

    def sync(self):
        capi.ifdlbm_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            capi.ifdlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
