"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point include/ifdlbm.h declares; argument validation happens before
any device work (no compute calls are made here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ifdlbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2306_07603_gb300 import capi
    if not os.path.exists(capi.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build libifdlbm.so")
        from paper_2306_07603_gb300 import build
        build.build()
    return capi.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ifdlbm_\w+)\s*\(", text)) - {"ifdlbm_alloc_fn", "ifdlbm_free_fn"})


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_covers_every_declared_symbol():
    from paper_2306_07603_gb300 import capi
    assert set(declared_functions()) <= set(capi._SIGS)


def test_default_options(lib):
    from paper_2306_07603_gb300 import capi
    o = capi.ifdlbm_default_options()
    assert (o.cfl, o.c, o.eta_b, o.rho0) == (0.5, 1.0, 0.5, 1.0)
    assert o.precision == capi.IFDLBM_FP64 and o.graph_chunk == 32
    # the FP32-deviation form keeps the power law in FP64 unless the opt-in is set
    assert o.power_fp32 == 0 and o.lambda_mode == capi.IFDLBM_LAMBDA_LAGGED


@pytest.mark.parametrize("args,frag", [
    ((4, 9, (1, 1, 60), 100, 0.75, 0.1), ">= 5"),
    ((9, 9, (1, 1, 0), 100, 0.75, 0.1), "theta"),
    ((9, 9, (1, 1, 91), 100, 0.75, 0.1), "theta"),
    ((9, 9, (0, 1, 60), 100, 0.75, 0.1), "L and H"),
    ((9, 9, (1, 1, 60), -1, 0.75, 0.1), "Re, n"),
    ((9, 9, (1, 1, 60), 100, 0.0, 0.1), "Re, n"),
    ((9, 9, (1, 1, 60), 100, 0.75, 0.0), "Re, n"),
])
def test_invalid_arguments_rejected_before_device_use(lib, args, frag):
    from paper_2306_07603_gb300 import capi
    with pytest.raises(capi.IfdlbmError) as e:
        capi.ifdlbm_create(*args)
    assert e.value.code == capi.IFDLBM_ERR_INVALID_ARG
    assert frag in str(e.value)


def test_invalid_options_rejected(lib):
    from paper_2306_07603_gb300 import capi
    for field, val in (("eta_b", 1.5), ("cfl", 0.0), ("precision", 7), ("graph_chunk", 3),
                       ("power_fp32", 1), ("power_fp32", 2), ("wall_pressure", 2)):
        o = capi.ifdlbm_default_options()
        setattr(o, field, val)
        with pytest.raises(capi.IfdlbmError) as e:
            capi.ifdlbm_create(9, 9, (1, 1, 60), 100, 0.75, 0.1, o)
        assert e.value.code == capi.IFDLBM_ERR_INVALID_ARG


def test_no_cpu_fallback_without_a_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2306_07603_gb300 import capi
    with pytest.raises(capi.IfdlbmError) as e:
        capi.ifdlbm_create(9, 9, (1, 1, 60), 100, 0.75, 0.1)
    assert e.value.code == capi.IFDLBM_ERR_CUDA


def test_first_order_wall_pressure_refuses_the_fused_kernel(lib):
    from paper_2306_07603_gb300 import capi
    o = capi.ifdlbm_default_options()
    o.wall_pressure, o.kernel = capi.IFDLBM_WALLP_FIRST, capi.IFDLBM_KERNEL_FUSED
    with pytest.raises(capi.IfdlbmError) as e:
        capi.ifdlbm_create(9, 9, (1, 1, 60), 100, 0.75, 0.1, o)
    assert e.value.code == capi.IFDLBM_ERR_INVALID_ARG and "staged" in str(e.value)


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2306_07603_gb300 import capi
    assert lib.ifdlbm_step(None, 1) == capi.IFDLBM_ERR_INVALID_ARG
    assert lib.ifdlbm_sync(None) == capi.IFDLBM_ERR_INVALID_ARG
    assert lib.ifdlbm_destroy(None) == capi.IFDLBM_OK
    assert lib.ifdlbm_state_bytes(None) == -1
    # the adjoint sweep's intermediates
    assert lib.ifdlbm_intermediate_bytes(None) == -1
    assert lib.ifdlbm_save_intermediates_dev(None, None) == capi.IFDLBM_ERR_INVALID_ARG
    assert lib.ifdlbm_adjoint_step_saved(None, None, None, None, None, None) == \
        capi.IFDLBM_ERR_INVALID_ARG


SKEW = ((0.1, -0.05), (1.3, 0.12), (-0.2, 0.9), (1.05, 1.1))


@pytest.mark.parametrize("corners,kw,frag", [
    (((0, 0), (1, 0), (1, 1), (0, 1)), {}, "convex"),          # top corners swapped: J < 0
    (((0, 0), (1, 0), (0, 1), (0.0, 1.0)), {}, "convex"),      # degenerate: J = 0 at a corner
    (((0, 0), (1, 0), (0, 1), (float("nan"), 1.0)), {}, "finite"),
    (SKEW, {"H": 0.0}, "H must"),
    (SKEW, {"Re": -1.0}, "Re, n"),
])
def test_invalid_quadrilaterals_rejected_before_device_use(lib, corners, kw, frag):
    from paper_2306_07603_gb300 import capi
    from paper_2306_07603_gb300.solver import quad_cavity
    args = dict(Re=100.0, n=0.75)
    args.update(kw)
    q = quad_cavity(9, 9, corners, **args)
    with pytest.raises(capi.IfdlbmError) as e:
        capi.ifdlbm_create_quad_batch([q])
    assert e.value.code == capi.IFDLBM_ERR_INVALID_ARG
    assert frag in str(e.value)


@pytest.mark.parametrize("field,val,frag", [("kernel", 2, "fused kernel needs FP32DEV"),
                                            ("dt_mode", 0, "dt_mode GRID")])
def test_quadrilateral_options_rejected(lib, field, val, frag):
    from paper_2306_07603_gb300 import capi
    from paper_2306_07603_gb300.solver import quad_cavity
    assert (capi.IFDLBM_KERNEL_FUSED, capi.IFDLBM_DT_GRID) == (2, 0)
    o = capi.ifdlbm_default_options()
    setattr(o, field, val)
    with pytest.raises(capi.IfdlbmError) as e:
        capi.ifdlbm_create_quad_batch([quad_cavity(9, 9, SKEW, 100.0, 0.75)], o)
    assert e.value.code == capi.IFDLBM_ERR_INVALID_ARG
    assert frag in str(e.value)


def test_quadrilateral_fused_kernel_accepted_for_fp32_lagged(lib):
    """The header's statement: for general quadrilaterals FUSED is accepted with
    FP32DEV and the lagged relaxation time (creation then gets past argument
    checking to the device, which is absent here), and INVALID_ARG with FP64
    or with the implicit relaxation time."""
    import torch

    from paper_2306_07603_gb300 import capi
    from paper_2306_07603_gb300.solver import quad_cavity
    q = [quad_cavity(9, 9, SKEW, 100.0, 0.75)]
    for prec, lmode, ok in ((capi.IFDLBM_FP32DEV, capi.IFDLBM_LAMBDA_LAGGED, True),
                            (capi.IFDLBM_FP64, capi.IFDLBM_LAMBDA_LAGGED, False),
                            (capi.IFDLBM_FP32DEV, capi.IFDLBM_LAMBDA_IMPLICIT, False)):
        o = capi.ifdlbm_default_options()
        o.kernel, o.precision, o.lambda_mode = capi.IFDLBM_KERNEL_FUSED, prec, lmode
        if ok and torch.cuda.is_available():
            continue
        with pytest.raises(capi.IfdlbmError) as e:
            capi.ifdlbm_create_quad_batch(q, o)
        assert e.value.code == (capi.IFDLBM_ERR_CUDA if ok else capi.IFDLBM_ERR_INVALID_ARG), (
            prec, lmode, str(e.value))
    text = open(HEADER).read()
    assert "FUSED is INVALID_ARG." not in text.split("ifdlbm_create_quad_batch")[0][-900:]


def test_static_residual_wrapper_rejects_what_the_c_entry_cannot_check(lib):
    """ifdlbm_residual_fields_static takes bare device pointers; the binding
    refuses host arrays, host tensors, other dtypes, non-contiguous or short
    tensors before anything reaches the library."""
    import numpy as np
    import torch

    from paper_2306_07603_gb300 import capi
    nx, ny = 8, 4
    host = np.zeros(nx * ny)
    with pytest.raises(TypeError):
        capi.ifdlbm_residual_fields_static(nx, ny, host, host, host, host, host, host, host)
    t = torch.zeros(nx * ny, dtype=torch.float64)
    with pytest.raises(ValueError, match="host"):
        capi.ifdlbm_residual_fields_static(nx, ny, t, t, t, t, t, t, t)
    if not torch.cuda.is_available():
        return
    d = torch.zeros(nx * ny, dtype=torch.float64, device="cuda")
    for bad, frag in ((d.float(), "float64"), (d[:-1], "needed"), (d.view(ny, nx).t(), "contiguous")):
        with pytest.raises(ValueError, match=frag):
            capi.ifdlbm_residual_fields_static(nx, ny, bad, d, d, d, d, d, d)
    with pytest.raises(ValueError, match="needed"):
        capi.ifdlbm_residual_fields_static(nx, ny, d, d, d, d, d, d, d[:2])


STRUCTS = ["ifdlbm_geometry", "ifdlbm_options", "ifdlbm_cavity", "ifdlbm_quad_cavity",
           "ifdlbm_info_t", "ifdlbm_tuning", "ifdlbm_eddy"]


def test_header_is_plain_c_and_the_binding_matches_its_layouts(tmp_path):
    """The ABI header compiles as C99, and every struct's size and field
    offsets in the ctypes binding equal the C compiler's."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import subprocess

    from paper_2306_07603_gb300 import capi
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ifdlbm.h"', "int main(void) {"]
    expect = []
    for name in STRUCTS:
        cls = getattr(capi, name)
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        expect.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {fname}));')
            expect.append(getattr(cls, fname).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == expect


def test_library_is_usable_from_c(lib, tmp_path):
    """A C program links libifdlbm.so and calls it through the header alone:
    options, argument checks, and create (IFDLBM_ERR_CUDA without a GPU; on a
    GPU one step, a residual read and destroy)."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import subprocess

    from paper_2306_07603_gb300 import capi
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include "ifdlbm.h"
int main(void) {
  ifdlbm_options o;
  if (ifdlbm_default_options(&o) != IFDLBM_OK || o.cfl != 0.5) return 10;
  ifdlbm_geometry g = {1.0, 1.0, 60.0};
  ifdlbm_handle h = 0;
  if (ifdlbm_create(3, 9, g, 100.0, 0.75, 0.1, &o, NULL, &h) != IFDLBM_ERR_INVALID_ARG) return 11;
  int rc = ifdlbm_create(17, 17, g, 100.0, 0.75, 0.1, &o, NULL, &h);
  if (rc == IFDLBM_ERR_CUDA) { printf("nogpu %s\n", ifdlbm_last_error(NULL)); return 0; }
  if (rc != IFDLBM_OK) return 12;
  double r[4];
  if (ifdlbm_step(h, 2) != IFDLBM_OK || ifdlbm_residual(h, r) != IFDLBM_OK) return 13;
  ifdlbm_destroy(h);
  printf("gpu %g\n", r[3]);
  return 0;
}
''')
    exe = tmp_path / "use"
    libdir = os.path.dirname(capi.LIB_PATH)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-lifdlbm",
                        f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.startswith(("nogpu", "gpu"))
