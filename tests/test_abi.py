"""Host-side checks of the C ABI: the in-tree library loads, exports every
function include/lbm_pf.h declares, and validates grids, parameters and
workspace sizes without touching a GPU."""
import ctypes
import os
import re

import numpy as np

import pytest

import workloads as W
from paper_2003_06342_b300 import _binding as B
from paper_2003_06342_b300.solver import make_grid, make_params

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if fn.endswith(".h"):
            src = open(os.path.join(HEADER_DIR, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(B.lib, n), n
    # and the binding declares every one of them
    assert names <= set(B.SIGNATURES)


def test_bounds_checking_build_exports_the_same_abi():
    """liblbmpf_debug.so (LBM_CHECK_BOUNDS) is a drop-in replacement."""
    path = os.path.join(os.path.dirname(B.LIB_PATH), "liblbmpf_debug.so")
    dbg = ctypes.CDLL(path)
    for n in sorted(declared_functions()):
        assert hasattr(dbg, n), n
    dbg.lbm_strerror.restype = ctypes.c_char_p
    assert dbg.lbm_strerror(B.LBM_EBOUNDS) == B.lib.lbm_strerror(B.LBM_EBOUNDS)


def _ws(w, storage="fp32"):
    g = make_grid(w.n, w.periodic)
    p = make_params(w.params, storage)
    out = ctypes.c_size_t()
    lat = B.LBM_D2Q9 if w.dim == 2 else B.LBM_D3Q19_D3Q7
    return B.lib.lbm_workspace_bytes(ctypes.byref(g), lat, ctypes.byref(p), ctypes.byref(out)), out.value, g, p, lat


def test_workspace_bytes_scale_with_storage():
    w = W.film_boiling_2d(64, 32)
    r32, b32, *_ = _ws(w, "fp32")
    r16, b16, *_ = _ws(w, "fp16")
    assert r32 == 0 and r16 == 0
    N = 64 * 32
    assert b32 >= 2 * 27 * 4 * N + 3 * 4 * N
    assert b16 >= 2 * 27 * 2 * N and b16 < b32
    w3 = W.film_boiling_3d(16, 8, 12, modes=1, z0=5.0)
    r3, b3, *_ = _ws(w3, "fp32")
    assert r3 == 0 and b3 >= 2 * 45 * 4 * w3.cells


@pytest.mark.parametrize("field,value", [("nu_l", 0.0), ("M_phi", -1.0), ("W", 0.0), ("rho_g", 0.0),
                                         ("alpha_g", float("nan"))])
def test_invalid_parameters_rejected(field, value):
    w = W.film_boiling_2d(16, 16)
    w.params[field] = value
    r, *_ = _ws(w)
    assert r == B.LBM_EINVAL


def test_collision_option_validated():
    w = W.film_boiling_2d(16, 16)
    w.params.update(collision=1, trt_magic=(0.25, 3.0 / 16.0, 0.25))
    assert _ws(w)[0] == B.LBM_OK
    for bad in ((0.0, 0.25, 0.25), (0.25, -1.0, 0.25), (0.25, 0.25, float("inf"))):
        w.params["trt_magic"] = bad
        assert _ws(w)[0] == B.LBM_EINVAL, bad
    w.params.update(collision=3, trt_magic=(0.25, 0.25, 0.25))
    assert _ws(w)[0] == B.LBM_EINVAL
    # MRT of the flow set: rates in (0, 2), the coupled model only (2D and 3D)
    w.params.update(collision=2, mrt_rates=(1.4, 1.4, 1.2))
    assert _ws(w)[0] == B.LBM_OK
    for bad in ((0.0, 1.4, 1.2), (1.4, 2.0, 1.2), (1.4, 1.4, float("nan"))):
        w.params["mrt_rates"] = bad
        assert _ws(w)[0] == B.LBM_EINVAL, bad
    w.params["mrt_rates"] = (1.4, 1.4, 1.2)
    w.params["mrt_rates_g"] = (0.0, 1.5, 0.0, 1.2)          # 0: the BGK rate
    assert _ws(w)[0] == B.LBM_OK
    for bad in ((-0.1, 1.5, 1.0, 1.2), (1.0, 2.0, 1.0, 1.0), (1.0, 1.0, float("inf"), 1.0)):
        w.params["mrt_rates_g"] = bad
        assert _ws(w)[0] == B.LBM_EINVAL, bad
    w.params["mrt_rates_g"] = (0.0, 0.0, 0.0, 0.0)
    w3 = W.film_boiling_3d(8, 8, 8, modes=1, z0=3.0)
    w3.params.update(collision=2, mrt_rates=(1.4, 1.4, 1.2))
    assert _ws(w3)[0] == B.LBM_OK
    w3.params["mrt_rates_g"] = (1.2, 0.0, 0.0, 2.0)
    assert _ws(w3)[0] == B.LBM_EINVAL
    vm = W.vortex_disk(n=33)
    vm.params.update(collision=2, mrt_rates=(1.4, 1.4, 1.2))
    assert _ws(vm)[0] == B.LBM_EUNSUPPORTED
    # the phase-field-only model and the adjoint are BGK only
    v = W.vortex_disk(n=33)
    v.params.update(collision=1, trt_magic=(0.25, 0.25, 0.25))
    assert _ws(v)[0] == B.LBM_EUNSUPPORTED
    w.params.update(collision=1)
    r, nbytes, g, p, lat = _ws(w)
    buf = (ctypes.c_uint8 * (nbytes + 512))()
    base = (ctypes.addressof(buf) + 255) // 256 * 256
    h = ctypes.c_void_p()
    assert B.lib.lbm_create(ctypes.byref(g), lat, ctypes.byref(p), ctypes.c_void_p(base), nbytes,
                            None, ctypes.byref(h)) == B.LBM_OK
    a, sc = ctypes.c_size_t(), ctypes.c_size_t()
    assert B.lib.lbm_adjoint_bytes(h, ctypes.byref(a), ctypes.byref(sc)) == B.LBM_EUNSUPPORTED
    B.lib.lbm_destroy(h)


def test_gradient_option_validated():
    w = W.film_boiling_2d(16, 16)
    w.params.update(grad_scheme=1)
    assert _ws(w)[0] == B.LBM_OK
    w.params.update(grad_scheme=3)
    assert _ws(w)[0] == B.LBM_EINVAL
    w3 = W.film_boiling_3d(16, 8, 12, modes=1, z0=5.0)
    w3.params.update(grad_scheme=1)
    assert _ws(w3)[0] == B.LBM_OK
    v = W.vortex_disk(n=33)
    v.params.update(grad_scheme=1)
    assert _ws(v)[0] == B.LBM_EUNSUPPORTED             # coupled model only


def test_invalid_grids_rejected():
    w = W.film_boiling_2d(16, 16)
    w.periodic = (False, False)            # two wall axes
    assert _ws(w)[0] == B.LBM_EINVAL
    w = W.film_boiling_2d(16, 16)
    w.n = (0, 16)
    assert _ws(w)[0] == B.LBM_EINVAL


def test_create_checks_workspace_without_gpu():
    w = W.film_boiling_2d(16, 16)
    r, nbytes, g, p, lat = _ws(w)
    buf = (ctypes.c_uint8 * (nbytes + 512))()
    base = (ctypes.addressof(buf) + 255) // 256 * 256          # stand-in pointer, never dereferenced
    h = ctypes.c_void_p()
    assert B.lib.lbm_create(ctypes.byref(g), lat, ctypes.byref(p), ctypes.c_void_p(base), nbytes - 1,
                            None, ctypes.byref(h)) == B.LBM_ENOMEM
    assert B.lib.lbm_create(ctypes.byref(g), lat, ctypes.byref(p), ctypes.c_void_p(base + 8), nbytes,
                            None, ctypes.byref(h)) == B.LBM_EINVAL           # misaligned
    assert B.lib.lbm_create(ctypes.byref(g), lat, ctypes.byref(p), ctypes.c_void_p(base), nbytes,
                            None, ctypes.byref(h)) == B.LBM_OK
    steps = ctypes.c_int64(-1)
    assert B.lib.lbm_steps_done(h, ctypes.byref(steps)) == 0 and steps.value == 0
    assert B.lib.lbm_step(h, -1) == B.LBM_EINVAL
    B.lib.lbm_destroy(h)


def test_strerror():
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert B.lib.lbm_strerror(code)
    assert B.lib.lbm_strerror(-99) == b"unknown error"


def test_calls_reject_bad_arguments_before_device_work():
    w = W.film_boiling_2d(16, 16)
    r, nbytes, g, p, lat = _ws(w)
    buf = (ctypes.c_uint8 * (nbytes + 512))()
    base = (ctypes.addressof(buf) + 255) // 256 * 256
    h = ctypes.c_void_p()
    assert B.lib.lbm_create(ctypes.byref(g), lat, ctypes.byref(p), ctypes.c_void_p(base), nbytes,
                            None, ctypes.byref(h)) == B.LBM_OK
    f = B.lbm_fields()                       # phi and T missing
    assert B.lib.lbm_init(h, ctypes.byref(f)) == B.LBM_EINVAL
    assert B.lib.lbm_get_fields(h, None) == B.LBM_EINVAL
    f.dtype = 7
    assert B.lib.lbm_get_fields(h, ctypes.byref(f)) == B.LBM_EINVAL
    assert B.lib.lbm_stream_map(h, 2, None, None) == B.LBM_EINVAL
    assert B.lib.lbm_set_kernel(h, 9) == B.LBM_EINVAL
    # periodic state check: a negative period, a non-positive or non-finite bound
    assert B.lib.lbm_set_health_check(None, 10, 0.6) == B.LBM_EINVAL
    assert B.lib.lbm_set_health_check(h, -1, 0.6) == B.LBM_EINVAL
    assert B.lib.lbm_set_health_check(h, 10, 0.0) == B.LBM_EINVAL
    assert B.lib.lbm_set_health_check(h, 10, float("nan")) == B.LBM_EINVAL
    assert B.lib.lbm_set_health_check(h, 10, 0.6) == B.LBM_OK
    assert B.lib.lbm_set_health_check(h, 0, 0.0) == B.LBM_OK         # off
    small = ctypes.c_size_t()
    assert B.lib.lbm_state_bytes(h, ctypes.byref(small)) == B.LBM_OK
    assert B.lib.lbm_get_state(h, ctypes.c_void_p(base), small.value - 1, 1) == B.LBM_ENOMEM
    # segment calls: a stride shorter than one state, a negative count
    assert B.lib.lbm_step_record(h, 2, ctypes.c_void_p(base), small.value - 4) == B.LBM_ENOMEM
    assert B.lib.lbm_step_record(h, -1, ctypes.c_void_p(base), small.value) == B.LBM_EINVAL
    vb = ctypes.c_void_p(base)
    assert B.lib.lbm_adjoint_steps(h, vb, small.value, -1, vb, ctypes.c_void_p(base + 4), vb, vb) == B.LBM_EINVAL
    assert B.lib.lbm_adjoint_steps(h, vb, small.value - 4, 1, vb, ctypes.c_void_p(base + 4), vb,
                                   vb) == B.LBM_ENOMEM
    # the adjoint exists for 2D FP32 only
    a, sc = ctypes.c_size_t(), ctypes.c_size_t()
    assert B.lib.lbm_adjoint_bytes(h, ctypes.byref(a), ctypes.byref(sc)) == B.LBM_OK
    # the adjoint state: the 29 state planes and the phi adjoint; scratch: four stencil planes
    assert a.value == 30 * 16 * 16 * 4 and sc.value == 4 * 16 * 16 * 4
    B.lib.lbm_destroy(h)
    p16 = make_params(w.params, "fp16")
    h2 = ctypes.c_void_p()
    r16 = ctypes.c_size_t()
    B.lib.lbm_workspace_bytes(ctypes.byref(g), lat, ctypes.byref(p16), ctypes.byref(r16))
    assert B.lib.lbm_create(ctypes.byref(g), lat, ctypes.byref(p16), ctypes.c_void_p(base), r16.value,
                            None, ctypes.byref(h2)) == B.LBM_OK
    assert B.lib.lbm_adjoint_bytes(h2, ctypes.byref(a), ctypes.byref(sc)) == B.LBM_EUNSUPPORTED
    B.lib.lbm_destroy(h2)


def test_phase_field_model_validation():
    w = W.vortex_disk(n=33)
    g = B.lbm_grid()
    g.nx, g.ny, g.nz = 33, 33, 1
    g.periodic[:] = [1, 1, 1]
    size = ctypes.c_size_t()
    p = make_params(w.params)
    assert B.lib.lbm_workspace_bytes(ctypes.byref(g), B.LBM_D2Q9, ctypes.byref(p), ctypes.byref(size)) == B.LBM_OK
    pc = make_params(dict(w.params, model=0))
    size_c = ctypes.c_size_t()
    B.lib.lbm_workspace_bytes(ctypes.byref(g), B.LBM_D2Q9, ctypes.byref(pc), ctypes.byref(size_c))
    assert size.value > size_c.value                       # room for the imposed velocity
    for bad in (dict(w.params, model=2), dict(w.params, source_on=1)):
        pb = make_params(bad)
        assert B.lib.lbm_workspace_bytes(ctypes.byref(g), B.LBM_D2Q9, ctypes.byref(pb),
                                         ctypes.byref(size_c)) == B.LBM_EINVAL
    g3 = B.lbm_grid()
    g3.nx, g3.ny, g3.nz = 8, 8, 8
    g3.periodic[:] = [1, 1, 1]
    size3, size3c = ctypes.c_size_t(), ctypes.c_size_t()
    assert B.lib.lbm_workspace_bytes(ctypes.byref(g3), B.LBM_D3Q19_D3Q7, ctypes.byref(p),
                                     ctypes.byref(size3)) == B.LBM_OK
    assert B.lib.lbm_workspace_bytes(ctypes.byref(g3), B.LBM_D3Q19_D3Q7, ctypes.byref(pc),
                                     ctypes.byref(size3c)) == B.LBM_OK
    assert size3.value >= size3c.value + 3 * 8 * 8 * 8 * 4          # three velocity planes
    # lbm_set_velocity belongs to the phase-field model only
    buf = (ctypes.c_uint8 * (size.value + 512))()
    base = (ctypes.addressof(buf) + 255) // 256 * 256
    h = ctypes.c_void_p()
    assert B.lib.lbm_create(ctypes.byref(g), B.LBM_D2Q9, ctypes.byref(pc), ctypes.c_void_p(base),
                            size.value, None, ctypes.byref(h)) == B.LBM_OK
    f = B.lbm_fields()
    ux = np.zeros(33 * 33)
    f.ux = f.uy = ux.ctypes.data
    f.on_device, f.dtype = 0, 1
    assert B.lib.lbm_set_velocity(h, ctypes.byref(f), 0.0) == B.LBM_EUNSUPPORTED
    B.lib.lbm_destroy(h)


def test_struct_layouts_match_the_header(tmp_path):
    """Every field of lbm_grid, lbm_params and lbm_fields sits at the same
    offset, and each struct has the same size, in the C header (compiled with
    the host C compiler) and in the ctypes binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = (B.lbm_grid, B.lbm_params, B.lbm_fields)
    body = ""
    for st in structs:
        t = st.__name__
        body += "".join(f'    printf("{t}.{f[0]} %zu\\n", offsetof({t}, {f[0]}));\n' for f in st._fields_)
        body += f'    printf("{t}.sizeof %zu\\n", sizeof({t}));\n'
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "lbm_pf.h"\nint main(void) {\n'
                   f'{body}    return 0;\n}}\n')
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for st in structs:
        t = st.__name__
        for f in st._fields_:
            assert int(out[f"{t}.{f[0]}"]) == getattr(st, f[0]).offset, (t, f[0])
        assert int(out[f"{t}.sizeof"]) == ctypes.sizeof(st), t
