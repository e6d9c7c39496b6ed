"""The C-ABI library builds, loads and exports every symbol include/sense.h declares; host
logic and argument checks that need no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "sense.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(sense_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_09233_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2604_09233_gb300 import native
    assert sorted(native.EXPORTED) == _declared()
    for n in native.EXPORTED:
        assert callable(getattr(native, n)), n


def test_library_is_sm103a_only():
    """The shared object carries sm_103a code only (no PTX for JIT, no other arch)."""
    from paper_2604_09233_gb300 import build
    assert ["-gencode", "arch=compute_103a,code=sm_103a"] == build.ARCH


def test_error_strings_and_null_arguments():
    from paper_2604_09233_gb300 import native
    lib = native._lib
    assert lib.sense_strerror(0) == b"ok"
    assert lib.sense_strerror(-1) == b"invalid argument"
    assert lib.sense_plan_create(None, None) == -1
    assert lib.sense_encode(None, 0, None, None, None) in (-1, -3)
    assert lib.sense_plan_destroy(None) == 0
    c = ctypes.c_int32()
    assert lib.sense_lcurve_corner(None, 3, ctypes.byref(c)) == -1


def test_plan_create_validates_before_touching_the_device():
    from paper_2604_09233_gb300 import native
    K, L, C = 4, 5, 2
    Km = np.zeros((K, 1))
    Rm = np.zeros((1, L))
    S = np.zeros((L, C), np.complex64)
    Km[1, 0] = np.nan
    with pytest.raises(native.SenseError) as e:
        native.sense_plan_create(Km, Rm, S)
    assert e.value.code == -4  # ENONFINITE
    with pytest.raises(native.SenseError) as e:
        native.sense_plan_create(np.zeros((K, 1)), Rm, np.zeros((L, 65), np.complex64))
    assert e.value.code == -6  # EUNSUPPORTED: > 64 coils


def test_plan_create_without_gpu_reports_no_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2604_09233_gb300 import native
    with pytest.raises(native.SenseError) as e:
        native.sense_plan_create(np.zeros((4, 1)), np.zeros((1, 5)), np.zeros((5, 2), np.complex64))
    assert e.value.code == -7  # ENODEVICE


def test_lcurve_corner_matches_oracle_picker():
    """The library's host-side corner picker agrees with the oracle's on a curved history."""
    import oracle
    from paper_2604_09233_gb300 import native
    n = np.arange(1, 40)
    res = 1.0 + 30.0 * np.exp(-n / 4.0)            # residual falls, then flattens
    sol = 1.0 + 0.02 * n + 0.002 * n ** 2           # solution norm keeps growing
    hist = np.stack([np.ones_like(res), sol, res], axis=1)
    c_lib = native.sense_lcurve_corner(hist)
    c_or = oracle.lcurve_corner(res, sol)
    assert c_lib == c_or and 0 < c_lib < len(n) - 1


def test_gradient_and_batch_entry_points_check_arguments_first():
    """The differentiation, batch and allocation-free entry points reject null handles and
    impossible sizes before any device work (so these checks need no GPU)."""
    from paper_2604_09233_gb300 import native
    lib = native._lib
    vp = ctypes.c_void_p
    assert lib.sense_grad_b0(None, 0, None, None, None, None, None) == -1
    assert lib.sense_cg_ckpt_bytes(None, 10, 2) == -1
    assert lib.sense_cg_solve_ckpt(None, None, None, None, 2, None, 0, None, None) == -1
    assert lib.sense_cg_backward(None, None, None, 0, None, None, None, None) == -1
    h = vp()
    assert lib.sense_batch_create(None, 0, ctypes.byref(h)) == -1
    assert lib.sense_batch_destroy(None) == 0
    assert lib.sense_batch_plan(None, 0, ctypes.byref(h)) == -1
    assert lib.sense_batch_info(None, (ctypes.c_int32 * 4)()) == -1
    assert lib.sense_batch_normal_op(None, 2, None, None, None) == -1
    assert lib.sense_batch_cg_solve(None, None, None, None, None, None) == -1
    assert lib.sense_batch_set_tuning(None, 16, 4) == -1
    assert lib.sense_batch_autotune(None, 2, None, None, None) == -1
    d = ctypes.c_double()
    buf = (ctypes.c_float * 8)()
    # the allocation-free encode: sizes first (L < 1), then its fixed scratch (K x 32 coils
    # one sample row beyond 2^21 complex values)
    assert lib.sense_encode_noalloc(0, 4, 8, 1, ctypes.addressof(d), ctypes.addressof(d),
                                    buf, None, buf, buf, None) == -1
    assert lib.sense_encode_noalloc(4, (1 << 21) // 32 + 1, 32, 1, ctypes.addressof(d),
                                    ctypes.addressof(d), buf, None, buf, buf, None) == -1
    assert b"scratch" in lib.sense_last_error()


def test_batch_create_without_gpu_reports_no_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2604_09233_gb300 import native
    with pytest.raises(native.SenseError) as e:
        native.sense_batch_create([(np.zeros((4, 1)), np.zeros((1, 5)),
                                    np.zeros((5, 2), np.complex64), None)])
    assert e.value.code == -7


def test_smoothing_and_filter_entry_points_check_arguments_first():
    """Map smoothing rejects null pointers, impossible grids, orders, field counts and
    preconditioner codes, and host memory, before any device work; the k-space filter mask
    rejects empty grids."""
    from paper_2604_09233_gb300 import native
    lib = native._lib
    buf = (ctypes.c_float * 64)()
    info = (native.SmoothInfo * 4)()

    def opts(**kw):
        base = dict(nx=4, ny=4, nz=1, order=2, alpha=0.5, max_iter=10, rel_tol=1e-6, precond=1,
                    n_fields=1)
        base.update(kw)
        return native.SmoothOpts(*[base[k] for k in ("nx", "ny", "nz", "order", "alpha",
                                                     "max_iter", "rel_tol", "precond",
                                                     "n_fields")])

    for bad in (dict(nx=0), dict(order=3), dict(alpha=-1.0), dict(max_iter=-1),
                dict(rel_tol=-1e-3), dict(precond=2), dict(n_fields=0), dict(n_fields=70000)):
        o = opts(**bad)
        assert lib.sense_smooth_map(ctypes.byref(o), buf, buf, buf, buf, info, None) == -1, bad
    o = opts()
    assert lib.sense_smooth_map(None, buf, buf, buf, buf, info, None) == -1
    assert lib.sense_smooth_map(ctypes.byref(o), None, buf, buf, buf, info, None) == -1
    # host arrays are refused (the solver works on device fields only)
    assert lib.sense_smooth_map(ctypes.byref(o), buf, buf, buf, buf, info, None) == -1
    assert b"device" in lib.sense_last_error()
    assert lib.sense_smooth_sensitivities(ctypes.byref(o), 0, buf, buf, buf, buf, info,
                                          None) == -1
    assert lib.sense_smooth_sensitivities(ctypes.byref(o), 40000, buf, buf, buf, buf, info,
                                          None) == -1
    kx = (ctypes.c_double * 3)(0.0, 1.0, 0.0)
    assert lib.sense_kspace_filter_mask(0, 4, 1e-3, 1e-3, kx, kx, 3, buf) == -1


def test_header_is_plain_c():
    """include/sense.h compiles as C99 and as C++17 on its own (plain C types only)."""
    import shutil
    import subprocess
    from paper_2604_09233_gb300 import build
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(build.__file__))),
                       "include", "sense.h")
    for cc, std, lang in (("gcc", "-std=c99", "c"), ("g++", "-std=c++17", "c++")):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not available")
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-x", lang,
                            hdr], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
