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
