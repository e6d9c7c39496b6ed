"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of an
oracle function (Python functions: a wrong weight index, stencil coefficient or sign, a dropped
square root, shifted rows, a skipped normalisation, an uncentred or unscaled transform, a
reversed curvature; the C operators and CG: a conjugated exponential, a missing conjugate or
term, a misplaced intensity correction, a broken CG recurrence, a gradient sign) and checks
that the pins of that function, which the real oracle passes, reject the copy. The mistakes are
planted on the CPU, in the oracle only."""
import ctypes
import inspect
import os
import shutil
import subprocess
import textwrap

import numpy as np
import pytest

import oracle
from oracle import oracle as om
import test_oracle_pins as pins


def _mutant(func, edits):
    """A copy of `func` with each (old, new) text replacement applied once, evaluated in the
    oracle module's namespace (so it calls the real versions of the other functions)."""
    src = textwrap.dedent(inspect.getsource(func))
    for old, new in edits:
        assert src.count(old) >= 1, old
        src = src.replace(old, new, 1)
    ns = dict(om.__dict__)
    exec(compile(src, f"<mutant of {func.__name__}>", "exec"), ns)
    return ns[func.__name__]


def _smooth_map_all(fn):
    pins.smooth_map_pins(fn)
    pins.smooth_map_weight_pin(fn)


CASES = [
    # smoothing (Eqs. 1 and 3)
    ("first-difference weight on the next voxel", om.smooth_map, _smooth_map_all,
     [("vals += [-wd[line[c]], wd[line[c]]]", "vals += [-wd[line[c + 1]], wd[line[c + 1]]]")]),
    ("second-difference centre coefficient", om.smooth_map, _smooth_map_all,
     [("vals += [wd[line[c]], -2 * wd[line[c]], wd[line[c]]]",
       "vals += [wd[line[c]], -1 * wd[line[c]], wd[line[c]]]")]),
    ("first-difference sign of one term", om.smooth_map, _smooth_map_all,
     [("vals += [-wd[line[c]], wd[line[c]]]", "vals += [wd[line[c]], wd[line[c]]]")]),
    ("alpha not square-rooted", om.smooth_map, _smooth_map_all,
     [("blocks.append(np.sqrt(alpha) *", "blocks.append(alpha *")]),
    ("second-difference rows shifted by one", om.smooth_map, _smooth_map_all,
     [("for c in range(1, m - 1):", "for c in range(0, m - 2):")]),
    ("data term weighted twice", om.smooth_map, _smooth_map_all,
     [("rhs = np.concatenate([w0 * np.asarray", "rhs = np.concatenate([w0 * w0 * np.asarray")]),
    ("unconstrained voxels solved too", om.smooth_map, _smooth_map_all,
     [("keep = N.diagonal() > 0", "keep = N.diagonal() >= 0")]),
    ("derivative rows only along the last axis", om.smooth_map, _smooth_map_all,
     [("for ax in range(len(shape)):", "for ax in range(len(shape) - 1, len(shape)):")]),
    # sensitivities (magnitude and normalised map per coil)
    ("recombined without normalising u", om.smooth_sensitivities,
     pins.smooth_sensitivities_pins,
     [("out[:, c] = np.where(a > 0, m * u / np.where(a > 0, a, 1.0), 0.0)",
       "out[:, c] = m * u")]),
    ("the map itself smoothed instead of the normalised map", om.smooth_sensitivities,
     pins.smooth_sensitivities_pins,
     [("u = smooth_map(shape, 2, alpha, m_t, m_r, unit)",
       "u = smooth_map(shape, 2, alpha, m_t, m_r, S_hat[:, c])")]),
    ("magnitude taken from the smoothed normalised map", om.smooth_sensitivities,
     pins.smooth_sensitivities_pins,
     [("out[:, c] = np.where(a > 0, m * u / np.where(a > 0, a, 1.0), 0.0)",
       "out[:, c] = np.where(a > 0, a * u / np.where(a > 0, a, 1.0), 0.0)")]),
    # k-space filter
    ("forward transform with the wrong sign", om.kspace_filter, pins.kspace_filter_pins,
     [("x = np.moveaxis(np.tensordot(W(n, +1)", "x = np.moveaxis(np.tensordot(W(n, -1)")]),
    ("inverse transform without 1/n", om.kspace_filter, pins.kspace_filter_pins,
     [("axes=(1, 0)) / n", "axes=(1, 0))")]),
    ("uncentred frequency index", om.kspace_filter, pins.kspace_filter_pins,
     [("c = np.arange(n) - n // 2", "c = np.arange(n)")]),
    # k-space mask
    ("mask grid not centred", om.kspace_mask, pins.kspace_mask_pins,
     [("u = 2 * np.pi * (np.arange(nx) - nx // 2) / (nx * dx)",
       "u = 2 * np.pi * np.arange(nx) / (nx * dx)")]),
    ("mask spacings swapped", om.kspace_mask, pins.kspace_mask_pins,
     [("u = 2 * np.pi * (np.arange(nx) - nx // 2) / (nx * dx)",
       "u = 2 * np.pi * (np.arange(nx) - nx // 2) / (nx * dy)")]),
    ("mask axes swapped", om.kspace_mask, pins.kspace_mask_pins,
     [("np.stack([U.ravel(), V.ravel()], axis=1)", "np.stack([V.ravel(), U.ravel()], axis=1)")]),
    # L-curve corner
    ("curvature sign reversed", om.lcurve_corner, pins.lcurve_pins,
     [("k = (dda * db - da * ddb) / den", "k = (da * ddb - dda * db) / den")]),
    ("minimum instead of maximum", om.lcurve_corner, pins.lcurve_pins,
     [("best, best_k = -1, -np.inf", "best, best_k = -1, np.inf"),
      ("if k > best_k:", "if k < best_k:")]),
    ("the start x_0 read as a point of the curve", om.lcurve_corner, pins.lcurve_pins,
     [("a = np.log(np.asarray(res_norm, np.float64)[1:])",
       "a = np.log(np.asarray(res_norm, np.float64))"),
      ("b = np.log(np.asarray(sol_norm, np.float64)[1:])",
       "b = np.log(np.asarray(sol_norm, np.float64))"),
      ("best, best_k = i + 1, k", "best, best_k = i, k")]),
]


def test_the_real_oracle_passes_every_pin_used_here():
    _smooth_map_all(om.smooth_map)
    pins.smooth_sensitivities_pins(om.smooth_sensitivities)
    pins.kspace_filter_pins(om.kspace_filter)
    pins.lcurve_pins(om.lcurve_corner)
    pins.kspace_mask_pins(om.kspace_mask)


@pytest.mark.parametrize("name,func,check,edits", CASES, ids=[c[0] for c in CASES])
def test_pins_reject_a_planted_mistake(name, func, check, edits):
    bad = _mutant(func, edits)
    with np.errstate(all="ignore"), pytest.raises(Exception):
        check(bad)


# ---------------------------------------------------------------------------------------
# The C part of the oracle: mutated copies of sense_oracle.c are compiled into a scratch
# library and put behind the same Python wrappers; the operator, CG and gradient pins (with
# fixtures built by the real library) must reject each one.
# ---------------------------------------------------------------------------------------
C_FUNCS = ["or_num_threads", "or_set_num_threads", "or_encode", "or_adjoint", "or_normal",
           "or_cg", "or_grad_omega", "or_grad_omega_adjoint"]

OPERATOR_PINS = ["test_closed_form_dft_matches_numpy_fft", "test_point_source_analytic_signal",
                 "test_adjointness", "test_normal_operator_hermitian_psd"]
CG_PINS = ["test_cg_converges_to_dense_normal_solution",
           "test_cg_iterates_minimise_error_over_krylov_space",
           "test_cg_history_and_residual_monotone"]
X0_PINS = ["test_cg_from_x0_minimises_error_over_shifted_krylov_space",
           "test_cg_from_the_solution_stops_at_once"]
GRAD_PINS = ["test_grad_omega_matches_central_differences",
             "test_grad_omega_adjoint_matches_central_differences"]

C_CASES = [
    ("E with the conjugate exponential", OPERATOR_PINS,
     [("const cplx e = cexp(I * phase_of(Km, Rm, L, P1, kappa, l));\n      const cplx w",
       "const cplx e = cexp(-I * phase_of(Km, Rm, L, P1, kappa, l));\n      const cplx w")]),
    ("E^H without the conjugate sensitivities", OPERATOR_PINS,
     [("v += conj(S[l * C + lam]) * acc[lam];", "v += S[l * C + lam] * acc[lam];")]),
    ("phase without the B0 row", OPERATOR_PINS,
     [("for (int p = 0; p < P1; ++p) phi +=", "for (int p = 1; p < P1; ++p) phi +=")]),
    ("E without the intensity correction", OPERATOR_PINS,
     [("const cplx e = cexp(I * phase_of(Km, Rm, L, P1, kappa, l));\n"
       "      const cplx w = m[l] * (j ? j[l] : 1.0);",
       "const cplx e = cexp(I * phase_of(Km, Rm, L, P1, kappa, l));\n"
       "      const cplx w = m[l];")]),
    ("CG step length inverted", CG_PINS,
     [("const cplx a_over_b = alpha / beta;", "const cplx a_over_b = beta / alpha;")]),
    ("CG without the direction recurrence", CG_PINS,
     [("p[l] = r[l] + ratio * p[l];", "p[l] = r[l];")]),
    ("CG inner product without the conjugate", CG_PINS,
     [("acc += conj(a[i]) * b[i];", "acc += a[i] * b[i];")]),
    ("CG ends dividing by j", CG_PINS,
     [("rho[l] *= j[l];", "rho[l] /= j[l];")]),
    ("CG from x0 keeps r_0 = E^H s", X0_PINS,
     [("for (int64_t l = 0; l < L; ++l) r[l] -= q[l];", "")]),
    ("CG from x0 starts at zero", X0_PINS,
     [("memcpy(rho, x0, sizeof(cplx) * (size_t)L);",
       "for (int64_t l = 0; l < L; ++l) rho[l] = 0.0;")]),
    ("CG tolerance relative to the start residual", X0_PINS,
     [("const double r0 = norm2(r, L);   /* ||E^H sigma||: the tolerance reference */",
       "double r0;"),
      ("  memcpy(p, r, sizeof(cplx) * (size_t)L);\n",
       "  memcpy(p, r, sizeof(cplx) * (size_t)L);\n  r0 = norm2(r, L);\n")]),
    ("B0 gradient with the wrong time factor sign", GRAD_PINS,
     [("(-I * Km[kappa * P1 + 0])", "(I * Km[kappa * P1 + 0])")]),
    ("adjoint B0 gradient with the wrong time factor sign", GRAD_PINS,
     [("const cplx dy = I * Km[kappa * P1 + 0]", "const cplx dy = -I * Km[kappa * P1 + 0]")]),
]


@pytest.fixture(scope="module")
def pin_fixtures():
    """The pins' fixtures (the same workloads as in test_oracle_pins), built with the real
    oracle library."""
    from paper_2604_09233_gb300 import synthetic
    small = synthetic.small_2d(seed=11, matrix=12, n_coils=4, n_samples=400, order=3,
                               with_j=True)
    wl = synthetic.small_2d(seed=21, matrix=6, n_coils=4, n_samples=180, order=2, R=1,
                            with_j=True)
    sigma = oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j) + wl.noise
    return {"small": small, "tiny": (wl, sigma, pins._dense_E(wl))}


def _run_pin(name, fixtures):
    fn = getattr(pins, name)
    params = list(inspect.signature(fn).parameters)
    fn(*[fixtures[p] for p in params])


def test_the_real_c_oracle_passes_the_pins_used_here(pin_fixtures):
    for name in OPERATOR_PINS + CG_PINS + X0_PINS + GRAD_PINS:
        _run_pin(name, pin_fixtures)


@pytest.mark.parametrize("name,pin_names,edits", C_CASES, ids=[c[0] for c in C_CASES])
def test_c_pins_reject_a_planted_mistake(name, pin_names, edits, pin_fixtures, repo_tmp,
                                         monkeypatch):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(om._SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    c_path = os.path.join(repo_tmp, "mutant.c")
    so_path = os.path.join(repo_tmp, "mutant.so")
    with open(c_path, "w") as fh:
        fh.write(src)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", c_path, "-o",
                    so_path, "-lm"], check=True)
    real = om.load()
    bad = ctypes.CDLL(so_path)
    for f in C_FUNCS:
        getattr(bad, f).argtypes = getattr(real, f).argtypes
        getattr(bad, f).restype = getattr(real, f).restype
    monkeypatch.setattr(om, "_lib", bad)
    caught = []
    for pin in pin_names:
        try:
            with np.errstate(all="ignore"):
                _run_pin(pin, pin_fixtures)
        except Exception:
            caught.append(pin)
    assert caught, f"no pin rejected: {name}"
