"""Thin Python binding of libsense (include/sense.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no arithmetic of
the method: all of E, E^H, E^H E and CG runs in the CUDA library. Arrays may be torch CUDA
tensors (device pointers, launched on the current torch stream) or host arrays (numpy /
CPU tensors; the library stages them). Complex arrays are complex64.

There is no fallback: if libsense.so is missing or fails to load, importing this module
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsense.so")

SENSE_PREC_FP32 = 0
SENSE_PREC_TC_FP16 = 1
SENSE_PREC_TC_SPLIT = 2
PRECISIONS = {"fp32": SENSE_PREC_FP32, "tc_fp16": SENSE_PREC_TC_FP16,
              "tc_split": SENSE_PREC_TC_SPLIT}

EXPORTED = ["sense_plan_create", "sense_plan_destroy", "sense_plan_set_b0", "sense_plan_info",
            "sense_encode", "sense_adjoint", "sense_normal_op", "sense_cg_solve",
            "sense_lcurve_corner", "sense_strerror", "sense_last_error", "sense_plan_profile",
            "sense_plan_stats", "sense_diag_sincos_rate", "sense_plan_get_tuning",
            "sense_plan_set_tuning", "sense_plan_sync", "sense_encode_noalloc",
            "sense_grad_b0", "sense_cg_ckpt_bytes", "sense_cg_solve_ckpt", "sense_cg_backward",
            "sense_batch_create", "sense_batch_destroy", "sense_batch_plan", "sense_batch_info",
            "sense_batch_normal_op", "sense_batch_cg_solve", "sense_batch_set_tuning",
            "sense_batch_autotune", "sense_cg_solve_iterates", "sense_kspace_filter_mask",
            "sense_kspace_filter", "sense_plan_store_p", "sense_smooth_map",
            "sense_kspace_filter_mask3d", "sense_smooth_sensitivities", "sense_diag_chunk_width",
            "sense_diag_stream_k_layout"]


class SenseError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.sense_strerror(code).decode()
        detail = _lib.sense_last_error().decode()
        super().__init__(f"{where}: {msg} ({code}){': ' + detail if detail else ''}")


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("timed", ctypes.c_int64 * 4),
                ("ms", ctypes.c_double * 4)]


KERNEL_CLASSES = ["tc_encode_pass", "tc_adjoint_pass", "fp32_encode", "fp32_adjoint"]


class Tuning(ctypes.Structure):
    _fields_ = [("seg_len", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("wait_limit_us", ctypes.c_int32), ("test_hold_stage", ctypes.c_int32),
                ("inner_chunk", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class _Problem(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("K", ctypes.c_int64), ("C", ctypes.c_int32),
                ("P1", ctypes.c_int32), ("Kmat", ctypes.c_void_p), ("Rmat", ctypes.c_void_p),
                ("S", ctypes.c_void_p), ("j", ctypes.c_void_p)]


class CGOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("rel_tol", ctypes.c_double), ("refine_every", ctypes.c_int32),
                ("apply_j", ctypes.c_int32), ("use_x0", ctypes.c_int32)]


class SmoothOpts(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("order", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("rel_tol", ctypes.c_double),
                ("precond", ctypes.c_int32), ("n_fields", ctypes.c_int32)]


class SmoothInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("rel_residual", ctypes.c_double)]


class CGInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rr0", ctypes.c_double), ("rr_final", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsense.so not built ({LIB_PATH}); run paper_2604_09233_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "sense_plan_create": ([ctypes.POINTER(_Problem), ctypes.POINTER(vp)], ctypes.c_int),
        "sense_plan_destroy": ([vp], ctypes.c_int),
        "sense_plan_set_b0": ([vp, vp, vp], ctypes.c_int),
        "sense_plan_info": ([vp, ctypes.POINTER(i64)], ctypes.c_int),
        "sense_encode": ([vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "sense_adjoint": ([vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "sense_normal_op": ([vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "sense_cg_solve": ([vp, vp, vp, ctypes.POINTER(CGOpts), vp, ctypes.POINTER(CGInfo), vp],
                           ctypes.c_int),
        "sense_lcurve_corner": ([vp, i32, ctypes.POINTER(i32)], ctypes.c_int),
        "sense_kspace_filter_mask": ([i32, i32, dbl, dbl, vp, vp, i64, vp], ctypes.c_int),
        "sense_kspace_filter": ([i32, i32, i32, vp, vp, vp], ctypes.c_int),
        "sense_kspace_filter_mask3d": ([i32, i32, i32, dbl, dbl, dbl, vp, vp, vp, i64, vp],
                                       ctypes.c_int),
        "sense_plan_store_p": ([vp, i32, vp], ctypes.c_int),
        "sense_smooth_map": ([ctypes.POINTER(SmoothOpts), vp, vp, vp, vp,
                              ctypes.POINTER(SmoothInfo), vp], ctypes.c_int),
        "sense_smooth_sensitivities": ([ctypes.POINTER(SmoothOpts), i32, vp, vp, vp, vp,
                                        ctypes.POINTER(SmoothInfo), vp], ctypes.c_int),
        "sense_cg_solve_iterates": ([vp, vp, vp, ctypes.POINTER(CGOpts), vp,
                                     ctypes.POINTER(CGInfo), vp], ctypes.c_int),
        "sense_plan_profile": ([vp, ctypes.c_int], ctypes.c_int),
        "sense_plan_sync": ([vp, vp], ctypes.c_int),
        "sense_encode_noalloc": ([i64, i64, i32, i32, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "sense_grad_b0": ([vp, i32, vp, vp, vp, vp, vp], ctypes.c_int),
        "sense_cg_ckpt_bytes": ([vp, i32, i32], i64),
        "sense_cg_solve_ckpt": ([vp, vp, vp, ctypes.POINTER(CGOpts), i32, vp, i64,
                                 ctypes.POINTER(CGInfo), vp], ctypes.c_int),
        "sense_cg_backward": ([vp, vp, vp, i64, vp, vp, vp, vp], ctypes.c_int),
        "sense_batch_create": ([ctypes.POINTER(_Problem), i32, ctypes.POINTER(vp)], ctypes.c_int),
        "sense_batch_destroy": ([vp], ctypes.c_int),
        "sense_batch_plan": ([vp, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "sense_batch_info": ([vp, ctypes.POINTER(i32)], ctypes.c_int),
        "sense_batch_normal_op": ([vp, i32, vp, vp, vp], ctypes.c_int),
        "sense_batch_cg_solve": ([vp, vp, vp, ctypes.POINTER(CGOpts), ctypes.POINTER(CGInfo), vp],
                                 ctypes.c_int),
        "sense_batch_set_tuning": ([vp, i32, i32], ctypes.c_int),
        "sense_batch_autotune": ([vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                  ctypes.POINTER(dbl)], ctypes.c_int),
        "sense_plan_get_tuning": ([vp, ctypes.POINTER(Tuning)], ctypes.c_int),
        "sense_plan_set_tuning": ([vp, ctypes.POINTER(Tuning)], ctypes.c_int),
        "sense_plan_stats": ([vp, ctypes.POINTER(Stats)], ctypes.c_int),
        "sense_diag_sincos_rate": ([dbl, ctypes.POINTER(dbl)], ctypes.c_int),
        "sense_diag_chunk_width": ([i64, i64, i32, i32, ctypes.POINTER(i64)], ctypes.c_int),
        "sense_diag_stream_k_layout": ([i64, i64, i64, i32, vp, vp, ctypes.POINTER(i32)],
                                       ctypes.c_int),
        "sense_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "sense_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def _check(rc, where):
    if rc != 0:
        raise SenseError(rc, where)


def _ptr(a, dtype=np.complex64):
    """(pointer, keepalive, stream) for a torch tensor or numpy array (no copies of device data)."""
    if a is None:
        return None, None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            want = {np.complex64: torch.complex64, np.float64: torch.float64,
                    np.float32: torch.float32, np.uint8: torch.uint8}[dtype]
            if a.dtype != want:
                raise TypeError(f"expected {want}, got {a.dtype}")
            stream = torch.cuda.current_stream(a.device).cuda_stream if a.is_cuda else None
            return a.data_ptr(), a, stream
    except ImportError:
        pass
    arr = np.asarray(a)
    if arr.dtype != dtype or not arr.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
    return arr.ctypes.data, arr, None


def _stream(*streams, explicit=None):
    if explicit is not None:
        return explicit
    for s in streams:
        if s is not None:
            return s
    return None


def sense_plan_create(Kmat, Rmat, S, j=None):
    """Create a plan from host arrays Kmat [K][P1], Rmat [P1][L] (float64), S [L][C]
    (complex64), j [L] (float32 or None). Returns an opaque handle (int)."""
    Kmat = np.ascontiguousarray(Kmat, np.float64)
    Rmat = np.ascontiguousarray(Rmat, np.float64)
    S = np.ascontiguousarray(S, np.complex64)
    jj = None if j is None else np.ascontiguousarray(j, np.float32)
    K, P1 = Kmat.shape
    L = Rmat.shape[1]
    if Rmat.shape[0] != P1 or S.shape[0] != L or (jj is not None and jj.shape != (L,)):
        raise ValueError("inconsistent shapes")
    prob = _Problem(L, K, S.shape[1], P1, Kmat.ctypes.data, Rmat.ctypes.data, S.ctypes.data,
                    None if jj is None else jj.ctypes.data)
    h = ctypes.c_void_p()
    _check(_lib.sense_plan_create(ctypes.byref(prob), ctypes.byref(h)), "sense_plan_create")
    return h.value


def sense_plan_destroy(plan):
    _check(_lib.sense_plan_destroy(plan), "sense_plan_destroy")


def sense_plan_set_b0(plan, omega, stream=None):
    om = np.ascontiguousarray(omega, np.float64)
    _check(_lib.sense_plan_set_b0(plan, om.ctypes.data, stream), "sense_plan_set_b0")


def sense_plan_info(plan):
    out = (ctypes.c_int64 * 8)()
    _check(_lib.sense_plan_info(plan, out), "sense_plan_info")
    keys = ["L", "K", "C", "P1", "rows_kept", "L_padded", "K_padded", "C_padded"]
    return dict(zip(keys, list(out)))


def sense_encode(plan, prec, m, s, stream=None):
    pm, km, sm = _ptr(m)
    ps, ks, ss = _ptr(s)
    _check(_lib.sense_encode(plan, int(prec), pm, ps, _stream(sm, ss, explicit=stream)),
           "sense_encode")


def sense_adjoint(plan, prec, s, m, stream=None):
    ps, ks, ss = _ptr(s)
    pm, km, sm = _ptr(m)
    _check(_lib.sense_adjoint(plan, int(prec), ps, pm, _stream(ss, sm, explicit=stream)),
           "sense_adjoint")


def sense_normal_op(plan, prec, m, out, stream=None):
    pm, km, sm = _ptr(m)
    po, ko, so = _ptr(out)
    _check(_lib.sense_normal_op(plan, int(prec), pm, po, _stream(sm, so, explicit=stream)),
           "sense_normal_op")


def sense_cg_solve(plan, s, x, max_iter, prec=SENSE_PREC_FP32, rel_tol=0.0, refine_every=0,
                   apply_j=True, history=True, stream=None, use_x0=False):
    """Returns (info dict, history array [iters+1][3] or None). use_x0: x holds the start."""
    ps, ks, ss = _ptr(s)
    px, kx, sx = _ptr(x)
    opts = CGOpts(int(max_iter), int(prec), float(rel_tol), int(refine_every),
                  1 if apply_j else 0, 1 if use_x0 else 0)
    info = CGInfo()
    hist = np.full((int(max_iter) + 1, 3), np.nan) if history else None
    _check(_lib.sense_cg_solve(plan, ps, px, ctypes.byref(opts),
                               None if hist is None else hist.ctypes.data, ctypes.byref(info),
                               _stream(ss, sx, explicit=stream)), "sense_cg_solve")
    out = dict(iters=info.iters, status=info.status, rr0=info.rr0, rr_final=info.rr_final)
    return out, (None if hist is None else hist[: info.iters + 1])


def sense_cg_solve_iterates(plan, s, iterates, max_iter, prec=SENSE_PREC_FP32, rel_tol=0.0,
                            refine_every=0, apply_j=True, stream=None, use_x0=False):
    """CG recording every iterate into iterates ([max_iter+1][L] complex64 CUDA tensor;
    with use_x0 row 0 holds the start on input). Returns (info dict, history [iters+1][3])."""
    ps, _, ss = _ptr(s)
    pX, _, sX = _ptr(iterates)
    opts = CGOpts(int(max_iter), int(prec), float(rel_tol), int(refine_every),
                  1 if apply_j else 0, 1 if use_x0 else 0)
    info = CGInfo()
    hist = np.full((int(max_iter) + 1, 3), np.nan)
    _check(_lib.sense_cg_solve_iterates(plan, ps, pX, ctypes.byref(opts), hist.ctypes.data,
                                        ctypes.byref(info), _stream(ss, sX, explicit=stream)),
           "sense_cg_solve_iterates")
    out = dict(iters=info.iters, status=info.status, rr0=info.rr0, rr_final=info.rr_final)
    return out, hist[: info.iters + 1]


def sense_plan_store_p(plan, enable=True, stream=None):
    """Stored-P mode on (precomputed phase tiles streamed from HBM) or off."""
    _check(_lib.sense_plan_store_p(plan, 1 if enable else 0, stream), "sense_plan_store_p")


SMOOTH_PRECOND = {"none": 0, "multigrid": 1}


def _smooth_opts(shape, order, alpha, max_iter, rel_tol, precond, n_fields):
    nz, ny, nx = (1,) + tuple(shape) if len(shape) == 2 else tuple(shape)
    pc = SMOOTH_PRECOND[precond] if isinstance(precond, str) else int(precond)
    return SmoothOpts(int(nx), int(ny), int(nz), int(order), float(alpha), int(max_iter),
                      float(rel_tol), pc, int(n_fields))


def sense_smooth_map(shape, order, alpha, w0, wd, xhat, x, max_iter=2000, rel_tol=1e-7,
                     precond="multigrid", stream=None):
    """Eq. 1 (order 2) / Eq. 3 (order 1) smoothing on a grid of `shape` ((ny, nx) or
    (nz, ny, nx)); w0, wd float32 and xhat, x complex64 CUDA tensors, [n] for one field or
    [F][n] for F fields solved together; precond "multigrid" (V-cycle preconditioned CG) or
    "none" (plain CG). Returns the info dict (one field) or a list of them."""
    n = int(np.prod(shape))
    F = 1 if xhat.ndim == 1 else int(xhat.shape[0])
    if xhat.numel() != F * n or x.numel() != F * n:
        raise ValueError("xhat and x must hold n_fields x prod(shape) values")
    o = _smooth_opts(shape, order, alpha, max_iter, rel_tol, precond, F)
    info = (SmoothInfo * F)()
    p0, _, s0 = _ptr(w0, np.float32)
    p1, _, _ = _ptr(wd, np.float32)
    p2, _, _ = _ptr(xhat)
    p3, _, _ = _ptr(x)
    _check(_lib.sense_smooth_map(ctypes.byref(o), p0, p1, p2, p3, info,
                                 _stream(s0, explicit=stream)), "sense_smooth_map")
    out = [{"iters": i.iters, "rel_residual": i.rel_residual} for i in info]
    return out[0] if xhat.ndim == 1 else out


def sense_smooth_sensitivities(shape, alpha, m_t, m_r, S_hat, S, max_iter=2000, rel_tol=1e-7,
                               precond="multigrid", stream=None):
    """Eq. 1 on every coil's sensitivity map: magnitude and magnitude-normalised map smoothed
    separately (2 C fields in one solve) and recombined. m_t (trusted mask), m_r
    (reconstruction mask): float32 [n]; S_hat, S: complex64 [n][C] CUDA tensors (may be the
    same tensor). Returns the per-field info dicts (magnitudes first)."""
    n = int(np.prod(shape))
    C = int(S_hat.shape[-1])
    if S_hat.numel() != n * C or S.numel() != n * C:
        raise ValueError("S_hat and S must be [prod(shape)][C]")
    o = _smooth_opts(shape, 2, alpha, max_iter, rel_tol, precond, 2 * C)
    info = (SmoothInfo * (2 * C))()
    p0, _, s0 = _ptr(m_t, np.float32)
    p1, _, _ = _ptr(m_r, np.float32)
    p2, _, _ = _ptr(S_hat)
    p3, _, _ = _ptr(S)
    _check(_lib.sense_smooth_sensitivities(ctypes.byref(o), C, p0, p1, p2, p3, info,
                                           _stream(s0, explicit=stream)),
           "sense_smooth_sensitivities")
    return [{"iters": i.iters, "rel_residual": i.rel_residual} for i in info]


def sense_kspace_filter_mask(nx, ny, dx, dy, kx, ky):
    """Convex-hull k-space filter [ny][nx] (float32 numpy) from first-order coefficients."""
    kx = np.ascontiguousarray(kx, np.float64)
    ky = np.ascontiguousarray(ky, np.float64)
    if kx.shape != ky.shape:
        raise ValueError("kx and ky differ in shape")
    mask = np.empty((int(ny), int(nx)), np.float32)
    _check(_lib.sense_kspace_filter_mask(int(nx), int(ny), float(dx), float(dy), kx.ctypes.data,
                                         ky.ctypes.data, int(kx.size), mask.ctypes.data),
           "sense_kspace_filter_mask")
    return mask


def sense_kspace_filter_mask3d(nx, ny, nz, dx, dy, dz, kx, ky, kz):
    """Convex-hull k-space filter [nz][ny][nx] (float32 numpy) for a stack of planar
    trajectories."""
    k = [np.ascontiguousarray(a, np.float64) for a in (kx, ky, kz)]
    if not (k[0].shape == k[1].shape == k[2].shape):
        raise ValueError("kx, ky, kz differ in shape")
    mask = np.empty((int(nz), int(ny), int(nx)), np.float32)
    _check(_lib.sense_kspace_filter_mask3d(int(nx), int(ny), int(nz), float(dx), float(dy),
                                           float(dz), k[0].ctypes.data, k[1].ctypes.data,
                                           k[2].ctypes.data, int(k[0].size), mask.ctypes.data),
           "sense_kspace_filter_mask3d")
    return mask


def sense_kspace_filter(image, mask, shape, stream=None):
    """Filter a complex64 CUDA image of `shape` ((ny, nx) or (nz, ny, nx)) in place with a
    float32 CUDA mask of the same shape."""
    nz, ny, nx = (1,) + tuple(shape) if len(shape) == 2 else tuple(shape)
    pi, _, si = _ptr(image)
    pm, _, _ = _ptr(mask, np.float32)
    _check(_lib.sense_kspace_filter(int(nx), int(ny), int(nz), pm, pi,
                                    _stream(si, explicit=stream)), "sense_kspace_filter")


def sense_encode_noalloc(Kmat, Rmat, S, m, s, j=None, stream=None):
    """s = E m without any device allocation by the library (see include/sense.h). All
    arrays are CUDA tensors: Kmat [K][P1] float64, Rmat [P1][L] float64, S [L][C]
    complex64, m [L] complex64, s [K][C] complex64 (output), j [L] float32 or None."""
    K, P1 = Kmat.shape
    L = Rmat.shape[1]
    C = S.shape[1]
    pk, _, sk = _ptr(Kmat, np.float64)
    pr, _, _ = _ptr(Rmat, np.float64)
    pS, _, _ = _ptr(S)
    pm, _, _ = _ptr(m)
    ps, _, _ = _ptr(s)
    pj = None if j is None else _ptr(j, np.float32)[0]
    _check(_lib.sense_encode_noalloc(int(L), int(K), int(C), int(P1), pk, pr, pS, pj, pm, ps,
                                     _stream(sk, explicit=stream)), "sense_encode_noalloc")


def sense_grad_b0(plan, prec, a, y, grad_omega, z=None, stream=None):
    """grad_omega = Im(conj(a) * E^H(t o y)) ([L] float32) and, if z is given, z = E^H y."""
    pa, _, sa = _ptr(a)
    py, _, sy = _ptr(y)
    pg, _, sg = _ptr(grad_omega, np.float32)
    pz, _, _ = _ptr(z)
    _check(_lib.sense_grad_b0(plan, int(prec), pa, py, pz, pg,
                              _stream(sa, sy, sg, explicit=stream)), "sense_grad_b0")


def sense_cg_ckpt_bytes(plan, max_iter, ckpt_every):
    n = _lib.sense_cg_ckpt_bytes(plan, int(max_iter), int(ckpt_every))
    if n < 0:
        raise SenseError(int(n), "sense_cg_ckpt_bytes")
    return int(n)


def sense_cg_solve_ckpt(plan, s, x, ckpt, max_iter, ckpt_every, prec=SENSE_PREC_FP32,
                        rel_tol=0.0, apply_j=True, stream=None):
    """CG solve that records checkpoints into ckpt (a uint8 CUDA tensor of at least
    sense_cg_ckpt_bytes bytes). Returns the info dict."""
    ps, _, ss = _ptr(s)
    px, _, sx = _ptr(x)
    pc, kc, _ = _ptr(ckpt, np.uint8)
    opts = CGOpts(int(max_iter), int(prec), float(rel_tol), 0, 1 if apply_j else 0, 0)
    info = CGInfo()
    _check(_lib.sense_cg_solve_ckpt(plan, ps, px, ctypes.byref(opts), int(ckpt_every), pc,
                                    int(kc.numel()), ctypes.byref(info),
                                    _stream(ss, sx, explicit=stream)), "sense_cg_solve_ckpt")
    return dict(iters=info.iters, status=info.status, rr0=info.rr0, rr_final=info.rr_final)


def sense_cg_backward(plan, s, ckpt, xbar, sbar=None, omega_bar=None, stream=None):
    """Reverse mode through the solve recorded in ckpt: sbar = dL/ds, omega_bar = dL/domega."""
    ps, _, ss = _ptr(s)
    pc, kc, _ = _ptr(ckpt, np.uint8)
    pxb, _, sxb = _ptr(xbar)
    psb, _, _ = _ptr(sbar)
    pwb, _, _ = _ptr(omega_bar, np.float32)
    _check(_lib.sense_cg_backward(plan, ps, pc, int(kc.numel()), pxb, psb, pwb,
                                  _stream(ss, sxb, explicit=stream)), "sense_cg_backward")


def _problem_struct(Kmat, Rmat, S, j, keep):
    Kmat = np.ascontiguousarray(Kmat, np.float64)
    Rmat = np.ascontiguousarray(Rmat, np.float64)
    S = np.ascontiguousarray(S, np.complex64)
    jj = None if j is None else np.ascontiguousarray(j, np.float32)
    K, P1 = Kmat.shape
    L = Rmat.shape[1]
    if Rmat.shape[0] != P1 or S.shape[0] != L or (jj is not None and jj.shape != (L,)):
        raise ValueError("inconsistent shapes")
    keep.extend([Kmat, Rmat, S, jj])
    return _Problem(L, K, S.shape[1], P1, Kmat.ctypes.data, Rmat.ctypes.data, S.ctypes.data,
                    None if jj is None else jj.ctypes.data)


def sense_batch_create(problems):
    """problems: sequence of (Kmat, Rmat, S, j). Returns an opaque batch handle (int)."""
    keep = []
    arr = (_Problem * len(problems))(*[_problem_struct(*p, keep) for p in problems])
    h = ctypes.c_void_p()
    _check(_lib.sense_batch_create(arr, len(problems), ctypes.byref(h)), "sense_batch_create")
    return h.value


def sense_batch_destroy(batch):
    _check(_lib.sense_batch_destroy(batch), "sense_batch_destroy")


def sense_batch_plan(batch, i):
    h = ctypes.c_void_p()
    _check(_lib.sense_batch_plan(batch, int(i), ctypes.byref(h)), "sense_batch_plan")
    return h.value


def sense_batch_info(batch):
    out = (ctypes.c_int32 * 4)()
    _check(_lib.sense_batch_info(batch, out), "sense_batch_info")
    return dict(zip(["n", "C_padded", "delta_rows", "chunk"], list(out)))


def _ptr_array(tensors):
    ptrs = [_ptr(t)[0] for t in tensors]
    return (ctypes.c_void_p * len(ptrs))(*ptrs)


def sense_batch_normal_op(batch, prec, m_list, out_list, stream=None):
    """out_list[b] = E_b^H E_b m_list[b] (complex64 CUDA tensors)."""
    st = stream if stream is not None else _ptr(m_list[0])[2]
    _check(_lib.sense_batch_normal_op(batch, int(prec), _ptr_array(m_list), _ptr_array(out_list),
                                      st), "sense_batch_normal_op")


def sense_batch_cg_solve(batch, s_list, x_list, max_iter, prec=SENSE_PREC_TC_SPLIT, rel_tol=0.0,
                         apply_j=True, stream=None):
    """CG for every instance (device tensors); returns the list of info dicts."""
    n = len(s_list)
    opts = CGOpts(int(max_iter), int(prec), float(rel_tol), 0, 1 if apply_j else 0, 0)
    infos = (CGInfo * n)()
    st = stream if stream is not None else _ptr(s_list[0])[2]
    _check(_lib.sense_batch_cg_solve(batch, _ptr_array(s_list), _ptr_array(x_list),
                                     ctypes.byref(opts), infos, st), "sense_batch_cg_solve")
    return [dict(iters=i.iters, status=i.status, rr0=i.rr0, rr_final=i.rr_final) for i in infos]


def sense_batch_set_tuning(batch, chunk=16, seg_len=4):
    _check(_lib.sense_batch_set_tuning(batch, int(chunk), int(seg_len)), "sense_batch_set_tuning")


def sense_batch_autotune(batch, prec=SENSE_PREC_TC_SPLIT):
    c, s, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(_lib.sense_batch_autotune(batch, int(prec), ctypes.byref(c), ctypes.byref(s),
                                     ctypes.byref(ms)), "sense_batch_autotune")
    return {"chunk": c.value, "seg_len": s.value, "ms": ms.value}


class Batch:
    """Owns a libsense batch of independent problems (sequence of (Kmat, Rmat, S, j))."""

    def __init__(self, problems):
        self.handle = sense_batch_create(problems)
        self.n = len(problems)
        self.dims = []
        for i in range(self.n):
            inf = sense_plan_info(sense_batch_plan(self.handle, i))
            self.dims.append((inf["L"], inf["K"], inf["C"]))

    def close(self):
        if self.handle:
            sense_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def normal(self, ms, prec=SENSE_PREC_TC_SPLIT):
        import torch
        outs = [torch.empty_like(m) for m in ms]
        sense_batch_normal_op(self.handle, prec, ms, outs)
        torch.cuda.synchronize()
        return outs

    def cg(self, ss, max_iter, prec=SENSE_PREC_TC_SPLIT, rel_tol=0.0, apply_j=True):
        import torch
        xs = [torch.empty(L, dtype=torch.complex64, device=s.device)
              for s, (L, _, _) in zip(ss, self.dims)]
        infos = sense_batch_cg_solve(self.handle, ss, xs, max_iter, prec, rel_tol, apply_j)
        return xs, infos


def sense_plan_sync(plan, stream=None):
    """Synchronise and raise SenseError if a device-side failure was recorded."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
    _check(_lib.sense_plan_sync(plan, stream), "sense_plan_sync")


def sense_plan_get_tuning(plan):
    t = Tuning()
    _check(_lib.sense_plan_get_tuning(plan, ctypes.byref(t)), "sense_plan_get_tuning")
    return {"seg_len": t.seg_len, "grid": t.grid, "wait_limit_us": t.wait_limit_us,
            "test_hold_stage": t.test_hold_stage, "inner_chunk": t.inner_chunk}


def sense_plan_set_tuning(plan, seg_len=0, grid=0, wait_limit_us=0, test_hold_stage=0,
                          inner_chunk=0):
    t = Tuning(int(seg_len), int(grid), int(wait_limit_us), int(test_hold_stage),
               int(inner_chunk))
    _check(_lib.sense_plan_set_tuning(plan, ctypes.byref(t)), "sense_plan_set_tuning")


def sense_plan_profile(plan, enable=True):
    _check(_lib.sense_plan_profile(plan, 1 if enable else 0), "sense_plan_profile")


def sense_plan_stats(plan):
    """dict(launches, per-class dict(n=timed launches, ms=summed event time))."""
    st = Stats()
    _check(_lib.sense_plan_stats(plan, ctypes.byref(st)), "sense_plan_stats")
    out = {"launches": st.launches}
    for i, name in enumerate(KERNEL_CLASSES):
        out[name] = {"n": st.timed[i], "ms": st.ms[i]}
    return out


def sense_diag_sincos_rate(ms_budget=200.0):
    v = ctypes.c_double()
    _check(_lib.sense_diag_sincos_rate(float(ms_budget), ctypes.byref(v)),
           "sense_diag_sincos_rate")
    return v.value


def sense_diag_chunk_width(n_outer, n_inner, cp, g):
    """Streamed blocks per stream-K chunk of a tensor-core pass (host only)."""
    w = ctypes.c_int64()
    _check(_lib.sense_diag_chunk_width(int(n_outer), int(n_inner), int(cp), int(g),
                                       ctypes.byref(w)), "sense_diag_chunk_width")
    return w.value


def sense_diag_stream_k_layout(n_outer, n_inner, chunk, g):
    """Slot bases [chunks][n_outer], slots per row block and the largest slot count of the
    chunked stream-K schedule (host only)."""
    nch = (int(n_inner) + int(chunk) - 1) // int(chunk)
    base = np.zeros((nch, int(n_outer)), np.int32)
    nslot = np.zeros(int(n_outer), np.int32)
    mx = ctypes.c_int32()
    _check(_lib.sense_diag_stream_k_layout(int(n_outer), int(n_inner), int(chunk), int(g),
                                           base.ctypes.data, nslot.ctypes.data,
                                           ctypes.byref(mx)), "sense_diag_stream_k_layout")
    return base, nslot, mx.value


def sense_strerror(code):
    return _lib.sense_strerror(int(code)).decode()


def sense_last_error():
    return _lib.sense_last_error().decode()


def sense_lcurve_corner(history):
    h = np.ascontiguousarray(history, np.float64)
    c = ctypes.c_int32()
    _check(_lib.sense_lcurve_corner(h.ctypes.data, int(h.shape[0]), ctypes.byref(c)),
           "sense_lcurve_corner")
    return c.value


class Plan:
    """Owns a libsense plan; methods allocate outputs and call the C entry points."""

    def __init__(self, Kmat, Rmat, S, j=None):
        self.handle = sense_plan_create(Kmat, Rmat, S, j)
        info = sense_plan_info(self.handle)
        self.L, self.K, self.C = info["L"], info["K"], info["C"]
        self.info = info

    def close(self):
        if self.handle:
            sense_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def encode(self, m, prec=SENSE_PREC_FP32):
        import torch
        s = torch.empty((self.K, self.C), dtype=torch.complex64, device=m.device)
        sense_encode(self.handle, prec, m, s)
        sense_plan_sync(self.handle)
        return s

    def adjoint(self, s, prec=SENSE_PREC_FP32):
        import torch
        m = torch.empty((self.L,), dtype=torch.complex64, device=s.device)
        sense_adjoint(self.handle, prec, s, m)
        sense_plan_sync(self.handle)
        return m

    def normal(self, m, prec=SENSE_PREC_FP32):
        import torch
        out = torch.empty((self.L,), dtype=torch.complex64, device=m.device)
        sense_normal_op(self.handle, prec, m, out)
        sense_plan_sync(self.handle)
        return out

    def cg(self, s, max_iter, prec=SENSE_PREC_FP32, rel_tol=0.0, refine_every=0, apply_j=True,
           x0=None):
        """CG from rho = 0, or from x0 ([L] complex64 tensor, the start before the final
        multiplication by j) when given."""
        import torch
        if x0 is None:
            x = torch.empty((self.L,), dtype=torch.complex64, device=s.device)
        else:
            x = x0.detach().to(device=s.device, dtype=torch.complex64).clone().contiguous()
        info, hist = sense_cg_solve(self.handle, s, x, max_iter, prec, rel_tol, refine_every,
                                    apply_j, use_x0=x0 is not None)
        sense_plan_sync(self.handle)
        return x, info, hist
