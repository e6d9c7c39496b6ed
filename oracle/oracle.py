"""ctypes loader and numpy marshalling for the FP64 oracle (``sense_oracle.c``).

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sense_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile sense_oracle.c with gcc into liboracle.so (OpenMP, -O2, no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.or_num_threads.restype = _int
        lib.or_set_num_threads.argtypes = [_int]
        lib.or_encode.argtypes = [_i64, _i64, _int, _int, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr,
                                  _i64, _ptr]
        lib.or_adjoint.argtypes = [_i64, _i64, _int, _int, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr,
                                   _i64, _ptr]
        lib.or_normal.argtypes = [_i64, _i64, _int, _int, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr,
                                  _ptr]
        lib.or_cg.argtypes = [_i64, _i64, _int, _int, _ptr, _ptr, _ptr, _ptr, _ptr, _int, _dbl,
                              _int, _ptr, _ptr, _ptr, _ptr]
        lib.or_cg.restype = _int
        lib.or_grad_omega.argtypes = [_i64, _i64, _int, _int, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr,
                                      _ptr]
        lib.or_grad_omega_adjoint.argtypes = [_i64, _i64, _int, _int, _ptr, _ptr, _ptr, _ptr,
                                              _ptr, _ptr, _ptr]
        _lib = lib
        return lib


def num_threads() -> int:
    return int(load().or_num_threads())


def set_num_threads(n: int) -> None:
    load().or_set_num_threads(int(n))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _geom(Kmat, Rmat, S, j):
    Kmat = _c(Kmat, np.float64)
    Rmat = _c(Rmat, np.float64)
    S = _c(S, np.complex128)
    K, P1 = Kmat.shape
    P1b, L = Rmat.shape
    if P1b != P1:
        raise ValueError("K has %d columns but R has %d rows" % (P1, P1b))
    if S.shape[0] != L:
        raise ValueError("S must be [L][C]")
    jj = None if j is None else _c(j, np.float64)
    if jj is not None and jj.shape != (L,):
        raise ValueError("j must be [L]")
    return Kmat, Rmat, S, jj, L, K, S.shape[1], P1


def encode(Kmat, Rmat, S, m, j=None, rows=None):
    """s = E m (Eq. 4); rows selects sample indices (default all)."""
    Kmat, Rmat, S, jj, L, K, C, P1 = _geom(Kmat, Rmat, S, j)
    m = _c(m, np.complex128)
    if rows is None:
        r, n = None, K
    else:
        r = _c(rows, np.int64)
        n = r.shape[0]
    out = np.empty((n, C), np.complex128)
    load().or_encode(L, K, C, P1, _p(Kmat), _p(Rmat), _p(S), _p(jj), _p(m), _p(r), n, _p(out))
    return out


def adjoint(Kmat, Rmat, S, s, j=None, vox=None):
    """m = E^H s (Eq. 5); vox selects voxel indices (default all)."""
    Kmat, Rmat, S, jj, L, K, C, P1 = _geom(Kmat, Rmat, S, j)
    s = _c(s, np.complex128).reshape(K, C)
    if vox is None:
        v, n = None, L
    else:
        v = _c(vox, np.int64)
        n = v.shape[0]
    out = np.empty(n, np.complex128)
    load().or_adjoint(L, K, C, P1, _p(Kmat), _p(Rmat), _p(S), _p(jj), _p(s), _p(v), n, _p(out))
    return out


def normal(Kmat, Rmat, S, m, j=None):
    """E^H E m."""
    Kmat, Rmat, S, jj, L, K, C, P1 = _geom(Kmat, Rmat, S, j)
    m = _c(m, np.complex128)
    out = np.empty(L, np.complex128)
    work = np.empty(K * C, np.complex128)
    load().or_normal(L, K, C, P1, _p(Kmat), _p(Rmat), _p(S), _p(jj), _p(m), _p(out), _p(work))
    return out


def cg(Kmat, Rmat, S, sigma, n_it, j=None, rel_tol=0.0, apply_j=True, history=False,
       iterates=False, x0=None):
    """The CG loop of Alg. 1 (Fig. 2). Returns dict(x, iters, history?, iterates?).

    x0: optional start rho_0 ([L], the iterate before the final multiplication by j);
    Alg. 1 starts from rho_0 = 0. rel_tol stops once ||r_n|| <= rel_tol ||E^H sigma||."""
    Kmat, Rmat, S, jj, L, K, C, P1 = _geom(Kmat, Rmat, S, j)
    sigma = _c(sigma, np.complex128).reshape(K, C)
    rho = np.empty(L, np.complex128)
    hist = np.full((n_it + 1, 3), np.nan) if history else None
    its = np.zeros((n_it + 1, L), np.complex128) if iterates else None
    xs = None if x0 is None else _c(x0, np.complex128)
    if xs is not None and xs.shape != (L,):
        raise ValueError("x0 must be [L]")
    n = load().or_cg(L, K, C, P1, _p(Kmat), _p(Rmat), _p(S), _p(jj), _p(sigma), int(n_it),
                     float(rel_tol), 1 if apply_j else 0, _p(xs), _p(rho), _p(hist), _p(its))
    out = {"x": rho, "iters": int(n)}
    if history:
        out["history"] = hist[: n + 1]
    if iterates:
        out["iterates"] = its[: n + 1]
    return out


def grad_omega(Kmat, Rmat, S, m, g, j=None):
    """d Loss / d R[0,:] given g = dLoss/dRe(Em) + i dLoss/dIm(Em)."""
    Kmat, Rmat, S, jj, L, K, C, P1 = _geom(Kmat, Rmat, S, j)
    m = _c(m, np.complex128)
    g = _c(g, np.complex128).reshape(K, C)
    out = np.empty(L, np.float64)
    load().or_grad_omega(L, K, C, P1, _p(Kmat), _p(Rmat), _p(S), _p(jj), _p(m), _p(g),
                         _p(out))
    return out


def grad_omega_adjoint(Kmat, Rmat, S, y, h, j=None):
    """d Loss / d R[0,:] through x = E^H y, given h = dLoss/dRe(x) + i dLoss/dIm(x)."""
    Kmat, Rmat, S, jj, L, K, C, P1 = _geom(Kmat, Rmat, S, j)
    y = _c(y, np.complex128).reshape(K, C)
    h = _c(h, np.complex128)
    out = np.empty(L, np.float64)
    load().or_grad_omega_adjoint(L, K, C, P1, _p(Kmat), _p(Rmat), _p(S), _p(jj), _p(y), _p(h),
                                 _p(out))
    return out


def smooth_map(shape, order, alpha, w0, wd, xhat):
    """Least-squares solution of Eq. 1 (order 2, second differences; w0 = M_T, wd = M_R) or
    Eq. 3 (order 1, first differences; w0 = 1, wd = the fit's standard error):
    A x = [w0 o xhat; 0; 0; 0], A = [diag(w0); sqrt(alpha) diag(wd) D_x; ... D_y; ... D_z],
    with the sparse A written out row by row (second-difference rows at interior voxels, first-
    difference rows where the next voxel exists, weight wd at the row's voxel) and the normal
    equations solved directly; voxels that no equation constrains keep xhat. shape: (ny, nx)
    or (nz, ny, nx); x fastest."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    shape = tuple(shape)
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    w0 = np.asarray(w0, float).ravel()
    wd = np.asarray(wd, float).ravel()
    blocks = [sp.diags(w0)]
    for ax in range(len(shape)):
        m = shape[ax]
        if m < 2:
            continue
        rows, cols, vals = [], [], []
        sl = np.moveaxis(idx, ax, -1).reshape(-1, m)
        r = 0
        for line in sl:
            if order == 1:
                for c in range(m - 1):
                    rows += [r, r]
                    cols += [line[c], line[c + 1]]
                    vals += [-wd[line[c]], wd[line[c]]]
                    r += 1
            else:
                for c in range(1, m - 1):
                    rows += [r, r, r]
                    cols += [line[c - 1], line[c], line[c + 1]]
                    vals += [wd[line[c]], -2 * wd[line[c]], wd[line[c]]]
                    r += 1
        blocks.append(np.sqrt(alpha) * sp.csr_matrix((vals, (rows, cols)), shape=(r, n)))
    A = sp.vstack(blocks).tocsc()
    rhs = np.concatenate([w0 * np.asarray(xhat, complex).ravel(),
                          np.zeros(A.shape[0] - n, complex)])
    N = (A.T @ A).tocsc()
    # voxels that no equation constrains (outside the data and derivative weights) keep xhat
    x = np.asarray(xhat, complex).ravel().copy()
    keep = N.diagonal() > 0
    if keep.any():
        x[keep] = spl.spsolve(N[keep][:, keep].tocsc(), (A.T @ rhs)[keep])
    return x


def smooth_sensitivities(shape, alpha, m_t, m_r, S_hat):
    """Sensitivity maps by Eq. 1 as the paper applies it: for every coil the magnitude of
    S_hat and the magnitude-normalised S_hat (0 where S_hat = 0) are smoothed separately (w0 =
    M_T, wd = M_R, second differences) and recombined as S = m u / |u| (0 where u = 0).
    S_hat: [n][C] complex; returns [n][C]."""
    S_hat = np.asarray(S_hat, complex)
    n, C = S_hat.shape
    out = np.zeros((n, C), complex)
    for c in range(C):
        mag = np.abs(S_hat[:, c])
        unit = np.where(mag > 0, S_hat[:, c] / np.where(mag > 0, mag, 1.0), 0.0)
        m = smooth_map(shape, 2, alpha, m_t, m_r, mag.astype(complex)).real
        u = smooth_map(shape, 2, alpha, m_t, m_r, unit)
        a = np.abs(u)
        out[:, c] = np.where(a > 0, m * u / np.where(a > 0, a, 1.0), 0.0)
    return out


def kspace_mask(nx, ny, dx, dy, kx, ky):
    """k-space filter of the paper's k-space filter section: 1 for the Cartesian k-space
    points 2 pi (u - n/2) / (n d) that lie in a triangle of the Delaunay triangulation of the
    first-order k-space coordinates (kx, ky), else 0 ([ny][nx])."""
    from scipy.spatial import Delaunay
    tri = Delaunay(np.stack([np.asarray(kx, float), np.asarray(ky, float)], axis=1))
    u = 2 * np.pi * (np.arange(nx) - nx // 2) / (nx * dx)
    v = 2 * np.pi * (np.arange(ny) - ny // 2) / (ny * dy)
    U, V = np.meshgrid(u, v)
    inside = tri.find_simplex(np.stack([U.ravel(), V.ravel()], axis=1)) >= 0
    return inside.reshape(ny, nx).astype(np.float64)


def kspace_filter(image, shape, mask):
    """rho <- IFFT(FFT(rho) o f) (the filtering that ends Alg. 1, Fig. 2) with the signal model's sign along every
    axis: F(k_u) = sum_x rho(x) e^{+i 2 pi (u - n/2)(x - n/2) / n}, then
    rho(x) = (1/n) sum_u F(k_u) f(u) e^{-i 2 pi (u - n/2)(x - n/2) / n}, written out as dense
    matrices (shape: (ny, nx) or (nz, ny, nx))."""
    x = np.asarray(image, np.complex128).reshape(shape)
    f = np.asarray(mask, np.float64).reshape(shape)

    def W(n, sgn):
        c = np.arange(n) - n // 2
        return np.exp(sgn * 2j * np.pi * np.outer(c, c) / n)

    for ax, n in enumerate(shape):
        x = np.moveaxis(np.tensordot(W(n, +1), np.moveaxis(x, ax, 0), axes=(1, 0)), 0, ax)
    x = x * f
    for ax, n in enumerate(shape):
        x = np.moveaxis(np.tensordot(W(n, -1), np.moveaxis(x, ax, 0), axes=(1, 0)) / n, 0, ax)
    return x.ravel()


def lcurve_corner(res_norm, sol_norm):
    """Iteration n of maximum L-curve curvature.

    res_norm[n], sol_norm[n] are ||E x_n - s|| and ||x_n|| for n = 0..N (the rows of a CG
    history). The L-curve is the parametric curve (a, b) = (log ||E x_n - s||, log ||x_n||)
    over the iterates n = 1..N; row 0 (the start x_0 = 0, whose log norm is -inf) is not a
    point of it and is never read. The proposed stop is the point of maximum curvature. CG
    first moves along the flat leg (the residual falls) and then up the steep leg (the
    solution norm grows), so the corner is a clockwise turn; the curvature is signed positive
    for clockwise turns: kappa = (a'' b' - a' b'') / (a'^2 + b'^2)^1.5, derivatives by central
    differences in n. Only interior points (n = 2..N-1) are candidates and the first maximum
    wins. Returns -1 when the curve has fewer than three points (N < 3).
    """
    a = np.log(np.asarray(res_norm, np.float64)[1:])
    b = np.log(np.asarray(sol_norm, np.float64)[1:])
    n = a.shape[0]
    if n < 3:
        return -1
    best, best_k = -1, -np.inf
    for i in range(1, n - 1):
        da = 0.5 * (a[i + 1] - a[i - 1])
        db = 0.5 * (b[i + 1] - b[i - 1])
        dda = a[i + 1] - 2.0 * a[i] + a[i - 1]
        ddb = b[i + 1] - 2.0 * b[i] + b[i - 1]
        den = (da * da + db * db) ** 1.5
        if den == 0.0:
            continue
        k = (dda * db - da * ddb) / den
        if k > best_k:
            best, best_k = i + 1, k      # point i of the curve is iteration i + 1
    return best
