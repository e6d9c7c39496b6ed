"""Pins of the FP64 oracle against results the paper and the mathematics fix.

None of these re-types the oracle's loops. Each targets a class of plausible mistake:
  closed-form DFT (numpy FFT)    -> exponent sign, operand transposition, index convention
  point source                   -> voxel / coil / intensity wiring of Eq. 4
  adjointness                    -> a missing conjugate or j factor in Eq. 5 vs Eq. 4
  phase-wrap invariance          -> range handling of large phases
  dense normal-equation solve    -> the CG recurrence of Fig. 2 Alg. 1 (LAPACK, not CG)
  Krylov minimisation            -> every early-stopped iterate (the paper stops at 7..56)
  data-residual monotonicity     -> CG minimises ||E(x - x*)|| over growing Krylov spaces
  finite differences             -> the B0-map gradient
  analytic curvature             -> the L-curve corner picker
"""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _crandn(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.fixture(scope="module")
def small():
    return synthetic.small_2d(seed=11, matrix=12, n_coils=4, n_samples=400, order=3, with_j=True)


def test_closed_form_dft_matches_numpy_fft():
    """Zero B0, no higher orders, Cartesian k-grid: E equals an inverse FFT of S_c*m."""
    ny, nx, fov_x, fov_y = 6, 10, 0.2, 0.15
    x, y, _ = synthetic.grid_positions((ny, nx), (fov_x, fov_y))
    L = nx * ny
    u = np.arange(nx) - nx // 2
    w = np.arange(ny) - ny // 2
    W, U = np.meshgrid(w, u, indexing="ij")
    kx = 2 * np.pi * U.ravel() / fov_x
    ky = 2 * np.pi * W.ravel() / fov_y
    K = kx.shape[0]
    t = np.arange(K) * 1e-5
    Km = np.stack([t, kx, ky], axis=1)
    Rm = np.stack([np.zeros(L), x, y])
    rng = np.random.default_rng(0)
    C = 3
    S = _crandn(rng, L, C)
    m = _crandn(rng, L)
    s = oracle.encode(Km, Rm, S, m)
    for c in range(C):
        v = (S[:, c] * m).reshape(ny, nx)
        F = nx * ny * np.fft.ifft2(v)          # sum_v v[iy,ix] e^{+2 pi i (w iy/ny + u ix/nx)}
        # positions are (i - N/2) d, which multiplies each coefficient by e^{-i pi (u + w)}
        # for even N; coefficient index (w, u) maps to FFT bin (w mod ny, u mod nx).
        expect = F[W.ravel() % ny, U.ravel() % nx] * np.exp(-1j * np.pi * (U.ravel() + W.ravel()))
        assert _rel(s[:, c], expect) < 1e-12


def test_point_source_analytic_signal(small):
    """m = a delta(l0): s(kappa, c) = S(l0, c) j(l0) a exp(i phi(kappa, l0))."""
    wl = small
    l0 = 37
    a = 0.7 - 0.2j
    m = np.zeros(wl.L, complex)
    m[l0] = a
    s = oracle.encode(wl.Kmat, wl.Rmat, wl.S, m, j=wl.j)
    phi = wl.Kmat @ wl.Rmat[:, l0]
    expect = np.exp(1j * phi)[:, None] * (wl.S[l0] * wl.j[l0] * a)[None, :]
    assert _rel(s, expect) < 1e-12
    # a subset of rows gives the same rows
    rows = np.array([5, 0, 399, 123])
    assert _rel(oracle.encode(wl.Kmat, wl.Rmat, wl.S, m, j=wl.j, rows=rows), s[rows]) == 0.0


def test_adjointness(small):
    wl = small
    rng = np.random.default_rng(1)
    x = _crandn(rng, wl.L)
    y = _crandn(rng, wl.K, wl.C)
    Ex = oracle.encode(wl.Kmat, wl.Rmat, wl.S, x, j=wl.j)
    EHy = oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y, j=wl.j)
    lhs = np.vdot(Ex, y)        # <Ex, y>
    rhs = np.vdot(x, EHy)       # <x, E^H y>
    assert abs(lhs - rhs) / (np.linalg.norm(Ex) * np.linalg.norm(y)) < 1e-12
    # voxel subset
    vox = np.array([3, 140, 0, 77])
    assert _rel(oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y, j=wl.j, vox=vox), EHy[vox]) == 0.0


def test_normal_operator_hermitian_psd(small):
    wl = small
    rng = np.random.default_rng(2)
    u, v = _crandn(rng, wl.L), _crandn(rng, wl.L)
    Au = oracle.normal(wl.Kmat, wl.Rmat, wl.S, u, j=wl.j)
    Av = oracle.normal(wl.Kmat, wl.Rmat, wl.S, v, j=wl.j)
    assert abs(np.vdot(u, Av) - np.vdot(Au, v)) / (np.linalg.norm(Au) * np.linalg.norm(v)) < 1e-12
    q = np.vdot(v, Av)
    assert q.real > 0 and abs(q.imag) < 1e-12 * q.real


def test_phase_wrap_invariance(small):
    """Adding 2 pi n / dwell to the B0 map changes every phase by 2 pi n kappa."""
    wl = small
    dwell = wl.Kmat[1, 0] - wl.Kmat[0, 0]
    Km = wl.Kmat.copy()
    Km[:, 0] = np.arange(wl.K) * dwell  # exact multiples of the dwell
    rng = np.random.default_rng(3)
    m = _crandn(rng, wl.L)
    s0 = oracle.encode(Km, wl.Rmat, wl.S, m, j=wl.j)
    Rw = wl.Rmat.copy()
    n = rng.integers(-3, 4, size=wl.L)
    Rw[0] = Rw[0] + 2 * np.pi * n / dwell
    s1 = oracle.encode(Km, Rw, wl.S, m, j=wl.j)
    assert _rel(s1, s0) < 1e-9


def _dense_E(wl):
    cols = []
    for l in range(wl.L):
        e = np.zeros(wl.L, complex)
        e[l] = 1.0
        cols.append(oracle.encode(wl.Kmat, wl.Rmat, wl.S, e, j=wl.j).ravel())
    return np.stack(cols, axis=1)


@pytest.fixture(scope="module")
def tiny():
    wl = synthetic.small_2d(seed=21, matrix=6, n_coils=4, n_samples=180, order=2, R=1,
                            with_j=True)
    sigma = oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j) + wl.noise
    return wl, sigma, _dense_E(wl)


def test_cg_converges_to_dense_normal_solution(tiny):
    wl, sigma, E = tiny
    A = E.conj().T @ E
    b = E.conj().T @ sigma.ravel()
    x_star = np.linalg.solve(A, b)
    out = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, 4 * wl.L, j=wl.j, apply_j=False)
    assert _rel(out["x"], x_star) < 1e-9
    # Alg. 1 ends by multiplying the output by j
    out_j = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, 4 * wl.L, j=wl.j, apply_j=True)
    assert _rel(out_j["x"], x_star * wl.j) < 1e-9


def test_cg_iterates_minimise_error_over_krylov_space(tiny):
    """x_n = argmin over K_n(A, b) of ||x - x*||_A: fixes every early-stopped iterate."""
    wl, sigma, E = tiny
    A = E.conj().T @ E
    b = E.conj().T @ sigma.ravel()
    n_it = 6
    out = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, n_it, j=wl.j, apply_j=False, iterates=True)
    its = out["iterates"]
    assert np.all(its[0] == 0)
    krylov = [b]
    for n in range(1, n_it + 1):
        V, _ = np.linalg.qr(np.stack(krylov, axis=1))
        xn = V @ np.linalg.solve(V.conj().T @ A @ V, V.conj().T @ b)
        assert _rel(its[n], xn) < 1e-8, n
        krylov.append(A @ krylov[-1] / np.linalg.norm(A @ krylov[-1]))


def test_cg_from_x0_minimises_error_over_shifted_krylov_space(tiny):
    """From a start x_0: x_n = x_0 + argmin over K_n(A, r_0) of ||x - x*||_A with
    r_0 = b - A x_0, and history row 0 holds ||r_0||, ||x_0||, ||E x_0 - s||."""
    wl, sigma, E = tiny
    A = E.conj().T @ E
    b = E.conj().T @ sigma.ravel()
    rng = np.random.default_rng(17)
    x0 = wl.m_true + 0.3 * _crandn(rng, wl.L)
    r0 = b - A @ x0
    n_it = 5
    out = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, n_it, j=wl.j, apply_j=False, iterates=True,
                    history=True, x0=x0)
    its, h = out["iterates"], out["history"]
    assert _rel(its[0], x0) == 0.0
    assert abs(h[0, 0] - np.linalg.norm(r0)) < 1e-10 * np.linalg.norm(b)
    assert abs(h[0, 1] - np.linalg.norm(x0)) < 1e-12 * np.linalg.norm(x0)
    assert abs(h[0, 2] - np.linalg.norm(E @ x0 - sigma.ravel())) < 1e-10 * np.linalg.norm(sigma)
    krylov = [r0 / np.linalg.norm(r0)]
    for n in range(1, n_it + 1):
        V, _ = np.linalg.qr(np.stack(krylov, axis=1))
        xn = x0 + V @ np.linalg.solve(V.conj().T @ A @ V, V.conj().T @ r0)
        assert _rel(its[n], xn) < 1e-8, n
        krylov.append(A @ krylov[-1] / np.linalg.norm(A @ krylov[-1]))


def test_cg_from_the_solution_stops_at_once(tiny):
    """Started at the dense solution x* the residual is already at rounding level: the
    tolerance stop (relative to ||E^H s||) ends the solve after 0 iterations at x*."""
    wl, sigma, E = tiny
    A = E.conj().T @ E
    b = E.conj().T @ sigma.ravel()
    x_star = np.linalg.solve(A, b)
    out = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, 10, j=wl.j, apply_j=False, rel_tol=1e-9,
                    x0=x_star, history=True)
    assert out["iters"] == 0
    assert _rel(out["x"], x_star) == 0.0
    assert out["history"][0, 0] < 1e-9 * np.linalg.norm(b)
    # a start near x* reaches the same tolerance in fewer iterations than x_0 = 0
    tol = 1e-4
    cold = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, 60, j=wl.j, apply_j=False, rel_tol=tol)
    rng = np.random.default_rng(3)
    warm = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, 60, j=wl.j, apply_j=False, rel_tol=tol,
                     x0=x_star + 1e-3 * np.linalg.norm(x_star) / np.sqrt(wl.L) * _crandn(rng, wl.L))
    assert 0 < warm["iters"] < cold["iters"]
    assert _rel(warm["x"], x_star) < 1e-3


def test_cg_history_and_residual_monotone(tiny):
    wl, sigma, E = tiny
    out = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, 12, j=wl.j, apply_j=False, history=True,
                    iterates=True)
    h = out["history"]
    b = E.conj().T @ sigma.ravel()
    assert abs(h[0, 0] - np.linalg.norm(b)) < 1e-12 * np.linalg.norm(b)
    assert h[0, 1] == 0.0
    assert abs(h[0, 2] - np.linalg.norm(sigma)) < 1e-12 * np.linalg.norm(sigma)
    for n in range(h.shape[0]):
        x = out["iterates"][n]
        assert abs(h[n, 1] - np.linalg.norm(x)) <= 1e-12 * max(1, np.linalg.norm(x))
        assert abs(h[n, 2] - np.linalg.norm(E @ x - sigma.ravel())) < 1e-10 * np.linalg.norm(sigma)
    assert np.all(np.diff(h[:, 2]) <= 1e-12 * h[0, 2])
    # recursive residual equals the true normal-equation residual b - A x
    A = E.conj().T @ E
    for n in (1, 5, 12):
        x = out["iterates"][n]
        assert abs(h[n, 0] - np.linalg.norm(b - A @ x)) < 1e-8 * np.linalg.norm(b)


def test_cg_relative_tolerance_stop(tiny):
    wl, sigma, _ = tiny
    full = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, 30, j=wl.j, history=True)
    tol = 1e-3
    out = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, 30, j=wl.j, rel_tol=tol, history=True)
    r = full["history"][:, 0]
    first = int(np.argmax(r <= tol * r[0]))
    assert out["iters"] == first
    assert _rel(out["x"], oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, first, j=wl.j)["x"]) == 0.0


def test_grad_omega_matches_central_differences(small):
    wl = small
    rng = np.random.default_rng(4)
    m = wl.m_true + 0.1 * _crandn(rng, wl.L)
    d = _crandn(rng, wl.K, wl.C)

    def loss(Rm):
        r = oracle.encode(wl.Kmat, Rm, wl.S, m, j=wl.j) - d
        return 0.5 * np.vdot(r, r).real

    g = oracle.encode(wl.Kmat, wl.Rmat, wl.S, m, j=wl.j) - d   # dLoss/dRe + i dLoss/dIm
    grad = oracle.grad_omega(wl.Kmat, wl.Rmat, wl.S, m, g, j=wl.j)
    h = 1e-2  # rad/s; phases change by ~t*h <= 2e-5 rad
    for l in (0, 17, 60, 143):
        Rp, Rn = wl.Rmat.copy(), wl.Rmat.copy()
        Rp[0, l] += h
        Rn[0, l] -= h
        fd = (loss(Rp) - loss(Rn)) / (2 * h)
        assert abs(fd - grad[l]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grad).max()), l


def test_grad_omega_adjoint_matches_central_differences(small):
    """x = E^H y: the B0 gradient of a loss of x, against central differences."""
    wl = small
    rng = np.random.default_rng(5)
    y = _crandn(rng, wl.K, wl.C)
    w = _crandn(rng, wl.L)

    def loss(Rm):
        x = oracle.adjoint(wl.Kmat, Rm, wl.S, y, j=wl.j)
        return np.vdot(w, x).real + 0.25 * np.vdot(x, x).real

    x0 = oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y, j=wl.j)
    h_up = w + 0.5 * x0                      # dLoss/dRe(x) + i dLoss/dIm(x)
    grad = oracle.grad_omega_adjoint(wl.Kmat, wl.Rmat, wl.S, y, h_up, j=wl.j)
    h = 1e-2
    for l in (0, 17, 60, 143):
        Rp, Rn = wl.Rmat.copy(), wl.Rmat.copy()
        Rp[0, l] += h
        Rn[0, l] -= h
        fd = (loss(Rp) - loss(Rn)) / (2 * h)
        assert abs(fd - grad[l]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grad).max()), l


def lcurve_pins(lcurve_corner):
    """(a, b) = (x, x^2) traversed right to left: curvature peaks (value 2) at the vertex.
    The arrays are CG-history columns: entry n belongs to iterate n, and entry 0 (the start
    x_0 = 0) is not a point of the L-curve (the curve runs over n = 1..N)."""
    xs = np.linspace(2.0, -1.0, 31)           # vertex at index 20
    idx = lcurve_corner(np.exp(xs), np.exp(xs ** 2))
    assert idx == 20
    # a shifted vertex moves the corner with it
    xs2 = xs + 0.5                             # vertex now where xs == -0.5 -> index 25
    assert lcurve_corner(np.exp(xs2), np.exp((xs2 - 0.0) ** 2)) == 25
    # fewer than three iterates (entries 1..N, N < 3): no corner
    assert lcurve_corner([1.0, 2.0], [1.0, 1.0]) == -1
    assert lcurve_corner([1.0, 2.0, 3.0], [0.0, 1.0, 2.0]) == -1
    # a real history starts with ||x_0|| = 0: entry 0 is never read (no log of zero)
    sol = np.exp(xs ** 2)
    sol[0] = 0.0
    with np.errstate(all="raise"):
        assert lcurve_corner(np.exp(xs), sol) == 20
    # vertex at iteration 2, the first interior point of the curve; an entry 0 that would make
    # iteration 1 the sharpest turn if it were a point does not move the corner
    h = 0.1
    x = np.array([3 * h] + [(2 - n) * h for n in range(1, 31)])
    res, sol = np.exp(x), np.exp(x ** 2)
    sol[0] = np.exp(3 * h)
    assert lcurve_corner(res, sol) == 2


def test_lcurve_corner_on_parabola_vertex():
    lcurve_pins(oracle.lcurve_corner)


def test_kspace_filter_keeps_inside_and_removes_outside_plane_waves():
    kspace_filter_pins(oracle.kspace_filter)


def kspace_filter_pins(kspace_filter):
    """A Cartesian plane wave rho(x) = e^{-i k_u r_x} has all of its k-space content at k_u:
    the filter returns it unchanged when f(u) = 1 and removes it when f(u) = 0; f = 1 is the
    identity; the transform is linear (checked on a sum)."""
    shape = (6, 10)
    ny, nx = shape
    y, x = np.mgrid[:ny, :nx]
    f = np.zeros(shape)
    f[2, 7] = 1.0

    def wave(u, v):
        return np.exp(-2j * np.pi * ((u - nx // 2) * (x - nx // 2) / nx
                                     + (v - ny // 2) * (y - ny // 2) / ny)).ravel()

    a, b = wave(7, 2), wave(3, 4)
    assert np.allclose(kspace_filter(a, shape, f), a, atol=1e-12)
    assert np.allclose(kspace_filter(b, shape, f), 0, atol=1e-12)
    assert np.allclose(kspace_filter(2 * a + b, shape, f), 2 * a, atol=1e-12)
    rng = np.random.default_rng(6)
    z = rng.normal(size=60) + 1j * rng.normal(size=60)
    assert np.allclose(kspace_filter(z, shape, np.ones(shape)), z, atol=1e-12)
    # 3D: the same along the third axis
    z3 = rng.normal(size=(3, 4, 5)) + 1j * rng.normal(size=(3, 4, 5))
    assert np.allclose(kspace_filter(z3, (3, 4, 5), np.ones((3, 4, 5))), z3.ravel())


def test_kspace_mask_of_a_square_of_samples():
    kspace_mask_pins(oracle.kspace_mask)


def kspace_mask_pins(kspace_mask):
    """Samples on the corners of a rectangle cover exactly the Cartesian points inside it; the
    grid spacing differs along x and y in the second case, and the grid is not square."""
    nx = ny = 8
    d = 0.01
    dk = 2 * np.pi / (nx * d)
    kx = np.array([-2.5, 2.5, 2.5, -2.5]) * dk
    ky = np.array([-1.5, -1.5, 1.5, 1.5]) * dk
    m = kspace_mask(nx, ny, d, d, kx, ky)
    expect = np.zeros((ny, nx))
    expect[4 - 1: 4 + 2, 4 - 2: 4 + 3] = 1.0
    assert np.array_equal(m, expect)
    # 10 x 6 grid, dx = 0.01, dy = 0.02: k steps 2 pi / 0.1 along x and 2 pi / 0.12 along y
    nx, ny, dx, dy = 10, 6, 0.01, 0.02
    dkx, dky = 2 * np.pi / (nx * dx), 2 * np.pi / (ny * dy)
    kx = np.array([-3.5, 1.5, 1.5, -3.5]) * dkx
    ky = np.array([-0.5, -0.5, 2.5, 2.5]) * dky
    m = kspace_mask(nx, ny, dx, dy, kx, ky)
    expect = np.zeros((ny, nx))
    expect[3 + 0: 3 + 3, 5 - 3: 5 + 2] = 1.0      # u - 5 in -3..1, v - 3 in 0..2
    assert np.array_equal(m, expect)


def test_smooth_map_pins():
    smooth_map_pins(oracle.smooth_map)


def smooth_map_pins(smooth_map):
    """Eq. 1 / Eq. 3 smoothing: a field in the null space of the derivative is returned unchanged
    for any alpha (linear for second differences, constant for first differences); with the
    data term on half the grid only (Eq. 1 with M_T a half, M_R everything) a linear field is
    continued exactly over the other half; alpha = 0 returns the data where w0 = 1; and the
    normal equations hold for a random field."""
    ny, nx = 7, 9
    y, x = np.mgrid[:ny, :nx]
    lin = (0.3 + 0.2j) * x - (0.1 - 0.4j) * y + 1.0
    ones = np.ones((ny, nx))
    assert np.allclose(smooth_map((ny, nx), 2, 5.0, ones, ones, lin), lin.ravel())
    const = np.full((ny, nx), 2.0 - 1.0j)
    rng = np.random.default_rng(7)
    eps = rng.uniform(0.5, 2.0, size=(ny, nx))
    assert np.allclose(smooth_map((ny, nx), 1, 3.0, ones, eps, const), const.ravel())
    half = (x < nx // 2).astype(float)
    garbage = np.where(half > 0, lin, 50.0 + 7j)            # data outside M_T is ignored
    assert np.allclose(smooth_map((ny, nx), 2, 0.7, half, ones, garbage), lin.ravel())
    z = rng.normal(size=(ny, nx)) + 1j * rng.normal(size=(ny, nx))
    assert np.allclose(smooth_map((ny, nx), 1, 0.0, ones, eps, z), z.ravel())
    # extrapolation along the other axes: trusted on half the rows (y), half the planes (z)
    half_y = (y < ny // 2).astype(float)
    garbage_y = np.where(half_y > 0, lin, -4.0 + 9j)
    assert np.allclose(smooth_map((ny, nx), 2, 0.7, half_y, ones, garbage_y), lin.ravel())
    # 3D: a linear field along all three axes is kept by second differences
    zz, yy, xx = np.mgrid[:4, :5, :6]
    lin3 = 1.0 + 0.5 * xx - 0.25 * yy + 0.125j * zz
    o3 = np.ones((4, 5, 6))
    assert np.allclose(smooth_map((4, 5, 6), 2, 2.0, o3, o3, lin3), lin3.ravel())
    half_z = (zz < 2).astype(float)
    garbage_z = np.where(half_z > 0, lin3, 3.0)
    assert np.allclose(smooth_map((4, 5, 6), 2, 2.0, half_z, o3, garbage_z), lin3.ravel())


def test_smooth_map_weight_sits_on_the_row_voxel():
    smooth_map_weight_pin(oracle.smooth_map)


def smooth_map_weight_pin(smooth_map):
    """Three voxels, first differences (Eq. 3), alpha = 1, weights (1, 2, 5): the rows are
    w_0 (x1 - x0) and w_1 (x2 - x1) (the last voxel has no row, its weight is unused), so the
    normal matrix is I + [[1, -1, 0], [-1, 1 + 4, -4], [0, -4, 4]]."""
    N = np.eye(3) + np.array([[1.0, -1.0, 0.0], [-1.0, 5.0, -4.0], [0.0, -4.0, 4.0]])
    xhat = np.array([1.0, -2.0, 0.5j])
    expect = np.linalg.solve(N, xhat)
    got = smooth_map((1, 3), 1, 1.0, np.ones(3), np.array([1.0, 2.0, 5.0]), xhat)
    assert np.allclose(got, expect)
    # alpha scales the derivative part of the normal matrix linearly (alpha = 2 here)
    got_a = smooth_map((1, 3), 1, 2.0, np.ones(3), np.array([1.0, 2.0, 5.0]), xhat)
    assert np.allclose(got_a, np.linalg.solve(np.eye(3) + 2.0 * (N - np.eye(3)), xhat))
    # a data weight w0 = (2, 1, 0.5) enters squared on both sides: diag(4, 1, 1/4) + the same
    # derivative part, right-hand side (4, 1, 1/4) o xhat
    N2 = np.diag([4.0, 1.0, 0.25]) + (N - np.eye(3))
    expect2 = np.linalg.solve(N2, np.array([4.0, 1.0, 0.25]) * xhat)
    got2 = smooth_map((1, 3), 1, 1.0, np.array([2.0, 1.0, 0.5]), np.array([1.0, 2.0, 5.0]), xhat)
    assert np.allclose(got2, expect2)
    # unconstrained voxels (w0 = 0, every touching row weighted 0) keep xhat; the others solve
    # I + [[1, -1], [-1, 1]] on their own
    xh4 = np.array([1.0 + 1.0j, -1.0, 7.0, -3.0j])
    got4 = smooth_map((1, 4), 1, 1.0, np.array([1.0, 1.0, 0.0, 0.0]),
                      np.array([1.0, 0.0, 0.0, 0.0]), xh4)
    sub = np.linalg.solve(np.array([[2.0, -1.0], [-1.0, 2.0]]), xh4[:2])
    assert np.allclose(got4, np.concatenate([sub, xh4[2:]]))


def test_smooth_sensitivities_pins():
    smooth_sensitivities_pins(oracle.smooth_sensitivities)


def smooth_sensitivities_pins(smooth_sensitivities):
    """Per-coil smoothing of magnitude and normalised map (Eq. 1 as the paper applies it):
    a map with positive linear magnitude and constant phase, trusted on half the grid only, is
    returned exactly over the whole grid (both parts lie in the null space of the second
    difference); a unit-magnitude map with a curved phase keeps magnitude 1 everywhere (the
    magnitude is processed on its own), while its phase is smoothed; coils are processed
    independently (permuting coils permutes the result); an all-zero coil stays zero."""
    ny, nx = 8, 10
    y, x = np.mgrid[:ny, :nx]
    half = (x < nx // 2).astype(float)
    ones = np.ones((ny, nx))
    exact = np.stack([(1.0 + 0.2 * x + 0.1 * y) * np.exp(0.7j),
                      (2.0 + 0.05 * x - 0.1 * y) * np.exp(-2.1j)], axis=-1).reshape(-1, 2)
    garbage = np.where(half.ravel()[:, None] > 0, exact, 9.0 - 4.0j)
    out = smooth_sensitivities((ny, nx), 0.8, half, ones, garbage)
    assert np.allclose(out, exact)
    phase = np.exp(1j * 0.08 * (x - 4.5) ** 2).reshape(-1, 1)
    rng = np.random.default_rng(3)
    S = np.concatenate([phase, exact[:, :1], np.zeros((ny * nx, 1)),
                        rng.normal(size=(ny * nx, 1)) + 1j * rng.normal(size=(ny * nx, 1))],
                       axis=1)
    out = smooth_sensitivities((ny, nx), 0.8, ones, ones, S)
    assert np.allclose(np.abs(out[:, 0]), 1.0)
    assert not np.allclose(out[:, 0], phase[:, 0], atol=1e-3)
    assert np.array_equal(out[:, 2], np.zeros(ny * nx))
    perm = [3, 0, 2, 1]
    assert np.allclose(smooth_sensitivities((ny, nx), 0.8, ones, ones, S[:, perm]),
                       out[:, perm])
    # very strong smoothing on a line of 5 voxels, all trusted: each field tends to its
    # least-squares straight line, so S -> line(|S|) line(u) / |line(u)| with u = S / |S|
    # (np.polyfit fits the lines); smoothing S itself would weight the phase by the magnitude
    xs = np.arange(5.0)
    S5 = ((np.array([1.0, 3.0, 0.5, 2.0, 4.0]) *
           np.exp(1j * np.array([0.0, 1.2, -0.7, 2.0, 0.4])))).reshape(5, 1)
    one5 = np.ones(5)
    got5 = smooth_sensitivities((1, 5), 1e8, one5, one5, S5)[:, 0]

    def line(v):
        re = np.polyval(np.polyfit(xs, v.real, 1), xs)
        im = np.polyval(np.polyfit(xs, v.imag, 1), xs) if np.iscomplexobj(v) else 0.0
        return re + 1j * im

    m_line = line(np.abs(S5[:, 0])).real
    u_line = line(S5[:, 0] / np.abs(S5[:, 0]))
    assert np.allclose(got5, m_line * u_line / np.abs(u_line), atol=1e-5)
