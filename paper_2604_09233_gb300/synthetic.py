"""Seeded synthetic inputs shaped like the paper's 2D and 3D spiral workloads.

This module builds the INPUTS of the reconstruction only: the temporal basis K, the
spatial basis R, coil sensitivities S, a ground-truth phantom and coil noise. It holds
none of the method's arithmetic (no phase K R, no exponential, no E, E^H or CG), so both
the CUDA path and the FP64 oracle can be fed from it without sharing method code.

Conventions (variable table of Fig. 2):
  K[kappa, 0] = t_kappa (s), K[kappa, p+1] = k_p(t_kappa)   temporal basis, [K][P+1]
  R[0, l]     = B0(r_l) as an angular frequency (rad/s)      spatial basis, [P+1][L]
  R[p+1, l]   = h_p(r_l), unnormalised real solid harmonics of the voxel position (m)
  S[l, c]     complex sensitivities; Sigma = coil data [K][C]
Positions on an N-point axis are (i - N/2) * dx, voxels flattened with x fastest.
The phase convention is exp(+i K R) (Eq. 4), so the 1st-order coefficients k_1..k_3 are
k-space coordinates in rad/m. All draws use numpy PCG64 with the given seed.

Values handed to the GPU in single precision (S, the phantom, the noise) are rounded to
complex64 here, so the oracle and the CUDA path see bit-identical inputs.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

# ---------------------------------------------------------------------------------------
# Spherical-harmonic field basis: unnormalised real solid harmonics up to 3rd order,
# 1 + 3 + 5 + 7 = 16 terms (the field-camera expansion used for dynamic field terms).
# Each entry: (order, callable(x, y, z)). The list order is the row order of R[1:].
# ---------------------------------------------------------------------------------------
SH_TERMS = [
    (0, lambda x, y, z: np.ones_like(x)),
    (1, lambda x, y, z: x),
    (1, lambda x, y, z: y),
    (1, lambda x, y, z: z),
    (2, lambda x, y, z: x * y),
    (2, lambda x, y, z: z * y),
    (2, lambda x, y, z: 2 * z * z - (x * x + y * y)),
    (2, lambda x, y, z: x * z),
    (2, lambda x, y, z: x * x - y * y),
    (3, lambda x, y, z: 3 * x * x * y - y ** 3),
    (3, lambda x, y, z: x * y * z),
    (3, lambda x, y, z: y * (4 * z * z - x * x - y * y)),
    (3, lambda x, y, z: z * (2 * z * z - 3 * x * x - 3 * y * y)),
    (3, lambda x, y, z: x * (4 * z * z - x * x - y * y)),
    (3, lambda x, y, z: z * (x * x - y * y)),
    (3, lambda x, y, z: x ** 3 - 3 * x * y * y),
]
N_TERMS_BY_ORDER = {1: 4, 2: 9, 3: 16}


@dataclasses.dataclass
class Workload:
    """One reconstruction problem: inputs of Fig. 2 plus the ground truth used to make Sigma."""

    name: str
    Kmat: np.ndarray            # [K][P1] float64
    Rmat: np.ndarray            # [P1][L] float64
    S: np.ndarray               # [L][C] complex128 holding complex64-representable values
    m_true: np.ndarray          # [L] complex128 (complex64-representable)
    noise: np.ndarray           # [K][C] complex128 (complex64-representable)
    j: Optional[np.ndarray]     # [L] float64 (float32-representable) or None
    shape: tuple                # image matrix (nz, ny, nx) or (ny, nx)
    n_iter: int                 # N_It of the configuration
    meta: dict

    @property
    def L(self):
        return self.Rmat.shape[1]

    @property
    def K(self):
        return self.Kmat.shape[0]

    @property
    def C(self):
        return self.S.shape[1]

    @property
    def P1(self):
        return self.Kmat.shape[1]


def _c64(a):
    return np.asarray(a, np.complex64).astype(np.complex128)


def grid_positions(shape, fov):
    """Voxel centres (x, y, z) in metres for a matrix `shape` ((ny, nx) or (nz, ny, nx))."""
    if len(shape) == 2:
        ny, nx = shape
        nz = 1
        fov = (fov[0], fov[1], 0.0) if len(fov) == 2 else fov
    else:
        nz, ny, nx = shape
    dx, dy = fov[0] / nx, fov[1] / ny
    dz = fov[2] / nz if nz > 1 else 0.0
    ix = (np.arange(nx) - nx // 2) * dx
    iy = (np.arange(ny) - ny // 2) * dy
    iz = (np.arange(nz) - nz // 2) * dz
    Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def phantom(rng, x, y, fov, n_ellipses=6, z=None, fov_z=None):
    """Random ellipses (ellipsoids in 3D), complex, |m| in [0, 1], smooth phase."""
    L = x.shape[0]
    mag = np.zeros(L)
    for _ in range(n_ellipses):
        cx, cy = rng.uniform(-0.25, 0.25, 2) * fov
        ax, ay = rng.uniform(0.08, 0.3, 2) * fov
        th = rng.uniform(0, np.pi)
        amp = rng.uniform(0.2, 1.0)
        xr = (x - cx) * np.cos(th) + (y - cy) * np.sin(th)
        yr = -(x - cx) * np.sin(th) + (y - cy) * np.cos(th)
        q = (xr / ax) ** 2 + (yr / ay) ** 2
        if z is not None and fov_z:
            cz = rng.uniform(-0.2, 0.2) * fov_z
            az = rng.uniform(0.25, 0.5) * fov_z
            q = q + ((z - cz) / az) ** 2
        mag += amp * (q <= 1.0)
    if mag.max() > 0:
        mag = mag / mag.max()
    c = rng.normal(size=6)
    xn, yn = 2 * x / fov, 2 * y / fov
    ph = 0.6 * (c[0] + c[1] * xn + c[2] * yn + 0.5 * (c[3] * xn * xn + c[4] * xn * yn + c[5] * yn * yn))
    return _c64(mag * np.exp(1j * ph))


def coils(rng, x, y, z, n_coils, fov, ring_radius_fovs=1.2, width_fovs=0.6, z_rings=None):
    """Gaussian-loop sensitivities on a ring of radius 1.2*FOV; max |S| = 1."""
    R0 = ring_radius_fovs * fov
    w = width_fovs * fov
    out = np.empty((x.shape[0], n_coils), np.complex128)
    for c in range(n_coils):
        th = 2 * np.pi * c / n_coils + rng.uniform(-0.1, 0.1)
        cx, cy = R0 * np.cos(th), R0 * np.sin(th)
        cz = 0.0 if not z_rings else z_rings[c % len(z_rings)]
        d2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        mag = np.exp(-d2 / (2 * w * w))
        ang = np.arctan2(y - cy, x - cx)
        out[:, c] = mag * np.exp(1j * (th + 0.5 * ang + rng.uniform(-0.3, 0.3)))
    out /= np.abs(out).max()
    return _c64(out)


def b0_map(rng, x, y, fov, f_max_hz, z=None, fov_z=None):
    """2nd-order polynomial plus 2 Gaussian blobs, scaled to +-f_max Hz; returns rad/s."""
    xn, yn = 2 * x / fov, 2 * y / fov
    zn = 2 * z / fov_z if (z is not None and fov_z) else np.zeros_like(x)
    c = rng.normal(size=10)
    f = (c[0] + c[1] * xn + c[2] * yn + c[3] * zn + c[4] * xn * xn + c[5] * yn * yn
         + c[6] * xn * yn + c[7] * zn * zn + c[8] * xn * zn + c[9] * yn * zn)
    for _ in range(2):
        bx, by = rng.uniform(-0.3, 0.3, 2) * fov
        bw = rng.uniform(0.05, 0.12) * fov
        d2 = (x - bx) ** 2 + (y - by) ** 2
        if z is not None and fov_z:
            d2 = d2 + (z - rng.uniform(-0.2, 0.2) * fov_z) ** 2
        f = f + rng.uniform(1.5, 3.0) * rng.choice([-1, 1]) * np.exp(-d2 / (2 * bw * bw))
    f = f - 0.5 * (f.max() + f.min())
    f = f_max_hz * f / np.abs(f).max()
    return 2 * np.pi * f


def spiral_2d(n_samples, matrix, fov, R):
    """Single-shot variable-density Archimedean spiral-out, k in rad/m.

    Radius k_max (tau + tau^2)/2 over tau in [0, 1] (denser centre, 3x wider turn spacing at
    the edge), constant angular rate; the number of turns makes the outer turn spacing R
    times the Nyquist spacing 2 pi / FOV.
    """
    k_max = np.pi * matrix / fov
    tau = np.arange(n_samples) / max(n_samples - 1, 1)
    n_turns = 1.5 * matrix / (2.0 * R)
    kr = k_max * 0.5 * (tau + tau * tau)
    ang = 2 * np.pi * n_turns * tau
    return kr * np.cos(ang), kr * np.sin(ang)


def _cubic_spline_coeffs(rng, t, n_knots=8):
    from scipy.interpolate import CubicSpline
    knots = np.linspace(t[0], t[-1], n_knots)
    vals = rng.normal(size=n_knots)
    return CubicSpline(knots, vals, bc_type="natural")(t)


def field_basis_rows(x, y, z, order):
    """h_p(r_l) for the first N_TERMS_BY_ORDER[order] solid harmonics, [P][L]."""
    n = N_TERMS_BY_ORDER[order]
    return np.stack([SH_TERMS[p][1](x, y, z) for p in range(n)])


def make_spiral_2d(name, seed, matrix, fov, n_coils, n_samples, dwell, R, f_max_hz,
                   order=1, ho_scale=1e-3, noise_sigma=1e-3, n_iter=20, with_j=False,
                   include_zero_order=None):
    """2D single-slice spiral problem (configs of the 2D spiral family)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (matrix, matrix)
    x, y, z = grid_positions(shape, (fov, fov))
    L = x.shape[0]
    t = np.arange(n_samples) * dwell
    kx, ky = spiral_2d(n_samples, matrix, fov, R)

    omega = b0_map(rng, x, y, fov, f_max_hz)
    if order == 1 and not include_zero_order:
        # plain k-space encoding: linear terms only (x, y; z = 0 in a 2D slice)
        Rm = np.stack([omega, x, y])
        Km = np.stack([t, kx, ky], axis=1)
    else:
        h = field_basis_rows(x, y, z, order)
        kt = np.zeros((n_samples, h.shape[0]))
        kt[:, 1], kt[:, 2] = kx, ky
        lin_max = np.max(np.hypot(kx, ky)) * np.max(np.hypot(x, y))
        for p in range(h.shape[0]):
            if SH_TERMS[p][0] == 1:
                continue
            spl = _cubic_spline_coeffs(rng, t)
            hmax = np.max(np.abs(h[p]))
            if hmax == 0.0:
                # vanishes in this slice: keep a coefficient of the same size as the others
                hmax = (np.max(np.hypot(x, y)) ** SH_TERMS[p][0]) or 1.0
            kt[:, p] = ho_scale * lin_max * spl / (np.max(np.abs(spl)) * hmax)
        Rm = np.vstack([omega[None, :], h])
        Km = np.hstack([t[:, None], kt])

    S = coils(rng, x, y, z, n_coils, fov)
    m = phantom(rng, x, y, fov)
    noise = _c64((rng.normal(size=(n_samples, n_coils)) + 1j * rng.normal(size=(n_samples, n_coils)))
                 * noise_sigma / np.sqrt(2.0))
    j = None
    if with_j:
        j = np.asarray(0.75 + 0.5 * rng.uniform(size=L), np.float32).astype(np.float64)
    meta = dict(fov=fov, dwell=dwell, R=R, f_max_hz=f_max_hz, order=order, seed=seed,
                T_acq_ms=n_samples * dwell * 1e3)
    return Workload(name, np.ascontiguousarray(Km), np.ascontiguousarray(Rm), S, m, noise, j,
                    shape, n_iter, meta)


def make_stack_of_spirals_3d(name, seed, shape, fov, fov_z, n_coils, n_arm_samples, dwell,
                             R_z, arms, R_arm, f_max_hz, order=2, ho_scale=1e-3,
                             noise_sigma=1e-3, n_iter=30):
    """3D stack of spirals. Every R_z-th of the nz kz planes is acquired; each plane carries
    `arms` spiral-out arms (each R_arm-fold undersampled, rotated by 2 pi / arms, the set
    turned by a further golden-angle step from plane to plane), so R = R_z R_arm / arms.
    Every arm is one readout: t restarts at 0. Linear terms are (kx, ky, kz); the other
    solid-harmonic terms up to `order` are smooth random cubic splines of t (shared by all
    arms) at ho_scale of the linear amplitude."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = shape
    x, y, z = grid_positions(shape, (fov, fov, fov_z))
    L = x.shape[0]
    kx0, ky0 = spiral_2d(n_arm_samples, nx, fov, R_arm)
    t_arm = np.arange(n_arm_samples) * dwell
    planes = np.arange(-(nz // 2), nz - nz // 2, R_z)
    golden = np.pi * (3.0 - np.sqrt(5.0))
    kx, ky, kz, t = [], [], [], []
    for ip, u in enumerate(planes):
        for a in range(arms):
            th = 2 * np.pi * a / arms + golden * ip
            kx.append(kx0 * np.cos(th) - ky0 * np.sin(th))
            ky.append(kx0 * np.sin(th) + ky0 * np.cos(th))
            kz.append(np.full(n_arm_samples, 2 * np.pi * u / fov_z))
            t.append(t_arm)
    kx, ky, kz, t = (np.concatenate(v) for v in (kx, ky, kz, t))
    K = t.shape[0]
    omega = b0_map(rng, x, y, fov, f_max_hz, z=z, fov_z=fov_z)
    h = field_basis_rows(x, y, z, order)
    kt = np.zeros((K, h.shape[0]))
    kt[:, 1], kt[:, 2], kt[:, 3] = kx, ky, kz
    r_max = np.max(np.sqrt(x * x + y * y + z * z))
    lin_max = np.max(np.sqrt(kx * kx + ky * ky + kz * kz)) * r_max
    for p in range(h.shape[0]):
        if SH_TERMS[p][0] == 1:
            continue
        spl = _cubic_spline_coeffs(rng, t_arm)
        hmax = np.max(np.abs(h[p])) or 1.0
        kt[:, p] = np.tile(ho_scale * lin_max * spl / (np.max(np.abs(spl)) * hmax),
                           K // n_arm_samples)
    Rm = np.vstack([omega[None, :], h])
    Km = np.hstack([t[:, None], kt])
    zr = [(-1.5 + k) * fov_z / 2 for k in range(4)]
    S = coils(rng, x, y, z, n_coils, fov, z_rings=zr)
    m = phantom(rng, x, y, fov, z=z, fov_z=fov_z)
    noise = _c64((rng.normal(size=(K, n_coils)) + 1j * rng.normal(size=(K, n_coils)))
                 * noise_sigma / np.sqrt(2.0))
    meta = dict(fov=fov, fov_z=fov_z, dwell=dwell, R=R_z * R_arm / arms, f_max_hz=f_max_hz,
                order=order, seed=seed, planes=len(planes), arms=arms,
                T_acq_ms=n_arm_samples * dwell * 1e3)
    return Workload(name, np.ascontiguousarray(Km), np.ascontiguousarray(Rm), S, m, noise, None,
                    shape, n_iter, meta)


# ---------------------------------------------------------------------------------------
# Named workloads. Seeds follow seed = 1000 * config + instance.
# ---------------------------------------------------------------------------------------

def plain_32():
    """2D 32x32, FOV 220 mm, 8 coils, 2048-sample spiral at 5 us (10.24 ms), R=2,
    B0 +-50 Hz, linear terms only, noise 1e-3, 20 CG iterations."""
    return make_spiral_2d("2d_32x32_8coil_2048samp", 1000, 32, 0.22, 8, 2048, 5e-6, 2, 50.0,
                          order=1, n_iter=20)


def precision_128():
    """2D 128x128, 32 coils, 16384-sample spiral at 2 us (32.8 ms), R=4, B0 +-100 Hz,
    3rd-order solid harmonics (16 terms) at 1e-3 of the linear amplitude, 30 iterations."""
    return make_spiral_2d("2d_128x128_32coil_16384samp_sh3", 2000, 128, 0.22, 32, 16384, 2e-6,
                          4, 100.0, order=3, n_iter=30)


def target_256():
    """2D 256x256, 32 coils, 35750-sample spiral at 2 us (71.5 ms), R=4, B0 +-150 Hz,
    3rd-order solid harmonics, 40 CG iterations."""
    return make_spiral_2d("2d_256x256_32coil_35750samp_sh3", 3000, 256, 0.22, 32, 35750, 2e-6,
                          4, 150.0, order=3, n_iter=40)


def stack_3d():
    """3D 96x96x48 (442368 voxels), FOV 220 x 220 x 96 mm, 32 coils on 4 rings; stack of
    spirals with 16 of 48 kz planes x 3 arms of 1300 samples at 2 us (62400 samples, R = 7);
    B0 3D polynomial plus blobs, +-200 Hz; 2nd-order solid harmonics (9 terms); 30 CG
    iterations."""
    return make_stack_of_spirals_3d("3d_96x96x48_32coil_62400samp_sh2", 4000, (48, 96, 96),
                                    0.22, 0.096, 32, 1300, 2e-6, 3, 3, 7, 200.0, order=2,
                                    n_iter=30)


def small_3d(seed=4100, shape=(8, 16, 16), n_coils=8, n_arm_samples=200, R_z=2, arms=2,
             R_arm=2, order=2):
    """Small stack of spirals of the same family for parity tests."""
    return make_stack_of_spirals_3d(f"small3d_{'x'.join(map(str, shape))}_{n_coils}c", seed,
                                    shape, 0.22, 0.096, n_coils, n_arm_samples, 4e-6, R_z, arms,
                                    R_arm, 100.0, order=order, n_iter=10)


def batch_64(n=64, seed=5000):
    """64 independent 2D spiral instances of uneven size: matrix uniform in
    {64,96,128,192,256}^2, coils in {8,16,32}, 4096-35750 samples at 2 us, R in {2,3,4},
    B0 +-50..150 Hz, field expansion of order 1..3; 50 CG iterations at most, stop at a
    relative residual of 1e-3. Instance i uses seed + i; the sizes are drawn with seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        matrix = int(rng.choice([64, 96, 128, 192, 256]))
        coils = int(rng.choice([8, 16, 32]))
        samples = int(rng.integers(4096, 35751))
        R = int(rng.choice([2, 3, 4]))
        order = int(rng.integers(1, 4))
        fmax = float(rng.uniform(50.0, 150.0))
        out.append(make_spiral_2d(f"b{i}_{matrix}x{matrix}_{coils}c_{samples}s_o{order}",
                                  seed + i, matrix, 0.22, coils, samples, 2e-6, R, fmax,
                                  order=order, n_iter=50))
    return out


def batch_small_64(n=64, seed=6000):
    """64 independent small 2D spiral instances, the case a persistent batched launch is for:
    matrix uniform in {64, 96}^2, coils in {8, 16}, 4096-8192 samples at 2 us, R in {2, 3, 4},
    B0 +-50..150 Hz, field expansion of order 1..3; stop at a relative residual of 1e-3 or 50
    iterations. Instance i uses seed + i; the sizes are drawn with seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        matrix = int(rng.choice([64, 96]))
        coils = int(rng.choice([8, 16]))
        samples = int(rng.integers(4096, 8193))
        R = int(rng.choice([2, 3, 4]))
        order = int(rng.integers(1, 4))
        fmax = float(rng.uniform(50.0, 150.0))
        out.append(make_spiral_2d(f"s{i}_{matrix}x{matrix}_{coils}c_{samples}s_o{order}",
                                  seed + i, matrix, 0.22, coils, samples, 2e-6, R, fmax,
                                  order=order, n_iter=50))
    return out


def small_batch(seed=7000):
    """Five small instances of uneven size for batch parity tests (ragged tiles, 1..32 coils,
    orders 1..3, one with intensity correction j)."""
    spec = [(24, 8, 1500, 3, True), (12, 3, 300, 1, False), (20, 32, 1000, 2, False),
            (8, 1, 100, 1, False), (16, 16, 600, 3, False)]
    return [small_2d(seed=seed + i, matrix=mtx, n_coils=c, n_samples=k, order=o, with_j=wj)
            for i, (mtx, c, k, o, wj) in enumerate(spec)]


def small_2d(seed=7, matrix=24, n_coils=8, n_samples=1500, order=3, R=2, f_max_hz=80.0,
             with_j=False, dwell=4e-6, n_iter=10):
    """Small problem of the same family for parity tests (oracle runs in well under a second)."""
    return make_spiral_2d(f"small_{matrix}_{n_coils}_{n_samples}_o{order}", seed, matrix, 0.22,
                          n_coils, n_samples, dwell, R, f_max_hz, order=order, n_iter=n_iter,
                          with_j=with_j)
