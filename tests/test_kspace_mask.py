"""The library's convex-hull k-space mask (host code) against the oracle's Delaunay
triangulation of the same k-space coordinates (the paper's procedure)."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic


@pytest.mark.parametrize("matrix,R,n", [(32, 2, 2048), (96, 3, 6000), (128, 4, 16384)])
def test_mask_matches_delaunay_membership(matrix, R, n):
    from paper_2604_09233_gb300 import native
    fov = 0.22
    kx, ky = synthetic.spiral_2d(n, matrix, fov, R)
    d = fov / matrix
    lib = native.sense_kspace_filter_mask(matrix, matrix, d, d, kx, ky)
    ref = oracle.kspace_mask(matrix, matrix, d, d, kx, ky)
    # points on the hull boundary may go either way: compare away from it
    from scipy.spatial import ConvexHull
    hull = ConvexHull(np.stack([kx, ky], 1))
    eq = hull.equations                      # a x + b y + c <= 0 inside, (a, b) unit
    u = 2 * np.pi * (np.arange(matrix) - matrix // 2) / (matrix * d)
    U, V = np.meshgrid(u, u)
    dist = np.max(eq[:, 0][None] * U.ravel()[:, None] + eq[:, 1][None] * V.ravel()[:, None]
                  + eq[:, 2][None], axis=1).reshape(matrix, matrix)
    away = np.abs(dist) > 1e-6 * (2 * np.pi / (matrix * d))
    assert np.array_equal(lib[away], ref[away].astype(np.float32))
    assert 0.3 < lib.mean() < 1.0


def test_mask_rejects_bad_input():
    from paper_2604_09233_gb300 import native
    with pytest.raises(native.SenseError):
        native.sense_kspace_filter_mask(8, 8, 0.01, 0.01, [0.0, 1.0], [0.0, 1.0])
    with pytest.raises(native.SenseError):
        native.sense_kspace_filter_mask(8, 8, 0.01, 0.01, [0.0, 1.0, np.nan], [0.0, 1.0, 2.0])


def _hull_inside(points, q, tol):
    """Membership in the convex hull of `points` by its facet planes (scipy / Qhull)."""
    from scipy.spatial import ConvexHull
    eq = ConvexHull(points).equations          # n . x + c <= 0 inside, n unit
    d = q @ eq[:, :-1].T + eq[:, -1][None]
    return d.max(axis=1), d.max(axis=1) <= tol


@pytest.mark.parametrize("shape,planes,arms", [((8, 16, 16), 4, 2), ((12, 20, 24), 5, 3)])
def test_3d_mask_matches_the_hull_of_a_stack(shape, planes, arms):
    from paper_2604_09233_gb300 import native
    nz, ny, nx = shape
    fov, fov_z = 0.22, 0.096
    rng = np.random.default_rng(8)
    kx0, ky0 = synthetic.spiral_2d(300, nx, fov, 2)
    kx, ky, kz = [], [], []
    zs = np.sort(rng.choice(np.arange(-(nz // 2), nz - nz // 2), planes, replace=False))
    for ip, u in enumerate(zs):
        for a in range(arms):
            th = 2 * np.pi * a / arms + 0.7 * ip
            kx.append(kx0 * np.cos(th) - ky0 * np.sin(th))
            ky.append(kx0 * np.sin(th) + ky0 * np.cos(th))
            kz.append(np.full(kx0.size, 2 * np.pi * u / fov_z))
    kx, ky, kz = (np.concatenate(v) for v in (kx, ky, kz))
    d, dz = fov / nx, fov_z / nz
    m = native.sense_kspace_filter_mask3d(nx, ny, nz, d, d, dz, kx, ky, kz)
    g = [2 * np.pi * (np.arange(n) - n // 2) / (n * s) for n, s in ((nz, dz), (ny, d), (nx, d))]
    Z, Y, X = np.meshgrid(*g, indexing="ij")
    q = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    dist, inside = _hull_inside(np.stack([kx, ky, kz], 1), q, 0.0)
    away = np.abs(dist) > 1e-6 * (2 * np.pi / (nx * d))
    assert np.array_equal(m.ravel()[away] > 0, inside[away])
    assert 0.05 < m.mean() < 0.95


def test_3d_mask_of_the_3d_configuration_on_sampled_grid_points():
    from paper_2604_09233_gb300 import native
    wl = synthetic.stack_3d()
    nz, ny, nx = wl.shape
    d, dz = wl.meta["fov"] / nx, wl.meta["fov_z"] / nz
    kx, ky, kz = wl.Kmat[:, 2], wl.Kmat[:, 3], wl.Kmat[:, 4]
    m = native.sense_kspace_filter_mask3d(nx, ny, nz, d, d, dz, kx, ky, kz)
    rng = np.random.default_rng(9)
    idx = rng.choice(m.size, 4000, replace=False)
    w, v, u = np.unravel_index(idx, m.shape)
    q = np.stack([2 * np.pi * (u - nx // 2) / (nx * d), 2 * np.pi * (v - ny // 2) / (ny * d),
                  2 * np.pi * (w - nz // 2) / (nz * dz)], axis=1)
    dist, inside = _hull_inside(np.stack([kx, ky, kz], 1), q, 0.0)
    away = np.abs(dist) > 1e-6 * (2 * np.pi / (nx * d))
    assert np.array_equal(m.ravel()[idx][away] > 0, inside[away])
