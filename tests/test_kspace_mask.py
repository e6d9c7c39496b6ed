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
