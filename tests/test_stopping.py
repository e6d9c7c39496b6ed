"""The SSIM used by the stopping-rule study, against what its definition fixes (Wang, Bovik,
Sheikh and Simoncelli, 2004)."""
import numpy as np

from paper_2604_09233_gb300.stopping import ssim


def _img(seed, shape=(24, 20)):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[: shape[0], : shape[1]]
    return np.sin(x / 3.0) + np.cos(y / 4.0) + 0.3 * rng.normal(size=shape)


def test_identical_images_score_one():
    a = _img(1)
    assert abs(ssim(a, a, a.shape) - 1.0) < 1e-12


def test_symmetric_for_a_fixed_data_range():
    a, b = _img(1), _img(2)
    assert abs(ssim(a, b, a.shape, data_range=4.0) - ssim(b, a, a.shape, data_range=4.0)) < 1e-12


def test_constant_images_give_the_luminance_term():
    """Zero local variances and covariance: the structure factor is C2 / C2 = 1 and the index
    is (2 c1 c2 + C1) / (c1^2 + c2^2 + C1)."""
    D = 2.0
    c1, c2 = 0.7, 1.3
    a = np.full((16, 16), c1)
    b = np.full((16, 16), c2)
    C1 = (0.01 * D) ** 2
    expect = (2 * c1 * c2 + C1) / (c1 * c1 + c2 * c2 + C1)
    assert abs(ssim(a, b, a.shape, data_range=D) - expect) < 1e-12


def test_more_noise_scores_lower():
    rng = np.random.default_rng(3)
    a = _img(4)
    n = rng.normal(size=a.shape)
    vals = [ssim(a + s * n, a, a.shape) for s in (0.0, 0.05, 0.2, 1.0)]
    assert vals[0] > vals[1] > vals[2] > vals[3]

