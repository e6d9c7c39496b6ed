"""Host helpers of the map-smoothing command-line tool: the synthetic masks are nested (the trusted mask
inside the reconstruction mask), grow with the dilation, and match a direct construction."""
import numpy as np

from paper_2604_09233_gb300 import maps, synthetic


def test_synthetic_masks_are_nested_and_dilated():
    wl = synthetic.small_2d(seed=3, matrix=24, n_coils=4, n_samples=600, order=1)
    m_t, m_r = maps.synthetic_masks(wl, dilate=2)
    assert m_t.dtype == np.float32 and m_t.shape == (wl.L,)
    assert set(np.unique(m_t)) <= {0.0, 1.0} and set(np.unique(m_r)) <= {0.0, 1.0}
    assert np.all(m_r >= m_t) and m_r.sum() > m_t.sum() > 0
    same_t, same_r = maps.synthetic_masks(wl, dilate=0)
    assert np.array_equal(same_t, same_r) and np.array_equal(same_t, m_t)
    support = np.abs(wl.m_true) > 0.1 * np.abs(wl.m_true).max()
    assert np.array_equal(m_t.astype(bool), support)
    # one dilation step adds exactly the 4-connected neighbours of the support
    _, m1 = maps.synthetic_masks(wl, dilate=1)
    s = support.reshape(wl.shape)
    grown = s.copy()
    grown[1:, :] |= s[:-1, :]
    grown[:-1, :] |= s[1:, :]
    grown[:, 1:] |= s[:, :-1]
    grown[:, :-1] |= s[:, 1:]
    assert np.array_equal(m1.reshape(wl.shape).astype(bool), grown)


def test_noisy_sensitivities_are_seeded():
    wl = synthetic.small_2d(seed=3, matrix=16, n_coils=3, n_samples=300, order=1)
    a, b = maps.noisy_sensitivities(wl), maps.noisy_sensitivities(wl)
    assert a.dtype == np.complex64 and a.shape == wl.S.shape and np.array_equal(a, b)
    assert 0.0 < np.abs(a - wl.S).std() < 0.2
