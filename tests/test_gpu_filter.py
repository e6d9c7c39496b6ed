"""The k-space filter that ends Alg. 1 (Fig. 2) through the C ABI against the oracle's dense
transforms."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("shape", [(32, 32), (96, 96), (17, 12), (6, 10, 8)])
def test_filter_matches_dense_transforms(shape):
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(51)
    img = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    mask = (rng.uniform(size=shape) < 0.6).astype(np.float32)
    x = torch.from_numpy(img.ravel().copy()).to(dev)
    native.sense_kspace_filter(x, torch.from_numpy(mask.ravel()).to(dev), shape)
    ref = oracle.kspace_filter(img.ravel(), shape, mask)
    e = _rel(x.cpu().numpy(), ref)
    ones = torch.from_numpy(img.ravel().copy()).to(dev)
    native.sense_kspace_filter(ones, torch.ones(int(np.prod(shape)), device=dev), shape)
    e1 = _rel(ones.cpu().numpy(), img.ravel())
    print(f"k-space filter {shape}: vs dense {e:.2e}, identity {e1:.2e}")
    assert e <= 1e-5 and e1 <= 1e-5


def test_filter_after_reconstruction():
    """The paper's last step on a 128x128 reconstruction: the hull mask of the spiral's k-space
    coordinates applied to the CG image (split tensor cores), against the oracle filter of the
    same image."""
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wl = synthetic.precision_128()
    fov, N = wl.meta["fov"], wl.shape[0]
    kx, ky = wl.Kmat[:, 2], wl.Kmat[:, 3]          # the 1st-order (x, y) coefficients
    mask = native.sense_kspace_filter_mask(N, N, fov / N, fov / N, kx, ky)
    with native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j) as plan:
        m = torch.from_numpy(wl.m_true.astype(np.complex64)).to(dev)
        s = plan.encode(m) + torch.from_numpy(wl.noise.astype(np.complex64)).to(dev)
        x, _, _ = plan.cg(s, 30, prec=native.SENSE_PREC_TC_SPLIT)
    before = x.cpu().numpy()
    native.sense_kspace_filter(x, torch.from_numpy(mask.ravel()).to(dev), wl.shape)
    ref = oracle.kspace_filter(before, wl.shape, mask)
    assert _rel(x.cpu().numpy(), ref) <= 1e-5
    assert 0.5 < mask.mean() < 1.0
