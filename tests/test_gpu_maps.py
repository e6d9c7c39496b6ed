"""Map smoothing (Eqs. 1 and 3) through the C ABI against the oracle's direct sparse solve."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.linspace(-1, 1, n) for n in shape], indexing="ij")
    r2 = sum(g * g for g in grids)
    smooth = np.exp(-r2) * np.exp(1j * (grids[-1] + 0.5 * grids[0]))
    xhat = smooth + 0.05 * (rng.normal(size=shape) + 1j * rng.normal(size=shape))
    m_r = (r2 < 0.9).astype(np.float32)                 # reconstruction mask
    m_t = (r2 < 0.5).astype(np.float32)                 # trusted mask inside it
    eps = rng.uniform(0.2, 2.0, size=shape).astype(np.float32)
    return xhat.astype(np.complex64), m_t, m_r, eps


@pytest.mark.parametrize("shape", [(24, 20), (6, 10, 8)])
@pytest.mark.parametrize("eq", [1, 3])
def test_smoothing_matches_direct_solve(shape, eq):
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    xhat, m_t, m_r, eps = _fields(shape, 71)
    if eq == 1:          # sensitivity maps: second differences, data only where trusted
        order, alpha, w0, wd = 2, 0.5, m_t, m_r
    else:                # B0 map: first differences weighted by the fit error
        order, alpha, w0, wd = 1, 2.0, np.ones(shape, np.float32), eps
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).to(dev)
    x = torch.empty(int(np.prod(shape)), dtype=torch.complex64, device=dev)
    info = native.sense_smooth_map(shape, order, alpha, t(w0), t(wd), t(xhat), x,
                                   max_iter=5000, rel_tol=1e-7)
    ref = oracle.smooth_map(shape, order, alpha, w0, wd, xhat.astype(complex))
    e = _rel(x.cpu().numpy(), ref)
    print(f"Eq. {eq} {shape}: {info['iters']} iterations, residual {info['rel_residual']:.1e}, "
          f"vs direct solve {e:.2e}")
    assert e <= 1e-4 and info["rel_residual"] <= 1e-7


def test_smoothing_keeps_the_null_space_and_extrapolates():
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    ny, nx = 16, 20
    y, x = np.mgrid[:ny, :nx]
    lin = ((0.3 + 0.2j) * x - (0.1 - 0.4j) * y + 1.0).astype(np.complex64)
    half = (x < nx // 2).astype(np.float32)
    data = np.where(half > 0, lin, 50.0 + 7j).astype(np.complex64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).to(dev)
    out = torch.empty(nx * ny, dtype=torch.complex64, device=dev)
    native.sense_smooth_map((ny, nx), 2, 0.7, t(half), t(np.ones((ny, nx), np.float32)), t(data),
                            out, max_iter=5000, rel_tol=1e-8)
    assert _rel(out.cpu().numpy(), lin.ravel()) <= 1e-4
