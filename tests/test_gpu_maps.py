"""Map smoothing (Eqs. 1 and 3) through the C ABI against the oracle's direct sparse solve."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.linspace(-1, 1, n) if n > 1 else np.zeros(1) for n in shape],
                        indexing="ij")
    r2 = sum(g * g for g in grids)
    smooth = np.exp(-r2) * np.exp(1j * (grids[-1] + 0.5 * grids[0]))
    xhat = smooth + 0.05 * (rng.normal(size=shape) + 1j * rng.normal(size=shape))
    m_r = (r2 < 0.9).astype(np.float32)                 # reconstruction mask
    m_t = (r2 < 0.5).astype(np.float32)                 # trusted mask inside it
    eps = rng.uniform(0.2, 2.0, size=shape).astype(np.float32)
    return xhat.astype(np.complex64), m_t, m_r, eps


@pytest.mark.parametrize("precond", ["none", "multigrid"])
@pytest.mark.parametrize("shape", [(24, 20), (6, 10, 8), (5, 7), (7, 1), (1, 7, 1), (4, 9, 33)])
@pytest.mark.parametrize("eq", [1, 3])
def test_smoothing_matches_direct_solve(shape, eq, precond):
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
                                   max_iter=5000, rel_tol=1e-7, precond=precond)
    ref = oracle.smooth_map(shape, order, alpha, w0, wd, xhat.astype(complex))
    e = _rel(x.cpu().numpy(), ref)
    print(f"Eq. {eq} {shape} {precond}: {info['iters']} iterations, residual "
          f"{info['rel_residual']:.1e}, vs direct solve {e:.2e}")
    assert e <= 1e-4 and info["rel_residual"] <= 1e-7


@pytest.mark.parametrize("eq", [1, 3])
def test_multigrid_on_a_larger_grid(eq):
    """96 x 80 and 20 x 24 x 16 grids (several coarse levels, ragged even and odd axes): the
    preconditioned solve reaches the direct solution in a small fraction of plain CG's
    iterations and stops at the requested tolerance."""
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    for shape in [(96, 80), (20, 24, 16)]:
        xhat, m_t, m_r, eps = _fields(shape, 72)
        if eq == 1:
            order, alpha, w0, wd = 2, 0.5, m_t, m_r
        else:
            order, alpha, w0, wd = 1, 2.0, np.ones(shape, np.float32), eps
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).to(dev)
        ref = oracle.smooth_map(shape, order, alpha, w0, wd, xhat.astype(complex))
        out = {}
        for pc in ("none", "multigrid"):
            x = torch.empty(int(np.prod(shape)), dtype=torch.complex64, device=dev)
            info = native.sense_smooth_map(shape, order, alpha, t(w0), t(wd), t(xhat), x,
                                           max_iter=40000, rel_tol=1e-6, precond=pc)
            out[pc] = info
            e = _rel(x.cpu().numpy(), ref)
            print(f"Eq. {eq} {shape} {pc}: {info['iters']} iterations, vs direct {e:.2e}")
            assert info["rel_residual"] <= 1e-6 and e <= 1e-3
        assert out["multigrid"]["iters"] * 4 <= out["none"]["iters"]


def test_multigrid_stops_at_max_iter_and_accepts_a_converged_start():
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    shape = (40, 36)
    xhat, m_t, m_r, _ = _fields(shape, 73)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).to(dev)
    x = torch.empty(int(np.prod(shape)), dtype=torch.complex64, device=dev)
    info = native.sense_smooth_map(shape, 2, 0.5, t(m_t), t(m_r), t(xhat), x, max_iter=3,
                                   rel_tol=1e-12)
    assert info["iters"] == 3
    info = native.sense_smooth_map(shape, 2, 0.5, t(m_t), t(m_r), t(xhat), x, max_iter=0)
    assert info["iters"] == 0 and torch.equal(x, t(xhat))
    # a start that already solves the equations (alpha = 0, w0 = 1: x = xhat)
    info = native.sense_smooth_map(shape, 2, 0.0, t(np.ones(shape, np.float32)), t(m_r),
                                   t(xhat), x, max_iter=50, rel_tol=1e-6)
    assert info["iters"] == 0 and torch.equal(x, t(xhat))
    with pytest.raises(native.SenseError):
        native.sense_smooth_map(shape, 2, 0.5, t(m_t), t(m_r), t(xhat), x, precond=7)


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
    for pc in ("none", "multigrid"):
        native.sense_smooth_map((ny, nx), 2, 0.7, t(half), t(np.ones((ny, nx), np.float32)),
                                t(data), out, max_iter=5000, rel_tol=1e-8, precond=pc)
        assert _rel(out.cpu().numpy(), lin.ravel()) <= 1e-4


def test_unconstrained_voxels_keep_xhat_under_both_solvers():
    """Voxels outside the trusted mask and outside every weighted derivative row (w0 = wd = 0
    in a corner block) are not touched by the solve."""
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    shape = (30, 28)
    xhat, m_t, _, _ = _fields(shape, 74)
    wd = np.ones(shape, np.float32)
    wd[:8, :8] = 0.0
    w0 = m_t.copy()
    w0[:8, :8] = 0.0
    ref = oracle.smooth_map(shape, 2, 0.5, w0, wd, xhat.astype(complex))
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).to(dev)
    for pc in ("none", "multigrid"):
        x = torch.empty(int(np.prod(shape)), dtype=torch.complex64, device=dev)
        native.sense_smooth_map(shape, 2, 0.5, t(w0), t(wd), t(xhat), x, max_iter=20000,
                                rel_tol=1e-7, precond=pc)
        got = x.cpu().numpy().reshape(shape)
        assert np.array_equal(got[:5, :5], xhat[:5, :5])
        assert _rel(got.ravel(), ref) <= 1e-4


@pytest.mark.parametrize("precond", ["none", "multigrid"])
def test_several_fields_in_one_solve(precond):
    """Five right-hand sides on one grid (Eq. 1 masks): each field matches its own direct
    solve, each stops on its own test, and the batch result equals five single-field calls."""
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    shape = (26, 22)
    n = int(np.prod(shape))
    _, m_t, m_r, _ = _fields(shape, 75)
    rng = np.random.default_rng(76)
    X = np.stack([_fields(shape, 80 + k)[0].ravel() * (1.0 + k) for k in range(4)] +
                 [rng.normal(size=n) + 0j]).astype(np.complex64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    out = torch.empty((5, n), dtype=torch.complex64, device=dev)
    infos = native.sense_smooth_map(shape, 2, 0.5, t(m_t.ravel()), t(m_r.ravel()), t(X), out,
                                    max_iter=20000, rel_tol=1e-7, precond=precond)
    assert len(infos) == 5
    for k in range(5):
        ref = oracle.smooth_map(shape, 2, 0.5, m_t, m_r, X[k].astype(complex))
        assert infos[k]["rel_residual"] <= 1e-7
        assert _rel(out[k].cpu().numpy(), ref) <= 1e-4
        one = torch.empty(n, dtype=torch.complex64, device=dev)
        inf1 = native.sense_smooth_map(shape, 2, 0.5, t(m_t.ravel()), t(m_r.ravel()), t(X[k]),
                                       one, max_iter=20000, rel_tol=1e-7, precond=precond)
        assert inf1["iters"] == infos[k]["iters"]
        assert _rel(out[k].cpu().numpy(), one.cpu().numpy()) <= 1e-6
    print(precond, [i["iters"] for i in infos])


@pytest.mark.parametrize("precond", ["none", "multigrid"])
@pytest.mark.parametrize("shape", [(24, 20), (6, 10, 8)])
def test_sensitivity_maps_match_oracle(shape, precond):
    """sense_smooth_sensitivities (magnitude and normalised map of 4 coils, smoothed and
    recombined on the device) against the oracle's per-coil direct solves; in place too."""
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    n = int(np.prod(shape))
    _, m_t, m_r, _ = _fields(shape, 77)
    S = np.stack([_fields(shape, 90 + c)[0].ravel() * np.exp(0.5j * c) for c in range(4)],
                 axis=-1).astype(np.complex64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ref = oracle.smooth_sensitivities(shape, 0.5, m_t.ravel(), m_r.ravel(), S.astype(complex))
    out = torch.empty((n, 4), dtype=torch.complex64, device=dev)
    infos = native.sense_smooth_sensitivities(shape, 0.5, t(m_t.ravel()), t(m_r.ravel()), t(S),
                                              out, max_iter=20000, rel_tol=1e-7,
                                              precond=precond)
    assert len(infos) == 8 and all(i["rel_residual"] <= 1e-7 for i in infos)
    e = _rel(out.cpu().numpy(), ref)
    print(f"sensitivities {shape} {precond}: {[i['iters'] for i in infos]}, vs oracle {e:.2e}")
    assert e <= 1e-4
    inplace = t(S)
    native.sense_smooth_sensitivities(shape, 0.5, t(m_t.ravel()), t(m_r.ravel()), inplace,
                                      inplace, max_iter=20000, rel_tol=1e-7, precond=precond)
    assert _rel(inplace.cpu().numpy(), out.cpu().numpy()) <= 1e-6
