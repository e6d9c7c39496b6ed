"""CG from a supplied start rho_0 (sense_cg_opts.use_x0) and resumed solves, against the
FP64 oracle's CG from the same start (the CG loop of Alg. 1, Fig. 2, with r_0 = E^H s -
E^H E rho_0 and p_0 = r_0; its pins fix every iterate as the minimiser over the shifted
Krylov space)."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 2: 1e-4}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(dev)


@pytest.fixture(scope="module")
def case():
    import torch
    from paper_2604_09233_gb300 import native
    wl = synthetic.small_2d(seed=1, matrix=24, n_coils=8, n_samples=1500, order=3, with_j=True)
    sigma = (oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j) + wl.noise).astype(
        np.complex64)
    plan = native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j)
    yield wl, sigma, plan, torch.device("cuda:0")
    plan.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_cg_from_x0_matches_oracle(case, prec):
    wl, sigma, plan, dev = case
    rng = np.random.default_rng(8)
    x0 = (wl.m_true + 0.2 * (rng.normal(size=wl.L) + 1j * rng.normal(size=wl.L))).astype(
        np.complex64)
    x, info, hist = plan.cg(_t(sigma, dev), 5, prec=prec, x0=_t(x0, dev))
    ref = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), 5, j=wl.j, x0=x0,
                    history=True)
    assert info["iters"] == 5 and info["status"] == 0
    assert _rel(x.cpu().numpy(), ref["x"]) <= TOL[prec]
    hr = ref["history"]
    # row 0 is the start: ||r_0||, ||rho_0||, ||E rho_0 - s||
    assert np.allclose(hist[0], hr[0], rtol=1e-4)
    assert np.allclose(hist[:, 0], hr[:, 0], rtol=1e-3, atol=1e-6 * hr[0, 0])


@pytest.mark.parametrize("prec", [0, 2])
def test_resumed_solve_matches_oracle(case, prec):
    """3 iterations, then 2 more from the result (CG restarted there, p_0 = r_0)."""
    wl, sigma, plan, dev = case
    s = _t(sigma, dev)
    x3, _, _ = plan.cg(s, 3, prec=prec, apply_j=False)
    x5, info, _ = plan.cg(s, 2, prec=prec, x0=x3)
    r3 = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), 3, j=wl.j, apply_j=False)
    r5 = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), 2, j=wl.j, x0=r3["x"])
    assert info["iters"] == 2
    assert _rel(x5.cpu().numpy(), r5["x"]) <= TOL[prec]


def test_iterates_from_x0(case):
    import torch
    from paper_2604_09233_gb300 import native
    wl, sigma, plan, dev = case
    rng = np.random.default_rng(9)
    x0 = (0.5 * wl.m_true + 0.1 * rng.normal(size=wl.L)).astype(np.complex64)
    n = 4
    its = torch.zeros((n + 1, wl.L), dtype=torch.complex64, device=dev)
    its[0] = _t(x0, dev)
    info, _ = native.sense_cg_solve_iterates(plan.handle, _t(sigma, dev), its, n, prec=2,
                                             apply_j=False, use_x0=True)
    torch.cuda.synchronize()
    ref = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), n, j=wl.j, apply_j=False,
                    x0=x0, iterates=True)["iterates"]
    X = its.cpu().numpy()
    assert np.array_equal(X[0], x0)
    for k in range(1, n + 1):
        assert _rel(X[k], ref[k]) <= 1e-4, k


def test_start_at_the_solution_stops_at_once(case):
    """A start that already meets the tolerance ends the solve after 0 iterations."""
    wl, sigma, plan, dev = case
    s = _t(sigma, dev)
    x40, _, _ = plan.cg(s, 60, prec=0, apply_j=False)
    _, _, hist40 = plan.cg(s, 1, prec=0, apply_j=False, x0=x40)
    nb = np.linalg.norm(oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), j=wl.j))
    tol = 2.0 * hist40[0, 0] / nb          # twice the start's relative residual
    x, info, _ = plan.cg(s, 60, prec=0, apply_j=False, x0=x40, rel_tol=tol)
    assert info["iters"] == 0 and info["status"] == 0
    assert np.array_equal(x.cpu().numpy(), x40.cpu().numpy())
