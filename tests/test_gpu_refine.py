"""Residual replacement in the tensor-core CG (refine_every > 0) against the FP64 oracle.

Every refine_every iterations the recursively updated residual is replaced by the true one,
r = b - E^H E x, computed with the FP32 CUDA-core operator (b = E^H s then also comes from the
FP32 operator), and the step ratio and the history row are recomputed from it (van der Vorst
and Ye's residual replacement, the reading of the north star's "outer iterative refinement
with residuals from an FP32 E^H E"). Checks:
  (a) the refined CG iterate after 5 iterations against the oracle's CG (the CG loop of
      Alg. 1, Fig. 2): split <= 1e-4, single FP16 <= 2e-3 (its operator bar); after 8, where
      FP64 CG itself moves by ~5e-5 under product noise of the split operator's size
      (tests/test_cg_sensitivity.py) and a replacement changes the recurrence itself:
      split <= 5e-4, single <= 5e-3;
  (b) after a replacement the history's ||r_n|| is the true residual ||b - E^H E x_n|| of the
      recorded iterate, evaluated by the oracle, to FP32 precision (2e-6 of ||b||), while
      without replacement the recursive residual of the single-FP16 CG drifts from it;
  (c) the tolerance stop (||r_n|| <= tol ||E^H s||) ends at the oracle's iteration."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

SPLIT, SINGLE = 2, 1
TOL = {SPLIT: 1e-4, SINGLE: 2e-3}
TOL_8 = {SPLIT: 5e-4, SINGLE: 5e-3}

CASES = {
    "sh3_24x24_c8_k1500_j": lambda: synthetic.small_2d(seed=1, matrix=24, n_coils=8,
                                                       n_samples=1500, order=3, with_j=True),
    "sh2_20x20_c32_k2000": lambda: synthetic.small_2d(seed=3, matrix=20, n_coils=32,
                                                      n_samples=2000, order=2, R=2),
}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(dev)


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    import torch
    from paper_2604_09233_gb300 import native
    wl = CASES[request.param]()
    sigma = (oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j) + wl.noise).astype(
        np.complex64)
    plan = native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j)
    ref = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), 8, j=wl.j, apply_j=False,
                    iterates=True, history=True)
    yield wl, sigma, plan, ref, torch.device("cuda:0")
    plan.close()


@pytest.mark.parametrize("prec", [SPLIT, SINGLE])
@pytest.mark.parametrize("k", [1, 4])
def test_refined_cg_matches_oracle(case, prec, k):
    wl, sigma, plan, ref, dev = case
    for n in (5, 8):
        x, info, hist = plan.cg(_t(sigma, dev), n, prec=prec, refine_every=k, apply_j=False)
        e = _rel(x.cpu().numpy(), ref["iterates"][n])
        print(f"{wl.name} prec {prec} refine_every {k}: {n} it. {e:.2e}")
        assert info["iters"] == n and info["status"] == 0
        assert e <= (TOL if n == 5 else TOL_8)[prec]


@pytest.mark.parametrize("prec", [SPLIT, SINGLE])
def test_replaced_residual_is_the_true_residual(case, prec):
    import torch
    from paper_2604_09233_gb300 import native
    wl, sigma, plan, _, dev = case
    n_it, k = 6, 2
    b = oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), j=wl.j)
    nb = np.linalg.norm(b)
    drift = {}
    for refine in (k, 0):
        its = torch.empty((n_it + 1, wl.L), dtype=torch.complex64, device=dev)
        info, hist = native.sense_cg_solve_iterates(plan.handle, _t(sigma, dev), its, n_it,
                                                    prec=prec, refine_every=refine,
                                                    apply_j=False)
        torch.cuda.synchronize()
        X = its.cpu().numpy()
        gaps = []
        for n in range(1, n_it):
            true = np.linalg.norm(b - oracle.normal(wl.Kmat, wl.Rmat, wl.S, X[n], j=wl.j))
            gaps.append(abs(hist[n, 0] - true) / nb)
            if refine and n % k == 0:
                # replaced at iterations k, 2k, ... (not after the last one)
                assert gaps[-1] <= 2e-6, (n, gaps[-1])
        drift[refine] = max(gaps)
        print(f"{wl.name} prec {prec} refine_every {refine}: max | ||r_n|| - true | / ||b|| "
              f"= {drift[refine]:.2e}")
    if prec == SINGLE:
        # without replacement the single-FP16 recursion drifts from the true residual
        assert drift[0] > 2e-6


def test_refined_cg_tolerance_stop(case):
    wl, sigma, plan, ref, dev = case
    full = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), 40, j=wl.j, history=True)
    r = full["history"][:, 0]
    tol = float(np.sqrt(r[5] * r[6]) / r[0])       # between iterations 5 and 6
    x, info, _ = plan.cg(_t(sigma, dev), 40, prec=SPLIT, refine_every=2, rel_tol=tol)
    assert info["iters"] == 6 and info["status"] == 0
    x6 = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), 6, j=wl.j)["x"]
    assert _rel(x.cpu().numpy(), x6) <= TOL[SPLIT]
