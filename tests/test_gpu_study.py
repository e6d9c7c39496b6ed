"""Iterate recording and the stopping-rule study through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def test_recorded_iterates_match_the_oracle_and_the_plain_solve():
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wl = synthetic.small_2d(seed=1, matrix=24, n_coils=8, n_samples=1500, order=3, with_j=True)
    sigma = (oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j) + wl.noise).astype(np.complex64)
    n = 8
    with native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j) as plan:
        s = torch.from_numpy(sigma).to(dev)
        X = torch.full((n + 1, wl.L), float("nan"), dtype=torch.complex64, device=dev)
        info, hist = native.sense_cg_solve_iterates(plan.handle, s, X, n)
        x, info2, hist2 = plan.cg(s, n)
        X = X.cpu().numpy()
    ref = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), n, j=wl.j, iterates=True)
    its = ref["iterates"] * wl.j[None, :]        # the recorded rows carry the j of the result
    assert np.all(X[0] == 0)
    for k in range(1, 6):
        assert _rel(X[k], its[k]) <= 1e-4, k
    assert np.array_equal(X[n], x.cpu().numpy())
    assert np.array_equal(hist, hist2) and info == info2


def test_stopping_study_on_the_32x32_configuration():
    from paper_2604_09233_gb300.stopping import study
    wl = synthetic.plain_32()
    out, series = study(wl, n_iter=60, prec="fp32", noise_scale=10.0)
    print(out)
    assert out["iterations"] == 60
    assert np.all(np.isfinite(series["rel_error"])) and np.all(np.isfinite(series["ssim"]))
    e = series["rel_error"]
    assert out["error_minimum"]["rel_error"] == pytest.approx(e.min())
    assert 0 < out["lcurve_corner"]["iteration"] < 60
    assert series["ssim"][0] < out["ssim_peak"]["ssim"] <= 1.0
