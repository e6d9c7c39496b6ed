"""Failure paths of the GPU path, in forms that fault, trap or hang nothing:
  - a bounded wait that runs out: the plan's wait limit is set to 2 ms and the loader warp of
    CTA 0 is told to withhold the arrival of its first stage, so the other warps' waits on it
    run out; the kernel records the failure, completes what it issued, frees its tensor
    memory and returns, and the call reports SENSE_ETIMEOUT; the same plan with the hold
    cleared, and a fresh plan, then match the FP64 oracle again;
  - coil data with a NaN: CG reports SENSE_ENONFINITE in its status, with a finite result
    (the last finite iterate, here the start rho = 0);
  - all-zero coil data: the solution is 0; CG stops at once with SENSE_OK and no NaN."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

SPLIT = 2
ETIMEOUT, ENONFINITE = -8, -4


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(dev)


@pytest.fixture(scope="module")
def wl():
    return synthetic.small_2d(seed=2, matrix=20, n_coils=8, n_samples=1000, order=3)


def test_wait_time_out_is_reported_and_recovers(wl):
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    m = _t(wl.m_true, dev)
    ref = oracle.normal(wl.Kmat, wl.Rmat, wl.S, wl.m_true)
    sigma = (oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true) + wl.noise).astype(np.complex64)
    ref_cg = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), 5)["x"]
    with native.Plan(wl.Kmat, wl.Rmat, wl.S) as plan:
        h = plan.handle
        native.sense_plan_set_tuning(h, wait_limit_us=2000, test_hold_stage=1)
        assert native.sense_plan_get_tuning(h)["test_hold_stage"] == 1
        out = torch.empty_like(m)
        native.sense_normal_op(h, SPLIT, m, out)
        with pytest.raises(native.SenseError) as e:
            native.sense_plan_sync(h)
        assert e.value.code == ETIMEOUT
        assert "timed out" in str(e.value)
        # a synchronising solve reports it directly
        x = torch.empty_like(m)
        with pytest.raises(native.SenseError) as e:
            native.sense_cg_solve(h, _t(sigma, dev), x, 3, prec=SPLIT)
        assert e.value.code == ETIMEOUT
        # hold cleared (default limit): the same plan is correct again
        native.sense_plan_set_tuning(h)
        q = plan.normal(m, prec=SPLIT).cpu().numpy()
        assert _rel(q, ref) <= 2e-5
        x, info, _ = plan.cg(_t(sigma, dev), 5, prec=SPLIT)
        assert info["status"] == 0 and _rel(x.cpu().numpy(), ref_cg) <= 1e-4
    with native.Plan(wl.Kmat, wl.Rmat, wl.S) as plan:
        q = plan.normal(m, prec=SPLIT).cpu().numpy()
        assert _rel(q, ref) <= 2e-5


@pytest.mark.parametrize("prec", [0, SPLIT])
def test_nan_in_coil_data_reports_nonfinite(wl, prec):
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    sigma = (oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true) + wl.noise).astype(np.complex64)
    sigma[17, 3] = np.nan
    with native.Plan(wl.Kmat, wl.Rmat, wl.S) as plan:
        x, info, hist = plan.cg(_t(sigma, dev), 5, prec=prec)
        xn = x.cpu().numpy()
    assert info["status"] == ENONFINITE
    assert info["iters"] == 0
    assert np.isfinite(xn).all() and not xn.any()


@pytest.mark.parametrize("prec", [0, SPLIT])
def test_zero_coil_data_stops_cleanly(wl, prec):
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    with native.Plan(wl.Kmat, wl.Rmat, wl.S) as plan:
        s = torch.zeros((wl.K, wl.C), dtype=torch.complex64, device=dev)
        x, info, hist = plan.cg(s, 5, prec=prec)
        xn = x.cpu().numpy()
    assert info["status"] == 0 and info["iters"] == 0
    assert np.isfinite(hist).all() and hist[0, 0] == 0.0
    assert not xn.any()
