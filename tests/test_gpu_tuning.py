"""Segment length and grid of the single-problem tensor-core passes against the FP64 oracle.

A pass accumulates at most seg_len blocks in the tensor-memory accumulators before the generator
warps drain them into FP32 running sums; a run (one CTA's piece of a row block) ends with a
drain and the run's output. Longer segments trade accuracy for fewer drains: the tensor cores
accumulate in FP32 with a rounding bias that grows with the chain of MMAs, so the split-FP16
bar of 2e-5 is kept up to its default length of 4, and longer segments (here up to 40 blocks in
one chain) are held to 5e-5 (2.5e-5 measured for E^H E with 64-block segments on 3 CTAs, where
the E^H runs span 40 sample blocks); single-FP16 tiles (default length 16) stay far inside their
2e-3 bar at any length. Split-FP16 tiles are generated by all 16 generator warps on every stage
and drained by all of them; single-FP16 tiles by two groups of 8 warps on alternating stages,
drained by the first group. Segment lengths of 1 (a drain after every block), odd lengths
(segments ending on either stage pattern of a run) and 64 (one segment per run), with the
default grid and with a narrow grid (long runs, several segments each), must all keep E, E^H and
E^H E within the precision's bar (for that segment length) of the oracle (Eq. 4, Eq. 5) and of
the default schedule. Out-of-range values are rejected and leave the tuning unchanged."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

SPLIT, SINGLE = 2, 1
TOL = {SPLIT: 2e-5, SINGLE: 2e-3}
DEFAULT_SEG = 4


def _tol(prec, seg_len):
    if prec == SPLIT and seg_len > DEFAULT_SEG:
        return 5e-5
    return TOL[prec]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(dev)


CASES = {
    # 13 voxel blocks x 40 sample blocks, 16 coils, 3rd order
    "sh3_40x40_c16_k5000": lambda: synthetic.small_2d(seed=8, matrix=40, n_coils=16,
                                                      n_samples=5000, order=3, R=2),
    # 5 voxel blocks x 12 sample blocks with j, 32 coils
    "sh2_24x24_c32_k1500_j": lambda: synthetic.small_2d(seed=4, matrix=24, n_coils=32,
                                                        n_samples=1500, order=2, with_j=True),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    import torch
    from paper_2604_09233_gb300 import native
    wl = CASES[request.param]()
    plan = native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j)
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(33)
    y = (rng.normal(size=(wl.K, wl.C)) + 1j * rng.normal(size=(wl.K, wl.C))).astype(np.complex64)
    ref = {"E": oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j),
           "EH": oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y.astype(complex), j=wl.j),
           "EHE": oracle.normal(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j)}

    def run(prec):
        m = _t(wl.m_true, dev)
        return {"E": plan.encode(m, prec=prec).cpu().numpy(),
                "EH": plan.adjoint(_t(y, dev), prec=prec).cpu().numpy(),
                "EHE": plan.normal(m, prec=prec).cpu().numpy()}

    default = {p: run(p) for p in (SPLIT, SINGLE)}
    yield plan, ref, default, run
    plan.close()


@pytest.mark.parametrize("prec", [SPLIT, SINGLE])
@pytest.mark.parametrize("seg_len,grid", [(1, 0), (3, 0), (7, 0), (64, 0), (1, 5), (3, 5),
                                          (64, 3)])
def test_segment_length_and_grid_match_oracle(case, prec, seg_len, grid):
    from paper_2604_09233_gb300 import native
    plan, ref, default, run = case
    native.sense_plan_set_tuning(plan.handle, seg_len=seg_len, grid=grid)
    try:
        t = native.sense_plan_get_tuning(plan.handle)
        assert t["seg_len"] == seg_len
        got = run(prec)
        tol = _tol(prec, seg_len)
        for k in ("E", "EH", "EHE"):
            assert _rel(got[k], ref[k]) <= tol, (k, prec, seg_len, grid)
            assert _rel(got[k], default[prec][k]) <= tol, (k, prec, seg_len, grid)
    finally:
        native.sense_plan_set_tuning(plan.handle)
    # the default schedule again reproduces its results bit for bit
    again = run(prec)
    for k in ("E", "EH", "EHE"):
        assert np.array_equal(again[k], default[prec][k]), k


@pytest.mark.parametrize("kw", [dict(seg_len=-1), dict(seg_len=65), dict(grid=-1)])
def test_out_of_range_tuning_is_rejected(case, kw):
    from paper_2604_09233_gb300 import native
    plan, ref, default, run = case
    before = native.sense_plan_get_tuning(plan.handle)
    with pytest.raises(native.SenseError):
        native.sense_plan_set_tuning(plan.handle, **kw)
    assert native.sense_plan_get_tuning(plan.handle) == before
