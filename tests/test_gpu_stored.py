"""Stored-P mode (the paper's precomputed P, streamed from HBM) through the C ABI: the tiles
are computed with the pass kernel's own per-element arithmetic, so the split-FP16 results
must be bit-identical to on-the-fly generation."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

SPLIT, SINGLE = 2, 1


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _crandn(rng, *shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2.0)


@pytest.mark.parametrize("case", [dict(seed=1, matrix=24, n_coils=8, n_samples=1500, order=3,
                                       with_j=True),
                                  dict(seed=3, matrix=16, n_coils=32, n_samples=600, order=2),
                                  dict(seed=5, matrix=12, n_coils=3, n_samples=300, order=1)])
def test_stored_tiles_reproduce_on_the_fly_results(case):
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wl = synthetic.small_2d(**case)
    rng = np.random.default_rng(61)
    m = torch.from_numpy(_crandn(rng, wl.L).astype(np.complex64)).to(dev)
    y = torch.from_numpy(_crandn(rng, wl.K, wl.C).astype(np.complex64)).to(dev)
    sig = torch.from_numpy((oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j)
                            + wl.noise).astype(np.complex64)).to(dev)
    with native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j) as plan:
        def run():
            return [plan.encode(m, SPLIT), plan.adjoint(y, SPLIT), plan.normal(m, SPLIT),
                    plan.cg(sig, 6, prec=SPLIT)[0], plan.normal(m, SINGLE)]
        fly = run()
        native.sense_plan_store_p(plan.handle, True)
        st = run()
        native.sense_plan_store_p(plan.handle, False)
        again = run()
    for a, b in zip(fly[:4], st[:4]):
        assert torch.equal(a, b)
    for a, b in zip(fly, again):
        assert torch.equal(a, b)
    # single FP16 from the split's hi part: equal except where FP16 rounding ties
    assert _rel(st[4].cpu().numpy(), fly[4].cpu().numpy()) <= 1e-4
    assert _rel(st[4].cpu().numpy(), oracle.normal(wl.Kmat, wl.Rmat, wl.S, m.cpu().numpy(),
                                                   j=wl.j)) <= 2e-3


def test_stored_tiles_follow_a_new_b0_map():
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wl = synthetic.small_2d(seed=2, matrix=20, n_coils=5, n_samples=1000, order=1)
    Rm = wl.Rmat.copy()
    Rm[0] = 1.3 * Rm[0] - 25.0
    m = torch.from_numpy(wl.m_true.astype(np.complex64)).to(dev)
    with native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j) as plan:
        native.sense_plan_store_p(plan.handle, True)
        native.sense_plan_set_b0(plan.handle, Rm[0])
        a = plan.normal(m, SPLIT)
    with native.Plan(wl.Kmat, Rm, wl.S, wl.j) as fresh:
        b = fresh.normal(m, SPLIT)
    assert torch.equal(a, b)


def test_stored_tiles_full_size():
    """256x256, 32 coils, 35750 samples: the stored-tile E^H E equals the generated one bit
    for bit; prints both apply times."""
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wl = synthetic.target_256()
    m = torch.from_numpy(wl.m_true.astype(np.complex64)).to(dev)
    with native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j) as plan:
        def timed():
            out = plan.normal(m, SPLIT)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                plan.normal(m, SPLIT)
            e1.record()
            torch.cuda.synchronize()
            return out, e0.elapsed_time(e1) / 3
        a, t_fly = timed()
        native.sense_plan_store_p(plan.handle, True)
        b, t_st = timed()
        native.sense_plan_store_p(plan.handle, False)
    print(f"256x256 E^H E split: generated {t_fly:.2f} ms, stored {t_st:.2f} ms")
    assert torch.equal(a, b)
