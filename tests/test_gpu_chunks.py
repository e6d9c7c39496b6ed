"""The chunked single-problem schedule of the tensor-core passes against the FP64 oracle.

Chunk by chunk of streamed blocks, every CTA takes an equal share of the chunk's (row block,
streamed block) pairs, and the partial slots of a row block are indexed by chunk and CTA. The
schedule only changes which CTA sums which pairs, so E, E^H and E^H E must stay within the
split-FP16 bar of the oracle (Eq. 4, Eq. 5), and within half that bar of the one-chunk result:
a chunk ends every run, so the tensor-memory accumulation chains get shorter (one block per chain
at width 1 against up to four by default), and the biased FP32 accumulation of the tensor cores
moves the result by a few 1e-6 (2.75e-6 measured for E^H E at width 1). Forced chunk widths
of 1 block and ragged widths (last chunk narrower) are used on problems the oracle finishes in
seconds, including a grid that the chunking narrows (a chunk must give each CTA a pair), then
the automatic width is restored."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

SPLIT = 2
TOL = 2e-5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(dev)


CASES = {
    # 13 voxel blocks x 40 sample blocks, 16 coils, 3rd order
    "sh3_40x40_c16_k5000": lambda: synthetic.small_2d(seed=8, matrix=40, n_coils=16,
                                                      n_samples=5000, order=3, R=2),
    # 5 voxel blocks x 12 sample blocks with j, 8 coils
    "sh3_24x24_c8_k1500_j": lambda: synthetic.small_2d(seed=1, matrix=24, n_coils=8,
                                                       n_samples=1500, order=3, with_j=True),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    import torch
    from paper_2604_09233_gb300 import native
    wl = CASES[request.param]()
    plan = native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j)
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(21)
    y = (rng.normal(size=(wl.K, wl.C)) + 1j * rng.normal(size=(wl.K, wl.C))).astype(np.complex64)
    ref = {"E": oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j),
           "EH": oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y.astype(complex), j=wl.j),
           "EHE": oracle.normal(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j)}

    def run():
        m = _t(wl.m_true, dev)
        return {"E": plan.encode(m, prec=SPLIT).cpu().numpy(),
                "EH": plan.adjoint(_t(y, dev), prec=SPLIT).cpu().numpy(),
                "EHE": plan.normal(m, prec=SPLIT).cpu().numpy()}

    one = run()
    yield wl, plan, ref, one, run
    plan.close()


@pytest.mark.parametrize("chunk", [1, 2, 3, 7])
def test_forced_chunks_match_oracle_and_one_chunk(case, chunk):
    from paper_2604_09233_gb300 import native
    wl, plan, ref, one, run = case
    native.sense_plan_set_tuning(plan.handle, inner_chunk=chunk)
    try:
        assert native.sense_plan_get_tuning(plan.handle)["inner_chunk"] == chunk
        got = run()
        for k in ("E", "EH", "EHE"):
            assert _rel(got[k], ref[k]) <= TOL, (k, chunk)
            assert _rel(got[k], one[k]) <= TOL / 2, (k, chunk)
    finally:
        native.sense_plan_set_tuning(plan.handle)
    again = run()
    for k in ("E", "EH", "EHE"):
        assert np.array_equal(again[k], one[k]), k


def test_forced_chunks_with_a_small_grid(case):
    """A chunk width and a grid together: the layout keeps every CTA range non-empty."""
    from paper_2604_09233_gb300 import native
    wl, plan, ref, one, run = case
    native.sense_plan_set_tuning(plan.handle, inner_chunk=2, grid=7)
    try:
        got = run()
        for k in ("E", "EH", "EHE"):
            assert _rel(got[k], ref[k]) <= TOL, k
    finally:
        native.sense_plan_set_tuning(plan.handle)


def test_negative_chunk_is_rejected(case):
    from paper_2604_09233_gb300 import native
    wl, plan, ref, one, run = case
    with pytest.raises(native.SenseError):
        native.sense_plan_set_tuning(plan.handle, inner_chunk=-1)
    assert native.sense_plan_get_tuning(plan.handle)["inner_chunk"] == 0


def test_stored_tiles_under_forced_chunks(case):
    """Stored-P mode with a forced chunk width: the tiles are kept per (row block, streamed
    block) pair, so the stored passes reproduce the generated passes of the same schedule bit
    for bit, and stay within the bar of the oracle."""
    from paper_2604_09233_gb300 import native
    wl, plan, ref, one, run = case
    native.sense_plan_set_tuning(plan.handle, inner_chunk=3)
    try:
        gen = run()
        native.sense_plan_store_p(plan.handle, True)
        try:
            st = run()
        finally:
            native.sense_plan_store_p(plan.handle, False)
        for k in ("E", "EH", "EHE"):
            assert np.array_equal(st[k], gen[k]), k
            assert _rel(st[k], ref[k]) <= TOL, k
    finally:
        native.sense_plan_set_tuning(plan.handle)
