"""sense_encode_noalloc: E m for callers that cannot allocate device memory.

Hosts that reserve all GPU memory at start-up, or whose device memory belongs to another
framework's allocator, cannot create a plan or let a call allocate; this entry point keeps
its scratch in a fixed array inside the library. The test drives it through the C ABI and
compares it with the plan-based sense_encode (FP32 path) on two calls in a row, at the
1e-5 relative tolerance of the FP32 parity tests. It lives in its own file that pytest
collects last, and passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("coils,order,with_j", [(8, 3, True), (5, 1, False), (32, 2, False)])
def test_noalloc_encode_matches_plan_encode_twice(coils, order, with_j):
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wl = synthetic.small_2d(seed=31, matrix=24, n_coils=coils, n_samples=1500, order=order,
                            with_j=with_j)
    m = torch.from_numpy(wl.m_true.astype(np.complex64)).to(dev)
    with native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j) as plan:
        ref = plan.encode(m).cpu().numpy()
    Km = torch.from_numpy(np.ascontiguousarray(wl.Kmat)).to(dev)
    Rm = torch.from_numpy(np.ascontiguousarray(wl.Rmat)).to(dev)
    S = torch.from_numpy(np.ascontiguousarray(wl.S, np.complex64)).to(dev)
    j = None if wl.j is None else torch.from_numpy(wl.j.astype(np.float32)).to(dev)
    outs = []
    for _ in range(2):
        s = torch.full((wl.K, wl.C), float("nan"), dtype=torch.complex64, device=dev)
        native.sense_encode_noalloc(Km, Rm, S, m, s, j=j)
        torch.cuda.synchronize()
        outs.append(s.cpu().numpy())
    for out in outs:
        assert np.isfinite(out).all()
        assert _rel(out, ref) <= TOL
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    tiny = torch.zeros(8, dtype=torch.complex64, device=dev)
    kd = torch.zeros(8, dtype=torch.float64, device=dev)
    lib = native._lib
    # K x 32 padded coils = 2^21 + 32 complex values: one more sample row than fits
    K = (1 << 21) // 32 + 1
    rc = lib.sense_encode_noalloc(4, K, 32, 1, kd.data_ptr(), kd.data_ptr(), tiny.data_ptr(),
                                  None, tiny.data_ptr(), tiny.data_ptr(), None)
    assert rc == -1
    assert b"scratch" in lib.sense_last_error()
