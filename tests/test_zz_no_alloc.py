"""sense_encode_noalloc: E m for callers that cannot allocate device memory.

Hosts that reserve all GPU memory at start-up, or whose device memory belongs to another
framework's allocator, cannot create a plan or let a call allocate; this entry point keeps
its scratch in a fixed array inside the library. The test drives it through the C ABI and
compares it with the FP64 oracle's E (Eq. 4) and with the plan-based sense_encode (FP32
path), on two calls in a row, at the 1e-5 relative tolerance of the FP32 parity tests. The
cases cover a ragged last voxel round (L not a multiple of the 64 voxels staged per round),
sample counts that are not multiples of the 128 samples per block, splits of several rounds
with an uneven last split, 48 coils (the 64-coil kernel), with and without the intensity
correction j. It lives in its own file that pytest collects last, and passes alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = {
    # 20x20 = 400 voxels: 6 full rounds of 64 and a tail of 16; 1000 samples = 7 blocks + 104
    "20x20_c8_k1000_o3_j": dict(matrix=20, n_coils=8, n_samples=1000, order=3, with_j=True),
    "20x20_c5_k777_o1": dict(matrix=20, n_coils=5, n_samples=777, order=1, with_j=False),
    # 39x39 = 1521 voxels, 40000 samples: 6 splits of 256 voxels (4 rounds), the last 241
    "39x39_c8_k40000_o2_j": dict(matrix=39, n_coils=8, n_samples=40000, order=2, with_j=True),
    # 48 coils run the 64-coil kernel
    "20x20_c48_k600_o2": dict(matrix=20, n_coils=48, n_samples=600, order=2, with_j=False),
    "24x24_c32_k1500_o3": dict(matrix=24, n_coils=32, n_samples=1500, order=3, with_j=False),
}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_encode_matches_oracle_and_plan_encode_twice(name):
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wl = synthetic.small_2d(seed=31, **CASES[name])
    ref = oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j)
    m = torch.from_numpy(wl.m_true.astype(np.complex64)).to(dev)
    with native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j) as plan:
        via_plan = plan.encode(m).cpu().numpy()
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
    e_or = _rel(outs[0], ref)
    e_plan = _rel(outs[0], via_plan)
    print(f"{name}: vs oracle {e_or:.2e}, vs plan encode {e_plan:.2e}")
    for out in outs:
        assert np.isfinite(out).all()
        assert _rel(out, ref) <= TOL
        assert _rel(out, via_plan) <= TOL
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
