"""GPU parity of the tcgen05 tensor-core path against the FP64 oracle, through the C ABI.

Bars (relative L2 versus FP64): split hi+lo FP16 operands with FP32 accumulation <= 2e-5;
single FP16 <= 2e-3; CG with the split operator at equal iteration count <= 1e-4.
"""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

SPLIT, SINGLE = 2, 1
TOL = {SPLIT: 2e-5, SINGLE: 2e-3}
TOL_CG = 1e-4


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(dev)


CASES = {
    "sh3_24x24_c8_k1500_j": lambda: synthetic.small_2d(seed=1, matrix=24, n_coils=8,
                                                       n_samples=1500, order=3, with_j=True),
    "lin_20x20_c5_k1000": lambda: synthetic.small_2d(seed=2, matrix=20, n_coils=5,
                                                     n_samples=1000, order=1),
    "sh2_16x16_c32_k600": lambda: synthetic.small_2d(seed=3, matrix=16, n_coils=32,
                                                     n_samples=600, order=2, R=1),
    "sh3_12x12_c64_k300": lambda: synthetic.small_2d(seed=4, matrix=12, n_coils=64,
                                                     n_samples=300, order=3, R=1),
    "tiny_6x6_c1_k100": lambda: synthetic.small_2d(seed=5, matrix=6, n_coils=1, n_samples=100,
                                                   order=1, R=1),
    "sh3_40x40_c16_k5000": lambda: synthetic.small_2d(seed=8, matrix=40, n_coils=16,
                                                      n_samples=5000, order=3, R=2),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    import torch
    from paper_2604_09233_gb300 import native
    wl = CASES[request.param]()
    plan = native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j)
    yield wl, plan, torch.device("cuda:0")
    plan.close()


@pytest.mark.parametrize("prec", [SPLIT, SINGLE])
def test_tc_encode(case, prec):
    wl, plan, dev = case
    s = plan.encode(_t(wl.m_true, dev), prec=prec).cpu().numpy()
    ref = oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j)
    assert _rel(s, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [SPLIT, SINGLE])
def test_tc_adjoint(case, prec):
    wl, plan, dev = case
    rng = np.random.default_rng(9)
    y = (rng.normal(size=(wl.K, wl.C)) + 1j * rng.normal(size=(wl.K, wl.C))).astype(np.complex64)
    m = plan.adjoint(_t(y, dev), prec=prec).cpu().numpy()
    ref = oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y.astype(complex), j=wl.j)
    assert _rel(m, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [SPLIT, SINGLE])
def test_tc_normal(case, prec):
    wl, plan, dev = case
    q = plan.normal(_t(wl.m_true, dev), prec=prec).cpu().numpy()
    ref = oracle.normal(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j)
    assert _rel(q, ref) <= TOL[prec]


def test_tc_split_cg_equal_iteration_count(case):
    """Early iterations (5): the split tensor-core CG iterate equals the FP64 one within 1e-4,
    for every case (1 to 64 coils). Deeper, FP64 CG itself moves by 1e-4..1e-2 under product
    noise of the split operator's size (3e-6; tests/test_cg_sensitivity.py measures the
    effect), so at 10 iterations the check is on what the iterate is for: its distance to the
    ground-truth image must agree with FP64 CG's to 2% (5% for the one-coil 6x6 case, whose 36
    unknowns are the worst conditioned here)."""
    wl, plan, dev = case
    sigma = (oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j) + wl.noise).astype(np.complex64)
    n_early, n_deep = 5, 10
    x, info, _ = plan.cg(_t(sigma, dev), n_early, prec=SPLIT)
    ref = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), n_early, j=wl.j)
    assert info["iters"] == n_early and info["status"] == 0
    assert _rel(x.cpu().numpy(), ref["x"]) <= TOL_CG
    x, info, _ = plan.cg(_t(sigma, dev), n_deep, prec=SPLIT)
    ref = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), n_deep, j=wl.j)
    truth = wl.m_true * (wl.j if wl.j is not None else 1.0)
    e_gpu = _rel(x.cpu().numpy(), truth)
    e_ref = _rel(ref["x"], truth)
    print(f"{wl.name}: 10 it. to truth {e_gpu:.5f} vs FP64 {e_ref:.5f}")
    assert abs(e_gpu - e_ref) <= (5e-2 if wl.C == 1 else 2e-2) * e_ref


def test_tc_results_are_deterministic(case):
    wl, plan, dev = case
    m = _t(wl.m_true, dev)
    a = plan.normal(m, prec=SPLIT)
    for _ in range(4):
        b = plan.normal(m, prec=SPLIT)
        assert bool((a == b).all())


@pytest.mark.parametrize("matrix,n_samples", [(20, 1000), (12, 300), (40, 5000)])
def test_tc_no_reads_of_unwritten_device_memory(matrix, n_samples):
    """Freshly allocated device memory is poisoned with NaN first (allocate, fill, hand back
    to the CUDA allocator), so any read of a workspace element that no kernel wrote shows up. Small
    problems (fewer block pairs than SMs) once summed partial slots of CTAs with no work."""
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    poison = torch.full((1 << 28,), float("nan"), dtype=torch.float32, device=dev)  # 1 GiB
    del poison
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    wl = synthetic.small_2d(seed=2, matrix=matrix, n_coils=5, n_samples=n_samples, order=1)
    ref_s = oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true)
    ref_q = oracle.normal(wl.Kmat, wl.Rmat, wl.S, wl.m_true)
    with native.Plan(wl.Kmat, wl.Rmat, wl.S) as plan:
        m = _t(wl.m_true, dev)
        for prec in (SPLIT, SINGLE, 0):
            s = plan.encode(m, prec=prec).cpu().numpy()
            q = plan.normal(m, prec=prec).cpu().numpy()
            tol = TOL.get(prec, 1e-5)
            assert np.isfinite(s).all() and np.isfinite(q).all()
            assert _rel(s, ref_s) <= tol and _rel(q, ref_q) <= tol


@pytest.fixture(scope="module")
def target():
    import torch
    from paper_2604_09233_gb300 import native
    wl = synthetic.target_256()
    plan = native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j)
    yield wl, plan, torch.device("cuda:0")
    plan.close()


def test_tc_full_size_sampled(target):
    """2D 256x256, 32 coils, 35750 samples, 3rd-order terms: sampled rows / voxels of the
    split tensor-core E and E^H against the oracle, in the launch configuration the
    benchmark uses."""
    wl, plan, dev = target
    rng = np.random.default_rng(23)
    rows = np.sort(rng.choice(wl.K, 48, replace=False))
    s = plan.encode(_t(wl.m_true, dev), prec=SPLIT).cpu().numpy()
    ref = oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, rows=rows)
    assert _rel(s[rows], ref) <= TOL[SPLIT]
    y = (rng.normal(size=(wl.K, wl.C)) + 1j * rng.normal(size=(wl.K, wl.C))).astype(np.complex64)
    vox = np.sort(rng.choice(wl.L, 48, replace=False))
    m = plan.adjoint(_t(y, dev), prec=SPLIT).cpu().numpy()
    refm = oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y.astype(complex), vox=vox)
    assert _rel(m[vox], refm) <= TOL[SPLIT]


def test_tc_full_size_matches_fp32_path(target):
    """Whole-vector check at full size: the split tensor-core E^H E against the FP32
    CUDA-core E^H E (itself within 1e-5 of FP64 on sampled outputs)."""
    import torch
    wl, plan, dev = target
    rng = np.random.default_rng(29)
    u = _t(rng.normal(size=wl.L) + 1j * rng.normal(size=wl.L), dev)
    a = plan.normal(u, prec=SPLIT)
    b = plan.normal(u, prec=0)
    assert (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item() <= 3e-5
