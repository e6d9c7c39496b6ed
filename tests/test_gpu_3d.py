"""3D stack-of-spirals problems (the 3D configuration: 96x96x48, 32 coils, 62400 samples,
2nd-order field terms): operators and CG against the FP64 oracle through the C ABI, on a
small volume in full and on the full-size volume on sampled rows and voxels."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tc_split": 2e-5, "tc_fp16": 2e-3}


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _crandn(rng, *shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2.0)


@pytest.fixture(scope="module")
def small():
    from paper_2604_09233_gb300 import native
    wl = synthetic.small_3d()
    plan = native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j)
    yield wl, plan
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "tc_split", "tc_fp16"])
def test_small_volume_operators(small, prec):
    import torch
    from paper_2604_09233_gb300 import native
    wl, plan = small
    p = native.PRECISIONS[prec]
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(31)
    m = _crandn(rng, wl.L).astype(np.complex64)
    y = _crandn(rng, wl.K, wl.C).astype(np.complex64)
    s = plan.encode(torch.from_numpy(m).to(dev), p).cpu().numpy()
    x = plan.adjoint(torch.from_numpy(y).to(dev), p).cpu().numpy()
    q = plan.normal(torch.from_numpy(m).to(dev), p).cpu().numpy()
    e = [_rel(s, oracle.encode(wl.Kmat, wl.Rmat, wl.S, m)),
         _rel(x, oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y)),
         _rel(q, oracle.normal(wl.Kmat, wl.Rmat, wl.S, m))]
    print(f"3D small {prec}: E {e[0]:.2e}  E^H {e[1]:.2e}  E^H E {e[2]:.2e}")
    assert max(e) <= TOL[prec]


def test_small_volume_cg(small):
    import torch
    wl, plan = small
    dev = torch.device("cuda:0")
    sigma = (oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true) + wl.noise).astype(np.complex64)
    from paper_2604_09233_gb300 import native
    x, info, _ = plan.cg(torch.from_numpy(sigma).to(dev), 5, prec=native.SENSE_PREC_TC_SPLIT)
    ref = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma.astype(complex), 5)["x"]
    e = _rel(x.cpu().numpy(), ref)
    print(f"3D small CG (5 iterations, split): {e:.2e}")
    assert info["iters"] == 5 and e <= 1e-4


def test_full_volume_sampled_rows_and_voxels():
    """96x96x48, 32 coils, 62400 samples: E on 16 random sample rows and E^H on 16 random
    voxels (tensor-core split path) against the oracle computed one row / voxel at a time;
    E^H E Hermitian and positive on random vectors."""
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wl = synthetic.stack_3d()
    rng = np.random.default_rng(32)
    p = native.SENSE_PREC_TC_SPLIT
    with native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j) as plan:
        m = wl.m_true.astype(np.complex64)
        s = plan.encode(torch.from_numpy(m).to(dev), p).cpu().numpy()
        rows = np.sort(rng.choice(wl.K, 16, replace=False))
        e_rows = _rel(s[rows], oracle.encode(wl.Kmat, wl.Rmat, wl.S, m, rows=rows))
        y = _crandn(rng, wl.K, wl.C).astype(np.complex64)
        x = plan.adjoint(torch.from_numpy(y).to(dev), p).cpu().numpy()
        vox = np.sort(rng.choice(wl.L, 16, replace=False))
        e_vox = _rel(x[vox], oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y, vox=vox))
        a = torch.from_numpy(_crandn(rng, wl.L).astype(np.complex64)).to(dev)
        b = torch.from_numpy(_crandn(rng, wl.L).astype(np.complex64)).to(dev)
        Aa, Ab = plan.normal(a, p), plan.normal(b, p)
        lhs = torch.vdot(b, Aa).item()
        rhs = torch.vdot(Ab, a).item()
        herm = abs(lhs - rhs) / abs(lhs)
        pos = torch.vdot(a, Aa).item()
    print(f"3D full: E rows {e_rows:.2e}, E^H voxels {e_vox:.2e}, Hermitian {herm:.2e}")
    assert e_rows <= TOL["tc_split"] and e_vox <= TOL["tc_split"]
    assert herm <= 1e-5 and pos.real > 0 and abs(pos.imag) <= 1e-5 * pos.real
