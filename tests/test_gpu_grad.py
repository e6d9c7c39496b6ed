"""B0-map and input gradients through the C ABI against the FP64 oracle and central
finite differences of the oracle's own forward (the oracle gradients are pinned by
finite differences in test_oracle_pins.py)."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL_PRIM = {"fp32": 1e-5, "tc_split": 5e-5, "tc_fp16": 5e-3}
TOL_AUTOGRAD = 2e-5
TOL_CG_GRAD = 2e-4


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _crandn(rng, *shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2.0)


def _problem(seed=1, matrix=24, coils=8, samples=1500, order=3, with_j=True):
    wl = synthetic.small_2d(seed=seed, matrix=matrix, n_coils=coils, n_samples=samples,
                            order=order, with_j=with_j)
    # the B0 map as the float32 tensor the autograd layer receives; the oracle uses the same
    Rm = wl.Rmat.copy()
    Rm[0] = Rm[0].astype(np.float32).astype(np.float64)
    return wl, Rm


@pytest.mark.parametrize("prec", ["fp32", "tc_split", "tc_fp16"])
def test_grad_b0_primitive_matches_oracle(prec):
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wl, Rm = _problem()
    rng = np.random.default_rng(11)
    m = _crandn(rng, wl.L).astype(np.complex64)
    g = _crandn(rng, wl.K, wl.C).astype(np.complex64)
    with native.Plan(wl.Kmat, Rm, wl.S, wl.j) as plan:
        p = native.PRECISIONS[prec]
        gw = torch.empty(wl.L, dtype=torch.float32, device=dev)
        z = torch.empty(wl.L, dtype=torch.complex64, device=dev)
        native.sense_grad_b0(plan.handle, p, torch.from_numpy(m).to(dev),
                             torch.from_numpy(g).to(dev), gw, z=z)
        native.sense_plan_sync(plan.handle)
        # E^H backward: a = h (upstream of x), y the input of E^H
        h = _crandn(rng, wl.L).astype(np.complex64)
        gw2 = np.empty(wl.L, np.float32)              # host output: staged path
        native.sense_grad_b0(plan.handle, p, h, g, gw2)
    ref = oracle.grad_omega(wl.Kmat, Rm, wl.S, m, g, j=wl.j)
    e1 = _rel(gw.cpu().numpy(), ref)
    e2 = _rel(z.cpu().numpy(), oracle.adjoint(wl.Kmat, Rm, wl.S, g, j=wl.j))
    e3 = _rel(gw2, oracle.grad_omega_adjoint(wl.Kmat, Rm, wl.S, g, h, j=wl.j))
    print(f"grad_b0 {prec}: E-backward {e1:.2e}  z {e2:.2e}  E^H-backward {e3:.2e}")
    assert e1 <= TOL_PRIM[prec] and e3 <= TOL_PRIM[prec]
    assert e2 <= TOL_PRIM[prec]


def test_autograd_encode_against_oracle_and_central_differences():
    """Loss 0.5 ||E(m; omega) - d||^2: gradients w.r.t. m and omega; omega also against
    central differences (step 1e-3 rad/s) of the oracle's loss on 64 random voxels."""
    import torch
    from paper_2604_09233_gb300.autograd import SenseOperator
    dev = torch.device("cuda:0")
    wl, Rm = _problem()
    rng = np.random.default_rng(12)
    m0 = (wl.m_true + 0.1 * _crandn(rng, wl.L)).astype(np.complex64)
    d = (oracle.encode(wl.Kmat, Rm, wl.S, wl.m_true, j=wl.j) + 0.05 * _crandn(rng, wl.K, wl.C))
    d = d.astype(np.complex64)
    op = SenseOperator(wl.Kmat, wl.Rmat, wl.S, wl.j, prec="fp32")
    m = torch.from_numpy(m0).to(dev).requires_grad_(True)
    omega = torch.from_numpy(Rm[0].astype(np.float32)).to(dev).requires_grad_(True)
    r = op.E(m, omega) - torch.from_numpy(d).to(dev)
    loss = 0.5 * (r.real ** 2 + r.imag ** 2).sum()
    loss.backward()
    g = oracle.encode(wl.Kmat, Rm, wl.S, m0, j=wl.j) - d
    gm_ref = oracle.adjoint(wl.Kmat, Rm, wl.S, g, j=wl.j)
    gw_ref = oracle.grad_omega(wl.Kmat, Rm, wl.S, m0, g, j=wl.j)
    gm, gw = m.grad.cpu().numpy(), omega.grad.cpu().numpy()
    print(f"autograd E: dm {_rel(gm, gm_ref):.2e}  domega {_rel(gw, gw_ref):.2e}")
    assert _rel(gm, gm_ref) <= TOL_AUTOGRAD
    assert _rel(gw, gw_ref) <= TOL_AUTOGRAD

    def oloss(R):
        rr = oracle.encode(wl.Kmat, R, wl.S, m0, j=wl.j) - d
        return 0.5 * np.vdot(rr, rr).real

    h = 1e-3
    vox = rng.choice(wl.L, 64, replace=False)
    worst = 0.0
    for l in vox:
        Rp, Rn = Rm.copy(), Rm.copy()
        Rp[0, l] += h
        Rn[0, l] -= h
        fd = (oloss(Rp) - oloss(Rn)) / (2 * h)
        worst = max(worst, abs(fd - gw[l]) / np.abs(gw_ref).max())
    print(f"autograd E: central differences on 64 voxels, worst {worst:.2e} of max|grad|")
    assert worst <= TOL_AUTOGRAD
    op.close()


def test_autograd_adjoint_against_oracle():
    import torch
    from paper_2604_09233_gb300.autograd import SenseOperator
    dev = torch.device("cuda:0")
    wl, Rm = _problem(seed=2, matrix=20, coils=5, samples=1000, order=1, with_j=False)
    rng = np.random.default_rng(13)
    y0 = _crandn(rng, wl.K, wl.C).astype(np.complex64)
    w = _crandn(rng, wl.L).astype(np.complex64)
    op = SenseOperator(wl.Kmat, wl.Rmat, wl.S, wl.j, prec="fp32")
    y = torch.from_numpy(y0).to(dev).requires_grad_(True)
    omega = torch.from_numpy(Rm[0].astype(np.float32)).to(dev).requires_grad_(True)
    x = op.EH(y, omega)
    wt = torch.from_numpy(w).to(dev)
    loss = (torch.conj(wt) * x).real.sum() + 0.25 * (x.real ** 2 + x.imag ** 2).sum()
    loss.backward()
    x0 = oracle.adjoint(wl.Kmat, Rm, wl.S, y0, j=wl.j)
    hup = w + 0.5 * x0
    gy_ref = oracle.encode(wl.Kmat, Rm, wl.S, hup, j=wl.j)
    gw_ref = oracle.grad_omega_adjoint(wl.Kmat, Rm, wl.S, y0, hup, j=wl.j)
    e_y, e_w = _rel(y.grad.cpu().numpy(), gy_ref), _rel(omega.grad.cpu().numpy(), gw_ref)
    print(f"autograd E^H: dy {e_y:.2e}  domega {e_w:.2e}")
    assert e_y <= TOL_AUTOGRAD and e_w <= TOL_AUTOGRAD
    op.close()


def _cg_case():
    wl, Rm = _problem()
    sigma = (oracle.encode(wl.Kmat, Rm, wl.S, wl.m_true, j=wl.j) + wl.noise).astype(np.complex64)
    return wl, Rm, sigma


def _cg_grads(op, sigma, omega0, w, n_it, every, dev, apply_j=True):
    import torch
    s = torch.from_numpy(sigma).to(dev).requires_grad_(True)
    omega = torch.from_numpy(omega0).to(dev).requires_grad_(True)
    x = op.cg(s, omega, n_iter=n_it, ckpt_every=every, apply_j=apply_j)
    loss = (torch.conj(torch.from_numpy(w).to(dev)) * x).real.sum()
    loss.backward()
    return x.detach().cpu().numpy(), s.grad.cpu().numpy(), omega.grad.cpu().numpy()


@pytest.mark.parametrize("apply_j", [True, False])
def test_cg_backward_against_central_differences_of_oracle_cg(apply_j):
    """Loss Re<w, x_N> with x_N the CG iterate after 6 iterations (checkpoints every 4:
    a full and a ragged segment); directional and per-voxel derivatives w.r.t. omega and a
    directional derivative w.r.t. s, against central differences of the FP64 oracle CG."""
    import torch
    from paper_2604_09233_gb300.autograd import SenseOperator
    dev = torch.device("cuda:0")
    wl, Rm, sigma = _cg_case()
    n_it = 6
    rng = np.random.default_rng(14)
    w = _crandn(rng, wl.L).astype(np.complex64)
    op = SenseOperator(wl.Kmat, wl.Rmat, wl.S, wl.j, prec="fp32")
    x, gs, gw = _cg_grads(op, sigma, Rm[0].astype(np.float32), w, n_it, 4, dev, apply_j)
    op.close()

    def oloss(R, s):
        xo = oracle.cg(wl.Kmat, R, wl.S, s, n_it, j=wl.j, apply_j=apply_j)["x"]
        return np.vdot(w.astype(complex), xo).real

    s64 = sigma.astype(complex)
    assert _rel(x, oracle.cg(wl.Kmat, Rm, wl.S, s64, n_it, j=wl.j, apply_j=apply_j)["x"]) <= 1e-4
    h = 1e-3
    d = rng.normal(size=wl.L)
    Rp, Rn = Rm.copy(), Rm.copy()
    Rp[0] += h * d
    Rn[0] -= h * d
    fd = (oloss(Rp, s64) - oloss(Rn, s64)) / (2 * h)
    e_dir = abs(float(np.dot(gw, d)) - fd) / abs(fd)
    worst = 0.0
    for l in rng.choice(wl.L, 12, replace=False):
        Rp, Rn = Rm.copy(), Rm.copy()
        Rp[0, l] += h
        Rn[0, l] -= h
        fdl = (oloss(Rp, s64) - oloss(Rn, s64)) / (2 * h)
        worst = max(worst, abs(fdl - gw[l]) / np.abs(gw).max())
    ds = _crandn(rng, wl.K, wl.C) * np.sqrt(np.mean(np.abs(s64) ** 2))
    hs = 1e-3
    fds = (oloss(Rm, s64 + hs * ds) - oloss(Rm, s64 - hs * ds)) / (2 * hs)
    e_s = abs(float(np.vdot(gs.astype(complex), ds).real) - fds) / abs(fds)
    print(f"CG backward (apply_j={apply_j}): omega dir {e_dir:.2e}, per-voxel worst {worst:.2e}, "
          f"s dir {e_s:.2e}")
    assert e_dir <= TOL_CG_GRAD and worst <= TOL_CG_GRAD and e_s <= TOL_CG_GRAD


def test_cg_backward_is_independent_of_checkpoint_spacing():
    """The replay from checkpoints is bit-identical to the forward, so every spacing
    (one per iteration, ragged, one segment, more than the iterations) gives the same
    gradients."""
    import torch
    from paper_2604_09233_gb300.autograd import SenseOperator
    dev = torch.device("cuda:0")
    wl, Rm, sigma = _cg_case()
    w = _crandn(np.random.default_rng(15), wl.L).astype(np.complex64)
    op = SenseOperator(wl.Kmat, wl.Rmat, wl.S, wl.j, prec="fp32")
    outs = [_cg_grads(op, sigma, Rm[0].astype(np.float32), w, 7, k, dev) for k in (1, 3, 7, 10)]
    op.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["tc_split"])
def test_cg_backward_tensor_core_close_to_fp32(prec):
    import torch
    from paper_2604_09233_gb300.autograd import SenseOperator
    dev = torch.device("cuda:0")
    wl, Rm, sigma = _cg_case()
    w = _crandn(np.random.default_rng(16), wl.L).astype(np.complex64)
    ops = [SenseOperator(wl.Kmat, wl.Rmat, wl.S, wl.j, prec=p) for p in ("fp32", prec)]
    a = _cg_grads(ops[0], sigma, Rm[0].astype(np.float32), w, 6, 4, dev)
    b = _cg_grads(ops[1], sigma, Rm[0].astype(np.float32), w, 6, 4, dev)
    for o in ops:
        o.close()
    e = [_rel(b[i], a[i]) for i in range(3)]
    print(f"CG backward {prec} vs fp32: x {e[0]:.2e} sbar {e[1]:.2e} omegabar {e[2]:.2e}")
    assert max(e) <= 5e-5


def test_grad_b0_full_size_sampled_voxels():
    """2D 256x256, 32 coils, 35750 samples, 3rd-order terms: E-backward B0 gradient on the
    tensor-core split path, 24 voxels recomputed by the oracle one by one."""
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wl = synthetic.target_256()
    rng = np.random.default_rng(17)
    m = wl.m_true.astype(np.complex64)
    g = _crandn(rng, wl.K, wl.C).astype(np.complex64)
    with native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j) as plan:
        gw = torch.empty(wl.L, dtype=torch.float32, device=dev)
        native.sense_grad_b0(plan.handle, native.SENSE_PREC_TC_SPLIT,
                             torch.from_numpy(m).to(dev), torch.from_numpy(g).to(dev), gw)
        native.sense_plan_sync(plan.handle)
        gw = gw.cpu().numpy()
    vox = rng.choice(wl.L, 24, replace=False)
    jv = None if wl.j is None else wl.j[vox]
    ref = oracle.grad_omega(wl.Kmat, wl.Rmat[:, vox], wl.S[vox], m[vox], g, j=jv)
    e = _rel(gw[vox], ref)
    print(f"full-size grad_b0 tc_split on 24 voxels: {e:.2e}")
    assert e <= 1e-4


def test_cg_backward_full_size():
    """The differentiation configuration (256x256, 32 coils, 35750 samples, split tensor
    cores): the 40-iteration gradients are finite and bit-identical for checkpoints every 8 and
    every 40 iterations; at 5 iterations (where single-precision CG still tracks exact CG) the
    omega and s gradients agree with central differences of the GPU's own solve along random
    directions."""
    import torch
    from paper_2604_09233_gb300.autograd import SenseOperator
    dev = torch.device("cuda:0")
    wl = synthetic.target_256()
    op = SenseOperator(wl.Kmat, wl.Rmat, wl.S, wl.j, prec="tc_split")
    omega0 = wl.Rmat[0].astype(np.float32)
    m = torch.from_numpy(wl.m_true.astype(np.complex64)).to(dev)
    sig = (op.E(m, torch.from_numpy(omega0).to(dev)).detach()
           + torch.from_numpy(wl.noise.astype(np.complex64)).to(dev)).cpu().numpy()
    rng = np.random.default_rng(18)
    w = _crandn(rng, wl.L).astype(np.complex64)
    a = _cg_grads(op, sig, omega0, w, 40, 8, dev)
    b = _cg_grads(op, sig, omega0, w, 40, 40, dev)
    for u, v in zip(a, b):
        assert np.isfinite(u).all() and np.array_equal(u, v)

    n_it = 5
    x, gs, gw = _cg_grads(op, sig, omega0, w, n_it, 2, dev)

    def loss(om, s):
        with torch.no_grad():
            xx = op.cg(torch.from_numpy(s).to(dev), torch.from_numpy(om).to(dev), n_iter=n_it,
                       ckpt_every=n_it)
        return float((np.conj(w.astype(complex)) * xx.cpu().numpy()).real.sum())

    d = rng.normal(size=wl.L).astype(np.float32)
    h = 0.5                                     # rad/s: phase changes of at most ~0.04 rad
    fd = (loss(omega0 + h * d, sig) - loss(omega0 - h * d, sig)) / (2 * h)
    e_w = abs(float(np.dot(gw.astype(np.float64), d)) - fd) / abs(fd)
    ds = (_crandn(rng, wl.K, wl.C) * np.sqrt(np.mean(np.abs(sig) ** 2))).astype(np.complex64)
    hs = 1e-2
    fds = (loss(omega0, sig + hs * ds) - loss(omega0, sig - hs * ds)) / (2 * hs)
    e_s = abs(float(np.vdot(gs.astype(complex), ds.astype(complex)).real) - fds) / abs(fds)
    op.close()
    print(f"full-size CG backward: omega dir {e_w:.2e}, s dir {e_s:.2e}")
    assert e_w <= 1e-2 and e_s <= 1e-2
