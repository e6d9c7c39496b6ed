"""Batched reconstruction through the C ABI: one persistent work-queue launch per E / E^H
over instances of uneven size, per-instance CG stopping, the captured iteration graph and
the autotuner. References: the FP64 oracle, and the single-problem tensor-core path on the
same plans (which differs only in the order of the partial sums)."""
import numpy as np
import pytest

import oracle
from paper_2604_09233_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = {"tc_split": 2e-5, "tc_fp16": 2e-3}
TOL_CG = 1e-4
# instances of small_batch() well enough conditioned for FP32 CG to track FP64 CG
CG_PARITY = {0, 2}


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _crandn(rng, *shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2.0)


@pytest.fixture(scope="module")
def small():
    from paper_2604_09233_gb300 import native
    wls = synthetic.small_batch()
    b = native.Batch([(w.Kmat, w.Rmat, w.S, w.j) for w in wls])
    yield wls, b
    b.close()


def _sigma(w):
    return (oracle.encode(w.Kmat, w.Rmat, w.S, w.m_true, j=w.j) + w.noise).astype(np.complex64)


@pytest.mark.parametrize("prec", ["tc_split", "tc_fp16"])
def test_batch_normal_matches_oracle_and_single_path(small, prec):
    import torch
    from paper_2604_09233_gb300 import native
    wls, b = small
    p = native.PRECISIONS[prec]
    dev = torch.device("cuda:0")
    info = native.sense_batch_info(b.handle)
    assert info["n"] == len(wls) and info["C_padded"] == 32
    rng = np.random.default_rng(21)
    ms = [_crandn(rng, w.L).astype(np.complex64) for w in wls]
    outs = b.normal([torch.from_numpy(m).to(dev) for m in ms], p)
    for i, (w, m, o) in enumerate(zip(wls, ms, outs)):
        ref = oracle.normal(w.Kmat, w.Rmat, w.S, m, j=w.j)
        e = _rel(o.cpu().numpy(), ref)
        single = torch.empty_like(o)
        native.sense_normal_op(native.sense_batch_plan(b.handle, i), p,
                               torch.from_numpy(m).to(dev), single)
        torch.cuda.synchronize()
        e_s = _rel(o.cpu().numpy(), single.cpu().numpy())
        print(f"batch normal {prec} instance {i} ({w.name}): vs oracle {e:.2e}, vs single {e_s:.2e}")
        assert e <= TOL[prec]
        assert e_s <= TOL[prec] / 4


def test_batch_cg_matches_oracle_at_early_iterations(small):
    import torch
    wls, b = small
    dev = torch.device("cuda:0")
    sig = [_sigma(w) for w in wls]
    xs, infos = b.cg([torch.from_numpy(s).to(dev) for s in sig], 5)
    for i, (w, x, inf) in enumerate(zip(wls, xs, infos)):
        assert inf["iters"] == 5 and inf["status"] == 0
        assert np.isfinite(x.cpu().numpy()).all()
        if i in CG_PARITY:
            ref = oracle.cg(w.Kmat, w.Rmat, w.S, sig[i].astype(complex), 5, j=w.j)["x"]
            e = _rel(x.cpu().numpy(), ref)
            print(f"batch CG instance {i}: {e:.2e}")
            assert e <= TOL_CG


def test_batch_cg_stops_each_instance_like_the_single_path(small):
    """rel_tol stopping per instance: the batch stops every instance at the iteration the
    single-problem solve (same plan, same precision) stops at, unless the residual ratio
    there is within 1% of the tolerance (summation order may then decide)."""
    import torch
    from paper_2604_09233_gb300 import native
    wls, b = small
    dev = torch.device("cuda:0")
    sig = [torch.from_numpy(_sigma(w)).to(dev) for w in wls]
    tol = 3e-2
    _, infos = b.cg(sig, 40, rel_tol=tol)
    iters = [inf["iters"] for inf in infos]
    assert len(set(iters)) > 1          # the instances do stop at different iterations
    for i, (w, s) in enumerate(zip(wls, sig)):
        x = torch.empty(w.L, dtype=torch.complex64, device=dev)
        inf, hist = native.sense_cg_solve(native.sense_batch_plan(b.handle, i), s, x, 40,
                                          prec=native.SENSE_PREC_TC_SPLIT, rel_tol=tol)
        r = hist[:, 0] / hist[0, 0]
        n = inf["iters"]
        ambiguous = abs(r[n] / tol - 1.0) < 0.01 or (n > 0 and abs(r[n - 1] / tol - 1.0) < 0.01)
        print(f"instance {i}: batch {iters[i]} single {n} (ratio {r[n]:.4g})")
        assert iters[i] == n or (ambiguous and abs(iters[i] - n) <= 1)


def test_batch_follows_a_member_plans_new_b0_map(small):
    """Replacing a member plan's B0 map rebuilds that plan's geometry; the batch picks up the
    new arrays on its next call (its descriptors would otherwise point at the old ones)."""
    import torch
    from paper_2604_09233_gb300 import native
    wls, b = small
    dev = torch.device("cuda:0")
    i = 2
    w = wls[i]
    Rm = w.Rmat.copy()
    Rm[0] = 1.5 * Rm[0] + 40.0
    native.sense_plan_set_b0(native.sense_batch_plan(b.handle, i), Rm[0])
    try:
        rng = np.random.default_rng(24)
        ms = [_crandn(rng, x.L).astype(np.complex64) for x in wls]
        outs = b.normal([torch.from_numpy(m).to(dev) for m in ms])
        ref = oracle.normal(w.Kmat, Rm, w.S, ms[i], j=w.j)
        assert _rel(outs[i].cpu().numpy(), ref) <= TOL["tc_split"]
        assert _rel(outs[0].cpu().numpy(), oracle.normal(wls[0].Kmat, wls[0].Rmat, wls[0].S,
                                                          ms[0], j=wls[0].j)) <= TOL["tc_split"]
    finally:
        native.sense_plan_set_b0(native.sense_batch_plan(b.handle, i), w.Rmat[0])


def test_batch_graph_replay_is_deterministic(small):
    import torch
    wls, b = small
    dev = torch.device("cuda:0")
    sig = [torch.from_numpy(_sigma(w)).to(dev) for w in wls]
    a, ia = b.cg(sig, 12, rel_tol=1e-3)
    c, ic = b.cg(sig, 12, rel_tol=1e-3)
    for x, y in zip(a, c):
        assert torch.equal(x, y)
    assert ia == ic


def test_batch_autotune_and_rejections(small):
    import torch
    from paper_2604_09233_gb300 import native
    wls, b = small
    t = native.sense_batch_autotune(b.handle)
    assert t["chunk"] in (8, 16, 32, 64) and t["seg_len"] in (2, 4) and t["ms"] > 0
    assert native.sense_batch_info(b.handle)["chunk"] == t["chunk"]
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(22)
    ms = [_crandn(rng, w.L).astype(np.complex64) for w in wls]
    outs = b.normal([torch.from_numpy(m).to(dev) for m in ms])
    for w, m, o in zip(wls, ms, outs):
        assert _rel(o.cpu().numpy(), oracle.normal(w.Kmat, w.Rmat, w.S, m, j=w.j)) <= TOL["tc_split"]
    xs = [torch.empty(w.L, dtype=torch.complex64, device=dev) for w in wls]
    ss = [torch.zeros((w.K, w.C), dtype=torch.complex64, device=dev) for w in wls]
    with pytest.raises(native.SenseError) as e:
        native.sense_batch_cg_solve(b.handle, ss, xs, 3, prec=native.SENSE_PREC_FP32)
    assert e.value.code == -1
    host = [np.zeros((w.K, w.C), np.complex64) for w in wls]
    with pytest.raises(native.SenseError):
        native.sense_batch_cg_solve(b.handle, host, xs, 3)


def test_batch_of_full_size_instances_matches_single_path():
    """The first 8 instances of the 64-instance batch workload (matrices 64..256, 8-32 coils,
    4096-35750 samples): batched E^H E against the single-problem path on the same plans,
    and per-instance stopping at relative residual 1e-3 within 50 iterations."""
    import torch
    from paper_2604_09233_gb300 import native
    dev = torch.device("cuda:0")
    wls = synthetic.batch_64()[:8]
    with native.Batch([(w.Kmat, w.Rmat, w.S, w.j) for w in wls]) as b:
        native.sense_batch_autotune(b.handle)
        rng = np.random.default_rng(23)
        ms = [torch.from_numpy(_crandn(rng, w.L).astype(np.complex64)).to(dev) for w in wls]
        outs = b.normal(ms)
        for i, (m, o) in enumerate(zip(ms, outs)):
            single = torch.empty_like(o)
            native.sense_normal_op(native.sense_batch_plan(b.handle, i),
                                   native.SENSE_PREC_TC_SPLIT, m, single)
            torch.cuda.synchronize()
            assert _rel(o.cpu().numpy(), single.cpu().numpy()) <= 5e-6
        sig = [torch.from_numpy((w.noise + 0).astype(np.complex64)).to(dev) for w in wls]
        for i, w in enumerate(wls):
            enc = torch.empty((w.K, w.C), dtype=torch.complex64, device=dev)
            native.sense_encode(native.sense_batch_plan(b.handle, i), native.SENSE_PREC_FP32,
                                torch.from_numpy(w.m_true.astype(np.complex64)).to(dev), enc)
            sig[i] += enc
        torch.cuda.synchronize()
        _, infos = b.cg(sig, 50, rel_tol=1e-3)
        for i, inf in enumerate(infos):
            x = torch.empty(wls[i].L, dtype=torch.complex64, device=dev)
            ref, _ = native.sense_cg_solve(native.sense_batch_plan(b.handle, i), sig[i], x, 50,
                                           prec=native.SENSE_PREC_TC_SPLIT, rel_tol=1e-3,
                                           history=False)
            print(f"{wls[i].name}: batch {inf['iters']} single {ref['iters']}")
            assert inf["status"] == 0 and abs(inf["iters"] - ref["iters"]) <= 1
