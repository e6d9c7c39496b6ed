"""Sensitivity and B0 map smoothing (Eqs. 1 and 3) on synthetic maps: masks and a command-line
tool that times the device solves.

The paper derives its masks from prescan data: the trusted mask M_T (voxels with enough signal)
and the reconstruction mask M_R (every voxel that may hold signal, a slightly dilated head
mask). For the synthetic phantoms M_T is the phantom's support and M_R that support dilated by a
few voxels, so Eq. 1 extrapolates the maps over the band between them.

Run:  python -m paper_2604_09233_gb300.maps --workload target_256 --precond multigrid none
"""
import argparse
import json

import numpy as np


def synthetic_masks(wl, dilate=8, level=0.1):
    """(M_T, M_R) as float32 [L]: |m_true| above `level` of its peak, and that support dilated
    by `dilate` voxels."""
    from scipy.ndimage import binary_dilation
    support = (np.abs(wl.m_true) > level * np.abs(wl.m_true).max()).reshape(wl.shape)
    m_r = binary_dilation(support, iterations=dilate) if dilate > 0 else support
    return support.astype(np.float32).ravel(), m_r.astype(np.float32).ravel()


def noisy_sensitivities(wl, sigma=0.05, seed=8):
    """The workload's coil sensitivities [L][C] with complex Gaussian noise of std sigma."""
    rng = np.random.default_rng(seed)
    noise = rng.normal(size=wl.S.shape) + 1j * rng.normal(size=wl.S.shape)
    return (wl.S + sigma * noise).astype(np.complex64)


def run(wl, precond=("multigrid", "none"), dilate=8, alpha=0.5, rel_tol=1e-6, max_iter=20000,
        device="cuda:0"):
    """Eq. 1 on every coil's noisy sensitivity map (2 C fields in one call) with each
    preconditioner; the second of two identical calls is timed with CUDA events."""
    import torch
    from . import native
    dev = torch.device(device)
    m_t, m_r = synthetic_masks(wl, dilate)
    dm_t, dm_r = torch.from_numpy(m_t).to(dev), torch.from_numpy(m_r).to(dev)
    dS = torch.from_numpy(noisy_sensitivities(wl)).to(dev)
    out = torch.empty_like(dS)
    stream = torch.cuda.current_stream(dev)
    res = {"workload": wl.name, "coils": wl.C, "fields": 2 * wl.C, "dilate": dilate,
           "trusted": int(m_t.sum()), "reconstructed": int(m_r.sum())}
    for pc in precond:
        def call():
            return native.sense_smooth_sensitivities(wl.shape, alpha, dm_t, dm_r, dS, out,
                                                     max_iter=max_iter, rel_tol=rel_tol,
                                                     precond=pc)
        call()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        infos = call()
        ev[1].record(stream)
        torch.cuda.synchronize()
        its = [i["iters"] for i in infos]
        res[pc] = {"ms": ev[0].elapsed_time(ev[1]), "iterations_max": max(its),
                   "iterations_mean": float(np.mean(its)),
                   "rel_residual_max": max(i["rel_residual"] for i in infos)}
    return res


def main():
    from . import synthetic
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="target_256")
    ap.add_argument("--precond", nargs="+", default=["multigrid", "none"])
    ap.add_argument("--dilate", type=int, default=8)
    args = ap.parse_args()
    wl = getattr(synthetic, args.workload)()
    print(json.dumps(run(wl, tuple(args.precond), args.dilate)), flush=True)


if __name__ == "__main__":
    main()
