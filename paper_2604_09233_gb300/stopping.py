"""Stopping rules for the CG reconstruction, studied on synthetic phantoms.

The paper chooses the number of CG iterations by hand and discusses two automatic rules: the
point of maximum curvature of the L-curve (log data residual against log solution norm over the
iterations) and the peak of the structural similarity (SSIM) with a reference image. With a
synthetic phantom the ground truth is known, so a long run can place both rules against the
iteration of minimum error. The solve records every iterate on the GPU
(`sense_cg_solve_iterates`); the image metrics below are evaluated afterwards on the host (they
are analysis, not part of the reconstruction).

Run:  python -m paper_2604_09233_gb300.stopping --workload precision_128 --iters 250
"""
import argparse
import json

import numpy as np


def ssim(a, b, shape, sigma=1.5, truncate=3.5, k1=0.01, k2=0.03, data_range=None):
    """Mean structural similarity of two real images of `shape` (Wang, Bovik, Sheikh and
    Simoncelli, 2004): Gaussian-weighted local means, variances and covariance (window
    standard deviation sigma, radius int(truncate*sigma + 0.5)), stabilisers C1 = (k1 D)^2
    and C2 = (k2 D)^2 with D the data range (default: the range of b, the reference), the
    SSIM map averaged over the voxels at least one window radius from the border."""
    from scipy.ndimage import gaussian_filter
    a = np.asarray(a, np.float64).reshape(shape)
    b = np.asarray(b, np.float64).reshape(shape)
    D = float(b.max() - b.min()) if data_range is None else float(data_range)
    c1, c2 = (k1 * D) ** 2, (k2 * D) ** 2

    def g(x):
        return gaussian_filter(x, sigma, truncate=truncate, mode="reflect")

    mu_a, mu_b = g(a), g(b)
    s_aa = g(a * a) - mu_a * mu_a
    s_bb = g(b * b) - mu_b * mu_b
    s_ab = g(a * b) - mu_a * mu_b
    m = ((2 * mu_a * mu_b + c1) * (2 * s_ab + c2)) / \
        ((mu_a * mu_a + mu_b * mu_b + c1) * (s_aa + s_bb + c2))
    r = int(truncate * sigma + 0.5)
    inner = tuple(slice(r, n - r) if n > 2 * r else slice(None) for n in m.shape)
    return float(m[inner].mean())


def study(wl, n_iter=250, prec="tc_split", noise_scale=1.0, device="cuda:0"):
    """Run n_iter CG iterations on the workload's data (E m_true + noise_scale * noise),
    recording every iterate, and place the L-curve corner and the SSIM peak against the
    iteration of minimum relative error to the ground truth."""
    import torch
    from . import native
    dev = torch.device(device)
    p = native.PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    truth = wl.m_true * (wl.j if wl.j is not None else 1.0)
    with native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j) as plan:
        m = torch.from_numpy(wl.m_true.astype(np.complex64)).to(dev)
        s = plan.encode(m) + noise_scale * torch.from_numpy(wl.noise.astype(np.complex64)).to(dev)
        X = torch.empty((n_iter + 1, wl.L), dtype=torch.complex64, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        info, hist = native.sense_cg_solve_iterates(plan.handle, s, X, n_iter, prec=p)
        ev[1].record()
        torch.cuda.synchronize()
        corner = native.sense_lcurve_corner(hist)
        X = X[: info["iters"] + 1].cpu().numpy()
    shape = wl.shape
    err = np.linalg.norm(X - truth[None, :], axis=1) / np.linalg.norm(truth)
    ref = np.abs(truth)
    sim = np.array([ssim(np.abs(x), ref, shape) for x in X])
    n_err = int(np.argmin(err))
    n_ssim = int(np.argmax(sim))
    out = {
        "workload": wl.name, "precision": prec, "noise_scale": noise_scale,
        "iterations": info["iters"], "solve_ms": ev[0].elapsed_time(ev[1]),
        "error_minimum": {"iteration": n_err, "rel_error": float(err[n_err]),
                          "ssim": float(sim[n_err])},
        "ssim_peak": {"iteration": n_ssim, "rel_error": float(err[n_ssim]),
                      "ssim": float(sim[n_ssim])},
        "lcurve_corner": {"iteration": int(corner),
                          "rel_error": float(err[corner]) if corner >= 0 else None,
                          "ssim": float(sim[corner]) if corner >= 0 else None},
        "final": {"rel_error": float(err[-1]), "ssim": float(sim[-1])},
    }
    return out, {"rel_error": err, "ssim": sim, "history": hist}


def main():
    from . import synthetic
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="precision_128")
    ap.add_argument("--iters", type=int, default=250)
    ap.add_argument("--prec", default="tc_split")
    ap.add_argument("--noise-scale", type=float, nargs="+", default=[1.0, 300.0])
    args = ap.parse_args()
    wl = getattr(synthetic, args.workload)()
    for ns in args.noise_scale:
        print(json.dumps(study(wl, args.iters, args.prec, ns)[0]), flush=True)


if __name__ == "__main__":
    main()
