"""Writes cg_target_256.txt: the FP64 oracle's CG iterates for the 2D 256x256, 32-coil,
35750-sample spiral with 3rd-order field terms (the CG loop of Alg. 1, Fig. 2, from rho = 0,
then rho <- rho o j), on every 64th voxel (1024 voxels, user order), after 5, 10 and 40
iterations.

Inputs: the seeded synthetic workload (paper_2604_09233_gb300.synthetic.target_256) with coil
data sigma = E m + noise, E applied by the oracle. Everything here is computed by oracle/;
nothing comes from the CUDA library. Run: python tests/golden/make_cg_target_256.py
(about 41 applications of the FP64 operator: tens of minutes on a few host cores).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2604_09233_gb300 import synthetic  # noqa: E402

ITERS = (5, 10, 40)
STRIDE = 64
OUT = os.path.join(HERE, "cg_target_256.txt")


def main():
    wl = synthetic.target_256()
    t0 = time.time()
    sigma = oracle.encode(wl.Kmat, wl.Rmat, wl.S, wl.m_true, j=wl.j) + wl.noise
    out = oracle.cg(wl.Kmat, wl.Rmat, wl.S, sigma, max(ITERS), j=wl.j, iterates=True)
    its = out["iterates"]
    jj = 1.0 if wl.j is None else wl.j
    vox = np.arange(0, wl.L, STRIDE)
    with open(OUT, "w") as fh:
        fh.write(f"# FP64 oracle CG iterates (CG loop of Alg. 1, Fig. 2, times j) for {wl.name}\n")
        fh.write(f"# written by tests/golden/make_cg_target_256.py in {time.time() - t0:.0f} s "
                 f"with {oracle.num_threads()} threads\n")
        fh.write(f"# sigma = oracle E m_true + noise; voxels l = 0, {STRIDE}, ... (user order)\n")
        fh.write("# columns: voxel " + " ".join(f"re_{n} im_{n}" for n in ITERS) + "\n")
        fh.write("# norms of the full iterates: " +
                 " ".join(f"{n}:{np.linalg.norm(its[n] * jj):.17e}" for n in ITERS) + "\n")
        for l in vox:
            vals = []
            for n in ITERS:
                v = its[n][l] * (jj if np.isscalar(jj) else jj[l])
                vals += [f"{v.real:.17e}", f"{v.imag:.17e}"]
            fh.write(f"{l} " + " ".join(vals) + "\n")


if __name__ == "__main__":
    main()
