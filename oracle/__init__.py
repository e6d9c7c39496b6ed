"""FP64 CPU oracle for the non-Fourier SENSE operator, its CG solve and its B0 gradient.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it; the product path never does. It
shares no code with the CUDA library. The arithmetic lives in ``sense_oracle.c`` (plain
complex128 loops); this module only loads it and marshals numpy arrays.

Functions and the passages they follow:
  encode       Eq. 4   s = P (S o (m 1^T)), P = e^{o iKR}, S <- S o j (Alg. 1, Fig. 2)
  adjoint      Eq. 5   m = (S* o (P^H Sigma)) 1
  normal       E^H E m (the normal-operator product inside Alg. 1, Fig. 2)
  cg           the CG loop of Alg. 1 (Fig. 2), then rho <- rho o j
  grad_omega   chain rule of Eq. 4 w.r.t. row 0 of R (the B0 map)
  grad_omega_adjoint  chain rule of Eq. 5 w.r.t. row 0 of R (backward of x = E^H y)
  smooth_map   Eqs. 1 and 3: smoothing and extrapolation of sensitivity / B0 maps as a sparse
               least-squares problem, solved directly
  smooth_sensitivities  Eq. 1 per coil on the magnitude and the magnitude-normalised map,
               recombined (sensitivity-map section)
  kspace_mask  the k-space filter: Cartesian points inside the Delaunay triangulation of the
               first-order k-space coordinates (k-space filter section)
  kspace_filter  rho <- IFFT(FFT(rho) o f), the filtering that ends Alg. 1 (Fig. 2),
                 as dense transforms
  lcurve_corner  maximum-curvature point of the L-curve (log residual norm vs log
                 solution norm over CG iterations), the stopping rule the paper evaluates

Each is pinned in tests/test_oracle_pins.py against results the paper and the mathematics
fix: a closed-form DFT, a point source, adjointness, a dense normal-equation solve, Krylov
minimisation of early iterates, finite differences, and an analytic curvature.
"""
from .oracle import (  # noqa: F401
    build,
    load,
    encode,
    adjoint,
    normal,
    cg,
    grad_omega,
    grad_omega_adjoint,
    kspace_mask,
    kspace_filter,
    smooth_map,
    smooth_sensitivities,
    lcurve_corner,
    num_threads,
    set_num_threads,
)
