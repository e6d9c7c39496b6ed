/*
 * FP64 CPU oracle for the non-Fourier SENSE encoding operator and its CG solve.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py use it. It shares no code, header, table or constant with
 * the CUDA library in paper_2604_09233_gb300/csrc.
 *
 * Everything is written as the plain definition, in complex128, with explicit
 * loops and no blocking, fusion or reordering beyond what the definition says:
 *
 *   phase      phi(kappa,l) = sum_p K(kappa,p) R(p,l)            Eq. 4, P = e^{o i K R}
 *   encode     s(kappa,lam) = sum_l P(kappa,l) S(l,lam) j(l) m(l) Eq. 4, with S <- S o j
 *                                                                (Alg. 1, Fig. 2)      
 *   adjoint    m(l) = j(l) sum_lam conj(S(l,lam)) sum_kappa conj(P(kappa,l)) s(kappa,lam)
 *                                                                Eq. 5
 *   normal     E^H E m
 *   cg         the CG loop of Alg. 1, Fig. 2 (from rho = 0, N_It iterations)
 *   grad_omega derivative of a real loss through E w.r.t. row 0 of R (the B0 map),
 *              written as the chain rule of the definition above.
 *
 * Array conventions (row-major, as in the variable table of Fig. 2):
 *   Km  [K][P1]  temporal basis; column 0 is t_kappa, column p+1 is k_p(t_kappa)
 *   Rm  [P1][L]  spatial basis;  row 0 is B0(r_l) (rad/s), row p+1 is h_p(r_l)
 *   S   [L][C]   complex sensitivities
 *   j   [L]      real intensity correction (NULL means all ones)
 *   s   [K][C]   complex coil data Sigma
 *   m   [L]      complex image
 *
 * Parity of every function here is pinned in tests/test_oracle_pins.py against
 * results the paper and the mathematics fix (closed-form DFT, point source,
 * adjointness, dense normal-equation solve, Krylov minimisation, finite
 * differences); none of those pins re-types these loops.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Eq. 4: one entry of K R (the argument of the element-wise exponential). */
static double phase_of(const double* Km, const double* Rm, int64_t L, int P1,
                       int64_t kappa, int64_t l) {
  double phi = 0.0;
  for (int p = 0; p < P1; ++p) phi += Km[kappa * P1 + p] * Rm[(int64_t)p * L + l];
  return phi;
}

/* Eq. 4: s = E m evaluated for the sample rows listed in `rows` (all K rows
 * when rows == NULL, then nrows must be K). Output row i goes to s[i][*]. */
void or_encode(int64_t L, int64_t K, int C, int P1, const double* Km, const double* Rm,
               const cplx* S, const double* j, const cplx* m, const int64_t* rows,
               int64_t nrows, cplx* s) {
  (void)K;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nrows; ++i) {
    const int64_t kappa = rows ? rows[i] : i;
    cplx* out = s + i * C;
    for (int lam = 0; lam < C; ++lam) out[lam] = 0.0;
    for (int64_t l = 0; l < L; ++l) {
      const cplx e = cexp(I * phase_of(Km, Rm, L, P1, kappa, l));
      const cplx w = m[l] * (j ? j[l] : 1.0);
      for (int lam = 0; lam < C; ++lam) out[lam] += e * S[l * C + lam] * w;
    }
  }
}

/* Eq. 5: m = E^H s evaluated for the voxels listed in `vox` (all L when NULL). */
void or_adjoint(int64_t L, int64_t K, int C, int P1, const double* Km, const double* Rm,
                const cplx* S, const double* j, const cplx* s, const int64_t* vox,
                int64_t nvox, cplx* m) {
#pragma omp parallel
  {
    cplx* acc = (cplx*)malloc(sizeof(cplx) * (size_t)C);
#pragma omp for schedule(dynamic, 4)
    for (int64_t i = 0; i < nvox; ++i) {
      const int64_t l = vox ? vox[i] : i;
      for (int lam = 0; lam < C; ++lam) acc[lam] = 0.0;
      for (int64_t kappa = 0; kappa < K; ++kappa) {
        const cplx e_conj = cexp(-I * phase_of(Km, Rm, L, P1, kappa, l));
        for (int lam = 0; lam < C; ++lam) acc[lam] += e_conj * s[kappa * C + lam];
      }
      cplx v = 0.0;
      for (int lam = 0; lam < C; ++lam) v += conj(S[l * C + lam]) * acc[lam];
      m[i] = v * (j ? j[l] : 1.0);
    }
    free(acc);
  }
}

/* E^H E m (all voxels). `work` holds K*C complex values. */
void or_normal(int64_t L, int64_t K, int C, int P1, const double* Km, const double* Rm,
               const cplx* S, const double* j, const cplx* m, cplx* out, cplx* work) {
  or_encode(L, K, C, P1, Km, Rm, S, j, m, NULL, K, work);
  or_adjoint(L, K, C, P1, Km, Rm, S, j, work, NULL, L, out);
}

static cplx dotc(const cplx* a, const cplx* b, int64_t n) { /* a^H b */
  cplx acc = 0.0;
  for (int64_t i = 0; i < n; ++i) acc += conj(a[i]) * b[i];
  return acc;
}

static double norm2(const cplx* a, int64_t n) { return sqrt(creal(dotc(a, a, n))); }

/* The CG loop of Alg. 1 (Fig. 2): CG on E^H E rho = E^H sigma from rho = 0.
 *
 *  n_it      N_It, the number of iterations (fixed-count stop, the paper's choice)
 *  rel_tol   extra stop when ||r_n|| <= rel_tol ||E^H sigma|| (0 disables; not in the paper;
 *            from rho_0 = 0 the threshold is rel_tol ||r_0||)
 *  x0        optional [L] start rho_0 (NULL: rho_0 = 0 as in Alg. 1); the first residual
 *            is then r_0 = E^H sigma - E^H E rho_0 and the first direction p_0 = r_0
 *  rho       output [L]; multiplied by j at the end (as Alg. 1 does) when apply_j != 0
 *  hist      optional [(n_it+1)][3]: ||r_n||, ||rho_n||, ||E rho_n - sigma|| for
 *            n = 0..iters (row 0 is the start, rho_0 = 0); unused rows are left as is
 *  iterates  optional [(n_it+1)][L]: rho_n before the final multiplication by j, n = 0..iters
 * Returns the number of iterations run. The update rates are kept complex, as
 * Alg. 1 keeps them (alpha = r^H r, beta = p^H q, rho += alpha/beta p ...).      */
int or_cg(int64_t L, int64_t K, int C, int P1, const double* Km, const double* Rm,
          const cplx* S, const double* j, const cplx* sigma, int n_it, double rel_tol,
          int apply_j, const cplx* x0, cplx* rho, double* hist, cplx* iterates) {
  cplx* p = (cplx*)malloc(sizeof(cplx) * (size_t)L);
  cplx* r = (cplx*)malloc(sizeof(cplx) * (size_t)L);
  cplx* q = (cplx*)malloc(sizeof(cplx) * (size_t)L);
  cplx* work = (cplx*)malloc(sizeof(cplx) * (size_t)(K * C));
  cplx* resid = hist ? (cplx*)malloc(sizeof(cplx) * (size_t)(K * C)) : NULL;

  /* start: r = E^H sigma (- E^H E rho_0), p = r, rho = rho_0 (0 in Alg. 1) */
  or_adjoint(L, K, C, P1, Km, Rm, S, j, sigma, NULL, L, r);
  const double r0 = norm2(r, L);   /* ||E^H sigma||: the tolerance reference */
  if (x0) {
    memcpy(rho, x0, sizeof(cplx) * (size_t)L);
    or_normal(L, K, C, P1, Km, Rm, S, j, rho, q, work);
    for (int64_t l = 0; l < L; ++l) r[l] -= q[l];
  } else {
    for (int64_t l = 0; l < L; ++l) rho[l] = 0.0;
  }
  memcpy(p, r, sizeof(cplx) * (size_t)L);

  int done = 0;
  for (int n = 0;; ++n) {
    if (hist) {
      or_encode(L, K, C, P1, Km, Rm, S, j, rho, NULL, K, resid);
      for (int64_t i = 0; i < K * C; ++i) resid[i] -= sigma[i];
      hist[3 * n + 0] = norm2(r, L);
      hist[3 * n + 1] = norm2(rho, L);
      hist[3 * n + 2] = norm2(resid, K * C);
    }
    if (iterates) memcpy(iterates + (int64_t)n * L, rho, sizeof(cplx) * (size_t)L);
    if (n >= n_it) break;                                   /* at most N_It iterations */
    if (rel_tol > 0.0 && norm2(r, L) <= rel_tol * r0) break;
    /* q = E^H E p */
    or_normal(L, K, C, P1, Km, Rm, S, j, p, q, work);
    /* alpha = r^H r, beta = p^H q */
    cplx alpha = dotc(r, r, L);
    cplx beta = dotc(p, q, L);
    if (beta == 0.0) break;
    /* rho += (alpha / beta) p, r -= (alpha / beta) q */
    const cplx a_over_b = alpha / beta;
    for (int64_t l = 0; l < L; ++l) {
      rho[l] += a_over_b * p[l];
      r[l] -= a_over_b * q[l];
    }
    /* new r^H r, ratio to the old one, direction update */
    beta = alpha;
    alpha = dotc(r, r, L);
    const cplx ratio = alpha / beta;
    for (int64_t l = 0; l < L; ++l) p[l] = r[l] + ratio * p[l];
    done = n + 1;
  }
  /* rho <- rho o j */
  if (apply_j && j)
    for (int64_t l = 0; l < L; ++l) rho[l] *= j[l];
  free(p);
  free(r);
  free(q);
  free(work);
  free(resid);
  return done;
}

/* Gradient of a real loss through y = E m with respect to row 0 of R (the B0
 * map, omega, rad/s), given g = dLoss/dRe(y) + i dLoss/dIm(y) ([K][C]):
 *     dLoss/domega(l) = sum_{kappa,lam} Re( conj(g(kappa,lam)) * dy(kappa,lam)/domega(l) ),
 *     dy(kappa,lam)/domega(l) = i K(kappa,0) S(l,lam) j(l) m(l) e^{i phi(kappa,l)}
 * (the chain rule of Eq. 4; K(kappa,0) = t_kappa multiplies R(0,l) = B0(r_l)). */
/* Gradient of a real loss through x = E^H y with respect to row 0 of R, given
 * h = dLoss/dRe(x) + i dLoss/dIm(x) ([L]):
 *     dLoss/domega(l) = Re( conj(h(l)) * dx(l)/domega(l) ),
 *     dx(l)/domega(l) = j(l) sum_lam conj(S(l,lam)) sum_kappa (-i K(kappa,0)) e^{-i phi(kappa,l)} y(kappa,lam)
 * (the chain rule of Eq. 5; x(l) depends on omega(l) alone). */
void or_grad_omega_adjoint(int64_t L, int64_t K, int C, int P1, const double* Km,
                           const double* Rm, const cplx* S, const double* j, const cplx* y,
                           const cplx* h, double* grad) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t l = 0; l < L; ++l) {
    cplx dx = 0.0;
    for (int64_t kappa = 0; kappa < K; ++kappa) {
      const cplx e = cexp(-I * phase_of(Km, Rm, L, P1, kappa, l));
      for (int lam = 0; lam < C; ++lam)
        dx += conj(S[l * C + lam]) * (-I * Km[kappa * P1 + 0]) * e * y[kappa * C + lam];
    }
    dx *= (j ? j[l] : 1.0);
    grad[l] = creal(conj(h[l]) * dx);
  }
}

void or_grad_omega(int64_t L, int64_t K, int C, int P1, const double* Km, const double* Rm,
                   const cplx* S, const double* j, const cplx* m, const cplx* g,
                   double* grad) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t l = 0; l < L; ++l) {
    double acc = 0.0;
    const cplx w = m[l] * (j ? j[l] : 1.0);
    for (int64_t kappa = 0; kappa < K; ++kappa) {
      const cplx e = cexp(I * phase_of(Km, Rm, L, P1, kappa, l));
      for (int lam = 0; lam < C; ++lam) {
        const cplx dy = I * Km[kappa * P1 + 0] * S[l * C + lam] * w * e;
        acc += creal(conj(g[kappa * C + lam]) * dy);
      }
    }
    grad[l] = acc;
  }
}
