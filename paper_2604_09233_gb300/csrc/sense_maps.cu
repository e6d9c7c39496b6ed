// Map smoothing and extrapolation (Eq. 1 for sensitivity maps, Eq. 3 for the B0 map).
//
// Both equations are least-squares systems A x = [w0 o xhat; 0; ...; 0] with
//   A = [diag(w0); sqrt(alpha) diag(wd) D_x; sqrt(alpha) diag(wd) D_y; sqrt(alpha) diag(wd) D_z]
// where D is the second difference (Eq. 1: w0 = the trusted mask M_T, wd = the reconstruction
// mask M_R) or the first difference (Eq. 3: w0 = 1, wd = the fit's standard error). Their normal
// equations (diag(w0^2) + alpha sum_d D_d^T diag(wd^2) D_d) x = diag(w0^2) xhat have a real,
// symmetric, positive semi-definite matrix N; it is applied matrix-free as a stencil and solved
// by CG on complex fields (real and imaginary parts share the matrix) starting from xhat.
// A derivative row exists at voxel c along an axis when the stencil fits: second differences
// x[c-1] - 2 x[c] + x[c+1] at interior voxels, first differences x[c+1] - x[c] wherever c + 1 is
// on the grid; the row's weight is wd[c]. Axes of length 1 have no rows.
//
// Preconditioner (optional). The paper suggests an incomplete-Cholesky factorisation, whose
// triangular solves are sequential. Here the preconditioner is one symmetric multigrid V-cycle:
//  - level 0 is N written out as an explicit stencil (a cross of half-width 1 or 2), with the
//    diagonal of unconstrained voxels (no equation touches them) set to 1;
//  - coarse grids halve every axis longer than 1 (n_c = (n + 1) / 2, coarse node J at fine
//    node 2J); prolongation P is linear interpolation along each axis (an odd fine node takes
//    the mean of its two coarse neighbours, or copies the one it has at an even-length edge);
//  - coarse operators are Galerkin products P^T A P (a box stencil of half-width 2 for Eq. 1,
//    1 for Eq. 3), assembled on the device;
//  - smoothing is a degree-3 Chebyshev polynomial in D^-1 A over [l/30, l], l = 1.2 x a
//    10-step power-iteration estimate of the largest eigenvalue of D^-1 A (capped by the
//    Gershgorin bound), the same polynomial before and after the coarse correction, so that
//    the cycle is a symmetric positive definite operator;
//  - the coarsest grid (at most 64 nodes) is solved approximately by 40 Chebyshev steps in one
//    thread block.
// The cycle's output is zeroed at unconstrained voxels, so those keep xhat as in plain CG.
//
// Each CG iteration is captured once in a CUDA graph and replayed; the host reads the device's
// stop flag (tolerance reached or breakdown) one batch of replays behind, and every kernel
// returns at once after the flag is set.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sense_internal.cuh"
#include "sense_reduce.cuh"

namespace sense {
namespace {

constexpr int CHEB_DEG = 3;            // smoothing steps before and after the coarse correction
constexpr double CHEB_RATIO = 30.0;    // smoothed part of the spectrum: [lmax / 30, lmax]
constexpr int POWER_STEPS = 10;        // power-iteration steps for lmax(D^-1 A)
constexpr double POWER_SAFETY = 1.2;   // factor on the power-iteration estimate
constexpr int COARSE_MAX = 64;         // nodes of the coarsest grid (one thread block)
constexpr int COARSE_DEG = 40;         // Chebyshev steps on the coarsest grid
constexpr int MAX_LEVELS = 40;
constexpr int POLL_EVERY = 8;          // graph replays between reads of the stop flag

struct Grid {
  int n[3];
  long long stride[3];
  long long total;
};

// Stencil shape. cross: the centre, then offsets -e..-1, 1..e along x, y, z in turn (axes with
// e = 0 contribute none); box: every offset of [-e0, e0] x [-e1, e1] x [-e2, e2], x fastest.
// Coefficients are stored offset-major: c[o * total + i] multiplies x[i + offset o].
struct Sten {
  int e[3];
  int box;
  int count;
  int center;
};

Sten make_cross(const int (&e)[3]) {
  Sten s{{e[0], e[1], e[2]}, 0, 1 + 2 * (e[0] + e[1] + e[2]), 0};
  return s;
}

Sten make_box(const int (&e)[3]) {
  Sten s{{e[0], e[1], e[2]}, 1, (2 * e[0] + 1) * (2 * e[1] + 1) * (2 * e[2] + 1), 0};
  s.center = (e[2] * (2 * e[1] + 1) + e[1]) * (2 * e[0] + 1) + e[0];
  return s;
}

__device__ __forceinline__ void coords(const Grid& g, long long i, int (&c)[3]) {
  c[0] = (int)(i % g.n[0]);
  c[1] = (int)((i / g.n[0]) % g.n[1]);
  c[2] = (int)(i / ((long long)g.n[0] * g.n[1]));
}

template <class F>
__device__ __forceinline__ void for_offsets(const Sten& s, F&& f) {
  if (s.box) {
    int o = 0;
    for (int dz = -s.e[2]; dz <= s.e[2]; ++dz)
      for (int dy = -s.e[1]; dy <= s.e[1]; ++dy)
        for (int dx = -s.e[0]; dx <= s.e[0]; ++dx) f(o++, dx, dy, dz);
  } else {
    f(0, 0, 0, 0);
    int o = 1;
    for (int d = 0; d < 3; ++d)
      for (int k = -s.e[d]; k <= s.e[d]; ++k) {
        if (k == 0) continue;
        f(o++, d == 0 ? k : 0, d == 1 ? k : 0, d == 2 ? k : 0);
      }
  }
}

// (A v)_i for an explicit stencil; neighbours off the grid are skipped (their coefficients
// are zero by construction)
__device__ __forceinline__ float2 sten_apply(const Grid& g, const Sten& s, const float* c,
                                             const float2* v, long long i, const int (&ci)[3]) {
  float2 acc = make_float2(0.f, 0.f);
  for_offsets(s, [&](int o, int dx, int dy, int dz) {
    const int x = ci[0] + dx, y = ci[1] + dy, z = ci[2] + dz;
    if (x < 0 || x >= g.n[0] || y < 0 || y >= g.n[1] || z < 0 || z >= g.n[2]) return;
    const float a = c[(long long)o * g.total + i];
    if (a == 0.f) return;
    const float2 w = v[i + dx * g.stride[0] + dy * g.stride[1] + dz * g.stride[2]];
    acc.x = fmaf(a, w.x, acc.x);
    acc.y = fmaf(a, w.y, acc.y);
  });
  return acc;
}

// (D x)_r for the row at voxel r along axis d (the caller checks that the row exists)
__device__ __forceinline__ float2 drow(const Grid& g, const float2* x, long long r, int d,
                                       int order) {
  const long long s = g.stride[d];
  if (order == 1) {
    const float2 a = x[r], b = x[r + s];
    return make_float2(b.x - a.x, b.y - a.y);
  }
  const float2 a = x[r - s], b = x[r], c = x[r + s];
  return make_float2(a.x - 2.f * b.x + c.x, a.y - 2.f * b.y + c.y);
}

// ---------------------------------------------------------------------------------------
// CG on the normal equations
// ---------------------------------------------------------------------------------------

// y = w0^2 x + alpha sum_d D_d^T diag(wd^2) D_d x (matrix-free)
__global__ void smooth_apply_kernel(Grid g, int order, float alpha, const float* __restrict__ w0,
                                    const float* __restrict__ wd, const float2* __restrict__ x,
                                    float2* __restrict__ y, const double* sc) {
  if (sc[2] != 0.0) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    int c[3];
    coords(g, i, c);
    const float a0 = w0[i] * w0[i];
    float2 acc = make_float2(a0 * x[i].x, a0 * x[i].y);
    for (int d = 0; d < 3; ++d) {
      const int n = g.n[d];
      if (n < 2) continue;
      const long long s = g.stride[d];
      float2 t = make_float2(0.f, 0.f);
      if (order == 1) {
        // rows r = i - 1 (coefficient +1 on x[i]) and r = i (coefficient -1)
        if (c[d] >= 1) {
          const float w = wd[i - s] * wd[i - s];
          const float2 v = drow(g, x, i - s, d, 1);
          t.x += w * v.x;
          t.y += w * v.y;
        }
        if (c[d] + 1 < n) {
          const float w = wd[i] * wd[i];
          const float2 v = drow(g, x, i, d, 1);
          t.x -= w * v.x;
          t.y -= w * v.y;
        }
      } else {
        // rows r = i - 1 and i + 1 (coefficient +1 on x[i]) and r = i (coefficient -2)
        if (c[d] >= 2) {
          const float w = wd[i - s] * wd[i - s];
          const float2 v = drow(g, x, i - s, d, 2);
          t.x += w * v.x;
          t.y += w * v.y;
        }
        if (c[d] >= 1 && c[d] + 1 < n) {
          const float w = wd[i] * wd[i];
          const float2 v = drow(g, x, i, d, 2);
          t.x -= 2.f * w * v.x;
          t.y -= 2.f * w * v.y;
        }
        if (c[d] + 2 < n) {
          const float w = wd[i + s] * wd[i + s];
          const float2 v = drow(g, x, i + s, d, 2);
          t.x += w * v.x;
          t.y += w * v.y;
        }
      }
      acc.x += alpha * t.x;
      acc.y += alpha * t.y;
    }
    y[i] = acc;
  }
}

// Scalars sc[]: 0 r^H r, 1 ||b||^2, 2 stop flag, 3 step length, 4 beta, 5 iterations,
// 6 r^H z (preconditioned).

// r = w0^2 xhat - y (y = N x_0), p = r; sums ||r||^2 and ||w0^2 xhat||^2
__global__ void __launch_bounds__(VB) smooth_init_kernel(const float* __restrict__ w0,
                                                         const float2* __restrict__ xhat,
                                                         const float2* __restrict__ y,
                                                         long long n, float2* r, float2* p,
                                                         double* part, unsigned* counter,
                                                         double* sc, double tol2) {
  __shared__ double sh[2 * VB / 32];
  double v[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a0 = w0[i] * w0[i];
    const float2 b = make_float2(a0 * xhat[i].x, a0 * xhat[i].y);
    const float2 ri = make_float2(b.x - y[i].x, b.y - y[i].y);
    r[i] = ri;
    p[i] = ri;
    v[0] += (double)ri.x * ri.x + (double)ri.y * ri.y;
    v[1] += (double)b.x * b.x + (double)b.y * b.y;
  }
  block_sum<2>(v, sh);
  double tot[2];
  if (finish_sums<2>(v, part, counter, tot)) {
    sc[0] = tot[0];   // r^H r
    sc[1] = tot[1];   // ||b||^2
    sc[2] = tot[0] <= tol2 * tot[1] ? 1.0 : 0.0;   // stop flag
  }
}

// step length = (r^H z or r^H r) / p^H N p (N real symmetric: p^H N p real)
__global__ void __launch_bounds__(VB) smooth_pap_kernel(const float2* __restrict__ p,
                                                        const float2* __restrict__ q, long long n,
                                                        double* part, unsigned* counter,
                                                        double* sc, int num) {
  if (sc[2] != 0.0) return;
  __shared__ double sh[VB / 32];
  double v[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[0] += (double)p[i].x * q[i].x + (double)p[i].y * q[i].y;
  block_sum<1>(v, sh);
  double tot[1];
  if (finish_sums<1>(v, part, counter, tot)) {
    if (!(tot[0] > 0.0)) {
      sc[2] = 1.0;
      return;
    }
    sc[3] = sc[num] / tot[0];
  }
}

// x += a p; r -= a q; the new r^H r, beta for plain CG, the iteration count and the stop test
__global__ void __launch_bounds__(VB) smooth_update_kernel(float2* x, float2* r,
                                                           const float2* __restrict__ p,
                                                           const float2* __restrict__ q,
                                                           long long n, double* part,
                                                           unsigned* counter, double* sc,
                                                           double tol2) {
  if (sc[2] != 0.0) return;
  __shared__ double sh[VB / 32];
  const float a = (float)sc[3];
  double v[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i].x += a * p[i].x;
    x[i].y += a * p[i].y;
    const float2 ri = make_float2(r[i].x - a * q[i].x, r[i].y - a * q[i].y);
    r[i] = ri;
    v[0] += (double)ri.x * ri.x + (double)ri.y * ri.y;
  }
  block_sum<1>(v, sh);
  double tot[1];
  if (finish_sums<1>(v, part, counter, tot)) {
    sc[4] = tot[0] / sc[0];   // beta (plain CG)
    sc[0] = tot[0];
    sc[5] += 1.0;             // iterations
    if (tot[0] <= tol2 * sc[1]) sc[2] = 1.0;
  }
}

// Preconditioned CG: z <- 0 at unconstrained voxels, r^H z, beta = r^H z / (previous r^H z)
// (first = 1: beta = 0, so that the next direction is z itself)
__global__ void __launch_bounds__(VB) smooth_rz_kernel(float2* z, const float2* __restrict__ r,
                                                       const unsigned char* __restrict__ keep,
                                                       long long n, double* part,
                                                       unsigned* counter, double* sc, int first) {
  if (sc[2] != 0.0) return;
  __shared__ double sh[VB / 32];
  double v[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float2 zi = z[i];
    if (!keep[i]) {
      zi = make_float2(0.f, 0.f);
      z[i] = zi;
    }
    v[0] += (double)r[i].x * zi.x + (double)r[i].y * zi.y;
  }
  block_sum<1>(v, sh);
  double tot[1];
  if (finish_sums<1>(v, part, counter, tot)) {
    if (!(tot[0] > 0.0)) {
      sc[2] = 1.0;   // breakdown (or r = 0)
      return;
    }
    sc[4] = first ? 0.0 : tot[0] / sc[6];
    sc[6] = tot[0];
  }
}

// p = z + beta p (z = r for plain CG)
__global__ void smooth_p_kernel(float2* p, const float2* __restrict__ z, long long n,
                                const double* sc) {
  if (sc[2] != 0.0) return;
  const float b = (float)sc[4];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = make_float2(z[i].x + b * p[i].x, z[i].y + b * p[i].y);
}

// ---------------------------------------------------------------------------------------
// Multigrid hierarchy
// ---------------------------------------------------------------------------------------

// Level 0: N as a cross stencil of half-width `order` along every axis longer than 1.
// Row i of alpha D_d^T diag(wd^2) D_d gathers the rows r of D_d that touch voxel i:
// coefficient wd[r]^2 * D[r][i] * D[r][j] on voxel j.
__global__ void mg_fine_kernel(Grid g, Sten s, int order, float alpha,
                               const float* __restrict__ w0, const float* __restrict__ wd,
                               float* coef, unsigned char* keep) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    int c[3];
    coords(g, i, c);
    float center = w0[i] * w0[i];
    int base = 1;   // first cross index of the current axis
    for (int d = 0; d < 3; ++d) {
      const int n = g.n[d];
      if (s.e[d] == 0) continue;
      const long long st = g.stride[d];
      float cd[5] = {0.f, 0.f, 0.f, 0.f, 0.f};   // offsets -2..2 along d
      if (order == 2) {
        // second-difference rows r = c - 1, c, c + 1 (interior r only); D[r][r +- 1] = 1,
        // D[r][r] = -2
        for (int ro = -1; ro <= 1; ++ro) {
          const int rr = c[d] + ro;
          if (rr < 1 || rr > n - 2) continue;
          const float w = wd[i + ro * st];
          const float wr = alpha * w * w;
          const float ci = ro == 0 ? -2.f : 1.f;
          for (int jo = -1; jo <= 1; ++jo) cd[ro + jo + 2] += wr * ci * (jo == 0 ? -2.f : 1.f);
        }
      } else {
        // first-difference rows r = c - 1 and c (r + 1 on the grid); D[r][r] = -1,
        // D[r][r + 1] = 1
        for (int ro = -1; ro <= 0; ++ro) {
          const int rr = c[d] + ro;
          if (rr < 0 || rr > n - 2) continue;
          const float w = wd[i + ro * st];
          const float wr = alpha * w * w;
          const float ci = ro == 0 ? -1.f : 1.f;
          for (int jo = 0; jo <= 1; ++jo) cd[ro + jo + 2] += wr * ci * (jo == 0 ? -1.f : 1.f);
        }
      }
      center += cd[2];
      const int e = s.e[d];
      for (int k = -e; k <= e; ++k) {
        if (k == 0) continue;
        const int o = base + (k < 0 ? k + e : k + e - 1);
        coef[(long long)o * g.total + i] = cd[k + 2];
      }
      base += 2 * e;
    }
    keep[i] = center > 0.f ? 1 : 0;
    coef[i] = center > 0.f ? center : 1.f;   // centre: offset 0
  }
}

// coarse nodes holding fine node f along one axis, with their interpolation weights
__device__ __forceinline__ int parents(int f, int nc, int (&J)[2], float (&w)[2]) {
  if ((f & 1) == 0) {
    J[0] = f >> 1;
    w[0] = 1.f;
    return 1;
  }
  J[0] = (f - 1) >> 1;
  J[1] = J[0] + 1;
  if (J[1] < nc) {
    w[0] = w[1] = 0.5f;
    return 2;
  }
  w[0] = 1.f;
  return 1;
}

// fine nodes interpolated from coarse node I along one axis, with the weights
__device__ __forceinline__ int children(int I, int nf, int nc, int (&f)[3], float (&w)[3]) {
  int k = 0;
  for (int a = 2 * I - 1; a <= 2 * I + 1; ++a) {
    if (a < 0 || a >= nf) continue;
    int J[2];
    float pw[2];
    const int np = parents(a, nc, J, pw);
    for (int t = 0; t < np; ++t)
      if (J[t] == I) {
        f[k] = a;
        w[k] = pw[t];
        ++k;
      }
  }
  return k;
}

// Galerkin coarse operator: Ac[I][J] = sum_{a, b} P[a][I] A[a][b] P[b][J], one thread per
// coarse row I (each thread writes only its own row; cc zeroed beforehand)
__global__ void mg_galerkin_kernel(Grid gf, Sten sf, const float* __restrict__ cf, Grid gc,
                                   Sten sc, float* cc) {
  for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I < gc.total;
       I += (long long)gridDim.x * blockDim.x) {
    int CI[3];
    coords(gc, I, CI);
    int fa[3][3];
    float wa[3][3];
    int na[3];
    for (int d = 0; d < 3; ++d) na[d] = children(CI[d], gf.n[d], gc.n[d], fa[d], wa[d]);
    for (int az = 0; az < na[2]; ++az)
      for (int ay = 0; ay < na[1]; ++ay)
        for (int ax = 0; ax < na[0]; ++ax) {
          const int a[3] = {fa[0][ax], fa[1][ay], fa[2][az]};
          const float pa = wa[0][ax] * wa[1][ay] * wa[2][az];
          const long long ia = a[0] + a[1] * gf.stride[1] + a[2] * gf.stride[2];
          for_offsets(sf, [&](int o, int dx, int dy, int dz) {
            const int b[3] = {a[0] + dx, a[1] + dy, a[2] + dz};
            for (int d = 0; d < 3; ++d)
              if (b[d] < 0 || b[d] >= gf.n[d]) return;
            const float v = cf[(long long)o * gf.total + ia];
            if (v == 0.f) return;
            int J[3][2];
            float wj[3][2];
            int nj[3];
            for (int d = 0; d < 3; ++d) nj[d] = parents(b[d], gc.n[d], J[d], wj[d]);
            for (int jz = 0; jz < nj[2]; ++jz)
              for (int jy = 0; jy < nj[1]; ++jy)
                for (int jx = 0; jx < nj[0]; ++jx) {
                  const int ox = J[0][jx] - CI[0], oy = J[1][jy] - CI[1], oz = J[2][jz] - CI[2];
                  if (ox < -sc.e[0] || ox > sc.e[0] || oy < -sc.e[1] || oy > sc.e[1] ||
                      oz < -sc.e[2] || oz > sc.e[2])
                    continue;   // cannot happen for the half-widths chosen by the host
                  const int oc =
                      ((oz + sc.e[2]) * (2 * sc.e[1] + 1) + (oy + sc.e[1])) * (2 * sc.e[0] + 1) +
                      (ox + sc.e[0]);
                  cc[(long long)oc * gc.total + I] += pa * v * wj[0][jx] * wj[1][jy] * wj[2][jz];
                }
          });
        }
  }
}

// D^-1 and the Gershgorin bound max_i sum_j |A_ij| / A_ii (non-negative floats order like
// their bit patterns, so an unsigned atomicMax finds the maximum)
__global__ void mg_diag_kernel(Grid g, Sten s, const float* __restrict__ c, float* dinv,
                               unsigned* gmax) {
  float m = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = c[(long long)s.center * g.total + i];
    float sum = 0.f;
    for (int o = 0; o < s.count; ++o) sum += fabsf(c[(long long)o * g.total + i]);
    const float inv = d > 0.f ? 1.f / d : 0.f;
    dinv[i] = inv;
    m = fmaxf(m, sum * inv);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(gmax, __float_as_uint(m));
}

// start vector of the power iteration: entries in [-1, 1) from the 32-bit finaliser of
// MurmurHash3 applied to the index (real part only)
__global__ void mg_vinit_kernel(float2* v, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u + 12345u;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    v[i] = make_float2((float)(h >> 8) * (2.f / 16777216.f) - 1.f, 0.f);
  }
}

// w = D^-1 A v and ||w||^2 (into *out)
__global__ void __launch_bounds__(VB) mg_power_kernel(Grid g, Sten s, const float* __restrict__ c,
                                                      const float* __restrict__ dinv,
                                                      const float2* __restrict__ v, float2* w,
                                                      double* part, unsigned* counter,
                                                      double* out) {
  __shared__ double sh[VB / 32];
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    coords(g, i, ci);
    const float2 a = sten_apply(g, s, c, v, i, ci);
    const float2 wi = make_float2(dinv[i] * a.x, dinv[i] * a.y);
    w[i] = wi;
    acc[0] += (double)wi.x * wi.x + (double)wi.y * wi.y;
  }
  block_sum<1>(acc, sh);
  double tot[1];
  if (finish_sums<1>(acc, part, counter, tot)) *out = tot[0];
}

__global__ void mg_normalize_kernel(const float2* __restrict__ w, float2* v, long long n,
                                    const double* nrm2) {
  const float s = *nrm2 > 0.0 ? (float)(1.0 / std::sqrt(*nrm2)) : 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = make_float2(w[i].x * s, w[i].y * s);
}

// ---------------------------------------------------------------------------------------
// V-cycle kernels (all return at once after the CG stop flag is set)
// ---------------------------------------------------------------------------------------

// Chebyshev start from x = 0: r = b, d = D^-1 b / theta, x = d
__global__ void cheb_first0_kernel(long long n, const float* __restrict__ dinv,
                                   const float2* __restrict__ b, float2* x, float2* r, float2* d,
                                   float inv_theta, const double* sc) {
  if (sc[2] != 0.0) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 bi = b[i];
    const float s = dinv[i] * inv_theta;
    const float2 di = make_float2(s * bi.x, s * bi.y);
    r[i] = bi;
    d[i] = di;
    x[i] = di;
  }
}

// Chebyshev start from x: r = b - A x, d = D^-1 r / theta, xo = x + d
__global__ void cheb_first_kernel(Grid g, Sten s, const float* __restrict__ c,
                                  const float* __restrict__ dinv, const float2* __restrict__ b,
                                  const float2* __restrict__ x, float2* xo, float2* r, float2* d,
                                  float inv_theta, const double* sc) {
  if (sc[2] != 0.0) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    coords(g, i, ci);
    const float2 a = sten_apply(g, s, c, x, i, ci);
    const float2 ri = make_float2(b[i].x - a.x, b[i].y - a.y);
    const float t = dinv[i] * inv_theta;
    const float2 di = make_float2(t * ri.x, t * ri.y);
    r[i] = ri;
    d[i] = di;
    xo[i] = make_float2(x[i].x + di.x, x[i].y + di.y);
  }
}

// Chebyshev step: r -= A dp; dn = c1 dp + c2 D^-1 r; x += dn
__global__ void cheb_step_kernel(Grid g, Sten s, const float* __restrict__ c,
                                 const float* __restrict__ dinv, const float2* __restrict__ dp,
                                 float2* dn, float2* r, float2* x, float c1, float c2,
                                 const double* sc) {
  if (sc[2] != 0.0) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    coords(g, i, ci);
    const float2 a = sten_apply(g, s, c, dp, i, ci);
    const float2 ri = make_float2(r[i].x - a.x, r[i].y - a.y);
    const float t = c2 * dinv[i];
    const float2 di = make_float2(c1 * dp[i].x + t * ri.x, c1 * dp[i].y + t * ri.y);
    r[i] = ri;
    dn[i] = di;
    x[i] = make_float2(x[i].x + di.x, x[i].y + di.y);
  }
}

// r = b - A x
__global__ void mg_resid_kernel(Grid g, Sten s, const float* __restrict__ c,
                                const float2* __restrict__ b, const float2* __restrict__ x,
                                float2* r, const double* sc) {
  if (sc[2] != 0.0) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    coords(g, i, ci);
    const float2 a = sten_apply(g, s, c, x, i, ci);
    r[i] = make_float2(b[i].x - a.x, b[i].y - a.y);
  }
}

// bc = P^T r
__global__ void mg_restrict_kernel(Grid gf, Grid gc, const float2* __restrict__ r, float2* bc,
                                   const double* sc) {
  if (sc[2] != 0.0) return;
  for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I < gc.total;
       I += (long long)gridDim.x * blockDim.x) {
    int CI[3];
    coords(gc, I, CI);
    int fa[3][3];
    float wa[3][3];
    int na[3];
    for (int d = 0; d < 3; ++d) na[d] = children(CI[d], gf.n[d], gc.n[d], fa[d], wa[d]);
    float2 acc = make_float2(0.f, 0.f);
    for (int az = 0; az < na[2]; ++az)
      for (int ay = 0; ay < na[1]; ++ay)
        for (int ax = 0; ax < na[0]; ++ax) {
          const float w = wa[0][ax] * wa[1][ay] * wa[2][az];
          const float2 v = r[fa[0][ax] + fa[1][ay] * gf.stride[1] + fa[2][az] * gf.stride[2]];
          acc.x = fmaf(w, v.x, acc.x);
          acc.y = fmaf(w, v.y, acc.y);
        }
    bc[I] = acc;
  }
}

// x += P xc
__global__ void mg_prolong_kernel(Grid gf, Grid gc, const float2* __restrict__ xc, float2* x,
                                  const double* sc) {
  if (sc[2] != 0.0) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < gf.total;
       i += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    coords(gf, i, ci);
    int J[3][2];
    float w[3][2];
    int nj[3];
    for (int d = 0; d < 3; ++d) nj[d] = parents(ci[d], gc.n[d], J[d], w[d]);
    float2 acc = x[i];
    for (int jz = 0; jz < nj[2]; ++jz)
      for (int jy = 0; jy < nj[1]; ++jy)
        for (int jx = 0; jx < nj[0]; ++jx) {
          const float ww = w[0][jx] * w[1][jy] * w[2][jz];
          const float2 v = xc[J[0][jx] + J[1][jy] * gc.stride[1] + J[2][jz] * gc.stride[2]];
          acc.x = fmaf(ww, v.x, acc.x);
          acc.y = fmaf(ww, v.y, acc.y);
        }
    x[i] = acc;
  }
}

// Coarsest grid (at most COARSE_MAX nodes, one block of COARSE_MAX threads): COARSE_DEG
// Chebyshev steps from x = 0 with the vectors in shared memory
__global__ void __launch_bounds__(COARSE_MAX) mg_coarse_kernel(Grid g, Sten s,
                                                               const float* __restrict__ c,
                                                               const float* __restrict__ dinv,
                                                               const float2* __restrict__ b,
                                                               float2* x, double theta,
                                                               double delta, const double* sc) {
  if (sc[2] != 0.0) return;   // uniform over the block
  __shared__ float2 sd[2][COARSE_MAX];
  const int i = threadIdx.x;
  const bool on = i < g.total;
  int ci[3] = {0, 0, 0};
  float2 ri = make_float2(0.f, 0.f), xi = make_float2(0.f, 0.f);
  float di_inv = 0.f;
  if (on) {
    coords(g, i, ci);
    di_inv = dinv[i];
    ri = b[i];
    const float t = di_inv * (float)(1.0 / theta);
    xi = make_float2(t * ri.x, t * ri.y);
    sd[0][i] = xi;
  }
  __syncthreads();
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  int cur = 0;
  for (int k = 1; k < COARSE_DEG; ++k) {
    const double rho_n = 1.0 / (2.0 * sigma - rho);
    const float c1 = (float)(rho_n * rho), c2 = (float)(2.0 * rho_n / delta);
    rho = rho_n;
    if (on) {
      float2 a = make_float2(0.f, 0.f);
      for_offsets(s, [&](int o, int dx, int dy, int dz) {
        const int xx = ci[0] + dx, yy = ci[1] + dy, zz = ci[2] + dz;
        if (xx < 0 || xx >= g.n[0] || yy < 0 || yy >= g.n[1] || zz < 0 || zz >= g.n[2]) return;
        const float cv = c[(long long)o * g.total + i];
        const float2 w = sd[cur][i + dx * g.stride[0] + dy * g.stride[1] + dz * g.stride[2]];
        a.x = fmaf(cv, w.x, a.x);
        a.y = fmaf(cv, w.y, a.y);
      });
      ri = make_float2(ri.x - a.x, ri.y - a.y);
      const float2 dp = sd[cur][i];
      const float t = c2 * di_inv;
      const float2 dn = make_float2(c1 * dp.x + t * ri.x, c1 * dp.y + t * ri.y);
      sd[cur ^ 1][i] = dn;
      xi = make_float2(xi.x + dn.x, xi.y + dn.y);
    }
    __syncthreads();
    cur ^= 1;
  }
  if (on) x[i] = xi;
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

struct Level {
  Grid g;
  Sten s;
  float* coef = nullptr;
  float* dinv = nullptr;
  float2 *b = nullptr, *x = nullptr, *xo = nullptr, *r = nullptr, *d0 = nullptr, *d1 = nullptr;
  double theta = 1.0, delta = 0.5;
  float c1[CHEB_DEG] = {}, c2[CHEB_DEG] = {};
  int grid = 1;
};

// device buffers of one call, freed (after the stream's work) when the call returns
struct Work {
  cudaStream_t st;
  std::vector<void*> bufs;
  explicit Work(cudaStream_t s) : st(s) {}
  ~Work() {
    cudaStreamSynchronize(st);
    for (void* p : bufs) cudaFree(p);
  }
  template <class T>
  T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    bufs.push_back(p);
    return (T*)p;
  }
};

Grid make_grid(int nx, int ny, int nz) {
  Grid g;
  g.n[0] = nx;
  g.n[1] = ny;
  g.n[2] = nz;
  g.stride[0] = 1;
  g.stride[1] = nx;
  g.stride[2] = (long long)nx * ny;
  g.total = (long long)nx * ny * nz;
  return g;
}

int grid_for(long long n, int sms) {
  return (int)std::max<long long>(1, std::min<long long>((n + VB - 1) / VB, 8LL * sms));
}

// V-cycle on level l: output in L[l].xo (or L[l].x on the coarsest level); returns that buffer
float2* vcycle(std::vector<Level>& L, size_t l, const float2* b, const double* sc,
               cudaStream_t st) {
  Level& v = L[l];
  if (l + 1 == L.size()) {
    mg_coarse_kernel<<<1, COARSE_MAX, 0, st>>>(v.g, v.s, v.coef, v.dinv, b, v.x, v.theta, v.delta,
                                               sc);
    return v.x;
  }
  const float inv_theta = (float)(1.0 / v.theta);
  // pre-smoothing from x = 0
  cheb_first0_kernel<<<v.grid, VB, 0, st>>>(v.g.total, v.dinv, b, v.x, v.r, v.d0, inv_theta, sc);
  float2 *dp = v.d0, *dn = v.d1;
  for (int k = 1; k < CHEB_DEG; ++k) {
    cheb_step_kernel<<<v.grid, VB, 0, st>>>(v.g, v.s, v.coef, v.dinv, dp, dn, v.r, v.x, v.c1[k],
                                            v.c2[k], sc);
    std::swap(dp, dn);
  }
  // coarse-grid correction
  mg_resid_kernel<<<v.grid, VB, 0, st>>>(v.g, v.s, v.coef, b, v.x, v.r, sc);
  Level& w = L[l + 1];
  mg_restrict_kernel<<<w.grid, VB, 0, st>>>(v.g, w.g, v.r, w.b, sc);
  const float2* xc = vcycle(L, l + 1, w.b, sc, st);
  mg_prolong_kernel<<<v.grid, VB, 0, st>>>(v.g, w.g, xc, v.x, sc);
  // post-smoothing (the same polynomial) from the corrected x
  cheb_first_kernel<<<v.grid, VB, 0, st>>>(v.g, v.s, v.coef, v.dinv, b, v.x, v.xo, v.r, v.d0,
                                           inv_theta, sc);
  dp = v.d0;
  dn = v.d1;
  for (int k = 1; k < CHEB_DEG; ++k) {
    cheb_step_kernel<<<v.grid, VB, 0, st>>>(v.g, v.s, v.coef, v.dinv, dp, dn, v.r, v.xo, v.c1[k],
                                            v.c2[k], sc);
    std::swap(dp, dn);
  }
  return v.xo;
}

}  // namespace
}  // namespace sense

using namespace sense;

extern "C" int sense_smooth_map(const sense_smooth_opts* o, const float* w0, const float* wd,
                                const float* xhat, float* x, sense_smooth_info* info,
                                void* stream) {
  if (!o || !w0 || !wd || !xhat || !x) return set_error(SENSE_EINVAL, "null argument");
  if (o->nx < 1 || o->ny < 1 || o->nz < 1 || (o->order != 1 && o->order != 2) ||
      !(o->alpha >= 0.0) || o->max_iter < 0 || !(o->rel_tol >= 0.0) ||
      (o->precond != SENSE_SMOOTH_PLAIN && o->precond != SENSE_SMOOTH_MULTIGRID))
    return set_error(SENSE_EINVAL,
                     "grid >= 1, order 1 or 2, alpha, max_iter, rel_tol >= 0, precond 0 or 1");
  const void* ptrs[] = {w0, wd, xhat, x};
  for (const void* p : ptrs)
    if (!is_device_pointer(p)) return set_error(SENSE_EINVAL, "fields must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  const Grid g = make_grid(o->nx, o->ny, o->nz);
  int dev = 0, sms = 1;
  SENSE_CUDA_TRY(cudaGetDevice(&dev));
  SENSE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = grid_for(g.total, sms);
  const bool mg = o->precond == SENSE_SMOOTH_MULTIGRID;

  Work W(st);
  float2* r = W.get<float2>(g.total);
  float2* p = W.get<float2>(g.total);
  float2* q = W.get<float2>(g.total);
  double* red = W.get<double>(grid * 2 + 8);
  unsigned* counter = W.get<unsigned>(1);
  if (!r || !p || !q || !red || !counter) return set_error(SENSE_ENOMEM, "smoothing workspace");
  double* sc = red + grid * 2;   // [rr, bb, stop, step, beta, iters, rz, -]
  float2* X = (float2*)x;
  const float2* XH = (const float2*)xhat;
  const float alpha = (float)o->alpha;
  const double tol2 = o->rel_tol * o->rel_tol;
  int rc = SENSE_OK;
  auto chk = [&](const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (rc == SENSE_OK && e != cudaSuccess) rc = cuda_error(e, what);
  };
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(sc, 0, 8 * sizeof(double), st) != cudaSuccess ||
      (X != XH && cudaMemcpyAsync(X, XH, (size_t)g.total * 8, cudaMemcpyDeviceToDevice, st) !=
                      cudaSuccess))
    return cuda_error(cudaGetLastError(), "smoothing set-up");

  // ------------------------------------------------------------ multigrid hierarchy
  std::vector<Level> L;
  unsigned char* keep = nullptr;
  float2* z = nullptr;
  if (mg) {
    keep = W.get<unsigned char>(g.total);
    z = nullptr;
    Grid gl = g;
    int e0[3];
    for (int d = 0; d < 3; ++d) e0[d] = g.n[d] > 1 ? o->order : 0;
    Sten sl = make_cross(e0);
    while (true) {
      Level v;
      v.g = gl;
      v.s = sl;
      v.grid = grid_for(gl.total, sms);
      const bool coarsest = gl.total <= COARSE_MAX || (int)L.size() + 1 >= MAX_LEVELS;
      v.coef = W.get<float>((size_t)sl.count * gl.total);
      v.dinv = W.get<float>(gl.total);
      v.x = W.get<float2>(gl.total);
      if (!v.coef || !v.dinv || !v.x || !keep) return set_error(SENSE_ENOMEM, "multigrid levels");
      if (!coarsest) {
        v.xo = W.get<float2>(gl.total);
        v.r = W.get<float2>(gl.total);
        v.d0 = W.get<float2>(gl.total);
        v.d1 = W.get<float2>(gl.total);
        if (!v.xo || !v.r || !v.d0 || !v.d1) return set_error(SENSE_ENOMEM, "multigrid levels");
      }
      if (!L.empty()) {
        v.b = W.get<float2>(gl.total);
        if (!v.b) return set_error(SENSE_ENOMEM, "multigrid levels");
      }
      L.push_back(v);
      if (coarsest) break;
      int ec[3];
      int nc[3];
      for (int d = 0; d < 3; ++d) {
        nc[d] = (gl.n[d] + 1) / 2;
        ec[d] = nc[d] > 1 ? (sl.e[d] + 2) / 2 : 0;
      }
      gl = make_grid(nc[0], nc[1], nc[2]);
      sl = make_box(ec);
    }
    if (gl.total > COARSE_MAX) return set_error(SENSE_EINVAL, "grid too large for the multigrid");
    // operators
    unsigned* gmax = W.get<unsigned>(L.size());
    double* lam2 = W.get<double>(L.size());
    float2* pw = W.get<float2>(g.total);
    float2* pv = W.get<float2>(g.total);
    if (!gmax || !lam2 || !pw || !pv) return set_error(SENSE_ENOMEM, "multigrid set-up");
    if (cudaMemsetAsync(gmax, 0, L.size() * sizeof(unsigned), st) != cudaSuccess)
      return cuda_error(cudaGetLastError(), "multigrid set-up");
    for (size_t l = 0; l < L.size() && rc == SENSE_OK; ++l) {
      Level& v = L[l];
      if (l == 0) {
        if (cudaMemsetAsync(v.coef, 0, (size_t)v.s.count * v.g.total * sizeof(float), st) !=
            cudaSuccess)
          return cuda_error(cudaGetLastError(), "multigrid set-up");
        mg_fine_kernel<<<v.grid, VB, 0, st>>>(v.g, v.s, o->order, alpha, w0, wd, v.coef, keep);
      } else {
        const Level& f = L[l - 1];
        if (cudaMemsetAsync(v.coef, 0, (size_t)v.s.count * v.g.total * sizeof(float), st) !=
            cudaSuccess)
          return cuda_error(cudaGetLastError(), "multigrid set-up");
        mg_galerkin_kernel<<<grid_for(v.g.total, sms), 128, 0, st>>>(f.g, f.s, f.coef, v.g, v.s,
                                                                     v.coef);
      }
      mg_diag_kernel<<<v.grid, VB, 0, st>>>(v.g, v.s, v.coef, v.dinv, gmax + l);
      mg_vinit_kernel<<<v.grid, VB, 0, st>>>(pv, v.g.total);
      for (int k = 0; k < POWER_STEPS; ++k) {
        mg_power_kernel<<<v.grid, VB, 0, st>>>(v.g, v.s, v.coef, v.dinv, pv, pw, red, counter,
                                               lam2 + l);
        mg_normalize_kernel<<<v.grid, VB, 0, st>>>(pw, pv, v.g.total, lam2 + l);
      }
      chk("multigrid set-up");
    }
    if (rc != SENSE_OK) return rc;
    std::vector<unsigned> hg(L.size());
    std::vector<double> hl(L.size());
    if (cudaMemcpyAsync(hg.data(), gmax, L.size() * sizeof(unsigned), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(hl.data(), lam2, L.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return cuda_error(cudaGetLastError(), "multigrid set-up");
    for (size_t l = 0; l < L.size(); ++l) {
      float gb;
      std::memcpy(&gb, &hg[l], sizeof(float));
      double hi = POWER_SAFETY * std::sqrt(std::max(hl[l], 0.0));
      if (!(hi > 0.0) || !(hi <= (double)gb)) hi = gb;
      if (!(hi > 0.0) || !std::isfinite(hi)) hi = 1.0;
      const double lo = hi / CHEB_RATIO;
      Level& v = L[l];
      v.theta = 0.5 * (hi + lo);
      v.delta = 0.5 * (hi - lo);
      const double sigma = v.theta / v.delta;
      double rho = 1.0 / sigma;
      for (int k = 1; k < CHEB_DEG; ++k) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        v.c1[k] = (float)(rn * rho);
        v.c2[k] = (float)(2.0 * rn / v.delta);
        rho = rn;
      }
    }
  }

  // ------------------------------------------------------------ CG start
  smooth_apply_kernel<<<grid, VB, 0, st>>>(g, o->order, alpha, w0, wd, X, q, sc);
  chk("smooth apply");
  smooth_init_kernel<<<grid, VB, 0, st>>>(w0, XH, q, g.total, r, p, red, counter, sc, tol2);
  chk("smooth init");
  if (mg && rc == SENSE_OK) {
    z = vcycle(L, 0, r, sc, st);
    smooth_rz_kernel<<<grid, VB, 0, st>>>(z, r, keep, g.total, red, counter, sc, 1);
    smooth_p_kernel<<<grid, VB, 0, st>>>(p, z, g.total, sc);
    chk("smooth preconditioner");
  }
  // one iteration, as a sequence of launches on stream s
  auto iteration = [&](cudaStream_t s) {
    smooth_apply_kernel<<<grid, VB, 0, s>>>(g, o->order, alpha, w0, wd, p, q, sc);
    smooth_pap_kernel<<<grid, VB, 0, s>>>(p, q, g.total, red, counter, sc, mg ? 6 : 0);
    smooth_update_kernel<<<grid, VB, 0, s>>>(X, r, p, q, g.total, red, counter, sc, tol2);
    if (mg) {
      float2* zz = vcycle(L, 0, r, sc, s);
      smooth_rz_kernel<<<grid, VB, 0, s>>>(zz, r, keep, g.total, red, counter, sc, 0);
      smooth_p_kernel<<<grid, VB, 0, s>>>(p, zz, g.total, sc);
    } else {
      smooth_p_kernel<<<grid, VB, 0, s>>>(p, r, g.total, sc);
    }
  };

  // ------------------------------------------------------------ iterations (graph replays)
  cudaGraphExec_t exec = nullptr;
  double* hflag = nullptr;
  cudaEvent_t ev = nullptr;
  if (rc == SENSE_OK && o->max_iter > 0) {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      rc = cuda_error(cudaGetLastError(), "capture stream");
    } else {
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "cudaStreamBeginCapture");
      } else {
        iteration(cs);
        const cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess) rc = cuda_error(e, "cudaStreamEndCapture");
      }
      if (rc == SENSE_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "cudaGraphInstantiate");
        exec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cs);
    }
    if (rc == SENSE_OK && (cudaMallocHost((void**)&hflag, sizeof(double)) != cudaSuccess ||
                           cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess))
      rc = cuda_error(cudaGetLastError(), "smoothing poll buffers");
    // replay in batches; the stop flag of batch k is read while batch k + 1 runs
    bool pending = false;
    for (int done = 0; rc == SENSE_OK && done < o->max_iter;) {
      const int nb = std::min(POLL_EVERY, o->max_iter - done);
      for (int k = 0; k < nb && rc == SENSE_OK; ++k)
        if (cudaGraphLaunch(exec, st) != cudaSuccess)
          rc = cuda_error(cudaGetLastError(), "cudaGraphLaunch");
      done += nb;
      if (rc != SENSE_OK) break;
      if (pending) {
        if (cudaEventSynchronize(ev) != cudaSuccess) {
          rc = cuda_error(cudaGetLastError(), "smoothing poll");
          break;
        }
        if (*hflag != 0.0) break;
      }
      if (cudaMemcpyAsync(hflag, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaEventRecord(ev, st) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "smoothing poll");
        break;
      }
      pending = true;
    }
  }
  double h[6] = {0, 0, 0, 0, 0, 0};
  if (rc == SENSE_OK &&
      (cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = cuda_error(cudaGetLastError(), "smoothing result");
  if (rc == SENSE_OK && info) {
    info->iters = (int32_t)h[5];
    info->rel_residual = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : 0.0;
  }
  cudaStreamSynchronize(st);
  if (exec) cudaGraphExecDestroy(exec);
  if (ev) cudaEventDestroy(ev);
  if (hflag) cudaFreeHost(hflag);
  return rc;
}
