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
// Several fields (right-hand sides) are solved together: the matrix depends only on w0, wd and
// alpha, so one hierarchy serves them all, and every kernel runs over all fields at once (the
// second grid dimension), each field with its own CG scalars and stop flag. The paper smooths the
// magnitude and the magnitude-normalised map of every coil; sense_smooth_sensitivities makes
// those 2 C fields, solves them in one call and recombines them.
//
// Each CG iteration is captured once in a CUDA graph and replayed; the host reads the count of
// stopped fields (tolerance reached or breakdown) one batch of replays behind, and every kernel
// returns at once for a field that has stopped.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
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
// CG on the normal equations, for F fields at once (blockIdx.y = field; field f's vectors
// start at f * n, its scalars at sc + 8 f, its reduction partials at part + f * pstride and
// its completion counter at counter[f]). Every kernel skips the fields that have stopped.
// ---------------------------------------------------------------------------------------

// Scalars of a field: 0 r^H r, 1 ||b||^2, 2 stop flag, 3 step length, 4 beta, 5 iterations,
// 6 r^H z (preconditioned). nstop counts the fields that have stopped.
constexpr int NSC = 8;

__device__ __forceinline__ void set_stop(double* s, unsigned* nstop) {
  if (s[2] == 0.0) {
    s[2] = 1.0;
    atomicAdd(nstop, 1u);
  }
}

// r = w0^2 xhat - y (y = N x_0), p = r; sums ||r||^2 and ||w0^2 xhat||^2 and the stop test
__global__ void __launch_bounds__(VB) smooth_init_kernel(const float* __restrict__ w0,
                                                         const float2* __restrict__ xhatb,
                                                         const float2* __restrict__ yb,
                                                         long long n, float2* rb, float2* pb,
                                                         double* part, long long pstride,
                                                         unsigned* counter, double* sc,
                                                         unsigned* nstop, double tol2) {
  __shared__ double sh[2 * VB / 32];
  const int f = blockIdx.y;
  const long long o = (long long)f * n;
  // per-thread partials in FP32 (a few elements each), block and grid sums in FP64
  float a[2] = {0.f, 0.f};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a0 = w0[i] * w0[i];
    const float2 xh = xhatb[o + i], y = yb[o + i];
    const float2 b = make_float2(a0 * xh.x, a0 * xh.y);
    const float2 ri = make_float2(b.x - y.x, b.y - y.y);
    rb[o + i] = ri;
    pb[o + i] = ri;
    a[0] = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, a[0]));
    a[1] = fmaf(b.x, b.x, fmaf(b.y, b.y, a[1]));
  }
  double v[2] = {(double)a[0], (double)a[1]};
  block_sum<2>(v, sh);
  double tot[2];
  if (finish_sums<2>(v, part + f * pstride, counter + f, tot)) {
    double* s = sc + f * NSC;
    s[0] = tot[0];   // r^H r
    s[1] = tot[1];   // ||b||^2
    if (tot[0] <= tol2 * tot[1]) set_stop(s, nstop);
  }
}

// step length = (r^H z or r^H r) / p^H N p (N real symmetric: p^H N p real)
__global__ void __launch_bounds__(VB) smooth_pap_kernel(const float2* __restrict__ pb,
                                                        const float2* __restrict__ qb, long long n,
                                                        double* part, long long pstride,
                                                        unsigned* counter, double* sc,
                                                        unsigned* nstop, int num) {
  const int f = blockIdx.y;
  double* s = sc + f * NSC;
  if (s[2] != 0.0) return;
  __shared__ double sh[VB / 32];
  const float2* p = pb + (long long)f * n;
  const float2* q = qb + (long long)f * n;
  float a = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    a = fmaf(p[i].x, q[i].x, fmaf(p[i].y, q[i].y, a));
  double v[1] = {(double)a};
  block_sum<1>(v, sh);
  double tot[1];
  if (finish_sums<1>(v, part + f * pstride, counter + f, tot)) {
    if (!(tot[0] > 0.0)) {
      set_stop(s, nstop);
      return;
    }
    s[3] = s[num] / tot[0];
  }
}

// x += a p; r -= a q; the new r^H r, beta for plain CG, the iteration count and the stop test
__global__ void __launch_bounds__(VB) smooth_update_kernel(float2* xb, float2* rb,
                                                           const float2* __restrict__ pb,
                                                           const float2* __restrict__ qb,
                                                           long long n, double* part,
                                                           long long pstride, unsigned* counter,
                                                           double* sc, unsigned* nstop,
                                                           double tol2) {
  const int f = blockIdx.y;
  double* s = sc + f * NSC;
  if (s[2] != 0.0) return;
  __shared__ double sh[VB / 32];
  const long long o = (long long)f * n;
  const float a = (float)s[3];
  float acc = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 pi = pb[o + i], qi = qb[o + i];
    float2 xi = xb[o + i];
    xi.x += a * pi.x;
    xi.y += a * pi.y;
    xb[o + i] = xi;
    const float2 ri = make_float2(rb[o + i].x - a * qi.x, rb[o + i].y - a * qi.y);
    rb[o + i] = ri;
    acc = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, acc));
  }
  double v[1] = {(double)acc};
  block_sum<1>(v, sh);
  double tot[1];
  if (finish_sums<1>(v, part + f * pstride, counter + f, tot)) {
    s[4] = tot[0] / s[0];   // beta (plain CG)
    s[0] = tot[0];
    s[5] += 1.0;            // iterations
    if (tot[0] <= tol2 * s[1]) set_stop(s, nstop);
  }
}

// Preconditioned CG: z <- 0 at unconstrained voxels, r^H z, beta = r^H z / (previous r^H z)
// (first = 1: beta = 0, so that the next direction is z itself)
__global__ void __launch_bounds__(VB) smooth_rz_kernel(float2* zb, const float2* __restrict__ rb,
                                                       const unsigned char* __restrict__ keep,
                                                       long long n, double* part,
                                                       long long pstride, unsigned* counter,
                                                       double* sc, unsigned* nstop, int first) {
  const int f = blockIdx.y;
  double* s = sc + f * NSC;
  if (s[2] != 0.0) return;
  __shared__ double sh[VB / 32];
  const long long o = (long long)f * n;
  float a = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float2 zi = zb[o + i];
    if (!keep[i]) {
      zi = make_float2(0.f, 0.f);
      zb[o + i] = zi;
    }
    a = fmaf(rb[o + i].x, zi.x, fmaf(rb[o + i].y, zi.y, a));
  }
  double v[1] = {(double)a};
  block_sum<1>(v, sh);
  double tot[1];
  if (finish_sums<1>(v, part + f * pstride, counter + f, tot)) {
    if (!(tot[0] > 0.0)) {
      set_stop(s, nstop);   // breakdown (or r = 0)
      return;
    }
    s[4] = first ? 0.0 : tot[0] / s[6];
    s[6] = tot[0];
  }
}

// p = z + beta p (z = r for plain CG)
__global__ void smooth_p_kernel(float2* pb, const float2* __restrict__ zb, long long n,
                                const double* sc) {
  const int f = blockIdx.y;
  const double* s = sc + f * NSC;
  if (s[2] != 0.0) return;
  const long long o = (long long)f * n;
  const float b = (float)s[4];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    pb[o + i] = make_float2(zb[o + i].x + b * pb[o + i].x, zb[o + i].y + b * pb[o + i].y);
}

// ---------------------------------------------------------------------------------------
// Multigrid hierarchy (shared by all fields)
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
// V-cycle kernels: blockIdx.y = field, vectors of level size n at f * n (the coarsest-grid
// kernel: one block per field); each returns at once for a field whose CG has stopped
// ---------------------------------------------------------------------------------------

// Chebyshev start from x = 0: r = b, d = D^-1 b / theta, x = d
__global__ void cheb_first0_kernel(long long n, const float* __restrict__ dinv,
                                   const float2* __restrict__ bb, float2* xb, float2* rb,
                                   float2* db, float inv_theta, const double* sc) {
  const int f = blockIdx.y;
  if (sc[f * NSC + 2] != 0.0) return;
  const long long o = (long long)f * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 bi = bb[o + i];
    const float s = dinv[i] * inv_theta;
    const float2 di = make_float2(s * bi.x, s * bi.y);
    rb[o + i] = bi;
    db[o + i] = di;
    xb[o + i] = di;
  }
}

// Stencil kernels take the fields in chunks of FC (blockIdx.y = chunk), so that every
// coefficient is loaded once per voxel and applied to FC fields.
constexpr int FC = 8;

// bit k set: field f0 + k exists and has not stopped (f0 = first field of this block's chunk)
__device__ __forceinline__ unsigned chunk_active(int F, const double* sc, int& f0) {
  f0 = blockIdx.y * FC;
  unsigned m = 0;
#pragma unroll
  for (int k = 0; k < FC; ++k)
    if (f0 + k < F && sc[(f0 + k) * NSC + 2] == 0.0) m |= 1u << k;
  return m;
}

// acc[k] = (A v_{f0 + k})_i for the active fields of the chunk
__device__ __forceinline__ void sten_apply_chunk(const Grid& g, const Sten& s, const float* c,
                                                 const float2* vb, long long i,
                                                 const int (&ci)[3], int f0, unsigned act,
                                                 float2 (&acc)[FC]) {
#pragma unroll
  for (int k = 0; k < FC; ++k) acc[k] = make_float2(0.f, 0.f);
  for_offsets(s, [&](int o, int dx, int dy, int dz) {
    const int x = ci[0] + dx, y = ci[1] + dy, z = ci[2] + dz;
    if (x < 0 || x >= g.n[0] || y < 0 || y >= g.n[1] || z < 0 || z >= g.n[2]) return;
    const float a = c[(long long)o * g.total + i];
    if (a == 0.f) return;
    const long long j = i + dx * g.stride[0] + dy * g.stride[1] + dz * g.stride[2];
#pragma unroll
    for (int k = 0; k < FC; ++k)
      if ((act >> k) & 1u) {
        const float2 w = vb[(long long)(f0 + k) * g.total + j];
        acc[k].x = fmaf(a, w.x, acc[k].x);
        acc[k].y = fmaf(a, w.y, acc[k].y);
      }
  });
}

// y = w0^2 x + alpha sum_d D_d^T diag(wd^2) D_d x, matrix-free (the differences are taken of x
// itself, so fields in the null space of D stay there exactly), FC fields per block
__global__ void smooth_apply_kernel(Grid g, int order, float alpha, const float* __restrict__ w0,
                                    const float* __restrict__ wd, const float2* __restrict__ xb,
                                    float2* __restrict__ yb, int F, const double* sc) {
  int f0;
  const unsigned act = chunk_active(F, sc, f0);
  if (!act) return;
  const long long n = g.total;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int c[3];
    coords(g, i, c);
    const float a0 = w0[i] * w0[i];
    float2 acc[FC];
#pragma unroll
    for (int k = 0; k < FC; ++k) {
      acc[k] = make_float2(0.f, 0.f);
      if ((act >> k) & 1u) {
        const float2 xi = xb[(long long)(f0 + k) * n + i];
        acc[k] = make_float2(a0 * xi.x, a0 * xi.y);
      }
    }
    for (int d = 0; d < 3; ++d) {
      const int nd = g.n[d];
      if (nd < 2) continue;
      const long long s = g.stride[d];
      if (order == 1) {
        // rows r = i - 1 (coefficient +1 on x[i]) and r = i (coefficient -1)
        const bool lo = c[d] >= 1, hi = c[d] + 1 < nd;
        const float wl = lo ? wd[i - s] * wd[i - s] : 0.f;
        const float wh = hi ? wd[i] * wd[i] : 0.f;
#pragma unroll
        for (int k = 0; k < FC; ++k) {
          if (!((act >> k) & 1u)) continue;
          const float2* x = xb + (long long)(f0 + k) * n;
          float2 t = make_float2(0.f, 0.f);
          if (lo) {
            const float2 v = drow(g, x, i - s, d, 1);
            t.x += wl * v.x;
            t.y += wl * v.y;
          }
          if (hi) {
            const float2 v = drow(g, x, i, d, 1);
            t.x -= wh * v.x;
            t.y -= wh * v.y;
          }
          acc[k].x += alpha * t.x;
          acc[k].y += alpha * t.y;
        }
      } else {
        // rows r = i - 1 and i + 1 (coefficient +1 on x[i]) and r = i (coefficient -2)
        const bool ra = c[d] >= 2, rb = c[d] >= 1 && c[d] + 1 < nd, rc = c[d] + 2 < nd;
        const float wa = ra ? wd[i - s] * wd[i - s] : 0.f;
        const float wb = rb ? wd[i] * wd[i] : 0.f;
        const float wc = rc ? wd[i + s] * wd[i + s] : 0.f;
#pragma unroll
        for (int k = 0; k < FC; ++k) {
          if (!((act >> k) & 1u)) continue;
          const float2* x = xb + (long long)(f0 + k) * n;
          float2 t = make_float2(0.f, 0.f);
          if (ra) {
            const float2 v = drow(g, x, i - s, d, 2);
            t.x += wa * v.x;
            t.y += wa * v.y;
          }
          if (rb) {
            const float2 v = drow(g, x, i, d, 2);
            t.x -= 2.f * wb * v.x;
            t.y -= 2.f * wb * v.y;
          }
          if (rc) {
            const float2 v = drow(g, x, i + s, d, 2);
            t.x += wc * v.x;
            t.y += wc * v.y;
          }
          acc[k].x += alpha * t.x;
          acc[k].y += alpha * t.y;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < FC; ++k)
      if ((act >> k) & 1u) yb[(long long)(f0 + k) * n + i] = acc[k];
  }
}

// Chebyshev start from x: r = b - A x, d = D^-1 r / theta, xo = x + d
__global__ void cheb_first_kernel(Grid g, Sten s, const float* __restrict__ c,
                                  const float* __restrict__ dinv, const float2* __restrict__ bb,
                                  const float2* __restrict__ xb, float2* xob, float2* rb,
                                  float2* db, float inv_theta, int F, const double* sc) {
  int f0;
  const unsigned act = chunk_active(F, sc, f0);
  if (!act) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    coords(g, i, ci);
    float2 a[FC];
    sten_apply_chunk(g, s, c, xb, i, ci, f0, act, a);
    const float t = dinv[i] * inv_theta;
#pragma unroll
    for (int k = 0; k < FC; ++k)
      if ((act >> k) & 1u) {
        const long long o = (long long)(f0 + k) * g.total + i;
        const float2 ri = make_float2(bb[o].x - a[k].x, bb[o].y - a[k].y);
        const float2 di = make_float2(t * ri.x, t * ri.y);
        rb[o] = ri;
        db[o] = di;
        xob[o] = make_float2(xb[o].x + di.x, xb[o].y + di.y);
      }
  }
}

// Chebyshev step: r -= A dp; dn = c1 dp + c2 D^-1 r; x += dn
__global__ void cheb_step_kernel(Grid g, Sten s, const float* __restrict__ c,
                                 const float* __restrict__ dinv, const float2* __restrict__ dpb,
                                 float2* dnb, float2* rb, float2* xb, float c1, float c2, int F,
                                 const double* sc) {
  int f0;
  const unsigned act = chunk_active(F, sc, f0);
  if (!act) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    coords(g, i, ci);
    float2 a[FC];
    sten_apply_chunk(g, s, c, dpb, i, ci, f0, act, a);
    const float t = c2 * dinv[i];
#pragma unroll
    for (int k = 0; k < FC; ++k)
      if ((act >> k) & 1u) {
        const long long o = (long long)(f0 + k) * g.total + i;
        const float2 ri = make_float2(rb[o].x - a[k].x, rb[o].y - a[k].y);
        const float2 dp = dpb[o];
        const float2 di = make_float2(c1 * dp.x + t * ri.x, c1 * dp.y + t * ri.y);
        rb[o] = ri;
        dnb[o] = di;
        xb[o] = make_float2(xb[o].x + di.x, xb[o].y + di.y);
      }
  }
}

// r = b - A x
__global__ void mg_resid_kernel(Grid g, Sten s, const float* __restrict__ c,
                                const float2* __restrict__ bb, const float2* __restrict__ xb,
                                float2* rb, int F, const double* sc) {
  int f0;
  const unsigned act = chunk_active(F, sc, f0);
  if (!act) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    coords(g, i, ci);
    float2 a[FC];
    sten_apply_chunk(g, s, c, xb, i, ci, f0, act, a);
#pragma unroll
    for (int k = 0; k < FC; ++k)
      if ((act >> k) & 1u) {
        const long long o = (long long)(f0 + k) * g.total + i;
        rb[o] = make_float2(bb[o].x - a[k].x, bb[o].y - a[k].y);
      }
  }
}

// bc = P^T r
__global__ void mg_restrict_kernel(Grid gf, Grid gc, const float2* __restrict__ rb, float2* bcb,
                                   const double* sc) {
  const int f = blockIdx.y;
  if (sc[f * NSC + 2] != 0.0) return;
  const float2* r = rb + (long long)f * gf.total;
  float2* bc = bcb + (long long)f * gc.total;
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
__global__ void mg_prolong_kernel(Grid gf, Grid gc, const float2* __restrict__ xcb, float2* xb,
                                  const double* sc) {
  const int f = blockIdx.y;
  if (sc[f * NSC + 2] != 0.0) return;
  const float2* xc = xcb + (long long)f * gc.total;
  float2* x = xb + (long long)f * gf.total;
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

// Coarsest grid (at most COARSE_MAX nodes; one block of COARSE_MAX threads per field):
// COARSE_DEG Chebyshev steps from x = 0 with the vectors in shared memory
__global__ void __launch_bounds__(COARSE_MAX) mg_coarse_kernel(Grid g, Sten s,
                                                               const float* __restrict__ c,
                                                               const float* __restrict__ dinv,
                                                               const float2* __restrict__ bb,
                                                               float2* xb, double theta,
                                                               double delta, const double* sc) {
  const int f = blockIdx.x;
  if (sc[f * NSC + 2] != 0.0) return;   // uniform over the block
  __shared__ float2 sd[2][COARSE_MAX];
  __shared__ float scoef[125 * COARSE_MAX];   // a box of half-width 2 in 3D at most
  for (int k = threadIdx.x; k < s.count * COARSE_MAX; k += blockDim.x) {
    const int oo = k / COARSE_MAX, ii = k - oo * COARSE_MAX;
    scoef[k] = ii < g.total ? c[(long long)oo * g.total + ii] : 0.f;
  }
  const long long o = (long long)f * g.total;
  const int i = threadIdx.x;
  const bool on = i < g.total;
  int ci[3] = {0, 0, 0};
  float2 ri = make_float2(0.f, 0.f), xi = make_float2(0.f, 0.f);
  float di_inv = 0.f;
  if (on) {
    coords(g, i, ci);
    di_inv = dinv[i];
    ri = bb[o + i];
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
      for_offsets(s, [&](int oo, int dx, int dy, int dz) {
        const int xx = ci[0] + dx, yy = ci[1] + dy, zz = ci[2] + dz;
        if (xx < 0 || xx >= g.n[0] || yy < 0 || yy >= g.n[1] || zz < 0 || zz >= g.n[2]) return;
        const float cv = scoef[oo * COARSE_MAX + i];
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
  if (on) xb[o + i] = xi;
}

// Sensitivity maps (Eq. 1 as the paper applies it): the magnitude and the magnitude-normalised
// map of every coil are smoothed as separate fields. Split S[l][c] into field c = |S| and field
// C + c = S / |S| (0 where S = 0), each [L] in raster order.
__global__ void sens_split_kernel(const float2* __restrict__ S, long long L, int C,
                                  float2* fields) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < L * C;
       t += (long long)gridDim.x * blockDim.x) {
    const long long l = t / C;
    const int c = (int)(t - l * C);
    const float2 v = S[t];
    const float m = hypotf(v.x, v.y);
    fields[(long long)c * L + l] = make_float2(m, 0.f);
    fields[(long long)(C + c) * L + l] =
        m > 0.f ? make_float2(v.x / m, v.y / m) : make_float2(0.f, 0.f);
  }
}

// Recombine: S[l][c] = m * u / |u| with m the smoothed magnitude (real part of field c) and u
// the smoothed normalised map (field C + c); 0 where u = 0
__global__ void sens_combine_kernel(const float2* __restrict__ fields, long long L, int C,
                                    float2* S) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < L * C;
       t += (long long)gridDim.x * blockDim.x) {
    const long long l = t / C;
    const int c = (int)(t - l * C);
    const float m = fields[(long long)c * L + l].x;
    const float2 u = fields[(long long)(C + c) * L + l];
    const float a = hypotf(u.x, u.y);
    S[t] = a > 0.f ? make_float2(m * u.x / a, m * u.y / a) : make_float2(0.f, 0.f);
  }
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
  int grid = 1;   // blocks of the single-field set-up kernels
  dim3 gF, gC;    // grids of the per-field and the field-chunk kernels
};

// Workspace comes from a stream-ordered memory pool of the library's own (one per device),
// which keeps up to 1 GiB of freed blocks for the next call: repeated solves then allocate in
// microseconds instead of one cudaMalloc per buffer.
cudaMemPool_t work_pool(int dev) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  uint64_t keep = 1ull << 30;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  pools[dev] = pool;
  return pool;
}

// device buffers of one call, allocated and freed in stream order on the call's stream
struct Work {
  cudaStream_t st;
  cudaMemPool_t pool = nullptr;
  std::vector<void*> bufs;
  explicit Work(cudaStream_t s) : st(s) {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) pool = work_pool(dev);
  }
  ~Work() {
    for (void* p : bufs) cudaFreeAsync(p, st);
  }
  template <class T>
  T* get(size_t count) {
    void* p = nullptr;
    if (!pool ||
        cudaMallocFromPoolAsync(&p, std::max<size_t>(count, 1) * sizeof(T), pool, st) !=
            cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    bufs.push_back(p);
    return (T*)p;
  }
};

// pinned word the host polls the stopped-field count into (one per host thread, kept)
unsigned* poll_word() {
  thread_local unsigned* w = nullptr;
  if (!w && cudaHostAlloc((void**)&w, sizeof(unsigned), cudaHostAllocPortable) != cudaSuccess) {
    cudaGetLastError();
    w = nullptr;
  }
  return w;
}

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

// grid of a kernel over `rows` fields (or field chunks) of n elements: about 8 blocks per SM in
// all, each thread taking several elements when there are many fields
dim3 grid_rows(long long n, int rows, int sms) {
  const long long per = std::max<long long>(1, (8LL * sms + rows - 1) / rows);
  return dim3((unsigned)std::max<long long>(1, std::min<long long>((n + VB - 1) / VB, per)),
              (unsigned)rows);
}

// V-cycle on level l for F fields: output in L[l].xo (or L[l].x on the coarsest level);
// returns that buffer
float2* vcycle(std::vector<Level>& L, size_t l, const float2* b, int F, const double* sc,
               cudaStream_t st) {
  Level& v = L[l];
  if (l + 1 == L.size()) {
    mg_coarse_kernel<<<F, COARSE_MAX, 0, st>>>(v.g, v.s, v.coef, v.dinv, b, v.x, v.theta, v.delta,
                                               sc);
    return v.x;
  }
  const dim3 grid = v.gF;
  const dim3 gridc = v.gC;
  const float inv_theta = (float)(1.0 / v.theta);
  // pre-smoothing from x = 0
  cheb_first0_kernel<<<grid, VB, 0, st>>>(v.g.total, v.dinv, b, v.x, v.r, v.d0, inv_theta, sc);
  float2 *dp = v.d0, *dn = v.d1;
  for (int k = 1; k < CHEB_DEG; ++k) {
    cheb_step_kernel<<<gridc, VB, 0, st>>>(v.g, v.s, v.coef, v.dinv, dp, dn, v.r, v.x, v.c1[k],
                                           v.c2[k], F, sc);
    std::swap(dp, dn);
  }
  // coarse-grid correction
  mg_resid_kernel<<<gridc, VB, 0, st>>>(v.g, v.s, v.coef, b, v.x, v.r, F, sc);
  Level& w = L[l + 1];
  mg_restrict_kernel<<<w.gF, VB, 0, st>>>(v.g, w.g, v.r, w.b, sc);
  const float2* xc = vcycle(L, l + 1, w.b, F, sc, st);
  mg_prolong_kernel<<<grid, VB, 0, st>>>(v.g, w.g, xc, v.x, sc);
  // post-smoothing (the same polynomial) from the corrected x
  cheb_first_kernel<<<gridc, VB, 0, st>>>(v.g, v.s, v.coef, v.dinv, b, v.x, v.xo, v.r, v.d0,
                                          inv_theta, F, sc);
  dp = v.d0;
  dn = v.d1;
  for (int k = 1; k < CHEB_DEG; ++k) {
    cheb_step_kernel<<<gridc, VB, 0, st>>>(v.g, v.s, v.coef, v.dinv, dp, dn, v.r, v.xo,
                                           v.c1[k], v.c2[k], F, sc);
    std::swap(dp, dn);
  }
  return v.xo;
}

// Solve N x_f = w0^2 xhat_f for the F fields of xhat (field-major, F x n complex) into x.
int smooth_solve(const sense_smooth_opts* o, int F, const float* w0, const float* wd,
                 const float2* XH, float2* X, sense_smooth_info* info, cudaStream_t st) {
  const Grid g = make_grid(o->nx, o->ny, o->nz);
  int dev = 0, sms = 1;
  SENSE_CUDA_TRY(cudaGetDevice(&dev));
  SENSE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = grid_for(g.total, sms);
  const dim3 gridF = grid_rows(g.total, F, sms);
  const dim3 gridC = grid_rows(g.total, (F + FC - 1) / FC, sms);
  // partial sums: 2 per block of each field's reduction kernels (gridF.x blocks); the
  // single-field set-up kernels of the hierarchy use field 0's region with up to `grid` blocks
  const long long pstride = 2LL * gridF.x;
  const long long nF = (long long)F * g.total;
  const bool mg = o->precond == SENSE_SMOOTH_MULTIGRID;

  Work W(st);
  float2* r = W.get<float2>(nF);
  float2* p = W.get<float2>(nF);
  float2* q = W.get<float2>(nF);
  double* part = W.get<double>((size_t)std::max<long long>(F * pstride, 2LL * grid));
  unsigned* counter = W.get<unsigned>(F + 1);
  double* sc = W.get<double>((size_t)F * NSC);
  if (!r || !p || !q || !part || !counter || !sc)
    return set_error(SENSE_ENOMEM, "smoothing workspace");
  unsigned* nstop = counter + F;
  const float alpha = (float)o->alpha;
  const double tol2 = o->rel_tol * o->rel_tol;
  int rc = SENSE_OK;
  auto chk = [&](const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (rc == SENSE_OK && e != cudaSuccess) rc = cuda_error(e, what);
  };
  if (cudaMemsetAsync(counter, 0, (F + 1) * sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(sc, 0, (size_t)F * NSC * sizeof(double), st) != cudaSuccess ||
      (X != XH &&
       cudaMemcpyAsync(X, XH, (size_t)nF * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess))
    return cuda_error(cudaGetLastError(), "smoothing set-up");

  // ------------------------------------------------------------ multigrid hierarchy
  std::vector<Level> L;
  unsigned char* keep = nullptr;
  if (mg) {
    keep = W.get<unsigned char>(g.total);
    if (!keep) return set_error(SENSE_ENOMEM, "multigrid levels");
    Grid gl = g;
    int e0[3];
    for (int d = 0; d < 3; ++d) e0[d] = g.n[d] > 1 ? o->order : 0;
    Sten sl = make_cross(e0);
    while (true) {
      Level v;
      v.g = gl;
      v.s = sl;
      v.grid = grid_for(gl.total, sms);
      v.gF = grid_rows(gl.total, F, sms);
      v.gC = grid_rows(gl.total, (F + FC - 1) / FC, sms);
      const bool coarsest = gl.total <= COARSE_MAX || (int)L.size() + 1 >= MAX_LEVELS;
      const size_t nl = (size_t)F * gl.total;
      v.coef = W.get<float>((size_t)sl.count * gl.total);
      v.dinv = W.get<float>(gl.total);
      v.x = W.get<float2>(nl);
      if (!v.coef || !v.dinv || !v.x) return set_error(SENSE_ENOMEM, "multigrid levels");
      if (!coarsest) {
        v.xo = W.get<float2>(nl);
        v.r = W.get<float2>(nl);
        v.d0 = W.get<float2>(nl);
        v.d1 = W.get<float2>(nl);
        if (!v.xo || !v.r || !v.d0 || !v.d1) return set_error(SENSE_ENOMEM, "multigrid levels");
      }
      if (!L.empty()) {
        v.b = W.get<float2>(nl);
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
    if (gl.total > COARSE_MAX || L.back().s.count > 125)
      return set_error(SENSE_EINVAL, "grid too large for the multigrid");
    // operators (field-independent)
    unsigned* gmax = W.get<unsigned>(L.size());
    double* lam2 = W.get<double>(L.size());
    float2* pw = W.get<float2>(g.total);
    float2* pv = W.get<float2>(g.total);
    if (!gmax || !lam2 || !pw || !pv) return set_error(SENSE_ENOMEM, "multigrid set-up");
    if (cudaMemsetAsync(gmax, 0, L.size() * sizeof(unsigned), st) != cudaSuccess)
      return cuda_error(cudaGetLastError(), "multigrid set-up");
    for (size_t l = 0; l < L.size() && rc == SENSE_OK; ++l) {
      Level& v = L[l];
      if (cudaMemsetAsync(v.coef, 0, (size_t)v.s.count * v.g.total * sizeof(float), st) !=
          cudaSuccess)
        return cuda_error(cudaGetLastError(), "multigrid set-up");
      if (l == 0) {
        mg_fine_kernel<<<v.grid, VB, 0, st>>>(v.g, v.s, o->order, alpha, w0, wd, v.coef, keep);
      } else {
        const Level& f = L[l - 1];
        mg_galerkin_kernel<<<grid_for(v.g.total, sms), 128, 0, st>>>(f.g, f.s, f.coef, v.g, v.s,
                                                                     v.coef);
      }
      mg_diag_kernel<<<v.grid, VB, 0, st>>>(v.g, v.s, v.coef, v.dinv, gmax + l);
      mg_vinit_kernel<<<v.grid, VB, 0, st>>>(pv, v.g.total);
      for (int k = 0; k < POWER_STEPS; ++k) {
        mg_power_kernel<<<v.grid, VB, 0, st>>>(v.g, v.s, v.coef, v.dinv, pv, pw, part, counter,
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
  smooth_apply_kernel<<<gridC, VB, 0, st>>>(g, o->order, alpha, w0, wd, X, q, F, sc);
  chk("smooth apply");
  smooth_init_kernel<<<gridF, VB, 0, st>>>(w0, XH, q, g.total, r, p, part, pstride, counter, sc,
                                           nstop, tol2);
  chk("smooth init");
  if (mg && rc == SENSE_OK) {
    float2* z = vcycle(L, 0, r, F, sc, st);
    smooth_rz_kernel<<<gridF, VB, 0, st>>>(z, r, keep, g.total, part, pstride, counter, sc,
                                           nstop, 1);
    smooth_p_kernel<<<gridF, VB, 0, st>>>(p, z, g.total, sc);
    chk("smooth preconditioner");
  }
  // one iteration, as a sequence of launches on stream s
  auto iteration = [&](cudaStream_t s) {
    smooth_apply_kernel<<<gridC, VB, 0, s>>>(g, o->order, alpha, w0, wd, p, q, F, sc);
    smooth_pap_kernel<<<gridF, VB, 0, s>>>(p, q, g.total, part, pstride, counter, sc, nstop,
                                           mg ? 6 : 0);
    smooth_update_kernel<<<gridF, VB, 0, s>>>(X, r, p, q, g.total, part, pstride, counter, sc,
                                              nstop, tol2);
    if (mg) {
      float2* z = vcycle(L, 0, r, F, sc, s);
      smooth_rz_kernel<<<gridF, VB, 0, s>>>(z, r, keep, g.total, part, pstride, counter, sc,
                                            nstop, 0);
      smooth_p_kernel<<<gridF, VB, 0, s>>>(p, z, g.total, sc);
    } else {
      smooth_p_kernel<<<gridF, VB, 0, s>>>(p, r, g.total, sc);
    }
  };

  // ------------------------------------------------------------ iterations (graph replays)
  cudaGraphExec_t exec = nullptr;
  unsigned* hstop = nullptr;
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
    hstop = poll_word();
    if (rc == SENSE_OK && (!hstop || cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) !=
                                         cudaSuccess))
      rc = cuda_error(cudaGetLastError(), "smoothing poll buffers");
    // replay in batches; the stopped-field count of batch k is read while batch k + 1 runs
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
        if (*hstop >= (unsigned)F) break;
      }
      if (cudaMemcpyAsync(hstop, nstop, sizeof(unsigned), cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaEventRecord(ev, st) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "smoothing poll");
        break;
      }
      pending = true;
    }
  }
  std::vector<double> h((size_t)F * NSC, 0.0);
  if (rc == SENSE_OK &&
      (cudaMemcpyAsync(h.data(), sc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
           cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = cuda_error(cudaGetLastError(), "smoothing result");
  if (rc == SENSE_OK && info)
    for (int f = 0; f < F; ++f) {
      const double* s = &h[(size_t)f * NSC];
      info[f].iters = (int32_t)s[5];
      info[f].rel_residual = s[1] > 0.0 ? std::sqrt(s[0] / s[1]) : 0.0;
    }
  cudaStreamSynchronize(st);
  if (exec) cudaGraphExecDestroy(exec);
  if (ev) cudaEventDestroy(ev);
  return rc;
}

int check_opts(const sense_smooth_opts* o) {
  if (o->nx < 1 || o->ny < 1 || o->nz < 1 || (o->order != 1 && o->order != 2) ||
      !(o->alpha >= 0.0) || o->max_iter < 0 || !(o->rel_tol >= 0.0) || o->n_fields < 1 ||
      o->n_fields > 65535 ||
      (o->precond != SENSE_SMOOTH_PLAIN && o->precond != SENSE_SMOOTH_MULTIGRID))
    return set_error(SENSE_EINVAL,
                     "grid >= 1, order 1 or 2, alpha, max_iter, rel_tol >= 0, n_fields in "
                     "[1, 65535], precond 0 or 1");
  return SENSE_OK;
}

}  // namespace
}  // namespace sense

using namespace sense;

extern "C" int sense_smooth_map(const sense_smooth_opts* o, const float* w0, const float* wd,
                                const float* xhat, float* x, sense_smooth_info* info,
                                void* stream) {
  if (!o || !w0 || !wd || !xhat || !x) return set_error(SENSE_EINVAL, "null argument");
  if (const int rc = check_opts(o)) return rc;
  const void* ptrs[] = {w0, wd, xhat, x};
  for (const void* p : ptrs)
    if (!is_device_pointer(p)) return set_error(SENSE_EINVAL, "fields must be device memory");
  return smooth_solve(o, o->n_fields, w0, wd, (const float2*)xhat, (float2*)x, info,
                      (cudaStream_t)stream);
}

extern "C" int sense_smooth_sensitivities(const sense_smooth_opts* o, int32_t C, const float* w0,
                                          const float* wd, const float* S_hat, float* S,
                                          sense_smooth_info* info, void* stream) {
  if (!o || !w0 || !wd || !S_hat || !S) return set_error(SENSE_EINVAL, "null argument");
  if (C < 1 || 2LL * C > 65535) return set_error(SENSE_EINVAL, "coils in [1, 32767]");
  sense_smooth_opts oo = *o;
  oo.n_fields = 2 * C;
  if (const int rc = check_opts(&oo)) return rc;
  const void* ptrs[] = {w0, wd, S_hat, S};
  for (const void* p : ptrs)
    if (!is_device_pointer(p)) return set_error(SENSE_EINVAL, "maps must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  const long long L = (long long)o->nx * o->ny * o->nz;
  int dev = 0, sms = 1;
  SENSE_CUDA_TRY(cudaGetDevice(&dev));
  SENSE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  Work W(st);
  float2* fields = W.get<float2>((size_t)2 * C * L);
  if (!fields) return set_error(SENSE_ENOMEM, "sensitivity fields");
  const int grid = grid_for(L * C, sms);
  sens_split_kernel<<<grid, VB, 0, st>>>((const float2*)S_hat, L, C, fields);
  SENSE_CUDA_TRY(cudaGetLastError());
  const int rc = smooth_solve(&oo, 2 * C, w0, wd, fields, fields, info, st);
  if (rc != SENSE_OK) return rc;
  sens_combine_kernel<<<grid, VB, 0, st>>>(fields, L, C, (float2*)S);
  SENSE_CUDA_TRY(cudaGetLastError());
  SENSE_CUDA_TRY(cudaStreamSynchronize(st));
  return SENSE_OK;
}
