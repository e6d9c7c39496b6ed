// Map smoothing and extrapolation (Eq. 1 for sensitivity maps, Eq. 3 for the B0 map).
//
// Both equations are least-squares systems A x = [w0 o xhat; 0; ...; 0] with
//   A = [diag(w0); sqrt(alpha) diag(wd) D_x; sqrt(alpha) diag(wd) D_y; sqrt(alpha) diag(wd) D_z]
// where D is the second difference (Eq. 1: w0 = the trusted mask M_T, wd = the reconstruction
// mask M_R) or the first difference (Eq. 3: w0 = 1, wd = the fit's standard error). Their normal
// equations (diag(w0^2) + alpha sum_d D_d^T diag(wd^2) D_d) x = diag(w0^2) xhat have a real,
// symmetric, positive semi-definite matrix; it is applied matrix-free as a stencil and solved by
// CG on complex fields (real and imaginary parts share the matrix) starting from xhat.
// A derivative row exists at voxel c along an axis when the stencil fits: second differences
// x[c-1] - 2 x[c] + x[c+1] at interior voxels, first differences x[c+1] - x[c] wherever c + 1 is
// on the grid; the row's weight is wd[c]. Axes of length 1 have no rows.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sense_internal.cuh"
#include "sense_reduce.cuh"

namespace sense {
namespace {

struct Grid {
  int n[3];
  long long stride[3];
  long long total;
};

__device__ __forceinline__ void coords(const Grid& g, long long i, int (&c)[3]) {
  c[0] = (int)(i % g.n[0]);
  c[1] = (int)((i / g.n[0]) % g.n[1]);
  c[2] = (int)(i / ((long long)g.n[0] * g.n[1]));
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

// y = w0^2 x + alpha sum_d D_d^T diag(wd^2) D_d x
__global__ void smooth_apply_kernel(Grid g, int order, float alpha, const float* __restrict__ w0,
                                    const float* __restrict__ wd, const float2* __restrict__ x,
                                    float2* __restrict__ y) {
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

// r = w0^2 xhat - y (y = A x_0), p = r; sums ||r||^2 and ||w0^2 xhat||^2
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

// alpha = r^H r / p^H A p (A real symmetric: p^H A p real); x += alpha p; r -= alpha A p;
// then the new r^H r and the stop test
__global__ void __launch_bounds__(VB) smooth_pap_kernel(const float2* __restrict__ p,
                                                        const float2* __restrict__ q, long long n,
                                                        double* part, unsigned* counter,
                                                        double* sc) {
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
    sc[3] = sc[0] / tot[0];   // step length
  }
}

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
    sc[4] = tot[0] / sc[0];   // beta
    sc[0] = tot[0];
    sc[5] += 1.0;             // iterations
    if (tot[0] <= tol2 * sc[1]) sc[2] = 1.0;
  }
}

__global__ void smooth_p_kernel(float2* p, const float2* __restrict__ r, long long n,
                                const double* sc) {
  if (sc[2] != 0.0) return;
  const float b = (float)sc[4];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = make_float2(r[i].x + b * p[i].x, r[i].y + b * p[i].y);
}

}  // namespace
}  // namespace sense

using namespace sense;

extern "C" int sense_smooth_map(const sense_smooth_opts* o, const float* w0, const float* wd,
                                const float* xhat, float* x, sense_smooth_info* info,
                                void* stream) {
  if (!o || !w0 || !wd || !xhat || !x) return set_error(SENSE_EINVAL, "null argument");
  if (o->nx < 1 || o->ny < 1 || o->nz < 1 || (o->order != 1 && o->order != 2) ||
      !(o->alpha >= 0.0) || o->max_iter < 0 || !(o->rel_tol >= 0.0))
    return set_error(SENSE_EINVAL, "grid >= 1, order 1 or 2, alpha, max_iter, rel_tol >= 0");
  const void* ptrs[] = {w0, wd, xhat, x};
  for (const void* p : ptrs)
    if (!is_device_pointer(p)) return set_error(SENSE_EINVAL, "fields must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  Grid g;
  g.n[0] = o->nx;
  g.n[1] = o->ny;
  g.n[2] = o->nz;
  g.stride[0] = 1;
  g.stride[1] = o->nx;
  g.stride[2] = (long long)o->nx * o->ny;
  g.total = (long long)o->nx * o->ny * o->nz;
  int dev = 0, sms = 1;
  SENSE_CUDA_TRY(cudaGetDevice(&dev));
  SENSE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::max<long long>(1, std::min<long long>((g.total + VB - 1) / VB, 8LL * sms));
  // workspace: r, p, q [n] complex; reduction partials, counter, scalars
  float2* ws = nullptr;
  double* red = nullptr;
  unsigned* counter = nullptr;
  if (cudaMalloc((void**)&ws, (size_t)g.total * 3 * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&red, (size_t)(grid * 2 + 8) * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&counter, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ws);
    cudaFree(red);
    cudaFree(counter);
    return set_error(SENSE_ENOMEM, "smoothing workspace");
  }
  float2 *r = ws, *p = ws + g.total, *q = ws + 2 * g.total;
  double* sc = red + grid * 2;   // [rr, bb, stop, step, beta, iters, -, -]
  float2* X = (float2*)x;
  const float2* XH = (const float2*)xhat;
  const float alpha = (float)o->alpha;
  const double tol2 = o->rel_tol * o->rel_tol;
  int rc = SENSE_OK;
  auto chk = [&](const char* what) {
    if (rc == SENSE_OK && cudaGetLastError() != cudaSuccess) rc = cuda_error(cudaGetLastError(), what);
  };
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(sc, 0, 8 * sizeof(double), st) != cudaSuccess ||
      (X != XH && cudaMemcpyAsync(X, XH, (size_t)g.total * 8, cudaMemcpyDeviceToDevice, st) !=
                      cudaSuccess))
    rc = cuda_error(cudaGetLastError(), "smoothing set-up");
  if (rc == SENSE_OK) {
    smooth_apply_kernel<<<grid, VB, 0, st>>>(g, o->order, alpha, w0, wd, X, q);
    chk("smooth apply");
    smooth_init_kernel<<<grid, VB, 0, st>>>(w0, XH, q, g.total, r, p, red, counter, sc, tol2);
    chk("smooth init");
  }
  for (int it = 0; it < o->max_iter && rc == SENSE_OK; ++it) {
    smooth_apply_kernel<<<grid, VB, 0, st>>>(g, o->order, alpha, w0, wd, p, q);
    smooth_pap_kernel<<<grid, VB, 0, st>>>(p, q, g.total, red, counter, sc);
    smooth_update_kernel<<<grid, VB, 0, st>>>(X, r, p, q, g.total, red, counter, sc, tol2);
    smooth_p_kernel<<<grid, VB, 0, st>>>(p, r, g.total, sc);
    chk("smooth iteration");
  }
  double h[6] = {0, 0, 0, 0, 0, 0};
  if (rc == SENSE_OK && (cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess))
    rc = cuda_error(cudaGetLastError(), "smoothing result");
  if (rc == SENSE_OK && info) {
    info->iters = (int32_t)h[5];
    info->rel_residual = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : 0.0;
  }
  cudaStreamSynchronize(st);
  cudaFree(ws);
  cudaFree(red);
  cudaFree(counter);
  return rc;
}
