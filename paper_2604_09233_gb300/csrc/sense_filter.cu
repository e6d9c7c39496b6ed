// k-space filter: rho <- IFFT(FFT(rho) o f) (the filtering that ends Alg. 1, Fig. 2).
//
// The filter keeps the Cartesian k-space points that lie inside the convex hull of the
// first-order field coefficients (the k-space coordinates of the samples): components far from
// every sample are the ill-conditioned ones. Mask construction is host geometry (2D: monotone
// chain hull, point-in-convex-polygon test). The transform follows the signal model's sign:
// on an n-point axis with positions r_x = (x - n/2) d and k-space points k_u = 2 pi (u - n/2) /
// (n d), the forward transform is F(u) = sum_x rho(x) e^{+i k_u r_x} (the noiseless sample a
// single-coil, uniform-sensitivity acquisition would record at k_u), the inverse
// rho(x) = (1/n) sum_u F(u) e^{-i k_u r_x}; with f = 1 the filter is the identity. Both are
// evaluated as direct sums along one axis at a time (any axis length; n <= 4096) with FP32
// twiddles from an FP64 table: at these sizes a few milliseconds at most, against tens of
// milliseconds of CG iterations.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sense_internal.cuh"

namespace sense {
namespace {

constexpr int MAX_N = 4096;
constexpr int DFT_THREADS = 256;

// One block per line along the transformed axis: the line (n complex) and the twiddles e^{i 2 pi
// m / n} (m = 0..n-1) in shared memory; output u = sum_x in(x) w^{sgn (u - n/2)(x - n/2)}.
// Element x of line l is at base + x * inner, base = (l / inner) * n * inner + l % inner.
// (in and out may be the same array: a block reads its whole line before writing it)
__global__ void dft_axis_kernel(const float2* in, float2* out, int n,
                                long long inner, long long lines, const float2* __restrict__ tw,
                                int sgn, float scale, const float* __restrict__ mask) {
  extern __shared__ float2 sh[];
  float2* line = sh;       // [n]
  float2* w = sh + n;      // [n]
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = tw[i];
  for (long long l = blockIdx.x; l < lines; l += gridDim.x) {
    const long long outer = l / inner, in_off = l % inner;
    const long long base = outer * (long long)n * inner + in_off;
    __syncthreads();
    for (int x = threadIdx.x; x < n; x += blockDim.x) line[x] = in[base + (long long)x * inner];
    __syncthreads();
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
      const int cu = u - n / 2;
      // exponent index e = (cu * (x - n/2)) mod n, advanced by cu mod n per x
      const int step = ((cu % n) + n) % n;
      int e = (int)((((long long)cu * (-(n / 2))) % n + n) % n);
      float2 acc = make_float2(0.f, 0.f);
      for (int x = 0; x < n; ++x, e = (e + step >= n) ? e + step - n : e + step) {
        float2 t = w[e];
        if (sgn < 0) t.y = -t.y;
        const float2 v = line[x];
        acc.x = fmaf(v.x, t.x, fmaf(-v.y, t.y, acc.x));
        acc.y = fmaf(v.x, t.y, fmaf(v.y, t.x, acc.y));
      }
      const long long o = base + (long long)u * inner;
      const float f = mask ? mask[o] * scale : scale;
      out[o] = make_float2(acc.x * f, acc.y * f);
    }
  }
}

// convex hull helpers (host)
struct Pt {
  double x, y;
};

double cross(const Pt& o, const Pt& a, const Pt& b) {
  return (a.x - o.x) * (b.y - o.y) - (a.y - o.y) * (b.x - o.x);
}

// counter-clockwise hull without collinear points (Andrew's monotone chain)
std::vector<Pt> convex_hull(std::vector<Pt> p) {
  std::sort(p.begin(), p.end(), [](const Pt& a, const Pt& b) {
    return a.x < b.x || (a.x == b.x && a.y < b.y);
  });
  p.erase(std::unique(p.begin(), p.end(),
                      [](const Pt& a, const Pt& b) { return a.x == b.x && a.y == b.y; }),
          p.end());
  if (p.size() < 3) return p;
  std::vector<Pt> h(2 * p.size());
  size_t k = 0;
  for (size_t i = 0; i < p.size(); ++i) {
    while (k >= 2 && cross(h[k - 2], h[k - 1], p[i]) <= 0) --k;
    h[k++] = p[i];
  }
  for (size_t i = p.size() - 1, t = k + 1; i > 0; --i) {
    while (k >= t && cross(h[k - 2], h[k - 1], p[i - 1]) <= 0) --k;
    h[k++] = p[i - 1];
  }
  h.resize(k - 1);
  return h;
}

// inside or on the boundary of a counter-clockwise convex polygon
bool inside(const std::vector<Pt>& h, const Pt& q, double eps) {
  if (h.size() < 3) return false;
  for (size_t i = 0; i < h.size(); ++i) {
    const Pt& a = h[i];
    const Pt& b = h[(i + 1) % h.size()];
    const double len = std::hypot(b.x - a.x, b.y - a.y);
    if (cross(a, b, q) < -eps * len) return false;
  }
  return true;
}

// Cartesian points (u, v) with k = (dkx (u - nx/2), dky (v - ny/2)) inside or on the convex
// CCW polygon h: per row, the polygon's interval on that row, the exact half-plane test only
// near its ends.
void raster_polygon(const std::vector<Pt>& h, int nx, int ny, double dkx, double dky, double eps,
                    float* mask) {
  if (h.size() < 3) return;
  for (int v = 0; v < ny; ++v) {
    const double y = dky * (v - ny / 2);
    double lo = INFINITY, hi = -INFINITY;
    for (size_t i = 0; i < h.size(); ++i) {
      const Pt& a = h[i];
      const Pt& b = h[(i + 1) % h.size()];
      if ((y < std::min(a.y, b.y) - eps) || (y > std::max(a.y, b.y) + eps)) continue;
      double xa, xb;
      if (std::fabs(b.y - a.y) <= eps) {
        xa = std::min(a.x, b.x);
        xb = std::max(a.x, b.x);
      } else {
        const double s = std::min(1.0, std::max(0.0, (y - a.y) / (b.y - a.y)));
        xa = xb = a.x + s * (b.x - a.x);
      }
      lo = std::min(lo, xa);
      hi = std::max(hi, xb);
    }
    if (!(lo <= hi)) continue;
    const int u0 = std::max(0, (int)std::floor(lo / dkx) + nx / 2 - 1);
    const int u1 = std::min(nx - 1, (int)std::ceil(hi / dkx) + nx / 2 + 1);
    for (int u = u0; u <= u1; ++u) {
      const double x = dkx * (u - nx / 2);
      const bool sure = x > lo + dkx && x < hi - dkx;
      if (sure || inside(h, {x, y}, eps)) mask[(size_t)v * nx + u] = 1.0f;
    }
  }
}

// Minkowski sum of two convex CCW polygons (each scaled): merge their edges by angle
std::vector<Pt> minkowski(const std::vector<Pt>& P, double sp, const std::vector<Pt>& Q,
                          double sq) {
  std::vector<Pt> out;
  if (P.empty() || Q.empty()) return out;
  if (P.size() < 3 || Q.size() < 3) {        // degenerate: all vertex sums
    for (const Pt& a : P)
      for (const Pt& b : Q) out.push_back({sp * a.x + sq * b.x, sp * a.y + sq * b.y});
    return convex_hull(out);
  }
  auto start = [](const std::vector<Pt>& H) {
    size_t k = 0;
    for (size_t i = 1; i < H.size(); ++i)
      if (H[i].y < H[k].y || (H[i].y == H[k].y && H[i].x < H[k].x)) k = i;
    return k;
  };
  const size_t i0 = start(P), j0 = start(Q), n = P.size(), m = Q.size();
  size_t i = 0, j = 0;
  while (i < n || j < m) {
    const Pt& a = P[(i0 + i) % n];
    const Pt& b = Q[(j0 + j) % m];
    out.push_back({sp * a.x + sq * b.x, sp * a.y + sq * b.y});
    const Pt& a1 = P[(i0 + i + 1) % n];
    const Pt& b1 = Q[(j0 + j + 1) % m];
    const Pt ea = {sp * (a1.x - a.x), sp * (a1.y - a.y)};
    const Pt eb = {sq * (b1.x - b.x), sq * (b1.y - b.y)};
    const double c = ea.x * eb.y - ea.y * eb.x;
    if (j >= m || (i < n && c > 0)) ++i;
    else if (i >= n || c < 0) ++j;
    else { ++i; ++j; }
  }
  return convex_hull(out);
}

}  // namespace
}  // namespace sense

using namespace sense;

extern "C" int sense_kspace_filter_mask3d(int32_t nx, int32_t ny, int32_t nz, double dx, double dy,
                                          double dz, const double* kx, const double* ky,
                                          const double* kz, int64_t K, float* mask) {
  if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0.0) || !(dy > 0.0) || !(dz > 0.0) || !kx || !ky ||
      !kz || K < 4 || !mask)
    return set_error(SENSE_EINVAL, "sizes, spacings, k-space coordinates (K >= 4) and mask");
  // group the samples by kz plane (stacks of planar trajectories)
  std::vector<std::pair<double, std::vector<Pt>>> planes;
  {
    std::vector<int64_t> order((size_t)K);
    for (int64_t i = 0; i < K; ++i) {
      if (!std::isfinite(kx[i]) || !std::isfinite(ky[i]) || !std::isfinite(kz[i]))
        return set_error(SENSE_ENONFINITE, "non-finite k-space coordinate");
      order[i] = i;
    }
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return kz[a] < kz[b]; });
    for (int64_t i : order) {
      if (planes.empty() || kz[i] != planes.back().first) {
        if (planes.size() >= 4096)
          return set_error(SENSE_EUNSUPPORTED, "3D mask: more than 4096 distinct kz planes");
        planes.push_back({kz[i], {}});
      }
      planes.back().second.push_back({kx[i], ky[i]});
    }
  }
  for (auto& pl : planes) pl.second = convex_hull(pl.second);
  const double dkx = 2.0 * M_PI / (nx * dx), dky = 2.0 * M_PI / (ny * dy),
               dkz = 2.0 * M_PI / (nz * dz);
  const double eps = 1e-9 * std::max(dkx, dky);
  const double ztol = 1e-9 * dkz;
  std::fill(mask, mask + (size_t)nx * ny * nz, 0.0f);
  // cross-section of the hull at height c: the convex hull of (1 - t) H_i + t H_j over all
  // plane pairs z_i <= c <= z_j (t = (c - z_i) / (z_j - z_i)), and of H_i for z_i = c
  for (int w = 0; w < nz; ++w) {
    const double c = dkz * (w - nz / 2);
    std::vector<Pt> pts;
    for (size_t i = 0; i < planes.size(); ++i) {
      const double zi = planes[i].first;
      if (std::fabs(zi - c) <= ztol)
        pts.insert(pts.end(), planes[i].second.begin(), planes[i].second.end());
      if (zi > c) continue;
      for (size_t j = i + 1; j < planes.size(); ++j) {
        const double zj = planes[j].first;
        if (zj < c || zj - zi <= ztol) continue;
        const double tt = (c - zi) / (zj - zi);
        const std::vector<Pt> s = minkowski(planes[i].second, 1.0 - tt, planes[j].second, tt);
        pts.insert(pts.end(), s.begin(), s.end());
      }
    }
    if (pts.size() < 3) continue;
    raster_polygon(convex_hull(pts), nx, ny, dkx, dky, eps, mask + (size_t)w * nx * ny);
  }
  return SENSE_OK;
}

extern "C" int sense_kspace_filter_mask(int32_t nx, int32_t ny, double dx, double dy,
                                        const double* kx, const double* ky, int64_t K,
                                        float* mask) {
  if (nx < 1 || ny < 1 || !(dx > 0.0) || !(dy > 0.0) || !kx || !ky || K < 3 || !mask)
    return set_error(SENSE_EINVAL, "sizes, spacings, k-space coordinates (K >= 3) and mask");
  std::vector<Pt> pts((size_t)K);
  for (int64_t i = 0; i < K; ++i) {
    if (!std::isfinite(kx[i]) || !std::isfinite(ky[i]))
      return set_error(SENSE_ENONFINITE, "non-finite k-space coordinate");
    pts[i] = {kx[i], ky[i]};
  }
  const std::vector<Pt> h = convex_hull(pts);
  // boundary tolerance: a tiny fraction of the grid's k-space spacing
  const double eps = 1e-9 * 2.0 * M_PI / std::max(nx * dx, ny * dy);
  const double dkx = 2.0 * M_PI / (nx * dx), dky = 2.0 * M_PI / (ny * dy);
  std::fill(mask, mask + (size_t)nx * ny, 0.0f);
  raster_polygon(h, nx, ny, dkx, dky, eps, mask);
  return SENSE_OK;
}

extern "C" int sense_kspace_filter(int32_t nx, int32_t ny, int32_t nz, const float* mask,
                                   float* image, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || nx > MAX_N || ny > MAX_N || nz > MAX_N || !mask || !image)
    return set_error(SENSE_EINVAL, "axis lengths 1..4096, mask and image required");
  if (!is_device_pointer(mask) || !is_device_pointer(image))
    return set_error(SENSE_EINVAL, "mask and image must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  const int n_axis[3] = {nx, ny, nz};
  const long long inner_of[3] = {1, nx, (long long)nx * ny};
  const long long total = (long long)nx * ny * nz;
  float2* img = (float2*)image;
  // twiddle tables (FP64 -> FP32) for each distinct axis length
  std::vector<float2*> tws(3, nullptr);
  int rc = SENSE_OK;
  for (int a = 0; a < 3 && rc == SENSE_OK; ++a) {
    const int n = n_axis[a];
    if (n == 1) continue;
    std::vector<float2> h((size_t)n);
    for (int m = 0; m < n; ++m)
      h[m] = make_float2((float)std::cos(2.0 * M_PI * m / n), (float)std::sin(2.0 * M_PI * m / n));
    if (cudaMalloc((void**)&tws[a], (size_t)n * 8) != cudaSuccess) {
      cudaGetLastError();
      rc = set_error(SENSE_ENOMEM, "twiddles");
      break;
    }
    if (cudaMemcpyAsync(tws[a], h.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      rc = cuda_error(cudaGetLastError(), "twiddles");
    // pageable source: wait before h goes out of scope
    if (rc == SENSE_OK && cudaStreamSynchronize(st) != cudaSuccess)
      rc = cuda_error(cudaGetLastError(), "twiddles");
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // forward transforms along every axis, the mask applied with the last one, then the inverse
  // transforms (scaled by 1/n each)
  int last = -1;
  for (int a = 0; a < 3; ++a)
    if (n_axis[a] > 1) last = a;
  for (int pass = 0; pass < 2 && rc == SENSE_OK; ++pass) {
    for (int a = 0; a < 3 && rc == SENSE_OK; ++a) {
      const int n = n_axis[a];
      if (n == 1) continue;
      const long long lines = total / n;
      const int grid = (int)std::min<long long>(lines, 64LL * sms);
      const size_t shm = (size_t)2 * n * sizeof(float2);
      const bool fwd = pass == 0;
      if (shm > 48 * 1024 &&
          cudaFuncSetAttribute(dft_axis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)shm) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "dft shared memory");
        break;
      }
      dft_axis_kernel<<<grid, DFT_THREADS, shm, st>>>(
          img, img, n, inner_of[a], lines, tws[a], fwd ? 1 : -1, fwd ? 1.0f : 1.0f / n,
          (fwd && a == last) ? mask : nullptr);
      if (cudaGetLastError() != cudaSuccess) rc = cuda_error(cudaGetLastError(), "dft launch");
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == SENSE_OK)
    rc = cuda_error(cudaGetLastError(), "filter");
  for (auto* p : tws) cudaFree(p);
  return rc;
}
