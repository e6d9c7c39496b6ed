// Plan creation: validation, voxel ordering, phase anchors (FP64 on the device), uploads.
//
// Phase evaluation used by every kernel (Eq. 4, phi = K R, here in turns = phi / 2pi):
//   with a sample block b(k) of TILE consecutive samples and a voxel block v(l) of TILE
//   spatially compact voxels, and block centres Kc(b) (a row of K) and Rc(v) (a column
//   of R),
//     phi(k,l) = Kc(b).R(l)  +  (K(k)-Kc(b)).Rc(v)  +  (K(k)-Kc(b)).(R(l)-Rc(v))
//              =   A(b,l)    +       B(v,k)         +          D(k,l)
//   A and B are computed once per plan in FP64 and stored reduced mod 1 as float; only
//   the local bilinear term D, whose size is bounded by the extent of one block in k and
//   in r, is evaluated per pair in FP32. Rows of K R that are constant inside every block
//   (or zero) contribute nothing to D and are dropped from it.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "sense_tc.cuh"

namespace sense {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  g_last_error = buf;
  return SENSE_ECUDA;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// --------------------------------------------------------------------------------------
// Voxel order: recursive median splits along the basis row with the largest phase
// spread (max_k |K(k,p)| times the range of R(p,.) in the current set), so that every
// block of TILE voxels is compact in the coordinates that drive the phase. Left halves
// always hold a multiple of TILE voxels, so only the last block can be partial.
// --------------------------------------------------------------------------------------
static void kd_order(std::vector<int32_t>& idx, int64_t lo, int64_t hi, const double* R,
                     int64_t L, int P1, const std::vector<double>& w) {
  const int64_t n = hi - lo;
  if (n <= TILE) return;
  int best = -1;
  double best_spread = 0.0;
  for (int p = 0; p < P1; ++p) {
    if (w[p] == 0.0) continue;
    double mn = INFINITY, mx = -INFINITY;
    for (int64_t i = lo; i < hi; ++i) {
      const double v = R[(int64_t)p * L + idx[i]];
      mn = std::min(mn, v);
      mx = std::max(mx, v);
    }
    const double s = w[p] * (mx - mn);
    if (s > best_spread) {
      best_spread = s;
      best = p;
    }
  }
  int64_t nl = ((n / 2 + TILE - 1) / TILE) * TILE;
  if (nl >= n) nl = n - 1;  // cannot happen for n > TILE, kept for safety
  if (best >= 0) {
    const double* row = R + (int64_t)best * L;
    std::nth_element(idx.begin() + lo, idx.begin() + lo + nl, idx.begin() + hi,
                     [row](int32_t a, int32_t b) {
                       return row[a] < row[b] || (row[a] == row[b] && a < b);
                     });
  }
  kd_order(idx, lo, lo + nl, R, L, P1, w);
  kd_order(idx, lo + nl, hi, R, L, P1, w);
}

// --------------------------------------------------------------------------------------
// FP64 anchor kernels.
// --------------------------------------------------------------------------------------
__device__ __forceinline__ float frac_turns(double v) { return (float)(v - rint(v)); }
__device__ __forceinline__ float frac_radians(double v) {
  return (float)(6.283185307179586 * (v - rint(v)));
}

// A(b, l) = frac(Kc(b) . R(l)), in turns (A) and in radians (AR)
__global__ void anchors_A_kernel(const double* __restrict__ Kc, const double* __restrict__ Rd,
                                 float* __restrict__ A, float* __restrict__ AR, int P1,
                                 int64_t Lp) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = blockIdx.y;
  if (l >= Lp) return;
  double acc = 0.0;
  for (int p = 0; p < P1; ++p) acc = fma(Kc[(int64_t)sb * P1 + p], Rd[(int64_t)p * Lp + l], acc);
  A[(int64_t)sb * Lp + l] = frac_turns(acc);
  AR[(int64_t)sb * Lp + l] = frac_radians(acc);
}

// B(v, k) = frac((K(k) - Kc(b(k))) . Rc(v)), in turns (B) and in radians (BR)
__global__ void anchors_B_kernel(const double* __restrict__ Kd, const double* __restrict__ Kc,
                                 const double* __restrict__ Rc, float* __restrict__ B,
                                 float* __restrict__ BR, int P1, int64_t Kp) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int vb = blockIdx.y;
  if (k >= Kp) return;
  const int64_t sb = k / TILE;
  double acc = 0.0;
  for (int p = 0; p < P1; ++p)
    acc = fma(Kd[k * P1 + p] - Kc[sb * P1 + p], Rc[(int64_t)vb * P1 + p], acc);
  B[(int64_t)vb * Kp + k] = frac_turns(acc);
  BR[(int64_t)vb * Kp + k] = frac_radians(acc);
}

// ---------------------------------------------------------------------------------------
// Operand images of the local bilinear phase for the tensor-core phase kernel. With the
// kept rows q, the phase in radians is D(k,l) = 2 pi sum_q dK(k,q) dR(l,q). Per row q a
// power of two u_q balances the two factors, and one more power of two S scales both so
// that the largest entry is below 2^12: kv = dK u_q S, rv = dR 2 pi / u_q S, D = (kv . rv) /
// S^2. Each value is split into FP16 hi = fp16(v) and lo = fp16(v - hi). An image row holds
// 64 FP16 (128 bytes) in the 128B-swizzled K-major layout of the MMA operands (16-byte chunk
// c of row n at n * 128 + (c ^ (n & 7)) * 16): FP16 h = part * 16 nkp + q of row n, part 0 =
// hi, 1 = lo. The row-side image of a block lists its 128 entities in order. The streamed-side
// image lists each 64-wide stage's entities in the order the generator warps read the phases
// back from tensor memory: MMA row n < 32 is element 16 (n / 8) + n % 8, n >= 32 is element
// 16 ((n - 32) / 8) + 8 + (n - 32) % 8; for nkp = 1 both stages share 64 rows (stage st in
// FP16 32 st + h), for nkp = 2 each stage has its own 64 rows (8 KB).
// ---------------------------------------------------------------------------------------
static inline size_t ph_off(int64_t n, int h) {
  return (size_t)n * 128 + (size_t)((((h >> 3) ^ (int)(n & 7))) << 4) + (size_t)(h & 7) * 2;
}

// hi / lo FP16 parts of v at FP16 positions h (hi) and h + 16 nkp (lo) of image row n
static void ph_put(uint8_t* img, int64_t n, int h, int nkp, double v) {
  const __half hi = __double2half(v);
  const __half lo = __double2half(v - (double)__half2float(hi));
  std::memcpy(img + ph_off(n, h), &hi, 2);
  std::memcpy(img + ph_off(n, h + 16 * nkp), &lo, 2);
}

// MMA row of streamed element j (0..63) of a stage
static inline int ph_perm_row(int j) {
  const int g = j >> 4, e = j & 15;
  return e < 8 ? 8 * g + e : 32 + 8 * g + (e - 8);
}

template <typename T>
static int dalloc(T** p, size_t n);

static int build_phase_images(sense_plan_s* P, const std::vector<double>& Kt,
                              const std::vector<double>& Kc, const std::vector<double>& Rd,
                              const std::vector<double>& Rc, cudaStream_t st) {
  const int P1 = P->P1, r = P->r;
  const int64_t Kp = P->Kp, Lp = P->Lp;
  const int nkp = P->RT <= 16 ? 1 : 2;
  P->nkp = nkp;
  const int colb = tc::tcp_col_bytes(nkp);
  std::vector<double> mk(std::max(1, r), 0.0), mr(std::max(1, r), 0.0);
  auto dk = [&](int64_t k, int q) {
    return Kt[(size_t)k * P1 + P->rows[q]] - Kc[(size_t)(k / TILE) * P1 + P->rows[q]];
  };
  auto dr = [&](int64_t i, int q) {
    return Rd[(size_t)P->rows[q] * Lp + i] - Rc[(size_t)(i / TILE) * P1 + P->rows[q]];
  };
  for (int q = 0; q < r; ++q) {
    for (int64_t k = 0; k < Kp; ++k) mk[q] = std::max(mk[q], std::fabs(dk(k, q)));
    for (int64_t i = 0; i < Lp; ++i) mr[q] = std::max(mr[q], std::fabs(dr(i, q)));
  }
  const double two_pi = 2.0 * M_PI;
  std::vector<double> u(std::max(1, r), 1.0);
  double vmax = 0.0;
  for (int q = 0; q < r; ++q) {
    if (mk[q] > 0.0 && mr[q] > 0.0)
      u[q] = std::ldexp(1.0, (int)std::lround(0.5 * std::log2(two_pi * mr[q] / mk[q])));
    vmax = std::max(vmax, std::max(mk[q] * u[q], two_pi * mr[q] / u[q]));
  }
  const double S = vmax > 0.0 ? std::ldexp(1.0, (int)std::floor(std::log2(4096.0 / vmax))) : 1.0;
  P->ph_unscale = (float)(1.0 / (S * S));
  std::vector<uint8_t> kr((size_t)P->nsb * tc::TCP_ROW_BYTES, 0), kc((size_t)P->nsb * colb, 0);
  std::vector<uint8_t> rr((size_t)P->nvb * tc::TCP_ROW_BYTES, 0), rc((size_t)P->nvb * colb, 0);
  for (int64_t k = 0; k < Kp; ++k) {
    const int64_t b = k / TILE, j = k % TILE;
    const int st = (int)(j >> 6), n = ph_perm_row((int)(j & 63));
    for (int q = 0; q < r; ++q) {
      const double v = dk(k, q) * u[q] * S;
      ph_put(kr.data() + (size_t)b * tc::TCP_ROW_BYTES, j, q, nkp, v);
      if (nkp == 1)
        ph_put(kc.data() + (size_t)b * colb, n, 32 * st + q, 1, v);
      else
        ph_put(kc.data() + (size_t)b * colb + (size_t)st * 8192, n, q, 2, v);
    }
  }
  for (int64_t i = 0; i < Lp; ++i) {
    const int64_t b = i / TILE, j = i % TILE;
    const int st = (int)(j >> 6), n = ph_perm_row((int)(j & 63));
    for (int q = 0; q < r; ++q) {
      const double v = dr(i, q) * (two_pi / u[q]) * S;
      ph_put(rr.data() + (size_t)b * tc::TCP_ROW_BYTES, j, q, nkp, v);
      if (nkp == 1)
        ph_put(rc.data() + (size_t)b * colb, n, 32 * st + q, 1, v);
      else
        ph_put(rc.data() + (size_t)b * colb + (size_t)st * 8192, n, q, 2, v);
    }
  }
  int rc_ = SENSE_OK;
  if ((rc_ = dalloc(&P->phK_row, kr.size())) != SENSE_OK) return rc_;
  if ((rc_ = dalloc(&P->phK_col, kc.size())) != SENSE_OK) return rc_;
  if ((rc_ = dalloc(&P->phR_row, rr.size())) != SENSE_OK) return rc_;
  if ((rc_ = dalloc(&P->phR_col, rc.size())) != SENSE_OK) return rc_;
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->phK_row, kr.data(), kr.size(), cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->phK_col, kc.data(), kc.size(), cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->phR_row, rr.data(), rr.size(), cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->phR_col, rc.data(), rc.size(), cudaMemcpyHostToDevice, st));
  // the host vectors die at return
  SENSE_CUDA_TRY(cudaStreamSynchronize(st));
  return SENSE_OK;
}

__global__ void deltas_kernel(const double* __restrict__ Kd, const double* __restrict__ Kc,
                              const double* __restrict__ Rd, const double* __restrict__ Rc,
                              const int* __restrict__ rows, int r, int RP, int P1, int64_t Kp,
                              int64_t Lp, float* __restrict__ dK, float* __restrict__ dR,
                              int RT, float* __restrict__ dKt, float* __restrict__ dRt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int RM = RP > RT ? RP : RT;
  if (i < Kp) {
    const int64_t sb = i / TILE, w = i % TILE;
    for (int q = 0; q < RM; ++q) {
      const float v = q < r ? (float)(Kd[i * P1 + rows[q]] - Kc[sb * P1 + rows[q]]) : 0.0f;
      if (q < RP) dK[i * RP + q] = v;
      if (q < RT) dKt[(sb * RT + q) * TILE + w] = v;
    }
  }
  if (i < Lp) {
    const int64_t vb = i / TILE, w = i % TILE;
    for (int q = 0; q < RM; ++q) {
      const float v =
          q < r ? (float)(Rd[(int64_t)rows[q] * Lp + i] - Rc[vb * P1 + rows[q]]) : 0.0f;
      if (q < RP) dR[i * RP + q] = v;
      if (q < RT) dRt[(vb * RT + q) * TILE + w] = v;
    }
  }
}

template <typename T>
static int dalloc(T** p, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(SENSE_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  return SENSE_OK;
}

#define SENSE_TRY(expr)          \
  do {                           \
    int _rc = (expr);            \
    if (_rc != SENSE_OK) return _rc; \
  } while (0)

static void free_geometry(sense_plan_s* P) {
  cudaFree(P->dKd); cudaFree(P->dRd); cudaFree(P->dKc); cudaFree(P->dRc);
  cudaFree(P->drows); cudaFree(P->dK); cudaFree(P->dR); cudaFree(P->Aanc); cudaFree(P->Banc);
  cudaFree(P->dKt); cudaFree(P->dRt);
  cudaFree(P->AancR); cudaFree(P->BancR);
  cudaFree(P->phK_row); cudaFree(P->phK_col); cudaFree(P->phR_row); cudaFree(P->phR_col);
  P->AancR = P->BancR = nullptr;
  P->phK_row = P->phK_col = P->phR_row = P->phR_col = nullptr;
  P->dKt = P->dRt = nullptr;
  P->dKd = P->dRd = P->dKc = P->dRc = nullptr;
  P->drows = nullptr;
  P->dK = P->dR = P->Aanc = P->Banc = nullptr;
}

// Build (or rebuild, after the B0 row changed) centres, kept rows, anchors and deltas.
static int build_geometry(sense_plan_s* P, cudaStream_t st) {
  const int64_t L = P->L, K = P->K, Lp = P->Lp, Kp = P->Kp;
  const int P1 = P->P1;
  const double inv2pi = 1.0 / (2.0 * M_PI);

  // K in turns, padded rows filled later with the block centre
  std::vector<double> Kt((size_t)Kp * P1);
  for (int64_t k = 0; k < K; ++k)
    for (int p = 0; p < P1; ++p) Kt[k * P1 + p] = P->Kh[k * P1 + p] * inv2pi;
  std::vector<double> Kc((size_t)P->nsb * P1);
  for (int sb = 0; sb < P->nsb; ++sb) {
    const int64_t k0 = (int64_t)sb * TILE, k1 = std::min<int64_t>(K, k0 + TILE);
    for (int p = 0; p < P1; ++p) {
      double mn = INFINITY, mx = -INFINITY;
      for (int64_t k = k0; k < k1; ++k) {
        mn = std::min(mn, Kt[k * P1 + p]);
        mx = std::max(mx, Kt[k * P1 + p]);
      }
      Kc[(size_t)sb * P1 + p] = 0.5 * (mn + mx);
    }
    for (int64_t k = k1; k < k0 + TILE; ++k)
      for (int p = 0; p < P1; ++p) Kt[k * P1 + p] = Kc[(size_t)sb * P1 + p];
  }
  // R in plan order
  std::vector<double> Rd((size_t)P1 * Lp);
  std::vector<double> Rc((size_t)P->nvb * P1);
  for (int vb = 0; vb < P->nvb; ++vb) {
    const int64_t l0 = (int64_t)vb * TILE;
    for (int p = 0; p < P1; ++p) {
      double mn = INFINITY, mx = -INFINITY;
      for (int64_t i = l0; i < l0 + TILE; ++i) {
        const int32_t u = P->perm[i];
        if (u < 0) continue;
        const double v = P->Rh[(int64_t)p * L + u];
        mn = std::min(mn, v);
        mx = std::max(mx, v);
      }
      const double c = 0.5 * (mn + mx);
      Rc[(size_t)vb * P1 + p] = c;
      for (int64_t i = l0; i < l0 + TILE; ++i) {
        const int32_t u = P->perm[i];
        Rd[(size_t)p * Lp + i] = u < 0 ? c : P->Rh[(int64_t)p * L + u];
      }
    }
  }
  // rows that vary inside blocks in both factors
  std::vector<int> rows;
  for (int p = 0; p < P1; ++p) {
    bool k_varies = false, r_varies = false;
    for (int64_t k = 0; k < Kp && !k_varies; ++k)
      k_varies = Kt[k * P1 + p] != Kc[(size_t)(k / TILE) * P1 + p];
    for (int64_t i = 0; i < Lp && !r_varies; ++i)
      r_varies = Rd[(size_t)p * Lp + i] != Rc[(size_t)(i / TILE) * P1 + p];
    if (k_varies && r_varies) rows.push_back(p);
  }
  if ((int)rows.size() > MAX_RP)
    return set_error(SENSE_EUNSUPPORTED, "more than 20 basis rows vary inside a block");
  P->rows = rows;
  P->r = (int)rows.size();
  P->RP = std::max(4, (P->r + 3) / 4 * 4);
  {
    static const int rt_sizes[] = {4, 6, 8, 10, 12, 16, 20};
    P->RT = 20;
    for (int v : rt_sizes)
      if (v >= std::max(P->r, P->min_rt)) {
        P->RT = v;
        break;
      }
  }

  free_geometry(P);
  ++P->geom_version;
  SENSE_TRY(dalloc(&P->dKd, (size_t)Kp * P1));
  SENSE_TRY(dalloc(&P->dRd, (size_t)P1 * Lp));
  SENSE_TRY(dalloc(&P->dKc, (size_t)P->nsb * P1));
  SENSE_TRY(dalloc(&P->dRc, (size_t)P->nvb * P1));
  SENSE_TRY(dalloc(&P->drows, (size_t)std::max(1, P->r)));
  SENSE_TRY(dalloc(&P->dK, (size_t)Kp * P->RP));
  SENSE_TRY(dalloc(&P->dR, (size_t)Lp * P->RP));
  SENSE_TRY(dalloc(&P->dKt, (size_t)Kp * P->RT));
  SENSE_TRY(dalloc(&P->dRt, (size_t)Lp * P->RT));
  SENSE_TRY(dalloc(&P->Aanc, (size_t)P->nsb * Lp));
  SENSE_TRY(dalloc(&P->Banc, (size_t)P->nvb * Kp));
  SENSE_TRY(dalloc(&P->AancR, (size_t)P->nsb * Lp));
  SENSE_TRY(dalloc(&P->BancR, (size_t)P->nvb * Kp));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->dKd, Kt.data(), Kt.size() * 8, cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->dRd, Rd.data(), Rd.size() * 8, cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->dKc, Kc.data(), Kc.size() * 8, cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->dRc, Rc.data(), Rc.size() * 8, cudaMemcpyHostToDevice, st));
  if (P->r > 0)
    SENSE_CUDA_TRY(cudaMemcpyAsync(P->drows, rows.data(), rows.size() * sizeof(int),
                                   cudaMemcpyHostToDevice, st));
  anchors_A_kernel<<<dim3((unsigned)((Lp + 255) / 256), P->nsb), 256, 0, st>>>(
      P->dKc, P->dRd, P->Aanc, P->AancR, P1, Lp);
  SENSE_CUDA_TRY(cudaGetLastError());
  anchors_B_kernel<<<dim3((unsigned)((Kp + 255) / 256), P->nvb), 256, 0, st>>>(
      P->dKd, P->dKc, P->dRc, P->Banc, P->BancR, P1, Kp);
  SENSE_CUDA_TRY(cudaGetLastError());
  const int64_t nmax = std::max(Kp, Lp);
  deltas_kernel<<<(unsigned)((nmax + 255) / 256), 256, 0, st>>>(
      P->dKd, P->dKc, P->dRd, P->dRc, P->drows, P->r, P->RP, P1, Kp, Lp, P->dK, P->dR, P->RT,
      P->dKt, P->dRt);
  SENSE_CUDA_TRY(cudaGetLastError());
  // the host vectors above die at return: make the copies complete first
  SENSE_CUDA_TRY(cudaStreamSynchronize(st));
  return build_phase_images(P, Kt, Kc, Rd, Rc, st);
}

static int upload_sens(sense_plan_s* P, cudaStream_t st) {
  const int64_t Lp = P->Lp;
  const int C = P->C, Cp = P->Cp;
  std::vector<float> Sp((size_t)Lp * Cp * 2, 0.0f), jp((size_t)Lp, 1.0f);
  for (int64_t i = 0; i < Lp; ++i) {
    const int32_t u = P->perm[i];
    if (u < 0) continue;
    const float jj = P->jh[u];
    jp[i] = jj;
    for (int c = 0; c < C; ++c) {
      Sp[((size_t)i * Cp + c) * 2 + 0] = P->Sh[((size_t)u * C + c) * 2 + 0] * jj;
      Sp[((size_t)i * Cp + c) * 2 + 1] = P->Sh[((size_t)u * C + c) * 2 + 1] * jj;
    }
  }
  std::vector<float> tk((size_t)P->Kp, 0.0f);
  for (int64_t k = 0; k < P->K; ++k) tk[k] = (float)P->Kh[k * P->P1 + 0];
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->S, Sp.data(), Sp.size() * 4, cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->jv, jp.data(), jp.size() * 4, cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->tk, tk.data(), tk.size() * 4, cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(P->dperm, P->perm.data(), P->perm.size() * 4,
                                 cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaStreamSynchronize(st));
  return SENSE_OK;
}

static void choose_split(int64_t outer, int64_t inner, int target, int* nsplit, int* per) {
  int64_t ns = (target + outer - 1) / outer;
  ns = std::max<int64_t>(1, std::min<int64_t>(ns, inner));
  int64_t pr = (inner + ns - 1) / ns;
  *per = (int)pr;
  *nsplit = (int)((inner + pr - 1) / pr);
}

static int alloc_workspace(sense_plan_s* P) {
  const int64_t Lp = P->Lp, Kp = P->Kp;
  const int target = P->num_sms * 16;
  choose_split(P->nsb, P->nvb, target, &P->nsplit_e, &P->vb_per_split);
  choose_split(P->nvb, P->nsb, target, &P->nsplit_a, &P->sb_per_split);
  SENSE_TRY(dalloc(&P->Ypart, (size_t)P->nsplit_e * Kp * P->Cp));
  SENSE_TRY(dalloc(&P->Y, (size_t)Kp * P->Cp));
  SENSE_TRY(dalloc(&P->Ydata, (size_t)Kp * P->Cp));
  SENSE_TRY(dalloc(&P->Xpart, (size_t)P->nsplit_a * Lp));
  SENSE_TRY(dalloc(&P->vx, Lp));
  SENSE_TRY(dalloc(&P->vr, Lp));
  SENSE_TRY(dalloc(&P->vp, Lp));
  SENSE_TRY(dalloc(&P->vq, Lp));
  SENSE_TRY(dalloc(&P->vb, Lp));
  SENSE_TRY(dalloc(&P->vm, Lp));
  SENSE_TRY(dalloc(&P->scal, SC_COUNT));
  // partials of the vector reductions: up to 8 blocks per SM, 4 sums per block
  P->red_blocks = 8 * P->num_sms;
  SENSE_TRY(dalloc(&P->red, (size_t)P->red_blocks * 4));
  SENSE_TRY(dalloc(&P->counter, 4));
  SENSE_CUDA_TRY(cudaMemset(P->counter, 0, 4 * sizeof(unsigned)));
  SENSE_TRY(dalloc(&P->stage_s, (size_t)P->K * P->C));
  SENSE_TRY(dalloc(&P->stage_m, (size_t)P->L));
  SENSE_TRY(tc_setup(P));
  return SENSE_OK;
}

static void plan_free_all(sense_plan_s* P) {
  if (!P) return;
  free_geometry(P);
  cudaFree(P->dperm); cudaFree(P->S); cudaFree(P->jv); cudaFree(P->tk);
  cudaFree(P->Ypart); cudaFree(P->Y); cudaFree(P->Ydata); cudaFree(P->Xpart);
  cudaFree(P->vx); cudaFree(P->vr); cudaFree(P->vp); cudaFree(P->vq); cudaFree(P->vb);
  cudaFree(P->vm); cudaFree(P->scal); cudaFree(P->hist); cudaFree(P->red);
  cudaFree(P->counter); cudaFree(P->stage_s); cudaFree(P->stage_m);
  tc_free(P);
  grad_free(P);
  prof_free(P);
  delete P;
}

}  // namespace sense

using namespace sense;

extern "C" int sense_plan_create(const sense_problem* prob, sense_plan* out) {
  return plan_create(prob, 0, 0, out);
}

namespace sense {

int plan_create(const sense_problem* prob, int min_cp, int min_rt, sense_plan_s** out) {
  NvtxRange nvtx("sense plan create");
  if (!prob || !out) return set_error(SENSE_EINVAL, "null problem or output pointer");
  *out = nullptr;
  if (prob->L < 1 || prob->K < 1 || prob->C < 1 || prob->P1 < 1)
    return set_error(SENSE_EINVAL, "L, K, C and P1 must be >= 1");
  if (!prob->Kmat || !prob->Rmat || !prob->S)
    return set_error(SENSE_EINVAL, "Kmat, Rmat and S are required");
  if (prob->C > MAX_CP) return set_error(SENSE_EUNSUPPORTED, "at most 64 coils");
  if (prob->L > (int64_t)1 << 30 || prob->K > (int64_t)1 << 30)
    return set_error(SENSE_EUNSUPPORTED, "L and K must be below 2^30");
  const int64_t L = prob->L, K = prob->K;
  const int C = prob->C, P1 = prob->P1;
  for (int64_t i = 0; i < K * P1; ++i)
    if (!std::isfinite(prob->Kmat[i])) return set_error(SENSE_ENONFINITE, "non-finite Kmat");
  for (int64_t i = 0; i < L * P1; ++i)
    if (!std::isfinite(prob->Rmat[i])) return set_error(SENSE_ENONFINITE, "non-finite Rmat");
  for (int64_t i = 0; i < L * C * 2; ++i)
    if (!std::isfinite(prob->S[i])) return set_error(SENSE_ENONFINITE, "non-finite S");
  if (prob->j)
    for (int64_t i = 0; i < L; ++i)
      if (!std::isfinite(prob->j[i])) return set_error(SENSE_ENONFINITE, "non-finite j");

  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return set_error(SENSE_ENODEVICE, "no CUDA device");
  }
  SENSE_CUDA_TRY(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  SENSE_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  if (prop.major != 10 || prop.minor != 3)
    return set_error(SENSE_ENODEVICE, "libsense is built for sm_103a (GB300) only");

  sense_plan_s* P = new sense_plan_s();
  P->device = dev;
  P->num_sms = prop.multiProcessorCount;
  {
    int khz = 0;
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess) {
      cudaGetLastError();
      khz = 0;
    }
    P->clock_khz = khz > 0 ? khz : 2100000;
  }
  P->L = L; P->K = K; P->C = C; P->P1 = P1;
  P->Lp = (L + TILE - 1) / TILE * TILE;
  P->Kp = (K + TILE - 1) / TILE * TILE;
  P->Cp = C <= 8 ? 8 : C <= 16 ? 16 : C <= 32 ? 32 : 64;
  P->Cp = std::max(P->Cp, min_cp);
  P->min_rt = min_rt;
  P->nsb = (int)(P->Kp / TILE);
  P->nvb = (int)(P->Lp / TILE);
  P->Kh.assign(prob->Kmat, prob->Kmat + K * P1);
  P->Rh.assign(prob->Rmat, prob->Rmat + L * P1);
  P->Sh.assign(prob->S, prob->S + L * C * 2);
  P->has_j = prob->j != nullptr;
  P->jh.assign((size_t)L, 1.0f);
  if (prob->j) std::copy(prob->j, prob->j + L, P->jh.begin());

  // voxel order
  std::vector<double> w(P1, 0.0);
  for (int64_t k = 0; k < K; ++k)
    for (int p = 0; p < P1; ++p) w[p] = std::max(w[p], std::fabs(P->Kh[k * P1 + p]));
  std::vector<int32_t> idx(L);
  std::iota(idx.begin(), idx.end(), 0);
  kd_order(idx, 0, L, P->Rh.data(), L, P1, w);
  P->perm.assign((size_t)P->Lp, -1);
  std::copy(idx.begin(), idx.end(), P->perm.begin());

  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    delete P;
    return cuda_error(cudaGetLastError(), "cudaStreamCreate");
  }
  int rc = SENSE_OK;
  do {
    if ((rc = dalloc(&P->dperm, (size_t)P->Lp)) != SENSE_OK) break;
    if ((rc = dalloc(&P->S, (size_t)P->Lp * P->Cp)) != SENSE_OK) break;
    if ((rc = dalloc(&P->jv, (size_t)P->Lp)) != SENSE_OK) break;
    if ((rc = dalloc(&P->tk, (size_t)P->Kp)) != SENSE_OK) break;
    if ((rc = build_geometry(P, st)) != SENSE_OK) break;
    if ((rc = upload_sens(P, st)) != SENSE_OK) break;
    if ((rc = alloc_workspace(P)) != SENSE_OK) break;
  } while (0);
  cudaStreamDestroy(st);
  if (rc != SENSE_OK) {
    plan_free_all(P);
    return rc;
  }
  *out = P;
  return SENSE_OK;
}

}  // namespace sense

extern "C" int sense_plan_destroy(sense_plan plan) {
  if (!plan) return SENSE_OK;
  cudaDeviceSynchronize();
  plan_free_all(plan);
  return SENSE_OK;
}

extern "C" int sense_plan_set_b0(sense_plan P, const double* omega, void* stream) {
  if (!P || !omega) return set_error(SENSE_EINVAL, "null plan or omega");
  for (int64_t l = 0; l < P->L; ++l)
    if (!std::isfinite(omega[l])) return set_error(SENSE_ENONFINITE, "non-finite omega");
  cudaStream_t st = (cudaStream_t)stream;
  SENSE_CUDA_TRY(cudaStreamSynchronize(st));
  std::copy(omega, omega + P->L, P->Rh.begin());
  const int rc = build_geometry(P, st);
  // stored phase tiles follow the new geometry
  if (rc != SENSE_OK || !P->p_enc) return rc;
  return tc_store_p(P, true, st);
}

extern "C" int sense_plan_info(sense_plan P, int64_t out[8]) {
  if (!P || !out) return set_error(SENSE_EINVAL, "null plan or output");
  out[0] = P->L; out[1] = P->K; out[2] = P->C; out[3] = P->P1;
  out[4] = P->r; out[5] = P->Lp; out[6] = P->Kp; out[7] = P->Cp;
  return SENSE_OK;
}

extern "C" const char* sense_strerror(int code) {
  switch (code) {
    case SENSE_OK: return "ok";
    case SENSE_EINVAL: return "invalid argument";
    case SENSE_ENOMEM: return "out of memory";
    case SENSE_ECUDA: return "CUDA error";
    case SENSE_ENONFINITE: return "non-finite value";
    case SENSE_EBREAKDOWN: return "CG breakdown";
    case SENSE_EUNSUPPORTED: return "unsupported size";
    case SENSE_ENODEVICE: return "no usable device";
    case SENSE_ETIMEOUT: return "device wait timed out";
    default: return "unknown error";
  }
}

extern "C" const char* sense_last_error(void) { return g_last_error.c_str(); }

extern "C" int sense_lcurve_corner(const double* h, int32_t n, int32_t* corner) {
  if (!h || !corner || n < 0) return set_error(SENSE_EINVAL, "null history/corner or n < 0");
  *corner = -1;
  // the curve's points are the iterates, rows 1..n-1 (row 0 is the start x_0 = 0, whose
  // log norm is -inf, and is never read); interior points 2..n-2 are the candidates
  if (n < 4) return SENSE_OK;
  double best = -INFINITY;
  for (int i = 2; i < n - 1; ++i) {
    // a = log data residual (column 2), b = log solution norm (column 1)
    const double am = std::log(h[3 * (i - 1) + 2]), a0 = std::log(h[3 * i + 2]),
                 ap = std::log(h[3 * (i + 1) + 2]);
    const double bm = std::log(h[3 * (i - 1) + 1]), b0 = std::log(h[3 * i + 1]),
                 bp = std::log(h[3 * (i + 1) + 1]);
    const double da = 0.5 * (ap - am), db = 0.5 * (bp - bm);
    const double dda = ap - 2.0 * a0 + am, ddb = bp - 2.0 * b0 + bm;
    const double den = std::pow(da * da + db * db, 1.5);
    if (!(den > 0.0) || !std::isfinite(den)) continue;
    const double k = (dda * db - da * ddb) / den;
    if (k > best) {
      best = k;
      *corner = i;
    }
  }
  return SENSE_OK;
}
